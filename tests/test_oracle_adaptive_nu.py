"""Pins of the oracle's adaptive number of nested iterations (or_nu_rule, a
reading: the paper asks for such a rule as future work in Sec. 4 and 5).

With two Gauss-Lobatto nodes (M = 1) the sweep's only free node is the output,
so the rule's whole decision can be recomputed from independent fixed-nu runs:
delta_l = |phi_{nu=l+1} - phi_{nu=l}| / |phi_{nu=l+1}| with phi_{nu=0} = phi^n
(iteration 0 compares against sweep k, the spread initial value)."""
import numpy as np
import pytest

import oracle as O

CASES = [(-100.0, -5.0), (-5.0, -5.0), (-5.0, -100.0), (-30.0, -30.0)]


def _rule_by_hand(phis, nu_max, eta, rho):
    """Nested iterations the rule runs, from phi_{nu=0..nu_max} of one sweep."""
    d = [abs(phis[l + 1] - phis[l]) / abs(phis[l + 1]) for l in range(nu_max)]
    ran = 1
    for l in range(nu_max):
        ran = l + 1
        if l >= 1 and l + 1 < nu_max and not (d[l] > eta * d[0] and d[l] < rho * d[l - 1]):
            break
    return ran


@pytest.mark.parametrize("d,r", CASES)
@pytest.mark.parametrize("eta,rho", [(0.1, 0.5), (0.3, 0.8), (0.02, 0.9), (1e-12, 0.999)])
def test_one_sweep_decision_matches_fixed_nu_runs(d, r, eta, rho):
    dt, phi0, nu_max = 0.1, 1.0, 6
    phis = [phi0] + [O.linear_step("CISDCQ", 1, 1, nu, dt, 0.0, d, r, phi0)[0] for nu in range(1, nu_max + 1)]
    want = _rule_by_hand(phis, nu_max, eta, rho)
    got, _, used = O.linear_step("CISDCQ", 1, 1, nu_max, dt, 0.0, d, r, phi0, nu_rule=(eta, rho))
    assert used[0] == want
    # stopping early leaves exactly the fixed-nu result of that many iterations
    assert got == phis[want]


@pytest.mark.parametrize("M", [1, 2, 4])
def test_rule_off_or_nu_two_is_fixed_nu(M):
    for nu in (1, 2, 4):
        want, inc_w = O.linear_step("CISDCQ", M, 5, nu, 0.1, 0.0, -20.0, -7.0)
        got, inc_g, used = O.linear_step("CISDCQ", M, 5, nu, 0.1, 0.0, -20.0, -7.0, nu_rule=(0.0, 0.5))
        assert got == want and np.array_equal(inc_g, inc_w) and np.all(used == nu)
    # nu_max = 2: iterations 0 and 1 always run, so the rule never stops early
    want, _ = O.linear_step("CISDCQ", M, 5, 2, 0.1, 0.0, -20.0, -7.0)
    got, _, used = O.linear_step("CISDCQ", M, 5, 2, 0.1, 0.0, -20.0, -7.0, nu_rule=(0.5, 0.1))
    assert got == want and np.all(used == 2)


@pytest.mark.parametrize("d,r", CASES[:3])
def test_adaptive_converges_to_the_collocation_solution_with_less_work(d, r):
    """Sweeps with adaptive nu still converge to the collocation solution (the
    fixed point every scheme shares), and reach it with fewer nested iterations
    in total than fixed nu = 6."""
    M, dt, sweeps = 2, 0.1, 30
    coll, _ = O.linear_step("CISDCQ", M, 60, 6, dt, 0.0, d, r)
    phi, inc, used = O.linear_step("CISDCQ", M, sweeps, 6, dt, 0.0, d, r, nu_rule=(0.1, 0.5))
    assert abs(phi - coll) <= 1e-13 * abs(coll)
    k_ad = next(i for i, v in enumerate(inc) if v < 1e-14)
    _, inc6 = O.linear_step("CISDCQ", M, sweeps, 6, dt, 0.0, d, r)
    k_6 = next(i for i, v in enumerate(inc6) if v < 1e-14)
    assert int(np.sum(used[: k_ad + 1])) < 6 * (k_6 + 1)
    assert np.all((used >= 2) & (used <= 6))
