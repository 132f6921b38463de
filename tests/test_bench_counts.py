"""The bench line's roofline arithmetic on the host: the algorithmic FP64 flops of
the reaction step follow the per cell-iteration counts (thermo 15N, rates
R(10 + 4 nubar), Jacobian 2 R nubar^2, LU 2n^3/3, one solve 2n^2 per iteration
and per certified or stored-step solve), applied to the device counters, and the
refinement rounds of the mixed diffusion solve follow the flame's dimension."""
import types

import bench


def test_counted_flops_follow_the_per_iteration_counts():
    N, R, nubar = 21, 84, 3.869047619047619
    n = N + 1
    stats = {"newton_iters": 1000, "newton_jacobians": 30, "newton_certified": 600,
             "newton_stored_steps": 250, "newton_solves": 900}
    flops, c = bench.newton_flops_counted(N, R, nubar, stats, mixed=True)
    ev = 1000 - 600 - 250   # iterations that evaluate the rates
    per_ev = 15 * N + R * (10 + 4 * nubar)
    per_jac = 2 * R * nubar ** 2 + 2.0 * n ** 3 / 3
    want = ev * per_ev + 30 * per_jac + (ev + 600 + 250) * 2 * n * n
    assert abs(flops - want) <= 1e-9 * want
    assert (c["rate_iterations"], c["jacobians"], c["certified"], c["stored_steps"]) == (ev, 30, 600, 250)
    assert c["per_rate_iteration"] == per_ev and c["per_solve"] == 2 * n * n
    # FP64 mode: every iteration evaluates the rates and assembles a Jacobian
    f64, c64 = bench.newton_flops_counted(N, R, nubar, stats, mixed=False)
    assert c64["rate_iterations"] == 1000 and c64["jacobians"] == 1000
    assert abs(f64 - 1000 * (per_ev + per_jac + 2 * n * n)) <= 1e-9 * f64


def test_refinement_rounds_follow_the_dimension():
    args = types.SimpleNamespace(lin_rounds=-1)
    assert [bench.lin_rounds_for(args, types.SimpleNamespace(dim=d)) for d in (1, 2, 3)] == [0, 0, 2]
    args.lin_rounds = 3
    assert bench.lin_rounds_for(args, types.SimpleNamespace(dim=3)) == 3
