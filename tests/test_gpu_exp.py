"""The FP64 exponential of the rate kernels (misdc_exp, Tang's table-driven method)
against the host's libm exp and CUDA's exp on the same arguments: within 2 ulp of
both everywhere in (-700, 700), equal to CUDA's exp outside (its fallback), and
exact at 0."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def ulp_err(a, b):
    """|a - b| in units of the last place of b."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_exp_within_two_ulp():
    from paper_1801_01201_gb300 import solver as S
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.uniform(-700, 700, 200_000),
        rng.uniform(-1, 1, 50_000),
        rng.uniform(-1e-6, 1e-6, 10_000),
        # arguments at and next to the reduction's break points k ln2/32 (round-half cases)
        (np.arange(-2000, 2000) + 0.5) * np.log(2) / 32,
        np.arange(-2000, 2000) * np.log(2) / 32,
        [0.0, -0.0, 1.0, -1.0, 699.999, -699.999, 709.0, -709.0, -745.0, 1e-300],
    ])
    xd = torch.as_tensor(x, device="cuda")
    got = S.exp(xd).cpu().numpy()
    cuda = torch.exp(xd).cpu().numpy()
    host = np.exp(x)
    inside = np.abs(x) < 700
    assert np.max(ulp_err(got[inside], host[inside])) <= 2.0
    assert np.max(ulp_err(got[inside], cuda[inside])) <= 2.0
    # outside (-700, 700) the kernel's fallback is CUDA's own exp
    assert np.array_equal(got[~inside], cuda[~inside])
    assert got[x == 0.0][0] == 1.0


def test_exp_special_values():
    from paper_1801_01201_gb300 import solver as S
    x = torch.tensor([np.nan, np.inf, -np.inf, 800.0, -800.0], dtype=torch.float64, device="cuda")
    got = S.exp(x).cpu().numpy()
    assert np.isnan(got[0]) and got[1] == np.inf and got[2] == 0.0 and got[3] == np.inf and got[4] == 0.0
