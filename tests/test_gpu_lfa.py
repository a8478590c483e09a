"""Legendre-element convergence maps (Secs. IV-V): la_lfa_maps on the GPU against the oracle's
direct evaluation (projection, constrained relaxation, residual norm and action) point by point."""
import numpy as np
import pytest

from oracle import lfa

pytestmark = pytest.mark.gpu

# FP64 on both sides by different routes (closed-form element matrices, Gram-Schmidt null spaces
# and elimination on the host, contracted matrices on the GPU, against quadrature matrices, SVD null
# spaces and direct evaluation).  log10 N ratios agree to 1e-8 and log10 |S| ratios to 1e-6, plus
# the rounding the problem itself amplifies, measured per point in tolerances().
TOL = 1e-8
TOL_S = 1e-6


def tolerances(method, nx, nt, kappa, nu, ks, ws):
    """Per-point bounds: the base tolerances plus ten times the disagreement of two backward-stable
    FP64 routes of the oracle itself (null-space and bordered least-squares solves), which measures
    how much rounding the problem amplifies (the constrained systems reach condition numbers of
    1.6e11 for two 8 x 8 elements at kappa = 10)."""
    nN, nS = lfa.ratio_map(method, nx, nt, kappa, nu, ks, ws)
    bN, bS = lfa.ratio_map(method, nx, nt, kappa, nu, ks, ws, solver="bordered")
    return TOL + 10 * np.abs(nN - bN), TOL_S + 10 * np.abs(nS - bS)


@pytest.mark.parametrize("method", ["one", "two", "transfer"])
@pytest.mark.parametrize("nx,nt", [(2, 2), (3, 3), (4, 5), (6, 6), (8, 8)])
def test_maps_match_the_oracle(method, nx, nt):
    from paper_1111_4363_gb300 import binding as B
    ks = np.array([-7.5, -2.0, 0.3, 1.0, 4.4])
    ws = np.array([-5.0, -0.6, 2.5, 6.1])
    cases = [(method, nx, nt, kappa, nu) for kappa, nu in lfa.KAPPA_NU]
    got = B.lfa_maps(cases, ks, ws)
    well = 0
    for c, (kappa, nu) in enumerate(lfa.KAPPA_NU):
        refN, refS = lfa.ratio_map(method, nx, nt, kappa, nu, ks, ws)
        tolN, tolS = tolerances(method, nx, nt, kappa, nu, ks, ws)
        assert np.all(np.abs(got[c, 0] - refN) < tolN), (kappa, nu)
        assert np.all(np.abs(got[c, 1] - refS) < tolS), (kappa, nu)
        if max(np.max(tolN), np.max(tolS)) < 1e-5:
            well += 1
    assert well >= 5       # most cases are checked to tight bounds
    if (nx, nt) == (2, 2) and method == "one":
        assert np.all(np.abs(got) < 1e-12)   # no free parameter: the trial is unchanged


def test_device_output_and_full_grid_samples():
    """The full map set the bench computes (8 (kappa, nu) pairs x 3 methods x 4 basis sizes on its
    256 x 256 grid, which avoids k = w = 0 where N or S of the trial vanishes for nu = 0), into a
    device array; sampled points against the oracle."""
    import torch
    from paper_1111_4363_gb300 import binding as B
    ks = np.linspace(-8.0, 8.0, 256)
    ws = np.linspace(-8.0, 8.0, 256)
    cases = [(m, s, s, kappa, nu) for m in ("one", "two", "transfer") for s in (3, 4, 6, 8)
             for kappa, nu in lfa.KAPPA_NU]
    out = torch.zeros((len(cases), 2, len(ws), len(ks)), dtype=torch.float64, device="cuda")
    B.lfa_maps(cases, ks, ws, out=out)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    rng = np.random.default_rng(7)
    for c in rng.choice(len(cases), 10, replace=False):
        m, nx, nt, kappa, nu = cases[c]
        a, b = rng.integers(0, len(ws)), rng.integers(0, len(ks))
        refN, refS = lfa.ratio_map(m, nx, nt, kappa, nu, ks[b:b + 1], ws[a:a + 1])
        tolN, tolS = tolerances(m, nx, nt, kappa, nu, ks[b:b + 1], ws[a:a + 1])
        assert abs(got[c, 0, a, b] - refN[0, 0]) < tolN[0, 0]
        assert abs(got[c, 1, a, b] - refS[0, 0]) < tolS[0, 0]


def test_invalid_cases_are_rejected():
    from paper_1111_4363_gb300 import binding as B
    with pytest.raises(B.LeastActionError):
        B.lfa_maps([("one", 1, 3, 0.0, 0.0)], [0.0], [0.0])
    with pytest.raises(B.LeastActionError):
        B.lfa_maps([("two", 3, 9, 0.0, 0.0)], [0.0], [0.0])
