"""la_action_noalloc: the residual norm for callers that cannot allocate device memory.

Such callers (code inside a framework that owns every device byte through its own pool, or a
process whose device budget is spent) get N through one entry point that allocates nothing and
keeps its scratch in a static device array.  It must agree with the oracle's N = r^dagger W r and
with the context-based la_residual on two calls in a row (the second call reuses the array the
first one left behind), for every dimension and residual-norm weight, on a side stream, and on a
grid of exactly LA_NOALLOC_MAX_POINTS points, where the partial sums fill the array.  This file is
collected last on purpose.
"""
import pytest

from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import oracle_system, small_3d, variant

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("make", [lambda: wl.softcore_2d(n=32, levels=3), lambda: wl.harmonic_1d()])
def test_noalloc_action_matches_la_residual_two_calls(make):
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = make()
    cfg = B.config_from_workload(w)
    V0 = torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda")
    ctx = B.Context(cfg)
    ctx.set_hamiltonian(V0, w.pulse)
    psi0 = torch.from_numpy(wl.initial_state(w).ravel()).cuda()
    for call, (seed, t0) in enumerate([(21, 0.3), (22, 1.15)]):
        c = torch.from_numpy(wl.random_state(w.nunknowns, seed) * 0.05).cuda()
        n_ref = ctx.residual(psi0, t0, c)
        n = B.action_noalloc(cfg, V0, w.pulse, psi0, t0, c)
        assert n == pytest.approx(n_ref, rel=1e-12), (call, n, n_ref)
    ctx.close()


WORKLOADS = {
    "1d": lambda: wl.harmonic_1d(),
    "2d": lambda: wl.softcore_2d(n=32, levels=3),
    "3d": lambda: small_3d(levels=2),
}


@pytest.mark.parametrize("weight", ["dual", "literal", "identity"])
@pytest.mark.parametrize("dim", ["1d", "2d", "3d"])
def test_noalloc_action_matches_the_oracle(dim, weight):
    """N of two coefficient vectors in a row against the oracle's assembled r^dagger W r (Eq. residnorm
    with each of the three weights)."""
    import torch
    from oracle import system
    from paper_1111_4363_gb300 import binding as B
    w = variant(WORKLOADS[dim](), weight=weight)
    cfg = B.config_from_workload(w)
    V0 = torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda")
    psi0 = wl.initial_state(w).ravel()
    for seed, t0 in [(31, 0.45), (32, 2.05)]:
        c = wl.random_state(w.nunknowns, seed) * 0.05
        _, M, f, W = oracle_system(w, psi0, t0)
        n_ref = system.action_norm(system.residual(M, f, c), W)
        n = B.action_noalloc(cfg, V0, w.pulse, torch.from_numpy(psi0).cuda(), t0, torch.from_numpy(c).cuda())
        assert n == pytest.approx(n_ref, rel=1e-12), (seed, n, n_ref)


def test_noalloc_action_at_the_point_limit_and_on_a_side_stream():
    """2048 x 2048 points = LA_NOALLOC_MAX_POINTS exactly (the last partial-sum slot and the result
    slot at the array's end), K = 4; the second call runs on a torch side stream."""
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = variant(wl.softcore_2d(n=32, levels=1), n=(2048, 2048, 1), nt=4, sub=(2, 2, 1), coarse_sub=None)
    assert w.npoints == 1 << 22
    cfg = B.config_from_workload(w)
    V0 = torch.tensor(wl.potential(w).ravel(), dtype=torch.float64, device="cuda")
    ctx = B.Context(cfg)
    ctx.set_hamiltonian(V0, w.pulse)
    psi0 = torch.from_numpy(wl.initial_state(w).ravel()).cuda()
    c = torch.from_numpy(wl.random_state(w.nunknowns, 41) * 0.05).cuda()
    n_ref = ctx.residual(psi0, 0.7, c)
    assert B.action_noalloc(cfg, V0, w.pulse, psi0, 0.7, c) == pytest.approx(n_ref, rel=1e-12)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        n = B.action_noalloc(cfg, V0, w.pulse, psi0, 0.7, c, stream=side)
    assert n == pytest.approx(n_ref, rel=1e-12)
    ctx.close()


def test_noalloc_rejects_grids_beyond_the_limit():
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = wl.softcore_2d(n=32, levels=1)
    cfg = B.config_from_workload(w)
    cfg.n[0] = cfg.n[1] = 4096          # 16.8 M points > LA_NOALLOC_MAX_POINTS
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.LeastActionError, match="LA_NOALLOC_MAX_POINTS"):
        B.action_noalloc(cfg, dummy.real.contiguous(), None, dummy, 0.0, dummy)
