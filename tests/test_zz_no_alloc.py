"""la_action_noalloc: the residual norm for callers that cannot allocate device memory.

Such callers (code inside a framework that owns every device byte through its own pool, or a
process whose device budget is spent) get N through one entry point that allocates nothing and
keeps its scratch in a static device array.  It must agree with the context-based la_residual on
two calls in a row (the second call reuses the array the first one left behind).  This file is
collected last on purpose.
"""
import pytest

from paper_1111_4363_gb300 import workloads as wl

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


def test_noalloc_rejects_grids_beyond_the_limit():
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = wl.softcore_2d(n=32, levels=1)
    cfg = B.config_from_workload(w)
    cfg.n[0] = cfg.n[1] = 4096          # 16.8 M points > LA_NOALLOC_MAX_POINTS
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.LeastActionError, match="LA_NOALLOC_MAX_POINTS"):
        B.action_noalloc(cfg, dummy.real.contiguous(), None, dummy, 0.0, dummy)
