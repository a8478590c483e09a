"""la_profile counters agree with the work a step reports (GB300 required)."""
import pytest

from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_counters_match_the_step_statistics(precision):
    w = wl.softcore_2d(n=64, levels=3)
    ctx = gpu_context(w, precision=precision)
    psi = wl.initial_state(w).ravel().copy()
    ctx.step(psi, 1, 0.0)                       # warm-up (first cycle runs outside a graph)
    ctx.profile_enable(True)
    nsteps = 3
    st, stats = ctx.step(psi, nsteps, w.dt, stats=True)
    p = ctx.profile_read()
    ctx.profile_enable(False)
    assert p["n_factor"] == nsteps
    assert p["n_sweep"] == sum(s[1] for s in stats)            # whole finest sweeps
    # residual stencil: one per cycle inside the V-cycle, one per action evaluation after a cycle; N(0)
    # of c = 0 is the weighted norm of f alone (no stencil) and is not counted
    cycles = sum(s[0] for s in stats)
    if precision == 0:
        assert p["n_resid"] == cycles + cycles and p["n_resid32"] == 0
    else:   # the V-cycle residual is complex64
        assert p["n_resid"] == cycles and p["n_resid32"] == cycles
    assert p["ms_factor"] > 0 and p["ms_sweep"] > 0 and p["ms_resid"] > 0 and p["launches"] > 0
    n = 4 * 4 * w.nt
    nsub = (w.n[0] // 4) * (w.n[1] // 4)
    assert p["flops_factor"] == pytest.approx(nsub * 4.0 / 3.0 * n ** 3)
    assert p["flops_sweep"] == pytest.approx(nsub * 8.0 * n ** 2)
    csize = 16 if precision == 0 else 8
    per_cycle = w.npoints * (csize * w.nt * 3 + 8)               # f, c in, z out, V0 in (V-cycle residual)
    per_action = w.npoints * (16 * w.nt * 3 + 8)                 # f, c in, r out, V0 in (FP64 action)
    if precision == 0:
        assert p["bytes_resid"] == pytest.approx(cycles * per_cycle + cycles * per_action)
    else:
        assert p["bytes_resid"] == pytest.approx(cycles * per_action)
        assert p["bytes_resid32"] == pytest.approx(cycles * per_cycle)
