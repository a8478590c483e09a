"""Bounded waits: a wait on an mbarrier that nothing completes gives up after its poll limit, sets
the status bit the staged kernels use, and leaves the device usable (no fault, no hang)."""
import numpy as np
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


def test_wait_gives_up_and_reports():
    import torch
    from paper_1111_4363_gb300 import binding as B
    assert B.wait_selftest(1 << 10) & 4
    torch.cuda.synchronize()
    # the device is still usable: a relaxation step runs and converges afterwards
    w = wl.softcore_2d(n=32, levels=3)
    ctx = gpu_context(w)
    c = np.zeros(w.nunknowns, dtype=np.complex128)
    st, (cycles, sweeps, N, rel) = ctx.solve_step(wl.initial_state(w).ravel(), 0.0, c)
    assert rel <= w.tol
    ctx.close()


def test_invalid_selftest_arguments():
    from paper_1111_4363_gb300 import binding as B
    with pytest.raises(B.LeastActionError):
        B.wait_selftest(0)
