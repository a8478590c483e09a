"""The action norm as a NaN/Inf canary, with the failure made on the host: one NaN written into an
input buffer.  Every relaxation path (la_step, la_backward, la_step_batch) must stop with
LA_ENOTCONV, whether or not a tolerance is set, and leave the device usable; a NaN in the potential
makes the subvolume matrices non-positive-definite, which the factorisation reports as LA_ECUDA."""
import dataclasses

import numpy as np
import pytest

from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def small():
    return wl.softcore_2d(n=32, levels=3, nsteps=4)


def nan_state(w, point=37):
    psi = wl.initial_state(w).ravel().copy()
    psi[point] = complex(np.nan, 0.0)
    return psi


@pytest.mark.parametrize("tol", [1e-10, 0.0])
def test_la_step_stops_on_a_non_finite_action(tol):
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = small()
    ctx = gpu_context(w, tol=tol, max_cycles=20)
    psi = torch.from_numpy(nan_state(w)).cuda()
    st, stats = ctx.step(psi, 2, 0.0, stats=True, allow_notconv=True)
    assert st == B.LA_ENOTCONV
    assert all(s[0] == 0 for s in stats)          # no cycle runs on a non-finite action
    assert "not finite" in ctx.last_error()
    # the device stays usable: a clean step on the same context converges
    psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
    st, stats = ctx.step(psi, 1, 0.0, stats=True)
    assert st == B.LA_OK and stats[0][0] > 0 and np.isfinite(stats[0][2])


@pytest.mark.parametrize("tol", [1e-10, 0.0])
def test_la_step_batch_flags_the_member_whatever_its_tolerance(tol):
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = small()
    ws = [w, dataclasses.replace(wl.batched_2d(3), n=(32, 32, 1), levels=3)]
    ctxs = [gpu_context(x, tol=tol, max_cycles=3) for x in ws]
    psis = [torch.from_numpy(nan_state(ws[0])).cuda(),
            torch.from_numpy(wl.initial_state(ws[1]).ravel().copy()).cuda()]
    with pytest.raises(B.LeastActionError) as e:
        B.step_batch(ctxs, psis, 2, [0.0, 0.0])
    assert e.value.status == B.LA_ENOTCONV
    assert "not finite" in ctxs[0].last_error()
    # the healthy member was stepped as if alone
    alone = gpu_context(ws[1], tol=tol, max_cycles=3)
    psi1 = torch.from_numpy(wl.initial_state(ws[1]).ravel().copy()).cuda()
    alone.step(psi1, 2, 0.0, allow_notconv=True)
    assert rel_l2(psis[1].cpu().numpy(), psi1.cpu().numpy()) < 1e-14


@pytest.mark.parametrize("tol", [1e-10, 0.0])
def test_la_backward_stops_on_a_non_finite_adjoint(tol):
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = small()
    ctx = gpu_context(w, tol=tol, max_cycles=4, ckpt_every=2)
    psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
    ctx.step(psi, 4, 0.0, allow_notconv=True)
    dJ = torch.from_numpy(nan_state(w, point=500)).cuda()
    with pytest.raises(B.LeastActionError) as e:
        ctx.backward(dJ, w.pulse.ncomp)
    assert e.value.status == B.LA_ENOTCONV
    assert "not finite" in ctx.last_error()


def test_nan_potential_is_reported_by_the_factorisation():
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = small()
    cfg = B.config_from_workload(w)
    ctx = B.Context(cfg)
    V0 = wl.potential(w).ravel().copy()
    V0[100] = np.nan
    ctx.set_hamiltonian(torch.from_numpy(V0).cuda(), w.pulse)
    psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
    with pytest.raises(B.LeastActionError) as e:
        ctx.step(psi, 1, 0.0)
    assert e.value.status == B.LA_ECUDA
    assert "positive definite" in ctx.last_error()
    ctx.close()
