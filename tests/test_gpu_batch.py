"""la_step_batch: independent propagations stepped together equal the oracle's propagations of the same
problems, and the same propagations stepped alone."""
import dataclasses

import pytest

from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, oracle_trial_propagation, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def members():
    a = wl.batched_2d(3)
    a = dataclasses.replace(a, n=(48, 48, 1), levels=3)
    b = wl.batched_2d(5)
    b = dataclasses.replace(b, n=(32, 32, 1), levels=2, sub=(2, 2, 1))
    c = wl.harmonic_1d()
    return [a, b, c]


@pytest.mark.parametrize("precision,trial", [(0, 0), (1, 0), (0, 3), (1, 3)])
def test_batch_equals_individual_steps(precision, trial):
    import torch
    from paper_1111_4363_gb300 import binding as B
    ws = [dataclasses.replace(w, trial=trial) for w in members()]
    nsteps = 3
    alone = []
    for w in ws:
        ctx = gpu_context(w, precision=precision)
        psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
        st, stats = ctx.step(psi, nsteps, 0.2, stats=True)
        alone.append((psi.cpu().numpy(), stats))
    ctxs = [gpu_context(w, precision=precision) for w in ws]
    psis = [torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda() for w in ws[:2]]
    psis.append(wl.initial_state(ws[2]).ravel().copy())            # host buffer for the third member
    stats = B.step_batch(ctxs, psis, nsteps, [0.2] * 3)
    for i, (psi_ref, st_ref) in enumerate(alone):
        got = psis[i].cpu().numpy() if hasattr(psis[i], "cpu") else psis[i]
        assert rel_l2(got, psi_ref) < 1e-14, i
        assert [s[0] for s in stats[i]] == [s[0] for s in st_ref]
        assert all(s[3] <= ws[i].tol for s in stats[i])


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_members_match_the_oracle(precision):
    """Members of the batched family (K = 4, own E0 and soft-core a) at 64^2 and 48^2 and the 1D workload
    in one la_step_batch call, each step two fixed cycles from the quadratic trial, against the oracle
    replaying the same schedule (FP64: 1e-11; mixed precision: its complex64 V-cycle on the correction
    equation leaves iterates that differ from the FP64 ones at the level of the FP32 rounding, 1e-5)."""
    import torch
    from paper_1111_4363_gb300 import binding as B
    a = dataclasses.replace(wl.batched_2d(7), n=(64, 64, 1), levels=3, trial=3)
    b = dataclasses.replace(wl.batched_2d(11), n=(48, 48, 1), levels=3, trial=3)
    c = dataclasses.replace(wl.harmonic_1d(), trial=3)
    ws = [a, b, c]
    assert a.pulse.amp != b.pulse.amp and a.softcore_a != b.softcore_a
    nsteps, ncyc, t0 = 3, 2, 0.15
    ctxs = [gpu_context(w, precision=precision, tol=0.0, max_cycles=ncyc) for w in ws]
    psis = [torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda() for w in ws]
    stats = B.step_batch(ctxs, psis, nsteps, [t0] * 3)
    tol = 1e-11 if precision == 0 else 1e-5
    for i, w in enumerate(ws):
        assert [s[0] for s in stats[i]] == [ncyc] * nsteps
        ref = oracle_trial_propagation(w, wl.initial_state(w).ravel(), nsteps, w.trial, ncyc, t0=t0)
        assert rel_l2(psis[i].cpu().numpy(), ref) < tol, (i, rel_l2(psis[i].cpu().numpy(), ref))


def test_batch_rejects_repeated_context():
    import torch
    from paper_1111_4363_gb300 import binding as B
    w = members()[1]
    ctx = gpu_context(w)
    psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
    with pytest.raises(B.LeastActionError):
        B.step_batch([ctx, ctx], [psi, psi.clone()], 1)


def test_batch_with_square_local_form():
    """Contexts of both local forms in one batch (the square form single-level, red-black)."""
    import torch
    from paper_1111_4363_gb300 import binding as B
    a, b, c = members()
    ws = [dataclasses.replace(a, levels=1, local_form="square", trial=3), b,
          dataclasses.replace(c, local_form="square")]
    nsteps = 3
    alone = []
    for w in ws:
        ctx = gpu_context(w)
        psi = torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda()
        st, stats = ctx.step(psi, nsteps, 0.2, stats=True)
        alone.append((psi.cpu().numpy(), stats))
    ctxs = [gpu_context(w) for w in ws]
    psis = [torch.from_numpy(wl.initial_state(w).ravel().copy()).cuda() for w in ws]
    stats = B.step_batch(ctxs, psis, nsteps, [0.2] * 3)
    for i, (psi_ref, st_ref) in enumerate(alone):
        assert rel_l2(psis[i].cpu().numpy(), psi_ref) < 1e-14, i
        assert [s[0] for s in stats[i]] == [s[0] for s in st_ref]
        assert all(s[3] <= ws[i].tol for s in stats[i])
