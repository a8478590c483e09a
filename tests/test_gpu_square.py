"""Square-form local solve (Sec. II, M_UU delta_U = (f - M c)_U, red-black colouring): CUDA path
vs the CPU oracle through the C ABI (GB300 required)."""
import dataclasses

import numpy as np
import pytest

from oracle import relax, system
from oracle.propagate import numpy_sub
from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, oracle_system, ragged_2d, rel_l2, small_3d

pytestmark = pytest.mark.gpu

# FP64 on both sides, different summation orders, LU with partial pivoting on each side (the
# pivot sequences may differ on near-ties): 1e-11 relative L2 as for the least-squares form.
TOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def square(w, **kw):
    return dataclasses.replace(w, levels=1, local_form="square", **kw)


WORKLOADS = {
    "1d": lambda: square(wl.harmonic_1d()),
    "2d": lambda: square(wl.softcore_2d(n=32, levels=1)),
    "2d_sub2": lambda: square(wl.softcore_2d(n=16, levels=1), sub=(2, 2, 1)),
    "2d_sub1": lambda: square(wl.softcore_2d(n=12, levels=1), sub=(1, 1, 1)),
    "2d_ragged": lambda: square(ragged_2d(levels=1)),
    "3d": lambda: square(small_3d(levels=1)),
}


def oracle_relaxation(w, psi0, t0):
    prob, M, f, W = oracle_system(w, psi0, t0)
    return prob, M.tocsr(), f, W, relax.SquareRelaxation(M, prob.shape, numpy_sub(w), prob.K)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_square_colour_pass(name):
    """One red-black pass (LU factor + sweep kernels) vs the oracle's square block updates."""
    w = WORKLOADS[name]()
    ctx = gpu_context(w)
    psi0 = wl.initial_state(w).ravel()
    t0 = 0.25
    prob, M, f, W, R = oracle_relaxation(w, psi0, t0)
    c0 = wl.random_state(M.shape[1], 3) * 0.05
    for colour in range(2):
        ref = c0.copy()
        R.colour_pass(ref, f, colour)
        got = c0.copy()
        ctx.relax_colour(psi0, t0, colour, got)
        assert rel_l2(got - c0, ref - c0) < 1e-10, colour
        assert rel_l2(got, ref) < TOL64
        # the relaxed subvolumes' residual rows vanish, the others' do not
        r = system.residual(M, f, got)
        rows = np.concatenate([idx for col, idx, _ in R.blocks if col == colour])
        others = np.setdiff1d(np.arange(M.shape[0]), rows)
        assert np.max(np.abs(r[rows])) <= 1e-11 * np.max(np.abs(f))
        assert np.max(np.abs(r[others])) > 1e-6 * np.max(np.abs(f))


@pytest.mark.parametrize("name", ["1d", "2d", "2d_ragged", "3d"])
def test_square_fixed_sweeps(name):
    """A fixed number of red-black sweeps from c = 0: the same iterate and action."""
    w = WORKLOADS[name]()
    ctx = gpu_context(w)
    psi0 = wl.initial_state(w).ravel()
    t0 = 0.1
    prob, M, f, W, R = oracle_relaxation(w, psi0, t0)
    ncycles = 2
    ref = np.zeros(M.shape[1], complex)
    for _ in range(ncycles * (w.nu1 + w.nu2)):
        R.sweep(ref, f)
    c = np.zeros(M.shape[1], dtype=np.complex128)
    st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, t0, c, ncycles=ncycles)
    assert cycles == ncycles and sweeps == ncycles * (w.nu1 + w.nu2)
    assert rel_l2(c, ref) < TOL64
    assert N == pytest.approx(system.action_norm(system.residual(M, f, ref), W), rel=1e-9)


def test_square_steps_converge_to_the_direct_solution():
    w = dataclasses.replace(WORKLOADS["2d"](), tol=1e-22, max_cycles=40)
    ctx = gpu_context(w)
    psi0 = wl.initial_state(w).ravel()
    t0 = 0.3
    prob, M, f, W = oracle_system(w, psi0, t0)
    c = np.zeros(M.shape[1], dtype=np.complex128)
    st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, t0, c)
    assert rel <= 1e-22
    xd = system.direct_solve(M, f)
    assert rel_l2(c, xd) < 1e-9


def test_square_divergence_matches_the_oracle():
    """kappa = 2.5 (dt = 0.2, h = 0.2): the square form diverges; the GPU follows the oracle's
    growing iterates pass for pass while N rises above N(0)."""
    w = square(wl.softcore_2d(n=16, levels=1), dt=0.2, nu1=1, nu2=0)
    ctx = gpu_context(w)
    psi0 = wl.initial_state(w).ravel()
    t0 = 0.0
    prob, M, f, W, R = oracle_relaxation(w, psi0, t0)
    N0 = system.action_norm(f, W)
    ref = np.zeros(M.shape[1], complex)
    rels = []
    for ncyc in (2, 6):
        while len(rels) < ncyc:
            R.sweep(ref, f)
            rels.append(system.action_norm(system.residual(M, f, ref), W) / N0)
        c = np.zeros(M.shape[1], dtype=np.complex128)
        st, (cycles, sweeps, N, rel) = ctx.solve_step(psi0, t0, c, ncycles=ncyc)
        assert rel_l2(c, ref) < 1e-9
        assert rel == pytest.approx(rels[-1], rel=1e-8)
    assert rels[-1] > 1.0 and rels[-1] > rels[0]


def test_square_form_rejects_the_adjoint():
    from paper_1111_4363_gb300 import binding as B
    w = dataclasses.replace(WORKLOADS["2d"](), nsteps=2)
    ctx = gpu_context(w, ckpt_every=2)
    import torch
    psi = torch.from_numpy(wl.initial_state(w).ravel()).to("cuda")
    ctx.step(psi, 2, 0.0, allow_notconv=True)
    with pytest.raises(B.LeastActionError) as e:
        ctx.backward(torch.zeros_like(psi), 0)
    assert e.value.status == B.LA_EINVAL
