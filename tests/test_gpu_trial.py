"""la_step with an extrapolated trial iterate (cfg.trial > 0) vs the oracle replaying the same schedule."""
import dataclasses

import pytest

from paper_1111_4363_gb300 import workloads as wl
from tests.helpers import gpu_context, oracle_trial_propagation, rel_l2, small_3d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name,trial", [("2d", 1), ("2d", 2), ("2d", 3), ("3d", 3)])
def test_fixed_schedule_with_trial_matches_oracle(name, trial):
    w = wl.softcore_2d(n=32, levels=3) if name == "2d" else small_3d(levels=2)
    w = dataclasses.replace(w, trial=trial)
    nsteps, ncycles = 5, 2
    psi0 = wl.initial_state(w).ravel()
    ref = oracle_trial_propagation(w, psi0, nsteps, trial, ncycles)
    ctx = gpu_context(w, tol=0.0, max_cycles=ncycles)
    psi = psi0.copy()
    ctx.step(psi, nsteps, 0.0)
    # and without the trial the result differs (the test would not see a dropped trial otherwise)
    cold = oracle_trial_propagation(w, psi0, nsteps, 0, ncycles)
    assert rel_l2(psi, ref) < 1e-11
    assert rel_l2(cold, ref) > 1e-9


def test_trial_keeps_the_tolerance_and_saves_cycles():
    w = wl.softcore_2d(n=32, levels=3)
    psi0 = wl.initial_state(w).ravel()
    nsteps = 8
    out = {}
    for trial in (0, 1, 3):
        ctx = gpu_context(dataclasses.replace(w, trial=trial))
        psi = psi0.copy()
        st, stats = ctx.step(psi, nsteps, 0.0, stats=True)
        assert all(s[3] <= w.tol for s in stats)
        out[trial] = (psi, sum(s[0] for s in stats))
    assert out[3][1] <= out[1][1] < out[0][1]
    # converged to the same relative action: the states agree to the accuracy of the stopping test
    assert rel_l2(out[3][0], out[0][0]) < 1e-6


def test_history_continues_across_calls_and_resets_on_a_jump():
    w = dataclasses.replace(wl.softcore_2d(n=32, levels=3), trial=3)
    psi0 = wl.initial_state(w).ravel()
    ctx = gpu_context(w, tol=0.0, max_cycles=2)
    a = psi0.copy()
    ctx.step(a, 4, 0.0)
    b = psi0.copy()
    ctx2 = gpu_context(w, tol=0.0, max_cycles=2)
    ctx2.step(b, 2, 0.0)
    ctx2.step(b, 2, 2 * w.dt)             # continues: same iterates as one call of 4 steps
    assert rel_l2(b, a) < 1e-14
    ctx3 = gpu_context(w, tol=0.0, max_cycles=2)
    d = psi0.copy()
    ctx3.step(d, 2, 0.0)
    ctx3.step(d, 2, 5 * w.dt)             # a jump in time clears the history
    ref = oracle_trial_propagation(w, oracle_trial_propagation(w, psi0, 2, 3, 2), 2, 3, 2, t0=5 * w.dt)
    assert rel_l2(d, ref) < 1e-11
