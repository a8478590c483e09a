"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import dataclasses
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(la_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("la_init", "la_set_hamiltonian", "la_step", "la_action", "la_finalize"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import binding
    lib = ctypes.CDLL(binding.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert b"sm_103a" in binding.lib().la_version()
    assert set(binding.EXPORTS) <= set(declared_functions())


def test_binding_status_codes_match_the_header():
    text = open(os.path.join(ROOT, "include", "leastaction.h")).read()
    codes = {int(v): k for k, v in re.findall(r"\b(LA_[A-Z]+) = (\d+)", text)}
    from paper_1111_4363_gb300 import binding as B
    assert codes == B.STATUS_NAMES
    for value, name in codes.items():
        assert getattr(B, name) == value


def test_init_rejects_invalid_configs_without_touching_the_gpu():
    from paper_1111_4363_gb300 import binding as B
    from paper_1111_4363_gb300 import workloads as wl
    w = wl.softcore_2d(n=32, levels=3)
    bad = [dict(dim=4), dict(nt=0), dict(nt=9), dict(dt=0.0), dict(levels=0), dict(max_cycles=0),
           dict(weight=3), dict(precision=2), dict(laser_axis=2), dict(nu1=0, nu2=0), dict(trial=4),
           dict(trial=-1), dict(coarse_cycle=1, coarse_nu1=-1), dict(local_form=2), dict(local_form=-1),
           dict(local_form=1, precision=1), dict(local_form=1, levels=2), dict(local_form=1, levels=1, nt=8),
           dict(factor_group=2), dict(factor_group=-1)]
    for kw in bad:
        cfg = B.config_from_workload(w, **kw)
        with pytest.raises(B.LeastActionError) as e:
            B.Context(cfg)
        assert e.value.status == B.LA_EINVAL, kw
    cfg = B.config_from_workload(w)
    cfg.sub[0] = 1
    with pytest.raises(B.LeastActionError, match="sub must be"):
        B.Context(cfg)
    cfg = B.config_from_workload(w)
    cfg.n[0] = 30          # not divisible by 2^(levels-1) = 4
    with pytest.raises(B.LeastActionError, match="divisible"):
        B.Context(cfg)
    cfg = B.config_from_workload(w)
    cfg.sub[0] = cfg.sub[1] = 8   # 64 points x K = 6 = 384 unknowns > 256
    with pytest.raises(B.LeastActionError, match="at most 64 points and 256 unknowns"):
        B.Context(cfg)
    w3 = dataclasses.replace(wl.hydrogen_3d(n=16, nsteps=4, ncomp=4, sub=4), coarse_sub=None)
    cfg = B.config_from_workload(w3)   # 4x4x4 finest subvolumes, Galerkin levels of the same size
    with pytest.raises(B.LeastActionError, match="Galerkin-level subvolume"):
        B.Context(cfg)
    cfg = B.config_from_workload(w3, levels=1)
    cfg.sub[0] = 5                     # 5x4x4 = 80 points
    with pytest.raises(B.LeastActionError, match="at most 64 points"):
        B.Context(cfg)


def test_allocation_failure_reports_enomem(monkeypatch):
    """LA_FAIL_ALLOC refuses every device allocation: la_init returns LA_ENOMEM and frees what it holds."""
    from paper_1111_4363_gb300 import binding as B
    from paper_1111_4363_gb300 import workloads as wl
    monkeypatch.setenv("LA_FAIL_ALLOC", "1")
    cfg = B.config_from_workload(wl.softcore_2d(n=32, levels=3))
    with pytest.raises(B.LeastActionError, match="LA_FAIL_ALLOC") as e:
        B.Context(cfg)
    assert e.value.status == B.LA_ENOMEM


def test_noalloc_rejects_oversized_grids_and_host_pointers_without_the_gpu():
    """la_action_noalloc checks every axis before it multiplies them (three axes of 2^31 - 1 points
    would overflow a 64-bit count), and rejects host buffers; both before any device work."""
    import numpy as np
    from paper_1111_4363_gb300 import binding as B
    from paper_1111_4363_gb300 import workloads as wl
    w = wl.hydrogen_3d(n=8, nsteps=4, ncomp=4, sub=2)
    host = np.zeros(8, dtype=np.complex128)
    for ext in [(2 ** 31 - 1,) * 3, (2 ** 22 + 1, 1, 1), (2048, 2048, 2)]:
        cfg = B.config_from_workload(w)
        for a in range(3):
            cfg.n[a] = ext[a]
        with pytest.raises(B.LeastActionError, match="LA_NOALLOC_MAX_POINTS") as e:
            B.action_noalloc(cfg, host.real.copy(), w.pulse, host, 0.0, host)
        assert e.value.status == B.LA_EINVAL
    cfg = B.config_from_workload(w)
    with pytest.raises(B.LeastActionError, match="device pointers") as e:
        B.action_noalloc(cfg, np.zeros(w.npoints), w.pulse, np.zeros(w.npoints, np.complex128), 0.0,
                         np.zeros(w.nunknowns, np.complex128))
    assert e.value.status == B.LA_EINVAL


def test_null_arguments_are_rejected_without_touching_the_gpu():
    """Every entry point checks its context and required pointers before any CUDA call: a null one
    returns LA_EINVAL (here, on a machine without a GPU), and la_last_error still answers."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import binding as B
    L = B.lib()
    d = ctypes.c_double(0.0)
    calls = {
        "la_init": lambda: L.la_init(None, None, None),
        "la_set_hamiltonian": lambda: L.la_set_hamiltonian(None, None, None),
        "la_step": lambda: L.la_step(None, None, 1, d, None),
        "la_action": lambda: L.la_action(None, None, None),
        "la_solve_step": lambda: L.la_solve_step(None, None, d, 1, None, None),
        "la_residual": lambda: L.la_residual(None, None, d, None, None, None),
        "la_relax_colour": lambda: L.la_relax_colour(None, None, d, 0, None),
        "la_time_matrices": lambda: L.la_time_matrices(None, d, None),
        "la_backward": lambda: L.la_backward(None, None, None, None),
        "la_step_batch": lambda: L.la_step_batch(None, 1, None, 1, None, None),
        "la_profile_enable": lambda: L.la_profile_enable(None, 1),
        "la_profile_read": lambda: L.la_profile_read(None, None),
        "la_action_noalloc": lambda: L.la_action_noalloc(None, None, None, None, d, None, None, None),
        "la_lfa_maps": lambda: L.la_lfa_maps(None, 1, None, 1, None, 1, None, None),
        "la_wait_selftest": lambda: L.la_wait_selftest(0, None, None),
        "la_fma_peaks": lambda: L.la_fma_peaks(None, None, None, None),
        "la_finalize": lambda: L.la_finalize(None),
    }
    assert set(calls) == set(B.EXPORTS) - {"la_last_error", "la_version"}
    for name, call in calls.items():
        assert call() == B.LA_EINVAL, name
    assert L.la_last_error(None)
