"""Autotuner candidates are configurations la_init accepts (checked on the CPU: with device
allocations refused, a valid configuration gets as far as LA_ENOMEM, an invalid one stops at LA_EINVAL)."""
import dataclasses

import pytest

from paper_1111_4363_gb300 import workloads as wl


@pytest.mark.parametrize("n", [64, 128, 256])
def test_every_candidate_passes_validation(monkeypatch, n):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1111_4363_gb300 import autotune
    from paper_1111_4363_gb300 import binding as B
    monkeypatch.setenv("LA_FAIL_ALLOC", "1")
    w = dataclasses.replace(wl.batched_2d(0), n=(n, n, 1), trial=3)
    cands = autotune.candidates(w)
    assert len(cands) >= 20
    shapes = {(c["levels"] > 1, c["nu1"], c["nu2"]) for c in cands}
    assert (True, 1, 2) in shapes and (False, 1, 0) in shapes
    for cand in cands:
        cfg = B.config_from_workload(dataclasses.replace(w, **cand))
        with pytest.raises(B.LeastActionError) as e:
            B.Context(cfg)
        assert e.value.status == B.LA_ENOMEM, (cand, str(e.value))


def test_cache_key_separates_precision_and_trial():
    from paper_1111_4363_gb300 import autotune
    w = wl.batched_2d(0)
    keys = {autotune.key(dataclasses.replace(w, trial=t), p) for t in (0, 3) for p in (0, 1)}
    assert len(keys) == 4
