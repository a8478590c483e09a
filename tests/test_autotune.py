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
    # K = 4 reaches the 8 x 8 subvolume (256 unknowns); every candidate also with one matrix per CTA
    assert any(c["sub"][:2] == (8, 8) for c in cands)
    cands = cands + [dict(c, factor_group=1) for c in cands[:3]]
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


def test_tune_ranks_by_time_among_converged_candidates_and_caches(monkeypatch, tmp_path):
    """tune() on the CPU with the GPU measurement replaced: the fastest candidate that reached the
    tolerance wins, candidates that did not converge or were rejected by la_init are skipped, the
    table is cached and a second call reads the cache without measuring."""
    from paper_1111_4363_gb300 import autotune
    from paper_1111_4363_gb300 import binding as B
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    w = dataclasses.replace(wl.batched_2d(0), n=(128, 128, 1), trial=3)
    cands = autotune.candidates(w)
    calls = []

    def fake_measure(wc, precision):
        i = len(calls)
        calls.append(wc)
        if wc.factor_group == 1:                    # packing pass: the second of the three is faster still
            return {"ms_per_step": 9.0 if i == len(cands) + 1 else 100.0, "cycles": 2.0, "rel": w.tol / 2}
        if i == 0:
            raise B.LeastActionError(B.LA_EINVAL, "rejected")
        rel = 1.0 if i == 1 else w.tol / 2          # candidate 1 is the fastest but does not converge
        return {"ms_per_step": 0.5 if i == 1 else 10.0 + (i * 7919) % 13, "cycles": 2.0, "rel": rel}

    monkeypatch.setattr(autotune, "measure", fake_measure)
    best = autotune.tune(w, 0)
    assert len(calls) == len(cands) + 3
    times = {i: 10.0 + (i * 7919) % 13 for i in range(2, len(cands))}
    ranked = sorted(times, key=lambda i: (times[i], i))
    assert best == dict(cands[ranked[1]], factor_group=1)
    assert [c.factor_group for c in calls[len(cands):]] == [1, 1, 1]
    monkeypatch.setattr(autotune, "measure", lambda *a: pytest.fail("measured despite the cache"))
    assert autotune.tune(w, 0) == best
    table = __import__("json").load(open(autotune.CACHE))[autotune.key(w, 0)]["table"]
    assert len(table) == len(cands) - 2 + 3


def test_tune_reports_when_nothing_converges(monkeypatch, tmp_path):
    from paper_1111_4363_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "measure", lambda wc, p: {"ms_per_step": 1.0, "cycles": 9.0, "rel": 1.0})
    with pytest.raises(RuntimeError, match="no candidate"):
        autotune.tune(dataclasses.replace(wl.batched_2d(0), n=(64, 64, 1)), 0)
