"""Autotuner candidate lists (host logic, no GPU): irregular blocking tries
threshold 0 over Algorithm 3's sample count, b_min and max_num, deduplicated
on the effective sample count S = min(sample_points, n / b_min), plus the
paper defaults at threshold 0.3; regular blocking tries the thresholds."""
from paper_2512_04389_b300 import tune as T


def _eff(c, n):
    return min(c["sample_points"], n // c["b_min"]), c["max_num"], c["dense_threshold"]


def test_irregular_candidates_unique_plans():
    for n in (64, 2304, 64_000, 200_000):
        cs = T.candidates("irregular", n)
        effs = [_eff(c, n) for c in cs]
        assert len(effs) == len(set(effs))
        assert {"dense_threshold": 0.3, "sample_points": 1000, "b_min": 32,
                "max_num": 3} in cs
        assert {c["max_num"] for c in cs} == {1, 2, 3}


def test_candidate_counts():
    # n = 64,000: S = min(sample_points, n / b_min) in {2000, 1000, 500}
    # (b_min 128 gives 500; 8 and 32 give no new S) x max_num + 1
    assert len(T.candidates("irregular", 64_000)) == 10
    # n = 2304: S in {72, 288, 36, 18} (sample_points irrelevant) x max_num + 1
    assert len(T.candidates("irregular", 2304)) == 13
    assert T.candidates("regular") == [{"dense_threshold": t} for t in T.THRESHOLDS]


def test_cache_key_covers_pattern_options_and_library(monkeypatch):
    import numpy as np
    cp, ri = np.array([0, 1, 2]), np.array([0, 1])
    k0 = T._key(2, cp, ri, {"precision": "fp64"})
    assert k0 == T._key(2, cp, ri, {"precision": "fp64"})
    assert k0 != T._key(2, cp, ri, {"precision": "fp32"})
    assert k0 != T._key(2, np.array([0, 2, 2]), np.array([0, 1]), {"precision": "fp64"})
    monkeypatch.setattr(T, "_SOURCES", "another build")
    assert k0 != T._key(2, cp, ri, {"precision": "fp64"})
