"""Host logic of the batched-plan autotuner (CPU only, fake timings)."""
import json

from paper_2401_14117_gb300 import autotune


def test_candidates_fit_the_sm():
    cands = autotune.candidates()
    assert cands
    for threads, ctas, smem in cands:
        assert threads % 32 == 0 and threads * ctas <= autotune.THREADS_PER_SM
        assert smem * ctas <= autotune.SMEM_PER_SM
        assert smem <= autotune.SMEM_PER_CTA_MAX


def test_choose_prefers_fastest_then_smaller():
    t = {(256, 1, 1000): 2.0, (128, 2, 1000): 1.0, (128, 1, 1000): 1.0}
    assert autotune.choose(t) == (128, 1, 1000)


def test_tune_measures_every_candidate_and_caches(tmp_path):
    calls = []

    def fake(p):
        calls.append(p)
        return 1.0 / (p[0] * p[1]) + p[2] * 1e-9

    path = str(tmp_path / "cache.json")
    best, timings = autotune.tune(fake, "gpu|n2^4-2^9", cache_path=path)
    assert len(calls) == len(autotune.candidates())
    assert best == min(timings, key=timings.get)
    saved = json.load(open(path))
    assert saved["gpu|n2^4-2^9"]["plan"] == list(best)
    calls.clear()
    best2, _ = autotune.tune(fake, "gpu|n2^4-2^9", cache_path=path)
    assert best2 == best and calls == []  # served from the cache


def test_bucket_key():
    assert autotune.bucket_key("GB300", [16, 512]) == "GB300|n2^4-2^9"
    assert autotune.bucket_key("GB300", [17, 500]) == "GB300|n2^4-2^9"
