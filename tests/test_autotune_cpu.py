"""Host-side choices of the autotuner (no device needed)."""
from paper_2609_05494_b300 import autotune


def _c(a, b, ms):
    return {"a": a, "b": b, "ms": ms}


def test_persistent_split_keeps_the_default_on_near_ties():
    # timings of the 64-case sweep's tuning horizon on one B300: the split by
    # particles x steps is within 0.3 % of the fastest and is kept
    cands = [_c(1.0, 0.0, 909.3), _c(1.0, 1.0, 731.6), _c(1.0, 0.5, 766.4), _c(0.5, 1.0, 729.8)]
    a, b, ms = autotune.choose_weight(cands)
    assert (a, b) == autotune.DEFAULT_WEIGHT and ms == 731.6


def test_persistent_split_takes_a_clearly_faster_candidate():
    cands = [_c(1.0, 1.0, 800.0), _c(0.5, 1.0, 700.0)]
    assert autotune.choose_weight(cands)[:2] == (0.5, 1.0)
    # without the default among the candidates, the fastest
    assert autotune.choose_weight([_c(1.0, 0.0, 5.0), _c(0.5, 1.0, 4.0)])[:2] == (0.5, 1.0)
    # the margin is a fraction of the fastest time
    assert autotune.choose_weight(cands, margin=0.2)[:2] == (1.0, 1.0)
