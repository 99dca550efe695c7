"""Host logic of the autotuner (no GPU): choosing the fastest candidate, skipping the ones the
library refuses, the signature and the JSON cache."""
from types import SimpleNamespace

import pytest

from paper_2005_11931_gb300 import autotune, tsu


def test_pick_takes_the_fastest_and_skips_refused_candidates():
    cands = [autotune.Choice(1, 0, 0), autotune.Choice(2, 4, 64), autotune.Choice(2, 4, 128),
             autotune.Choice(3, 8, 128)]
    cost = {cands[0]: 9.0, cands[1]: 3.0, cands[2]: 2.5, cands[3]: 1.0}
    calls = []

    def run(c):
        calls.append(c)
        if c.kernel == 3:
            raise tsu.TsuError(tsu.TSU_EINVAL, "run", "refused")


    def timer(fn):
        fn()
        return cost[calls[-1]]

    best, times = autotune.pick(cands, run, timer, repeats=3)
    assert best == cands[2]
    assert cands[3] not in times
    # every accepted candidate: one untimed run, then three timed
    assert sum(1 for c in calls if c == cands[1]) == 4


def test_pick_fails_when_nothing_runs():
    def run(c):
        raise tsu.TsuError(tsu.TSU_EINVAL, "run", "no")

    with pytest.raises(RuntimeError):
        autotune.pick([autotune.Choice(2, 4, 0)], run, lambda fn: 0.0)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = autotune.Cache(path)
    assert c.get("k") is None
    c.put("k", autotune.Choice(2, 4, 96, True))
    assert autotune.Cache(path).get("k") == autotune.Choice(2, 4, 96, True)


def test_signature_ignores_problem_order():
    a = SimpleNamespace(g=SimpleNamespace(nx=100, ny=90, ld=128), dtype=0, form=1)
    b = SimpleNamespace(g=SimpleNamespace(nx=300, ny=300, ld=320), dtype=0, form=1)
    assert autotune.signature("batch", [a, b]) == autotune.signature("batch", [b, a])
    assert autotune.signature("batch", [a, b]) != autotune.signature("step", [a, b])


def test_candidates_are_valid_configurations():
    for c in autotune.batch_candidates():
        assert c.kernel in (2, 3) and (c.tdepth in (2, 4) if c.kernel == 2 else c.tdepth in (4, 8))
    for c in autotune.step_candidates():
        assert c.kernel in (1, 2, 3, 4)
        if c.kernel == 4:  # the persistent pass has one depth (4 steps per pass)
            assert c.tdepth in (0, 4)
