"""Host logic of the tuning table (no GPU): the autotuner's rule for the fan-out threshold,
and the build step that compiles tuning.json into the library's initialisers."""
import importlib
import json
import os

import pytest

from paper_1606_05973_gb300 import tile_sweep

# the module (the package exports a function of the same name)
build = importlib.import_module("paper_1606_05973_gb300.build")

SIDES = tile_sweep.STREAM_SIDES  # 4096, 6144, 8192, 12288, 16384


def test_fanout_threshold_from_recorded_sweeps():
    """The GB300 sweeps recorded in profiles/tuning_sweep.txt (ms per call, fanned out / three
    launches): one clears the 5% margin from 4096^2, the earliest only from 8192^2 (6144^2
    was 1.4% faster, under the margin), the latest from 6144^2 (it lost at 4096^2)."""
    later = ([0.2430, 0.4542, 0.7153, 1.5433, 2.6444], [0.2572, 0.5316, 0.8890, 1.9557, 3.4222])
    earlier = ([0.2510, 0.5256, 0.8032, 1.6725, 2.7880], [0.2568, 0.5331, 0.8986, 1.9608, 3.4332])
    latest = ([0.2658, 0.4547, 0.7132, 1.5380, 2.6623], [0.2495, 0.5299, 0.8971, 1.9536, 3.4111])
    assert tile_sweep.fanout_threshold(SIDES, *later) == 4096 * 4096
    assert tile_sweep.fanout_threshold(SIDES, *earlier) == 8192 * 8192
    assert tile_sweep.fanout_threshold(SIDES, *latest) == 6144 * 6144


def test_fanout_threshold_needs_every_larger_side():
    three = [1.0] * len(SIDES)
    win, tie, loss = 0.9, 0.96, 1.1
    assert tile_sweep.fanout_threshold(SIDES, [win] * 5, three) == SIDES[0] ** 2
    assert tile_sweep.fanout_threshold(SIDES, [loss] * 5, three) == -1
    # a win only at the largest side; a loss in the middle hides the wins below it
    assert tile_sweep.fanout_threshold(SIDES, [loss, loss, loss, loss, win], three) == SIDES[-1] ** 2
    assert tile_sweep.fanout_threshold(SIDES, [win, win, loss, win, win], three) == SIDES[3] ** 2
    # faster, but by less than the margin, counts as no win
    assert tile_sweep.fanout_threshold(SIDES, [win, win, win, win, tie], three) == -1


def test_tuning_source_compiles_the_committed_table():
    with open(build.TUNING) as f:
        t = json.load(f)
    src = build.tuning_source()
    assert src.count("LL, {") == len(t["rows"])
    assert f"kTuneStreamsMinPx = {int(t['streams_min_px'])}LL;" in src
    assert f"kTuneSingleFusedMaxPx = {int(t['single_fused_max_px'])}LL;" in src


def test_tuning_source_defaults_and_checks(tmp_path):
    with open(build.TUNING) as f:
        t = json.load(f)
    del t["streams_min_px"]  # a table written before the fan-out: never fan out
    p = os.path.join(tmp_path, "t.json")
    with open(p, "w") as f:
        json.dump(t, f)
    assert "kTuneStreamsMinPx = -1LL;" in build.tuning_source(p)
    t["rows"][-1]["max_px"] = 123  # the last row must be unbounded
    with open(p, "w") as f:
        json.dump(t, f)
    with pytest.raises(AssertionError):
        build.tuning_source(p)
