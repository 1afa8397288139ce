"""Host logic of the block-size autotuner (no device: timings are injected)."""
from dataclasses import replace

import workloads as W
from paper_2411_03416_b300 import autotune


def test_tuner_picks_fastest_per_bucket_and_round_trips():
    calls = []

    def fake_timer(pb, op, prec):
        calls.append((pb.N, op.plan_threads))
        # a synthetic latency model: small blocks win on short horizons, large on long ones
        return abs(op.plan_threads - (32 if pb.N < 100 else 256)) + 1.0

    short = W.c1_point2d(N=50)
    long_ = W.c1_point2d(N=700)
    long_twin = W.c1_point2d(request=3, N=600)        # same bucket as N = 700
    tuner = autotune.Tuner()
    table = tuner.tune([short, long_, long_twin], precision=1, timer=fake_timer)
    assert table[autotune.bucket(short[0])] == 32
    assert table[autotune.bucket(long_[0])] == 256
    assert len(calls) == 2 * len(autotune.CANDIDATES)  # one sample per bucket
    assert tuner.apply(*long_twin).plan_threads == 256
    again = autotune.Tuner.from_json(tuner.to_json())
    assert again.table == tuner.table


def test_untuned_bucket_falls_back_to_the_rule():
    tuner = autotune.Tuner()
    for N, want in [(10, 32), (200, 64), (1000, 256)]:
        pb, op = W.c1_point2d(N=N)
        assert tuner.choose(pb) == want == autotune.default_threads(pb)
        assert tuner.apply(pb, op).plan_threads == want
        assert replace(op, plan_threads=0).plan_threads == 0   # options are not mutated
