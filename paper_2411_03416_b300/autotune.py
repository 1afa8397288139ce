"""Autotuner for the execution form of served plans.

The block form's one tunable shape is the thread-block size per plan (32, 64,
128 or 256 threads sharing the plan's time axis).  More threads shorten the
cyclic-reduction levels and the per-state loops but leave fewer blocks per SM
for the plans that share the GPU, so the best size depends on the load: alone,
the largest block is fastest; on a busy GPU a middle size finishes a burst of
plans sooner.  The tuner times, for each (state dimension, dynamics kind,
horizon bucket), a batch of `copies` plans of one sample request in every
candidate size (copies = 1: an idle GPU; a few per SM: a loaded one), keeps
the fastest, and answers `choose(problem)` for requests, which the server
honours when it is created with plan_threads = -1.  Tables are plain JSON so
that a tuned table can be reused across runs.
"""
from __future__ import annotations

import json
import math
import time
from dataclasses import replace
from typing import Callable, Dict, Iterable, Optional, Tuple

CANDIDATES = (32, 64, 128, 256)

Key = Tuple[int, int, int]   # (n, dyn_kind, horizon bucket)


def bucket(problem) -> Key:
    """Horizon buckets by powers of two of the state count (the number of
    cyclic-reduction levels)."""
    return (int(problem.n), int(problem.dyn_kind), int(math.ceil(math.log2(problem.N + 1))))


def default_threads(problem) -> int:
    """Fallback without a measurement: about one thread per four states,
    within 32..256."""
    t = 32
    while t < 256 and 4 * t < problem.N + 1:
        t *= 2
    return t


def _time_on_device(problem, options, precision: int, repeats: int, copies: int) -> float:
    import torch

    from . import _lib
    probs, opts = [problem] * copies, [options] * copies
    _lib.solve(probs[:1], opts[:1], precision)            # module load and warm caches
    best = math.inf
    for _ in range(repeats):
        torch.cuda.synchronize()
        t = time.perf_counter()
        _lib.solve(probs, opts, precision)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
    return best


class Tuner:
    def __init__(self, table: Optional[Dict[Key, int]] = None):
        self.table: Dict[Key, int] = dict(table or {})
        self.timings: Dict[Key, Dict[int, float]] = {}

    def tune(self, samples: Iterable, precision: int, candidates=CANDIDATES, repeats: int = 2, copies: int = 1,
             timer: Optional[Callable] = None) -> Dict[Key, int]:
        """Times every candidate size on one sample (problem, options) per
        bucket, as a batch of `copies` plans, and keeps the fastest.
        `timer(problem, options, precision)` replaces the device timing (tests)."""
        timer = timer or (lambda p, o, prec: _time_on_device(p, o, prec, repeats, copies))
        for pb, op in samples:
            k = bucket(pb)
            if k in self.table:
                continue
            t = {c: timer(pb, replace(op, plan_threads=c), precision) for c in candidates}
            self.timings[k] = t
            self.table[k] = min(t, key=lambda c: (t[c], c))
        return self.table

    def choose(self, problem) -> int:
        return self.table.get(bucket(problem), default_threads(problem))

    def apply(self, problem, options):
        """The request's options with the tuned block size."""
        return replace(options, plan_threads=self.choose(problem))

    def to_json(self) -> str:
        return json.dumps({"table": [[list(k), v] for k, v in sorted(self.table.items())]})

    @classmethod
    def from_json(cls, text: str) -> "Tuner":
        d = json.loads(text)
        return cls({tuple(k): int(v) for k, v in d["table"]})
