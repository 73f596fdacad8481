"""Device-time measurement of one launch with CUDA events.

GB300's event clock advances in steps of about 2 us, and an event pair around
a single short launch also counts the launch's own start-up, so a kernel of a
few microseconds cannot be timed launch by launch.  Two ways are used here:

- operands larger than L2 (no flush): the trimmed mean of per-launch event
  intervals (launches of 100 us and more; the tick is noise there);
- operands that fit in L2: `reps` pairs (L2 flush, launch) are queued back to
  back inside ONE event interval, the same number of flushes alone inside
  another (three interleaved rounds, median difference), and the difference
  divided by `reps` is the launch's cost in the stream, with a cold L2 at
  every launch; a launch lost in the flushes' own jitter reads as 0.  The
  flush reads a buffer larger than L2, which evicts it without leaving dirty
  lines behind.
"""
from __future__ import annotations

import statistics
from typing import Callable, List, Optional

import torch


def trimmed_mean(times: List[float], cut: float = 0.2) -> float:
    """Mean of the values left after dropping the lowest and highest `cut`
    fraction (at least one value is kept)."""
    t = sorted(times)
    k = int(len(t) * cut)
    mid = t[k:len(t) - k] or t
    return statistics.fmean(mid)


def _interval_ms(body: Callable[[], None], stream) -> float:
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    body()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def launch_time_us(fn: Callable[[], None], reps: int, flush: Optional[torch.Tensor] = None,
                   stream=None) -> float:
    """Device time of one call of `fn` (which launches on `stream`, default the
    current stream), in microseconds; see the module docstring."""
    if stream is None:
        stream = torch.cuda.current_stream()
    reps = max(int(reps), 1)
    if flush is None:
        return trimmed_mean([_interval_ms(fn, stream) * 1e3 for _ in range(reps)])

    def flushes():
        for _ in range(reps):
            flush.sum()

    def pairs():
        for _ in range(reps):
            flush.sum()
            fn()

    with torch.cuda.stream(stream):
        _interval_ms(flushes, stream)        # brings the clocks up; discarded
        diffs = []
        for _ in range(3):                   # interleaved against clock drift
            t_f = _interval_ms(flushes, stream)
            t_b = _interval_ms(pairs, stream)
            diffs.append(t_b - t_f)
    return max(statistics.median(diffs) * 1e3 / reps, 0.0)


def warm_time_us(fn: Callable[[], None], reps: int, stream=None) -> float:
    """Device time of one call of `fn` with its operands left in L2 by the
    previous call: `reps` calls back to back in one event interval (after one
    call to warm L2), in microseconds."""
    if stream is None:
        stream = torch.cuda.current_stream()
    reps = max(int(reps), 1)

    def calls():
        for _ in range(reps):
            fn()

    with torch.cuda.stream(stream):
        fn()
        return _interval_ms(calls, stream) * 1e3 / reps
