"""Autotuner of batched runs.

A batch shares the GPU among many catalogs, so the launch settings each context would pick
for a whole GPU are not the best ones: persistent grids sized for the whole GPU crowd out
the other catalogs' work, and a sort or a median tile with fewer threads can pack better.
The tuner times the batch itself (device time of the whole launch) over the settings that
leave results unchanged (sub_set_tuning): first the grid divisor, then, at the best
divisor, the sort's elements per thread and the median's threads per tile, keeping each
choice that is faster.
"""
from __future__ import annotations

from . import gbsub

DIVISORS = (1, 2, 4, 8, 16, 32)
SORT_WIDTHS = (0, 4, 8)          # 0: automatic (2 for the default window)
MEDIAN_THREADS = (0, 256, 128)   # 0: automatic (512 for the default window)


def _time(batch, repeats):
    batch.run()  # rebuilds the graph and warms up
    best = None
    for _ in range(repeats):
        batch.run()
        best = batch.last_ms if best is None else min(best, batch.last_ms)
    return best


def _apply(subs, knob, value):
    """Set a knob on every context; False when a context does not allow the value."""
    try:
        for s in subs:
            gbsub.sub_set_tuning(s.ctx, knob, value)
        return True
    except gbsub.SubError:
        for s in subs:
            gbsub.sub_set_tuning(s.ctx, knob, 0 if knob != gbsub.TUNE_GRID_DIV else 1)
        return False


def tune_batch(batch: "gbsub.Batch", subs, divisors=DIVISORS, sort_widths=SORT_WIDTHS,
               median_threads=MEDIAN_THREADS, repeats=3):
    """Set the fastest settings on every context of the batch.  Returns (settings, timings):
    settings {"grid_div", "sort_e", "median_threads"} (0: automatic), timings {label: ms}."""
    timings = {}
    for div in divisors:
        _apply(subs, gbsub.TUNE_GRID_DIV, div)
        timings["grid_div=%d" % div] = _time(batch, repeats)
    div = min(divisors, key=lambda d: timings["grid_div=%d" % d])
    _apply(subs, gbsub.TUNE_GRID_DIV, div)
    settings = {"grid_div": div, "sort_e": 0, "median_threads": 0}
    best = timings["grid_div=%d" % div]
    for name, knob, values in (("sort_e", gbsub.TUNE_SORT_E, sort_widths),
                               ("median_threads", gbsub.TUNE_MEDIAN_THREADS, median_threads)):
        for v in values:
            if v == 0 or not _apply(subs, knob, v):
                continue
            ms = _time(batch, repeats)
            timings["%s=%d" % (name, v)] = ms
            if ms < best:
                best, settings[name] = ms, v
        _apply(subs, knob, settings[name])
    batch.run()
    return settings, timings
