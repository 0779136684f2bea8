"""Autotuner of batched runs.

A batch shares the GPU among many catalogs, so the persistent grids each context would
size for the whole GPU are too large: their idle CTAs crowd out the other catalogs' work.
The tuner times the batch itself (device time of the whole launch) for each candidate
grid divisor and keeps the fastest; results do not depend on the divisor.
"""
from __future__ import annotations

from . import gbsub

DIVISORS = (1, 2, 4, 8, 16, 32)


def tune_batch(batch: "gbsub.Batch", subs, divisors=DIVISORS, repeats=3):
    """Set the best divisor on every context of the batch; returns (best, {div: ms})."""
    timing = {}
    for div in divisors:
        for s in subs:
            gbsub.sub_set_grid_div(s.ctx, div)
        batch.run()  # rebuilds the graph and warms up
        best = None
        for _ in range(repeats):
            batch.run()
            best = batch.last_ms if best is None else min(best, batch.last_ms)
        timing[div] = best
    choice = min(timing, key=timing.get)
    for s in subs:
        gbsub.sub_set_grid_div(s.ctx, choice)
    batch.run()
    return choice, timing
