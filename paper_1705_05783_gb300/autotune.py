"""Per-shape choice of the engine's equivalent kernel schedules.

The ILU(0) wavefront sweeps run either one 8x4-row tile per warp or 2x2
tiles per CTA (the same arithmetic, bitwise-equal results), and the
symmetric coarse solve runs in one CTA or across a thread-block cluster.
Which is faster depends on the grid, the coarse grid and the precision, so
`tune` times a few C-AMS iterations of a live handle under every schedule the
handle accepts (cams_set_schedule refuses those this GPU or grid cannot run)
and keeps the fastest.  `ScheduleCache` remembers the choice per shape, so
that handles of the same shape (members of an ensemble) are timed once.

Everything here drives the C-ABI; the timings are host wall clock around
calls that return only when their GPU work is done (cams_iterate reads each
residual norm back).
"""
from __future__ import annotations

import itertools
import time

from . import cams

# (ilu_cta, coarse_cluster)
CANDIDATES = tuple(itertools.product((0, 1), (0, 1)))


def tune(h, p_n, dt, bc, iters=3, repeats=2, candidates=CANDIDATES, clock=time.perf_counter):
    """Time `repeats` runs of `iters` C-AMS iterations from p_n (the system
    assembled at p_n, the basis built once) under every candidate schedule,
    set the fastest and leave the handle assembled at p_n.  Returns
    (choice, {candidate: best seconds}); choice is None when the handle
    accepts no candidate (the level-scheduled sweeps)."""
    cams.cams_assemble(h, p_n, p_n, dt, bc)
    cams.cams_update_basis(h, True)
    times = {}
    for cand in candidates:
        try:
            cams.cams_set_schedule(h, *cand)
        except cams.CamsError:
            continue
        # one untimed run: it captures the iteration graph of the new schedule
        cams.cams_assemble(h, p_n, p_n, dt, bc)
        cams.cams_iterate(h, 1)
        best = float("inf")
        for _ in range(repeats):
            cams.cams_assemble(h, p_n, p_n, dt, bc)
            t0 = clock()
            cams.cams_iterate(h, iters)
            best = min(best, clock() - t0)
        times[cand] = best
    choice = min(times, key=times.get) if times else None
    if choice is not None:
        cams.cams_set_schedule(h, *choice)
    cams.cams_assemble(h, p_n, p_n, dt, bc)
    return choice, times


def tune_ensemble(handles, run, repeats=2, candidates=CANDIDATES, clock=time.perf_counter):
    """Tune the schedule of an ensemble as it runs: under each candidate
    (set on every handle that accepts it; the others keep theirs) time
    `repeats` calls of run(), which runs the whole ensemble once, after one
    untimed call (graph capture); keep the fastest candidate on every handle.
    Members that run concurrently share the GPU, so a schedule timed on one
    handle alone need not be the fastest among them.  Returns
    (choice, {candidate: best seconds})."""
    times = {}
    for cand in candidates:
        accepted = 0
        for h in handles:
            try:
                cams.cams_set_schedule(h, *cand)
                accepted += 1
            except cams.CamsError:
                pass
        if accepted == 0:
            continue
        run()
        best = float("inf")
        for _ in range(repeats):
            t0 = clock()
            run()
            best = min(best, clock() - t0)
        times[cand] = best
    choice = min(times, key=times.get) if times else None
    if choice is not None:
        for h in handles:
            try:
                cams.cams_set_schedule(h, *choice)
            except cams.CamsError:
                pass
    return choice, times


def shape_key(nx, ny, nz, coarse, precision, restriction):
    return (int(nx), int(ny), int(nz), tuple(int(b) for b in coarse), int(precision),
            int(restriction))


class ScheduleCache:
    """Tuned schedules per shape key (see shape_key)."""

    def __init__(self):
        self.table = {}

    def apply(self, h, key, p_n, dt, bc, **kw):
        """Give h the schedule tuned for its shape, tuning on h the first
        time the shape is seen; returns the schedule (or None)."""
        if key in self.table:
            if self.table[key] is not None:
                cams.cams_set_schedule(h, *self.table[key])
            return self.table[key]
        choice, _ = tune(h, p_n, dt, bc, **kw)
        self.table[key] = choice
        return choice
