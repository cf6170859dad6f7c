"""The paper's parallel processing scheme on one GPU (Sec. "Simulating live and
parallel processing"): the positions are split into disjoint subsets, each
subset is iterated independently for a few sweeps from the common object and
illumination, and the results are averaged for synchronisation, a hybrid
between ePIE and batch methods (after Nashed et al. 2014).  The paper notes
that the result depends on the number of subsets.

Each subset is an engine handle with its own stream; a round runs their
sweeps concurrently (epie_iterate_many) and then averages on the device
(epie_average_state).  Subset q draws its visiting order from seed + q.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B


class ParallelAveraging:
    def __init__(self, N, obj_h, obj_w, probe0, subsets_pos, object0=None, mode=B.EPIE_SEQUENTIAL,
                 seed=0, capacity=None, device=0, flags=0, **kw):
        self.engines = [B.Engine(N, obj_h, obj_w, probe0, object0, mode=mode, seed=seed + q,
                                 capacity=capacity or max(len(p), 1), device=device, flags=flags,
                                 **kw)
                        for q, p in enumerate(subsets_pos)]

    def append(self, q, frames, pos):
        """Frames of subset q (live: subsets may grow round-robin)."""
        self.engines[q].append(frames, pos)

    def round(self, sweeps):
        """`sweeps` independent sweeps per subset, then the average.  Returns the
        per-subset sweep errors [n_subsets, sweeps]."""
        errs = B.epie_iterate_many([e.h for e in self.engines], sweeps)
        B.epie_average_state([e.h for e in self.engines])
        return errs

    def object(self):
        return self.engines[0].object()

    def probe(self):
        return self.engines[0].probe()

    def close(self):
        for e in self.engines:
            e.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
