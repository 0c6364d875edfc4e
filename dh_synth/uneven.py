"""Seeded batches of windows of several frame sizes (the uneven-size workload).

Each frame size gets its own reconstruction distance z ~ U(0.25, 0.45) m; its windows
alternate between 32 and 64 frames and are laid end to end in one frame sequence of that
size; every window is drawn from its own speckle stream whose dynamic-speckle Doppler spread
is sigma_D ~ U(0.1, 1.0) rad per frame. Frames only: none of the method's arithmetic.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .speckle import SpeckleParams, SpeckleStream


@dataclass
class SizeGroup:
    n: int                  # frames are n x n
    z: float                # reconstruction distance of this size, metres
    frames: torch.Tensor    # uint16 [F, n, n]
    windows: list = field(default_factory=list)  # (first frame, T, sigma_D) per window

    def starts(self, T: int) -> list[int]:
        return [s for s, t, _ in self.windows if t == T]


def uneven_batch(sizes=((512, 40), (1024, 16), (2048, 4)), lengths=(32, 64), seed: int = 3000,
                 device="cpu") -> list[SizeGroup]:
    """One SizeGroup per (n, n_windows) of `sizes`; windows alternate through `lengths`."""
    rng = np.random.default_rng(seed)
    groups = []
    for gi, (n, nwin) in enumerate(sizes):
        z = float(rng.uniform(0.25, 0.45))
        ts = [lengths[w % len(lengths)] for w in range(nwin)]
        sig = rng.uniform(0.1, 1.0, size=nwin)
        frames = torch.empty((sum(ts), n, n), dtype=torch.uint16, device=device)
        g = SizeGroup(n=n, z=z, frames=frames)
        off = 0
        for w, (t, s) in enumerate(zip(ts, sig)):
            st = SpeckleStream(SpeckleParams(n, n, sigma_doppler=float(s)),
                               seed=seed * 1000 + gi * 100 + w, device=device)
            frames[off:off + t] = st.next(t)
            g.windows.append((off, t, float(s)))
            off += t
        groups.append(g)
    return groups
