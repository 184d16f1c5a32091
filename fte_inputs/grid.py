"""Spherical snapshot grid description and memory layout (the data interface).

A background is a sequence of `n_snap` snapshots of cell-centred data on a
spherical (r, theta, phi) grid (finite-volume output, Sec. 2.2).  Each cell holds
one record of REC float32 values:

    0..2   B  (Cartesian, nT)
    3..5   V  (Cartesian, au/s), in the frame the snapshot is given in
    6..14  dV_i/dx_j, row-major i (component) then j (direction), 1/s
    15..17 d|B|/dx_j (nT/au)
    18..23 padding (zero): 96-byte records, so that two r-neighbours form one
           32-byte aligned 192-byte block

Array order is [snap][phi][theta][r][REC] (r fastest).  Cell k along an axis
spans faces edge_k .. edge_{k+1}; phi covers [0, 2 pi) periodically.  With
radial='log' the r faces are geometric (grid stretching, Sec. 4).
"""
from dataclasses import dataclass, asdict
import math
import numpy as np

NFIELD = 18
REC = 24


@dataclass
class GridSpec:
    nr: int
    nth: int
    nph: int
    r_min: float = 0.1                 # au
    r_max: float = 2.0                 # au
    th_min: float = math.radians(30.0)
    th_max: float = math.radians(150.0)
    radial: str = "linear"             # 'linear' | 'log'
    n_snap: int = 1
    periodic: bool = False             # snapshot sequence periodic in time
    t_snap0: float = 0.0               # s, time of snapshot 0
    dt_snap: float = 3600.0            # s

    def cells(self):
        return self.nr * self.nth * self.nph

    def snapshot_bytes(self):
        return self.cells() * REC * 4

    def as_dict(self):
        return asdict(self)


def cell_centres(g: GridSpec):
    """Cell-centre coordinates (r, theta, phi) along each axis, float64."""
    i = np.arange(g.nr) + 0.5
    if g.radial == "log":
        dl = math.log(g.r_max / g.r_min) / g.nr
        r = g.r_min * np.exp(i * dl)
    else:
        r = g.r_min + i * (g.r_max - g.r_min) / g.nr
    th = g.th_min + (np.arange(g.nth) + 0.5) * (g.th_max - g.th_min) / g.nth
    ph = (np.arange(g.nph) + 0.5) * (2.0 * math.pi / g.nph)
    return r, th, ph
