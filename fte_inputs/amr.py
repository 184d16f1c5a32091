"""Block-AMR spherical grids (Sec. 2.2 / 2.4): tree, lookup table and per-leaf data.

Geometry: the domain [r_min, r_max] x [th_min, th_max] x [0, 2 pi) is split into
nbr x nbt x nbp base blocks (level 0) of B^3 cells; each refinement halves a
block in every direction (Sec. 2.4), up to `levels - 1` times.  Neighbouring
leaves (faces, edges and corners) differ by at most one level (2:1 nesting,
Sec. 2.4).  Radial coordinate: uniform in ln r ("log", the stretched grid of
Sec. 4) or in r ("linear").

Data handed to both implementations:
* leaves  int32 [n_leaf, 4] = (level, bi, bj, bk), block index at its own level,
          sorted by the Morton key of the block's origin at the finest level;
* table   int32 [nbp 2^L, nbt 2^L, nbr 2^L] (L = levels - 1): the leaf covering
          each finest-level block position;
* fields  float32 [n_snap, n_leaf, B+2, B+2, B+2, REC] (phi, theta, r order),
          interior cells filled, the one-cell ghost layer left zero.

Field values come from the same analytic winds as the uniform grids; the
gradients are second-order central differences at the leaf's own resolution,
using the analytic field one cell beyond the block (a halo), mapped to
Cartesian derivatives.
"""
from dataclasses import dataclass
import math

import numpy as np
import torch

from . import backgrounds as bgm
from .grid import REC

_F64 = torch.float64


@dataclass
class AmrSpec:
    nbr: int = 32
    nbt: int = 8
    nbp: int = 24
    bsize: int = 16
    levels: int = 3
    r_min: float = 0.1
    r_max: float = 2.0
    th_min: float = math.radians(30.0)
    th_max: float = math.radians(150.0)
    radial: str = "log"
    n_snap: int = 1
    periodic: bool = False
    t_snap0: float = 0.0
    dt_snap: float = 3600.0

    @property
    def L(self):
        return self.levels - 1

    def cells(self, level):
        f = (1 << level) * self.bsize
        return self.nbr * f, self.nbt * f, self.nbp * f

    def finest_blocks(self):
        f = 1 << self.L
        return self.nbr * f, self.nbt * f, self.nbp * f


def _r_of(spec, u):
    """r at normalised radial coordinate u in [0, 1]."""
    if spec.radial == "log":
        return spec.r_min * np.exp(u * math.log(spec.r_max / spec.r_min))
    return spec.r_min + u * (spec.r_max - spec.r_min)


def centres_1d(spec, level, axis, idx):
    """Cell-centre coordinate of global level-`level` cell indices idx along axis 0 (r), 1 (th), 2 (ph)."""
    n = spec.cells(level)[axis]
    u = (np.asarray(idx, dtype=np.float64) + 0.5) / n
    if axis == 0:
        return _r_of(spec, u)
    if axis == 1:
        return spec.th_min + u * (spec.th_max - spec.th_min)
    return u * 2.0 * math.pi


def morton3(a, b, c, bits=10):
    """Interleave the bits of (c, b, a) -> key (a lowest)."""
    key = np.zeros(np.shape(a), dtype=np.int64)
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    for k in range(bits):
        key |= ((a >> k) & 1) << (3 * k)
        key |= ((b >> k) & 1) << (3 * k + 1)
        key |= ((c >> k) & 1) << (3 * k + 2)
    return key


def finest_table(spec, leaves):
    """int32 [nbp 2^L, nbt 2^L, nbr 2^L] of leaf ids covering each finest-level block."""
    fr, ft, fp = spec.finest_blocks()
    tab = np.full((fp, ft, fr), -1, dtype=np.int32)
    for n, (lv, bi, bj, bk) in enumerate(leaves):
        s = 1 << (spec.L - lv)
        tab[bk * s:(bk + 1) * s, bj * s:(bj + 1) * s, bi * s:(bi + 1) * s] = n
    return tab


def _split(lv, bi, bj, bk):
    return [(lv + 1, 2 * bi + a, 2 * bj + b, 2 * bk + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]


def build_leaves(spec, refine):
    """Leaves after refining every block for which refine(level, bi, bj, bk) holds, then
    enforcing 2:1 nesting across faces, edges and corners; Morton-sorted int32 [n, 4]."""
    from scipy import ndimage
    leaves = [(0, i, j, k) for k in range(spec.nbp) for j in range(spec.nbt) for i in range(spec.nbr)]
    for lv in range(spec.L):
        nxt = []
        for leaf in leaves:
            if leaf[0] == lv and refine(*leaf):
                nxt.extend(_split(*leaf))
            else:
                nxt.append(leaf)
        leaves = nxt
    while True:      # 2:1 balance: refine any leaf with a neighbour two levels finer
        tab = finest_table(spec, leaves)
        lev = np.array([l[0] for l in leaves], dtype=np.int32)[tab]
        nb = ndimage.maximum_filter(lev, size=3, mode=("wrap", "nearest", "nearest"))
        marks = set()
        for n, (lv, bi, bj, bk) in enumerate(leaves):
            s = 1 << (spec.L - lv)
            if nb[bk * s:(bk + 1) * s, bj * s:(bj + 1) * s, bi * s:(bi + 1) * s].max() > lv + 1:
                marks.add(n)
        if not marks:
            break
        nxt = []
        for n, leaf in enumerate(leaves):
            nxt.extend(_split(*leaf) if n in marks else [leaf])
        leaves = nxt
    arr = np.array(leaves, dtype=np.int32)
    s = (1 << (spec.L - arr[:, 0])).astype(np.int64)
    key = morton3(arr[:, 1] * s, arr[:, 2] * s, arr[:, 3] * s)
    return np.ascontiguousarray(arr[np.argsort(key, kind="stable")])


def check_balance(spec, leaves):
    """True if every pair of touching leaves differs by at most one level."""
    from scipy import ndimage
    tab = finest_table(spec, leaves)
    if (tab < 0).any():
        return False
    lev = leaves[:, 0][tab]
    hi = ndimage.maximum_filter(lev, size=3, mode=("wrap", "nearest", "nearest"))
    lo = ndimage.minimum_filter(lev, size=3, mode=("wrap", "nearest", "nearest"))
    return bool((hi - lev).max() <= 1 and (lev - lo).max() <= 1)


# ---------------------------------------------------------------------------
# fields
# ---------------------------------------------------------------------------
def _leaf_lattice(spec, leaf, halo=1):
    lv, bi, bj, bk = (int(v) for v in leaf)
    B = spec.bsize
    idx = np.arange(-halo, B + halo)
    r = centres_1d(spec, lv, 0, bi * B + idx)
    th = centres_1d(spec, lv, 1, bj * B + idx)
    ph = centres_1d(spec, lv, 2, bk * B + idx)
    return r, th, ph


def _pack_leaf(rec, B_, V_, r, th, ph):
    """Interior records of one leaf from Cartesian B, V on the (B+2)^3 lattice [ph, th, r]."""
    R = torch.as_tensor(r, dtype=_F64)[None, None, :]
    TH = torch.as_tensor(th, dtype=_F64)[None, :, None]
    PH = torch.as_tensor(ph, dtype=_F64)[:, None, None]
    P = len(r)
    basis = bgm._basis(TH, PH)
    ST = torch.sin(TH)
    rhat, that, phat = [[torch.broadcast_to(c, (P, P, P)) for c in v] for v in basis]
    Rt = torch.as_tensor(r, dtype=_F64)
    Tt = torch.as_tensor(th, dtype=_F64)
    dph = float(ph[1] - ph[0])

    def grad(f):
        # central differences on the interior (non-uniform in r)
        h1 = (Rt[1:-1] - Rt[:-2])[None, None, :]
        h2 = (Rt[2:] - Rt[1:-1])[None, None, :]
        fr = (-h2 / (h1 * (h1 + h2)) * f[1:-1, 1:-1, :-2] + (h2 - h1) / (h1 * h2) * f[1:-1, 1:-1, 1:-1]
              + h1 / (h2 * (h1 + h2)) * f[1:-1, 1:-1, 2:])
        dth = float(Tt[1] - Tt[0])
        ft = (f[1:-1, 2:, 1:-1] - f[1:-1, :-2, 1:-1]) / (2 * dth)
        fp = (f[2:, 1:-1, 1:-1] - f[:-2, 1:-1, 1:-1]) / (2 * dph)
        Ri = R[:, :, 1:-1]
        Si = ST[:, 1:-1, :]
        return [fr * rhat[j][1:-1, 1:-1, 1:-1] + ft * that[j][1:-1, 1:-1, 1:-1] / Ri
                + fp * phat[j][1:-1, 1:-1, 1:-1] / (Ri * Si) for j in range(3)]

    out = torch.from_numpy(rec)
    inner = (slice(1, -1),) * 3
    for i in range(3):
        out[inner + (i,)] = B_[i][1:-1, 1:-1, 1:-1]
        out[inner + (3 + i,)] = V_[i][1:-1, 1:-1, 1:-1]
        g = grad(V_[i])
        for j in range(3):
            out[inner + (6 + 3 * i + j,)] = g[j]
    Bm = torch.sqrt(B_[0] ** 2 + B_[1] ** 2 + B_[2] ** 2)
    g = grad(Bm)
    for j in range(3):
        out[inner + (15 + j,)] = g[j]


def fields(spec, leaves, model="cir", **kw):
    """float32 [n_snap, n_leaf, B+2, B+2, B+2, REC]; interior filled, ghost layer zero."""
    B = spec.bsize
    P = B + 2
    out = np.zeros((spec.n_snap, len(leaves), P, P, P, REC), dtype=np.float32)
    for s in range(spec.n_snap):
        t = spec.t_snap0 + s * spec.dt_snap
        for n, leaf in enumerate(leaves):
            r, th, ph = _leaf_lattice(spec, leaf)
            R = torch.as_tensor(r, dtype=_F64)[None, None, :]
            TH = torch.as_tensor(th, dtype=_F64)[None, :, None]
            PH = torch.as_tensor(ph, dtype=_F64)[:, None, None]
            if model == "cir":
                B_, V_ = bgm.cir_fields(R, TH, PH, t, **kw)
            elif model == "parker":
                B_, V_ = bgm.parker_fields(R, TH, PH, **kw)
            else:
                raise ValueError(model)
            B_ = [torch.broadcast_to(b, (P, P, P)) for b in B_]
            V_ = [torch.broadcast_to(v, (P, P, P)) for v in V_]
            _pack_leaf(out[s, n], B_, V_, r, th, ph)
    return out


def from_uniform(spec, uniform):
    """Level-0 leaves (no refinement) carrying the cells of a uniform-grid array
    [n_snap, nph, nth, nr, REC] whose geometry equals the AMR base level."""
    leaves = build_leaves(spec, lambda *a: False)
    B = spec.bsize
    P = B + 2
    out = np.zeros((uniform.shape[0], len(leaves), P, P, P, REC), dtype=np.float32)
    for n, (lv, bi, bj, bk) in enumerate(leaves):
        out[:, n, 1:-1, 1:-1, 1:-1] = uniform[:, bk * B:(bk + 1) * B, bj * B:(bj + 1) * B,
                                              bi * B:(bi + 1) * B]
    return leaves, out


def divv_refiner(spec, threshold, model="cir", t=0.0, r_from=0.0, **kw):
    """refine(level, bi, bj, bk): |div V| of the analytic wind exceeds `threshold` (1/s) at
    some cell centre of the block (div V by central differences at the block's resolution)."""
    def refine(lv, bi, bj, bk):
        r, th, ph = _leaf_lattice(spec, (lv, bi, bj, bk))
        if r[-1] < r_from:
            return False
        R = torch.as_tensor(r, dtype=_F64)[None, None, :]
        TH = torch.as_tensor(th, dtype=_F64)[None, :, None]
        PH = torch.as_tensor(ph, dtype=_F64)[:, None, None]
        if model == "cir":
            _, V = bgm.cir_fields(R, TH, PH, t, **kw)
        else:
            _, V = bgm.parker_fields(R, TH, PH, **kw)
        P = spec.bsize + 2
        V = [torch.broadcast_to(v, (P, P, P)) for v in V]
        rec = np.zeros((P, P, P, REC), np.float32)
        Bz = [torch.zeros((P, P, P), dtype=_F64) + 1.0 for _ in range(3)]
        _pack_leaf(rec, Bz, V, r, th, ph)
        dv = rec[1:-1, 1:-1, 1:-1, 6] + rec[1:-1, 1:-1, 1:-1, 10] + rec[1:-1, 1:-1, 1:-1, 14]
        return bool(np.abs(dv).max() > threshold)
    return refine


def affine(spec, leaves, seed=0, phi_ref=math.pi):
    """Every field affine in (r, theta, phi - phi_ref) (phi unwrapped to [0, 2 pi)), per
    snapshot s plus a term linear in s; returns (fields, coef) like backgrounds.affine."""
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=(18, 5))
    B = spec.bsize
    P = B + 2
    out = np.zeros((spec.n_snap, len(leaves), P, P, P, REC), dtype=np.float32)
    for n, (lv, bi, bj, bk) in enumerate(leaves):
        idx = np.arange(B)
        r = centres_1d(spec, lv, 0, bi * B + idx)
        th = centres_1d(spec, lv, 1, bj * B + idx)
        ph = centres_1d(spec, lv, 2, bk * B + idx) - phi_ref
        for s in range(spec.n_snap):
            for f in range(18):
                c = coef[f]
                out[s, n, 1:-1, 1:-1, 1:-1, f] = (c[0] + c[1] * r[None, None, :] + c[2] * th[None, :, None]
                                                   + c[3] * ph[:, None, None] + c[4] * s)
    return out, coef
