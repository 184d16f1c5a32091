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
        if getattr(refine, "batched", False):      # refine(blocks) -> bool per block
            cand = [leaf for leaf in leaves if leaf[0] == lv]
            hit = set(map(tuple, np.asarray(cand)[refine(cand)].tolist())) if cand else set()
        else:
            hit = {leaf for leaf in leaves if leaf[0] == lv and refine(*leaf)}
        nxt = []
        for leaf in leaves:
            if tuple(leaf) in hit:
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


def fields_batched(spec, leaves, model="cir", device="cpu", batch=1024, snaps=None, out=None, t=None, **kw):
    """Same values as `fields`, evaluated for many leaves at once (torch, on `device`).
    Returns (or fills `out`) a float32 tensor [n_snap, n_leaf, B+2, B+2, B+2, REC] on
    `device`; ghost cells are left as they are.  `t` overrides the snapshot times."""
    B = spec.bsize
    P = B + 2
    snaps = range(spec.n_snap) if snaps is None else snaps
    if out is None:
        out = torch.zeros((len(snaps), len(leaves), P, P, P, REC), dtype=torch.float32, device=device)
    lv_all = np.asarray(leaves)
    idx = np.arange(-1, B + 1)
    for si, s in enumerate(snaps):
        ts = spec.t_snap0 + s * spec.dt_snap if t is None else t
        for a in range(0, len(lv_all), batch):
            chunk = lv_all[a:a + batch]
            n = len(chunk)
            r = np.stack([centres_1d(spec, int(l[0]), 0, int(l[1]) * B + idx) for l in chunk])
            th = np.stack([centres_1d(spec, int(l[0]), 1, int(l[2]) * B + idx) for l in chunk])
            ph = np.stack([centres_1d(spec, int(l[0]), 2, int(l[3]) * B + idx) for l in chunk])
            Rt = torch.as_tensor(r, dtype=_F64, device=device)          # [n, P]
            Tt = torch.as_tensor(th, dtype=_F64, device=device)
            Pt = torch.as_tensor(ph, dtype=_F64, device=device)
            R = Rt[:, None, None, :]
            TH = Tt[:, None, :, None]
            PH = Pt[:, :, None, None]
            if model == "cir":
                B_, V_ = bgm.cir_fields(R, TH, PH, ts, **kw)
            else:
                B_, V_ = bgm.parker_fields(R, TH, PH, **kw)
            shape = (n, P, P, P)
            B_ = [torch.broadcast_to(b, shape) for b in B_]
            V_ = [torch.broadcast_to(v, shape) for v in V_]
            basis = bgm._basis(TH, PH)
            rhat, that, phat = [[torch.broadcast_to(c, shape)[:, 1:-1, 1:-1, 1:-1] for c in v] for v in basis]
            Ri = R[:, :, :, 1:-1]
            Si = torch.sin(TH)[:, :, 1:-1, :]
            h1 = (Rt[:, 1:-1] - Rt[:, :-2])[:, None, None, :]
            h2 = (Rt[:, 2:] - Rt[:, 1:-1])[:, None, None, :]
            dth = (Tt[:, 1] - Tt[:, 0])[:, None, None, None]
            dph = (Pt[:, 1] - Pt[:, 0])[:, None, None, None]

            def grad(f):
                fr = (-h2 / (h1 * (h1 + h2)) * f[:, 1:-1, 1:-1, :-2] + (h2 - h1) / (h1 * h2) * f[:, 1:-1, 1:-1, 1:-1]
                      + h1 / (h2 * (h1 + h2)) * f[:, 1:-1, 1:-1, 2:])
                ft = (f[:, 1:-1, 2:, 1:-1] - f[:, 1:-1, :-2, 1:-1]) / (2 * dth)
                fp = (f[:, 2:, 1:-1, 1:-1] - f[:, :-2, 1:-1, 1:-1]) / (2 * dph)
                return [fr * rhat[j] + ft * that[j] / Ri + fp * phat[j] / (Ri * Si) for j in range(3)]

            o = out[si, a:a + n]
            inner = (slice(None),) + (slice(1, -1),) * 3
            for i in range(3):
                o[inner + (i,)] = B_[i][inner].float()
                o[inner + (3 + i,)] = V_[i][inner].float()
                gi = grad(V_[i])
                for j in range(3):
                    o[inner + (6 + 3 * i + j,)] = gi[j].float()
            Bm = torch.sqrt(B_[0] ** 2 + B_[1] ** 2 + B_[2] ** 2)
            gB = grad(Bm)
            for j in range(3):
                o[inner + (15 + j,)] = gB[j].float()
    return out


def divv_marks(spec, blocks, threshold, model="cir", t=0.0, r_from=0.0, device="cpu", batch=512, **kw):
    """Batched form of `divv_refiner`: one bool per block (level, bi, bj, bk)."""
    blocks = np.asarray(blocks, dtype=np.int64).reshape(-1, 4)
    marks = np.zeros(len(blocks), dtype=bool)
    one = AmrSpec(**{**spec.__dict__, "n_snap": 1})
    for a in range(0, len(blocks), batch):
        chunk = blocks[a:a + batch]
        f = fields_batched(one, chunk, model=model, device=device, batch=batch, t=t, **kw)[0]
        inner = f[:, 1:-1, 1:-1, 1:-1]
        dv = (inner[..., 6] + inner[..., 10]) + inner[..., 14]
        m = (dv.abs().reshape(len(chunk), -1).amax(dim=1) > threshold).cpu().numpy()
        for n, (lv, bi, bj, bk) in enumerate(chunk):
            r_last = centres_1d(spec, int(lv), 0, np.array([(int(bi) + 1) * spec.bsize]))[0]
            if r_last < r_from:
                m[n] = False
        marks[a:a + len(chunk)] = m
    return marks


def divv_refiner_batched(spec, threshold, model="cir", t=0.0, r_from=0.0, device="cpu", **kw):
    """`divv_refiner` for `build_leaves` that tests many blocks at once."""
    def refine(blocks):
        return divv_marks(spec, blocks, threshold, model=model, t=t, r_from=r_from, device=device, **kw)
    refine.batched = True
    return refine
