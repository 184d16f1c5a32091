"""Synthetic solar-wind backgrounds sampled on a spherical grid.

The paper's backgrounds are Icarus / EUHFORIA MHD snapshots (Sec. 2.2-2.3); they
are not available, so these analytic winds stand in for them:

* ``parker``   - radial wind of constant speed with a Parker-spiral field,
                 static (one snapshot), inertial frame.
* ``cir``      - a corotating interaction region pattern in the frame corotating
                 with the Sun: a slow/fast stream structure set by a tanh profile
                 in the spiral phase psi = phi + Omega (r - r_B) / U (Eq. 6), with
                 forward and reverse shocks (tanh jumps of compression ratio s)
                 switched on beyond 1 au, B parallel to V so that E = 0 in the
                 corotating frame (Sec. 2.3, inner-boundary remark), and a weak
                 24-hour modulation of the fast-stream speed so that hourly
                 snapshots differ.
* ``affine``   - every field an affine function of (r, theta, phi, snapshot);
                 used to check that interpolation reproduces linear data exactly.

Gradients dV_i/dx_j and d|B|/dx_j are second-order finite differences along the
grid lines (one-sided second order at the r and theta faces, periodic in phi),
mapped to Cartesian derivatives with dr/dx = r_hat, dtheta/dx = theta_hat / r,
dphi/dx = phi_hat / (r sin theta).  This mirrors what a post-processor of
finite-volume MHD output provides; the stored gradients are data.

Evaluation uses float64 CPU torch tensors (multi-threaded elementwise work); the
result is a float32 numpy array [n_snap, nph, nth, nr, REC].
"""
import math
import numpy as np
import torch

from .grid import GridSpec, REC, cell_centres
from .units import OMEGA_SUN, KMS

_F64 = torch.float64


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


def _axes(g: GridSpec):
    r, th, ph = cell_centres(g)
    return _t(r), _t(th), _t(ph)


def _basis(TH, PH):
    st, ct = torch.sin(TH), torch.cos(TH)
    sp, cp = torch.sin(PH), torch.cos(PH)
    zero = torch.zeros((), dtype=_F64)
    rhat = (st * cp, st * sp, ct + zero * cp)
    that = (ct * cp, ct * sp, -st + zero * cp)
    phat = (-sp + zero * st, cp + zero * st, zero * st * sp)
    return rhat, that, phat


def _sph_to_cart(vr, vt, vp, basis):
    rhat, that, phat = basis
    return [vr * rhat[i] + vt * that[i] + vp * phat[i] for i in range(3)]


def _d_axis(f, x, axis):
    """Second-order derivative of f along `axis` with (possibly non-uniform) coordinates x."""
    n = x.shape[0]
    f = f.movedim(axis, -1)
    out = torch.empty_like(f)
    if n < 3:
        d = (f[..., 1] - f[..., 0]) / (x[1] - x[0])
        out[..., 0] = d
        out[..., 1] = d
        return out.movedim(-1, axis)
    h1 = x[1:-1] - x[:-2]
    h2 = x[2:] - x[1:-1]
    out[..., 1:-1] = (-h2 / (h1 * (h1 + h2)) * f[..., :-2]
                      + (h2 - h1) / (h1 * h2) * f[..., 1:-1]
                      + h1 / (h2 * (h1 + h2)) * f[..., 2:])
    a, b = x[1] - x[0], x[2] - x[1]
    out[..., 0] = (-(2 * a + b) / (a * (a + b)) * f[..., 0] + (a + b) / (a * b) * f[..., 1]
                   - a / (b * (a + b)) * f[..., 2])
    a, b = x[-2] - x[-3], x[-1] - x[-2]
    out[..., -1] = (b / (a * (a + b)) * f[..., -3] - (a + b) / (a * b) * f[..., -2]
                    + (a + 2 * b) / (b * (a + b)) * f[..., -1])
    return out.movedim(-1, axis)


def _grad_cart(f, r, th, ph, basis, R, ST):
    """Cartesian gradient of a cell-centred scalar f[phi, theta, r]."""
    dfr = _d_axis(f, r, 2)
    dft = _d_axis(f, th, 1)
    dph = float(ph[1] - ph[0]) if ph.shape[0] > 1 else 2 * math.pi
    dfp = (torch.roll(f, -1, 0) - torch.roll(f, 1, 0)) / (2.0 * dph)
    rhat, that, phat = basis
    return [dfr * rhat[j] + dft * that[j] / R + dfp * phat[j] / (R * ST) for j in range(3)]


def _pack(out, s, B, V, r, th, ph):
    """Fill snapshot s of out[s, phi, theta, r, REC] from Cartesian B, V (full 3-D tensors)."""
    PH = ph[:, None, None]
    TH = th[None, :, None]
    R = r[None, None, :]
    basis = _basis(TH, PH)
    ST = torch.sin(TH)
    rec = torch.from_numpy(out[s])
    for i in range(3):
        rec[..., i] = B[i]
        rec[..., 3 + i] = V[i]
    for i in range(3):
        gr = _grad_cart(V[i], r, th, ph, basis, R, ST)
        for j in range(3):
            rec[..., 6 + 3 * i + j] = gr[j]
    Bm = torch.sqrt(B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    gr = _grad_cart(Bm, r, th, ph, basis, R, ST)
    for j in range(3):
        rec[..., 15 + j] = gr[j]
    rec[..., 18:] = 0.0


def _alloc(g: GridSpec):
    return np.zeros((g.n_snap, g.nph, g.nth, g.nr, REC), dtype=np.float32)


def _full(a, shape):
    return torch.broadcast_to(a, shape).contiguous()


# ----------------------------------------------------------------------------
# Parker spiral
# ----------------------------------------------------------------------------
def parker_B_r1(v_kms=400.0, b1_nt=5.0):
    """Radial field at 1 au such that |B|(1 au, 90 deg) = b1_nt."""
    v = v_kms * KMS
    return b1_nt / math.sqrt(1.0 + (OMEGA_SUN * 1.0 / v) ** 2)


def parker_fields(R, TH, PH, v_kms=400.0, b1_nt=5.0):
    """Analytic Parker wind: V = v r_hat, B_r = B_r1 / r^2, B_phi = -B_r Omega r sin(theta) / v.

    Arguments are broadcastable float64 tensors; returns Cartesian (B, V) lists."""
    v = v_kms * KMS
    br1 = parker_B_r1(v_kms, b1_nt)
    R, TH, PH = torch.broadcast_tensors(R, TH, PH)
    basis = _basis(TH, PH)
    br = br1 / R ** 2
    bp = -br * OMEGA_SUN * R * torch.sin(TH) / v
    B = _sph_to_cart(br, 0.0 * br, bp, basis)
    V = _sph_to_cart(v + 0.0 * R, 0.0 * R, 0.0 * R, basis)
    return B, V


def parker(g: GridSpec, v_kms=400.0, b1_nt=5.0):
    r, th, ph = _axes(g)
    shape = (g.nph, g.nth, g.nr)
    out = _alloc(g)
    B, V = parker_fields(r[None, None, :], th[None, :, None], ph[:, None, None], v_kms, b1_nt)
    B = [_full(b, shape) for b in B]
    V = [_full(v, shape) for v in V]
    for s in range(g.n_snap):
        _pack(out, s, B, V, r, th, ph)
    return out


# ----------------------------------------------------------------------------
# Corotating interaction region
# ----------------------------------------------------------------------------
CIR_DEFAULTS = dict(
    v_slow=330.0, v_fast=700.0,       # km/s
    u_spiral=500.0,                   # km/s, U of Eq. 6
    r_b=0.1,                          # au, inner boundary
    slow=((0.5 * math.pi, math.pi), (1.5 * math.pi, 2.0 * math.pi)),  # slow-stream psi intervals
    w_psi=0.1,                        # rad, stream-edge width at the source
    s=2.5,                            # shock compression ratio
    w_shock=0.01,                     # au, shock width
    w_iface=0.03,                     # au, stream-interface width
    r_on=1.0, w_on=0.05,              # au, shocks switched on beyond r_on
    h0=0.02, h1=0.08,                 # au, half-separation of the shocks h = h0 + h1 (r - r_on)
    br_b=350.0,                       # nT, B_r at r_b
    mod_amp=0.05, mod_period=86400.0, # fast-stream modulation
)


def _T(u):
    return 0.5 * (1.0 + torch.tanh(u))


def _wrap(a):
    return torch.remainder(a + math.pi, 2.0 * math.pi) - math.pi


def cir_fields(R, TH, PH, t, **kw):
    """Analytic CIR wind (corotating frame) at broadcastable float64 tensors (R, TH, PH), time t."""
    p = dict(CIR_DEFAULTS)
    p.update(kw)
    vs = p["v_slow"] * KMS
    vf = p["v_fast"] * KMS * (1.0 + p["mod_amp"] * math.sin(2.0 * math.pi * t / p["mod_period"]))
    U = p["u_spiral"] * KMS
    s = p["s"]
    R, TH, PH = torch.broadcast_tensors(R, TH, PH)
    ST = torch.sin(TH)
    psi = PH + OMEGA_SUN * (R - p["r_b"]) / U
    # smooth stream structure: slow inside the listed psi intervals
    S = torch.zeros_like(psi)
    for a, b in p["slow"]:
        S += _T(_wrap(psi - a) / p["w_psi"]) * (1.0 - _T(_wrap(psi - b) / p["w_psi"]))
    vr = vf - (vf - vs) * S
    comp = torch.ones_like(psi)
    on = _T((R - p["r_on"]) / p["w_on"])
    h = p["h0"] + p["h1"] * torch.clamp(R - p["r_on"], min=0.0)
    v_r2 = U + (vf - U) / s       # downstream of the reverse shock
    v_f2 = U + (vs - U) / s       # downstream of the forward shock
    norm = 1.0 / torch.sqrt(1.0 + (OMEGA_SUN * R * ST / U) ** 2)
    ws, wi = p["w_shock"], p["w_iface"]
    for a, _b in p["slow"]:       # compression boundary = start of each slow interval
        dpsi = _wrap(psi - a)
        x = R * ST * dpsi * norm  # distance normal to the spiral
        up = _T((x + h) / ws)
        dn = _T((x - h) / ws)
        shocked = vf + (v_r2 - vf) * up + (v_f2 - v_r2) * _T(x / wi) + (vs - v_f2) * dn
        step = vf + (vs - vf) * _T(dpsi / p["w_psi"])
        vr = vr + on * (shocked - step)
        comp = comp + on * (s - 1.0) * (up - dn)
    vphi = -OMEGA_SUN * R * ST
    basis = _basis(TH, PH)
    V = _sph_to_cart(vr, 0.0 * vr, vphi, basis)
    br = p["br_b"] * (p["r_b"] / R) ** 2 * comp
    B = _sph_to_cart(br, 0.0 * br, br * vphi / vr, basis)
    return B, V


def cir(g: GridSpec, **kw):
    r, th, ph = _axes(g)
    out = _alloc(g)
    for s in range(g.n_snap):
        t = g.t_snap0 + s * g.dt_snap
        B, V = cir_fields(r[None, None, :], th[None, :, None], ph[:, None, None], t, **kw)
        _pack(out, s, B, V, r, th, ph)
    return out


# ----------------------------------------------------------------------------
# Affine test data
# ----------------------------------------------------------------------------
def affine(g: GridSpec, seed=0):
    """Every stored value (18 fields, every snapshot) affine in (r, theta, phi, snap).

    Returns (data, coef) with data[s, k, j, i, f] = c0 + cr r_i + ct theta_j + cp phi_k + cs s.
    """
    rng = np.random.default_rng(seed)
    coef = rng.normal(size=(18, 5))
    r, th, ph = cell_centres(g)
    out = _alloc(g)
    for s in range(g.n_snap):
        for f in range(18):
            c = coef[f]
            out[s, ..., f] = (c[0] + c[1] * r[None, None, :] + c[2] * th[None, :, None]
                              + c[3] * ph[:, None, None] + c[4] * s)
    return out, coef
