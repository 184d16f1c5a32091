"""Pins of the oracle's background access (Sec. 2.4) and of the synthetic backgrounds.

Sec. 2.4: the particle is located on the grid, the values of the surrounding grid
points are read and interpolated trilinearly at every step.  Reading: cell-centred
data (finite-volume output), weights in the physical coordinates (r, theta, phi),
values held constant beyond the outermost cell centres in r and theta, phi
periodic, snapshots interpolated linearly in time.  Trilinear interpolation
reproduces any field affine in (r, theta, phi) exactly, which pins the cell
index, the weights and the corner order.
"""
import math

import numpy as np
import pytest

from fte_inputs import backgrounds, configs
from fte_inputs.grid import GridSpec, REC, cell_centres
from fte_inputs.units import OMEGA_SUN, KMS
from oracle import oracle as O


def _cart(r, th, ph):
    return (r * math.sin(th) * math.cos(ph), r * math.sin(th) * math.sin(ph), r * math.cos(th))


def _affine_value(coef, r, th, ph, s):
    return coef[:, 0] + coef[:, 1] * r + coef[:, 2] * th + coef[:, 3] * ph + coef[:, 4] * s


def _field_vector(out):
    return np.concatenate([out["B"], out["V"], out["G"].ravel(), out["gB"]])


@pytest.mark.parametrize("radial", ["linear", "log"])
def test_affine_data_reproduced(radial):
    g = GridSpec(nr=12, nth=7, nph=9, r_min=0.2, r_max=1.7, radial=radial, n_snap=1)
    data, coef = backgrounds.affine(g, seed=1)
    bg = O.grid_background(g, data)
    r_c, th_c, ph_c = cell_centres(g)
    rng = np.random.default_rng(5)
    scale = np.abs(data).max()
    for _ in range(200):
        r = rng.uniform(r_c[0], r_c[-1])
        th = rng.uniform(th_c[0], th_c[-1])
        ph = rng.uniform(ph_c[0], ph_c[-1])
        got = _field_vector(O.eval_fields(bg, *_cart(r, th, ph), 0.0))
        assert np.abs(got - _affine_value(coef, r, th, ph, 0)).max() < 2e-6 * scale


def test_clamped_beyond_outer_centres_and_phi_seam():
    g = GridSpec(nr=10, nth=6, nph=8, r_min=0.2, r_max=1.2, n_snap=1)
    data, coef = backgrounds.affine(g, seed=2)
    bg = O.grid_background(g, data)
    r_c, th_c, ph_c = cell_centres(g)
    scale = np.abs(data).max()
    th, ph = 0.5 * (th_c[1] + th_c[2]), ph_c[3] + 0.1
    # inside the first half-cell in r the value equals the value at the first centre
    a = _field_vector(O.eval_fields(bg, *_cart(0.5 * (g.r_min + r_c[0]), th, ph), 0.0))
    b = _field_vector(O.eval_fields(bg, *_cart(r_c[0], th, ph), 0.0))
    assert np.abs(a - b).max() < 1e-6 * scale
    # same at the theta faces
    a = _field_vector(O.eval_fields(bg, *_cart(0.7, g.th_max - 1e-4, ph), 0.0))
    b = _field_vector(O.eval_fields(bg, *_cart(0.7, th_c[-1], ph), 0.0))
    assert np.abs(a - b).max() < 1e-6 * scale
    # across phi = 0 the interpolant is continuous and is the mean of the last and first cells
    r, th = 0.63, th_c[2]
    lo = _field_vector(O.eval_fields(bg, *_cart(r, th, -1e-9), 0.0))
    hi = _field_vector(O.eval_fields(bg, *_cart(r, th, 1e-9), 0.0))
    assert np.abs(lo - hi).max() < 1e-6 * scale
    mid = 0.5 * (_affine_value(coef, r, th, ph_c[0], 0) + _affine_value(coef, r, th, ph_c[-1], 0))
    assert np.abs(hi - mid).max() < 2e-6 * scale


def test_time_interpolation_and_dvdt():
    g = GridSpec(nr=8, nth=6, nph=8, r_min=0.2, r_max=1.2, n_snap=4, periodic=False,
                 t_snap0=100.0, dt_snap=50.0)
    data, coef = backgrounds.affine(g, seed=3)
    bg = O.grid_background(g, data)
    r_c, th_c, ph_c = cell_centres(g)
    r, th, ph = 0.71, th_c[2] + 0.05, ph_c[4] + 0.02
    scale = np.abs(data).max()
    for t in (100.0, 117.5, 150.0, 233.0):
        s = (t - 100.0) / 50.0
        out = O.eval_fields(bg, *_cart(r, th, ph), t)
        assert np.abs(_field_vector(out) - _affine_value(coef, r, th, ph, s)).max() < 2e-6 * scale
        assert out["dVdt"] == pytest.approx(coef[3:6, 4] / 50.0, rel=1e-5)
    # before the first and after the last snapshot: frozen, no time derivative
    out = O.eval_fields(bg, *_cart(r, th, ph), 50.0)
    assert np.abs(_field_vector(out) - _affine_value(coef, r, th, ph, 0)).max() < 2e-6 * scale
    assert np.all(out["dVdt"] == 0)
    for t in (250.0, 400.0):
        out = O.eval_fields(bg, *_cart(r, th, ph), t)
        assert np.abs(_field_vector(out) - _affine_value(coef, r, th, ph, 3)).max() < 2e-6 * scale
        assert np.all(out["dVdt"] == 0)
    # periodic sequence: between the last and the first snapshot
    g.periodic = True
    bg = O.grid_background(g, data)
    out = O.eval_fields(bg, *_cart(r, th, ph), 100.0 + 3.5 * 50.0)
    expect = 0.5 * (_affine_value(coef, r, th, ph, 3) + _affine_value(coef, r, th, ph, 0))
    assert np.abs(_field_vector(out) - expect).max() < 2e-6 * scale
    assert out["dVdt"] == pytest.approx(-3 * coef[3:6, 4] / 50.0, rel=1e-5)


def test_interpolant_gradient_of_B():
    """dB_i/dx_j of the trilinear interpolant of affine data: c_r r_hat + c_th theta_hat / r
    + c_ph phi_hat / (r sin theta)."""
    g = GridSpec(nr=12, nth=7, nph=9, r_min=0.2, r_max=1.7, n_snap=1)
    data, coef = backgrounds.affine(g, seed=4)
    bg = O.grid_background(g, data)
    r_c, th_c, ph_c = cell_centres(g)
    r, th, ph = 0.93, th_c[3] + 0.03, ph_c[5] + 0.1
    out = O.eval_fields(bg, *_cart(r, th, ph), 0.0)
    rh = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    thh = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    phh = np.array([-math.sin(ph), math.cos(ph), 0.0])
    for i in range(3):
        expect = coef[i, 1] * rh + coef[i, 2] * thh / r + coef[i, 3] * phh / (r * math.sin(th))
        assert out["dB"][i] == pytest.approx(expect, rel=2e-5, abs=1e-5)


# -------------------------------------------------------------------------------------------
# the synthetic backgrounds (inputs): finite-difference gradients are second order
# -------------------------------------------------------------------------------------------
def _parker_grad_error(n):
    g = GridSpec(nr=8 * n, nth=4 * n, nph=8 * n, r_min=0.5, r_max=1.5, th_min=math.radians(60),
                 th_max=math.radians(120), n_snap=1)
    f = backgrounds.parker(g)
    r_c, th_c, ph_c = cell_centres(g)
    i, j, k = 4 * n, 2 * n, 3 * n       # an interior cell
    r, th, ph = r_c[i], th_c[j], ph_c[k]
    rec = f[0, k, j, i].astype(np.float64)
    V0 = 400 * KMS
    rh = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    G = V0 * (np.eye(3) - np.outer(rh, rh)) / r
    errV = np.abs(rec[6:15].reshape(3, 3) - G).max() / np.abs(G).max()

    def bmag(x):
        import torch
        rr = math.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
        tt = math.atan2(math.hypot(x[0], x[1]), x[2])
        pp = math.atan2(x[1], x[0])
        B, _ = backgrounds.parker_fields(torch.tensor(rr, dtype=torch.float64),
                                         torch.tensor(tt, dtype=torch.float64),
                                         torch.tensor(pp, dtype=torch.float64))
        return math.sqrt(sum(float(b) ** 2 for b in B))
    x0 = np.array(_cart(r, th, ph))
    h = 1e-6
    gB = np.array([(bmag(x0 + h * e) - bmag(x0 - h * e)) / (2 * h) for e in np.eye(3)])
    errB = np.abs(rec[15:18] - gB).max() / np.abs(gB).max()
    return errV, errB


def test_parker_gradients_second_order():
    e1 = _parker_grad_error(1)
    e2 = _parker_grad_error(2)
    for a, b in zip(e1, e2):
        assert b < 0.02
        assert a / b > 3.0          # halving the spacing cuts the error ~4x


def test_cir_background_structure():
    g = GridSpec(nr=96, nth=12, nph=72, n_snap=2, periodic=True, dt_snap=3600.0)
    f = backgrounds.cir(g)
    B, V = f[..., 0:3].astype(np.float64), f[..., 3:6].astype(np.float64)
    # B parallel to V (E = 0 in the corotating frame)
    cross = np.linalg.norm(np.cross(B, V), axis=-1)
    assert np.all(cross <= 1e-5 * np.linalg.norm(B, axis=-1) * np.linalg.norm(V, axis=-1))
    # azimuthal velocity of the corotating frame
    r_c, th_c, ph_c = cell_centres(g)
    phh = np.stack([-np.sin(ph_c), np.cos(ph_c), 0 * ph_c], -1)[:, None, None, :]
    vphi = (V[0] * phh).sum(-1)
    expect = -OMEGA_SUN * r_c[None, None, :] * np.sin(th_c)[None, :, None]
    assert np.allclose(vphi, expect, rtol=1e-5, atol=1e-12)
    # compression (div V < 0) exists beyond 1 au and the two snapshots differ
    dv = f[0, ..., 6] + f[0, ..., 10] + f[0, ..., 14]
    assert (dv[..., r_c > 1.1] < 0).mean() > 0.02
    assert np.abs(f[0] - f[1]).max() > 0
    # speeds within the slow/fast range plus the corotation speed
    vr = (V[0] * np.stack([np.sin(th_c)[None, :, None] * np.cos(ph_c)[:, None, None],
                           np.sin(th_c)[None, :, None] * np.sin(ph_c)[:, None, None],
                           np.cos(th_c)[None, :, None] + 0 * ph_c[:, None, None]], -1)).sum(-1)
    assert vr.min() > 300 * KMS and vr.max() < 760 * KMS
