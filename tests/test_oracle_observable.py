"""Pins of the oracle's smooth observable (the kernel-smoothed intensity whose
gradients fit transport parameters): J_i = sum over alive steps n of
w dt K(r_n, E_n, t_n), K a product of Gaussians in r, ln E and t, evaluated on
the start-of-step state.  Particles with known closed-form paths fix it."""
import math

import numpy as np
import pytest

from fte_inputs.configs import Params, SmoothObserver
from oracle import oracle as O


def _K(ob, r, E, t):
    return (np.exp(-0.5 * ((r - ob.r_o) / ob.sigma_r) ** 2) * np.exp(-0.5 * (np.log(E / ob.e_c) / ob.sigma_lnE) ** 2)
            * np.exp(-0.5 * ((t - ob.t_c) / ob.sigma_t) ** 2))


def test_resting_particle():
    """V = 0, uniform B, mu = 0, no scattering: the particle stays put; J is the time sum."""
    bg = O.analytic_background("uniform_b", [5.0])
    ob = SmoothObserver(r_o=1.0, sigma_r=0.05, e_c=0.1, sigma_lnE=0.3, t_c=3000.0, sigma_t=900.0)
    p = math.sqrt(0.12 / O.MC2 * (0.12 / O.MC2 + 2))
    P = O.make_particles(1, 1.03, 0.0, 0.0, 0.0, p)
    P["w"] = 0.7
    prm = Params(dmumu="iso", lambda_par=1e300, dt=10.0, t0=5.0)
    J = O.observe(bg, prm, P, 0, 600, ob)
    t = 5.0 + 10.0 * np.arange(600)
    E = O.MC2 * p * p / (math.sqrt(1 + p * p) + 1)
    expect = 0.7 * 10.0 * np.sum(_K(ob, 1.03, E, t))
    assert J[0] == pytest.approx(expect, rel=1e-12)
    assert P["x"][0] == 1.03 and P["status"][0] == 0


def test_streaming_particle_start_of_step_state():
    """mu = 1 along a uniform B = B z_hat: z_n = z_0 + n v dt; the tally uses the state before each step."""
    bg = O.analytic_background("uniform_b", [5.0])
    ob = SmoothObserver(r_o=1.0, sigma_r=0.02, e_c=0.05, sigma_lnE=0.2, t_c=0.0, sigma_t=1e9)
    e0 = 0.05
    p = math.sqrt(e0 / O.MC2 * (e0 / O.MC2 + 2))
    v = O.speed_of_p(p)
    P = O.make_particles(1, 0.0, 0.0, 0.9, 1.0, p)
    prm = Params(dmumu="iso", lambda_par=1e300, dt=5.0)
    n = 400
    J = O.observe(bg, prm, P, 0, n, ob)
    z = 0.9 + v * 5.0 * np.arange(n)
    expect = 5.0 * np.sum(_K(ob, z, e0, 5.0 * np.arange(n)))
    assert J[0] == pytest.approx(expect, rel=1e-10)
    assert P["z"][0] == pytest.approx(0.9 + v * 5.0 * n, rel=1e-12)


def test_absorbed_particle_stops_contributing():
    bg = O.analytic_background("uniform_b", [5.0], domain="sphere", dom=(0.1, 1.0, 0.0, math.pi))
    ob = SmoothObserver(r_o=0.95, sigma_r=0.1, e_c=0.05, sigma_lnE=0.2, t_c=0.0, sigma_t=1e9)
    e0 = 0.05
    p = math.sqrt(e0 / O.MC2 * (e0 / O.MC2 + 2))
    v = O.speed_of_p(p)
    P = O.make_particles(1, 0.0, 0.0, 0.9, 1.0, p)
    prm = Params(dmumu="iso", lambda_par=1e300, dt=5.0)
    J = O.observe(bg, prm, P, 0, 10_000, ob)
    steps = int(math.floor((1.0 - 0.9) / (v * 5.0))) + 1     # steps taken before leaving r <= 1
    z = 0.9 + v * 5.0 * np.arange(steps)
    assert P["status"][0] == 2
    assert J[0] == pytest.approx(5.0 * np.sum(_K(ob, z, e0, 0.0)), rel=1e-10)
