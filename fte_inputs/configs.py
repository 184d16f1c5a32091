"""Workload definitions: background, injection, transport parameters, observers.

Plain data only.  Field names follow the paper's notation (lambda_par for the
parallel mean free path, q and H of the quasi-linear pitch-angle coefficient,
eps of Eq. 5, lambda_perp for the cross-field mean free path).

Workloads (the three that run on one spherical grid; names say what they are):

* ``parker_1e4``      - static Parker wind on a 128x16x32 grid, 1e4 protons at
                         100 keV from (0.1 au, 90 deg, 0 deg), QLT D_mumu with
                         q = 5/3, H = 0.05, lambda_par = 0.3 au, dt = 10 s for
                         one day, tally on the 1 au shell.
* ``cir_uniform_1e6`` - synthetic CIR on a 512x60x180 grid with 24 hourly
                         periodic snapshots, 1e6 protons at 50 keV spread over
                         the div V < 0 region of one CIR between 1 and 2 au at
                         theta = 90 +- 2 deg with weight 1/r^2 (Eq. 7),
                         lambda_par = 0.1 au, dt = 10 s for four days.
* ``cir_amr_1e7``     - the same CIR on a log-r block-AMR grid (16^3-cell blocks,
                         base 32x8x24 blocks, 3 levels, refined where |div V|
                         exceeds 6e-5 /s: about 40k leaves), two hourly
                         snapshots, 1e7 protons with an E^-3 spectrum over
                         50 keV - 5 MeV, dt = 2 s for one simulated hour,
                         four observer boxes at 0.5, 1, 1.5 and 1.8 au.
* ``cir_ensemble_64`` - the cir_uniform_1e6 background and transport with 64
                         parameter sets (lambda_par log-uniform in 0.05-1 au,
                         H uniform in 0.01-0.2, injection energy log-uniform
                         in 20-200 keV, particle counts log-uniform in
                         1e4-1e6 rescaled to 2e7 in total), six simulated
                         hours, per-set tallies at the 1 au box.
"""
from dataclasses import dataclass, field, replace
import math
from typing import List, Optional

import numpy as np

from .grid import GridSpec
from .units import OMEGA_SUN, KMS

DEG = math.pi / 180.0


@dataclass
class InjectSpec:
    region: str = "point"            # 'point' | 'box'
    r: float = 0.1                   # point position (au, rad)
    th: float = 90 * DEG
    ph: float = 0.0
    r1: float = 1.0                  # box: volume-uniform in r^2 dr dcos(theta) dphi
    r2: float = 2.0
    th1: float = 88 * DEG
    th2: float = 92 * DEG
    ph1: float = 0.0
    ph2: float = 2 * math.pi
    divv_max: Optional[float] = None # accept only cells whose stored div V < divv_max
    divv_snap: int = 0               # snapshot whose cell values decide acceptance
    max_tries: int = 256
    energy: str = "mono"             # 'mono' | 'powerlaw'
    e0: float = 0.1                  # MeV
    e1: float = 0.05
    e2: float = 5.0
    gamma: float = 3.0               # dN/dE ~ E^-gamma
    weight: str = "unit"             # 'unit' | 'r-2'
    mu: str = "isotropic"            # 'isotropic' | 'fixed'
    mu0: float = 0.0
    seed: int = 0
    set_id: int = 0
    spiral: float = 0.0              # box: ph1..ph2 bound the spiral phase phi + spiral (r - spiral_rb)
    spiral_rb: float = 0.1           # au


@dataclass
class Params:
    dmumu: str = "qlt"               # 'qlt' | 'paper' | 'iso'
    lambda_par: float = 0.3          # au, at momentum p_ref
    p_ref: float = 0.0               # m_p c; 0 -> lambda_par independent of p
    alpha: float = 0.0               # lambda_par ~ (p / p_ref)^alpha
    q: float = 5.0 / 3.0
    H: float = 0.05
    eps: float = 0.048
    mu_floor: float = 1e-4
    lambda_perp: float = 0.0         # au; 0 switches cross-field diffusion off
    kappa_drift: int = 1
    dvdt_term: int = 1
    p_update: str = "exp"            # 'exp' | 'euler'
    dt: float = 10.0                 # s
    t0: float = 0.0                  # s, time of step 0
    seed: int = 0
    set_id: int = 0
    sort_every: int = 0              # steps between spatial reorderings (performance only)
    tally_layout: str = "global"     # 'global' (warp-merged FP64 atomics) | 'shared' (per-block histograms)


@dataclass
class Observer:
    kind: str = "shell"              # 'shell' | 'box' | 'slab' | 'ring' (longitude profile:
                                     # nt bins in phi over [0, 2 pi), time integrated)
    r: float = 1.0
    dr: float = 0.01
    th: float = 90 * DEG
    dth: float = 2 * DEG
    ph: float = 0.0
    dph: float = 2 * DEG
    e_lo: float = 0.01               # MeV
    e_hi: float = 1.0
    ne: int = 16
    t_lo: float = 0.0                # s
    t_hi: float = 86400.0
    nt: int = 144


@dataclass
class SmoothObserver:
    """Kernel-smoothed intensity for parameter gradients: every alive step adds
    w dt exp(-(r-r_o)^2/(2 sigma_r^2)) exp(-ln(E/e_c)^2/(2 sigma_lnE^2)) exp(-(t-t_c)^2/(2 sigma_t^2))."""
    r_o: float = 1.0                 # au
    sigma_r: float = 0.02            # au
    e_c: float = 0.1                 # MeV
    sigma_lnE: float = 0.1           # natural log
    t_c: float = 2 * 86400.0         # s
    sigma_t: float = 3600.0          # s
    lr_window: float = -1.0          # gradient estimator: score-form window around mu = 0 (< 0: default)


@dataclass
class Workload:
    name: str
    grid: GridSpec
    background: str                  # 'parker' | 'cir'
    inject: InjectSpec
    n_particles: int
    params: Params
    observers: List[Observer] = field(default_factory=list)
    n_steps: int = 0
    amr_divv: Optional[float] = None   # block-AMR grids: refinement threshold on |div V| (1/s)
    sets: Optional[list] = None        # ensembles: EnsembleSet per parameter set


CIR_PSI_C = 1.5 * math.pi            # spiral phase of the observed CIR's compression boundary


def cir_observer_phi(r_obs=1.0, psi_c=CIR_PSI_C, u_kms=500.0, r_b=0.1):
    """Longitude where the CIR whose compression boundary sits at spiral phase psi_c crosses r_obs."""
    return (psi_c - OMEGA_SUN * (r_obs - r_b) / (u_kms * KMS)) % (2 * math.pi)


def parker_1e4():
    g = GridSpec(nr=128, nth=16, nph=32, r_min=0.1, r_max=2.0, n_snap=1)
    inj = InjectSpec(region="point", r=0.1, th=90 * DEG, ph=0.0, energy="mono", e0=0.1,
                     weight="unit", seed=0)
    prm = Params(dmumu="qlt", lambda_par=0.3, q=5.0 / 3.0, H=0.05, dt=10.0, seed=0)
    obs = [Observer(kind="shell", r=1.0, dr=0.01, e_lo=0.01, e_hi=1.0, ne=16,
                    t_lo=0.0, t_hi=86400.0, nt=144)]
    return Workload("parker_1e4", g, "parker", inj, 10_000, prm, obs, n_steps=8640)


def cir_uniform_1e6():
    g = GridSpec(nr=512, nth=60, nph=180, r_min=0.1, r_max=2.0, n_snap=24, periodic=True,
                 t_snap0=0.0, dt_snap=3600.0)
    inj = InjectSpec(region="box", r1=1.0, r2=2.0, th1=88 * DEG, th2=92 * DEG,
                     ph1=math.pi, ph2=2 * math.pi, divv_max=0.0, divv_snap=0,
                     energy="mono", e0=0.05, weight="r-2", seed=0)
    prm = Params(dmumu="qlt", lambda_par=0.1, q=5.0 / 3.0, H=0.05, dt=10.0, seed=0, sort_every=64)
    four_days = 4 * 86400.0
    obs = [Observer(kind="box", r=1.0, dr=0.02, th=90 * DEG, dth=2 * DEG,
                    ph=cir_observer_phi(1.0), dph=2 * DEG, e_lo=0.01, e_hi=10.0, ne=16,
                    t_lo=0.0, t_hi=four_days, nt=144)]
    return Workload("cir_uniform_1e6", g, "cir", inj, 1_000_000, prm, obs, n_steps=34_560)


def cir_amr_1e7(n_particles=10_000_000, n_steps=1800, spec=None):
    from .amr import AmrSpec
    g = spec or AmrSpec(nbr=32, nbt=8, nbp=24, bsize=16, levels=3, radial="log", n_snap=2,
                        periodic=False, t_snap0=0.0, dt_snap=3600.0)
    # one CIR from 0.12 to 2 au (Sec. 2.3), selected by the spiral region criterion
    # phi_hat = phi + (r - r_B) Omega / U within +-10 deg of the CIR's compression boundary
    # (the observers sit on it): the synthetic wind compresses (div V < 0) only beyond
    # ~0.65 au, so the band stands in for the shock-traced div V < 0 region
    inj = InjectSpec(region="box", r1=0.12, r2=2.0, th1=88 * DEG, th2=92 * DEG,
                     ph1=CIR_PSI_C - 10 * DEG, ph2=CIR_PSI_C + 10 * DEG,
                     spiral=OMEGA_SUN / (500.0 * KMS), spiral_rb=0.1,
                     energy="powerlaw", e1=0.05, e2=5.0, gamma=3.0, weight="r-2", seed=0)
    prm = Params(dmumu="qlt", lambda_par=0.1, q=5.0 / 3.0, H=0.05, dt=2.0, seed=0, sort_every=64)
    t_end = n_steps * prm.dt
    obs = [Observer(kind="box", r=r, dr=0.02, th=90 * DEG, dth=2 * DEG, ph=cir_observer_phi(r),
                    dph=2 * DEG, e_lo=0.01, e_hi=10.0, ne=16, t_lo=0.0, t_hi=t_end, nt=144)
           for r in (0.5, 1.0, 1.5, 1.8)]
    return Workload("cir_amr_1e7", g, "cir", inj, n_particles, prm, obs, n_steps=n_steps, amr_divv=6e-5)


@dataclass
class EnsembleSet:
    """One parameter set of an ensemble: its transport parameters, Philox key,
    particle count and injection."""
    lambda_par: float
    q: float
    H: float
    eps: float
    seed: int
    set_id: int
    count: int
    inject: InjectSpec


def ensemble_sets(n_sets=64, total=20_000_000, lo=10_000, hi=1_000_000, base_inject=None,
                  q=5.0 / 3.0, eps=0.048, rng_seed=2024):
    """Seeded parameter sets: lambda_par log-uniform on [0.05, 1] au, H uniform on
    [0.01, 0.2], mono injection energy log-uniform on [20, 200] keV, counts
    log-uniform on [lo, hi] rescaled to add up to `total`; set s has Philox key
    (seed s, set_id s)."""
    rng = np.random.default_rng(rng_seed)
    lam = np.exp(rng.uniform(math.log(0.05), math.log(1.0), n_sets))
    H = rng.uniform(0.01, 0.2, n_sets)
    e0 = np.exp(rng.uniform(math.log(0.02), math.log(0.2), n_sets))
    raw = np.exp(rng.uniform(math.log(lo), math.log(hi), n_sets))
    counts = np.floor(raw * total / raw.sum()).astype(np.int64)
    counts[np.argmax(counts)] += total - counts.sum()
    base = base_inject or InjectSpec()
    return [EnsembleSet(float(lam[s]), q, float(H[s]), eps, s, s, int(counts[s]),
                        replace(base, energy="mono", e0=float(e0[s]), seed=s, set_id=s))
            for s in range(n_sets)]


def cir_ensemble_64(n_sets=64, total=20_000_000, n_steps=2160):
    w = cir_uniform_1e6()
    t_end = n_steps * w.params.dt
    obs = [replace(w.observers[0], t_hi=t_end)]
    sets = ensemble_sets(n_sets, total, base_inject=w.inject)
    return replace(w, name="cir_ensemble_64", n_particles=total, observers=obs, n_steps=n_steps, sets=sets)


def scaled(w: Workload, nr=None, nth=None, nph=None, n_particles=None, n_steps=None,
           n_snap=None):
    """A smaller copy of a workload (same physics, coarser grid / fewer particles or steps)."""
    g = replace(w.grid)
    if nr: g.nr = nr
    if nth: g.nth = nth
    if nph: g.nph = nph
    if n_snap: g.n_snap = n_snap
    return replace(w, grid=g,
                   n_particles=n_particles or w.n_particles,
                   n_steps=n_steps or w.n_steps)


def build_background(w: Workload):
    from . import backgrounds
    if w.background == "parker":
        return backgrounds.parker(w.grid)
    if w.background == "cir":
        return backgrounds.cir(w.grid)
    raise ValueError(w.background)
