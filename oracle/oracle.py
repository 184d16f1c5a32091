"""ctypes binding of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs import this module.  It loads oracle/libfte_oracle.so (built by
oracle/build.py) and converts the plain-data inputs of fte_inputs into the
oracle's structs.  It never imports the CUDA package.
"""
import ctypes as C
import math
import os

import numpy as np

from . import build as _build

OR_BG = dict(grid=0, uniform_b=1, hubble=2, monopole=3, radial_wind=4, planar_shock=5)
OR_DOM = dict(sphere=0, slab_x=1, none=2)
OR_DMUMU = dict(qlt=0, paper=1, iso=2)
ALIVE, ABS_INNER, ABS_OUTER, ABS_THETA, NAN, INJ_FAIL = range(6)


class Background(C.Structure):
    _fields_ = [("kind", C.c_int32), ("domain", C.c_int32), ("a", C.c_double * 8),
                ("dom", C.c_double * 4),
                ("nr", C.c_int32), ("nth", C.c_int32), ("nph", C.c_int32), ("radial", C.c_int32),
                ("n_snap", C.c_int32), ("periodic", C.c_int32), ("rec", C.c_int32),
                ("pad", C.c_int32),
                ("r_min", C.c_double), ("r_max", C.c_double), ("th_min", C.c_double),
                ("th_max", C.c_double), ("t_snap0", C.c_double), ("dt_snap", C.c_double),
                ("fields", C.c_void_p),
                ("amr_levels", C.c_int32), ("amr_bsize", C.c_int32), ("n_leaves", C.c_int32),
                ("pad2", C.c_int32), ("leaves", C.c_void_p), ("table", C.c_void_p)]


class ParamsC(C.Structure):
    _fields_ = [("dmumu", C.c_int32), ("p_update", C.c_int32), ("kappa_drift", C.c_int32),
                ("dvdt_term", C.c_int32),
                ("lambda_par", C.c_double), ("p_ref", C.c_double), ("alpha", C.c_double),
                ("q", C.c_double), ("H", C.c_double), ("eps", C.c_double),
                ("mu_floor", C.c_double), ("lambda_perp", C.c_double),
                ("dt", C.c_double), ("t0", C.c_double),
                ("seed", C.c_uint32), ("set_id", C.c_uint32), ("shock_divv", C.c_double)]


class InjectC(C.Structure):
    _fields_ = [("region", C.c_int32), ("energy", C.c_int32), ("weight", C.c_int32),
                ("mu_mode", C.c_int32),
                ("r", C.c_double), ("th", C.c_double), ("ph", C.c_double),
                ("r1", C.c_double), ("r2", C.c_double), ("th1", C.c_double),
                ("th2", C.c_double), ("ph1", C.c_double), ("ph2", C.c_double),
                ("use_divv", C.c_int32), ("divv_snap", C.c_int32), ("max_tries", C.c_int32),
                ("pad", C.c_int32), ("divv_max", C.c_double),
                ("e0", C.c_double), ("e1", C.c_double), ("e2", C.c_double),
                ("gamma", C.c_double), ("mu0", C.c_double),
                ("seed", C.c_uint32), ("set_id", C.c_uint32),
                ("spiral", C.c_double), ("spiral_rb", C.c_double)]


class ObserverC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ne", C.c_int32), ("nt", C.c_int32), ("pad", C.c_int32),
                ("r", C.c_double), ("dr", C.c_double), ("th", C.c_double), ("dth", C.c_double),
                ("ph", C.c_double), ("dph", C.c_double), ("e_lo", C.c_double),
                ("e_hi", C.c_double), ("t_lo", C.c_double), ("t_hi", C.c_double)]


PARTICLE = np.dtype([("x", "f8"), ("y", "f8"), ("z", "f8"), ("mu", "f8"), ("p", "f8"),
                     ("w", "f8"), ("n_div", "i8"), ("id", "u4"), ("status", "i4"),
                     ("flags", "i4"), ("n_sens", "i4"), ("amp_log", "f8")])
assert PARTICLE.itemsize == 80

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.or_uniforms.argtypes = [C.c_uint32] * 5 + [P(C.c_double)]
        L.or_normals.argtypes = [C.c_uint32] * 4 + [P(C.c_double)]
        L.or_norm_integral.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        L.or_norm_integral.restype = C.c_double
        L.or_dmumu.argtypes = [P(ParamsC), C.c_double, C.c_double, C.c_double, P(C.c_double)]
        L.or_eval_fields.argtypes = [P(Background), C.c_double, C.c_double, C.c_double,
                                     C.c_double, P(C.c_double)]
        L.or_inject.argtypes = [P(Background), P(InjectC), C.c_void_p, C.c_int64, C.c_void_p,
                                P(C.c_double), P(C.c_uint64)]
        L.or_advance.argtypes = [P(Background), P(ParamsC), P(ObserverC), C.c_int, C.c_void_p,
                                 C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, P(C.c_double), P(C.c_uint64),
                                 C.c_int]
        L.or_step_terms.argtypes = [P(Background), P(ParamsC), C.c_void_p, C.c_int64,
                                    P(C.c_double)]
        L.or_intensity.argtypes = [P(ObserverC), C.c_void_p, C.c_void_p]
        L.or_observe.argtypes = [P(Background), P(ParamsC), P(SmoothObsC), C.c_void_p, C.c_int64,
                                 C.c_int64, C.c_int64, C.c_void_p, C.c_int]
        L.or_mu_logpdf.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_mu_logpdf.restype = C.c_double
        L.or_observe_lr.argtypes = [P(Background), P(ParamsC), P(SmoothObsC), C.c_double, C.c_void_p,
                                    C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_double, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_int]
        L.or_max_threads.restype = C.c_int
        L.or_amr_cell.argtypes = [P(Background), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                  P(C.c_double)]
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# conversions from fte_inputs plain data
# --------------------------------------------------------------------------
class Bg:
    """An oracle background plus the arrays it points to (kept alive here)."""

    def __init__(self, c, keep=None):
        self.c = c
        self.keep = keep


def grid_background(grid, fields):
    """Background from a GridSpec and its float32 [n_snap, nph, nth, nr, REC] array."""
    f = np.ascontiguousarray(fields, dtype=np.float32)
    assert f.shape[:4] == (grid.n_snap, grid.nph, grid.nth, grid.nr)
    c = Background()
    c.kind = OR_BG["grid"]
    c.domain = OR_DOM["sphere"]
    c.dom[:] = [grid.r_min, grid.r_max, grid.th_min, grid.th_max]
    c.nr, c.nth, c.nph = grid.nr, grid.nth, grid.nph
    c.radial = 1 if grid.radial == "log" else 0
    c.n_snap, c.periodic, c.rec = grid.n_snap, int(grid.periodic), f.shape[4]
    c.r_min, c.r_max, c.th_min, c.th_max = grid.r_min, grid.r_max, grid.th_min, grid.th_max
    c.t_snap0, c.dt_snap = grid.t_snap0, grid.dt_snap
    c.fields = f.ctypes.data
    return Bg(c, f)


def amr_background(spec, leaves, fields):
    """Background from an fte_inputs.amr.AmrSpec, its Morton-sorted leaves and padded fields
    [n_snap, n_leaf, B+2, B+2, B+2, REC] (ghost layer ignored)."""
    from fte_inputs import amr as amr_mod
    f = np.ascontiguousarray(fields, dtype=np.float32)
    lv = np.ascontiguousarray(leaves, dtype=np.int32)
    tab = np.ascontiguousarray(amr_mod.finest_table(spec, lv), dtype=np.int32)
    B = spec.bsize
    c = Background()
    c.kind = OR_BG["grid"]
    c.domain = OR_DOM["sphere"]
    c.dom[:] = [spec.r_min, spec.r_max, spec.th_min, spec.th_max]
    c.nr, c.nth, c.nph = spec.nbr * B, spec.nbt * B, spec.nbp * B
    c.radial = 1 if spec.radial == "log" else 0
    c.n_snap, c.periodic, c.rec = spec.n_snap, int(spec.periodic), f.shape[-1]
    c.r_min, c.r_max, c.th_min, c.th_max = spec.r_min, spec.r_max, spec.th_min, spec.th_max
    c.t_snap0, c.dt_snap = spec.t_snap0, spec.dt_snap
    c.fields = f.ctypes.data
    c.amr_levels, c.amr_bsize, c.n_leaves = spec.levels, B, len(lv)
    c.leaves = lv.ctypes.data
    c.table = tab.ctypes.data
    return Bg(c, (f, lv, tab))


def amr_cell(bg, snap, leaf, li, lj, lk):
    o = (C.c_double * 18)()
    lib().or_amr_cell(C.byref(bg.c), snap, leaf, li, lj, lk, o)
    return np.array(o)


def analytic_background(kind, a=(), domain="none", dom=()):
    c = Background()
    c.kind = OR_BG[kind]
    c.domain = OR_DOM[domain]
    for i, v in enumerate(a):
        c.a[i] = v
    for i, v in enumerate(dom):
        c.dom[i] = v
    return Bg(c)


def params_c(p, shock_divv=0.0):
    c = ParamsC()
    c.dmumu = OR_DMUMU[p.dmumu]
    c.p_update = 0 if p.p_update == "exp" else 1
    c.kappa_drift, c.dvdt_term = int(p.kappa_drift), int(p.dvdt_term)
    c.lambda_par, c.p_ref, c.alpha = p.lambda_par, p.p_ref, p.alpha
    c.q, c.H, c.eps, c.mu_floor, c.lambda_perp = p.q, p.H, p.eps, p.mu_floor, p.lambda_perp
    c.dt, c.t0 = p.dt, p.t0
    c.seed, c.set_id = p.seed & 0xFFFFFFFF, p.set_id & 0xFFFFFFFF
    c.shock_divv = shock_divv
    return c


def inject_c(s):
    c = InjectC()
    c.region = {"point": 0, "box": 1}[s.region]
    c.energy = {"mono": 0, "powerlaw": 1}[s.energy]
    c.weight = {"unit": 0, "r-2": 1}[s.weight]
    c.mu_mode = {"isotropic": 0, "fixed": 1}[s.mu]
    c.r, c.th, c.ph = s.r, s.th, s.ph
    c.r1, c.r2, c.th1, c.th2, c.ph1, c.ph2 = s.r1, s.r2, s.th1, s.th2, s.ph1, s.ph2
    c.use_divv = 0 if s.divv_max is None else 1
    c.divv_snap, c.max_tries = s.divv_snap, s.max_tries
    c.divv_max = 0.0 if s.divv_max is None else s.divv_max
    c.e0, c.e1, c.e2, c.gamma, c.mu0 = s.e0, s.e1, s.e2, s.gamma, s.mu0
    c.seed, c.set_id = s.seed & 0xFFFFFFFF, s.set_id & 0xFFFFFFFF
    c.spiral, c.spiral_rb = getattr(s, "spiral", 0.0), getattr(s, "spiral_rb", 0.1)
    return c


def observer_c(o):
    c = ObserverC()
    c.kind = {"shell": 0, "box": 1, "slab": 2, "ring": 3}[o.kind]
    c.ne, c.nt = o.ne, o.nt
    c.r, c.dr, c.th, c.dth, c.ph, c.dph = o.r, o.dr, o.th, o.dth, o.ph, o.dph
    c.e_lo, c.e_hi, c.t_lo, c.t_hi = o.e_lo, o.e_hi, o.t_lo, o.t_hi
    return c


# --------------------------------------------------------------------------
# API
# --------------------------------------------------------------------------
def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*[x & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[x & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    L.or_philox4x32_10(c, k, o)
    return list(o)


def uniforms(seed, set_id, c0, pid, tag):
    u = (C.c_double * 4)()
    lib().or_uniforms(seed, set_id, c0, pid, tag, u)
    return list(u)


def normals(seed, set_id, n, pid):
    z = (C.c_double * 3)()
    lib().or_normals(seed, set_id, n, pid, z)
    return list(z)


def norm_integral(model, q=5.0 / 3.0, H=0.05, eps=0.048):
    return lib().or_norm_integral(OR_DMUMU[model], q, H, eps)


def dmumu(params, mu, v, p):
    o = (C.c_double * 3)()
    pc = params_c(params)
    lib().or_dmumu(C.byref(pc), mu, v, p, o)
    return list(o)


def eval_fields(bg, x, y, z, t):
    o = (C.c_double * 40)()
    lib().or_eval_fields(C.byref(bg.c), x, y, z, t, o)
    a = np.array(o)
    return dict(B=a[0:3], V=a[3:6], G=a[6:15].reshape(3, 3), gB=a[15:18], dVdt=a[18:21],
                dB=a[21:30].reshape(3, 3), divv=a[30])


class Ledger:
    def __init__(self):
        self.w = (C.c_double * 8)()
        self.n = (C.c_uint64 * 8)()

    def as_dict(self):
        return dict(w=np.array(self.w), n=np.array(self.n, dtype=np.uint64))


def inject(bg, spec, ids, ledger=None):
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.zeros(len(ids), dtype=PARTICLE)
    led = ledger or Ledger()
    sc = inject_c(spec)
    lib().or_inject(C.byref(bg.c), C.byref(sc), ids.ctypes.data, len(ids), out.ctypes.data,
                    led.w, led.n)
    return out, led


class Tally:
    def __init__(self, observers):
        self.observers = list(observers)
        self.nb = [o.ne * o.nt for o in self.observers]
        n = max(sum(self.nb), 1)
        self.S = np.zeros(n)
        self.S2 = np.zeros(n)
        self.C = np.zeros(n, dtype=np.uint64)
        self.A = np.zeros(n, dtype=np.uint64)
        # the tally S by particle id mod 32: [bin][class]
        self.SC = np.zeros((n, 32))
        self.oc = (ObserverC * max(len(self.observers), 1))(
            *[observer_c(o) for o in self.observers])

    def obs_view(self, o, arr):
        off = sum(self.nb[:o])
        ob = self.observers[o]
        return arr[off:off + self.nb[o]].reshape(ob.ne, ob.nt)

    def classes(self, o):
        """Observer o's S by particle id mod 32, [ne, nt, 32]."""
        off = sum(self.nb[:o])
        ob = self.observers[o]
        return self.SC[off:off + self.nb[o]].reshape(ob.ne, ob.nt, 32)

    def intensity(self, o):
        S = np.ascontiguousarray(self.obs_view(o, self.S))
        J = np.zeros_like(S)
        lib().or_intensity(C.byref(self.oc[o]), S.ctypes.data, J.ctypes.data)
        return J


class SmoothObsC(C.Structure):
    _fields_ = [("r_o", C.c_double), ("sigma_r", C.c_double), ("e_c", C.c_double),
                ("sigma_lnE", C.c_double), ("t_c", C.c_double), ("sigma_t", C.c_double)]


def observe(bg, params, particles, n_start, n_end, obs, threads=None):
    """Advance particles (in place, no tally) and return each one's smooth observable
    J_i = sum over alive steps of w dt K(start-of-step state); `obs` has r_o, sigma_r,
    e_c, sigma_lnE, t_c, sigma_t."""
    assert particles.dtype == PARTICLE and particles.flags.c_contiguous
    L = lib()
    J = np.zeros(len(particles))
    k = SmoothObsC(obs.r_o, obs.sigma_r, obs.e_c, obs.sigma_lnE, obs.t_c, obs.sigma_t)
    nthreads = threads or int(os.environ.get("FTE_ORACLE_THREADS", "0")) or L.or_max_threads()
    rc = L.or_observe(C.byref(bg.c), C.byref(params_c(params)), C.byref(k), particles.ctypes.data,
                      len(particles), n_start, n_end, J.ctypes.data, nthreads)
    if rc != 0:
        raise RuntimeError(f"or_observe failed ({rc})")
    return J


LR_PARAMS = ("lambda_par", "q", "H", "eps")


def mu_logpdf(mu1, m, s):
    """Log density (without -ln(2 pi)/2) of the pitch-angle cosine after a step whose
    Gaussian increment has mean m and width s, reflected at +-1."""
    return lib().or_mu_logpdf(float(mu1), float(m), float(s))


def observe_lr(bg, params, particles, n_start, n_end, obs, window, names=("lambda_par",), rel=1e-6,
               threads=None):
    """or_observe plus each particle's hybrid pathwise / score gradient of J_i with respect
    to `names` (a subset of LR_PARAMS): steps whose Gaussian pitch-angle increment has its
    mean within `window` widths of mu = 0 enter by the likelihood ratio of the held
    mu_{n+1}.  Returns (J [n], {name: gradient [n]}, flags [n]); particles advance in place."""
    assert particles.dtype == PARTICLE and particles.flags.c_contiguous
    L = lib()
    n = len(particles)
    J = np.zeros(n)
    G = np.zeros((n, 4))
    fl = np.zeros(n, dtype=np.int32)
    which = 0
    for nm in names:
        which |= 1 << LR_PARAMS.index(nm)
    k = SmoothObsC(obs.r_o, obs.sigma_r, obs.e_c, obs.sigma_lnE, obs.t_c, obs.sigma_t)
    nthreads = threads or int(os.environ.get("FTE_ORACLE_THREADS", "0")) or L.or_max_threads()
    rc = L.or_observe_lr(C.byref(bg.c), C.byref(params_c(params)), C.byref(k), float(window),
                         particles.ctypes.data, n, n_start, n_end, which, float(rel), J.ctypes.data,
                         G.ctypes.data, fl.ctypes.data, nthreads)
    if rc != 0:
        raise RuntimeError(f"or_observe_lr failed ({rc})")
    return J, {nm: G[:, LR_PARAMS.index(nm)].copy() for nm in names}, fl


def convolve(G, dt_bin, src=None):
    """Time-dependent source from the Green's function tally (Sec. 2.3: all particles
    injected at t = 0, then convolved with the source's time profile): for every
    energy row e, out[e, k] = dt_bin * sum_{m=0..k} src[m] * G[e, k - m], src[m] the
    source rate in time bin m (1 in every bin if None, which accumulates towards the
    steady state).  G: [ne, nt] array (occupancy sums or intensities)."""
    G = np.asarray(G, dtype=np.float64)
    ne, nt = G.shape
    src = np.ones(nt) if src is None else np.asarray(src, dtype=np.float64)
    out = np.zeros((ne, nt))
    for e in range(ne):
        for k in range(nt):
            acc = 0.0
            for m in range(k + 1):
                acc += src[m] * G[e, k - m]
            out[e, k] = dt_bin * acc
    return out


def advance(bg, params, particles, n_start, n_end, tally=None, ledger=None, threads=None,
            shock_divv=0.0):
    """Advance particles (structured PARTICLE array, in place) from step n_start to n_end."""
    assert particles.dtype == PARTICLE and particles.flags.c_contiguous
    L = lib()
    tally = tally if tally is not None else Tally([])
    led = ledger or Ledger()
    pc = params_c(params, shock_divv)
    nthreads = threads or int(os.environ.get("FTE_ORACLE_THREADS", "0")) or L.or_max_threads()
    rc = L.or_advance(C.byref(bg.c), C.byref(pc), tally.oc, len(tally.observers),
                      particles.ctypes.data, len(particles), n_start, n_end,
                      tally.S.ctypes.data, tally.S2.ctypes.data, tally.C.ctypes.data,
                      tally.A.ctypes.data, tally.SC.ctypes.data, led.w, led.n, nthreads)
    if rc != 0:
        raise RuntimeError(f"or_advance failed ({rc})")
    return tally, led


def step_terms(bg, params, particle, n):
    o = (C.c_double * 32)()
    p = np.ascontiguousarray(np.atleast_1d(particle).astype(PARTICLE))
    lib().or_step_terms(C.byref(bg.c), C.byref(params_c(params)), p.ctypes.data, n, o)
    a = list(o)
    keys = ["v", "gamma", "D", "dD", "mudot", "pdot_p", "divb", "divv", "bbgv", "bdvdt",
            "bx", "by", "bz", "Vx", "Vy", "Vz", "z0", "z1", "z2", "kappa", "ux", "uy", "uz",
            "x1", "y1", "z1_", "mu1", "p1", "E", "scale", "t", "event"]
    return dict(zip(keys, a))


def make_particles(n, x=0.0, y=0.0, z=0.0, mu=0.0, p=0.01, w=1.0, ids=None):
    P = np.zeros(n, dtype=PARTICLE)
    P["x"], P["y"], P["z"], P["mu"], P["p"], P["w"] = x, y, z, mu, p, w
    P["id"] = np.arange(n, dtype=np.uint32) if ids is None else ids
    P["n_div"] = -1
    P["n_sens"] = -1
    return P


C_AU = 299792458.0 / 1.495978707e11
MC2 = 938.27208816


def speed_of_p(p):
    return C_AU * p / math.sqrt(1.0 + p * p)
