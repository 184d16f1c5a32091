"""Python binding of the C ABI (argument marshalling only).

Device memory is allocated with PyTorch and handed to the library as raw
pointers; the CUDA stream is torch's current stream unless one is given.  The
function names are those of include/fte.h; every computation runs in the
library's kernels.
"""
import ctypes as C
import math

import numpy as np
import torch

from . import _abi as A
from ._abi import check

DEG = math.pi / 180.0


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# plain-data -> C struct conversions (fields follow fte_inputs.configs)
# ---------------------------------------------------------------------------
DTYPES = {"f32": A.FTE_F32, "bf16": A.FTE_BF16, "f16": A.FTE_F16}


LAYOUTS_REC = {"cell": A.FTE_LAYOUT_CELL, "pair": A.FTE_LAYOUT_PAIR}


def grid_c(g, dtype="f32", ring=0, layout="cell"):
    c = A.fte_grid()
    c.dtype = DTYPES[dtype]
    c.ring = int(ring)
    c.layout = LAYOUTS_REC[layout]
    c.nr, c.nth, c.nph = g.nr, g.nth, g.nph
    c.radial = 1 if g.radial == "log" else 0
    c.r_min, c.r_max, c.th_min, c.th_max = g.r_min, g.r_max, g.th_min, g.th_max
    c.n_snap, c.periodic = g.n_snap, int(bool(g.periodic))
    c.t_snap0, c.dt_snap = g.t_snap0, g.dt_snap
    return c


def inject_c(s, id_base=0):
    c = A.fte_inject_spec()
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
    c.id_base = id_base
    c.spiral, c.spiral_rb = getattr(s, "spiral", 0.0), getattr(s, "spiral_rb", 0.1)
    return c


def params_c(p):
    c = A.fte_params()
    c.dmumu = {"qlt": 0, "paper": 1, "iso": 2}[p.dmumu]
    c.p_update = 0 if p.p_update == "exp" else 1
    c.kappa_drift, c.dvdt_term = int(p.kappa_drift), int(p.dvdt_term)
    c.lambda_par, c.p_ref, c.alpha = p.lambda_par, p.p_ref, p.alpha
    c.q, c.H, c.eps, c.mu_floor, c.lambda_perp = p.q, p.H, p.eps, p.mu_floor, p.lambda_perp
    c.dt, c.t0 = p.dt, p.t0
    c.seed, c.set_id = p.seed & 0xFFFFFFFF, p.set_id & 0xFFFFFFFF
    c.sort_every = int(getattr(p, "sort_every", 0))
    c.tally_layout = {"global": A.FTE_LAYOUT_GLOBAL, "shared": A.FTE_LAYOUT_SHARED}[getattr(p, "tally_layout", "global")]
    return c


def observer_c(o):
    c = A.fte_observer()
    c.kind = {"shell": 0, "box": 1, "slab": 2, "ring": 3}[o.kind]
    c.ne, c.nt = o.ne, o.nt
    c.r, c.dr, c.th, c.dth, c.ph, c.dph = o.r, o.dr, o.th, o.dth, o.ph, o.dph
    c.e_lo, c.e_hi, c.t_lo, c.t_hi = o.e_lo, o.e_hi, o.t_lo, o.t_hi
    return c


# ---------------------------------------------------------------------------
# device-memory holders
# ---------------------------------------------------------------------------
class Background:
    """Device copy of a snapshot sequence (fte_background); dtype 'f32', 'bf16' or 'f16';
    record layout 'cell' or 'pair'."""

    def __init__(self, grid, device="cuda", dtype="f32", ring=0, layout="cell"):
        self.grid = grid
        self.dtype = dtype
        self.layout = layout
        self.gc = grid_c(grid, dtype, ring, layout)
        nbytes = A.lib().fte_background_bytes(C.byref(self.gc))
        if nbytes == 0:
            raise ValueError("invalid grid")
        self.nbytes = nbytes
        self.dev = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
        self.c = A.fte_background(self.gc, self.dev.data_ptr(), None, None)


def amr_grid_c(spec, n_leaves, dtype="f32", ring=0, layout="cell"):
    """fte_grid of an fte_inputs.amr.AmrSpec with n_leaves leaves."""
    c = A.fte_grid()
    c.ring = int(ring)
    c.layout = LAYOUTS_REC[layout]
    B = spec.bsize
    c.nr, c.nth, c.nph = spec.nbr * B, spec.nbt * B, spec.nbp * B
    c.radial = 1 if spec.radial == "log" else 0
    c.r_min, c.r_max, c.th_min, c.th_max = spec.r_min, spec.r_max, spec.th_min, spec.th_max
    c.n_snap, c.periodic = spec.n_snap, int(bool(spec.periodic))
    c.t_snap0, c.dt_snap = spec.t_snap0, spec.dt_snap
    c.dtype = DTYPES[dtype]
    c.amr_levels, c.amr_bsize, c.n_leaves = spec.levels, B, int(n_leaves)
    return c


class AmrBackground(Background):
    """Device block-AMR background: padded leaf fields, leaves and finest-level table.
    A 16-bit copy shares the leaves and table of the FP32 background it is quantized from."""

    def __init__(self, spec, leaves, device="cuda", dtype="f32", share=None, ring=0, layout="cell"):
        self.grid = spec
        self.dtype = dtype
        self.layout = layout
        self.gc = amr_grid_c(spec, len(leaves), dtype, ring, layout)
        nbytes = A.lib().fte_background_bytes(C.byref(self.gc))
        if nbytes == 0:
            raise ValueError("invalid AMR grid: " + A.lib().fte_last_error().decode())
        self.nbytes = nbytes
        self.dev = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
        if share is not None:
            self.leaves_dev, self.table_dev = share.leaves_dev, share.table_dev
        else:
            self.leaves_dev = torch.as_tensor(np.ascontiguousarray(leaves, dtype=np.int32)).to(device)
            tb = A.lib().fte_amr_table_bytes(C.byref(self.gc))
            self.table_dev = torch.empty(tb // 4, dtype=torch.int32, device=device)
        self.c = A.fte_background(self.gc, self.dev.data_ptr(), self.leaves_dev.data_ptr(),
                                  self.table_dev.data_ptr())


def fte_amr_prepare(bg, stream=None):
    check(A.lib().fte_amr_prepare(C.byref(bg.c), _stream(stream)), "fte_amr_prepare")


def fte_load_background(bg, host_fields, stream=None):
    """Copy host snapshot data (numpy float32 or CPU tensor, record layout) into bg."""
    if isinstance(host_fields, np.ndarray):
        host = np.ascontiguousarray(host_fields, dtype=np.float32)
        ptr, n = host.ctypes.data, host.nbytes
    else:
        assert host_fields.dtype == torch.float32 and host_fields.device.type == "cpu"
        host = host_fields.contiguous()
        ptr, n = host.data_ptr(), host.numel() * 4
    if n != bg.nbytes:
        raise ValueError(f"host data has {n} bytes, the grid needs {bg.nbytes}")
    check(A.lib().fte_load_background(C.byref(bg.gc), C.c_void_p(ptr), C.c_void_p(bg.dev.data_ptr()),
                                      bg.nbytes, _stream(stream)), "fte_load_background")
    return host


def fte_quantize_background(bg_half, bg_f32, stream=None):
    """Fill bg_half (16-bit and/or pair layout) from the FP32 cell-layout background bg_f32
    (same geometry)."""
    if bg_f32.dtype != "f32" or getattr(bg_f32, "layout", "cell") != "cell":
        raise ValueError("convert from an f32 cell-layout background")
    if bg_half.dtype == "f32" and getattr(bg_half, "layout", "cell") == "cell":
        raise ValueError("the target must be 16-bit or use the pair layout")
    if bg_half.gc.amr_levels != bg_f32.gc.amr_levels:
        raise ValueError("quantize between backgrounds of the same kind")
    check(A.lib().fte_quantize_background(C.byref(bg_half.gc), C.c_void_p(bg_f32.dev.data_ptr()),
                                          C.c_void_p(bg_half.dev.data_ptr()), bg_half.nbytes,
                                          _stream(stream)), "fte_quantize_background")


def device_bytes(bg):
    """Host copy of a background's device array as raw bytes."""
    return bg.dev.view(torch.uint8)[: bg.nbytes].cpu().numpy()


class Particles:
    """Device particle pool (fte_particles, structure of arrays)."""

    def __init__(self, capacity, device="cuda"):
        f = lambda: torch.zeros(capacity, dtype=torch.float32, device=device)
        self.x, self.y, self.z, self.mu, self.p, self.w = f(), f(), f(), f(), f(), f()
        self.id = torch.zeros(capacity, dtype=torch.int32, device=device)
        self.status = torch.full((capacity,), A.FTE_INJ_FAIL, dtype=torch.uint8, device=device)
        self.c = A.fte_particles(self.x.data_ptr(), self.y.data_ptr(), self.z.data_ptr(),
                                 self.mu.data_ptr(), self.p.data_ptr(), self.w.data_ptr(),
                                 self.id.data_ptr(), self.status.data_ptr(), capacity, 0)

    @property
    def count(self):
        return self.c.count

    def state(self):
        """Host copy of the used part of the pool as a dict of numpy arrays."""
        n = self.count
        out = {k: getattr(self, k)[:n].cpu().numpy() for k in ("x", "y", "z", "mu", "p", "w")}
        out["id"] = self.id[:n].cpu().numpy().view(np.uint32)
        out["status"] = self.status[:n].cpu().numpy()
        return out

    def load_state(self, st):
        """Restore a pool saved with state() (a checkpoint): with the step index it is the whole
        state of a run, since every random number is a function of (seed, set, step, id)."""
        n = len(st["x"])
        if n > self.c.capacity:
            raise ValueError("pool capacity %d < %d" % (self.c.capacity, n))
        for k in ("x", "y", "z", "mu", "p", "w"):
            getattr(self, k)[:n].copy_(torch.from_numpy(np.ascontiguousarray(st[k], dtype=np.float32)))
        self.id[:n].copy_(torch.from_numpy(np.ascontiguousarray(st["id"]).view(np.int32)))
        self.status[:n].copy_(torch.from_numpy(np.ascontiguousarray(st["status"], dtype=np.uint8)))
        self.c.count = n


class Tally:
    """Device tally accumulators and ledger (fte_tally_buf); n_sets blocks of bins
    for an ensemble."""

    def __init__(self, observers, device="cuda", n_sets=1):
        self.observers = list(observers)
        if len(self.observers) > A.FTE_MAX_OBS:
            raise ValueError("too many observers")
        self.nb = [o.ne * o.nt for o in self.observers]
        self.n_sets = int(n_sets)
        n = max(sum(self.nb), 1) * max(self.n_sets, 1)
        self.S = torch.zeros(n, dtype=torch.float64, device=device)
        self.S2 = torch.zeros(n, dtype=torch.float64, device=device)
        self.C = torch.zeros(n, dtype=torch.int64, device=device)
        self.ledger_w = torch.zeros(A.FTE_LEDGER, dtype=torch.float64, device=device)
        self.ledger_n = torch.zeros(A.FTE_LEDGER, dtype=torch.int64, device=device)
        # the tally by particle-id class: [set][bin][class]
        self.S_class = torch.zeros((max(self.n_sets, 1), max(sum(self.nb), 1), A.FTE_NCLASS),
                                   dtype=torch.float64, device=device)
        self.out = torch.zeros(max(self.nb + [1]), dtype=torch.float64, device=device)
        c = A.fte_tally_buf()
        c.n_obs = len(self.observers)
        c.n_sets = self.n_sets
        for i, o in enumerate(self.observers):
            c.obs[i] = observer_c(o)
        c.S, c.S2, c.C = self.S.data_ptr(), self.S2.data_ptr(), self.C.data_ptr()
        c.ledger_w, c.ledger_n = self.ledger_w.data_ptr(), self.ledger_n.data_ptr()
        c.S_class = self.S_class.data_ptr()
        self.c = c

    def classes(self, obs=0, set=0):
        """Observer `obs`'s bins by particle-id class, float64 numpy [ne, nt, FTE_NCLASS]."""
        off = sum(self.nb[:obs])
        ob = self.observers[obs]
        c = self.S_class[set, off:off + self.nb[obs]].double().cpu().numpy()
        return c.reshape(ob.ne, ob.nt, A.FTE_NCLASS)

    def batch_sigma(self, obs=0, set=0):
        """Standard error of every bin of observer `obs` from its FTE_NCLASS particle-id
        class sums (batch means), float64 numpy [ne, nt]."""
        c = self.classes(obs, set)
        return (c.shape[-1] * c.var(axis=-1, ddof=1)) ** 0.5

    def batch_means(self, obs=0, set=0):
        """Observer `obs`'s total occupancy (sum of w dt over its tallied steps) and the
        relative standard error of that total from its FTE_NCLASS particle-id class sums
        (batch means: the particles are independent, so the class sums are independent
        estimates of 1/FTE_NCLASS of the total).  Returns (total, rel_err or None)."""
        c = self.classes(obs, set).reshape(-1, A.FTE_NCLASS).sum(axis=0)
        tot = float(c.sum())
        if tot <= 0:
            return tot, None
        k = len(c)
        return tot, float((k * c.var(ddof=1)) ** 0.5 / tot)


class Workspace:
    """Device scratch for fte_advance, grown on demand."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = torch.empty(0, dtype=torch.uint8, device=device)

    def ensure(self, nbytes):
        if self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


# ---------------------------------------------------------------------------
# the C ABI, one wrapper per entry point
# ---------------------------------------------------------------------------
def fte_workspace_bytes(bg, tally, n_particles, n_steps, device=None):
    dev = torch.cuda.current_device() if device is None else device
    n = A.lib().fte_workspace_bytes(dev, C.byref(bg.gc), C.byref(tally.c), int(n_particles), int(n_steps))
    if n == 0:
        raise RuntimeError("fte_workspace_bytes: " + A.lib().fte_last_error().decode())
    return n


def fte_tally_reset(tally, stream=None):
    check(A.lib().fte_tally_reset(C.byref(tally.c), _stream(stream)), "fte_tally_reset")


def fte_inject(pool, bg, spec, n, tally, id_base=None, check_failed=True, stream=None):
    """Append n particles drawn per `spec`; returns the number of failed injections
    (None if check_failed is False, in which case the call does not synchronise)."""
    base = pool.count if id_base is None else id_base
    sc = inject_c(spec, base)
    nf = C.c_uint64(0)
    st = A.lib().fte_inject(C.byref(pool.c), C.byref(bg.c), C.byref(sc), int(n), C.byref(tally.c),
                            C.byref(nf) if check_failed else None, _stream(stream))
    if st == A.FTE_ERANGE:
        return nf.value
    check(st, "fte_inject")
    return nf.value if check_failed else None


def fte_advance(pool, bg, params, tally, n_start, n_end, ws=None, stream=None):
    ws = ws if ws is not None else Workspace(bg.dev.device)
    buf = ws.ensure(fte_workspace_bytes(bg, tally, pool.count, n_end - n_start, bg.dev.device.index))
    pc = params_c(params)
    check(A.lib().fte_advance(C.byref(pool.c), C.byref(bg.c), C.byref(pc), C.byref(tally.c),
                              int(n_start), int(n_end), C.c_void_p(buf.data_ptr()), buf.numel(),
                              _stream(stream)), "fte_advance")
    return ws


def fte_advance_noalloc(pool, bg, params, tally, n_start, n_end, stream=None):
    """fte_advance without a workspace: the library's own statically placed
    device scratch is used, for callers that cannot allocate device memory."""
    pc = params_c(params)
    check(A.lib().fte_advance_noalloc(C.byref(pool.c), C.byref(bg.c), C.byref(pc), C.byref(tally.c),
                                      int(n_start), int(n_end), _stream(stream)), "fte_advance_noalloc")


def fte_tally(tally, obs, kind=A.FTE_TALLY_S, stream=None):
    """Observer `obs`'s [ne, nt] array of `kind` (S, S2, C or INTENSITY) on the host."""
    ob = tally.observers[obs]
    host = np.zeros((ob.ne, ob.nt), dtype=np.float64)
    check(A.lib().fte_tally(C.byref(tally.c), int(obs), int(kind), C.c_void_p(tally.out.data_ptr()),
                            C.c_void_p(host.ctypes.data), host.nbytes, _stream(stream)), "fte_tally")
    return host


def fte_probe_gather_l1(buf, threads, records, spread, out, stream=None):
    """The transport kernel's record loads from the L1-sized device tensor `buf` of FP32
    cell records (measurement aid, include/fte_probe.h)."""
    check(A.lib().fte_probe_gather_l1(C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                      int(threads), int(records), int(spread), C.c_void_p(out.data_ptr()),
                                      _stream(stream)), "fte_probe_gather_l1")


def fte_probe_step_timing(capacity):
    """Record CUDA events around up to `capacity` step-kernel launches of fte_advance
    (0: stop; measurement aid, include/fte_probe.h)."""
    check(A.lib().fte_probe_step_timing(int(capacity)), "fte_probe_step_timing")


def fte_probe_step_intervals(capacity=1 << 16):
    """(start, end) in ms of every recorded step-kernel launch since the last read,
    relative to the first start (float64 array [n, 2]); synchronises the events."""
    out = np.zeros(2 * capacity, dtype=np.float64)
    n = C.c_int(0)
    check(A.lib().fte_probe_step_intervals(C.c_void_p(out.ctypes.data), int(capacity), C.byref(n)),
          "fte_probe_step_intervals")
    return out[:2 * n.value].reshape(-1, 2)


def fte_probe_sectors(buf, threads, loads, out, stream=None):
    """Random 32-byte sector reads of the device tensor `buf` (measurement aid,
    include/fte_probe.h)."""
    check(A.lib().fte_probe_sectors(C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(),
                                    int(threads), int(loads), C.c_void_p(out.data_ptr()),
                                    _stream(stream)), "fte_probe_sectors")


def fte_ledger(tally, stream=None):
    w = (C.c_double * A.FTE_LEDGER)()
    n = (C.c_uint64 * A.FTE_LEDGER)()
    check(A.lib().fte_ledger(C.byref(tally.c), w, n, _stream(stream)), "fte_ledger")
    return np.array(w), np.array(n, dtype=np.uint64)


# ---------------------------------------------------------------------------
# ensembles, the launch-configuration autotuner and CUDA graphs
# ---------------------------------------------------------------------------
LAYOUTS = {"shared": A.FTE_LAYOUT_SHARED, "global": A.FTE_LAYOUT_GLOBAL}
LAYOUT_NAMES = {v: k for k, v in LAYOUTS.items()}


def sets_c(sets):
    """fte_set array of fte_inputs.configs.EnsembleSet entries."""
    arr = (A.fte_set * len(sets))()
    for i, e in enumerate(sets):
        arr[i] = A.fte_set(e.lambda_par, e.q, e.H, e.eps, e.seed & 0xFFFFFFFF, e.set_id & 0xFFFFFFFF, int(e.count))
    return arr


def config_c(cfg):
    """fte_launch_config of a dict {threads, steps_per_launch, tally_layout} (None: library default)."""
    if cfg is None:
        return None
    return A.fte_launch_config(int(cfg["threads"]), int(cfg["steps_per_launch"]),
                               LAYOUTS[cfg["tally_layout"]], 0)


def _config_dict(c):
    return {"threads": c.threads, "steps_per_launch": c.steps_per_launch,
            "tally_layout": LAYOUT_NAMES.get(c.tally_layout, str(c.tally_layout))}


def fte_workspace_bytes_batched(bg, tally, n_particles, n_steps, device=None):
    dev = torch.cuda.current_device() if device is None else device
    n = A.lib().fte_workspace_bytes_batched(dev, C.byref(bg.gc), C.byref(tally.c), int(n_particles), int(n_steps))
    if n == 0:
        raise RuntimeError("fte_workspace_bytes_batched: " + A.lib().fte_last_error().decode())
    return n


def fte_inject_batched(pool, bg, sets, tally, stream=None):
    """Inject every set (EnsembleSet.inject, EnsembleSet.count) one after another; ids restart
    at 0 in every set.  Asynchronous."""
    specs = (A.fte_inject_spec * len(sets))()
    for i, e in enumerate(sets):
        specs[i] = inject_c(e.inject, 0)
    counts = (C.c_uint64 * len(sets))(*[int(e.count) for e in sets])
    check(A.lib().fte_inject_batched(C.byref(pool.c), C.byref(bg.c), specs, counts, len(sets),
                                     C.byref(tally.c), _stream(stream)), "fte_inject_batched")


def fte_advance_batched(pool, bg, params, sets, tally, n_start, n_end, ws=None, config=None, stream=None):
    ws = ws if ws is not None else Workspace(bg.dev.device)
    buf = ws.ensure(fte_workspace_bytes_batched(bg, tally, pool.count, n_end - n_start, bg.dev.device.index))
    pc = params_c(params)
    sc = sets_c(sets)
    cc = config_c(config)
    check(A.lib().fte_advance_batched(C.byref(pool.c), C.byref(bg.c), C.byref(pc), sc, len(sets),
                                      C.byref(tally.c), int(n_start), int(n_end),
                                      C.byref(cc) if cc is not None else None,
                                      C.c_void_p(buf.data_ptr()), buf.numel(), _stream(stream)),
          "fte_advance_batched")
    return ws


def fte_autotune_batched(pool, bg, params, sets, tally, n_start, n_end, ws=None, stream=None):
    """Advance steps n_start..n_end while timing every launch configuration on a slice of them;
    returns (best configuration, [(configuration, alive particle-steps per second), ...])."""
    ws = ws if ws is not None else Workspace(bg.dev.device)
    buf = ws.ensure(fte_workspace_bytes_batched(bg, tally, pool.count, n_end - n_start, bg.dev.device.index))
    pc = params_c(params)
    sc = sets_c(sets)
    best = A.fte_launch_config()
    tried = (A.fte_launch_config * 16)()
    rates = (C.c_double * 16)()
    n_tried = C.c_int(0)
    check(A.lib().fte_autotune_batched(C.byref(pool.c), C.byref(bg.c), C.byref(pc), sc, len(sets),
                                       C.byref(tally.c), int(n_start), int(n_end),
                                       C.c_void_p(buf.data_ptr()), buf.numel(), C.byref(best), tried, rates,
                                       C.byref(n_tried), _stream(stream)), "fte_autotune_batched")
    return _config_dict(best), [(_config_dict(tried[k]), rates[k]) for k in range(n_tried.value)]


def fte_tally_set(tally, set_index, obs, kind=A.FTE_TALLY_S, stream=None):
    """fte_tally for parameter set `set_index` of an ensemble tally."""
    ob = tally.observers[obs]
    host = np.zeros((ob.ne, ob.nt), dtype=np.float64)
    check(A.lib().fte_tally_set(C.byref(tally.c), int(set_index), int(obs), int(kind),
                                C.c_void_p(tally.out.data_ptr()), C.c_void_p(host.ctypes.data), host.nbytes,
                                _stream(stream)), "fte_tally_set")
    return host


class Graph:
    """A CUDA graph of library calls: `with g.capture(stream): ...` records the asynchronous
    fte_* calls made on `stream` (not torch's default stream); g.launch(stream) replays them."""

    def __init__(self):
        self.h = C.c_void_p(0)

    def capture(self, stream):
        graph = self

        class _Cap:
            def __enter__(self):
                check(A.lib().fte_graph_begin(_stream(stream)), "fte_graph_begin")
                return graph

            def __exit__(self, *exc):
                h = C.c_void_p(0)
                st = A.lib().fte_graph_end(_stream(stream), C.byref(h))
                if exc[0] is None:
                    check(st, "fte_graph_end")
                graph.h = h
                return False
        return _Cap()

    def launch(self, stream=None):
        check(A.lib().fte_graph_launch(self.h, _stream(stream)), "fte_graph_launch")

    def __del__(self):
        try:
            if self.h and self.h.value:
                A.lib().fte_graph_destroy(self.h)
        except Exception:
            pass


def fte_tally_convolve(tally, obs, kind=A.FTE_TALLY_INTENSITY, src=None, set_index=0, stream=None):
    """Observer `obs`'s Green's-function tally convolved with the source rate per time bin
    (`src`: device tensor of nt doubles, None for a constant unit source), on the host."""
    ob = tally.observers[obs]
    host = np.zeros((ob.ne, ob.nt), dtype=np.float64)
    sp = C.c_void_p(src.data_ptr()) if src is not None else None
    check(A.lib().fte_tally_convolve(C.byref(tally.c), int(set_index), int(obs), int(kind), sp,
                                     C.c_void_p(tally.out.data_ptr()), C.c_void_p(host.ctypes.data), host.nbytes,
                                     _stream(stream)), "fte_tally_convolve")
    return host


# ---------------------------------------------------------------------------
# pathwise adjoint of a smooth observable, and its torch.autograd.Function
# ---------------------------------------------------------------------------
GRAD_NAMES = ("lambda_par", "q", "H", "eps", "gamma")


def smooth_c(o):
    return A.fte_smooth_obs(o.r_o, o.sigma_r, o.e_c, o.sigma_lnE, o.t_c, o.sigma_t,
                            float(getattr(o, "lr_window", -1.0)))


def fte_adjoint_workspace_bytes(bg, n_particles, n_steps, checkpoint_every, device=None):
    dev = torch.cuda.current_device() if device is None else device
    n = A.lib().fte_adjoint_workspace_bytes(dev, C.byref(bg.gc), int(n_particles), int(n_steps),
                                             int(checkpoint_every))
    if n == 0:
        raise RuntimeError("fte_adjoint_workspace_bytes: " + A.lib().fte_last_error().decode())
    return n


class Adjoint:
    """One checkpointed forward pass and its reverse pass (fte_adjoint_forward / _reverse) for a
    particle pool, a background, transport parameters and a smooth observable."""

    def __init__(self, bg, params, obs, n_start, n_end, checkpoint_every=256, ws=None, device="cuda"):
        self.bg, self.params, self.obs = bg, params, obs
        self.n_start, self.n_end, self.K = int(n_start), int(n_end), int(checkpoint_every)
        self.ws = ws if ws is not None else Workspace(device)
        self.out = torch.zeros(1 + A.FTE_NGRAD, dtype=torch.float64, device=device)

    def forward(self, pool, stream=None, per_particle=False):
        """Advance `pool` and return J (a 0-d device tensor, valid once the stream reaches it);
        with per_particle also each particle's J_i (float64 device tensor [n])."""
        buf = self.ws.ensure(fte_adjoint_workspace_bytes(self.bg, pool.count, self.n_end - self.n_start, self.K))
        Ji = torch.zeros(pool.count, dtype=torch.float64, device=buf.device) if per_particle else None
        check(A.lib().fte_adjoint_forward(C.byref(pool.c), C.byref(self.bg.c), C.byref(params_c(self.params)),
                                          C.byref(smooth_c(self.obs)), self.n_start, self.n_end, self.K,
                                          C.c_void_p(self.out.data_ptr()),
                                          C.c_void_p(Ji.data_ptr()) if Ji is not None else None,
                                          C.c_void_p(buf.data_ptr()), buf.numel(), _stream(stream)),
              "fte_adjoint_forward")
        self.n_particles = pool.count
        return (self.out[0], Ji) if per_particle else self.out[0]

    def reverse(self, pool, inject=None, per_particle=False, stream=None):
        """Gradients of J (device tensor of FTE_NGRAD doubles, in GRAD_NAMES order); with
        per_particle also each particle's [J_i, gradients] (float32 [n, 1 + FTE_NGRAD])."""
        buf = self.ws.buf
        pp = torch.zeros((pool.count, 1 + A.FTE_NGRAD), dtype=torch.float32, device=buf.device) \
            if per_particle else None
        spec = inject_c(inject, 0) if inject is not None else None
        check(A.lib().fte_adjoint_reverse(C.byref(pool.c), C.byref(self.bg.c), C.byref(params_c(self.params)),
                                          C.byref(smooth_c(self.obs)), C.byref(spec) if spec is not None else None,
                                          self.n_start, self.n_end, self.K, C.c_void_p(self.out.data_ptr()),
                                          C.c_void_p(pp.data_ptr()) if pp is not None else None,
                                          C.c_void_p(buf.data_ptr()), buf.numel(), _stream(stream)),
              "fte_adjoint_reverse")
        return (self.out[1:], pp) if per_particle else self.out[1:]


class SmoothIntensity(torch.autograd.Function):
    """J(theta) for theta = (lambda_par, q, H, eps, gamma): forward injects `run.n_particles`
    particles per run.inject (power-law index gamma), advances them through the checkpointed
    forward pass and returns J; backward runs the reverse pass.  `run` carries bg, params,
    inject, obs, n_steps, n_particles and checkpoint_every (plain attributes)."""

    @staticmethod
    def forward(ctx, theta, run):
        import dataclasses
        th = [float(v) for v in theta.detach().cpu().tolist()]
        prm = dataclasses.replace(run.params, lambda_par=th[0], q=th[1], H=th[2], eps=th[3])
        inj = dataclasses.replace(run.inject, gamma=th[4])
        pool = Particles(run.n_particles, device=run.bg.dev.device)
        tally = Tally([], device=run.bg.dev.device)
        fte_tally_reset(tally)
        fte_inject(pool, run.bg, inj, run.n_particles, tally, id_base=0, check_failed=False)
        adj = Adjoint(run.bg, prm, run.obs, 0, run.n_steps, run.checkpoint_every, device=run.bg.dev.device)
        J = adj.forward(pool)
        ctx.adj, ctx.pool, ctx.inj = adj, pool, inj
        ctx.theta_device, ctx.theta_dtype = theta.device, theta.dtype
        return J.detach().clone().to(theta.device, theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.adj.reverse(ctx.pool, ctx.inj).to(ctx.theta_device, ctx.theta_dtype)
        return grad_out * g, None


# ---------------------------------------------------------------------------
# snapshot streaming through a ring of resident slots
# ---------------------------------------------------------------------------
def fte_snapshot_bytes(bg):
    return A.lib().fte_snapshot_bytes(C.byref(bg.gc))


def fte_stream_plan(bg, params, n_start, n_end):
    """Runs of steps sharing a snapshot pair: int64 array [runs, 3] = (first, end, key); key >= 0 is
    the unwrapped earlier snapshot of the pair, key < 0 freezes the fields at snapshot -1 - key."""
    pc = params_c(params)
    count = C.c_int64(0)
    st = A.lib().fte_stream_plan(C.byref(bg.gc), C.byref(pc), int(n_start), int(n_end), None, 0, C.byref(count))
    if st not in (A.FTE_OK, A.FTE_ENOMEM):
        check(st, "fte_stream_plan")
    out = np.zeros((max(count.value, 1), 3), dtype=np.int64)
    check(A.lib().fte_stream_plan(C.byref(bg.gc), C.byref(pc), int(n_start), int(n_end),
                                  C.c_void_p(out.ctypes.data), count.value, C.byref(count)), "fte_stream_plan")
    return out[:count.value]


class SnapshotStream:
    """Host snapshots (page-locked FP32 cell records) and the ring's slot bookkeeping for
    fte_advance_streamed; `copy_stream` carries the uploads.  A 16-bit or pair-layout ring
    also gets a device staging snapshot, and a 16-bit ring its per-field scales from all
    host snapshots (fte_stream_scales) here, before any slot is filled."""

    def __init__(self, bg, host_fields, device="cuda"):
        if bg.gc.ring < 2:
            raise ValueError("the background has no ring")
        t = host_fields if isinstance(host_fields, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(host_fields))
        self.host = t if t.is_pinned() else t.pin_memory()
        need = fte_snapshot_bytes(bg) * bg.gc.n_snap
        if self.host.numel() * self.host.element_size() < need:
            raise ValueError("host snapshots hold %d bytes, need %d" % (self.host.numel() * self.host.element_size(), need))
        self.slots = np.full(bg.gc.ring, -1, dtype=np.int64)
        self.copy_stream = torch.cuda.Stream(device=device)
        self.bg = bg
        nst = A.lib().fte_stream_staging_bytes(C.byref(bg.gc))
        self.staging = torch.empty(nst, dtype=torch.uint8, device=bg.dev.device) if nst else None
        if bg.gc.dtype != A.FTE_F32:
            cur = torch.cuda.current_stream()
            self.copy_stream.wait_stream(cur)
            check(A.lib().fte_stream_scales(C.byref(bg.c), C.c_void_p(self.host.data_ptr()), *self._staging(),
                                            _stream(self.copy_stream)), "fte_stream_scales")
            cur.wait_stream(self.copy_stream)

    def _staging(self):
        if self.staging is None:
            return C.c_void_p(None), 0
        return C.c_void_p(self.staging.data_ptr()), self.staging.numel()

    def load(self, u, stream=None):
        """Copy unwrapped snapshot u into its slot, e.g. the injection snapshot before fte_inject:
        on the copy stream, after the work already on `stream` (torch's current stream by
        default), which then waits for the copy."""
        cur = stream if stream is not None else torch.cuda.current_stream()
        self.copy_stream.wait_stream(cur)
        check(A.lib().fte_stream_load(C.byref(self.bg.c), C.c_void_p(self.host.data_ptr()), int(u),
                                      C.c_void_p(self.slots.ctypes.data), *self._staging(),
                                      _stream(self.copy_stream)),
              "fte_stream_load")
        cur.wait_stream(self.copy_stream)


def fte_advance_streamed(pool, bg, stream_state, params, tally, n_start, n_end, ws=None, stream=None):
    """fte_advance over a ring background, uploading snapshots as the run reaches them."""
    ws = ws if ws is not None else Workspace(bg.dev.device)
    # a time table for the whole range lets the library advance several runs per call
    buf = ws.ensure(fte_workspace_bytes(bg, tally, pool.count, n_end - n_start, bg.dev.device.index))
    pc = params_c(params)
    check(A.lib().fte_advance_streamed(C.byref(pool.c), C.byref(bg.c), C.c_void_p(stream_state.host.data_ptr()),
                                       C.byref(pc), C.byref(tally.c), int(n_start), int(n_end),
                                       C.c_void_p(stream_state.slots.ctypes.data), *stream_state._staging(),
                                       C.c_void_p(buf.data_ptr()), buf.numel(), _stream(stream),
                                       _stream(stream_state.copy_stream)),
          "fte_advance_streamed")
    return ws
