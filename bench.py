"""Throughput benchmark of the focused-transport pusher on GB300.

Workload (one bench step = one full pass of the hot path over one batch):
  synthetic CIR in the corotating frame on a 512 r x 60 theta x 180 phi grid,
  24 hourly snapshots (periodic), 1e6 protons injected at 50 keV uniformly over
  the div V < 0 cells of one CIR between 1 and 2 au at theta = 90 +- 2 deg with
  weight 1/r^2, quasi-linear D_mumu (q = 5/3, H = 0.05, lambda_par = 0.1 au),
  dt = 10 s for 4 days (34,560 steps), occupancy tally at a 1 au observer box
  (16 log energy bins x 144 time bins).  Per step: inject, advance, read the tally.

Metric: alive particle-steps per second (whole job, all ranks).
`value` times the device work with the inputs resident in HBM; `e2e` times the
same step through the C ABI starting from host buffers: the snapshots stream
from page-locked memory into a ring of one slot per snapshot (each copied once
per step, overlapped with the steps of earlier intervals), and the tally and
ledger are read back.  `e2e.breakdown` splits the gap between the two on the box
that runs it (rank 0's own particles): the streamed calls without copies, a
device-timed step with them, and the copies alone with the host's time to issue
them.

Multi-GPU: every rank runs its own batch of 1e6 particles (distinct particle
ids, weak scaling) and the tallies are summed over ranks after each step.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.

The device background uses the cell record layout by default (`--layout pair`
measures records that hold a cell and its upper r-neighbour, converted on the
device from the uploaded cell records).  The default
line also carries the 16-bit storage forms (`forms`), the adjoint's cost on a
slice of the workload (`adjoint`), the 64-set ensemble (`ensemble`, the same three
arms as `--case ensemble`) and the block-AMR workload (`amr`).  Other cases, each one
JSON line: `--case amr` (the CIR on a 39,520-leaf block-AMR grid, 1e7 protons,
FP32/BF16/FP16), `--case ensemble` (64 parameter sets, 2e7 protons: set after
set, one ensemble launch, autotuned and graph-captured), `--case adjoint` (the
full 4-day adjoint with a finite-difference check), `--case profile` (small
cases for ncu captures), `--case slices` (the rate per 1024-step slice of the 4-day run, against
the number of alive particles).
"""
import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from fte_inputs import configs  # noqa: E402

METRIC = "FTE particle-steps/s on 1 GB300 at stated tally error; % gather roofline; adj/fwd"
UNIT = "particle-steps/s"
ALG_BYTES = 2 * 8 * 18 * 4          # 2 snapshots x 8 corners x 18 fields x 4 B per particle-step

# Error of the 16-bit storage forms against the FP64 oracle on the FP32 fields, per output: the
# bounds tests/test_gpu_precision.py::test_storage_error_per_output and
# tests/test_gpu_adjoint.py::test_gradient_storage_error assert (both import this table), and
# what they measured on GB300 (small CIR grid, 4000 particles).
STORAGE_ERROR = {
    "bf16": {"trajectory_p99_at_400_steps": {"pos_rel": 3e-4, "mu": 3e-3, "p_rel": 3e-3},
             "measured": {"trajectory_p99_at_400_steps": {"pos_rel": 4.4e-5, "mu": 3.7e-4, "p_rel": 3.9e-4},
                          "tally_bins": {"max_abs_z": 0.07, "share_beyond_3_sigma": 0.0, "mean_z": -0.01},
                          "ledger_absorbed_count_differences": {"inner": 0, "outer": -1, "theta": 0},
                          "adjoint_total_rel": {"J": -1.9e-5, "lambda_par": 1.3e-2, "q": 3.0e-2, "H": -3.1e-3}}},
    "f16": {"trajectory_p99_at_400_steps": {"pos_rel": 3e-5, "mu": 3e-4, "p_rel": 3e-4},
            "measured": {"trajectory_p99_at_400_steps": {"pos_rel": 4.5e-6, "mu": 3.9e-5, "p_rel": 4.4e-5},
                         "tally_bins": {"max_abs_z": 0.03, "share_beyond_3_sigma": 0.0, "mean_z": 0.0},
                         "ledger_absorbed_count_differences": {"inner": 0, "outer": 0, "theta": 0},
                         "adjoint_total_rel": {"J": -6.8e-6, "lambda_par": 2.2e-3, "q": 2.0e-2, "H": 1.4e-2}}},
}
STORAGE_ERROR_COMMON = {
    "trajectory": "99th percentile over the particles of |16-bit run - FP64 oracle| before the first "
                  "divergence event (position relative to r, mu absolute, p relative)",
    "tally_bins": {"max_share_beyond_3_sigma": 0.05, "max_abs_mean_z": 1.0,
                   "sigma": "batch-means standard error of the bin difference (32 particle-id classes, both sides)"},
    "ledger": "absorbed counts per face within 4 binomial sigma of the oracle's",
    "adjoint": {"J_rel": 0.02, "gradient_total_sigma": 4.0, "gradient_total_rel": 0.05,
                "gradient_total": "|16-bit total - FP32-field oracle total| within gradient_total_sigma batch-means "
                                  "sigma of the per-particle differences + gradient_total_rel of the oracle total"},
    "source": "tests/test_gpu_precision.py::test_storage_error_per_output, "
              "tests/test_gpu_adjoint.py::test_gradient_storage_error",
}
# steps per fte_advance call: larger than every run here, so each run is one call (a call
# ends with its two half-pools joined and a partial reordering chunk; 1024-step calls
# measured 0.3 % slower than the streamed path's longer calls)
CHUNK = 1 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "advance_kernel_traffic.json")
KERNEL_SOURCES = ("fte_advance.cu", "fte_device.cuh", "fte_kernels.cuh", "fte_step.cuh", "fte_sort.cu", "fte_api.cu")


def kernel_sources_hash():
    """sha256 of the step kernel's sources, of the particle ordering that sets its access
    pattern and of the library code that shapes its launches: DRAM traffic measured by ncu is
    reported only while all are unchanged."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2404_12164_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(layout, dtype="f32"):
    """The committed ncu record of the step kernel for one storage type (DRAM bytes per alive
    particle-step of the profile case, and its L1 data-pipe figures), or None when the kernel
    sources changed since, the record is for another record layout or has no capture of
    `dtype` ("f32", "bf16", "f16" on the uniform grid, "amr_f32" on the block-AMR grid)."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("sources_sha256") != kernel_sources_hash() or d.get("record_layout") != layout:
        return None
    e = d.get("by_dtype", {}).get(dtype)
    if not e:
        return None
    return {"dram_bytes_per_particle_step": e.get("dram_bytes_per_particle_step"),
            "source": TRAFFIC_FILE.split(ROOT + os.sep)[-1] + " (" + dtype + ")", "l1": e.get("l1")}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def device_background(api, w, fields, layout, dtype="f32"):
    """The workload's background on the device in the given record layout and storage dtype
    (converted on the device from the FP32 cell records)."""
    import torch
    cell = api.Background(w.grid)
    src = fields if isinstance(fields, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(fields))
    api.fte_load_background(cell, src)
    if layout == "cell" and dtype == "f32":
        return cell
    bg = api.Background(w.grid, dtype=dtype, layout=layout)
    api.fte_quantize_background(bg, cell)
    torch.cuda.synchronize()
    del cell
    torch.cuda.empty_cache()
    return bg


def build_workload():
    w = configs.cir_uniform_1e6()
    cache = os.environ.get("FTE_BG_CACHE")
    path = os.path.join(cache, "cir_uniform_512x60x180x24.npy") if cache else None
    if path and os.path.exists(path):
        return w, np.load(path, mmap_mode="r")
    f = configs.build_background(w)
    if path:
        os.makedirs(cache, exist_ok=True)
        np.save(path, f)
    return w, f


def e2e_breakdown(api, pool, ring_bg, sstream, w, tally, wsp, id_base, stream, barrier):
    """Where the end-to-end step's time goes, from three more steps on the streamed ring:
    the streamed calls with every snapshot already in its slot (the cost of advancing in
    snapshot-interval groups, no copy), a step with every snapshot copied (device-timed,
    without the host's read of the results), and the page-locked host-to-device copy rate
    of the snapshots with nothing else running.  (An event recorded on the copy stream
    after the streamed call returns does not mark its last copy: the call enqueues more
    launches than CUDA's launch queue holds, so it returns near the end of the step.)"""
    import torch

    def ev():
        return torch.cuda.Event(enable_timing=True)

    n_part, n_steps = w.n_particles, w.n_steps
    res = {}
    # 1. no copies: after a streamed step every slot holds its snapshot (periodic sequence)
    barrier()
    a, b = ev(), ev()
    a.record(stream)
    pool.c.count = 0
    api.fte_tally_reset(tally)
    api.fte_inject(pool, ring_bg, w.inject, n_part, tally, id_base=id_base, check_failed=False)
    api.fte_advance_streamed(pool, ring_bg, sstream, w.params, tally, 0, n_steps, wsp)
    b.record(stream)
    barrier()
    ms = a.elapsed_time(b)
    res["streamed_no_copy"] = {"value": int(tally.ledger_n.cpu().numpy()[6]) / (ms / 1e3), "ms": ms}
    # 2. a step with every snapshot copied
    a, b = ev(), ev()
    a.record(stream)
    pool.c.count = 0
    sstream.slots[:] = -1
    api.fte_tally_reset(tally)
    sstream.load(0)
    api.fte_inject(pool, ring_bg, w.inject, n_part, tally, id_base=id_base, check_failed=False)
    api.fte_advance_streamed(pool, ring_bg, sstream, w.params, tally, 0, n_steps, wsp)
    b.record(stream)
    barrier()
    ms = a.elapsed_time(b)
    res["streamed_with_copies"] = {"value": int(tally.ledger_n.cpu().numpy()[6]) / (ms / 1e3), "ms": ms}
    # 3. the snapshot copies alone, one after another on the copy stream; the host's time to
    # issue them tells whether the copies ran asynchronously (a copy from memory that is not
    # page-locked, or one the driver stages, returns only when done and keeps the host from
    # enqueuing the compute meanwhile)
    sstream.slots[:] = -1
    barrier()
    a, b = ev(), ev()
    a.record(sstream.copy_stream)
    t0 = time.perf_counter()
    for u in range(w.grid.n_snap):
        sstream.load(u)
    host_ms = (time.perf_counter() - t0) * 1e3
    b.record(sstream.copy_stream)
    barrier()
    ms = a.elapsed_time(b)
    res["h2d_copies_alone"] = {"gbs": w.grid.n_snap * api.fte_snapshot_bytes(ring_bg) / (ms / 1e3) / 1e9,
                               "ms": ms, "host_issue_ms": host_ms,
                               "host_buffer_page_locked": bool(sstream.host.is_pinned())}
    return res


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2404_12164_gb300 import api, build
    from paper_2404_12164_gb300 import _abi as A
    from paper_2404_12164_gb300 import dist as pdist

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w, fields = build_workload()
    w.params.sort_every = args.sort_every
    n_part, n_steps = w.n_particles, w.n_steps
    stream = torch.cuda.current_stream()

    host = torch.from_numpy(np.ascontiguousarray(fields)).pin_memory()
    src = api.Background(w.grid)               # FP32 cell records, as uploaded from the host
    bg = src if args.layout == "cell" else api.Background(w.grid, layout=args.layout)
    pool = api.Particles(n_part)
    tally = api.Tally(w.observers)
    wsp = api.Workspace()
    wsp.ensure(api.fte_workspace_bytes(bg, tally, n_part, min(CHUNK, n_steps)))
    id_base = pdist.id_base(rank, n_part)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def one_step():
        """inject + advance (chunked calls) + tally reduction over ranks."""
        pool.c.count = 0
        api.fte_tally_reset(tally)
        api.fte_inject(pool, bg, w.inject, n_part, tally, id_base=id_base, check_failed=False)
        for c in range(0, n_steps, CHUNK):
            api.fte_advance(pool, bg, w.params, tally, c, min(c + CHUNK, n_steps), wsp)
        pdist.reduce_tally(tally)

    def upload():
        """host snapshots -> device, converted to the measured record layout"""
        api.fte_load_background(src, host)
        if bg is not src:
            api.fte_quantize_background(bg, src)

    # device-resident arm ------------------------------------------------------
    upload()
    torch.cuda.synchronize()

    def measure(background, steps, warmup, clocks=None):
        """W warm-up + K timed steps on `background`; returns (ms, step-kernel launch intervals
        of this rank, alive particle-steps of this rank).  The library records a CUDA event pair
        around every step-kernel launch on the stream of that launch (fte_probe_step_timing)."""
        nonlocal bg
        saved, bg = bg, background
        for _ in range(warmup):
            one_step()
        done = 0
        barrier()
        api.fte_probe_step_timing(1 << 16)
        if clocks:
            clocks.start()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            one_step()
            ln = tally.ledger_n.cpu().numpy()
            done += int(ln[6]) // ws
        t1.record(stream)
        barrier()
        if clocks:
            clocks.result = clocks.stop()
        iv = api.fte_probe_step_intervals(1 << 16)
        api.fte_probe_step_timing(0)
        bg = saved
        ms = t0.elapsed_time(t1)
        (ms,) = pdist.max_over_ranks([ms], device="cuda")
        return ms, iv, done

    clocks = Clocks(local)
    ms, intervals, steps_total = measure(bg, args.steps, args.warmup, clocks)
    cl = clocks.result
    total_steps = steps_total * ws
    value = total_steps / (ms / 1e3)
    S_f32 = api.fte_tally(tally, 0, A.FTE_TALLY_S)

    # tally error: relative standard error of the observer's total occupancy, by batch means
    # over the 32 particle-id classes; the per-step figure sqrt(sum S2) / sum S treats a
    # particle's consecutive steps inside the observer as independent and understates it
    S = api.fte_tally(tally, 0, A.FTE_TALLY_S)
    S2 = api.fte_tally(tally, 0, A.FTE_TALLY_S2)
    _, rel_err = tally.batch_means(0)
    rel_err_per_step = math.sqrt(S2.sum()) / S.sum() if S.sum() > 0 else None

    # end-to-end arm: host buffers through the C ABI ---------------------------
    # The snapshots stream from page-locked host memory into a ring of one slot per
    # snapshot of the periodic sequence (fte_advance_streamed): every step starts with
    # empty slots, so each snapshot is copied once per step, overlapped with the steps
    # of the earlier intervals; the tally and ledger are read back at the end.
    out_host = np.zeros((w.observers[0].ne, w.observers[0].nt))
    ring_bg = api.Background(w.grid, ring=w.grid.n_snap, layout=args.layout)
    sstream = api.SnapshotStream(ring_bg, host)
    plan = api.fte_stream_plan(ring_bg, w.params, 0, n_steps)
    h2d_bytes = ring_uploads(plan, w.grid.n_snap, w.grid.n_snap, w.grid.periodic) * api.fte_snapshot_bytes(ring_bg)
    wsp.ensure(api.fte_workspace_bytes(ring_bg, tally, n_part, n_steps))

    def e2e_step():
        pool.c.count = 0
        sstream.slots[:] = -1
        api.fte_tally_reset(tally)
        sstream.load(0)                # the injection reads snapshot 0
        api.fte_inject(pool, ring_bg, w.inject, n_part, tally, id_base=id_base, check_failed=False)
        api.fte_advance_streamed(pool, ring_bg, sstream, w.params, tally, 0, n_steps, wsp)
        pdist.reduce_tally(tally)
        h = api.fte_tally(tally, 0, A.FTE_TALLY_S)
        out_host[:] = h
        return api.fte_ledger(tally)

    for _ in range(1):
        e2e_step()
    barrier()
    e0 = time.perf_counter()
    e_steps = 0
    for _ in range(args.steps):
        lw, ln = e2e_step()
        e_steps += int(ln[6]) // (ws if ws > 1 else 1)
    barrier()
    e_s = time.perf_counter() - e0
    (e_s,) = pdist.max_over_ranks([e_s], device="cuda")
    e2e_value = e_steps * ws / e_s
    e2e_parts = e2e_breakdown(api, pool, ring_bg, sstream, w, tally, wsp, id_base, stream, barrier)
    del sstream, ring_bg
    torch.cuda.empty_cache()

    # ceilings of the memory levels that serve the gathers (measured in this run)
    l1 = l1_probe()
    l2_gbs = l2_probe()
    # reduced-precision storage forms (same workload, background quantized on the device)
    forms = {}
    if not args.no_forms:
        for dt in ("bf16", "f16"):
            bh = api.Background(w.grid, dtype=dt, layout=args.layout)
            api.fte_quantize_background(bh, src)
            f_ms, f_iv, f_steps = measure(bh, args.steps, max(1, args.warmup // 3))
            Sh = api.fte_tally(tally, 0, A.FTE_TALLY_S)
            _, f_rel = tally.batch_means(0)
            forms[dt] = {"value": f_steps * ws / (f_ms / 1e3), "unit": UNIT,
                         "speedup_vs_f32": (f_steps / f_ms) / (steps_total / ms),
                         "roofline": roofline_record(f_iv, f_steps, ALG_BYTES // 2, l1, None,
                                                      measured_traffic(args.layout, dt)),
                         "tally_total_rel_diff_vs_f32": float(abs(Sh.sum() - S_f32.sum()) / S_f32.sum()),
                         "tally_rel_err": f_rel,
                         "stated_storage_error": dict(STORAGE_ERROR[dt], **STORAGE_ERROR_COMMON),
                         "background_bytes": int(bh.nbytes)}
            del bh
            torch.cuda.empty_cache()

    adjoint = None
    if not args.no_adjoint:
        adjoint = adjoint_times(api, bg, w, n_part, args.adj_slice, args.checkpoint_every, args.sort_every)
        adjoint["note"] = ("first %d of the workload's %d steps, E^-3 injection over 50 keV-5 MeV, smoothed "
                           "intensity at 1 au (E_c 100 keV, t_c %.0f s)" % (min(args.adj_slice, n_steps), n_steps,
                                                                          adjoint["t_c"]))

    roofline = roofline_record(intervals, total_steps // ws, ALG_BYTES, l1, l2_gbs, measured_traffic(args.layout))
    # our kernels per timed step: inject, and per advance call the two normalisation
    # kernels and the step table, then per launch chunk the step kernel, (with the
    # shared-memory tally) the partial-histogram reduction and (with reordering) the
    # five sort kernels
    # a pool of at least one wave of threads (at most 3 blocks of 256 per SM) is advanced as
    # two halves, each with its own reordering and launches (global tally, reordering on)
    wave = torch.cuda.get_device_properties(local).multi_processor_count * 3 * 256
    halves = 2 if (w.params.sort_every > 0 and w.params.tally_layout == "global" and n_part >= wave) else 1

    def kernels_per_call(s):
        chunk = min(w.params.sort_every, CHUNK) if w.params.sort_every > 0 else CHUNK
        per_chunk = 1 + (1 if w.params.tally_layout == "shared" else 0) + (5 if w.params.sort_every > 0 else 0)
        return 3 + math.ceil(s / chunk) * per_chunk * halves
    launches_per_step = 1 + sum(kernels_per_call(min(CHUNK, n_steps - c)) for c in range(0, n_steps, CHUNK))
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "cir_uniform_1e6: synthetic CIR 512x60x180 grid, 24 hourly snapshots, "
                               "1e6 protons at 50 keV in div V<0 cells (1-2 au, 90+-2 deg, w=1/r^2), "
                               "QLT D_mumu q=5/3 H=0.05 lambda_par=0.1 au, dt=10 s x 34560 (4 days), "
                               "1 au box tally 16x144",
                   "particles_per_gpu": n_part, "steps_per_particle": n_steps, "record_layout": args.layout,
                   "background_bytes": int(bg.nbytes), "l2": "inputs larger than L2 (background %.1f GB)" % (bg.nbytes / 1e9),
                   "tally_rel_err": rel_err,
                   "tally_rel_err_method": "relative standard error of the 1 au observer's total occupancy from "
                                           "32 batch means over particle-id classes (id mod 32)",
                   "tally_rel_err_per_step": rel_err_per_step,
                   "tally_rel_err_per_step_note": "sqrt(sum S2)/sum S counts every tallied step as an "
                                                  "independent event; a particle's consecutive steps in the "
                                                  "observer are correlated, so it understates the error"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d_bytes),
                "d2h_bytes_per_step": int(out_host.nbytes + 2 * 8 * A.FTE_LEDGER),
                "path": "fte_advance_streamed, %d-slot ring, each snapshot copied once per step" % w.grid.n_snap,
                "of_value": e2e_value / value, "breakdown": e2e_parts},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "clocks": cl,
        "forms": forms,
        "adjoint": adjoint,
    }
    if ws == 1 and not args.no_ensemble:
        # the 64-set ensemble on the same background (one GPU only)
        eclk = Clocks(local)
        eclk.start()
        result["ensemble"] = ensemble_measure(api, args, bg)
        result["ensemble"]["clocks"] = eclk.stop()
    if ws == 1 and not args.no_amr:
        # the block-AMR workload (the largest single-GPU configuration), one GPU only
        aclk = Clocks(local)
        result["amr"] = amr_measure(api, args, l1=l1, forms=False, cpu=rank == 0 and not args.no_cpu_baseline,
                                    clocks=aclk)
        result["amr"]["clocks"] = aclk.result
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, fields, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# oracle arms (host cores)
# ---------------------------------------------------------------------------
def _oracle_sample(w, fields, n_sample, n_steps=None, threads=None):
    from oracle import oracle as O
    bg = O.grid_background(w.grid, fields)
    ids = np.arange(n_sample, dtype=np.uint32)
    P, led = O.inject(bg, w.inject, ids)
    T = O.Tally(w.observers)
    t = time.perf_counter()
    O.advance(bg, w.params, P, 0, n_steps or w.n_steps, tally=T, ledger=led, threads=threads)
    el = time.perf_counter() - t
    return int(led.as_dict()["n"][6]), el


def cpu_baseline(w, fields, budget_s=20.0):
    from oracle import oracle as O
    threads = O.lib().or_max_threads()
    # calibrate on a tiny sample, then size the sample to ~budget_s of CPU work
    s0, e0 = _oracle_sample(w, fields, 200, threads=threads)
    rate = s0 / max(e0, 1e-6)
    n = int(max(200, min(200_000, 200 * budget_s / max(e0, 1e-3))))
    steps, el = _oracle_sample(w, fields, n, threads=threads)
    return {"value": steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} of the workload's 1e6 particles over the full 4 days "
                      f"({steps} alive particle-steps, {el:.1f} s)"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    w, fields = build_workload()
    threads = O.lib().or_max_threads()
    n_sample = int(os.environ.get("FTE_REF_SAMPLE", "5000"))
    for _ in range(args.warmup):
        _oracle_sample(w, fields, max(50, n_sample // 20), threads=threads)
    total, el = 0, 0.0
    for _ in range(args.steps):
        s, e = _oracle_sample(w, fields, n_sample, threads=threads)
        total += s
        el += e
    v = total / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "cir_uniform_1e6 (sampled: first %d particles per step, full 4 days)" % n_sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_sample} particles x 4 days per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_profile_case(args):
    """Small case of the same kernels for ncu captures: the full-resolution CIR grid with two
    snapshots (884 MB of cell records, 1.5 GB of pair records: larger than L2), 2^18 particles,
    a few launches of 256 steps, in the record layout of --layout."""
    import torch
    from paper_2404_12164_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    if args.grid == "amr":
        # block-AMR form of the same: base 16x4x8 blocks of 16^3 cells, 3 levels (3,872 leaves,
        # 4.3 GB for two snapshots)
        from fte_inputs.amr import AmrSpec
        spec = AmrSpec(nbr=16, nbt=4, nbp=8, bsize=16, levels=3, n_snap=2, dt_snap=3600.0)
        w = configs.cir_amr_1e7(n_particles=1 << 18, n_steps=256 * args.launches, spec=spec)
        w.params.sort_every = args.sort_every
        bg, leaves = build_amr_background(w, api)
        if args.layout != "cell" or args.dtype != "f32":
            cell = bg
            bg = api.AmrBackground(w.grid, leaves, dtype=args.dtype, share=cell, layout=args.layout)
            api.fte_quantize_background(bg, cell)
            torch.cuda.synchronize()
            del cell
    else:
        w = configs.scaled(configs.cir_uniform_1e6(), n_snap=2, n_particles=args.profile_particles)
        w.params.sort_every = args.sort_every
        bg = device_background(api, w, configs.build_background(w), args.layout, args.dtype)
    if args.no_obs:
        w.observers = []
    if args.profile_adjoint:
        # the adjoint's kernels on the same small case: forward and reverse over the launches'
        # steps (E^-3 injection, smoothed intensity at the middle of the run), no checks
        res = adjoint_times(api, bg, w, w.n_particles, 256 * args.launches, args.checkpoint_every,
                            args.sort_every, fd=False)
        print(json.dumps({"case": "profile", "grid": args.grid, "dtype": args.dtype, "adjoint": True,
                          **{k: res[k] for k in ("particles", "steps", "alive_particle_steps", "plain_s",
                                                 "adjoint_forward_s", "adjoint_forward_reverse_s",
                                                 "adj_over_fwd")}}))
        return
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, w.n_particles, tally)
    wsp = api.Workspace()
    wsp.ensure(api.fte_workspace_bytes(bg, tally, w.n_particles, 256))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for c in range(args.launches):
        api.fte_advance(pool, bg, w.params, tally, 256 * c, 256 * (c + 1), wsp)
    e1.record()
    lw, ln = api.fte_ledger(tally)
    torch.cuda.synchronize()
    per_step = ALG_BYTES if args.dtype == "f32" else ALG_BYTES // 2
    print(json.dumps({"case": "profile", "grid": args.grid, "dtype": args.dtype, "launches": args.launches,
                      "particles": w.n_particles, "observers": len(w.observers),
                      "particle_steps": int(ln[6]), "alg_bytes": int(ln[6]) * per_step,
                      "rate": int(ln[6]) / (e0.elapsed_time(e1) / 1e3)}))


def build_amr_background(w, api, device="cuda"):
    """Leaves and FP32 fields of a block-AMR workload, generated on the device straight into
    the background buffer; then the lookup table and ghost layers (fte_amr_prepare)."""
    import torch
    from fte_inputs import amr
    from fte_inputs.grid import REC
    spec = w.grid
    leaves = amr.build_leaves(spec, amr.divv_refiner_batched(spec, w.amr_divv, device=device))
    bg = api.AmrBackground(spec, leaves, device=device)
    P = spec.bsize + 2
    view = bg.dev.view(spec.n_snap, len(leaves), P, P, P, REC)
    view.zero_()
    amr.fields_batched(spec, leaves, device=device, out=view)
    api.fte_amr_prepare(bg)
    torch.cuda.synchronize()
    return bg, leaves


def amr_measure(api, args, l1=None, forms=True, cpu=True, clocks=None):
    """Block-AMR workload (cir_amr_1e7): FP32 rate with its roofline and batch-means tally
    errors at the 4 observers, optionally the BF16/FP16 forms and the oracle on a bounded
    sample; returns a dict."""
    import torch
    from paper_2404_12164_gb300 import _abi as A
    w = configs.cir_amr_1e7(n_particles=args.amr_particles, n_steps=args.amr_steps)
    w.params.sort_every = args.sort_every
    t_gen = time.perf_counter()
    bg, leaves = build_amr_background(w, api)
    t_gen = time.perf_counter() - t_gen
    n_part, n_steps = w.n_particles, w.n_steps
    stream = torch.cuda.current_stream()
    pool = api.Particles(n_part)
    tally = api.Tally(w.observers)
    wsp = api.Workspace()
    wsp.ensure(api.fte_workspace_bytes(bg, tally, n_part, min(CHUNK, n_steps)))
    alg = ALG_BYTES + 4                  # + the 4-byte finest-level table entry
    if l1 is None:
        l1 = l1_probe()

    def one_step(b):
        pool.c.count = 0
        api.fte_tally_reset(tally)
        api.fte_inject(pool, b, w.inject, n_part, tally, check_failed=False)
        for c in range(0, n_steps, CHUNK):
            api.fte_advance(pool, b, w.params, tally, c, min(c + CHUNK, n_steps), wsp)

    def measure(b, steps, warmup, clk=None):
        for _ in range(warmup):
            one_step(b)
        torch.cuda.synchronize()
        api.fte_probe_step_timing(1 << 16)
        if clk:
            clk.start()
        done = 0
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            one_step(b)
            done += int(tally.ledger_n.cpu().numpy()[6])
        t1.record(stream)
        torch.cuda.synchronize()
        if clk:
            clk.result = clk.stop()
        iv = api.fte_probe_step_intervals(1 << 16)
        api.fte_probe_step_timing(0)
        ms = t0.elapsed_time(t1)
        errs = [tally.batch_means(o)[1] for o in range(len(w.observers))]
        S = np.array([tally.classes(o).sum() for o in range(len(w.observers))])
        return ms, iv, done, S, errs

    layout = getattr(args, "layout", "cell")
    bm = bg
    if layout != "cell":
        bm = api.AmrBackground(w.grid, leaves, share=bg, layout=layout)
        api.fte_quantize_background(bm, bg)
    ms, iv, done, S, errs = measure(bm, args.steps, args.warmup, clocks)
    if bm is not bg:
        del bm
        torch.cuda.empty_cache()
    out_forms = {}
    if forms:
        for dt in ("bf16", "f16"):
            bh = api.AmrBackground(w.grid, leaves, dtype=dt, share=bg, layout=layout)
            api.fte_quantize_background(bh, bg)
            f_ms, f_iv, f_done, Sh, f_errs = measure(bh, args.steps, max(1, args.warmup // 3))
            out_forms[dt] = {"value": f_done / (f_ms / 1e3), "unit": UNIT,
                             "speedup_vs_f32": (f_done / f_ms) / (done / ms),
                             "roofline": roofline_record(f_iv, f_done, ALG_BYTES // 2 + 4, l1, None, None),
                             "tally_total_rel_diff_vs_f32": [float(abs(a - b) / b) if b > 0 else None
                                                             for a, b in zip(Sh, S)],
                             "tally_rel_err": f_errs,
                             "background_bytes": int(bh.nbytes)}
            del bh
            torch.cuda.empty_cache()
    lv = np.bincount(leaves[:, 0], minlength=w.grid.levels)
    res = {
        "value": done / (ms / 1e3), "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "dtype": "f32",
        "config": {"workload": "cir_amr_1e7: synthetic CIR on a log-r 3-level block-AMR grid (16^3 blocks, "
                               "base 32x8x24, refined where |div V| > 6e-5/s), 2 hourly snapshots, "
                               f"{n_part:.0e} protons E^-3 over 50 keV-5 MeV injected over one CIR's spiral band "
                               "(phi + (r - 0.1 au) Omega/U within +-10 deg of its compression boundary) from "
                               "0.12 to 2 au at 90+-2 deg, w=1/r^2, "
                               f"QLT q=5/3 H=0.05 lambda_par=0.1 au, dt=2 s x {n_steps}, "
                               "4 observer boxes (0.5, 1, 1.5, 1.8 au) 16x144",
                   "leaves": int(len(leaves)), "leaves_per_level": lv.tolist(), "record_layout": layout,
                   "background_bytes": int(bg.nbytes), "generate_s": t_gen,
                   "l2": "inputs larger than L2 (background %.1f GB)" % (bg.nbytes / 1e9),
                   "tally_rel_err": errs,
                   "tally_rel_err_method": "per observer: relative standard error of the total occupancy from "
                                           "32 batch means over particle-id classes"},
        "roofline": roofline_record(iv, done, alg, l1, None,
                                    measured_traffic(layout, "amr_f32") if layout == "cell" else None),
        "forms": out_forms,
    }
    if cpu:
        res["cpu_baseline"] = amr_cpu_baseline(w, bg, leaves, budget_s=args.cpu_budget / 2)
    del bg
    torch.cuda.empty_cache()
    return res


def amr_cpu_baseline(w, bg, leaves, budget_s=10.0):
    """The FP64 oracle on the host cores over a bounded sample of the AMR workload: the first
    1e4 particles for as many of the workload's steps as fit the budget (a host copy of the
    lattices)."""
    from oracle import oracle as O
    from fte_inputs.grid import REC
    spec = w.grid
    P_ = spec.bsize + 2
    fields = bg.dev.view(spec.n_snap, len(leaves), P_, P_, P_, REC).cpu().numpy()
    obg = O.amr_background(spec, leaves, fields)
    threads = O.lib().or_max_threads()
    n = 10_000
    P, led = O.inject(obg, w.inject, np.arange(n, dtype=np.uint32))
    t = time.perf_counter()
    O.advance(obg, w.params, P.copy(), 0, 20, threads=threads)
    per_step = (time.perf_counter() - t) / 20
    steps = int(max(20, min(w.n_steps, budget_s / max(per_step, 1e-6))))
    led = O.Ledger()
    t = time.perf_counter()
    O.advance(obg, w.params, P, 0, steps, ledger=led, threads=threads)
    el = time.perf_counter() - t
    done = int(led.as_dict()["n"][6])
    return {"value": done / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} of the workload's particles over its first {steps} steps "
                      f"({done} alive particle-steps, {el:.1f} s)"}


def run_amr_case(args):
    """Block-AMR workload (cir_amr_1e7): FP32, BF16 and FP16 storage, one line of JSON."""
    import torch
    from paper_2404_12164_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    clocks = Clocks(0)
    res = amr_measure(api, args, forms=not args.no_forms, cpu=not args.no_cpu_baseline, clocks=clocks)
    print(json.dumps({"case": "amr", "metric": METRIC, "n_gpus": 1, "higher_is_better": True,
                      "data": "synthetic", **res, "clocks": clocks.result}), flush=True)


def run_slices_case(args):
    """Rate of the benchmark workload per slice of --slice-steps steps: one pass (inject + 4 days)
    with CUDA events around each fte_advance call of one slice, after one untimed pass; shows how
    the rate follows the number of alive particles as absorption empties the pool."""
    import torch
    from paper_2404_12164_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    w, fields = build_workload()
    w.params.sort_every = args.sort_every
    bg = device_background(api, w, fields, args.layout)
    del fields
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers)
    wsp = api.Workspace()
    wsp.ensure(api.fte_workspace_bytes(bg, tally, w.n_particles, args.slice_steps))
    S = args.slice_steps

    def one_pass(record):
        pool.c.count = 0
        api.fte_tally_reset(tally)
        api.fte_inject(pool, bg, w.inject, w.n_particles, tally, check_failed=False)
        out, prev = [], 0
        for c in range(0, w.n_steps, S):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            api.fte_advance(pool, bg, w.params, tally, c, min(c + S, w.n_steps), wsp)
            e1.record()
            if record:
                torch.cuda.synchronize()
                done = int(tally.ledger_n.cpu().numpy()[6])
                out.append({"first_step": c, "steps": min(S, w.n_steps - c), "particle_steps": done - prev,
                            "ms": e0.elapsed_time(e1)})
                prev = done
        torch.cuda.synchronize()
        return out

    one_pass(False)
    sl = one_pass(True)
    for x in sl:
        x["alive_mean"] = x["particle_steps"] / x["steps"]
        x["rate"] = x["particle_steps"] / (x["ms"] / 1e3)
    tot_ms = sum(x["ms"] for x in sl)
    print(json.dumps({"case": "slices", "workload": "cir_uniform_1e6", "slice_steps": S,
                      "rate": sum(x["particle_steps"] for x in sl) / (tot_ms / 1e3),
                      "note": "rate of the slices' sum; one fte_advance call per slice, so every slice ends "
                              "with both half-pools joined",
                      "slices": sl}), flush=True)


def run_ensemble_case(args):
    """Ensemble workload (cir_ensemble_64) on its own: see ensemble_measure."""
    import torch
    from paper_2404_12164_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    w0, fields = build_workload()
    bg = device_background(api, w0, fields, args.layout)
    del fields
    print(json.dumps(ensemble_measure(api, args, bg)), flush=True)


def ensemble_measure(api, args, bg):
    """Ensemble workload (cir_ensemble_64): 64 parameter sets with uneven counts on the
    cir_uniform_1e6 background `bg`.  Three arms on the same particles: the single-set kernel run
    set after set; the ensemble kernel with the default launch configuration; the autotuned
    configuration replayed as one CUDA graph."""
    import torch
    w = configs.cir_ensemble_64(n_steps=args.ens_steps)
    w.params.sort_every = args.sort_every
    sets, n_steps, n_tot = w.sets, w.n_steps, w.n_particles
    side = torch.cuda.Stream()
    pool = api.Particles(n_tot)
    tally = api.Tally(w.observers, n_sets=len(sets))
    ws = api.Workspace()
    ws.ensure(max(api.fte_workspace_bytes_batched(bg, tally, n_tot, n_steps),
                  api.fte_workspace_bytes(bg, api.Tally(w.observers), n_tot, n_steps)))
    torch.cuda.synchronize()

    def timed(fn, count, steps, warmup):
        """Rate and time per step of `fn`; every step repeats the same work, so the alive
        particle-steps of the last one (`count`, read after the timed region) times the
        number of steps is the total."""
        for _ in range(warmup):
            fn()
        side.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):
            e0.record(side)
            for _ in range(steps):
                fn()
            e1.record(side)
        side.synchronize()
        done = count() * steps
        return done / (e0.elapsed_time(e1) / 1e3), e0.elapsed_time(e1) / steps

    def ensemble_count():
        return int(tally.ledger_n.cpu().numpy()[6])

    # arm 1: the single-set kernel, set after set (each set its own pool and tally)
    sub_pools = [api.Particles(s.count) for s in sets]
    sub_tallies = [api.Tally(w.observers) for _ in sets]
    set_params = [dataclasses.replace(w.params, lambda_par=s.lambda_par, q=s.q, H=s.H, eps=s.eps, seed=s.seed,
                                      set_id=s.set_id) for s in sets]

    def plain_step():
        for s, sub, tl, prm in zip(sets, sub_pools, sub_tallies, set_params):
            sub.c.count = 0
            api.fte_tally_reset(tl, stream=side)
            api.fte_inject(sub, bg, s.inject, s.count, tl, id_base=0, check_failed=False, stream=side)
            api.fte_advance(sub, bg, prm, tl, 0, n_steps, ws, stream=side)

    def plain_count():
        return sum(int(tl.ledger_n.cpu().numpy()[6]) for tl in sub_tallies)
    with torch.cuda.stream(side):
        plain_rate, plain_ms = timed(plain_step, plain_count, args.ens_timed, 1)
    side.synchronize()
    rel_plain = [e for e in (tl.batch_means(0)[1] for tl in sub_tallies) if e is not None]
    del sub_pools, sub_tallies
    torch.cuda.empty_cache()

    # arm 2: ensemble kernel, default configuration, eager calls
    def batched_step(cfg=None):
        pool.c.count = 0
        api.fte_tally_reset(tally, stream=side)
        api.fte_inject_batched(pool, bg, sets, tally, stream=side)
        api.fte_advance_batched(pool, bg, w.params, sets, tally, 0, n_steps, ws, config=cfg, stream=side)
    with torch.cuda.stream(side):
        eager_rate, eager_ms = timed(batched_step, ensemble_count, args.ens_timed, 1)

    # arm 3: autotune on one pass, then capture one pass into a graph and replay it
    with torch.cuda.stream(side):
        pool.c.count = 0
        api.fte_tally_reset(tally, stream=side)
        api.fte_inject_batched(pool, bg, sets, tally, stream=side)
        best, tried = api.fte_autotune_batched(pool, bg, w.params, sets, tally, 0, n_steps, ws, stream=side)
        side.synchronize()
        g = api.Graph()
        with g.capture(side):
            batched_step(best)
        graph_rate, graph_ms = timed(lambda: g.launch(side), ensemble_count, args.ens_timed, 1)
    # per-set tally errors by batch means over the 32 particle-id classes (graph arm's last step)
    rel = [e for e in (tally.batch_means(0, set=k)[1] for k in range(len(sets))) if e is not None]
    counts = [s.count for s in sets]
    del g, pool, tally, ws
    torch.cuda.empty_cache()
    return {
        "case": "ensemble", "metric": METRIC, "value": graph_rate, "unit": UNIT, "n_gpus": 1,
        "steps": args.ens_timed, "warmup": 1, "ms_per_step": graph_ms, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"cir_ensemble_64: cir_uniform_1e6 background, {len(sets)} parameter sets "
                               "(lambda_par log-U[0.05,1] au, H U[0.01,0.2], E_inj log-U[20,200] keV), "
                               f"{n_tot:.0e} protons (counts {min(counts)}-{max(counts)}), dt=10 s x {n_steps}, "
                               "per-set 1 au box tallies 16x144",
                   "sort_every": w.params.sort_every, "record_layout": args.layout,
                   "tally_rel_err_median": float(np.median(rel)) if rel else None,
                   "tally_rel_err_method": "per set: relative standard error of the 1 au total occupancy from 32 "
                                           "batch means over particle-id classes; median over the sets with hits",
                   "sets_with_hits": len(rel)},
        "arms": {"single_set_kernel_set_after_set": {"value": plain_rate, "ms_per_step": plain_ms,
                                                     "tally_rel_err_median": float(np.median(rel_plain))
                                                     if rel_plain else None},
                 "ensemble_kernel_default_config": {"value": eager_rate, "ms_per_step": eager_ms},
                 "ensemble_kernel_autotuned_graph": {"value": graph_rate, "ms_per_step": graph_ms,
                                                     "config": best}},
        "speedup_vs_single_set_kernel": graph_rate / plain_rate,
        "autotune": [{"config": c, "rate": r} for c, r in tried],
    }


ADJ_OBS = dict(r_o=1.0, sigma_r=0.02, e_c=0.1, sigma_lnE=0.1, t_c=2 * 86400.0, sigma_t=3600.0)


def batch_sigma(x, nb=32):
    """Standard error of sum(x) over particles from the sums of nb classes of particle index
    (batch means: particles are independent, so the class sums are independent)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.bincount(np.arange(len(x)) % nb, weights=x, minlength=nb)
    return float(math.sqrt(nb * s.var(ddof=1)))


def adjoint_times(api, bg, w, n_part, n_steps, K, sort_every, reps=1, fd=True, fd_names=("lambda_par", "q", "H"),
                  fd_rel=2e-2):
    """Times of the plain step kernel, of the adjoint's forward pass and of forward + reverse on
    the same particles (1e6-style power-law injection of the CIR workload); with `fd` a check of
    each gradient in fd_names against central differences (fd_rel of the parameter) of the
    forward pass with common random numbers, both with batch-means standard errors over 32
    particle-index classes, and the pathwise-only total (score window 0) beside them."""
    import torch
    inj = dataclasses.replace(w.inject, energy="powerlaw", e1=0.05, e2=5.0, gamma=3.0)
    # a run shorter than the observable's time centre looks at its middle instead
    t_c = min(ADJ_OBS["t_c"], 0.5 * n_steps * w.params.dt)
    obs = configs.SmoothObserver(**{**ADJ_OBS, "t_c": t_c})
    prm = dataclasses.replace(w.params, sort_every=sort_every)
    pool = api.Particles(n_part)
    tally = api.Tally(w.observers)
    ws = api.Workspace()
    adj = api.Adjoint(bg, prm, obs, 0, n_steps, K)
    stream = torch.cuda.current_stream()

    def inject():
        pool.c.count = 0
        api.fte_tally_reset(tally)
        api.fte_inject(pool, bg, inj, n_part, tally, id_base=0, check_failed=False)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    def plain():
        inject()
        for c in range(0, n_steps, CHUNK):
            api.fte_advance(pool, bg, prm, tally, c, min(c + CHUNK, n_steps), ws)

    t_plain = timed(plain)
    alive_steps = int(tally.ledger_n.cpu().numpy()[6])

    def fwd():
        inject()
        adj.forward(pool)

    def fwd_rev():
        fwd()
        adj.reverse(pool, inj)

    t_fwd = timed(fwd)
    t_adj = timed(fwd_rev)
    out = {"particles": n_part, "steps": n_steps, "checkpoint_every": K, "t_c": t_c, "alive_particle_steps": alive_steps,
           "plain_s": t_plain, "adjoint_forward_s": t_fwd, "adjoint_forward_reverse_s": t_adj,
           "adj_over_fwd": t_adj / t_plain, "J": float(adj.out[0]),
           "grad": dict(zip(api.GRAD_NAMES, adj.out[1:].cpu().numpy().tolist())),
           "estimator": "pathwise, with the steps whose pitch-angle Gaussian reaches mu = 0 in score form "
                        "(window %s widths)" % ("4" if prm.dmumu != "iso" else "0")}
    if fd:
        def per_particle(a):
            inject()
            a.forward(pool)
            _, pp = a.reverse(pool, inj, per_particle=True)
            return pp.double().cpu().numpy()

        pp = per_particle(adj)
        pw = per_particle(api.Adjoint(bg, prm, dataclasses.replace(obs, lr_window=0.0), 0, n_steps, K, ws=adj.ws))
        checks = {}
        for nm in fd_names:
            col = 1 + list(api.GRAD_NAMES).index(nm)
            v0 = getattr(prm, nm)
            h = fd_rel * v0
            Js = []
            for v in (v0 + h, v0 - h):
                a2 = api.Adjoint(bg, dataclasses.replace(prm, **{nm: v}), obs, 0, n_steps, K, ws=adj.ws)
                inject()
                Js.append(a2.forward(pool, per_particle=True)[1].cpu().numpy())
            fdp = (Js[0] - Js[1]) / (2 * h)
            d, sd = float(fdp.sum()), batch_sigma(fdp)
            g, sg = float(pp[:, col].sum()), batch_sigma(pp[:, col])
            g0, sg0 = float(pw[:, col].sum()), batch_sigma(pw[:, col])
            comb = math.sqrt(sd * sd + sg * sg)
            checks[nm] = {"central_difference": d, "central_difference_sigma": sd, "adjoint": g, "adjoint_sigma": sg,
                          "rel_diff": abs(d - g) / abs(d) if d else None,
                          "diff_in_sigma": abs(d - g) / comb if comb > 0 else None,
                          "pathwise_only": g0, "pathwise_only_sigma": sg0,
                          "pathwise_only_diff_in_sigma": abs(d - g0) / math.sqrt(sd * sd + sg0 * sg0)
                          if sd > 0 or sg0 > 0 else None}
        out["fd_check"] = {"step": f"{fd_rel:g} of each parameter, common random numbers",
                           "sigma": "batch means over 32 particle-index classes", "params": checks}
    return out


def run_adjoint_case(args):
    """Adjoint workload: the cir_uniform_1e6 background and transport, 1e6 protons with an E^-3
    spectrum over 50 keV - 5 MeV, gradients of the smoothed 1 au intensity (E_c = 100 keV,
    sigma_lnE = 0.1, t_c = 2 d, sigma_t = 1 h, sigma_r = 0.02 au) with respect to lambda_par, q, H
    and the injection index; checkpoints every 256 steps.  Reports the plain step kernel's time,
    the adjoint's forward + reverse time, their ratio, and central-difference checks of
    dJ/dlambda_par, dJ/dq and dJ/dH with common random numbers."""
    import torch
    from paper_2404_12164_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    w, fields = build_workload()
    bg = device_background(api, w, fields, args.layout)
    del fields
    res = adjoint_times(api, bg, w, args.adj_particles, args.adj_steps, args.checkpoint_every, args.sort_every,
                        reps=args.steps, fd=True)
    print(json.dumps({
        "case": "adjoint", "metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"cir_uniform_1e6 background and transport, {args.adj_particles:.0e} protons E^-3 "
                               f"over 50 keV-5 MeV, dt=10 s x {args.adj_steps}, smoothed 1 au intensity (E_c 100 keV, "
                               "sigma_lnE 0.1, t_c 2 d, sigma_t 1 h, sigma_r 0.02 au)"},
        "forward_plain_kernel": {"value": res["alive_particle_steps"] / res["plain_s"], "s": res["plain_s"]},
        "adjoint_forward_pass": {"value": res["alive_particle_steps"] / res["adjoint_forward_s"],
                                 "s": res["adjoint_forward_s"]},
        "adjoint_forward_plus_reverse": {"value": res["alive_particle_steps"] / res["adjoint_forward_reverse_s"],
                                         "s": res["adjoint_forward_reverse_s"]},
        "adj_over_fwd": res["adj_over_fwd"], "J": res["J"], "grad": res["grad"], "estimator": res["estimator"],
        "fd_check": res["fd_check"],
    }), flush=True)


def ring_uploads(plan, R, n_snap, periodic, group_runs=8):
    """Snapshot copies of one streamed step: the injection snapshot, then the library's rule.
    Runs are taken in groups (1, 1, 2, 4, then `group_runs` runs per advance call) whose
    snapshots fit the ring with one slot to spare (R >= 3); each group's snapshots are
    brought in, and after its launches the next group's snapshots are prefetched into the
    slots the group does not use; a slot holding the snapshot (for a periodic sequence, the
    same snapshot of another period) is not copied again."""
    slots = [-1] * R
    n = 0

    def ensure(u, busy=(), prefetch=False):
        nonlocal n
        k = u % R
        if slots[k] == u:
            return
        if periodic and slots[k] >= 0 and slots[k] % n_snap == u % n_snap:
            slots[k] = u
            return
        if prefetch and k in busy:
            return
        slots[k] = u
        n += 1

    def lo(key):
        return int(key) if key >= 0 else -1 - int(key)

    def hi(key):
        return int(key) + 1 if key >= 0 else -1 - int(key)

    ensure(0)
    keys = [int(key) for _, _, key in plan]
    span_max = R - 1 if R >= 3 else R
    groups, k = [], 0
    while k < len(keys):
        gi = len(groups)
        want = 1 if gi < 2 else (2 if gi == 2 else (4 if gi == 3 else group_runs))
        k1, ulo, uhi = k + 1, lo(keys[k]), hi(keys[k])
        while k1 < len(keys) and k1 - k < want:
            lo2, hi2 = min(ulo, lo(keys[k1])), max(uhi, hi(keys[k1]))
            if hi2 - lo2 + 1 > span_max:
                break
            ulo, uhi, k1 = lo2, hi2, k1 + 1
        groups.append((ulo, uhi))
        k = k1
    for gi, (ulo, uhi) in enumerate(groups):
        busy = {u % R for u in range(ulo, uhi + 1)}
        for u in range(ulo, uhi + 1):
            ensure(u)
        if gi + 1 < len(groups):
            nlo, nhi = groups[gi + 1]
            for nx in range(max(nlo, uhi + 1), nhi + 1):
                if not periodic and nx > n_snap - 1:
                    break
                ensure(nx, busy, True)
    return n


def run_stream_case(args):
    """The cir_uniform_1e6 workload with only `--ring` snapshot slots on the device: the 24 hourly
    snapshots stay in page-locked host memory (FP32 cell records) and are copied into their slots
    as the 4 days advance (each copy overlapped with the previous interval's steps; pair-layout
    or 16-bit slots are filled through a staging snapshot converted on the device).  Reports the
    streamed and the fully resident rates on the same particles in the same storage
    (`--layout`, `--stream-dtype`), and the host-to-device copy bandwidth measured beside them."""
    import torch
    from paper_2404_12164_gb300 import api, build
    build.build()
    torch.cuda.set_device(0)
    w, fields = build_workload()
    w.params.sort_every = args.sort_every
    host = torch.from_numpy(np.ascontiguousarray(fields)).pin_memory()
    n_part, n_steps = w.n_particles, w.n_steps
    dtype, layout = args.stream_dtype, args.layout
    pool = api.Particles(n_part)
    tally = api.Tally(w.observers)
    ws = api.Workspace()
    stream = torch.cuda.current_stream()

    def timed(step, reps, warmup):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        for _ in range(reps):
            step()
            done += int(tally.ledger_n.cpu().numpy()[6])
        e1.record(stream)
        torch.cuda.synchronize()
        return done / (e0.elapsed_time(e1) / 1e3), e0.elapsed_time(e1) / reps

    ring_bg = api.Background(w.grid, dtype=dtype, ring=args.ring, layout=layout)
    st = api.SnapshotStream(ring_bg, host)
    snap = api.fte_snapshot_bytes(ring_bg)

    # host-to-device bandwidth of whole-snapshot copies on the copy stream, into the staging
    # buffer or a slot (nothing runs beside them)
    flat = host.view(torch.uint8).view(-1)
    dst = st.staging if st.staging is not None else ring_bg.dev.view(torch.uint8)[:snap]
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st.copy_stream):
        c0.record(st.copy_stream)
        for k in range(8):
            dst[:snap].copy_(flat[k * snap:(k + 1) * snap], non_blocking=True)
        c1.record(st.copy_stream)
    torch.cuda.synchronize()
    h2d_gbs = 8 * snap / (c0.elapsed_time(c1) / 1e3) / 1e9
    st.slots[:] = -1                   # the probe overwrote slot contents

    def streamed():
        pool.c.count = 0
        api.fte_tally_reset(tally)
        st.load(0)                     # the injection reads snapshot 0 (slot 0)
        api.fte_inject(pool, ring_bg, w.inject, n_part, tally, check_failed=False)
        api.fte_advance_streamed(pool, ring_bg, st, w.params, tally, 0, n_steps, ws)

    v_str, ms_str = timed(streamed, args.steps, 1)
    ring_bytes = int(ring_bg.nbytes) + (st.staging.numel() if st.staging is not None else 0)
    del st, ring_bg
    torch.cuda.empty_cache()
    res_bg = device_background(api, w, host, layout, dtype)

    def resident():
        pool.c.count = 0
        api.fte_tally_reset(tally)
        api.fte_inject(pool, res_bg, w.inject, n_part, tally, check_failed=False)
        for c in range(0, n_steps, CHUNK):
            api.fte_advance(pool, res_bg, w.params, tally, c, min(c + CHUNK, n_steps), ws)

    v_res, ms_res = timed(resident, args.steps, 1)
    plan = api.fte_stream_plan(res_bg, w.params, 0, n_steps)
    uploads = ring_uploads(plan, args.ring, w.grid.n_snap, w.grid.periodic)
    print(json.dumps({
        "case": "stream", "metric": METRIC, "value": v_str, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "ms_per_step": ms_str, "higher_is_better": True, "dtype": dtype, "data": "synthetic",
        "config": {"workload": "cir_uniform_1e6 with %d resident snapshot slots (24 hourly snapshots in "
                               "page-locked host memory), %s %s records" % (args.ring, dtype, layout),
                   "device_background_bytes": ring_bytes, "resident_background_bytes": int(res_bg.nbytes),
                   "snapshot_uploads_per_step": uploads, "h2d_bytes_per_step": int(uploads * snap)},
        "h2d_gbs": h2d_gbs,
        "resident": {"value": v_res, "ms_per_step": ms_res},
        "streamed_over_resident": v_str / v_res,
    }), flush=True)


def l1_probe(kib=64, records=4096, reps=5, spreads=(1, 2, 4, 8, 32)):
    """Delivered GB/s of the transport kernel's record loads (ld.global.nc.v8 x 2 + v2, 72 B
    per record) from an L1-resident buffer of FP32 cell records, for several numbers of
    distinct records per warp (`spread`); best of reps each.  Returns {spread: GB/s}."""
    import torch
    from paper_2404_12164_gb300 import api
    from paper_2404_12164_gb300 import _abi as A
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    threads = sms * 2048
    buf = torch.rand(kib * 1024 // 4, dtype=torch.float32, device="cuda")
    out = torch.empty(threads, dtype=torch.float32, device="cuda")
    res = {}
    for sp in spreads:
        api.fte_probe_gather_l1(buf, threads, 64, sp, out)
        best = 0.0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            api.fte_probe_gather_l1(buf, threads, records, sp, out)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, threads * records * (A.FTE_NFIELD * 4) / (e0.elapsed_time(e1) / 1e3) / 1e9)
        res[sp] = best
    return res


def union_ms(iv):
    """Length of the union of [start, end] intervals (ms)."""
    if len(iv) == 0:
        return 0.0
    iv = iv[np.argsort(iv[:, 0])]
    tot, cs, ce = 0.0, iv[0, 0], iv[0, 1]
    for s, e in iv[1:]:
        if s > ce:
            tot += ce - cs
            cs, ce = s, e
        else:
            ce = max(ce, e)
    return tot + (ce - cs)


def roofline_record(intervals, particle_steps, alg_per_step, l1, l2_gbs, traffic):
    """Roofline of the step kernel over the timed region from its recorded launches: the
    algorithmic bytes of all launches over the time the kernel ran (the union of its launch
    intervals; the two half-pool streams overlap), in units of one launch."""
    hbm, hbm_kind = _peaks()
    n = len(intervals)
    u = union_ms(intervals)
    alg = particle_steps * alg_per_step
    achieved = alg / (u / 1e3) / 1e9 if u > 0 else None
    peak = max(l1.values()) if l1 else None
    durs = intervals[:, 1] - intervals[:, 0] if n else np.zeros(0)
    return {"bound": "l1", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved and peak else None,
            "traffic": traffic["dram_bytes_per_particle_step"] * particle_steps / n if traffic and n else None,
            "traffic_source": (traffic["source"] + ": DRAM bytes per alive particle-step of the profile case x "
                               "this run's particle-steps per launch") if traffic else None,
            "kernel": "advance_kernel", "alg_bytes_per_particle_step": alg_per_step,
            "alg_bytes_per_launch": alg / n if n else None,
            "kernel_launches": n, "kernel_ms_total": float(durs.sum()), "kernel_ms_union": u,
            "kernel_ms_mean_launch": float(durs.mean()) if n else None,
            "peak_source": "L1 probe of the step kernel's record loads (fte_probe_gather_l1, 64 KiB of records, "
                           "best over lane spreads), measured in this run",
            "l1_probe_gbs_by_spread": {str(k): v for k, v in l1.items()},
            "l1_wavefronts": traffic.get("l1") if traffic else None,
            "hbm": {"peak": hbm, "peak_source": f"{hbm_kind} hbm_gbs (MEASURED_PEAKS.json)",
                    "frac": achieved / hbm if achieved else None},
            "l2_random_sector_gbs": l2_gbs,
            "frac_of_l2": achieved / l2_gbs if achieved and l2_gbs else None}


def l2_probe(mib=64, threads=152 * 2048, loads=256, reps=5):
    """Random 32-byte sector read bandwidth of an L2-resident buffer (GB/s), best of reps."""
    import torch
    from paper_2404_12164_gb300 import api
    buf = torch.ones(mib * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    out = torch.empty(threads, dtype=torch.float32, device="cuda")
    api.fte_probe_sectors(buf, threads, 8, out)
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        api.fte_probe_sectors(buf, threads, loads, out)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, threads * loads * 32 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="bench",
                    choices=["bench", "profile", "amr", "ensemble", "adjoint", "stream", "slices"])
    ap.add_argument("--slice-steps", type=int, default=1024, help="steps per slice of --case slices")
    ap.add_argument("--ring", type=int, default=3, help="resident snapshot slots of --case stream")
    ap.add_argument("--stream-dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="storage of the slots (and of the resident comparison) of --case stream")
    ap.add_argument("--adj-particles", type=int, default=1_000_000)
    ap.add_argument("--adj-steps", type=int, default=34_560)
    ap.add_argument("--checkpoint-every", type=int, default=256)
    ap.add_argument("--ens-steps", type=int, default=2160)
    ap.add_argument("--ens-timed", type=int, default=2)
    ap.add_argument("--amr-particles", type=int, default=10_000_000)
    ap.add_argument("--amr-steps", type=int, default=1800)
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--grid", default="uniform", choices=["uniform", "amr"], help="grid of --case profile")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"], help="storage of --case profile")
    ap.add_argument("--profile-particles", type=int, default=1 << 18, help="particles of --case profile")
    ap.add_argument("--no-obs", action="store_true", help="--case profile without observers")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="--case profile: time the adjoint's forward and reverse passes instead")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--layout", default="cell", choices=["cell", "pair"],
                    help="record layout of the device background (pair: a cell and its r-neighbour per record)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-amr", action="store_true", help="leave the block-AMR workload out of the default line")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="leave the 64-set ensemble workload out of the default line")
    ap.add_argument("--adj-slice", type=int, default=34_560,
                    help="steps of the adjoint measurement in the default run (default: the whole 4 days)")
    ap.add_argument("--sort-every", type=int, default=64,
                    help="steps between spatial reorderings of the alive particles (0: off)")
    args = ap.parse_args()
    if args.case == "profile":
        run_profile_case(args)
    elif args.case == "amr":
        run_amr_case(args)
    elif args.case == "ensemble":
        run_ensemble_case(args)
    elif args.case == "slices":
        run_slices_case(args)
    elif args.case == "adjoint":
        run_adjoint_case(args)
    elif args.case == "stream":
        run_stream_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
