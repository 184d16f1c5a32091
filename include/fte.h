/*
 * fte.h - C ABI of the GB300 focused-transport particle pusher.
 *
 * The library integrates the focused transport equation (Husidic et al. 2024,
 * Sec. 2.1, Eq. 1) for independent pseudo-particles as Ito stochastic
 * differential equations forward in time, with the coefficients of Eq. 2 (dx/dt),
 * Eq. 3 (dmu/dt) and Eq. 4 (dp/dt), pitch-angle diffusion D_mumu (Eq. 5 or the
 * quasi-linear form of Sec. 2.1), optional cross-field diffusion (lambda_perp,
 * Sec. 2.1), through gridded solar-wind snapshots that are located, read and
 * interpolated trilinearly at every step (Sec. 2.4), with injection per Eq. 7
 * and occupancy tallies of the intensity (Sec. 3, Figs. 5-8).
 *
 * Conventions
 *   - Units: lengths au, times s, speeds au/s, B nT, energies MeV, momentum
 *     p in units of m_p c.  Cartesian frame: z = rotation axis, theta
 *     colatitude, phi longitude in [0, 2 pi).
 *   - Memory: every pointer named "dev" / documented DEVICE is device memory
 *     owned by the caller (the Python binding allocates it with PyTorch).  The
 *     library allocates no device memory and keeps no state between calls, with
 *     one exception: fte_advance_noalloc's statically placed 24 MiB scratch
 *     array (present on every device that loads the library) and the device
 *     address of it that the library looks up once per device.
 *     Pointers documented HOST are host memory owned by the caller.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *     work is enqueued asynchronously on it unless the call says it synchronises.
 *   - Errors: every call returns an fte_status, and fte_last_error() returns a
 *     message (thread-local, valid until the next call on the same thread).  No
 *     C++ exception crosses the ABI.  Argument errors are found before anything
 *     is enqueued, so the caller's buffers are unchanged.  A CUDA error returned
 *     by a launch, copy or event call (FTE_ECUDA) can come after part of the
 *     call's work was enqueued; that work stays enqueued, a call that forked a
 *     second stream (the half-pools of fte_advance and of the adjoint passes) has
 *     not joined it back, and, as after any CUDA error, the context may be
 *     unusable.
 *   - Random numbers: one Philox4x32-10 block (Salmon et al. 2011) per particle
 *     and step, key (seed, set_id), counter (step, particle id, tag, 0); tag 0
 *     transport, tag 1 injection draw, tag 2 injection position attempt.
 *   - Time: step n is at t_n = t0 + n dt.  Time bin of an event at t:
 *     floor(((t - t_lo) * nt) / (t_hi - t_lo)), evaluated in double precision.
 */
#ifndef FTE_H
#define FTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FTE_ABI_VERSION 3
#define FTE_NFIELD 18          /* stored fields per cell */
#define FTE_NCLASS 32          /* particle-id classes of the class-resolved tally S_class */
#define FTE_REC 24             /* floats per stored cell record (96 bytes) */
#define FTE_HREC 32            /* 16-bit values per reduced-precision cell record (64 bytes) */
#define FTE_HHDR 32            /* floats of the per-field scale header of a reduced-precision background */
#define FTE_MAX_OBS 8          /* observers per tally */
#define FTE_LEDGER 8           /* ledger slots */
#define FTE_MAX_SETS 64        /* parameter sets per ensemble call */

typedef enum fte_status {
    FTE_OK = 0,
    FTE_EINVAL = 1,    /* invalid argument (null pointer, bad size, bad range) */
    FTE_ENOMEM = 2,    /* a caller buffer is too small */
    FTE_ECUDA = 3,     /* a CUDA runtime call failed */
    FTE_ERANGE = 4,    /* injection found no acceptable position for some particles */
    FTE_ENOTSUP = 5    /* configuration outside what this build supports */
} fte_status;

/* particle status codes (uint8 per particle) */
enum { FTE_ALIVE = 0, FTE_ABS_INNER = 1, FTE_ABS_OUTER = 2, FTE_ABS_THETA = 3,
       FTE_DEAD_NAN = 4, FTE_INJ_FAIL = 5 };
/* ledger slots: weight (double) and count (uint64) per slot
   0 injected; 1 absorbed at r_min; 2 absorbed at r_max; 3 absorbed at a theta
   face; 4 non-finite state; 5 failed injections (count); 6 alive particle-steps
   (count); 7 tally events inside an observer but outside its E/t range (count) */

/* ---------------------------------------------------------------------------
 * Background: spherical grid of cell-centred snapshots (Sec. 2.2-2.4).
 * Cell k along an axis spans faces edge_k .. edge_{k+1}; r faces are uniform
 * (radial = 0) or geometric (radial = 1, the radially stretched grid of Sec. 4);
 * theta faces uniform on [th_min, th_max]; phi uniform and periodic on [0, 2 pi).
 * Record layout (24 floats, 96 bytes): 0-2 B, 3-5 V, 6-14 dV_i/dx_j (row i =
 * component), 15-17 d|B|/dx_j, 18-23 unused.  Array order [snap][phi][theta][r][FTE_REC],
 * so the two r-neighbours of a cell are one contiguous, 32-byte aligned 192-byte read.
 * Snapshot s holds the fields at t_snap0 + s dt_snap; between snapshots the
 * fields are interpolated linearly in time and dV/dt gains (V_{s+1}-V_s)/dt_snap;
 * periodic != 0 wraps the sequence; otherwise the fields are frozen (and
 * dV/dt = 0) before the first and from the last snapshot on.
 *
 * Reduced precision (dtype FTE_BF16 / FTE_F16): the device array starts with a
 * header of FTE_HHDR floats whose first 18 are per-field scales s_f (the largest
 * |value| of field f over all cells and snapshots, 1 for an all-zero field),
 * followed by records of FTE_HREC 16-bit values holding round-to-nearest-even
 * (v_f / s_f) (the quotient rounded to float first), slots 18-31 zero.  The
 * field used by the transport is the stored value times s_f.  Such arrays are
 * produced on the device by fte_quantize_background (or copied in ready-made).
 * ------------------------------------------------------------------------- */
enum { FTE_F32 = 0, FTE_BF16 = 1, FTE_F16 = 2 };
/* Record layout.  FTE_LAYOUT_CELL: one record per cell as above.  FTE_LAYOUT_PAIR:
   record k holds the fields of cell k and of its upper r-neighbour k + 1 (zero
   for the last cell of an r-row): FP32 40 floats (160 bytes: 0-17 cell k,
   18-35 cell k + 1, 36-39 zero), 16-bit 48 values (96 bytes: 0-17, 18-35, then
   zero), so that the two r-neighbours of a corner pair are one 32-byte aligned
   read of five (FP32) or three (16-bit) sectors instead of six or four. */
enum { FTE_LAYOUT_CELL = 0, FTE_LAYOUT_PAIR = 1 };
typedef struct fte_grid {
    int32_t nr, nth, nph;      /* cells per axis, each >= 2 */
    int32_t radial;            /* 0 linear, 1 logarithmic */
    double r_min, r_max;       /* au, 0 < r_min < r_max; absorbing faces */
    double th_min, th_max;     /* rad, 0 <= th_min < th_max <= pi; absorbing faces */
    int32_t n_snap;            /* >= 1 */
    int32_t periodic;
    double t_snap0, dt_snap;   /* s; dt_snap > 0 when n_snap > 1 */
    int32_t dtype;             /* FTE_F32, FTE_BF16 or FTE_F16 */
    int32_t amr_levels;        /* 0: uniform grid; 1..4: block AMR with this many levels */
    int32_t amr_bsize;         /* AMR: cells per block edge B (nr, nth, nph multiples of B) */
    int32_t n_leaves;          /* AMR: number of leaf blocks */
    int32_t ring;              /* 0: all n_snap snapshots resident; 2 .. n_snap: the device
                                  array holds `ring` snapshot slots, snapshot u (counted in
                                  time order, periodic sequences unwrapped) in slot u mod ring,
                                  filled on demand by fte_advance_streamed (any dtype and
                                  layout: host snapshots are FP32 cell records) */
    int32_t layout;            /* FTE_LAYOUT_CELL or FTE_LAYOUT_PAIR (see below) */
} fte_grid;

/* Block AMR (Sec. 2.4, Fig. 4): nr x nth x nph are the base-level (level 0) cells,
   split into blocks of B^3 cells; a block of level l is halved in every direction
   to give 8 blocks of level l+1; touching leaves (faces, edges, corners) differ by
   at most one level.  Leaf n is (level, bi, bj, bk): block indices at its own
   level.  Fields: [snap][leaf][B+2][B+2][B+2] records (phi, theta, r order) - the
   leaf's cells with a one-cell ghost layer that fte_amr_prepare fills from the
   neighbours (same level: copy; finer: trilinear interpolation of the finer
   lattice at the ghost centre; coarser: of the coarser lattice, where a coarser
   lattice cell covered by finer leaves takes the interpolation of the finer
   lattice at its centre; outside the domain in r and theta: the nearest
   interior cell; phi periodic), so that every point of a leaf interpolates
   trilinearly on the leaf's padded lattice. */
typedef struct fte_background {
    fte_grid grid;
    const float* fields;       /* DEVICE, fte_background_bytes(&grid) bytes, 32-byte aligned */
    const int32_t* leaves;     /* AMR: DEVICE [n_leaves][4] (level, bi, bj, bk) */
    int32_t* table;            /* AMR: DEVICE, fte_amr_table_bytes(&grid) bytes: the leaf
                                  covering each finest-level block, built by fte_amr_prepare */
} fte_background;

/* Bytes of the device array holding all snapshots of `g` (0 if g is invalid). */
size_t fte_background_bytes(const fte_grid* g);

/* Validate `g` and copy `host_fields` (HOST, fte_background_bytes(g) bytes, in
   the record layout above; page-locked memory makes the copy asynchronous) to
   `dev_fields` (DEVICE, 32-byte aligned, at least that many bytes).  EINVAL on an invalid grid or
   null pointer, ENOMEM if dev_bytes is too small, ECUDA if the copy fails. */
fte_status fte_load_background(const fte_grid* g, const float* host_fields, void* dev_fields,
                               size_t dev_bytes, void* stream);

/* Bytes of the finest-level lookup table of an AMR grid (0 if not AMR or invalid). */
size_t fte_amr_table_bytes(const fte_grid* g);

/* AMR set-up, once per background after its interior cells and leaves are on the
   device (FP32 fields): builds bg->table, checks that the leaves tile the domain
   without overlap and with 2:1 nesting (EINVAL otherwise; this check
   synchronises `stream`), then fills the ghost layer of every leaf and snapshot
   in bg->fields.  A 16-bit copy is then made with fte_quantize_background.  For
   a ring background in 16-bit or pair storage only the table is built (its
   slots are filled, ghosts included, as snapshots stream in). */
fte_status fte_amr_prepare(const fte_background* bg, void* stream);

/* Convert an FP32 cell-layout background to the storage form of `g_half`: a
   16-bit dtype (FTE_BF16 or FTE_F16: per-field scales and rounded records) and/or
   the pair layout; the other fields give the geometry of both arrays.
   `dev_f32` (DEVICE, the FP32 cell-layout array of the same geometry; for AMR
   after fte_amr_prepare) is read and `dev_out` (DEVICE, 32-byte aligned,
   out_bytes >= fte_background_bytes(g_half)) receives the converted array.
   EINVAL if g_half is FP32 with the cell layout.  Asynchronous on `stream`. */
fte_status fte_quantize_background(const fte_grid* g_half, const float* dev_f32, void* dev_out,
                                   size_t out_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Particle pool: structure of arrays in DEVICE memory, `capacity` entries each.
 * `count` (host field) is the number of entries in use; fte_inject appends.
 * ------------------------------------------------------------------------- */
typedef struct fte_particles {
    float *x, *y, *z;          /* position, au (inertial or snapshot frame) */
    float *mu;                 /* pitch-angle cosine in the wind frame */
    float *p;                  /* momentum, m_p c */
    float *w;                  /* statistical weight */
    uint32_t* id;              /* Philox counter word 1 */
    uint8_t* status;           /* FTE_ALIVE ... */
    uint64_t capacity;
    uint64_t count;
} fte_particles;

/* ---------------------------------------------------------------------------
 * Injection (Sec. 2.3, Eq. 7).  region 0: all at the point (r, th, ph); region 1:
 * uniform in volume over r in [r1, r2], cos(theta) between cos th1 and cos th2,
 * phi in [ph1, ph2] (with spiral != 0: the spiral phase phi_hat = phi + spiral
 * (r - spiral_rb) in [ph1, ph2], i.e. a band along an Archimedean spiral such as
 * the CIR region criterion phi_hat = phi + (r - r_B) Omega / U of Sec. 2.3; the
 * volume element is unchanged), optionally accepting only positions whose containing cell
 * of snapshot `divv_snap` (of a ring background: slot `divv_snap`, which the caller
 * must have filled) has stored div V (dV_x/dx + dV_y/dy + dV_z/dz, summed in
 * float in that order) < divv_max, with at most max_tries attempts per particle.
 * energy 0: e0; energy 1: dN/dE ~ E^-gamma on [e1, e2] by inverse CDF.
 * weight 0: 1; weight 1: 1/r^2 (r in au).  mu_mode 0: mu uniform in [-1, 1];
 * 1: mu = mu0.  Particle ids are id_base + index within this call.
 * ------------------------------------------------------------------------- */
typedef struct fte_inject_spec {
    int32_t region, energy, weight, mu_mode;
    double r, th, ph;
    double r1, r2, th1, th2, ph1, ph2;
    int32_t use_divv, divv_snap, max_tries, pad0;
    double divv_max;
    double e0, e1, e2, gamma, mu0;
    uint32_t seed, set_id;
    uint32_t id_base, pad1;
    double spiral;             /* box: rad per au; phi = phi_hat - spiral (r - spiral_rb) */
    double spiral_rb;          /* au */
} fte_inject_spec;

/* ---------------------------------------------------------------------------
 * Transport parameters (Sec. 2.1).
 * dmumu 0 quasi-linear: D = (nu/2)(1-mu^2)(|mu|^(q-1) + H), nu = 3 v I / (2 lambda),
 *         I = int_0^1 (1-mu^2)/(mu^(q-1)+H) dmu; the factor |mu|^(q-2) of dD/dmu
 *         uses max(|mu|, mu_floor)
 *       1 Eq. 5: D = D0 (|mu|/(1+|mu|) + eps)(1-mu^2), D0 = 3 v J / (4 lambda),
 *         J = int_0^1 (1-mu^2)/(mu/(1+mu)+eps) dmu
 *       2 isotropic: D = (v / (2 lambda)) (1-mu^2)
 * lambda = lambda_par (p / p_ref)^alpha when p_ref > 0 and alpha != 0, else lambda_par.
 * Cross-field diffusion kappa_perp = (v lambda_perp / 3)(I - bb) when lambda_perp > 0,
 * with Ito drift div(kappa_perp) when kappa_drift != 0.
 * dvdt_term != 0 keeps the b.dV/dt terms of Eqs. 3-4.
 * p_update 0: p' = p exp(pdot/p dt); 1: p' = p (1 + pdot/p dt).
 * sort_every: see the field; it only changes which thread advances which particle.
 * ------------------------------------------------------------------------- */
typedef struct fte_params {
    int32_t dmumu, p_update, kappa_drift, dvdt_term;
    double lambda_par, p_ref, alpha, q, H, eps, mu_floor, lambda_perp;
    double dt, t0;
    uint32_t seed, set_id;
    int32_t sort_every;        /* > 0: reorder the alive particles by interpolation stencil
                                  (and sign of mu) every sort_every steps (performance
                                  only: results do not depend on it); 0: no reordering */
    int32_t tally_layout;      /* fte_advance: FTE_LAYOUT_GLOBAL (or 0): lanes of a warp in the
                                  same bin are merged and added to the tally with FP64 atomics;
                                  FTE_LAYOUT_SHARED: per-block histograms in shared memory
                                  (at most 16384 bins), reduced after each launch.  The
                                  counts are the same; the sums differ in rounding only */
} fte_params;

/* ---------------------------------------------------------------------------
 * Tallies.  An observer is kind 0 shell |r - r_o| <= dr; kind 1 box additionally
 * |theta - th| <= dth and |phi - ph| <= dph (phi difference wrapped to [-pi, pi]);
 * kind 2 slab |x - r| <= dr; kind 3 ring |r - r_o| <= dr and |theta - th| <= dth,
 * the longitude profile of Figs. 5-7.  Bins: ne logarithmic energy bins on [e_lo, e_hi]
 * (i_E = floor(ne ln(E/e_lo) / ln(e_hi/e_lo))) times nt time bins on [t_lo, t_hi)
 * (ring: nt longitude bins floor(phi nt / 2 pi), counting steps in [t_lo, t_hi)).
 * At every step, the start-of-step state of every alive particle inside an
 * observer adds w dt to S, (w dt)^2 to S2 and 1 to C of its bin (occupancy
 * estimator).  Accumulators are DEVICE arrays over all observers' bins,
 * observer o starting at offset sum_{o' < o} ne*nt, bin index i_E * nt + i_t.
 * ------------------------------------------------------------------------- */
typedef struct fte_observer {
    int32_t kind, ne, nt, pad;
    double r, dr, th, dth, ph, dph;
    double e_lo, e_hi, t_lo, t_hi;
} fte_observer;

typedef struct fte_tally_buf {
    int32_t n_obs;
    int32_t n_sets;                   /* ensembles: one block of bins per parameter set
                                         (0 or 1: a single block); at most FTE_MAX_SETS */
    fte_observer obs[FTE_MAX_OBS];
    double* S;                        /* DEVICE, max(n_sets, 1) * fte_tally_bins() doubles */
    double* S2;                       /* DEVICE, max(n_sets, 1) * fte_tally_bins() doubles */
    unsigned long long* C;            /* DEVICE, max(n_sets, 1) * fte_tally_bins() counts */
    double* ledger_w;                 /* DEVICE, FTE_LEDGER doubles */
    unsigned long long* ledger_n;     /* DEVICE, FTE_LEDGER counts */
    double* S_class;                  /* DEVICE, optional (NULL: not kept): max(n_sets, 1) *
                                         fte_tally_bins() * FTE_NCLASS doubles, [set][bin][class]: S of
                                         the bin from the particles whose id % FTE_NCLASS is `class`,
                                         for batch-means error estimates of bins and observer totals */
} fte_tally_buf;

/* Total bins over all observers of one set (0 if the tally description is invalid). */
size_t fte_tally_bins(const fte_tally_buf* t);

/* Zero S, S2, C of every set, S_class (when kept) and the ledger (asynchronous). */
fte_status fte_tally_reset(const fte_tally_buf* t, void* stream);

/* Scratch (DEVICE) needed by fte_advance on `device` for grid `g`, tally `t`, a
   pool of `n_particles` entries and `n_steps` steps per call: per-block partial
   histograms, launch counters, the per-step time table, the normalisation
   constants and the particle-ordering buffers.  0 on error. */
size_t fte_workspace_bytes(int device, const fte_grid* g, const fte_tally_buf* t,
                           uint64_t n_particles, int64_t n_steps);

/* Append n particles to P (requires P->count + n <= P->capacity) drawn per `spec`
   on the device (Sec. 2.3, Eq. 7), positions in the frame of `bg`.  Adds the
   injected weight to ledger slot 0 and failed injections to slot 5 of t.  On
   success P->count += n.  If n_failed (HOST) is non-NULL the call synchronises
   `stream`, stores the number of particles that found no acceptable position
   (status FTE_INJ_FAIL, weight 0) and returns FTE_ERANGE if it is non-zero. */
fte_status fte_inject(fte_particles* P, const fte_background* bg, const fte_inject_spec* spec,
                      uint64_t n, const fte_tally_buf* t, uint64_t* n_failed, void* stream);

/* Advance every alive particle of P from step n_start to step n_end (Sec. 2.1:
   Euler-Maruyama steps of Eqs. 2-4 with the Ito drift of D_mumu, reflection at
   mu = +-1, exponential momentum update; Sec. 2.4: trilinear interpolation of
   the bracketing snapshots), tallying the start-of-step state of each step into
   t and absorbing particles that leave [r_min, r_max] x [th_min, th_max] (ledger
   slots 1-3).  ws (DEVICE, ws_bytes >= fte_workspace_bytes(device, &bg->grid, t,
   P->count, n_end - n_start)) is scratch; its contents on return are unspecified.
   Asynchronous on `stream`.  With the global tally layout, reordering on and at
   least one wave of threads' worth of particles, the two halves of P are
   advanced concurrently, one on `stream` and one on a stream the call creates,
   forks from `stream` and joins back to it before returning (so all work is
   ordered after earlier and before later work on `stream`); under stream capture
   the call keeps to `stream`. */
fte_status fte_advance(fte_particles* P, const fte_background* bg, const fte_params* prm,
                       const fte_tally_buf* t, int64_t n_start, int64_t n_end, void* ws,
                       size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Snapshot streaming (Sec. 4 names loading only what is needed as the way to cut
 * the cost of whole snapshot files): with grid.ring = R > 0 only R snapshots are
 * resident and fte_advance_streamed moves snapshot files from host memory into
 * their slots as the simulated time reaches them, on a copy stream, overlapped
 * with the steps of earlier intervals (R >= 3: each group of intervals prefetches
 * the next group's snapshots while it computes).
 * ------------------------------------------------------------------------- */

/* Plan of a streamed advance: the steps n_start .. n_end-1 split into runs that
   use the same snapshot pair.  out (HOST, 3 entries per run): first step, end
   step, and the unwrapped index u of the earlier snapshot (the pair u, u+1), or
   -1 - u when the fields are frozen at snapshot u (before the first or from the
   last snapshot of a non-periodic sequence).  *count receives the number of
   runs; ENOMEM if it exceeds max_runs (out then holds the first max_runs). */
fte_status fte_stream_plan(const fte_grid* g, const fte_params* prm, int64_t n_start, int64_t n_end,
                           int64_t* out, int64_t max_runs, int64_t* count);

/* Bytes of one host snapshot: FP32 cell records (96 bytes per cell; AMR: the
   padded leaf lattices, ghost values ignored), the unit fte_advance_streamed copies. */
size_t fte_snapshot_bytes(const fte_grid* g);

/* Bytes of the DEVICE staging buffer that streaming into a ring of `g` needs: 0
   for FP32 cell-layout slots (a snapshot is copied straight into its slot);
   otherwise one host snapshot (fte_snapshot_bytes), into which each snapshot is
   copied and from which it is converted into its slot as fte_quantize_background
   converts a resident background (0 if g is invalid). */
size_t fte_stream_staging_bytes(const fte_grid* g);

/* 16-bit ring backgrounds: set the per-field scale header of bg->fields from all
   n_snap host snapshots (each copied into `staging`, AMR ghost layer refilled,
   largest |value| per field; the scales fte_quantize_background computes for the
   fully resident background of the same snapshots, so the stored values are
   identical).  Once, before the first fte_stream_load or fte_advance_streamed;
   AMR: after fte_amr_prepare.  EINVAL for FP32 backgrounds or a NULL argument,
   ENOMEM if staging_bytes < fte_stream_staging_bytes.  Asynchronous on `stream`. */
fte_status fte_stream_scales(const fte_background* bg, const void* host_snapshots, void* staging,
                             size_t staging_bytes, void* stream);

/* fte_advance over a ring background (grid.ring >= 2): for every run of the
   plan, the snapshots it needs are copied from host_snapshots (HOST, page-locked for overlap: the n_snap snapshots in
   order, each fte_snapshot_bytes(g) bytes of FP32 cell records) into their slots
   on copy_stream - for a 16-bit or pair-layout ring through `staging` (DEVICE,
   32-byte aligned, fte_stream_staging_bytes(g) bytes; may be NULL when that is
   0) and a conversion into the slot; for AMR the ghost cells of a copied
   snapshot are refilled on the device - and the run is advanced on
   compute_stream once its slots are filled; a slot is overwritten only after
   the steps using it are done; a slot already holding the snapshot (periodic
   sequences: the same snapshot of another period) is not copied again, so a
   ring of n_snap slots over a periodic sequence copies each snapshot once.
   slot_state (HOST, ring entries, caller-owned, -1 = empty before the first
   call) records the unwrapped snapshot each slot holds and is updated.  Consecutive
   runs are advanced together, one fte_advance call per group of up to 8 runs
   (ramping 1, 1, 2, 4, 8 from the call's start), as long as a group's snapshots fit
   the ring with one slot to spare (ring >= 3) and its steps fit ws's time table:
   ws as for fte_advance with n_steps at least the longest run of the plan
   (n_end - n_start steps allow full groups).  With ring >= 3, once a group's
   launches are enqueued the next group's snapshots are copied into the slots the
   group does not use, so that the group's compute covers them (also where a
   copy call returns only when done).
   Work of earlier calls on either stream is waited for.  EINVAL/ENOMEM for a
   missing or undersized staging buffer.  Asynchronous. */
fte_status fte_advance_streamed(fte_particles* P, const fte_background* bg, const void* host_snapshots,
                                const fte_params* prm, const fte_tally_buf* t, int64_t n_start, int64_t n_end,
                                int64_t* slot_state, void* staging, size_t staging_bytes, void* ws,
                                size_t ws_bytes, void* compute_stream, void* copy_stream);

/* Copy unwrapped snapshot u (periodic sequences: any u, snapshot u mod n_snap;
   otherwise 0 <= u < n_snap) from host_snapshots into slot u mod ring on
   `stream` (through `staging` as above; AMR: and refill its ghost layer), and
   record it in slot_state, for instance the injection snapshot before
   fte_inject.  Asynchronous. */
fte_status fte_stream_load(const fte_background* bg, const void* host_snapshots, int64_t u, int64_t* slot_state,
                           void* staging, size_t staging_bytes, void* stream);

/* Allocation-free variant of fte_advance (the paper has no counterpart: this is
   an interface for callers that cannot allocate device memory at run time, such
   as a host code whose own allocator owns all of the GPU's memory, or a service
   that must not call cudaMalloc once running).  Same arguments and stream
   semantics as fte_advance, but without the workspace: the scratch is a 24 MiB
   array that the library places in device memory statically, held by every GPU
   that loads the library until the process exits.  It always tallies through
   per-block shared-memory histograms (prm->tally_layout must still be a valid
   value and is otherwise not used) and never reorders the particles
   (prm->sort_every is not used): particle states, ledger and tally counts equal
   those of fte_advance with tally_layout = FTE_LAYOUT_SHARED, tally sums up to
   the order of FP32 partial sums.  The first call on a device (with that device
   current) looks up the array's device address; make that first call before
   any stream capture.  That address belongs to the device's primary context: a
   cudaDeviceReset (or any teardown of that context) invalidates it, after which
   the process must not call this entry point on that device again.  All calls
   share the array: calls whose work overlaps on the GPU race on it.  Returns
   FTE_ENOMEM when the tally's per-block partial histograms (12 bytes per bin) do
   not fit the array for at least one block per SM (about 13,800 bins on a
   152-SM GB300). */
fte_status fte_advance_noalloc(fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_tally_buf* t, int64_t n_start, int64_t n_end, void* stream);

/* ---------------------------------------------------------------------------
 * Ensembles: many parameter sets advanced together (the paper runs one set per
 * simulation; this is a batching of independent runs, Sec. 2.1 per set).
 * The pool holds the sets one after another: set s is the counts[s] entries
 * starting at counts[0] + ... + counts[s-1] (fte_set.count), and the counts
 * add up to P->count.  Set s replaces lambda_par, q, H, eps, seed and set_id of
 * the shared fte_params by its own; the D_mumu model, dt, t0, lambda_perp,
 * p_ref/alpha, toggles and sort_every are shared.  Set s tallies into block s
 * of the accumulators (bin b of set s at s * fte_tally_bins(t) + b; t->n_sets
 * >= n_sets).  A particle of set s follows exactly the trajectory fte_advance
 * gives it with prm carrying set s's values.
 * ------------------------------------------------------------------------- */
typedef struct fte_set {
    double lambda_par, q, H, eps;
    uint32_t seed, set_id;
    uint64_t count;            /* particles of this set in the pool */
} fte_set;

/* Launch configuration of the ensemble step kernel (results do not depend on it). */
enum { FTE_LAYOUT_SHARED = 1, FTE_LAYOUT_GLOBAL = 2 };
typedef struct fte_launch_config {
    int32_t threads;           /* threads per block: 128 or 256 */
    int32_t steps_per_launch;  /* 1 .. 1024 steps per step-kernel launch; with prm->sort_every > 0
                                  the alive particles are reordered before every launch */
    int32_t tally_layout;      /* FTE_LAYOUT_SHARED: every block keeps all sets' bins in shared
                                  memory (n_sets * bins <= 16384 and the block must fit on an SM),
                                  reduced into t after each launch; FTE_LAYOUT_GLOBAL: lanes of a
                                  warp in the same bin are merged and added to t with FP64 atomics */
    int32_t pad;
} fte_launch_config;

/* Scratch (DEVICE) for fte_advance_batched / fte_autotune_batched with any
   launch configuration: grid g, tally t (t->n_sets sets), n_particles pool
   entries, n_steps steps per call.  0 on error. */
size_t fte_workspace_bytes_batched(int device, const fte_grid* g, const fte_tally_buf* t,
                                   uint64_t n_particles, int64_t n_steps);

/* Inject every set of an ensemble: for s = 0 .. n_sets-1, append counts[s]
   particles drawn per specs[s] (HOST arrays) exactly as fte_inject would, with
   ids specs[s].id_base + index within the set.  Asynchronous (failed
   injections are in ledger slot 5).  EINVAL if n_sets is outside
   1..FTE_MAX_SETS, ENOMEM if the pool cannot hold them all. */
fte_status fte_inject_batched(fte_particles* P, const fte_background* bg, const fte_inject_spec* specs,
                              const uint64_t* counts, int n_sets, const fte_tally_buf* t, void* stream);

/* Advance every set of an ensemble from step n_start to n_end in the same
   launches (sets: HOST array of n_sets entries; cfg: HOST, NULL for 256
   threads, prm->sort_every (or 1024) steps per launch and the shared layout
   when it fits, else the global one).  ws (DEVICE, ws_bytes >=
   fte_workspace_bytes_batched(...)) is scratch.  Asynchronous; makes no
   synchronising CUDA call, so it can be captured into a graph. */
fte_status fte_advance_batched(fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_set* sets, int n_sets, const fte_tally_buf* t, int64_t n_start,
                               int64_t n_end, const fte_launch_config* cfg, void* ws, size_t ws_bytes,
                               void* stream);

/* Autotuner of the ensemble launch configuration: advances steps n_start ..
   n_end exactly as fte_advance_batched would (the trajectories and tallies do
   not depend on the configuration), trying in turn every configuration of
   {128, 256 threads} x {32, 64, 128, 256 steps per launch (1024 when
   prm->sort_every == 0)} x {shared layout where it fits, global layout} on
   consecutive slices of the steps, twice (forward, then backward order), and
   stores in *best (HOST) the one with the highest rate of alive particle-steps
   per second (CUDA events on `stream`, which it synchronises).  tried/rates
   (HOST, optional, room for 16 entries) receive every configuration and its
   rate, *n_tried their number.  n_end - n_start must allow at least
   two launches per trial: ENOTSUP otherwise. */
fte_status fte_autotune_batched(fte_particles* P, const fte_background* bg, const fte_params* prm,
                                const fte_set* sets, int n_sets, const fte_tally_buf* t, int64_t n_start,
                                int64_t n_end, void* ws, size_t ws_bytes, fte_launch_config* best,
                                fte_launch_config* tried, double* rates, int* n_tried, void* stream);

/* CUDA graphs of library calls (the paper has no counterpart): fte_graph_begin
   starts capturing `stream` (not the legacy NULL stream; thread-local capture
   mode), every asynchronous fte_* call enqueued on it until fte_graph_end is
   recorded instead of run, and fte_graph_end instantiates the graph into *out
   (a handle the caller owns until fte_graph_destroy).  fte_graph_launch runs
   it on `stream`; it reuses the pointers and sizes of the capture, so every
   buffer the captured calls used must stay allocated and unchanged in size.
   Calls that synchronise (fte_tally with a host buffer, fte_ledger,
   fte_inject with n_failed, fte_autotune_batched) must not be captured. */
typedef struct fte_graph fte_graph;
fte_status fte_graph_begin(void* stream);
fte_status fte_graph_end(void* stream, fte_graph** out);
fte_status fte_graph_launch(const fte_graph* g, void* stream);
fte_status fte_graph_destroy(fte_graph* g);

/* ---------------------------------------------------------------------------
 * Pathwise adjoint: gradients of a smooth observable with respect to the
 * transport parameters, for fitting them to intensities (the paper runs
 * forward simulations only; this differentiates the same Euler-Maruyama map of
 * Sec. 2.1 with every step's Philox noise held fixed).
 * Observable: J = sum_i w_i sum_n dt K(r_n, E_n, t_n) over the alive steps
 * n = n_start .. n_end-1 of every particle (start-of-step state, t_n = t0 + n dt),
 * K = exp(-(r - r_o)^2 / (2 sigma_r^2)) exp(-ln(E / e_c)^2 / (2 sigma_lnE^2))
 *     exp(-(t - t_c)^2 / (2 sigma_t^2)).
 * Gradients (FTE_NGRAD): dJ/dlambda_par, dJ/dq, dJ/dH, dJ/deps (through D_mumu,
 * its mu derivative and the normalisation integral), dJ/dgamma of the injected
 * power law (likelihood ratio of each particle's injected energy).
 * Each step's pitch-angle increment is a Gaussian of mean m = mu + (mudot +
 * dD/dmu) dt and width s = sqrt(2 D dt), reflected at mu = +-1 (Sec. 2.1).  Eq. 5's
 * dD/dmu jumps at mu = 0 and the quasi-linear one is singular there, so the
 * derivative of a realised path misses the part of dE[J]/dtheta carried by
 * paths whose mu passes 0.  Steps whose m lies within lr_window widths of a value
 * that lands at mu = 0 (min(|m|, ||m| - 2|) < lr_window s) therefore enter in the
 * score (likelihood-ratio) form: mu' is held and the derivative of the log of its
 * transition density (with the reflection's images) multiplies the observable
 * accumulated after the step; every other step is differentiated pathwise with its
 * Philox noise held.  The estimate is unbiased for the discretised chain up to the
 * Gaussian tail beyond lr_window widths.  lr_window < 0 selects 4 for Eq. 5 and the
 * quasi-linear form and 0 (pathwise everywhere) for the isotropic form, whose
 * coefficients are smooth in mu.  Other discrete decisions (cell, absorption) are
 * held fixed.
 * Supported: lambda_perp = 0, lambda independent of p (p_ref = 0 or alpha = 0).
 * ------------------------------------------------------------------------- */
#define FTE_NGRAD 5
typedef struct fte_smooth_obs {
    double r_o, sigma_r;       /* au */
    double e_c, sigma_lnE;     /* MeV; natural log */
    double t_c, sigma_t;       /* s */
    double lr_window;          /* widths of the score-form window around mu = 0; < 0: the default */
} fte_smooth_obs;

/* Scratch (DEVICE) for fte_adjoint_forward/reverse: checkpoints every
   `checkpoint_every` steps (20 bytes per particle each), per-particle step
   counts and observables, the replay scratch of the reverse pass (the states
   of one segment: checkpoint_every x 20 bytes per particle, e.g. 5.1 GB for
   1e6 particles and 256 steps), the particle orders of its 64-step chunks and
   the time table.  A pool of at least one wave of the forward kernel's threads
   (reordering on) gets two such regions, one per half of the pool (below).
   0 on error. */
size_t fte_adjoint_workspace_bytes(int device, const fte_grid* g, uint64_t n_particles, int64_t n_steps,
                                   int checkpoint_every);

/* Forward pass: advances P from n_start to n_end exactly as fte_advance would
   (no tally, no ledger), storing checkpoints in ws, and writes J to dev_out[0]
   (DEVICE, 1 + FTE_NGRAD doubles; the rest is zeroed).  dev_J_particle (DEVICE,
   optional, P->count doubles): each particle's J_i.  With reordering on
   (prm->sort_every > 0), a pool of at least one wave of the forward kernel's
   threads is advanced as two halves, each in its own region of ws, on `stream`
   and a second stream forked from and joined back to it (in turn on `stream`
   while it is being captured); every particle's results are those of one pool.
   Asynchronous. */
fte_status fte_adjoint_forward(fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_smooth_obs* obs, int64_t n_start, int64_t n_end, int checkpoint_every,
                               double* dev_out, double* dev_J_particle, void* ws, size_t ws_bytes, void* stream);

/* Reverse pass after fte_adjoint_forward with the same P, bg, prm, obs, steps,
   checkpoint interval and ws: writes the FTE_NGRAD gradients to dev_out[1..].
   Segment by segment from the last, it replays the segment from its checkpoint
   in chunks of 64 steps and then runs the step VJPs backwards over them, with
   the particles reordered by position per chunk (prm->sort_every > 0).
   spec (HOST, optional): the injection that produced P at n_start; with a power
   law (energy 1) the dJ/dgamma entry is filled, otherwise it is 0.
   dev_per_particle (DEVICE, optional, n x (1 + FTE_NGRAD) floats): each
   particle's J_i and gradients.  The pool is split into the same halves as in
   the forward pass.  Asynchronous. */
fte_status fte_adjoint_reverse(const fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_smooth_obs* obs, const fte_inject_spec* spec, int64_t n_start,
                               int64_t n_end, int checkpoint_every, double* dev_out, float* dev_per_particle,
                               void* ws, size_t ws_bytes, void* stream);

/* Tally output kinds for fte_tally(). */
enum { FTE_TALLY_S = 0, FTE_TALLY_S2 = 1, FTE_TALLY_C = 2, FTE_TALLY_INTENSITY = 3 };

/* Write observer `obs`'s [ne][nt] array of `kind` as doubles to dev_out (DEVICE,
   ne*nt doubles).  INTENSITY is j = S v(E_c) / (4 pi V_obs dt_bin dE) with E_c
   the geometric bin centre and V_obs the observer volume (au^3; 2 dr for a slab;
   one longitude bin of a ring, whose dt_bin is the whole window t_hi - t_lo):
   particles / (au^2 s sr MeV) per unit weight.  If host_out (HOST, `bytes` >=
   ne*nt*8) is non-NULL the array is also copied there and the call synchronises
   `stream`. */
fte_status fte_tally(const fte_tally_buf* t, int obs, int kind, double* dev_out, void* host_out,
                     size_t bytes, void* stream);

/* fte_tally for parameter set `set` of an ensemble tally (0 <= set < max(t->n_sets, 1)). */
fte_status fte_tally_set(const fte_tally_buf* t, int set, int obs, int kind, double* dev_out, void* host_out,
                         size_t bytes, void* stream);

/* Green's function to time-dependent source (Sec. 2.3: the particles are all
   injected at t = 0; the solution for a source with a given time profile is the
   convolution of that Green's-function solution with the profile).  For
   observer `obs` of set `set`, with time bins of width dt_b = (t_hi - t_lo)/nt:
   out[e][k] = dt_b * sum_{m=0..k} src[m] X[e][k-m], X the observer's S or
   INTENSITY array (`kind`) and src[m] the source rate (injected populations per
   second) in time bin m (dev_src: DEVICE, nt doubles, or NULL for 1 in every
   bin, so that out[e][k] accumulates towards the steady state of a constant
   source).  dev_out (DEVICE, ne*nt doubles); host_out/bytes as in fte_tally.
   EINVAL for ring observers (their bins are longitudes, not times). */
fte_status fte_tally_convolve(const fte_tally_buf* t, int set, int obs, int kind, const double* dev_src,
                              double* dev_out, void* host_out, size_t bytes, void* stream);

/* Copy the ledger to HOST arrays (FTE_LEDGER entries each); synchronises `stream`. */
fte_status fte_ledger(const fte_tally_buf* t, double* host_w, uint64_t* host_n, void* stream);

const char* fte_last_error(void);
const char* fte_status_string(int status);
int fte_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
