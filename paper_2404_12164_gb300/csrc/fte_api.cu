// C ABI of the focused-transport pusher: argument validation, workspace
// layout and kernel launches.  No device memory is allocated here; every
// buffer comes from the caller.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <mutex>
#include <new>
#include <vector>

#include "fte_kernels.cuh"
#include "fte_probe.h"

using namespace fte;

namespace {

thread_local char g_err[512] = "";

fte_status fail(fte_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

fte_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(FTE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FTE_CUDA(call, what)                      \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

const double kPiD = 3.141592653589793;

fte_status check_grid(const fte_grid* g)
{
    if (!g) return fail(FTE_EINVAL, "grid is NULL");
    if (g->nr < 2 || g->nth < 2 || g->nph < 2) return fail(FTE_EINVAL, "grid needs >= 2 cells per axis");
    if (g->radial != 0 && g->radial != 1) return fail(FTE_EINVAL, "radial must be 0 or 1");
    if (!(g->r_min > 0.0 && g->r_max > g->r_min)) return fail(FTE_EINVAL, "need 0 < r_min < r_max");
    if (!(g->th_min >= 0.0 && g->th_max > g->th_min && g->th_max <= kPiD + 1e-12))
        return fail(FTE_EINVAL, "need 0 <= th_min < th_max <= pi");
    if (g->n_snap < 1) return fail(FTE_EINVAL, "n_snap must be >= 1");
    if (g->n_snap > 1 && !(g->dt_snap > 0.0)) return fail(FTE_EINVAL, "dt_snap must be > 0");
    if (g->dtype != FTE_F32 && g->dtype != FTE_BF16 && g->dtype != FTE_F16)
        return fail(FTE_EINVAL, "dtype must be FTE_F32, FTE_BF16 or FTE_F16");
    if (g->ring != 0 && (g->ring < 2 || g->ring > g->n_snap))
        return fail(FTE_EINVAL, "ring must be 0 or in [2, n_snap]");
    if (g->layout != FTE_LAYOUT_CELL && g->layout != FTE_LAYOUT_PAIR)
        return fail(FTE_EINVAL, "layout must be FTE_LAYOUT_CELL or FTE_LAYOUT_PAIR");
    if (g->amr_levels < 0 || g->amr_levels > 4) return fail(FTE_EINVAL, "amr_levels must be in [0, 4]");
    if (g->amr_levels > 0) {
        const int B = g->amr_bsize;
        if (B < 2 || g->nr % B || g->nth % B || g->nph % B)
            return fail(FTE_EINVAL, "AMR: block size must be >= 2 and divide nr, nth, nph");
        if (g->n_leaves < 1) return fail(FTE_EINVAL, "AMR: n_leaves must be >= 1");
        const double P = B + 2.0;
        if ((double)g->n_leaves * P * P * P > 2.0e9) return fail(FTE_EINVAL, "AMR: too many records per snapshot");
        const double nf = (double)(g->nr / B) * (g->nth / B) * (g->nph / B) * pow(8.0, g->amr_levels - 1);
        if (nf > 2.0e9) return fail(FTE_EINVAL, "AMR: finest-level table too large");
    } else if ((double)g->nr * g->nth * g->nph > 2.0e9) {
        return fail(FTE_EINVAL, "too many cells per snapshot");
    }
    const double cells = (double)g->nr * g->nth * g->nph * g->n_snap;
    if (cells * FTE_REC > 9.0e18 / 4.0) return fail(FTE_EINVAL, "grid too large");
    return FTE_OK;
}

size_t snapshot_records(const fte_grid* g)
{
    if (g->amr_levels > 0) {
        const size_t P = (size_t)g->amr_bsize + 2;
        return (size_t)g->n_leaves * P * P * P;
    }
    return (size_t)g->nr * g->nth * g->nph;
}

// snapshots held on the device: all of them, or the ring's slots
int resident_snapshots(const fte_grid* g) { return g->ring > 0 ? g->ring : g->n_snap; }

size_t grid_records(const fte_grid* g)
{
    return snapshot_records(g) * (size_t)resident_snapshots(g);
}

// bytes of one stored record for the grid's dtype and layout
size_t record_bytes(const fte_grid* g)
{
    const bool pair = g->layout == FTE_LAYOUT_PAIR;
    if (g->dtype == FTE_F32) return (pair ? kPairRec : FTE_REC) * sizeof(float);
    return (pair ? kPairHRec : FTE_HREC) * sizeof(uint16_t);
}

size_t grid_bytes(const fte_grid* g)
{
    const size_t head = g->dtype == FTE_F32 ? 0 : FTE_HHDR * sizeof(float);
    return head + grid_records(g) * record_bytes(g);
}

// cells per r-row of the stored lattice (the pair layout pairs within a row)
int row_cells(const fte_grid* g) { return g->amr_levels > 0 ? g->amr_bsize + 2 : g->nr; }

GridK make_gridk(const fte_background* bg)
{
    const fte_grid& g = bg->grid;
    GridK k;
    k.dtype = g.dtype;
    k.pair = g.layout == FTE_LAYOUT_PAIR ? 1 : 0;
    k.fields = bg->fields;
    k.scale = bg->fields;
    k.hfields = reinterpret_cast<const uint32_t*>(bg->fields + FTE_HHDR);
    k.snap_recs = (long long)snapshot_records(&g);
    k.nr = g.nr; k.nth = g.nth; k.nph = g.nph; k.radial = g.radial;
    k.r_min = (float)g.r_min; k.r_max = (float)g.r_max;
    k.th_min = (float)g.th_min; k.th_max = (float)g.th_max;
    k.cos_th_min = (float)cos(g.th_min); k.cos_th_max = (float)cos(g.th_max);
    if (g.radial) {
        const double dl = log(g.r_max / g.r_min) / g.nr;
        k.dr = (float)dl;
        k.inv_dr = (float)(1.0 / dl);
    } else {
        k.dr = (float)((g.r_max - g.r_min) / g.nr);
        k.inv_dr = (float)(g.nr / (g.r_max - g.r_min));
    }
    k.dth = (float)((g.th_max - g.th_min) / g.nth);
    k.inv_dth = (float)(g.nth / (g.th_max - g.th_min));
    k.inv_dph = (float)(g.nph / (2.0 * kPiD));
    k.inv_dt_snap = g.n_snap > 1 ? (float)(1.0 / g.dt_snap) : 0.f;
    k.amr = g.amr_levels;
    k.B = g.amr_bsize;
    k.P = g.amr_bsize + 2;
    k.L = g.amr_levels > 0 ? g.amr_levels - 1 : 0;
    k.amr_leaves = g.n_leaves;
    if (g.amr_levels > 0) {
        k.nf0 = (g.nr / g.amr_bsize) << k.L;
        k.nf1 = (g.nth / g.amr_bsize) << k.L;
        k.nf2 = (g.nph / g.amr_bsize) << k.L;
    } else {
        k.nf0 = k.nf1 = k.nf2 = 0;
    }
    k.leaves = reinterpret_cast<const int4*>(bg->leaves);
    k.table = bg->table;
    k.inv_lnr = (float)(g.radial ? 1.0 / log(g.r_max / g.r_min) : 1.0 / (g.r_max - g.r_min));
    k.inv_thspan = (float)(1.0 / (g.th_max - g.th_min));
    return k;
}

fte_status check_background(const fte_background* bg)
{
    if (!bg) return fail(FTE_EINVAL, "background is NULL");
    fte_status s = check_grid(&bg->grid);
    if (s != FTE_OK) return s;
    if (!bg->fields) return fail(FTE_EINVAL, "background fields pointer is NULL");
    if ((uintptr_t)bg->fields % 32) return fail(FTE_EINVAL, "background fields must be 32-byte aligned");
    if (bg->grid.amr_levels > 0 && (!bg->leaves || !bg->table || (uintptr_t)bg->leaves % 16))
        return fail(FTE_EINVAL, "AMR background needs 16-byte aligned leaves and a table");
    return FTE_OK;
}

fte_status check_tally(const fte_tally_buf* t, size_t* nbins)
{
    if (!t) return fail(FTE_EINVAL, "tally is NULL");
    if (t->n_obs < 0 || t->n_obs > FTE_MAX_OBS) return fail(FTE_EINVAL, "n_obs must be in [0, %d]", FTE_MAX_OBS);
    if (t->n_sets < 0 || t->n_sets > FTE_MAX_SETS) return fail(FTE_EINVAL, "n_sets must be in [0, %d]", FTE_MAX_SETS);
    size_t nb = 0;
    for (int o = 0; o < t->n_obs; ++o) {
        const fte_observer& ob = t->obs[o];
        if (ob.kind < 0 || ob.kind > 3) return fail(FTE_EINVAL, "observer %d: bad kind", o);
        if (ob.ne < 1 || ob.nt < 1 || ob.nt > 32767) return fail(FTE_EINVAL, "observer %d: bad bin counts", o);
        if (!(ob.e_lo > 0.0 && ob.e_hi > ob.e_lo)) return fail(FTE_EINVAL, "observer %d: need 0 < e_lo < e_hi", o);
        if (!(ob.t_hi > ob.t_lo)) return fail(FTE_EINVAL, "observer %d: need t_lo < t_hi", o);
        if (!(ob.dr >= 0.0)) return fail(FTE_EINVAL, "observer %d: dr < 0", o);
        nb += (size_t)ob.ne * ob.nt;
    }
    if (!t->ledger_w || !t->ledger_n) return fail(FTE_EINVAL, "ledger pointers are NULL");
    if (nb && (!t->S || !t->S2 || !t->C)) return fail(FTE_EINVAL, "tally accumulator pointers are NULL");
    *nbins = nb;
    return FTE_OK;
}

const BatchArgs g_no_batch = {};    // the single-set kernels ignore their ensemble argument

// Kernel-side observers: bins of observer o start at the sum of the earlier observers' bins.
void fill_observers(const fte_tally_buf* t, AdvanceArgs* a)
{
    size_t off = 0;
    for (int o = 0; o < t->n_obs; ++o) {
        const fte_observer& ob = t->obs[o];
        ObsK& k = a->obs[o];
        k.kind = ob.kind; k.ne = ob.ne; k.nt = ob.nt; k.off = (int)off;
        k.r = (float)ob.r; k.dr = (float)ob.dr; k.th = (float)ob.th; k.dth = (float)ob.dth;
        k.ph = (float)ob.ph; k.dph = (float)ob.dph;
        k.e_lo = (float)ob.e_lo; k.ne_over_lnratio = (float)(ob.ne / log(ob.e_hi / ob.e_lo));
        k.phi_scale = (float)(ob.nt / (2.0 * 3.141592653589793));
        off += (size_t)ob.ne * ob.nt;
    }
    a->n_obs = t->n_obs;
    a->cls = t->S_class;
}

// Layout of the fte_advance workspace.
struct WsLayout {
    size_t off_fetch, off_norm, off_npart, off_table, off_part, off_sort, total;
    int blocks;       // resident blocks of the step kernel on the device
    int threads;      // threads per block of its build (advance_threads)
};

constexpr int kMaxSmemBins = 16384;    // 3 x 4 B per bin in shared memory
constexpr long long kChunkSteps = 1024;
constexpr size_t kStreamGroupRuns = 8;   // snapshot intervals per fte_advance call of a streamed run
// Work counters of the step kernel: one per SM range (warp_fetch_sm), for up to 1024 SM ids.
constexpr unsigned kFetchSlots = 1024;
constexpr size_t kFetchBytes = kFetchSlots * sizeof(unsigned long long);

int device_sms(int device)
{
    static int cache[64];
    if (device < 0 || device >= 64) return 0;
    if (!cache[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
        cache[device] = v;
    }
    return cache[device];
}

// shared memory of a single-set step kernel: the partial histogram, or none
size_t single_smem(int mode, size_t nbins)
{
    return mode == kModeSingle ? 3 * sizeof(float) * (nbins ? nbins : 1) : 0;
}

// Reordering scratch of fte_advance: one sort of the whole pool, or, when the pool is
// advanced as two halves on two streams, one sort per half and a second fetch counter.
size_t advance_sort_bytes(const GridK& g, unsigned long long n)
{
    const unsigned long long h = n / 2;
    const size_t one = sort_scratch_bytes(g, n);
    const size_t two = sort_scratch_bytes(g, h) + sort_scratch_bytes(g, n - h) + kFetchBytes;
    return one > two ? one : two;
}

// A second stream and the events that fork it from and join it back to the
// caller's stream; released when the call returns (the device finishes the work).
// Measurement aid (fte_probe_step_timing): a CUDA event before and after every
// step-kernel launch of fte_advance, recorded on the stream of that launch, while
// recording is on (and the stream is not being captured).
struct StepTiming {
    std::atomic<int> on{0};
    std::mutex mu;
    std::vector<cudaEvent_t> ev;    // start, stop of launch i at 2 i, 2 i + 1
    int used = 0;
};
StepTiming g_timing;

cudaError_t launch_advance_timed(const AdvanceArgs& a, int kperp, int mode, int blocks, size_t smem, cudaStream_t s,
                                 bool capturing)
{
    const int nt = advance_threads(kperp, a.g.dtype, mode, a.g.amr > 0);
    if (!g_timing.on.load(std::memory_order_relaxed) || capturing)
        return launch_advance(a, g_no_batch, kperp, mode, nt, blocks, smem, s);
    std::lock_guard<std::mutex> lock(g_timing.mu);
    const bool rec = g_timing.used + 2 <= (int)g_timing.ev.size();
    if (rec) cudaEventRecord(g_timing.ev[g_timing.used], s);
    const cudaError_t e = launch_advance(a, g_no_batch, kperp, mode, nt, blocks, smem, s);
    if (rec) {
        cudaEventRecord(g_timing.ev[g_timing.used + 1], s);
        g_timing.used += 2;
    }
    return e;
}

struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~SideStream()
    {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s) cudaStreamDestroy(s);
    }
};

fte_status layout(int device, int kperp, int dtype, int pair, int amr, int mode, size_t nbins, long long n_steps,
                  size_t sort_bytes, WsLayout* L)
{
    const int sms = device_sms(device);
    if (sms <= 0) return fail(FTE_ECUDA, "cannot query device %d", device);
    const size_t smem = single_smem(mode, nbins);
    int per_sm = 0;
    int cur = 0;
    FTE_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != device) FTE_CUDA(cudaSetDevice(device), "cudaSetDevice");
    L->threads = advance_threads(kperp, dtype, mode, amr);
    cudaError_t e = advance_occupancy(kperp, dtype, mode, L->threads, pair, amr, smem, &per_sm);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(FTE_ENOTSUP, "step kernel does not fit on an SM with %zu bytes of tally", smem);
    L->blocks = sms * per_sm;
    size_t off = 0;
    L->off_fetch = off; off += kFetchBytes;
    L->off_norm = off; off += 64;
    L->off_npart = off; off += kNormPartials * sizeof(double);
    L->off_table = off; off += (size_t)(n_steps > 0 ? n_steps : 1) * sizeof(StepEntry);
    off = (off + 255) & ~(size_t)255;
    L->off_part = off;
    if (mode == kModeSingle) off += (size_t)L->blocks * 3 * (nbins ? nbins : 1) * sizeof(float);
    off = (off + 255) & ~(size_t)255;
    L->off_sort = off; off += sort_bytes;
    L->total = off;
    return FTE_OK;
}

}  // namespace

extern "C" {

const char* fte_last_error(void) { return g_err; }

const char* fte_status_string(int s)
{
    switch (s) {
    case FTE_OK: return "ok";
    case FTE_EINVAL: return "invalid argument";
    case FTE_ENOMEM: return "buffer too small";
    case FTE_ECUDA: return "CUDA error";
    case FTE_ERANGE: return "injection region has no acceptable position";
    case FTE_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

int fte_abi_version(void) { return FTE_ABI_VERSION; }

size_t fte_background_bytes(const fte_grid* g)
{
    if (check_grid(g) != FTE_OK) return 0;
    return grid_bytes(g);
}

fte_status fte_load_background(const fte_grid* g, const float* host_fields, void* dev_fields,
                               size_t dev_bytes, void* stream)
{
    fte_status s = check_grid(g);
    if (s != FTE_OK) return s;
    if (!host_fields || !dev_fields) return fail(FTE_EINVAL, "NULL field pointer");
    if ((uintptr_t)dev_fields % 32) return fail(FTE_EINVAL, "device fields must be 32-byte aligned");
    const size_t need = grid_bytes(g);
    if (dev_bytes < need) return fail(FTE_ENOMEM, "device buffer has %zu bytes, needs %zu", dev_bytes, need);
    FTE_CUDA(cudaMemcpyAsync(dev_fields, host_fields, need, cudaMemcpyHostToDevice, (cudaStream_t)stream),
             "background copy");
    return FTE_OK;
}

size_t fte_amr_table_bytes(const fte_grid* g)
{
    if (check_grid(g) != FTE_OK || g->amr_levels < 1) return 0;
    const int L = g->amr_levels - 1;
    const size_t nf = ((size_t)(g->nr / g->amr_bsize) << L) * ((size_t)(g->nth / g->amr_bsize) << L) *
                      ((size_t)(g->nph / g->amr_bsize) << L);
    return nf * sizeof(int32_t) + 64;   // table, then four status counters
}

fte_status fte_amr_prepare(const fte_background* bg, void* stream)
{
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    if (bg->grid.amr_levels < 1) return fail(FTE_EINVAL, "not an AMR background");
    const bool table_only = bg->grid.ring > 0 && (bg->grid.dtype != FTE_F32 || bg->grid.layout != FTE_LAYOUT_CELL);
    if (!table_only && (bg->grid.dtype != FTE_F32 || bg->grid.layout != FTE_LAYOUT_CELL))
        return fail(FTE_EINVAL, "prepare the FP32 cell-layout background, then convert it");
    const GridK g = make_gridk(bg);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nt = (size_t)g.nf0 * g.nf1 * g.nf2;
    unsigned* status = reinterpret_cast<unsigned*>(bg->table + nt);
    FTE_CUDA(launch_amr_table(g, bg->table, status, st), "AMR table launch");
    unsigned h[4] = {0, 0, 0, 0};
    FTE_CUDA(cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st), "AMR status copy");
    FTE_CUDA(cudaStreamSynchronize(st), "stream sync");
    if (h[0] || h[1] || h[2] || h[3])
        return fail(FTE_EINVAL, "AMR leaves: %u malformed, %u overlapping finest blocks, %u uncovered, "
                    "%u nesting violations", h[0], h[1], h[2], h[3]);
    if (table_only) return FTE_OK;     // the slots are filled (ghosts included) as snapshots stream in
    FTE_CUDA(launch_amr_ghosts(g, resident_snapshots(&bg->grid), bg->grid.r_min, bg->grid.r_max, bg->grid.th_min,
                               bg->grid.th_max, st), "AMR ghost launch");
    return FTE_OK;
}

fte_status fte_quantize_background(const fte_grid* g_half, const float* dev_f32, void* dev_out,
                                   size_t out_bytes, void* stream)
{
    fte_status s = check_grid(g_half);
    if (s != FTE_OK) return s;
    if (g_half->dtype == FTE_F32 && g_half->layout == FTE_LAYOUT_CELL)
        return fail(FTE_EINVAL, "conversion target must be 16-bit or use the pair layout");
    if (!dev_f32 || !dev_out) return fail(FTE_EINVAL, "NULL field pointer");
    if ((uintptr_t)dev_f32 % 32 || (uintptr_t)dev_out % 32) return fail(FTE_EINVAL, "arrays must be 32-byte aligned");
    const size_t need = grid_bytes(g_half);
    if (out_bytes < need) return fail(FTE_ENOMEM, "output buffer has %zu bytes, needs %zu", out_bytes, need);
    FTE_CUDA(launch_quantize(dev_f32, (long long)grid_records(g_half), row_cells(g_half), g_half->dtype,
                             g_half->layout == FTE_LAYOUT_PAIR, dev_out, (cudaStream_t)stream),
             "conversion launch");
    return FTE_OK;
}

size_t fte_tally_bins(const fte_tally_buf* t)
{
    size_t nb = 0;
    if (!t || t->n_obs < 0 || t->n_obs > FTE_MAX_OBS || t->n_sets < 0 || t->n_sets > FTE_MAX_SETS) return 0;
    for (int o = 0; o < t->n_obs; ++o) {
        if (t->obs[o].ne < 1 || t->obs[o].nt < 1) return 0;
        nb += (size_t)t->obs[o].ne * t->obs[o].nt;
    }
    return nb;
}

fte_status fte_tally_reset(const fte_tally_buf* t, void* stream)
{
    size_t nb = 0;
    fte_status s = check_tally(t, &nb);
    if (s != FTE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    nb *= (size_t)(t->n_sets > 1 ? t->n_sets : 1);
    if (nb) {
        FTE_CUDA(cudaMemsetAsync(t->S, 0, nb * sizeof(double), st), "memset S");
        FTE_CUDA(cudaMemsetAsync(t->S2, 0, nb * sizeof(double), st), "memset S2");
        FTE_CUDA(cudaMemsetAsync(t->C, 0, nb * sizeof(unsigned long long), st), "memset C");
    }
    if (t->S_class && nb)
        FTE_CUDA(cudaMemsetAsync(t->S_class, 0, nb * FTE_NCLASS * sizeof(double), st), "memset S_class");
    FTE_CUDA(cudaMemsetAsync(t->ledger_w, 0, FTE_LEDGER * sizeof(double), st), "memset ledger");
    FTE_CUDA(cudaMemsetAsync(t->ledger_n, 0, FTE_LEDGER * sizeof(unsigned long long), st), "memset ledger");
    return FTE_OK;
}

size_t fte_workspace_bytes(int device, const fte_grid* g, const fte_tally_buf* t,
                           uint64_t n_particles, int64_t n_steps)
{
    size_t nb = 0;
    if (check_grid(g) != FTE_OK) return 0;
    if (check_tally(t, &nb) != FTE_OK || n_steps < 0) return 0;
    fte_background tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.grid = *g;
    const size_t sort_bytes = advance_sort_bytes(make_gridk(&tmp), n_particles);
    size_t best = 0;
    for (int dtype = FTE_F32; dtype <= FTE_F16; ++dtype)
        for (int kperp = 0; kperp < 2; ++kperp)
            for (int pair = 0; pair < 2; ++pair)
                for (int mode : {kModeSingle, kModeSingleGlobal}) {
                    if (mode == kModeSingle && nb > (size_t)kMaxSmemBins) continue;
                    WsLayout L;
                    if (layout(device, kperp, dtype, pair, g->amr_levels > 0, mode, nb, n_steps, sort_bytes, &L) != FTE_OK)
                        return 0;
                    if (L.total > best) best = L.total;
                }
    return best;
}

fte_status fte_inject(fte_particles* P, const fte_background* bg, const fte_inject_spec* spec,
                      uint64_t n, const fte_tally_buf* t, uint64_t* n_failed, void* stream)
{
    if (!P || !spec) return fail(FTE_EINVAL, "NULL particles or spec");
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    size_t nb = 0;
    s = check_tally(t, &nb);
    if (s != FTE_OK) return s;
    if (!P->x || !P->y || !P->z || !P->mu || !P->p || !P->w || !P->id || !P->status)
        return fail(FTE_EINVAL, "NULL particle array");
    if (P->count + n > P->capacity) return fail(FTE_ENOMEM, "pool capacity %llu < %llu", (unsigned long long)P->capacity,
                                                (unsigned long long)(P->count + n));
    if (spec->region != 0 && spec->region != 1) return fail(FTE_EINVAL, "bad region");
    if (spec->energy != 0 && spec->energy != 1) return fail(FTE_EINVAL, "bad energy mode");
    if (spec->energy == 0 && !(spec->e0 > 0)) return fail(FTE_EINVAL, "e0 must be > 0");
    if (spec->energy == 1 && !(spec->e1 > 0 && spec->e2 > spec->e1)) return fail(FTE_EINVAL, "need 0 < e1 < e2");
    if (spec->region == 1) {
        if (!(spec->r2 > spec->r1 && spec->r1 > 0)) return fail(FTE_EINVAL, "need 0 < r1 < r2");
        if (spec->max_tries < 1) return fail(FTE_EINVAL, "max_tries must be >= 1");
        if (spec->use_divv && (spec->divv_snap < 0 || spec->divv_snap >= resident_snapshots(&bg->grid)))
            return fail(FTE_EINVAL, "divv_snap out of range");
    }
    if (spec->mu_mode == 1 && !(spec->mu0 >= -1.0 && spec->mu0 <= 1.0)) return fail(FTE_EINVAL, "mu0 outside [-1, 1]");
    if ((uint64_t)spec->id_base + n > 0x100000000ull) return fail(FTE_EINVAL, "particle ids exceed 32 bits");
    if (n == 0) {
        if (n_failed) *n_failed = 0;
        return FTE_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long before = 0;
    if (n_failed) FTE_CUDA(cudaMemcpyAsync(&before, t->ledger_n + 5, sizeof(before), cudaMemcpyDeviceToHost, st), "ledger read");
    InjectArgs a;
    memset(&a, 0, sizeof(a));
    a.g = make_gridk(bg);
    a.n_snap = bg->grid.n_snap;
    a.region = spec->region; a.energy = spec->energy; a.weight = spec->weight; a.mu_mode = spec->mu_mode;
    a.use_divv = spec->use_divv; a.divv_snap = spec->divv_snap; a.max_tries = spec->max_tries;
    a.r = (float)spec->r; a.th = (float)spec->th; a.ph = (float)spec->ph;
    a.r1 = (float)spec->r1; a.r2 = (float)spec->r2; a.th1 = (float)spec->th1; a.th2 = (float)spec->th2;
    a.ph1 = (float)spec->ph1; a.ph2 = (float)spec->ph2; a.divv_max = (float)spec->divv_max;
    a.e0 = (float)spec->e0; a.e1 = (float)spec->e1; a.e2 = (float)spec->e2; a.gamma = (float)spec->gamma;
    a.mu0 = (float)spec->mu0;
    a.spiral = (float)spec->spiral; a.spiral_rb = (float)spec->spiral_rb;
    a.seed = spec->seed; a.set_id = spec->set_id; a.id_base = spec->id_base;
    a.offset = P->count; a.n = n;
    a.x = P->x; a.y = P->y; a.z = P->z; a.mu = P->mu; a.p = P->p; a.w = P->w; a.id = P->id; a.status = P->status;
    a.ledger_w = t->ledger_w; a.ledger_n = t->ledger_n;
    FTE_CUDA(launch_inject(a, st), "inject launch");
    P->count += n;
    if (n_failed) {
        unsigned long long after = 0;
        FTE_CUDA(cudaMemcpyAsync(&after, t->ledger_n + 5, sizeof(after), cudaMemcpyDeviceToHost, st), "ledger read");
        FTE_CUDA(cudaStreamSynchronize(st), "stream sync");
        *n_failed = after - before;
        if (after != before) return fail(FTE_ERANGE, "%llu particles found no acceptable position", after - before);
    }
    return FTE_OK;
}

fte_status fte_advance(fte_particles* P, const fte_background* bg, const fte_params* prm,
                       const fte_tally_buf* t, int64_t n_start, int64_t n_end, void* ws,
                       size_t ws_bytes, void* stream)
{
    if (!P || !prm) return fail(FTE_EINVAL, "NULL particles or params");
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    size_t nb = 0;
    s = check_tally(t, &nb);
    if (s != FTE_OK) return s;
    if (prm && prm->tally_layout != 0 && prm->tally_layout != FTE_LAYOUT_SHARED && prm->tally_layout != FTE_LAYOUT_GLOBAL)
        return fail(FTE_EINVAL, "bad tally layout");
    // the warp-merged FP64 atomics unless the shared-memory histogram is asked for
    const int mode = (prm && prm->tally_layout == FTE_LAYOUT_SHARED) ? kModeSingle : kModeSingleGlobal;
    if (mode == kModeSingle && nb > (size_t)kMaxSmemBins)
        return fail(FTE_ENOTSUP, "%zu tally bins exceed %d", nb, kMaxSmemBins);
    if (n_end < n_start || n_start < 0) return fail(FTE_EINVAL, "need 0 <= n_start <= n_end");
    if (n_end > 0xFFFFFFFFll) return fail(FTE_EINVAL, "step index exceeds 32 bits");
    if (!(prm->dt > 0.0)) return fail(FTE_EINVAL, "dt must be > 0");
    if (!(prm->lambda_par > 0.0)) return fail(FTE_EINVAL, "lambda_par must be > 0");
    if (prm->dmumu < 0 || prm->dmumu > 2) return fail(FTE_EINVAL, "bad dmumu model");
    if (prm->dmumu == 0 && !(prm->q > 1.0 && prm->q <= 2.0 && prm->H >= 0.0)) return fail(FTE_EINVAL, "need 1 < q <= 2, H >= 0");
    if (prm->dmumu == 1 && !(prm->eps > 0.0)) return fail(FTE_EINVAL, "eps must be > 0");
    if (prm->lambda_perp < 0.0) return fail(FTE_EINVAL, "lambda_perp must be >= 0");
    if (!ws) return fail(FTE_EINVAL, "NULL workspace");
    if (!P->x || !P->y || !P->z || !P->mu || !P->p || !P->w || !P->id || !P->status)
        return fail(FTE_EINVAL, "NULL particle array");
    if (n_end == n_start || P->count == 0) return FTE_OK;

    int device = 0;
    FTE_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    const int kperp = prm->lambda_perp > 0.0 ? 1 : 0;
    const long long nsteps = n_end - n_start;
    const GridK gk = make_gridk(bg);
    const int sorting = prm->sort_every > 0;
    WsLayout L;
    s = layout(device, kperp, bg->grid.dtype, gk.pair, gk.amr > 0, mode, nb, nsteps,
               sorting ? advance_sort_bytes(gk, P->count) : 0,
               &L);
    if (s != FTE_OK) return s;
    if (ws_bytes < L.total) return fail(FTE_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
    char* w = (char*)ws;
    cudaStream_t st = (cudaStream_t)stream;

    double* norm = (double*)(w + L.off_norm);
    FTE_CUDA(launch_norm(prm->dmumu, prm->q, prm->H, prm->eps, norm, (double*)(w + L.off_npart), st),
             "norm launch");

    StepTableArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.tab = (StepEntry*)(w + L.off_table);
    ta.n0 = n_start; ta.count = nsteps; ta.t0 = prm->t0; ta.dt = prm->dt;
    ta.n_snap = bg->grid.n_snap; ta.periodic = bg->grid.periodic; ta.ring = bg->grid.ring;
    ta.t_snap0 = bg->grid.t_snap0; ta.dt_snap = bg->grid.dt_snap;
    ta.n_obs = t->n_obs;
    for (int o = 0; o < t->n_obs; ++o) {
        ta.ot[o].t_lo = t->obs[o].t_lo; ta.ot[o].t_hi = t->obs[o].t_hi; ta.ot[o].nt = t->obs[o].nt;
    }
    FTE_CUDA(launch_step_table(ta, st), "step table launch");

    AdvanceArgs a;
    memset(&a, 0, sizeof(a));
    a.g = gk;
    a.prm.dmumu = prm->dmumu; a.prm.p_update = prm->p_update; a.prm.kappa_drift = prm->kappa_drift;
    a.prm.dvdt_term = prm->dvdt_term;
    a.prm.use_rig = (prm->p_ref > 0.0 && prm->alpha != 0.0) ? 1 : 0;
    a.prm.lambda_par = (float)prm->lambda_par; a.prm.p_ref = (float)prm->p_ref; a.prm.alpha = (float)prm->alpha;
    a.prm.inv_lambda_par = (float)(1.0 / prm->lambda_par);
    a.prm.q = (float)prm->q; a.prm.H = (float)prm->H; a.prm.eps = (float)prm->eps;
    a.prm.mu_floor = (float)prm->mu_floor; a.prm.lambda_perp = (float)prm->lambda_perp;
    a.prm.dt = (float)prm->dt; a.prm.seed = prm->seed; a.prm.set_id = prm->set_id;
    SortArgs sa;
    memset(&sa, 0, sizeof(sa));
    if (sorting) {
        sort_carve(gk, P->count, w + L.off_sort, &sa);
        sa.g = gk;
        sa.x = P->x; sa.y = P->y; sa.z = P->z; sa.mu = P->mu; sa.status = P->status; sa.n = P->count;
        a.order = sa.order;
        a.n_order = sa.hist + sa.nb;
    }
    fill_observers(t, &a);
    a.nbins = (int)(nb ? nb : 1);
    a.x = P->x; a.y = P->y; a.z = P->z; a.mu = P->mu; a.p = P->p; a.w = P->w; a.id = P->id; a.status = P->status;
    a.n_particles = P->count;
    a.n_table0 = n_start;
    a.table = ta.tab;
    a.norm = norm;
    a.part = (float*)(w + L.off_part);
    a.gS = t->S; a.gS2 = t->S2; a.gC = t->C;
    a.fetch = (unsigned long long*)(w + L.off_fetch);
    // per-SM ranges for FP32 records (L1 hits 95 -> 97 %; 16-bit records measured 2-3 % slower)
    a.fetch_slots = bg->grid.dtype == FTE_F32 ? kFetchSlots : 0u;
    a.ledger_w = t->ledger_w; a.ledger_n = t->ledger_n;

    // Grid: an equal number of particles per thread (no partial last wave); with
    // reordering the alive count is only known on the device, so all resident
    // blocks are launched.
    const unsigned long long lanes = (unsigned long long)L.blocks * L.threads;
    const unsigned long long per = (P->count + lanes - 1) / lanes;
    const unsigned long long threads = (P->count + per - 1) / per;
    int blocks = (int)((threads + L.threads - 1) / L.threads);
    if (blocks > L.blocks || sorting) blocks = L.blocks;
    if (blocks < 1) blocks = 1;
    const long long chunk = sorting ? (prm->sort_every < kChunkSteps ? prm->sort_every : kChunkSteps) : kChunkSteps;
    const size_t smem = single_smem(mode, nb);
    int per_sm = 0;
    FTE_CUDA(advance_occupancy(kperp, bg->grid.dtype, mode, L.threads, bg->grid.layout == FTE_LAYOUT_PAIR, gk.amr > 0,
                               smem, &per_sm), "occupancy");

    // Two halves on two streams: while the last particles of one half's launch run, the
    // other half's reordering and launch fill the idle SMs (the step kernel launches one
    // wave of persistent blocks and its end waits for its slowest thread).  Only with the
    // global tally (no per-block partials), a pool of at least one wave, and outside
    // stream capture; each particle's result does not depend on it.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FTE_CUDA(cudaStreamIsCapturing(st, &cap), "capture query");
    if (sorting && mode == kModeSingleGlobal && P->count >= lanes && cap == cudaStreamCaptureStatusNone) {
        SideStream side;
        FTE_CUDA(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking), "stream create");
        FTE_CUDA(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming), "event create");
        FTE_CUDA(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming), "event create");
        AdvanceArgs ah[2] = {a, a};
        SortArgs sh[2];
        cudaStream_t hs[2] = {st, side.s};
        const unsigned long long half = P->count / 2;
        char* p = w + L.off_sort;
        for (int k = 0; k < 2; ++k) {
            const unsigned long long base = k ? half : 0, cnt = k ? P->count - half : half;
            AdvanceArgs& ak = ah[k];
            ak.x = P->x + base; ak.y = P->y + base; ak.z = P->z + base; ak.mu = P->mu + base;
            ak.p = P->p + base; ak.w = P->w + base; ak.id = P->id + base; ak.status = P->status + base;
            ak.n_particles = cnt;
            ak.compact = 1;
            memset(&sh[k], 0, sizeof(SortArgs));
            sort_carve(gk, cnt, p, &sh[k]);
            p += sort_scratch_bytes(gk, cnt);
            sh[k].g = gk;
            sh[k].x = ak.x; sh[k].y = ak.y; sh[k].z = ak.z; sh[k].mu = ak.mu; sh[k].status = ak.status;
            sh[k].n = cnt;
            ak.order = sh[k].order;
            ak.n_order = sh[k].hist + sh[k].nb;
        }
        ah[1].fetch = reinterpret_cast<unsigned long long*>(p);
        FTE_CUDA(cudaEventRecord(side.fork, st), "fork");
        FTE_CUDA(cudaStreamWaitEvent(side.s, side.fork, 0), "fork");
        for (long long c0 = n_start; c0 < n_end; c0 += chunk) {
            for (int k = 0; k < 2; ++k) {
                ah[k].n_start = c0;
                ah[k].n_end = (c0 + chunk < n_end) ? c0 + chunk : n_end;
                FTE_CUDA(launch_sort(sh[k], hs[k]), "sort launch");
                FTE_CUDA(cudaMemsetAsync(ah[k].fetch, 0, kFetchBytes, hs[k]), "fetch reset");
                FTE_CUDA(launch_advance_timed(ah[k], kperp, mode, blocks, smem, hs[k], false), "step kernel launch");
            }
        }
        FTE_CUDA(cudaEventRecord(side.join, side.s), "join");
        FTE_CUDA(cudaStreamWaitEvent(st, side.join, 0), "join");
        return FTE_OK;
    }

    for (long long c0 = n_start; c0 < n_end; c0 += chunk) {
        a.n_start = c0;
        a.n_end = (c0 + chunk < n_end) ? c0 + chunk : n_end;
        if (sorting) FTE_CUDA(launch_sort(sa, st), "sort launch");
        FTE_CUDA(cudaMemsetAsync(a.fetch, 0, kFetchBytes, st), "fetch reset");
        FTE_CUDA(launch_advance_timed(a, kperp, mode, blocks, smem, st, cap != cudaStreamCaptureStatusNone),
                 "step kernel launch");
        if (nb && mode == kModeSingle)
            FTE_CUDA(launch_reduce(a.part, blocks, (int)nb, t->S, t->S2, t->C, st), "reduce launch");
    }
    return FTE_OK;
}

fte_status fte_tally(const fte_tally_buf* t, int obs, int kind, double* dev_out, void* host_out,
                     size_t bytes, void* stream)
{
    return fte_tally_set(t, 0, obs, kind, dev_out, host_out, bytes, stream);
}

}  // extern "C"

namespace {

// Validated description of one observer's block of bins (set `set`) for the output kernels.
fte_status obs_out(const fte_tally_buf* t, int set, int obs, ObsOut* o, size_t* n)
{
    size_t nb = 0;
    fte_status s = check_tally(t, &nb);
    if (s != FTE_OK) return s;
    if (set < 0 || set >= (t->n_sets > 1 ? t->n_sets : 1)) return fail(FTE_EINVAL, "set %d out of range", set);
    if (obs < 0 || obs >= t->n_obs) return fail(FTE_EINVAL, "observer %d out of range", obs);
    const fte_observer& ob = t->obs[obs];
    *n = (size_t)ob.ne * ob.nt;
    o->kind = ob.kind; o->ne = ob.ne; o->nt = ob.nt;
    size_t off = (size_t)set * nb;
    for (int k = 0; k < obs; ++k) off += (size_t)t->obs[k].ne * t->obs[k].nt;
    o->off = (int)off;
    o->r = ob.r; o->dr = ob.dr; o->th = ob.th; o->dth = ob.dth; o->dph = ob.dph;
    o->e_lo = ob.e_lo; o->e_hi = ob.e_hi; o->t_lo = ob.t_lo; o->t_hi = ob.t_hi;
    return FTE_OK;
}

fte_status copy_out(void* host_out, const double* dev_out, size_t n, cudaStream_t st)
{
    if (host_out) {
        FTE_CUDA(cudaMemcpyAsync(host_out, dev_out, n * sizeof(double), cudaMemcpyDeviceToHost, st), "tally copy");
        FTE_CUDA(cudaStreamSynchronize(st), "stream sync");
    }
    return FTE_OK;
}

}  // namespace

extern "C" {

fte_status fte_tally_set(const fte_tally_buf* t, int set, int obs, int kind, double* dev_out, void* host_out,
                         size_t bytes, void* stream)
{
    ObsOut o;
    size_t n = 0;
    fte_status s = obs_out(t, set, obs, &o, &n);
    if (s != FTE_OK) return s;
    if (kind < FTE_TALLY_S || kind > FTE_TALLY_INTENSITY) return fail(FTE_EINVAL, "bad tally kind");
    if (!dev_out) return fail(FTE_EINVAL, "NULL device output");
    if (host_out && bytes < n * sizeof(double)) return fail(FTE_ENOMEM, "host buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    FTE_CUDA(launch_tally_out(t->S, t->S2, t->C, o, kind, dev_out, st), "tally output launch");
    return copy_out(host_out, dev_out, n, st);
}

fte_status fte_tally_convolve(const fte_tally_buf* t, int set, int obs, int kind, const double* dev_src,
                              double* dev_out, void* host_out, size_t bytes, void* stream)
{
    ObsOut o;
    size_t n = 0;
    fte_status s = obs_out(t, set, obs, &o, &n);
    if (s != FTE_OK) return s;
    if (kind != FTE_TALLY_S && kind != FTE_TALLY_INTENSITY) return fail(FTE_EINVAL, "kind must be S or INTENSITY");
    if (o.kind == 3) return fail(FTE_EINVAL, "observer %d bins longitude, not time", obs);
    if (!dev_out) return fail(FTE_EINVAL, "NULL device output");
    if (host_out && bytes < n * sizeof(double)) return fail(FTE_ENOMEM, "host buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    FTE_CUDA(launch_convolve(t->S, o, kind, dev_src, dev_out, st), "convolution launch");
    return copy_out(host_out, dev_out, n, st);
}

fte_status fte_probe_gather_l1(const void* buf, size_t bytes, int threads, int records, int spread,
                               float* dev_out, void* stream)
{
    if (!buf || !dev_out) return fail(FTE_EINVAL, "NULL pointer");
    if ((uintptr_t)buf % 32) return fail(FTE_EINVAL, "buffer must be 32-byte aligned");
    const unsigned long long nrec = bytes / (FTE_REC * sizeof(float));
    if (nrec < 64) return fail(FTE_EINVAL, "buffer holds %llu records, fewer than 64", nrec);
    if (spread < 1 || spread > 32) return fail(FTE_EINVAL, "spread must be in [1, 32]");
    if (threads < 256 || threads % 256 || records < 1)
        return fail(FTE_EINVAL, "threads must be a multiple of 256, records >= 1");
    FTE_CUDA(launch_probe_l1((const float*)buf, (unsigned)nrec, threads, records, spread, dev_out,
                             (cudaStream_t)stream), "probe launch");
    return FTE_OK;
}

fte_status fte_probe_step_timing(int capacity)
{
    if (capacity < 0 || capacity > (1 << 20)) return fail(FTE_EINVAL, "capacity must be in [0, 2^20]");
    std::lock_guard<std::mutex> lock(g_timing.mu);
    g_timing.on.store(0);
    for (cudaEvent_t e : g_timing.ev) cudaEventDestroy(e);
    g_timing.ev.clear();
    g_timing.used = 0;
    if (capacity == 0) return FTE_OK;
    g_timing.ev.resize(2 * (size_t)capacity, nullptr);
    for (auto& e : g_timing.ev) {
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) {
            for (cudaEvent_t x : g_timing.ev)
                if (x) cudaEventDestroy(x);
            g_timing.ev.clear();
            return cuda_fail(r, "cudaEventCreate");
        }
    }
    g_timing.on.store(1);
    return FTE_OK;
}

fte_status fte_probe_step_intervals(double* host_ms, int capacity, int* count)
{
    if (!count || (capacity > 0 && !host_ms)) return fail(FTE_EINVAL, "NULL pointer");
    std::lock_guard<std::mutex> lock(g_timing.mu);
    const int n = g_timing.used / 2;
    *count = n;
    if (n > capacity) return fail(FTE_ENOMEM, "%d launches recorded, room for %d", n, capacity);
    for (int i = 0; i < 2 * n; ++i) FTE_CUDA(cudaEventSynchronize(g_timing.ev[i]), "event synchronize");
    for (int i = 0; i < 2 * n; ++i) {
        float ms = 0.f;
        FTE_CUDA(cudaEventElapsedTime(&ms, g_timing.ev[0], g_timing.ev[i]), "event elapsed");
        host_ms[i] = ms;
    }
    g_timing.used = 0;
    return FTE_OK;
}

fte_status fte_probe_sectors(const void* buf, size_t bytes, int threads, int loads, float* dev_out,
                             void* stream)
{
    if (!buf || !dev_out) return fail(FTE_EINVAL, "NULL pointer");
    if ((uintptr_t)buf % 32 || bytes < 32) return fail(FTE_EINVAL, "buffer must be 32-byte aligned, >= 32 bytes");
    if (threads < 256 || threads % 256 || loads < 1) return fail(FTE_EINVAL, "threads must be a multiple of 256, loads >= 1");
    FTE_CUDA(launch_probe((const float*)buf, bytes / 32, threads, loads, dev_out, (cudaStream_t)stream),
             "probe launch");
    return FTE_OK;
}

fte_status fte_ledger(const fte_tally_buf* t, double* host_w, uint64_t* host_n, void* stream)
{
    if (!t || !t->ledger_w || !t->ledger_n || !host_w || !host_n) return fail(FTE_EINVAL, "NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    FTE_CUDA(cudaMemcpyAsync(host_w, t->ledger_w, FTE_LEDGER * sizeof(double), cudaMemcpyDeviceToHost, st), "ledger copy");
    FTE_CUDA(cudaMemcpyAsync(host_n, t->ledger_n, FTE_LEDGER * sizeof(uint64_t), cudaMemcpyDeviceToHost, st), "ledger copy");
    FTE_CUDA(cudaStreamSynchronize(st), "stream sync");
    return FTE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of fte_advance.
//
// Some callers cannot hand the library a scratch buffer: a host code that has
// reserved all device memory for its own pool at start-up, or a service that
// must not call cudaMalloc once it runs (the call can synchronise the device
// and can fail under memory pressure).  For them the scratch of the step loop
// lives in this file-scope device array.  Every GPU that loads the library
// holds it until the process exits.  All calls share it, so two calls whose
// work overlaps on the GPU (for example on two streams) race on it; it keeps
// the contents of the last call, and every value that must start at zero is
// cleared by the call itself.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kNoAllocBytes = 24u << 20;           // 24 MiB of scratch per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64];

// Device address of the scratch array for the current device, looked up once
// per device (the host-side name of the array is not a device address).  The
// address belongs to the device's primary context: after cudaDeviceReset (or
// any teardown of that context) it is no longer valid, and this process must
// not call fte_advance_noalloc on that device again.
fte_status noalloc_scratch(int device, char** out)
{
    if (device < 0 || device >= 64) return fail(FTE_ENOTSUP, "device index %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[device] = p;
    }
    *out = (char*)g_noalloc_ptr[device];
    return FTE_OK;
}

}  // namespace

extern "C" fte_status fte_advance_noalloc(fte_particles* P, const fte_background* bg,
                                          const fte_params* prm, const fte_tally_buf* t,
                                          int64_t n_start, int64_t n_end, void* stream)
{
    if (!P || !prm) return fail(FTE_EINVAL, "NULL particles or params");
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    size_t nb = 0;
    s = check_tally(t, &nb);
    if (s != FTE_OK) return s;
    if (nb > (size_t)kMaxSmemBins) return fail(FTE_ENOTSUP, "%zu tally bins exceed %d", nb, kMaxSmemBins);
    if (n_end < n_start || n_start < 0) return fail(FTE_EINVAL, "need 0 <= n_start <= n_end");
    if (n_end > 0xFFFFFFFFll) return fail(FTE_EINVAL, "step index exceeds 32 bits");
    if (!(prm->dt > 0.0)) return fail(FTE_EINVAL, "dt must be > 0");
    if (!(prm->lambda_par > 0.0)) return fail(FTE_EINVAL, "lambda_par must be > 0");
    if (prm->dmumu < 0 || prm->dmumu > 2) return fail(FTE_EINVAL, "bad dmumu model");
    if (prm->dmumu == 0 && !(prm->q > 1.0 && prm->q <= 2.0 && prm->H >= 0.0)) return fail(FTE_EINVAL, "need 1 < q <= 2, H >= 0");
    if (prm->dmumu == 1 && !(prm->eps > 0.0)) return fail(FTE_EINVAL, "eps must be > 0");
    if (prm->lambda_perp < 0.0) return fail(FTE_EINVAL, "lambda_perp must be >= 0");
    // the tally always goes through per-block shared-memory histograms here; other layout
    // values are refused as fte_advance refuses them
    if (prm->tally_layout != 0 && prm->tally_layout != FTE_LAYOUT_SHARED && prm->tally_layout != FTE_LAYOUT_GLOBAL)
        return fail(FTE_EINVAL, "bad tally_layout %d", prm->tally_layout);
    if (!P->x || !P->y || !P->z || !P->mu || !P->p || !P->w || !P->id || !P->status)
        return fail(FTE_EINVAL, "NULL particle array");

    int device = 0;
    FTE_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    char* w = nullptr;
    s = noalloc_scratch(device, &w);
    if (s != FTE_OK) return s;
    if (n_end == n_start || P->count == 0) return FTE_OK;

    // scratch layout: fetch counter, normalisation, the time table of one
    // launch, then per-block partial histograms
    const int kperp = prm->lambda_perp > 0.0 ? 1 : 0;
    const size_t off_fetch = 0, off_norm = 64, off_npart = 128;
    const size_t off_table = off_npart + kNormPartials * sizeof(double);
    const size_t off_part = (off_table + (size_t)kChunkSteps * sizeof(StepEntry) + 255) & ~(size_t)255;
    const size_t part_block = 3 * sizeof(float) * (nb ? nb : 1);
    const int sms = device_sms(device);
    if (sms <= 0) return fail(FTE_ECUDA, "cannot query device %d", device);
    const size_t fit = (kNoAllocBytes - off_part) / part_block;
    if (fit < (size_t)sms)
        return fail(FTE_ENOMEM, "a tally of %zu bins needs %zu bytes of scratch per block; the "
                    "allocation-free variant holds %zu bytes, less than one block per SM (%d)",
                    nb, part_block, kNoAllocBytes, sms);
    const size_t smem = part_block;
    int per_sm = 0;
    FTE_CUDA(advance_occupancy(kperp, bg->grid.dtype, kModeSingle, kThreads, bg->grid.layout == FTE_LAYOUT_PAIR,
                                bg->grid.amr_levels > 0, smem, &per_sm), "occupancy");
    if (per_sm < 1) return fail(FTE_ENOTSUP, "step kernel does not fit on an SM with %zu bytes of tally", smem);
    long long max_blocks = (long long)sms * per_sm;
    if ((size_t)max_blocks > fit) max_blocks = (long long)fit;

    cudaStream_t st = (cudaStream_t)stream;
    double* norm = (double*)(w + off_norm);
    FTE_CUDA(launch_norm(prm->dmumu, prm->q, prm->H, prm->eps, norm, (double*)(w + off_npart), st),
             "norm launch");

    AdvanceArgs a;
    memset(&a, 0, sizeof(a));
    a.g = make_gridk(bg);
    a.prm.dmumu = prm->dmumu; a.prm.p_update = prm->p_update; a.prm.kappa_drift = prm->kappa_drift;
    a.prm.dvdt_term = prm->dvdt_term;
    a.prm.use_rig = (prm->p_ref > 0.0 && prm->alpha != 0.0) ? 1 : 0;
    a.prm.lambda_par = (float)prm->lambda_par; a.prm.p_ref = (float)prm->p_ref; a.prm.alpha = (float)prm->alpha;
    a.prm.inv_lambda_par = (float)(1.0 / prm->lambda_par);
    a.prm.q = (float)prm->q; a.prm.H = (float)prm->H; a.prm.eps = (float)prm->eps;
    a.prm.mu_floor = (float)prm->mu_floor; a.prm.lambda_perp = (float)prm->lambda_perp;
    a.prm.dt = (float)prm->dt; a.prm.seed = prm->seed; a.prm.set_id = prm->set_id;
    fill_observers(t, &a);
    a.nbins = (int)(nb ? nb : 1);
    a.x = P->x; a.y = P->y; a.z = P->z; a.mu = P->mu; a.p = P->p; a.w = P->w; a.id = P->id; a.status = P->status;
    a.n_particles = P->count;
    a.table = (const StepEntry*)(w + off_table);
    a.norm = norm;
    a.part = (float*)(w + off_part);
    a.fetch = (unsigned long long*)(w + off_fetch);
    a.ledger_w = t->ledger_w; a.ledger_n = t->ledger_n;

    const unsigned long long lanes = (unsigned long long)max_blocks * kThreads;
    const unsigned long long per = (P->count + lanes - 1) / lanes;
    const unsigned long long threads = (P->count + per - 1) / per;
    long long blocks = (long long)((threads + kThreads - 1) / kThreads);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;

    StepTableArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.tab = (StepEntry*)(w + off_table);
    ta.t0 = prm->t0; ta.dt = prm->dt;
    ta.n_snap = bg->grid.n_snap; ta.periodic = bg->grid.periodic; ta.ring = bg->grid.ring;
    ta.t_snap0 = bg->grid.t_snap0; ta.dt_snap = bg->grid.dt_snap;
    ta.n_obs = t->n_obs;
    for (int o = 0; o < t->n_obs; ++o) {
        ta.ot[o].t_lo = t->obs[o].t_lo; ta.ot[o].t_hi = t->obs[o].t_hi; ta.ot[o].nt = t->obs[o].nt;
    }
    for (long long c0 = n_start; c0 < n_end; c0 += kChunkSteps) {
        const long long c1 = (c0 + kChunkSteps < n_end) ? c0 + kChunkSteps : n_end;
        ta.n0 = c0;
        ta.count = c1 - c0;
        FTE_CUDA(launch_step_table(ta, st), "step table launch");
        a.n_start = c0;
        a.n_end = c1;
        a.n_table0 = c0;
        FTE_CUDA(cudaMemsetAsync(a.fetch, 0, sizeof(unsigned long long), st), "fetch reset");
        FTE_CUDA(launch_advance(a, g_no_batch, kperp, kModeSingle, kThreads, (int)blocks, smem, st), "step kernel launch");
        if (nb) FTE_CUDA(launch_reduce(a.part, (int)blocks, (int)nb, t->S, t->S2, t->C, st), "reduce launch");
    }
    return FTE_OK;
}

// ---------------------------------------------------------------------------
// Ensembles: many parameter sets per launch, the launch-configuration
// autotuner and CUDA graphs of library calls.
// ---------------------------------------------------------------------------
namespace {

struct EnsLayout {
    size_t off_fetch, off_norm, off_npart, off_table, off_part, off_sort, total;
    int blocks;     // resident blocks (SMs x blocks per SM)
};

size_t shared_bins(int n_sets, size_t nb) { return (size_t)n_sets * nb; }

bool shared_fits(int n_sets, size_t nb) { return nb > 0 && shared_bins(n_sets, nb) <= (size_t)kMaxSmemBins; }

size_t ens_smem(int mode, int n_sets, size_t nb)
{
    return mode == kModeShared ? 3 * sizeof(float) * shared_bins(n_sets, nb) : 0;
}

fte_status ens_layout(int device, int kperp, int dtype, int pair, int mode, int nt, int n_sets, size_t nb,
                      long long n_steps, size_t sort_bytes, EnsLayout* L)
{
    const int sms = device_sms(device);
    if (sms <= 0) return fail(FTE_ECUDA, "cannot query device %d", device);
    const size_t smem = ens_smem(mode, n_sets, nb);
    int per_sm = 0, cur = 0;
    FTE_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != device) FTE_CUDA(cudaSetDevice(device), "cudaSetDevice");
    cudaError_t e = advance_occupancy(kperp, dtype, mode, nt, pair, 0, smem, &per_sm);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(FTE_ENOTSUP, "ensemble step kernel does not fit on an SM with %zu bytes of tally", smem);
    L->blocks = sms * per_sm;
    size_t off = 0;
    L->off_fetch = off; off += kFetchBytes;
    L->off_norm = off; off += FTE_MAX_SETS * sizeof(double);
    L->off_npart = off; off += (size_t)FTE_MAX_SETS * kNormPartials * sizeof(double);
    L->off_table = off; off += (size_t)(n_steps > 0 ? n_steps : 1) * sizeof(StepEntry);
    off = (off + 255) & ~(size_t)255;
    L->off_part = off;
    if (mode == kModeShared) off += (size_t)L->blocks * 3 * shared_bins(n_sets, nb) * sizeof(float);
    off = (off + 255) & ~(size_t)255;
    L->off_sort = off; off += sort_bytes;
    L->total = off;
    return FTE_OK;
}

fte_status check_params(const fte_params* prm)
{
    if (!(prm->dt > 0.0)) return fail(FTE_EINVAL, "dt must be > 0");
    if (prm->dmumu < 0 || prm->dmumu > 2) return fail(FTE_EINVAL, "bad dmumu model");
    if (prm->lambda_perp < 0.0) return fail(FTE_EINVAL, "lambda_perp must be >= 0");
    return FTE_OK;
}

fte_status check_sets(const fte_params* prm, const fte_set* sets, int n_sets, const fte_particles* P,
                      const fte_tally_buf* t)
{
    if (!sets) return fail(FTE_EINVAL, "NULL sets");
    if (n_sets < 1 || n_sets > FTE_MAX_SETS) return fail(FTE_EINVAL, "n_sets must be in [1, %d]", FTE_MAX_SETS);
    if ((t->n_sets > 1 ? t->n_sets : 1) < n_sets) return fail(FTE_EINVAL, "tally holds fewer than %d sets", n_sets);
    unsigned long long total = 0;
    for (int s = 0; s < n_sets; ++s) {
        const fte_set& k = sets[s];
        if (!(k.lambda_par > 0.0)) return fail(FTE_EINVAL, "set %d: lambda_par must be > 0", s);
        if (prm->dmumu == 0 && !(k.q > 1.0 && k.q <= 2.0 && k.H >= 0.0))
            return fail(FTE_EINVAL, "set %d: need 1 < q <= 2, H >= 0", s);
        if (prm->dmumu == 1 && !(k.eps > 0.0)) return fail(FTE_EINVAL, "set %d: eps must be > 0", s);
        total += k.count;
    }
    if (total != P->count) return fail(FTE_EINVAL, "set counts add up to %llu, the pool holds %llu", total,
                                       (unsigned long long)P->count);
    return FTE_OK;
}

struct EnsConfig {
    int nt, steps, mode;
};

// The ensemble advance of steps [n_start, n_end) with one launch configuration.
// Validation is done by the callers.
fte_status ens_run(fte_particles* P, const fte_background* bg, const fte_params* prm, const fte_set* sets,
                   int n_sets, const fte_tally_buf* t, size_t nb, int64_t n_start, int64_t n_end,
                   const EnsConfig& cfg, void* ws, size_t ws_bytes, cudaStream_t st)
{
    int device = 0;
    FTE_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    const int kperp = prm->lambda_perp > 0.0 ? 1 : 0;
    const long long nsteps = n_end - n_start;
    const GridK gk = make_gridk(bg);
    const int sorting = prm->sort_every > 0;
    EnsLayout L;
    fte_status s = ens_layout(device, kperp, bg->grid.dtype, gk.pair, cfg.mode, cfg.nt, n_sets, nb, nsteps,
                              sorting ? advance_sort_bytes(gk, P->count) : 0, &L);
    if (s != FTE_OK) return s;
    if (ws_bytes < L.total) return fail(FTE_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
    char* w = (char*)ws;

    NormSets ns;
    memset(&ns, 0, sizeof(ns));
    for (int k = 0; k < n_sets; ++k) { ns.q[k] = sets[k].q; ns.H[k] = sets[k].H; ns.eps[k] = sets[k].eps; }
    double* norm = (double*)(w + L.off_norm);
    FTE_CUDA(launch_norm_sets(prm->dmumu, ns, n_sets, norm, (double*)(w + L.off_npart), st), "norm launch");

    StepTableArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.tab = (StepEntry*)(w + L.off_table);
    ta.n0 = n_start; ta.count = nsteps; ta.t0 = prm->t0; ta.dt = prm->dt;
    ta.n_snap = bg->grid.n_snap; ta.periodic = bg->grid.periodic; ta.ring = bg->grid.ring;
    ta.t_snap0 = bg->grid.t_snap0; ta.dt_snap = bg->grid.dt_snap;
    ta.n_obs = t->n_obs;
    for (int o = 0; o < t->n_obs; ++o) {
        ta.ot[o].t_lo = t->obs[o].t_lo; ta.ot[o].t_hi = t->obs[o].t_hi; ta.ot[o].nt = t->obs[o].nt;
    }
    FTE_CUDA(launch_step_table(ta, st), "step table launch");

    AdvanceArgs a;
    memset(&a, 0, sizeof(a));
    a.g = gk;
    a.prm.dmumu = prm->dmumu; a.prm.p_update = prm->p_update; a.prm.kappa_drift = prm->kappa_drift;
    a.prm.dvdt_term = prm->dvdt_term;
    a.prm.use_rig = (prm->p_ref > 0.0 && prm->alpha != 0.0) ? 1 : 0;
    a.prm.p_ref = (float)prm->p_ref; a.prm.alpha = (float)prm->alpha;
    a.prm.mu_floor = (float)prm->mu_floor; a.prm.lambda_perp = (float)prm->lambda_perp;
    a.prm.dt = (float)prm->dt;
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    b.n_sets = n_sets;
    unsigned long long end = 0;
    for (int k = 0; k < n_sets; ++k) {
        end += sets[k].count;
        b.end[k] = end;
        b.set[k].lambda_par = (float)sets[k].lambda_par; b.set[k].q = (float)sets[k].q;
        b.set[k].H = (float)sets[k].H; b.set[k].eps = (float)sets[k].eps;
        b.set[k].seed = sets[k].seed; b.set[k].set_id = sets[k].set_id;
    }
    SortArgs sa;
    memset(&sa, 0, sizeof(sa));
    if (sorting) {
        sort_carve(gk, P->count, w + L.off_sort, &sa);
        sa.g = gk;
        sa.x = P->x; sa.y = P->y; sa.z = P->z; sa.mu = P->mu; sa.status = P->status; sa.n = P->count;
        a.order = sa.order;
        a.n_order = sa.hist + sa.nb;
    }
    fill_observers(t, &a);
    a.nbins = (int)(nb ? nb : 1);
    a.x = P->x; a.y = P->y; a.z = P->z; a.mu = P->mu; a.p = P->p; a.w = P->w; a.id = P->id; a.status = P->status;
    a.n_particles = P->count;
    a.n_table0 = n_start;
    a.table = ta.tab;
    a.norm = norm;
    a.gS = t->S; a.gS2 = t->S2; a.gC = t->C;
    a.part = (float*)(w + L.off_part);
    a.fetch = (unsigned long long*)(w + L.off_fetch);
    // per-SM ranges for FP32 records (L1 hits 95 -> 97 %; 16-bit records measured 2-3 % slower)
    a.fetch_slots = bg->grid.dtype == FTE_F32 ? kFetchSlots : 0u;
    a.ledger_w = t->ledger_w; a.ledger_n = t->ledger_n;

    const unsigned long long lanes = (unsigned long long)L.blocks * cfg.nt;
    const unsigned long long per = (P->count + lanes - 1) / lanes;
    const unsigned long long threads = (P->count + per - 1) / per;
    int blocks = (int)((threads + cfg.nt - 1) / cfg.nt);
    if (blocks > L.blocks || sorting) blocks = L.blocks;
    if (blocks < 1) blocks = 1;
    const size_t smem = ens_smem(cfg.mode, n_sets, nb);
    const int reduce_bins = (int)shared_bins(n_sets, nb);

    // two halves of the pool on two streams, as in fte_advance (global tally only); each
    // half's set boundaries are taken relative to its first entry
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FTE_CUDA(cudaStreamIsCapturing(st, &cap), "capture query");
    if (sorting && cfg.mode == kModeGlobal && P->count >= lanes && cap == cudaStreamCaptureStatusNone) {
        SideStream side;
        FTE_CUDA(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking), "stream create");
        FTE_CUDA(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming), "event create");
        FTE_CUDA(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming), "event create");
        AdvanceArgs ah[2] = {a, a};
        BatchArgs bh[2] = {b, b};
        SortArgs sh[2];
        cudaStream_t hs[2] = {st, side.s};
        const unsigned long long half = P->count / 2;
        char* p = w + L.off_sort;
        for (int k = 0; k < 2; ++k) {
            const unsigned long long base = k ? half : 0, cnt = k ? P->count - half : half;
            AdvanceArgs& ak = ah[k];
            ak.x = P->x + base; ak.y = P->y + base; ak.z = P->z + base; ak.mu = P->mu + base;
            ak.p = P->p + base; ak.w = P->w + base; ak.id = P->id + base; ak.status = P->status + base;
            ak.n_particles = cnt;
            for (int q = 0; q < n_sets; ++q) {
                const long long e = (long long)b.end[q] - (long long)base;
                bh[k].end[q] = e < 0 ? 0ULL : ((unsigned long long)e > cnt ? cnt : (unsigned long long)e);
            }
            memset(&sh[k], 0, sizeof(SortArgs));
            sort_carve(gk, cnt, p, &sh[k]);
            p += sort_scratch_bytes(gk, cnt);
            sh[k].g = gk;
            sh[k].x = ak.x; sh[k].y = ak.y; sh[k].z = ak.z; sh[k].mu = ak.mu; sh[k].status = ak.status;
            sh[k].n = cnt;
            ak.order = sh[k].order;
            ak.n_order = sh[k].hist + sh[k].nb;
        }
        ah[1].fetch = reinterpret_cast<unsigned long long*>(p);
        FTE_CUDA(cudaEventRecord(side.fork, st), "fork");
        FTE_CUDA(cudaStreamWaitEvent(side.s, side.fork, 0), "fork");
        for (long long c0 = n_start; c0 < n_end; c0 += cfg.steps) {
            for (int k = 0; k < 2; ++k) {
                ah[k].n_start = c0;
                ah[k].n_end = (c0 + cfg.steps < n_end) ? c0 + cfg.steps : n_end;
                FTE_CUDA(launch_sort(sh[k], hs[k]), "sort launch");
                FTE_CUDA(cudaMemsetAsync(ah[k].fetch, 0, kFetchBytes, hs[k]), "fetch reset");
                FTE_CUDA(launch_advance(ah[k], bh[k], kperp, cfg.mode, cfg.nt, blocks, smem, hs[k]),
                         "step kernel launch");
            }
        }
        FTE_CUDA(cudaEventRecord(side.join, side.s), "join");
        FTE_CUDA(cudaStreamWaitEvent(st, side.join, 0), "join");
        return FTE_OK;
    }

    for (long long c0 = n_start; c0 < n_end; c0 += cfg.steps) {
        a.n_start = c0;
        a.n_end = (c0 + cfg.steps < n_end) ? c0 + cfg.steps : n_end;
        if (sorting) FTE_CUDA(launch_sort(sa, st), "sort launch");
        FTE_CUDA(cudaMemsetAsync(a.fetch, 0, kFetchBytes, st), "fetch reset");
        FTE_CUDA(launch_advance(a, b, kperp, cfg.mode, cfg.nt, blocks, smem, st), "step kernel launch");
        if (cfg.mode == kModeShared && nb)
            FTE_CUDA(launch_reduce(a.part, blocks, reduce_bins, t->S, t->S2, t->C, st), "reduce launch");
    }
    return FTE_OK;
}

fte_status ens_check(fte_particles* P, const fte_background* bg, const fte_params* prm, const fte_set* sets,
                     int n_sets, const fte_tally_buf* t, int64_t n_start, int64_t n_end, void* ws, size_t* nb)
{
    if (!P || !prm) return fail(FTE_EINVAL, "NULL particles or params");
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    s = check_tally(t, nb);
    if (s != FTE_OK) return s;
    s = check_params(prm);
    if (s != FTE_OK) return s;
    s = check_sets(prm, sets, n_sets, P, t);
    if (s != FTE_OK) return s;
    if (n_end < n_start || n_start < 0) return fail(FTE_EINVAL, "need 0 <= n_start <= n_end");
    if (n_end > 0xFFFFFFFFll) return fail(FTE_EINVAL, "step index exceeds 32 bits");
    if (!ws) return fail(FTE_EINVAL, "NULL workspace");
    if (!P->x || !P->y || !P->z || !P->mu || !P->p || !P->w || !P->id || !P->status)
        return fail(FTE_EINVAL, "NULL particle array");
    return FTE_OK;
}

fte_status to_config(const fte_launch_config* c, const fte_params* prm, int n_sets, size_t nb, EnsConfig* out)
{
    const long long def_steps = prm->sort_every > 0 ? (prm->sort_every < kChunkSteps ? prm->sort_every : kChunkSteps)
                                                    : kChunkSteps;
    out->nt = c && c->threads ? c->threads : 256;
    out->steps = (int)(c && c->steps_per_launch ? c->steps_per_launch : def_steps);
    const int layout = c && c->tally_layout ? c->tally_layout
                                            : (shared_fits(n_sets, nb) ? FTE_LAYOUT_SHARED : FTE_LAYOUT_GLOBAL);
    if (out->nt != 128 && out->nt != 256) return fail(FTE_EINVAL, "threads must be 128 or 256");
    if (out->steps < 1 || out->steps > kChunkSteps) return fail(FTE_EINVAL, "steps_per_launch must be in [1, %lld]", kChunkSteps);
    if (layout == FTE_LAYOUT_SHARED) {
        if (!shared_fits(n_sets, nb)) return fail(FTE_ENOTSUP, "%d sets x %zu bins do not fit the shared layout", n_sets, nb);
        out->mode = kModeShared;
    } else if (layout == FTE_LAYOUT_GLOBAL) {
        out->mode = kModeGlobal;
    } else {
        return fail(FTE_EINVAL, "bad tally layout");
    }
    return FTE_OK;
}

}  // namespace

struct fte_graph {
    cudaGraphExec_t exec;
};

extern "C" {

size_t fte_workspace_bytes_batched(int device, const fte_grid* g, const fte_tally_buf* t,
                                   uint64_t n_particles, int64_t n_steps)
{
    size_t nb = 0;
    if (check_grid(g) != FTE_OK) return 0;
    if (check_tally(t, &nb) != FTE_OK || n_steps < 0) return 0;
    const int n_sets = t->n_sets > 1 ? t->n_sets : 1;
    fte_background tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.grid = *g;
    const size_t sort_bytes = advance_sort_bytes(make_gridk(&tmp), n_particles);
    size_t best = 0;
    for (int dtype = FTE_F32; dtype <= FTE_F16; ++dtype)
        for (int kperp = 0; kperp < 2; ++kperp)
            for (int mode = kModeShared; mode <= kModeGlobal; ++mode)
                for (int nt = 128; nt <= 256; nt *= 2) {
                    if (mode == kModeShared && !shared_fits(n_sets, nb)) continue;
                    EnsLayout L;
                    for (int pair = 0; pair < 2; ++pair) {
                        const fte_status s = ens_layout(device, kperp, dtype, pair, mode, nt, n_sets, nb, n_steps,
                                                        sort_bytes, &L);
                        if (s == FTE_ENOTSUP) continue;
                        if (s != FTE_OK) return 0;
                        if (L.total > best) best = L.total;
                    }
                }
    return best;
}

fte_status fte_inject_batched(fte_particles* P, const fte_background* bg, const fte_inject_spec* specs,
                              const uint64_t* counts, int n_sets, const fte_tally_buf* t, void* stream)
{
    if (!P || !specs || !counts) return fail(FTE_EINVAL, "NULL particles, specs or counts");
    if (n_sets < 1 || n_sets > FTE_MAX_SETS) return fail(FTE_EINVAL, "n_sets must be in [1, %d]", FTE_MAX_SETS);
    unsigned long long total = 0;
    for (int s = 0; s < n_sets; ++s) total += counts[s];
    if (P->count + total > P->capacity) return fail(FTE_ENOMEM, "pool capacity %llu < %llu",
                                                    (unsigned long long)P->capacity,
                                                    (unsigned long long)(P->count + total));
    for (int s = 0; s < n_sets; ++s) {
        const fte_status st = fte_inject(P, bg, specs + s, counts[s], t, nullptr, stream);
        if (st != FTE_OK) return st;
    }
    return FTE_OK;
}

fte_status fte_advance_batched(fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_set* sets, int n_sets, const fte_tally_buf* t, int64_t n_start,
                               int64_t n_end, const fte_launch_config* cfg, void* ws, size_t ws_bytes,
                               void* stream)
{
    size_t nb = 0;
    fte_status s = ens_check(P, bg, prm, sets, n_sets, t, n_start, n_end, ws, &nb);
    if (s != FTE_OK) return s;
    EnsConfig c;
    s = to_config(cfg, prm, n_sets, nb, &c);
    if (s != FTE_OK) return s;
    if (n_end == n_start || P->count == 0) return FTE_OK;
    return ens_run(P, bg, prm, sets, n_sets, t, nb, n_start, n_end, c, ws, ws_bytes, (cudaStream_t)stream);
}

fte_status fte_autotune_batched(fte_particles* P, const fte_background* bg, const fte_params* prm,
                                const fte_set* sets, int n_sets, const fte_tally_buf* t, int64_t n_start,
                                int64_t n_end, void* ws, size_t ws_bytes, fte_launch_config* best,
                                fte_launch_config* tried, double* rates, int* n_tried, void* stream)
{
    size_t nb = 0;
    fte_status s = ens_check(P, bg, prm, sets, n_sets, t, n_start, n_end, ws, &nb);
    if (s != FTE_OK) return s;
    if (!best) return fail(FTE_EINVAL, "NULL best");
    cudaStream_t st = (cudaStream_t)stream;
    // candidates
    fte_launch_config cand[16];
    int nc = 0;
    const int steps_sorted[4] = {32, 64, 128, 256};
    const int n_steps_opts = prm->sort_every > 0 ? 4 : 1;
    for (int ti = 0; ti < 2; ++ti)
        for (int si = 0; si < n_steps_opts; ++si)
            for (int li = 0; li < 2; ++li) {
                const int layout = li == 0 ? FTE_LAYOUT_SHARED : FTE_LAYOUT_GLOBAL;
                if (layout == FTE_LAYOUT_SHARED && !shared_fits(n_sets, nb)) continue;
                fte_launch_config& c = cand[nc++];
                c.threads = ti == 0 ? 128 : 256;
                c.steps_per_launch = prm->sort_every > 0 ? steps_sorted[si] : (int)kChunkSteps;
                c.tally_layout = layout;
                c.pad = 0;
            }
    double secs[16] = {0}, done[16] = {0};
    int ran[16] = {0};
    const long long trial = prm->sort_every > 0 ? 256 : kChunkSteps;   // steps per trial
    long long n = n_start;
    cudaEvent_t e0, e1;
    FTE_CUDA(cudaEventCreate(&e0), "event create");
    FTE_CUDA(cudaEventCreate(&e1), "event create");
    fte_status result = FTE_OK;
    for (int round = 0; round < 2 && result == FTE_OK; ++round)
        for (int q = 0; q < nc && result == FTE_OK; ++q) {
            const int k = round == 0 ? q : nc - 1 - q;
            if (n + trial > n_end || P->count == 0) break;
            EnsConfig c;
            result = to_config(&cand[k], prm, n_sets, nb, &c);
            if (result != FTE_OK) break;
            unsigned long long before = 0, after = 0;
            if (cudaMemcpyAsync(&before, t->ledger_n + 6, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaEventRecord(e0, st) != cudaSuccess) { result = cuda_fail(cudaGetLastError(), "trial start"); break; }
            result = ens_run(P, bg, prm, sets, n_sets, t, nb, n, n + trial, c, ws, ws_bytes, st);
            if (result != FTE_OK) break;
            if (cudaEventRecord(e1, st) != cudaSuccess ||
                cudaMemcpyAsync(&after, t->ledger_n + 6, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) { result = cuda_fail(cudaGetLastError(), "trial end"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            secs[k] += ms * 1e-3;
            done[k] += (double)(after - before);
            ran[k] = 1;
            n += trial;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != FTE_OK) return result;
    int bi = -1;
    double brate = -1.0;
    for (int k = 0; k < nc; ++k) {
        const double r = (ran[k] && secs[k] > 0) ? done[k] / secs[k] : 0.0;
        if (tried) tried[k] = cand[k];
        if (rates) rates[k] = r;
        if (ran[k] && r > brate) { brate = r; bi = k; }
    }
    if (n_tried) *n_tried = nc;
    if (bi < 0) {   // no trial ran: the default configuration
        EnsConfig c;
        s = to_config(nullptr, prm, n_sets, nb, &c);
        if (s != FTE_OK) return s;
        best->threads = c.nt; best->steps_per_launch = c.steps;
        best->tally_layout = c.mode == kModeShared ? FTE_LAYOUT_SHARED : FTE_LAYOUT_GLOBAL;
        best->pad = 0;
    } else {
        *best = cand[bi];
    }
    if (n < n_end && P->count) {
        EnsConfig c;
        s = to_config(best, prm, n_sets, nb, &c);
        if (s != FTE_OK) return s;
        return ens_run(P, bg, prm, sets, n_sets, t, nb, n, n_end, c, ws, ws_bytes, st);
    }
    return FTE_OK;
}

fte_status fte_graph_begin(void* stream)
{
    if (!stream) return fail(FTE_EINVAL, "the legacy NULL stream cannot be captured");
    FTE_CUDA(cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    return FTE_OK;
}

fte_status fte_graph_end(void* stream, fte_graph** out)
{
    if (!stream || !out) return fail(FTE_EINVAL, "NULL stream or output");
    *out = nullptr;
    cudaGraph_t g = nullptr;
    FTE_CUDA(cudaStreamEndCapture((cudaStream_t)stream, &g), "end capture");
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    fte_graph* h = new (std::nothrow) fte_graph;
    if (!h) {
        cudaGraphExecDestroy(ex);
        return fail(FTE_ENOMEM, "out of host memory");
    }
    h->exec = ex;
    *out = h;
    return FTE_OK;
}

fte_status fte_graph_launch(const fte_graph* g, void* stream)
{
    if (!g) return fail(FTE_EINVAL, "NULL graph");
    FTE_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream), "graph launch");
    return FTE_OK;
}

fte_status fte_graph_destroy(fte_graph* g)
{
    if (!g) return FTE_OK;
    const cudaError_t e = cudaGraphExecDestroy(g->exec);
    delete g;
    if (e != cudaSuccess) return cuda_fail(e, "graph destroy");
    return FTE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Pathwise adjoint: workspace layout, argument checks, forward and reverse.
// ---------------------------------------------------------------------------
namespace {

// Steps per reverse-pass launch (the reordering interval of the reverse pass).
constexpr long long kAdjChunk = 64;
// Per-particle values carried between reverse launches: state adjoint (5), parameter
// adjoint (4), observable accumulated after the current step (1).
constexpr int kAdjRows = 10;

struct AdjLayout {
    size_t off_fetch, off_norm, off_npart, off_normd, off_ndpart, off_table, off_ckpt, off_ndead, off_jpart,
        off_adj, off_scratch, off_carry, off_orders, off_counts, off_sort, total;
    int fwd_blocks, rev_blocks, rep_blocks;
    long long nseg;
};

fte_status adj_layout(int device, const fte_grid* g, unsigned long long n, long long n_steps, int K, bool sorting,
                      AdjLayout* L)
{
    const int sms = device_sms(device);
    if (sms <= 0) return fail(FTE_ECUDA, "cannot query device %d", device);
    int pf = 0, pr = 0, pp = 0, cur = 0;
    FTE_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != device) FTE_CUDA(cudaSetDevice(device), "cudaSetDevice");
    const int pair = g->layout == FTE_LAYOUT_PAIR;
    cudaError_t e = adjoint_blocks(g->dtype, pair, 0, &pf);
    if (e == cudaSuccess) e = adjoint_blocks(g->dtype, pair, 1, &pr);
    if (e == cudaSuccess) e = adjoint_blocks(g->dtype, pair, 2, &pp);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (pf < 1 || pr < 1 || pp < 1) return fail(FTE_ENOTSUP, "adjoint kernels do not fit on an SM");
    L->fwd_blocks = sms * pf;
    L->rev_blocks = sms * pr;
    L->rep_blocks = sms * pp;
    L->nseg = n_steps > 0 ? (n_steps + K - 1) / K : 1;
    const size_t nn = n ? n : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = (off + bytes + 255) & ~(size_t)255; return o; };
    L->off_fetch = take(kFetchBytes);
    L->off_norm = take(64);
    L->off_npart = take(kNormPartials * sizeof(double));
    L->off_normd = take(64);
    L->off_ndpart = take(256 * sizeof(double));
    L->off_table = take((size_t)(n_steps > 0 ? n_steps : 1) * sizeof(StepEntry));
    L->off_ckpt = take((size_t)L->nseg * 5 * nn * sizeof(float));
    L->off_ndead = take(nn * sizeof(int));
    L->off_jpart = take(nn * sizeof(double));
    L->off_adj = take(kAdjRows * nn * sizeof(float));
    L->off_scratch = take((size_t)K * 5 * nn * sizeof(float));    // a segment's states, per particle
    L->off_carry = take(5 * nn * sizeof(float));
    const long long nch = sorting ? (K + kAdjChunk - 1) / kAdjChunk : 1;
    L->off_orders = take(sorting ? (size_t)nch * nn * sizeof(uint32_t) : 0);   // each chunk's order
    L->off_counts = take((size_t)nch * sizeof(unsigned));
    fte_background tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.grid = *g;
    L->off_sort = take(sorting ? sort_scratch_bytes(make_gridk(&tmp), nn) : 0);
    L->total = off;
    return FTE_OK;
}

fte_status adj_check(const fte_particles* P, const fte_background* bg, const fte_params* prm,
                     const fte_smooth_obs* obs, int64_t n_start, int64_t n_end, int K, const void* ws)
{
    if (!P || !prm || !obs) return fail(FTE_EINVAL, "NULL particles, params or observable");
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    s = check_params(prm);
    if (s != FTE_OK) return s;
    if (!(prm->lambda_par > 0.0)) return fail(FTE_EINVAL, "lambda_par must be > 0");
    if (prm->dmumu == 0 && !(prm->q > 1.0 && prm->q <= 2.0 && prm->H >= 0.0)) return fail(FTE_EINVAL, "need 1 < q <= 2, H >= 0");
    if (prm->dmumu == 1 && !(prm->eps > 0.0)) return fail(FTE_EINVAL, "eps must be > 0");
    if (prm->lambda_perp > 0.0) return fail(FTE_ENOTSUP, "the adjoint needs lambda_perp = 0");
    if (prm->p_ref > 0.0 && prm->alpha != 0.0) return fail(FTE_ENOTSUP, "the adjoint needs lambda independent of p");
    if (!(obs->sigma_r > 0.0 && obs->sigma_lnE > 0.0 && obs->sigma_t > 0.0 && obs->e_c > 0.0))
        return fail(FTE_EINVAL, "observable widths and e_c must be > 0");
    if (!(obs->lr_window <= 1e30)) return fail(FTE_EINVAL, "lr_window must be finite");
    if (K < 1 || K > 65536) return fail(FTE_EINVAL, "checkpoint_every must be in [1, 65536]");
    if (n_end < n_start || n_start < 0) return fail(FTE_EINVAL, "need 0 <= n_start <= n_end");
    if (n_end - n_start > 0x7FFFFFFFll) return fail(FTE_EINVAL, "more than 2^31 - 1 steps");
    if (n_end > 0xFFFFFFFFll) return fail(FTE_EINVAL, "step index exceeds 32 bits");
    if (!ws) return fail(FTE_EINVAL, "NULL workspace");
    if (!P->x || !P->y || !P->z || !P->mu || !P->p || !P->w || !P->id || !P->status)
        return fail(FTE_EINVAL, "NULL particle array");
    return FTE_OK;
}

// Kernel arguments shared by both passes; launches the time table and the
// normalisation integrals when `setup` is set.
fte_status adj_args(const fte_particles* P, const fte_background* bg, const fte_params* prm,
                    const fte_smooth_obs* obs, int64_t n_start, int64_t n_end, int K, char* w, const AdjLayout& L,
                    double* dev_out, bool setup, cudaStream_t st, AdvanceArgs* a, AdjK* k)
{
    const long long nsteps = n_end - n_start;
    double* norm = (double*)(w + L.off_norm);
    double* normd = (double*)(w + L.off_normd);
    StepTableArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.tab = (StepEntry*)(w + L.off_table);
    ta.n0 = n_start; ta.count = nsteps; ta.t0 = prm->t0; ta.dt = prm->dt;
    ta.n_snap = bg->grid.n_snap; ta.periodic = bg->grid.periodic; ta.ring = bg->grid.ring;
    ta.t_snap0 = bg->grid.t_snap0; ta.dt_snap = bg->grid.dt_snap;
    if (setup) {
        FTE_CUDA(launch_norm(prm->dmumu, prm->q, prm->H, prm->eps, norm, (double*)(w + L.off_npart), st), "norm launch");
        FTE_CUDA(launch_norm_derivs(prm->dmumu, prm->q, prm->H, prm->eps, normd, (double*)(w + L.off_ndpart), st),
                 "norm derivative launch");
        if (nsteps > 0) FTE_CUDA(launch_step_table(ta, st), "step table launch");
    }
    memset(a, 0, sizeof(*a));
    a->g = make_gridk(bg);
    a->prm.dmumu = prm->dmumu; a->prm.p_update = prm->p_update; a->prm.kappa_drift = prm->kappa_drift;
    a->prm.dvdt_term = prm->dvdt_term;
    a->prm.lambda_par = (float)prm->lambda_par; a->prm.p_ref = (float)prm->p_ref; a->prm.alpha = (float)prm->alpha;
    a->prm.inv_lambda_par = (float)(1.0 / prm->lambda_par);
    a->prm.q = (float)prm->q; a->prm.H = (float)prm->H; a->prm.eps = (float)prm->eps;
    a->prm.mu_floor = (float)prm->mu_floor; a->prm.lambda_perp = 0.f;
    a->prm.dt = (float)prm->dt; a->prm.seed = prm->seed; a->prm.set_id = prm->set_id;
    a->x = P->x; a->y = P->y; a->z = P->z; a->mu = P->mu; a->p = P->p; a->w = P->w; a->id = P->id;
    a->status = P->status;
    a->n_particles = P->count;
    a->n_start = n_start; a->n_end = n_end; a->n_table0 = n_start;
    a->table = ta.tab;
    a->norm = norm;
    a->nbins = 1;
    a->fetch = (unsigned long long*)(w + L.off_fetch);
    a->fetch_slots = bg->grid.dtype == FTE_F32 ? kFetchSlots : 0u;
    memset(k, 0, sizeof(*k));
    k->K = K;
    k->ckpt = (float*)(w + L.off_ckpt);
    k->scratch = (float*)(w + L.off_scratch);
    k->carry = (float*)(w + L.off_carry);
    k->adj = (float*)(w + L.off_adj);
    k->n_dead = (int*)(w + L.off_ndead);
    k->J_part = (double*)(w + L.off_jpart);
    k->out = dev_out;
    k->normd = normd;
    k->r_o = (float)obs->r_o; k->inv_sr = (float)(1.0 / obs->sigma_r);
    k->inv_ec = (float)(1.0 / obs->e_c); k->inv_se = (float)(1.0 / obs->sigma_lnE);
    k->t_c = obs->t_c; k->inv_st = 1.0 / obs->sigma_t; k->t0 = prm->t0; k->dt = prm->dt;
    k->c0 = (float)((prm->t0 - obs->t_c) / obs->sigma_t);
    k->cstep = (float)(prm->dt / obs->sigma_t);
    k->lr_window = obs->lr_window < 0.0 ? (prm->dmumu == 2 ? 0.f : 4.f) : (float)obs->lr_window;
    return FTE_OK;
}

// A pool of at least one wave of the forward kernel's threads is advanced, in both
// passes, as two halves, each with its own region of the workspace (its own strides,
// orders, checkpoints and counters), on the caller's stream and a second stream forked
// from and joined back to it, as fte_advance does with its half-pools: one half's
// launches fill the SMs that the end of the other half's launches leaves idle.  Every
// particle's result is unchanged (only the order of the FP64 sums of the totals is
// not).  The split depends only on the pool, the device and whether reordering is on,
// so a forward and a reverse pass over the same pool lay out the workspace alike.
struct AdjPlan {
    int halves;
    unsigned long long base[2], cnt[2];
    AdjLayout L[2];
    size_t off[2], total;
};

fte_status adj_plan(int device, const fte_grid* g, unsigned long long n, long long n_steps, int K, bool sorting,
                    AdjPlan* p)
{
    AdjLayout full;
    fte_status s = adj_layout(device, g, n, n_steps, K, sorting, &full);
    if (s != FTE_OK) return s;
    const unsigned long long wave = (unsigned long long)full.fwd_blocks * 256ull;
    p->base[0] = p->base[1] = 0;
    p->cnt[1] = 0;
    p->off[0] = p->off[1] = 0;
    if (!sorting || n < wave || n < 2) {
        p->halves = 1;
        p->cnt[0] = n;
        p->L[0] = full;
        p->total = full.total;
        return FTE_OK;
    }
    p->halves = 2;
    p->cnt[0] = n / 2;
    p->base[1] = n / 2;
    p->cnt[1] = n - n / 2;
    for (int h = 0; h < 2; ++h) {
        s = adj_layout(device, g, p->cnt[h], n_steps, K, sorting, &p->L[h]);
        if (s != FTE_OK) return s;
    }
    p->off[1] = (p->L[0].total + 255) & ~(size_t)255;
    p->total = p->off[1] + p->L[1].total;
    return FTE_OK;
}

// The particles [base, base + cnt) of P as a pool of their own.
fte_particles sub_pool(const fte_particles* P, unsigned long long base, unsigned long long cnt)
{
    fte_particles h = *P;
    h.x += base; h.y += base; h.z += base; h.mu += base; h.p += base; h.w += base;
    h.id += base; h.status += base;
    h.count = cnt;
    h.capacity = cnt;
    return h;
}

// A second stream that starts after the work already on `st`.
fte_status fork_side(cudaStream_t st, SideStream* side)
{
    FTE_CUDA(cudaStreamCreateWithFlags(&side->s, cudaStreamNonBlocking), "stream create");
    FTE_CUDA(cudaEventCreateWithFlags(&side->fork, cudaEventDisableTiming), "event create");
    FTE_CUDA(cudaEventCreateWithFlags(&side->join, cudaEventDisableTiming), "event create");
    FTE_CUDA(cudaEventRecord(side->fork, st), "fork");
    FTE_CUDA(cudaStreamWaitEvent(side->s, side->fork, 0), "fork");
    return FTE_OK;
}

// `st` waits for everything enqueued on the second stream.
fte_status join_side(cudaStream_t st, SideStream* side)
{
    FTE_CUDA(cudaEventRecord(side->join, side->s), "join");
    FTE_CUDA(cudaStreamWaitEvent(st, side->join, 0), "join");
    return FTE_OK;
}

// Mean ln E of dN/dE ~ E^-gamma on [e1, e2].
double mean_ln_energy(double e1, double e2, double gamma)
{
    const double a = log(e1), b = log(e2);
    if (fabs(gamma - 1.0) < 1e-12) return 0.5 * (a + b);
    const double s = 1.0 - gamma;
    const double Z = (exp(s * b) - exp(s * a)) / s;
    const double F = exp(s * b) * (b / s - 1.0 / (s * s)) - exp(s * a) * (a / s - 1.0 / (s * s));
    return F / Z;
}

}  // namespace

extern "C" {

size_t fte_adjoint_workspace_bytes(int device, const fte_grid* g, uint64_t n_particles, int64_t n_steps,
                                   int checkpoint_every)
{
    if (check_grid(g) != FTE_OK || n_steps < 0 || checkpoint_every < 1) return 0;
    AdjPlan plan;
    if (adj_plan(device, g, n_particles, n_steps, checkpoint_every, true, &plan) != FTE_OK) return 0;
    return plan.total;
}

fte_status fte_adjoint_forward(fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_smooth_obs* obs, int64_t n_start, int64_t n_end, int checkpoint_every,
                               double* dev_out, double* dev_J_particle, void* ws, size_t ws_bytes, void* stream)
{
    fte_status s = adj_check(P, bg, prm, obs, n_start, n_end, checkpoint_every, ws);
    if (s != FTE_OK) return s;
    if (!dev_out) return fail(FTE_EINVAL, "NULL output");
    int device = 0;
    FTE_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    const bool sorting = prm->sort_every > 0;
    AdjPlan plan;
    s = adj_plan(device, &bg->grid, P->count, n_end - n_start, checkpoint_every, sorting, &plan);
    if (s != FTE_OK) return s;
    if (ws_bytes < plan.total) return fail(FTE_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, plan.total);
    cudaStream_t st = (cudaStream_t)stream;
    FTE_CUDA(cudaMemsetAsync(dev_out, 0, (1 + FTE_NGRAD) * sizeof(double), st), "output reset");
    if (P->count == 0) return FTE_OK;
    // the halves share the caller's stream while it is being captured into a graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FTE_CUDA(cudaStreamIsCapturing(st, &cap), "capture query");
    const bool forked = plan.halves == 2 && cap == cudaStreamCaptureStatusNone;
    SideStream side;
    cudaStream_t hs[2] = {st, st};
    if (forked) {
        s = fork_side(st, &side);
        if (s != FTE_OK) return s;
        hs[1] = side.s;
    }
    const int H = plan.halves;
    fte_particles ph[2];
    AdvanceArgs a[2];
    AdjK k[2];
    SortArgs sa[2];
    for (int h = 0; h < H; ++h) {
        ph[h] = sub_pool(P, plan.base[h], plan.cnt[h]);
        char* w = (char*)ws + plan.off[h];
        s = adj_args(&ph[h], bg, prm, obs, n_start, n_end, checkpoint_every, w, plan.L[h], dev_out, true, hs[h],
                     &a[h], &k[h]);
        if (s != FTE_OK) return s;
        FTE_CUDA(cudaMemsetAsync(k[h].n_dead, 0, ph[h].count * sizeof(int), hs[h]), "step count reset");
        FTE_CUDA(cudaMemsetAsync(k[h].J_part, 0, ph[h].count * sizeof(double), hs[h]), "observable reset");
        memset(&sa[h], 0, sizeof(SortArgs));
        if (sorting) {
            sort_carve(a[h].g, ph[h].count, w + plan.L[h].off_sort, &sa[h]);
            sa[h].g = a[h].g;
            sa[h].x = ph[h].x; sa[h].y = ph[h].y; sa[h].z = ph[h].z; sa[h].mu = ph[h].mu;
            sa[h].status = ph[h].status; sa[h].n = ph[h].count;
            a[h].order = sa[h].order;
            a[h].n_order = sa[h].hist + sa[h].nb;
        }
    }
    // each segment in launches of sort_every steps (reordered before each, as the plain
    // step kernel is); the first launch of a segment stores its checkpoint.  The halves'
    // launches alternate, so that both streams always have work queued.
    const long long sub = sorting ? (prm->sort_every < checkpoint_every ? prm->sort_every : checkpoint_every)
                                  : checkpoint_every;
    for (long long seg = 0; seg < plan.L[0].nseg && n_end > n_start; ++seg) {
        const long long s0 = n_start + seg * checkpoint_every;
        const long long s1 = s0 + checkpoint_every < n_end ? s0 + checkpoint_every : n_end;
        for (long long c0 = s0; c0 < s1; c0 += sub) {
            for (int h = 0; h < H; ++h) {
                k[h].seg = (int)seg;
                a[h].n_start = c0;
                a[h].n_end = c0 + sub < s1 ? c0 + sub : s1;
                k[h].ckpt_on = c0 == s0;
                if (sorting) FTE_CUDA(launch_sort(sa[h], hs[h]), "sort launch");
                FTE_CUDA(cudaMemsetAsync(a[h].fetch, 0, kFetchBytes, hs[h]), "fetch reset");
                FTE_CUDA(launch_adjoint_forward(a[h], k[h], plan.L[h].fwd_blocks, hs[h]), "adjoint forward launch");
            }
        }
    }
    for (int h = 0; h < H; ++h)
        if (dev_J_particle)
            FTE_CUDA(cudaMemcpyAsync(dev_J_particle + plan.base[h], k[h].J_part, ph[h].count * sizeof(double),
                                     cudaMemcpyDeviceToDevice, hs[h]),
                     "per-particle observable copy");
    if (forked) return join_side(st, &side);
    return FTE_OK;
}

fte_status fte_adjoint_reverse(const fte_particles* P, const fte_background* bg, const fte_params* prm,
                               const fte_smooth_obs* obs, const fte_inject_spec* spec, int64_t n_start,
                               int64_t n_end, int checkpoint_every, double* dev_out, float* dev_per_particle,
                               void* ws, size_t ws_bytes, void* stream)
{
    fte_status s = adj_check(P, bg, prm, obs, n_start, n_end, checkpoint_every, ws);
    if (s != FTE_OK) return s;
    if (!dev_out) return fail(FTE_EINVAL, "NULL output");
    if (spec && spec->energy == 1 && !(spec->e1 > 0.0 && spec->e2 > spec->e1))
        return fail(FTE_EINVAL, "need 0 < e1 < e2");
    int device = 0;
    FTE_CUDA(cudaGetDevice(&device), "cudaGetDevice");
    const bool sorting = prm->sort_every > 0;
    AdjPlan plan;
    s = adj_plan(device, &bg->grid, P->count, n_end - n_start, checkpoint_every, sorting, &plan);
    if (s != FTE_OK) return s;
    if (ws_bytes < plan.total) return fail(FTE_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, plan.total);
    cudaStream_t st = (cudaStream_t)stream;
    FTE_CUDA(cudaMemsetAsync(dev_out + 1, 0, FTE_NGRAD * sizeof(double), st), "output reset");
    if (P->count == 0) return FTE_OK;
    // the halves share the caller's stream while it is being captured into a graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FTE_CUDA(cudaStreamIsCapturing(st, &cap), "capture query");
    const bool forked = plan.halves == 2 && cap == cudaStreamCaptureStatusNone;
    SideStream side;
    cudaStream_t hs[2] = {st, st};
    if (forked) {
        s = fork_side(st, &side);
        if (s != FTE_OK) return s;
        hs[1] = side.s;
    }
    const int H = plan.halves;
    fte_particles ph[2];
    AdvanceArgs a[2];
    AdjK k[2];
    SortArgs sa[2];
    uint32_t* orders[2];
    unsigned* counts[2];
    for (int h = 0; h < H; ++h) {
        ph[h] = sub_pool(P, plan.base[h], plan.cnt[h]);
        char* w = (char*)ws + plan.off[h];
        s = adj_args(&ph[h], bg, prm, obs, n_start, n_end, checkpoint_every, w, plan.L[h], dev_out, false, hs[h],
                     &a[h], &k[h]);
        if (s != FTE_OK) return s;
        k[h].per_particle = dev_per_particle ? dev_per_particle + plan.base[h] * (1 + FTE_NGRAD) : nullptr;
        if (spec && spec->energy == 1) {
            k[h].score_on = 1;
            k[h].mean_lnE = mean_ln_energy(spec->e1, spec->e2, spec->gamma);
        }
        const size_t n = ph[h].count;
        if (k[h].per_particle)
            FTE_CUDA(cudaMemsetAsync(k[h].per_particle, 0, n * (1 + FTE_NGRAD) * sizeof(float), hs[h]),
                     "per-particle reset");
        FTE_CUDA(cudaMemsetAsync(k[h].adj, 0, kAdjRows * n * sizeof(float), hs[h]), "adjoint reset");
        memset(&sa[h], 0, sizeof(SortArgs));
        if (sorting) {
            sort_carve(a[h].g, n, w + plan.L[h].off_sort, &sa[h]);
            sa[h].g = a[h].g;
            sa[h].steps = k[h].n_dead;
            sa[h].n = n;
            a[h].order = sa[h].order;
            a[h].n_order = sa[h].hist + sa[h].nb;
        }
        orders[h] = (uint32_t*)(w + plan.L[h].off_orders);
        counts[h] = (unsigned*)(w + plan.L[h].off_counts);
    }
    // every segment from the last: replay its chunks forwards, then run the VJPs over
    // its chunks backwards; each chunk's particles (those alive at its start) are
    // reordered by their position there, and its backward launch reuses that order.  The
    // halves' launches alternate, so that both streams always have work queued.
    const long long chunk = sorting ? (kAdjChunk < checkpoint_every ? kAdjChunk : checkpoint_every) : checkpoint_every;
    for (long long seg = plan.L[0].nseg - 1; seg >= 0; --seg) {
        const long long n0 = n_start + seg * checkpoint_every;
        const long long se = n0 + checkpoint_every < n_end ? n0 + checkpoint_every : n_end;
        const long long nch = (se - n0 + chunk - 1) / chunk;
        for (long long q = 0; q < nch; ++q) {
            for (int h = 0; h < H; ++h) {
                const size_t n = ph[h].count;
                k[h].seg = (int)seg;
                k[h].last = seg == 0;
                k[h].c_start = n0 + q * chunk;
                k[h].c_end = k[h].c_start + chunk < se ? k[h].c_start + chunk : se;
                if (sorting) {
                    const float* c = q == 0 ? k[h].ckpt + (size_t)seg * 5 * n : k[h].carry;
                    sa[h].x = c; sa[h].y = c + n; sa[h].z = c + 2 * n; sa[h].mu = c + 3 * n;
                    sa[h].steps_min = k[h].c_start - n_start;
                    sa[h].order = orders[h] + (size_t)q * n;
                    FTE_CUDA(launch_sort(sa[h], hs[h]), "sort launch");
                    FTE_CUDA(cudaMemcpyAsync(counts[h] + q, sa[h].hist + sa[h].nb, sizeof(unsigned),
                                             cudaMemcpyDeviceToDevice, hs[h]),
                             "order count");
                    a[h].order = sa[h].order;
                    a[h].n_order = counts[h] + q;
                }
                FTE_CUDA(cudaMemsetAsync(a[h].fetch, 0, kFetchBytes, hs[h]), "fetch reset");
                FTE_CUDA(launch_adjoint_replay(a[h], k[h], plan.L[h].rep_blocks, hs[h]), "adjoint replay launch");
            }
        }
        for (long long q = nch - 1; q >= 0; --q) {
            for (int h = 0; h < H; ++h) {
                k[h].c_start = n0 + q * chunk;
                k[h].c_end = k[h].c_start + chunk < se ? k[h].c_start + chunk : se;
                if (sorting) {
                    a[h].order = orders[h] + (size_t)q * ph[h].count;
                    a[h].n_order = counts[h] + q;
                }
                FTE_CUDA(cudaMemsetAsync(a[h].fetch, 0, kFetchBytes, hs[h]), "fetch reset");
                FTE_CUDA(launch_adjoint_back(a[h], k[h], plan.L[h].rev_blocks, hs[h]), "adjoint backward launch");
            }
        }
    }
    if (forked) return join_side(st, &side);
    return FTE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Snapshot streaming through a ring of resident slots.
// ---------------------------------------------------------------------------
#include <vector>

namespace {

struct Run {
    int64_t a, b, key;     // steps [a, b); key >= 0: pair (key, key + 1); key < 0: frozen at -1 - key
};

// The snapshot pair of every step, by the step table's own rule (double
// precision, each operation rounded: the host code is built without contraction).
void stream_runs(const fte_grid* g, const fte_params* prm, int64_t n0, int64_t n1, std::vector<Run>& runs)
{
    runs.clear();
    for (int64_t n = n0; n < n1; ++n) {
        int64_t key = -1;
        if (g->n_snap > 1) {
            const double t = prm->t0 + (double)n * prm->dt;
            const double tau = (t - g->t_snap0) / g->dt_snap;
            if (g->periodic) key = (int64_t)floor(tau);
            else if (tau < 0.0) key = -1;
            else if (tau >= (double)(g->n_snap - 1)) key = -1 - (int64_t)(g->n_snap - 1);
            else key = (int64_t)floor(tau);
        }
        if (!runs.empty() && runs.back().key == key && runs.back().b == n) runs.back().b = n + 1;
        else runs.push_back(Run{n, n + 1, key});
    }
}

int64_t pmod(int64_t u, int64_t m) { return ((u % m) + m) % m; }

// A ring slot receives host snapshots (FP32 cell records) directly, or through
// a staging snapshot converted into the slot's storage form.
bool converts(const fte_grid& g) { return g.dtype != FTE_F32 || g.layout != FTE_LAYOUT_CELL; }

size_t host_snapshot_bytes(const fte_grid& g) { return snapshot_records(&g) * FTE_REC * sizeof(float); }

// Copy host snapshot `logical` into `dst` (FP32 cell records) on `xs` and, for
// AMR, refill the ghost layer of that one snapshot.
cudaError_t upload_f32(const fte_background* bg, const void* host_snapshots, int64_t logical, float* dst,
                       cudaStream_t xs)
{
    const fte_grid& g = bg->grid;
    const size_t bytes = host_snapshot_bytes(g);
    cudaError_t e = cudaMemcpyAsync(dst, (const char*)host_snapshots + (size_t)logical * bytes, bytes,
                                    cudaMemcpyHostToDevice, xs);
    if (e == cudaSuccess && g.amr_levels > 0) {
        GridK one = make_gridk(bg);
        one.dtype = FTE_F32;
        one.pair = 0;
        one.fields = dst;
        e = launch_amr_ghosts(one, 1, g.r_min, g.r_max, g.th_min, g.th_max, xs);
    }
    return e;
}

// Bring unwrapped snapshot u into its ring slot on stream `xs`: straight into an
// FP32 cell-layout slot, otherwise into `staging` and converted from there
// (16-bit: with the scales already in the header).
cudaError_t load_slot(const fte_background* bg, const void* host_snapshots, int64_t u, float* staging,
                      cudaStream_t xs)
{
    const fte_grid& g = bg->grid;
    const size_t nrec = snapshot_records(&g);
    const int64_t slot = pmod(u, g.ring);
    const int64_t logical = g.periodic ? pmod(u, g.n_snap) : u;
    const size_t head = g.dtype == FTE_F32 ? 0 : FTE_HHDR * sizeof(float);
    char* slot_ptr = const_cast<char*>(reinterpret_cast<const char*>(bg->fields)) + head +
                     (size_t)slot * nrec * record_bytes(&g);
    if (!converts(g)) return upload_f32(bg, host_snapshots, logical, reinterpret_cast<float*>(slot_ptr), xs);
    cudaError_t e = upload_f32(bg, host_snapshots, logical, staging, xs);
    if (e != cudaSuccess) return e;
    return launch_convert(staging, (long long)nrec, row_cells(&g), g.dtype, g.layout == FTE_LAYOUT_PAIR,
                          bg->fields, slot_ptr, xs);
}

fte_status check_stream(const fte_background* bg, const void* host_snapshots, const int64_t* slot_state,
                        const void* staging, size_t staging_bytes)
{
    fte_status s = check_background(bg);
    if (s != FTE_OK) return s;
    if (bg->grid.ring < 2) return fail(FTE_EINVAL, "streaming needs a ring background (grid.ring >= 2)");
    if (!host_snapshots || !slot_state) return fail(FTE_EINVAL, "NULL argument");
    if (converts(bg->grid)) {
        if (!staging) return fail(FTE_EINVAL, "a 16-bit or pair-layout ring needs a staging buffer");
        if ((uintptr_t)staging % 32) return fail(FTE_EINVAL, "staging buffer must be 32-byte aligned");
        if (staging_bytes < host_snapshot_bytes(bg->grid))
            return fail(FTE_ENOMEM, "staging buffer has %zu bytes, needs %zu", staging_bytes,
                        host_snapshot_bytes(bg->grid));
    }
    return FTE_OK;
}

}  // namespace

extern "C" {

size_t fte_snapshot_bytes(const fte_grid* g)
{
    if (check_grid(g) != FTE_OK) return 0;
    return host_snapshot_bytes(*g);
}

size_t fte_stream_staging_bytes(const fte_grid* g)
{
    if (check_grid(g) != FTE_OK || !converts(*g)) return 0;
    return host_snapshot_bytes(*g);
}

fte_status fte_stream_scales(const fte_background* bg, const void* host_snapshots, void* staging,
                             size_t staging_bytes, void* stream)
{
    int64_t unused = -1;
    fte_status s = check_stream(bg, host_snapshots, &unused, staging, staging_bytes);
    if (s != FTE_OK) return s;
    const fte_grid& g = bg->grid;
    if (g.dtype == FTE_F32) return fail(FTE_EINVAL, "FP32 backgrounds have no scales");
    cudaStream_t st = (cudaStream_t)stream;
    float* hdr = const_cast<float*>(bg->fields);
    float* stage = reinterpret_cast<float*>(staging);
    for (int u = 0; u < g.n_snap; ++u) {
        FTE_CUDA(upload_f32(bg, host_snapshots, u, stage, st), "snapshot copy");
        FTE_CUDA(launch_scales(stage, (long long)snapshot_records(&g), hdr, u == 0, u == g.n_snap - 1, st),
                 "scale launch");
    }
    return FTE_OK;
}

fte_status fte_stream_plan(const fte_grid* g, const fte_params* prm, int64_t n_start, int64_t n_end,
                           int64_t* out, int64_t max_runs, int64_t* count)
{
    fte_status s = check_grid(g);
    if (s != FTE_OK) return s;
    if (!prm || !count || (max_runs > 0 && !out)) return fail(FTE_EINVAL, "NULL argument");
    if (!(prm->dt > 0.0)) return fail(FTE_EINVAL, "dt must be > 0");
    if (n_end < n_start || n_start < 0) return fail(FTE_EINVAL, "need 0 <= n_start <= n_end");
    std::vector<Run> runs;
    stream_runs(g, prm, n_start, n_end, runs);
    *count = (int64_t)runs.size();
    for (int64_t k = 0; k < (int64_t)runs.size() && k < max_runs; ++k) {
        out[3 * k] = runs[k].a; out[3 * k + 1] = runs[k].b; out[3 * k + 2] = runs[k].key;
    }
    if ((int64_t)runs.size() > max_runs) return fail(FTE_ENOMEM, "%zu runs, room for %lld", runs.size(), (long long)max_runs);
    return FTE_OK;
}

fte_status fte_stream_load(const fte_background* bg, const void* host_snapshots, int64_t u, int64_t* slot_state,
                           void* staging, size_t staging_bytes, void* stream)
{
    fte_status s = check_stream(bg, host_snapshots, slot_state, staging, staging_bytes);
    if (s != FTE_OK) return s;
    if (!bg->grid.periodic && (u < 0 || u >= bg->grid.n_snap)) return fail(FTE_EINVAL, "snapshot %lld out of range", (long long)u);
    FTE_CUDA(load_slot(bg, host_snapshots, u, reinterpret_cast<float*>(staging), (cudaStream_t)stream),
             "snapshot copy");
    slot_state[pmod(u, bg->grid.ring)] = u;
    return FTE_OK;
}

fte_status fte_advance_streamed(fte_particles* P, const fte_background* bg, const void* host_snapshots,
                                const fte_params* prm, const fte_tally_buf* t, int64_t n_start, int64_t n_end,
                                int64_t* slot_state, void* staging, size_t staging_bytes, void* ws,
                                size_t ws_bytes, void* compute_stream, void* copy_stream)
{
    fte_status s = check_stream(bg, host_snapshots, slot_state, staging, staging_bytes);
    if (s != FTE_OK) return s;
    const fte_grid& g = bg->grid;
    if (!prm) return fail(FTE_EINVAL, "NULL params");
    if (!(prm->dt > 0.0)) return fail(FTE_EINVAL, "dt must be > 0");
    if (n_end < n_start || n_start < 0) return fail(FTE_EINVAL, "need 0 <= n_start <= n_end");
    std::vector<Run> runs;
    stream_runs(&g, prm, n_start, n_end, runs);
    const int R = g.ring;
    cudaStream_t cs = (cudaStream_t)compute_stream, xs = (cudaStream_t)copy_stream;
    std::vector<cudaEvent_t> ready(R, nullptr), freed(R, nullptr);
    std::vector<char> has_ready(R, 0), has_freed(R, 0);
    cudaEvent_t fence_c = nullptr, fence_x = nullptr;
    fte_status result = FTE_OK;
    auto fail_cuda = [&](cudaError_t e, const char* what) {
        if (result == FTE_OK) result = cuda_fail(e, what);
        return result;
    };
    auto mk = [&](cudaEvent_t* e) {
        const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
        if (r != cudaSuccess) fail_cuda(r, "event create");
    };
    for (int k = 0; k < R && result == FTE_OK; ++k) { mk(&ready[k]); mk(&freed[k]); }
    if (result == FTE_OK) mk(&fence_c);
    if (result == FTE_OK) mk(&fence_x);
    // order against earlier work: copies after earlier steps, steps after earlier copies
    if (result == FTE_OK) {
        cudaError_t e = cudaEventRecord(fence_c, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, fence_c, 0);
        if (e == cudaSuccess) e = cudaEventRecord(fence_x, xs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, fence_x, 0);
        if (e != cudaSuccess) fail_cuda(e, "stream ordering");
    }
    // bring unwrapped snapshot u into its slot (unless already there - for a
    // periodic sequence, the same snapshot of an earlier period counts - or, for a
    // prefetch, the slot is in use by the current group)
    auto ensure = [&](int64_t u, const std::function<bool(int)>& busy, bool prefetch) {
        if (result != FTE_OK) return;
        const int slot = (int)pmod(u, R);
        if (slot_state[slot] == u) return;
        if (g.periodic && slot_state[slot] >= 0 && pmod(slot_state[slot], g.n_snap) == pmod(u, g.n_snap)) {
            slot_state[slot] = u;
            return;
        }
        if (prefetch && busy(slot)) return;
        if (has_freed[slot]) {
            const cudaError_t e = cudaStreamWaitEvent(xs, freed[slot], 0);
            if (e != cudaSuccess) { fail_cuda(e, "copy wait"); return; }
        }
        cudaError_t e = load_slot(bg, host_snapshots, u, reinterpret_cast<float*>(staging), xs);
        if (e == cudaSuccess) e = cudaEventRecord(ready[slot], xs);
        if (e != cudaSuccess) { fail_cuda(e, "snapshot copy"); return; }
        has_ready[slot] = 1;
        slot_state[slot] = u;
    };
    // Consecutive runs are advanced in groups, one fte_advance call each, ramping up as
    // 1, 1, 2, 4, then kStreamGroupRuns runs per call: every call ends with its two
    // halves joined and a partial reordering chunk, so one call per snapshot interval
    // leaves the GPU idle at each interval's end; the ramp lets the first intervals
    // start as soon as their own snapshots are in, and lets each group's compute cover
    // the copies of the next group's snapshots.  A group's snapshots must fit the ring
    // together, leaving one slot to prefetch into (R >= 3), and its steps the
    // workspace's time table.
    auto run_lo = [](const Run& r) { return r.key >= 0 ? r.key : -1 - r.key; };
    auto run_hi = [](const Run& r) { return r.key >= 0 ? r.key + 1 : -1 - r.key; };
    const int64_t span_max = R >= 3 ? R - 1 : R;
    int device = 0;
    if (result == FTE_OK) {
        const cudaError_t e = cudaGetDevice(&device);
        if (e != cudaSuccess) fail_cuda(e, "cudaGetDevice");
    }
    const size_t ws0 = result == FTE_OK ? fte_workspace_bytes(device, &g, t, P->count, 0) : 0;
    auto fits = [&](int64_t steps) { return ws0 + (size_t)steps * sizeof(StepEntry) + 256 <= ws_bytes; };
    struct Group {
        size_t k, k1;          // runs [k, k1)
        int64_t ulo, uhi;      // the unwrapped snapshots they read
    };
    std::vector<Group> groups;
    for (size_t k = 0; k < runs.size();) {
        const size_t gi = groups.size();
        const size_t want = gi < 2 ? 1 : (gi == 2 ? 2 : (gi == 3 ? 4 : kStreamGroupRuns));
        size_t k1 = k + 1;
        int64_t ulo = run_lo(runs[k]), uhi = run_hi(runs[k]);
        while (k1 < runs.size() && k1 - k < want) {
            const int64_t lo2 = std::min(ulo, run_lo(runs[k1])), hi2 = std::max(uhi, run_hi(runs[k1]));
            if (hi2 - lo2 + 1 > span_max || !fits(runs[k1].b - runs[k].a)) break;
            ulo = lo2; uhi = hi2; ++k1;
        }
        groups.push_back(Group{k, k1, ulo, uhi});
        k = k1;
    }
    for (size_t gi = 0; gi < groups.size() && result == FTE_OK; ++gi) {
        const Group& G = groups[gi];
        auto busy = [&](int slot) { return pmod(slot - G.ulo, R) <= G.uhi - G.ulo; };
        for (int64_t u = G.ulo; u <= G.uhi && result == FTE_OK; ++u) ensure(u, busy, false);
        if (result != FTE_OK) break;
        for (int64_t u = G.ulo; u <= G.uhi; ++u) {
            const int sl = (int)pmod(u, R);
            if (has_ready[sl]) {
                const cudaError_t e = cudaStreamWaitEvent(cs, ready[sl], 0);
                if (e != cudaSuccess) { fail_cuda(e, "compute wait"); break; }
            }
        }
        if (result != FTE_OK) break;
        const fte_status st = fte_advance(P, bg, prm, t, runs[G.k].a, runs[G.k1 - 1].b, ws, ws_bytes, compute_stream);
        if (st != FTE_OK) { result = st; break; }
        for (int64_t u = G.ulo; u <= G.uhi; ++u) {
            const int sl = (int)pmod(u, R);
            const cudaError_t e = cudaEventRecord(freed[sl], cs);
            if (e != cudaSuccess) { fail_cuda(e, "event record"); break; }
            has_freed[sl] = 1;
        }
        if (result != FTE_OK || gi + 1 == groups.size()) break;
        // the next group's snapshots that are not in their slots yet, into the slots that
        // this group does not use, copied while it computes: issued only now, after this
        // group's launches, so that even copy calls that hold the host thread until they
        // are done (where the driver stages them) overlap this group's compute
        const Group& N = groups[gi + 1];
        for (int64_t nx = std::max(N.ulo, G.uhi + 1); nx <= N.uhi && result == FTE_OK; ++nx) {
            if (!g.periodic && nx > g.n_snap - 1) break;
            ensure(nx, busy, true);
        }
    }
    for (int k = 0; k < R; ++k) {
        if (ready[k]) cudaEventDestroy(ready[k]);
        if (freed[k]) cudaEventDestroy(freed[k]);
    }
    if (fence_c) cudaEventDestroy(fence_c);
    if (fence_x) cudaEventDestroy(fence_x);
    return result;
}

}  // extern "C"
