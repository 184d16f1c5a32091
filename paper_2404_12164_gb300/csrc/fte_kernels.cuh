// Kernel declarations and launch arguments shared by the API and kernel files.
#pragma once

#include "fte_device.cuh"

namespace fte {

// Step-kernel modes: one parameter set; an ensemble with all sets' tallies in
// shared memory; an ensemble with FP64 atomics into the global tally.
constexpr int kModeSingle = 0;
constexpr int kModeShared = 1;
constexpr int kModeGlobal = 2;
constexpr int kModeSingleGlobal = 3;   // one parameter set, warp-merged FP64 atomics to the tally

__host__ __device__ constexpr bool single_set(int mode) { return mode == kModeSingle || mode == kModeSingleGlobal; }
__host__ __device__ constexpr bool global_tally(int mode) { return mode == kModeGlobal || mode == kModeSingleGlobal; }

// Per-set transport parameters of an ensemble (everything else is shared).
struct SetK {
    float lambda_par, q, H, eps;
    uint32_t seed, set_id;
};

struct BatchArgs {
    int n_sets, pad;
    unsigned long long end[FTE_MAX_SETS];   // pool entries [end[s-1], end[s]) belong to set s
    SetK set[FTE_MAX_SETS];
};

struct AdvanceArgs {
    GridK g;
    ParamsK prm;
    ObsK obs[FTE_MAX_OBS];
    int n_obs, nbins;
    float *x, *y, *z, *mu, *p, *w;
    const uint32_t* id;
    uint8_t* status;
    unsigned long long n_particles;
    long long n_start, n_end;     // steps advanced by this launch
    long long n_table0;           // step index of table[0]
    const StepEntry* table;
    const double* norm;           // normalisation integral of D_mumu (one per set)
    double* gS;                   // global tally modes: FP64 accumulators [set][bin]
    double* gS2;
    unsigned long long* gC;
    const uint32_t* order;        // alive particles in spatial order (NULL: all, by index)
    const unsigned* n_order;      // number of entries of `order` (device)
    float* part;                  // per-block partial histograms [grid][3][nbins]
    unsigned long long* fetch;    // particle counter for dynamic assignment
    unsigned fetch_slots;         // > 0: `fetch` holds that many per-SM range counters
    int compact;                  // one of two half-pools on two streams: a launch with fewer ordered
                                  // particles than resident threads keeps one per thread (see advance_kernel)
    double* ledger_w;
    unsigned long long* ledger_n;
    double* cls;                  // optional [set][bin][FTE_NCLASS]: S by particle-id class
};

struct SortArgs {
    GridK g;
    const float *x, *y, *z;
    const float* mu;              // pitch-angle cosine (NULL: ordered by position only)
    const uint8_t* status;        // entries with status FTE_ALIVE are ordered ...
    const int* steps;             // ... or, when set, entries with steps[i] > steps_min
    long long steps_min;
    unsigned long long n;
    unsigned* hist;               // bucket counts, then exclusive offsets; total at hist[nb]
    unsigned* tiles;
    int* key;
    int* rank;
    uint32_t* order;
    int nb, ntiles;
};

struct ObsTime {
    double t_lo, t_hi;
    int nt, pad;
};

struct StepTableArgs {
    StepEntry* tab;
    long long n0, count;
    double t0, dt;
    int n_snap, periodic;
    double t_snap0, dt_snap;
    int n_obs;
    int ring;                     // > 0: snapshot u (unwrapped, in time order) is in slot u mod ring
    ObsTime ot[FTE_MAX_OBS];
};

struct ObsOut {
    int kind, ne, nt, off;
    double r, dr, th, dth, dph;
    double e_lo, e_hi, t_lo, t_hi;
};

struct InjectArgs {
    GridK g;
    int n_snap, region, energy, weight, mu_mode, use_divv, divv_snap, max_tries;
    float r, th, ph, r1, r2, th1, th2, ph1, ph2, divv_max, e0, e1, e2, gamma, mu0;
    float spiral, spiral_rb;      // box: longitude = sampled spiral phase - spiral (r - spiral_rb)
    uint32_t seed, set_id, id_base;
    unsigned long long offset, n;
    float *x, *y, *z, *mu, *p, *w;
    uint32_t* id;
    uint8_t* status;
    double* ledger_w;
    unsigned long long* ledger_n;
};

static_assert(sizeof(AdvanceArgs) + sizeof(BatchArgs) <= 4096, "step kernel parameters exceed 4 KB");

// Per-set inputs of the D_mumu normalisation integral.
struct NormSets {
    double q[FTE_MAX_SETS], H[FTE_MAX_SETS], eps[FTE_MAX_SETS];
};

// Pathwise adjoint (fte_adjoint.cu): checkpoints, replay scratch and outputs.
struct AdjK {
    int K;                        // steps between checkpoints
    int score_on;                 // injection-index gradient by the likelihood ratio
    int seg;                      // segment of this launch: steps n_start + seg K ..
    int last;                     // reverse: 1 for the first segment of the run (seg 0)
    int ckpt_on;                  // forward: this launch starts a segment (stores its checkpoint)
    long long c_start, c_end;     // reverse: steps of this launch's chunk of the segment
    float* ckpt;                  // [segment][5][n]: x, y, z, mu, p at n_start + segment K
    float* scratch;               // [K][5][n]: replayed start-of-step states of the segment, at
                                  // each particle's position in its chunk's order (coalesced)
    float* carry;                 // [5][n]: state at the start of the next chunk, by particle
    float* adj;                   // [10][n]: state adjoint (5), parameter adjoint (4) and the observable
                                  // accumulated after the current step (the score terms' weight), between launches
    float lr_window;              // score form for steps whose pitch-angle mean is within this many widths
                                  // of a value landing at mu = 0 (0: pathwise everywhere)
    int* n_dead;                  // [n]: steps each particle took (alive at their start)
    double* J_part;               // [n]: each particle's observable
    double* out;                  // [1 + FTE_NGRAD]: J, then the gradients
    float* per_particle;          // optional [n][1 + FTE_NGRAD]
    const double* normd;          // dI/dq and dI/dH (or dJ/deps) of the normalisation integral
    float r_o, inv_sr, inv_ec, inv_se;
    double t_c, inv_st, t0, dt;   // observable time centre and width; step times t0 + n dt
    float c0, cstep;              // (t0 - t_c) inv_st and dt inv_st: time argument c0 + n cstep
    double mean_lnE;              // mean ln E of the injected spectrum
};

// launchers (return cudaGetLastError())
// step kernel of (kperp, dtype, mode, threads per block); for the single-set modes nt must
// be advance_threads() of the same arguments
cudaError_t launch_advance(const AdvanceArgs& a, const BatchArgs& b, int kperp, int mode, int nt, int blocks,
                           size_t smem, cudaStream_t s);
// resident blocks per SM of a step kernel (`pair`: record layout of a single-set kernel)
cudaError_t advance_occupancy(int kperp, int dtype, int mode, int nt, int pair, int amr, size_t smem,
                              int* blocks_per_sm);
// Builds of the single-set step kernel.  Block AMR with the global tally and no
// cross-field diffusion (its chain of dependent loads, table -> leaf -> records, needs
// more resident warps) runs a register-limited build: FP32 records 5 blocks of 128
// threads per SM (at most 102 registers, 20 warps: 1.997e10 particle-steps/s against
// 1.912e10 with 24 warps at 85 registers and 1.892e10 with 16 unconstrained), 16-bit
// records 3 blocks of 256 (85 registers, 24 warps).  Uniform grids keep the
// unconstrained build of 256 threads in every storage form (under the tighter limits it
// spills: 16-bit storage measured 1.018x FP32 with the 3-block build and 1.069x without).
// advance_threads: threads per block of the build that advance_fn selects.
int advance_threads(int kperp, int dtype, int mode, int amr);
// the ensemble variants live in their own translation unit (fte_batched.cu)
const void* advance_fn_batched(int kperp, int dtype, int mode, int nt, int pair);
cudaError_t launch_advance_batched(const AdvanceArgs& a, const BatchArgs& b, int kperp, int mode, int nt,
                                   int blocks, size_t smem, cudaStream_t s);
cudaError_t launch_reduce(const float* part, int nblk, int nbins, double* S, double* S2,
                          unsigned long long* C, cudaStream_t s);
cudaError_t launch_step_table(const StepTableArgs& a, cudaStream_t s);
// normalisation integral; `part` holds kNormPartials doubles of scratch
constexpr int kNormPartials = 128;
cudaError_t launch_norm(int model, double q, double H, double eps, double* out, double* part,
                        cudaStream_t s);
// the same for n_sets sets at once: out[s], scratch part[n_sets][kNormPartials]
cudaError_t launch_norm_sets(int model, const NormSets& ns, int n_sets, double* out, double* part,
                             cudaStream_t s);
cudaError_t launch_tally_out(const double* S, const double* S2, const unsigned long long* C,
                             const ObsOut& ob, int kind, double* out, cudaStream_t s);
cudaError_t launch_convolve(const double* S, const ObsOut& ob, int kind, const double* src, double* out,
                            cudaStream_t s);
cudaError_t launch_inject(const InjectArgs& a, cudaStream_t s);
// adjoint (fte_adjoint.cu)
// resident blocks per SM of an adjoint kernel (kind 0 forward, 1 backward VJP, 2 replay)
cudaError_t adjoint_blocks(int dtype, int pair, int kind, int* blocks_per_sm);
cudaError_t launch_adjoint_forward(const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s);
cudaError_t launch_adjoint_replay(const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s);
cudaError_t launch_adjoint_back(const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s);
cudaError_t launch_norm_derivs(int model, double q, double H, double eps, double* out, double* part,
                               cudaStream_t s);
// spatial ordering of the alive particles (fte_sort.cu)
size_t sort_scratch_bytes(const GridK& g, unsigned long long n);
void sort_carve(const GridK& g, unsigned long long n, char* p, SortArgs* a);
cudaError_t launch_sort(const SortArgs& a, cudaStream_t s);
// block AMR set-up (fte_amr.cu): status[0] malformed leaves, [1] overlaps,
// [2] uncovered finest blocks, [3] 2:1 nesting violations
cudaError_t launch_amr_table(const GridK& g, int* table, unsigned* status, cudaStream_t s);
cudaError_t launch_amr_ghosts(const GridK& g, int n_snap, double r_min, double r_max, double th_min,
                              double th_max, cudaStream_t s);
// random-sector read probe (fte_probe.cu)
cudaError_t launch_probe_l1(const float* buf, unsigned nrec, int threads, int records, int spread, float* out,
                            cudaStream_t s);
cudaError_t launch_probe(const float* buf, unsigned long long nsec, int threads, int loads, float* out,
                         cudaStream_t s);
// storage conversion of `nrec` FP32 cell records (r-rows of `row` cells): 16-bit
// (scale header + records) in the cell or pair layout, or FP32 pair records
cudaError_t launch_quantize(const float* f32, long long nrec, int row, int dtype, int pair, void* out,
                            cudaStream_t s);
// the two halves of launch_quantize, for one snapshot at a time: per-field
// scales folded over calls (first: zero the header; last: finalise), and the
// conversion of nrec records into `out_recs` with the scales in `hdr`
cudaError_t launch_scales(const float* f32, long long nrec, float* hdr, bool first, bool last, cudaStream_t s);
cudaError_t launch_convert(const float* f32, long long nrec, int row, int dtype, int pair, const float* hdr,
                           void* out_recs, cudaStream_t s);

}  // namespace fte
