// Transport kernels: the per-particle step loop with the fused occupancy tally,
// the FP64 reduction of per-block partial histograms, the FP64 per-step time
// table, the D_mumu normalisation integral and the intensity output.
#include "fte_step.cuh"

namespace fte {

template <int MODE, int LAY>
static const void* single_fn(int kperp, int dtype)
{
    if (dtype == FTE_BF16)
        return kperp ? (const void*)advance_kernel<true, FTE_BF16, MODE, kThreads, LAY>
                     : (const void*)advance_kernel<false, FTE_BF16, MODE, kThreads, LAY>;
    if (dtype == FTE_F16)
        return kperp ? (const void*)advance_kernel<true, FTE_F16, MODE, kThreads, LAY>
                     : (const void*)advance_kernel<false, FTE_F16, MODE, kThreads, LAY>;
    return kperp ? (const void*)advance_kernel<true, FTE_F32, MODE, kThreads, LAY>
                 : (const void*)advance_kernel<false, FTE_F32, MODE, kThreads, LAY>;
}

// the register-limited builds of block AMR (global tally, no cross-field diffusion):
// 16-bit records 3 blocks of 256 threads per SM (at most 85 registers), FP32 records
// 5 blocks of 128 (at most 102)
constexpr int kDenseBlocks = 768 / kThreads;
constexpr int kAmr32Threads = 128;
constexpr int kAmr32Blocks = 5;
template <int LAY>
static const void* dense_fn(int dtype)
{
    if (dtype == FTE_BF16) return (const void*)advance_kernel<false, FTE_BF16, kModeSingleGlobal, kThreads, LAY, kDenseBlocks>;
    if (dtype == FTE_F16) return (const void*)advance_kernel<false, FTE_F16, kModeSingleGlobal, kThreads, LAY, kDenseBlocks>;
    return (const void*)advance_kernel<false, FTE_F32, kModeSingleGlobal, kAmr32Threads, LAY, kAmr32Blocks>;
}

static bool dense_variant(int kperp, int mode, int amr)
{
    return mode == kModeSingleGlobal && !kperp && amr;
}

int advance_threads(int kperp, int dtype, int mode, int amr)
{
    return single_set(mode) && dense_variant(kperp, mode, amr) && dtype == FTE_F32 ? kAmr32Threads : kThreads;
}

// the single-set kernels come in one variant per record layout (pair: 1) and tally
// mode, and for block AMR in a register-limited build
static const void* advance_fn(int kperp, int dtype, int mode, int nt, int pair, int amr)
{
    if (!single_set(mode)) return advance_fn_batched(kperp, dtype, mode, nt, pair);
    if (nt != advance_threads(kperp, dtype, mode, amr)) return nullptr;
    if (dense_variant(kperp, mode, amr)) return pair ? dense_fn<kLayPair>(dtype) : dense_fn<kLayCell>(dtype);
    if (mode == kModeSingleGlobal)
        return pair ? single_fn<kModeSingleGlobal, kLayPair>(kperp, dtype)
                    : single_fn<kModeSingleGlobal, kLayCell>(kperp, dtype);
    return pair ? single_fn<kModeSingle, kLayPair>(kperp, dtype) : single_fn<kModeSingle, kLayCell>(kperp, dtype);
}

cudaError_t advance_occupancy(int kperp, int dtype, int mode, int nt, int pair, int amr, size_t smem,
                              int* blocks_per_sm)
{
    const void* fn = advance_fn(kperp, dtype, mode, nt, pair, amr);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, nt, smem);
}

cudaError_t launch_advance(const AdvanceArgs& a, const BatchArgs& b, int kperp, int mode, int nt, int blocks,
                           size_t smem, cudaStream_t s)
{
    if (!single_set(mode)) return launch_advance_batched(a, b, kperp, mode, nt, blocks, smem, s);
    const void* fn = advance_fn(kperp, a.g.dtype, mode, nt, a.g.pair, a.g.amr > 0);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&a, (void*)&b};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(nt), args, smem, s);
}

// ---------------------------------------------------------------------------
// Quantization of an FP32 background to 16-bit storage with per-field scales:
// (1) largest |value| per field (atomic max of the non-negative float bits),
// (2) zero scales become 1, (3) each record is encoded as the round-to-nearest-
// even of (value / scale), the quotient correctly rounded in FP32.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) maxabs_kernel(const float* __restrict__ f, long long nrec,
                                                     unsigned* hdr)
{
    float m[FTE_NFIELD];
#pragma unroll
    for (int k = 0; k < FTE_NFIELD; ++k) m[k] = 0.f;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrec;
         r += (long long)gridDim.x * blockDim.x) {
        float a[FTE_REC];
#pragma unroll
        for (int q = 0; q < FTE_REC / 8; ++q) ldg8(f + r * FTE_REC + 8 * q, a + 8 * q);
#pragma unroll
        for (int k = 0; k < FTE_NFIELD; ++k) m[k] = fmaxf(m[k], fabsf(a[k]));
    }
#pragma unroll
    for (int k = 0; k < FTE_NFIELD; ++k) {
        float v = m[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(hdr + k, __float_as_uint(v));
    }
}

__global__ void scale_final_kernel(float* hdr)
{
    const int k = threadIdx.x;
    if (k < FTE_HHDR) hdr[k] = (k < FTE_NFIELD) ? (hdr[k] > 0.f ? hdr[k] : 1.f) : 0.f;
}

template <int DT>
__device__ __forceinline__ uint32_t encode16(float v)
{
    if (DT == FTE_BF16) return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    return (uint32_t)__half_as_ushort(__float2half_rn(v));
}

// 16-bit records: cell layout (18 values, padded to FTE_HREC) or pair layout
// (the cell's 18 values, then those of its upper r-neighbour - zero at the end of
// an r-row of `row` cells - padded to kPairHRec).
template <int DT, bool PAIR>
__global__ void __launch_bounds__(256) encode_kernel(const float* __restrict__ f, long long nrec, int row,
                                                     const float* __restrict__ hdr, uint32_t* out)
{
    constexpr int kWords = (PAIR ? kPairHRec : FTE_HREC) / 2;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    uint32_t w[kWords];
#pragma unroll
    for (int k = 0; k < kWords; ++k) w[k] = 0u;
    const bool hi_in_row = (r % row) != row - 1;
#pragma unroll
    for (int c = 0; c < (PAIR ? 2 : 1); ++c) {
        if (c == 1 && !hi_in_row) break;
        float a[FTE_REC];
#pragma unroll
        for (int q = 0; q < FTE_REC / 8; ++q) ldg8(f + (r + c) * FTE_REC + 8 * q, a + 8 * q);
#pragma unroll
        for (int k = 0; k < FTE_NFIELD; ++k) {
            const uint32_t h = encode16<DT>(__fdiv_rn(a[k], __ldg(hdr + k)));
            const int slot = c * FTE_NFIELD + k;
            w[slot >> 1] |= (slot & 1) ? (h << 16) : h;
        }
    }
    uint4* o = reinterpret_cast<uint4*>(out + r * kWords);
#pragma unroll
    for (int q = 0; q < kWords / 4; ++q) o[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

// FP32 pair records from FP32 cell records.
__global__ void __launch_bounds__(256) pair_f32_kernel(const float* __restrict__ f, long long nrec, int row,
                                                       float* out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    float a[kPairRec];
#pragma unroll
    for (int k = 0; k < kPairRec; ++k) a[k] = 0.f;
    float b[FTE_REC];
#pragma unroll
    for (int q = 0; q < FTE_REC / 8; ++q) ldg8(f + r * FTE_REC + 8 * q, b + 8 * q);
#pragma unroll
    for (int k = 0; k < FTE_NFIELD; ++k) a[k] = b[k];
    if ((r % row) != row - 1) {
#pragma unroll
        for (int q = 0; q < FTE_REC / 8; ++q) ldg8(f + (r + 1) * FTE_REC + 8 * q, b + 8 * q);
#pragma unroll
        for (int k = 0; k < FTE_NFIELD; ++k) a[FTE_NFIELD + k] = b[k];
    }
    float4* o = reinterpret_cast<float4*>(out + r * kPairRec);
#pragma unroll
    for (int q = 0; q < kPairRec / 4; ++q) o[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
}

// Per-field scales of FP32 cell records: `first` zeroes the header, each call
// folds nrec records into the running maxima, `last` turns them into scales.
cudaError_t launch_scales(const float* f32, long long nrec, float* hdr, bool first, bool last, cudaStream_t s)
{
    if (first) {
        const cudaError_t e = cudaMemsetAsync(hdr, 0, FTE_HHDR * sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    if (nrec > 0) maxabs_kernel<<<1216, 256, 0, s>>>(f32, nrec, reinterpret_cast<unsigned*>(hdr));
    if (last) scale_final_kernel<<<1, 32, 0, s>>>(hdr);
    return cudaGetLastError();
}

// FP32 cell records into pair and/or 16-bit records (16-bit: with the scales
// already in `hdr`), nrec records starting at `out_recs`.
cudaError_t launch_convert(const float* f32, long long nrec, int row, int dtype, int pair, const float* hdr,
                           void* out_recs, cudaStream_t s)
{
    const long long blocks = (nrec + 255) / 256;
    if (nrec <= 0) return cudaSuccess;
    if (dtype == FTE_F32) {
        if (!pair) return cudaErrorInvalidValue;
        pair_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(f32, nrec, row, reinterpret_cast<float*>(out_recs));
        return cudaGetLastError();
    }
    uint32_t* recs = reinterpret_cast<uint32_t*>(out_recs);
#define FTE_ENC(D, P) encode_kernel<D, P><<<(unsigned)blocks, 256, 0, s>>>(f32, nrec, row, hdr, recs)
    if (dtype == FTE_BF16) { if (pair) FTE_ENC(FTE_BF16, true); else FTE_ENC(FTE_BF16, false); }
    else { if (pair) FTE_ENC(FTE_F16, true); else FTE_ENC(FTE_F16, false); }
#undef FTE_ENC
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float* f32, long long nrec, int row, int dtype, int pair, void* out,
                            cudaStream_t s)
{
    if (dtype == FTE_F32) return launch_convert(f32, nrec, row, dtype, pair, nullptr, out, s);
    float* hdr = reinterpret_cast<float*>(out);
    const cudaError_t e = launch_scales(f32, nrec, hdr, true, true, s);
    if (e != cudaSuccess) return e;
    return launch_convert(f32, nrec, row, dtype, pair, hdr, reinterpret_cast<char*>(out) + FTE_HHDR * sizeof(float), s);
}

// ---------------------------------------------------------------------------
// FP64 sum of the per-block partial histograms into the tally (deterministic
// order: each bin's blocks are summed by 8 warps, then combined in order).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) reduce_kernel(const float* __restrict__ part, int nblk,
                                                     int nbins, double* S, double* S2,
                                                     unsigned long long* C)
{
    __shared__ double rs[8][32], rs2[8][32];
    __shared__ unsigned long long rc[8][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    double s = 0.0, s2 = 0.0;
    unsigned long long c = 0;
    if (b < nbins) {
        for (int k = wid; k < nblk; k += 8) {
            const float* q = part + (size_t)k * 3 * nbins;
            s += (double)q[b];
            s2 += (double)q[nbins + b];
            c += __float_as_uint(q[2 * nbins + b]);
        }
    }
    rs[wid][lane] = s;
    rs2[wid][lane] = s2;
    rc[wid][lane] = c;
    __syncthreads();
    if (wid == 0 && b < nbins) {
        for (int k = 1; k < 8; ++k) { s += rs[k][lane]; s2 += rs2[k][lane]; c += rc[k][lane]; }
        S[b] += s;
        S2[b] += s2;
        C[b] += c;
    }
}

cudaError_t launch_reduce(const float* part, int nblk, int nbins, double* S, double* S2,
                          unsigned long long* C, cudaStream_t s)
{
    reduce_kernel<<<(nbins + 31) / 32, 256, 0, s>>>(part, nblk, nbins, S, S2, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-step time table in FP64: t_n = t0 + n dt, bracketing snapshots and the
// time weight, and the time bin of every observer (rounded operations, no
// contraction, so that edges fall exactly where the definition puts them).
// ---------------------------------------------------------------------------
__global__ void step_table_kernel(const StepTableArgs a)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.count) return;
    const long long n = a.n0 + k;
    const double t = __dadd_rn(a.t0, __dmul_rn((double)n, a.dt));
    StepEntry e;
    e.s0 = 0; e.s1 = 0; e.wt = 0.f; e.two = 0;
    if (a.n_snap > 1) {
        const double tau = __ddiv_rn(__dsub_rn(t, a.t_snap0), a.dt_snap);
        // u0, u1: the snapshots in time order (periodic sequences unwrapped)
        long long u0 = 0, u1 = 0;
        if (a.periodic) {
            const double kf = floor(tau);
            u0 = (long long)kf;
            u1 = u0 + 1;
            e.wt = (float)(tau - kf);
            e.two = 1;
        } else if (tau < 0.0) {
            u0 = u1 = 0;
        } else if (tau >= (double)(a.n_snap - 1)) {
            u0 = u1 = a.n_snap - 1;
        } else {
            const double kf = floor(tau);
            u0 = (long long)kf;
            u1 = u0 + 1;
            e.wt = (float)(tau - kf);
            e.two = 1;
        }
        // storage slot: the snapshot itself, or its place in the ring
        const long long m = a.ring > 0 ? a.ring : a.n_snap;
        e.s0 = (int)(((u0 % m) + m) % m);
        e.s1 = (int)(((u1 % m) + m) % m);
    }
    for (int o = 0; o < FTE_MAX_OBS; ++o) {
        short it = -1;
        if (o < a.n_obs) {
            const ObsTime& ot = a.ot[o];
            const double f = floor(__ddiv_rn(__dmul_rn(__dsub_rn(t, ot.t_lo), (double)ot.nt),
                                             __dsub_rn(ot.t_hi, ot.t_lo)));
            if (f >= 0.0 && f < (double)ot.nt) it = (short)f;
        }
        e.it[o] = it;
    }
    a.tab[k] = e;
}

cudaError_t launch_step_table(const StepTableArgs& a, cudaStream_t s)
{
    const int blocks = (int)((a.count + 255) / 256);
    if (blocks > 0) step_table_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Normalisation of D_mumu from lambda_par: I (quasi-linear) or J (Eq. 5), by
// composite Simpson in FP64 after mu = s^3; 1 for the isotropic form.  Stage 1:
// one node per thread, block sums in a fixed tree order; stage 2: one thread adds
// the block sums in order.
// ---------------------------------------------------------------------------
constexpr int kNormIntervals = 16384;
constexpr int kNormThreads = 256;
constexpr int kNormBlocks = kNormIntervals / kNormThreads + 1;   // nodes 0 .. kNormIntervals
static_assert(kNormBlocks <= kNormPartials, "norm partials");

__global__ void __launch_bounds__(kNormThreads) norm_partial_kernel(int model, double q, double H,
                                                                    double eps, double* part)
{
    __shared__ double sh[kNormThreads];
    const int i = blockIdx.x * kNormThreads + threadIdx.x;
    double f = 0.0;
    if (model != 2 && i <= kNormIntervals) {
        const double h = 1.0 / kNormIntervals;
        const double s = i * h;
        const double m = s * s * s;
        const double den = (model == 0) ? pow(m, q - 1.0) + H : m / (1.0 + m) + eps;
        const double wgt = (i == 0 || i == kNormIntervals) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        f = wgt * 3.0 * s * s * (1.0 - m * m) / den;
    }
    sh[threadIdx.x] = f;
    __syncthreads();
    for (int o = kNormThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void norm_final_kernel(int model, const double* part, double* out)
{
    double acc = 0.0;
    for (int b = 0; b < kNormBlocks; ++b) acc += part[b];
    out[0] = (model == 2) ? 1.0 : acc / (3.0 * kNormIntervals);
}

// one block row per set (blockIdx.y), same quadrature
__global__ void __launch_bounds__(kNormThreads) norm_sets_partial_kernel(int model, const NormSets ns,
                                                                         double* part)
{
    const int s = blockIdx.y;
    __shared__ double sh[kNormThreads];
    const int i = blockIdx.x * kNormThreads + threadIdx.x;
    double f = 0.0;
    if (model != 2 && i <= kNormIntervals) {
        const double h = 1.0 / kNormIntervals;
        const double u = i * h;
        const double m = u * u * u;
        const double den = (model == 0) ? pow(m, ns.q[s] - 1.0) + ns.H[s] : m / (1.0 + m) + ns.eps[s];
        const double wgt = (i == 0 || i == kNormIntervals) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        f = wgt * 3.0 * u * u * (1.0 - m * m) / den;
    }
    sh[threadIdx.x] = f;
    __syncthreads();
    for (int o = kNormThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)s * kNormPartials + blockIdx.x] = sh[0];
}

__global__ void norm_sets_final_kernel(int model, int n_sets, const double* part, double* out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sets) return;
    double acc = 0.0;
    for (int b = 0; b < kNormBlocks; ++b) acc += part[(size_t)s * kNormPartials + b];
    out[s] = (model == 2) ? 1.0 : acc / (3.0 * kNormIntervals);
}

cudaError_t launch_norm_sets(int model, const NormSets& ns, int n_sets, double* out, double* part,
                             cudaStream_t s)
{
    norm_sets_partial_kernel<<<dim3(kNormBlocks, n_sets), kNormThreads, 0, s>>>(model, ns, part);
    norm_sets_final_kernel<<<1, 64, 0, s>>>(model, n_sets, part, out);
    return cudaGetLastError();
}

cudaError_t launch_norm(int model, double q, double H, double eps, double* out, double* part,
                        cudaStream_t s)
{
    norm_partial_kernel<<<kNormBlocks, kNormThreads, 0, s>>>(model, q, H, eps, part);
    norm_final_kernel<<<1, 1, 0, s>>>(model, part, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tally output for one observer: S, S2, C (as doubles) or the intensity
// j = S v(E_c) / (4 pi V_obs dt_bin dE).
// ---------------------------------------------------------------------------
// v(E_c) / (4 pi V dt dE) of energy row ie: the factor from the occupancy sum to the
// intensity.  Ring observers: V of one longitude bin, dt the whole time window.
__device__ double intensity_factor(const ObsOut& ob, int ie)
{
    const double pi = 3.141592653589793;
    double vol;
    if (ob.kind == 0) {
        const double lo = ob.r - ob.dr, hi = ob.r + ob.dr;
        vol = 4.0 * pi / 3.0 * (hi * hi * hi - lo * lo * lo);
    } else if (ob.kind == 1) {
        const double lo = ob.r - ob.dr, hi = ob.r + ob.dr;
        vol = (hi * hi * hi - lo * lo * lo) / 3.0 * (cos(ob.th - ob.dth) - cos(ob.th + ob.dth))
              * 2.0 * ob.dph;
    } else if (ob.kind == 3) {
        const double lo = ob.r - ob.dr, hi = ob.r + ob.dr;
        vol = (hi * hi * hi - lo * lo * lo) / 3.0 * (cos(ob.th - ob.dth) - cos(ob.th + ob.dth))
              * 2.0 * pi / ob.nt;
    } else {
        vol = 2.0 * ob.dr;
    }
    const double e0 = ob.e_lo * pow(ob.e_hi / ob.e_lo, (double)ie / ob.ne);
    const double e1 = ob.e_lo * pow(ob.e_hi / ob.e_lo, (double)(ie + 1) / ob.ne);
    const double ec = sqrt(e0 * e1);
    const double T = ec / 938.27208816;
    const double pm = sqrt(T * (T + 2.0));
    const double v = (299792458.0 / 1.495978707e11) * pm / sqrt(1.0 + pm * pm);
    const double dtb = ob.kind == 3 ? ob.t_hi - ob.t_lo : (ob.t_hi - ob.t_lo) / ob.nt;
    return v / (4.0 * pi * vol * dtb * (e1 - e0));
}

__global__ void tally_out_kernel(const double* S, const double* S2, const unsigned long long* C,
                                 const ObsOut ob, int kind, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ob.ne * ob.nt) return;
    const int b = ob.off + k;
    if (kind == FTE_TALLY_S) { out[k] = S[b]; return; }
    if (kind == FTE_TALLY_S2) { out[k] = S2[b]; return; }
    if (kind == FTE_TALLY_C) { out[k] = (double)C[b]; return; }
    out[k] = S[b] * intensity_factor(ob, k / ob.nt);
}

// Green's function -> time-dependent source (Sec. 2.3): out[e][k] = dt_bin *
// sum_{m <= k} src[m] X[e][k - m], X = S or the intensity; src NULL = 1.
__global__ void convolve_kernel(const double* S, const ObsOut ob, int kind, const double* src, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ob.ne * ob.nt) return;
    const int ie = k / ob.nt, it = k - ie * ob.nt;
    const double* row = S + ob.off + (size_t)ie * ob.nt;
    double acc = 0.0;
    for (int m = 0; m <= it; ++m) acc += (src ? src[m] : 1.0) * row[it - m];
    const double dtb = (ob.t_hi - ob.t_lo) / ob.nt;
    out[k] = dtb * acc * (kind == FTE_TALLY_INTENSITY ? intensity_factor(ob, ie) : 1.0);
}

cudaError_t launch_convolve(const double* S, const ObsOut& ob, int kind, const double* src, double* out,
                            cudaStream_t s)
{
    const int n = ob.ne * ob.nt;
    convolve_kernel<<<(n + 127) / 128, 128, 0, s>>>(S, ob, kind, src, out);
    return cudaGetLastError();
}

cudaError_t launch_tally_out(const double* S, const double* S2, const unsigned long long* C,
                             const ObsOut& ob, int kind, double* out, cudaStream_t s)
{
    const int n = ob.ne * ob.nt;
    tally_out_kernel<<<(n + 255) / 256, 256, 0, s>>>(S, S2, C, ob, kind, out);
    return cudaGetLastError();
}

}  // namespace fte
