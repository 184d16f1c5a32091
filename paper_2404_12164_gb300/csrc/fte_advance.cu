// Transport kernels: the per-particle step loop with the fused occupancy tally,
// the FP64 reduction of per-block partial histograms, the FP64 per-step time
// table, the D_mumu normalisation integral and the intensity output.
#include "fte_kernels.cuh"

namespace fte {

// ---------------------------------------------------------------------------
// Occupancy tally (start-of-step state, w dt per step).  Lanes of a warp that
// hit the same bin are merged first (__match_any_sync), then one lane per bin
// adds the merged sums to the block's shared-memory histogram.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_tally(float* shS, float* shS2, unsigned* shC, int bin,
                                           float val)
{
    const unsigned m = __activemask();
    if (!__any_sync(m, bin >= 0)) return;
    const unsigned grp = __match_any_sync(m, bin);
    if (bin < 0) return;
    float s = 0.f, s2 = 0.f;
    unsigned mm = grp;
    while (mm) {
        const int src = __ffs(mm) - 1;
        mm &= mm - 1;
        const float v = __shfl_sync(grp, val, src);
        s += v;
        s2 += v * v;
    }
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) {
        atomicAdd(&shS[bin], s);
        atomicAdd(&shS2[bin], s2);
        atomicAdd(&shC[bin], (unsigned)__popc(grp));
    }
}

// One Euler-Maruyama step of Eqs. 2-4 for one particle (Sec. 2.1), with the
// background interpolated at the start-of-step position and time (Sec. 2.4).
template <bool KPERP, int DT>
__device__ __forceinline__ int step(const AdvanceArgs& a, float I, long long n, uint32_t pid,
                                    float& x, float& y, float& z, float& mu, float& p, float w,
                                    float* shS, float* shS2, unsigned* shC, const float* sc,
                                    unsigned long long& noor)
{
    const StepEntry* ep = a.table + (n - a.n_table0);
    StepEntry e;
    {
        const int4 h = __ldg(reinterpret_cast<const int4*>(ep));   // s0, s1, wt, two
        e.s0 = h.x; e.s1 = h.y; e.wt = __int_as_float(h.z); e.two = h.w;
    }
    const float rho2 = x * x + y * y;
    const float r = sqrtf(rho2 + z * z);
    const float rho = sqrtf(rho2);
    const float th = atan2f(rho, z);
    float ph = atan2f(y, x);
    if (ph < 0.f) ph += kTwoPi;

    Loc L;
    locate(a.g, r, th, ph, L);
    Fields<KPERP> F;
    gather<KPERP, DT>(a.g, e, L, sc, F);
    const float* B = F.f;
    const float* V = F.f + 3;
    const float* G = F.f + 6;
    const float* gB = F.f + 15;

    // derived background quantities
    const float invB = rsqrtf(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    const float b0 = B[0] * invB, b1 = B[1] * invB, b2 = B[2] * invB;
    const float divb = -(b0 * gB[0] + b1 * gB[1] + b2 * gB[2]) * invB;   // 1 / L
    const float divv = G[0] + G[4] + G[8];
    const float bbgv = b0 * (G[0] * b0 + G[1] * b1 + G[2] * b2)
                     + b1 * (G[3] * b0 + G[4] * b1 + G[5] * b2)
                     + b2 * (G[6] * b0 + G[7] * b1 + G[8] * b2);
    float bdvdt = 0.f;
    if (a.prm.dvdt_term) {
        const float s = e.two ? a.g.inv_dt_snap : 0.f;   // dV/dt = dV/dt|_x + (V.grad) V
        const float a0 = F.dv[0] * s + G[0] * V[0] + G[1] * V[1] + G[2] * V[2];
        const float a1 = F.dv[1] * s + G[3] * V[0] + G[4] * V[1] + G[5] * V[2];
        const float a2 = F.dv[2] * s + G[6] * V[0] + G[7] * V[1] + G[8] * V[2];
        bdvdt = b0 * a0 + b1 * a1 + b2 * a2;
    }

    const float v = speed_of(p);
    float D, dD;
    dmumu(a.prm, I, mu, v, p, D, dD);

    const uint4 rb = philox4x32_10(make_uint4((uint32_t)n, pid, 0u, 0u),
                                   make_uint2(a.prm.seed, a.prm.set_id));
    const float amp0 = sqrtf(-2.f * logf(u01(rb.x)));
    float s1, c1;
    sincospif(2.f * u01(rb.y), &s1, &c1);
    const float dt = a.prm.dt;

    // Eq. 3 + Ito pitch-angle diffusion, reflecting at mu = +-1
    const float omm = 1.f - mu * mu;
    const float mudot = 0.5f * omm * (v * divb + mu * divv - 3.f * mu * bbgv - (2.f / v) * bdvdt);
    float mun = mu + (mudot + dD) * dt + sqrtf(2.f * D * dt) * (amp0 * c1);
    if (mun > 1.f) mun = 2.f - mun;
    if (mun < -1.f) mun = -2.f - mun;
    mun = fminf(fmaxf(mun, -1.f), 1.f);

    // Eq. 2 (V_d = 0) + cross-field diffusion kappa_perp = (v lambda_perp / 3)(I - bb)
    float ux = V[0] + mu * v * b0, uy = V[1] + mu * v * b1, uz = V[2] + mu * v * b2;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (KPERP) {
        const float kap = v * a.prm.lambda_perp * (1.f / 3.f);
        if (a.prm.kappa_drift) {
            const float cth = z / r, sth = rho / r;
            const float cph = rho > 0.f ? x / rho : 1.f, sph = rho > 0.f ? y / rho : 0.f;
            const float br = (b0 * cph + b1 * sph) * sth + b2 * cth;        // b . r_hat
            const float bt = ((b0 * cph + b1 * sph) * cth - b2 * sth) / r;  // b . theta_hat / r
            const float bp = (-b0 * sph + b1 * cph) / rho;                  // b . phi_hat / (r sin th)
            float g3[3];
#pragma unroll
            for (int m = 0; m < 3; ++m)
                g3[m] = F.dBa[3 * m + 0] * br + F.dBa[3 * m + 1] * bt + F.dBa[3 * m + 2] * bp;
            const float par = b0 * g3[0] + b1 * g3[1] + b2 * g3[2];
            // div(kappa_perp) = -kappa [(div b) b + (b.grad) b]
            ux -= kap * (divb * b0 + (g3[0] - b0 * par) * invB);
            uy -= kap * (divb * b1 + (g3[1] - b1 * par) * invB);
            uz -= kap * (divb * b2 + (g3[2] - b2 * par) * invB);
        }
        float e10, e11, e12;
        const float cz = sqrtf(b0 * b0 + b1 * b1);       // |b x z_hat|
        if (cz >= 0.1f) {
            e10 = b1 / cz; e11 = -b0 / cz; e12 = 0.f;
        } else {
            const float cx = sqrtf(b1 * b1 + b2 * b2);   // |b x x_hat|
            e10 = 0.f; e11 = b2 / cx; e12 = -b1 / cx;
        }
        const float e20 = b1 * e12 - b2 * e11, e21 = b2 * e10 - b0 * e12, e22 = b0 * e11 - b1 * e10;
        const float z1 = amp0 * s1;
        const float z2 = sqrtf(-2.f * logf(u01(rb.z))) * cospif(2.f * u01(rb.w));
        const float amp = sqrtf(2.f * kap * dt);
        nx = amp * (z1 * e10 + z2 * e20);
        ny = amp * (z1 * e11 + z2 * e21);
        nz = amp * (z1 * e12 + z2 * e22);
    }
    const float xn = x + ux * dt + nx, yn = y + uy * dt + ny, zn = z + uz * dt + nz;

    // Eq. 4
    const float pdot = 0.5f * (1.f - 3.f * mu * mu) * bbgv - 0.5f * omm * divv - (mu / v) * bdvdt;
    const float pn = (a.prm.p_update == 0) ? p * expf(pdot * dt) : p * (1.f + pdot * dt);

    // occupancy tally of the start-of-step state
    if (a.n_obs) {
        const float E = energy_of(p);
        for (int o = 0; o < a.n_obs; ++o) {
            const ObsK& ob = a.obs[o];
            bool in;
            if (ob.kind == 2) {
                in = fabsf(x - ob.r) <= ob.dr;
            } else {
                in = fabsf(r - ob.r) <= ob.dr;
                if (ob.kind == 1) {
                    float d = ph - ob.ph;
                    if (d > kPi) d -= kTwoPi;
                    if (d < -kPi) d += kTwoPi;
                    in = in && fabsf(th - ob.th) <= ob.dth && fabsf(d) <= ob.dph;
                }
            }
            int bin = -1;
            if (in) {
                const float le = logf(E / ob.e_lo) * ob.ne_over_lnratio;
                const int it = __ldg(&ep->it[o]);
                if (le >= 0.f && le < (float)ob.ne && it >= 0)
                    bin = ob.off + (int)le * ob.nt + it;
                else
                    ++noor;
            }
            warp_tally(shS, shS2, shC, bin, w * dt);
        }
    }

    x = xn; y = yn; z = zn; mu = mun; p = pn;
    if (!(isfinite(xn) && isfinite(yn) && isfinite(zn) && isfinite(mun) && isfinite(pn)))
        return FTE_DEAD_NAN;
    const float rn = sqrtf(xn * xn + yn * yn + zn * zn);
    if (rn < a.g.r_min) return FTE_ABS_INNER;
    if (rn > a.g.r_max) return FTE_ABS_OUTER;
    // theta < th_min  <=>  z > r cos(th_min); theta > th_max  <=>  z < r cos(th_max)
    if (zn > rn * a.g.cos_th_min || zn < rn * a.g.cos_th_max) return FTE_ABS_THETA;
    return FTE_ALIVE;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Persistent step kernel: each thread takes particles from a shared counter and
// keeps each one in registers for all steps [n_start, n_end) of the launch.
template <bool KPERP, int DT>
__global__ void __launch_bounds__(kThreads) advance_kernel(const AdvanceArgs a)
{
    extern __shared__ float sh[];
    float* shS = sh;
    float* shS2 = sh + a.nbins;
    unsigned* shC = reinterpret_cast<unsigned*>(sh + 2 * a.nbins);
    __shared__ float sc[FTE_NFIELD];      // per-field scales of 16-bit storage
    for (int b = threadIdx.x; b < 3 * a.nbins; b += blockDim.x) sh[b] = 0.f;
    if (DT != FTE_F32 && threadIdx.x < FTE_NFIELD) sc[threadIdx.x] = __ldg(a.g.scale + threadIdx.x);
    __syncthreads();

    const float I = (float)__ldg(a.norm);
    const unsigned long long n_work = a.order ? (unsigned long long)__ldg(a.n_order) : a.n_particles;
    unsigned long long nsteps = 0, noor = 0;
    for (;;) {
        const unsigned long long f = atomicAdd(a.fetch, 1ULL);
        if (f >= n_work) break;
        const unsigned long long i = a.order ? (unsigned long long)__ldg(a.order + f) : f;
        if (!a.order && a.status[i] != FTE_ALIVE) continue;
        float x = a.x[i], y = a.y[i], z = a.z[i], mu = a.mu[i], p = a.p[i];
        const float w = a.w[i];
        const uint32_t pid = a.id[i];
        int st = FTE_ALIVE;
        for (long long n = a.n_start; n < a.n_end; ++n) {
            ++nsteps;
            st = step<KPERP, DT>(a, I, n, pid, x, y, z, mu, p, w, shS, shS2, shC, sc, noor);
            if (st != FTE_ALIVE) break;
        }
        a.x[i] = x; a.y[i] = y; a.z[i] = z; a.mu[i] = mu; a.p[i] = p;
        if (st != FTE_ALIVE) {
            a.status[i] = (uint8_t)st;
            atomicAdd(&a.ledger_w[st], (double)w);
            atomicAdd(&a.ledger_n[st], 1ULL);
        }
    }

    __syncthreads();   // all tally updates of this block are in shared memory
    float* out = a.part + (size_t)blockIdx.x * 3 * a.nbins;
    for (int b = threadIdx.x; b < 3 * a.nbins; b += blockDim.x) out[b] = sh[b];
    nsteps = warp_sum_u64(nsteps);
    noor = warp_sum_u64(noor);
    if ((threadIdx.x & 31) == 0) {
        if (nsteps) atomicAdd(&a.ledger_n[6], nsteps);
        if (noor) atomicAdd(&a.ledger_n[7], noor);
    }
}

static const void* advance_fn(int kperp, int dtype)
{
    if (dtype == FTE_BF16)
        return kperp ? (const void*)advance_kernel<true, FTE_BF16> : (const void*)advance_kernel<false, FTE_BF16>;
    if (dtype == FTE_F16)
        return kperp ? (const void*)advance_kernel<true, FTE_F16> : (const void*)advance_kernel<false, FTE_F16>;
    return kperp ? (const void*)advance_kernel<true, FTE_F32> : (const void*)advance_kernel<false, FTE_F32>;
}

cudaError_t advance_occupancy(int kperp, int dtype, size_t smem, int* blocks_per_sm)
{
    const void* fn = advance_fn(kperp, dtype);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kThreads, smem);
}

cudaError_t launch_advance(const AdvanceArgs& a, int kperp, int blocks, size_t smem, cudaStream_t s)
{
    const int dt = a.g.dtype;
#define FTE_LAUNCH(K, D) advance_kernel<K, D><<<blocks, kThreads, smem, s>>>(a)
    if (dt == FTE_BF16) { if (kperp) FTE_LAUNCH(true, FTE_BF16); else FTE_LAUNCH(false, FTE_BF16); }
    else if (dt == FTE_F16) { if (kperp) FTE_LAUNCH(true, FTE_F16); else FTE_LAUNCH(false, FTE_F16); }
    else { if (kperp) FTE_LAUNCH(true, FTE_F32); else FTE_LAUNCH(false, FTE_F32); }
#undef FTE_LAUNCH
    return cudaGetLastError();
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

template <int DT>
__global__ void __launch_bounds__(256) encode_kernel(const float* __restrict__ f, long long nrec,
                                                     const float* __restrict__ hdr, uint32_t* out)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    float a[FTE_REC];
#pragma unroll
    for (int q = 0; q < FTE_REC / 8; ++q) ldg8(f + r * FTE_REC + 8 * q, a + 8 * q);
    uint32_t w[FTE_HREC / 2];
#pragma unroll
    for (int k = 0; k < FTE_HREC / 2; ++k) w[k] = 0u;
#pragma unroll
    for (int k = 0; k < FTE_NFIELD; ++k) {
        const uint32_t h = encode16<DT>(__fdiv_rn(a[k], __ldg(hdr + k)));
        w[k >> 1] |= (k & 1) ? (h << 16) : h;
    }
    uint4* o = reinterpret_cast<uint4*>(out + r * (FTE_HREC / 2));
#pragma unroll
    for (int q = 0; q < FTE_HREC / 8; ++q) o[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
}

cudaError_t launch_quantize(const float* f32, long long nrec, int dtype, void* out, cudaStream_t s)
{
    float* hdr = reinterpret_cast<float*>(out);
    uint32_t* recs = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(out) + FTE_HHDR * sizeof(float));
    cudaError_t e = cudaMemsetAsync(hdr, 0, FTE_HHDR * sizeof(float), s);
    if (e != cudaSuccess) return e;
    maxabs_kernel<<<1216, 256, 0, s>>>(f32, nrec, reinterpret_cast<unsigned*>(hdr));
    scale_final_kernel<<<1, 32, 0, s>>>(hdr);
    const long long blocks = (nrec + 255) / 256;
    if (dtype == FTE_BF16) encode_kernel<FTE_BF16><<<(unsigned)blocks, 256, 0, s>>>(f32, nrec, hdr, recs);
    else encode_kernel<FTE_F16><<<(unsigned)blocks, 256, 0, s>>>(f32, nrec, hdr, recs);
    return cudaGetLastError();
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
        if (a.periodic) {
            const double kf = floor(tau);
            const long long kk = (long long)kf;
            const int s0 = (int)(((kk % a.n_snap) + a.n_snap) % a.n_snap);
            e.s0 = s0;
            e.s1 = (s0 + 1) % a.n_snap;
            e.wt = (float)(tau - kf);
            e.two = 1;
        } else if (tau < 0.0) {
            e.s0 = e.s1 = 0;
        } else if (tau >= (double)(a.n_snap - 1)) {
            e.s0 = e.s1 = a.n_snap - 1;
        } else {
            const double kf = floor(tau);
            e.s0 = (int)kf;
            e.s1 = e.s0 + 1;
            e.wt = (float)(tau - kf);
            e.two = 1;
        }
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
__global__ void tally_out_kernel(const double* S, const double* S2, const unsigned long long* C,
                                 const ObsOut ob, int kind, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ob.ne * ob.nt) return;
    const int b = ob.off + k;
    if (kind == FTE_TALLY_S) { out[k] = S[b]; return; }
    if (kind == FTE_TALLY_S2) { out[k] = S2[b]; return; }
    if (kind == FTE_TALLY_C) { out[k] = (double)C[b]; return; }
    const double pi = 3.141592653589793;
    double vol;
    if (ob.kind == 0) {
        const double lo = ob.r - ob.dr, hi = ob.r + ob.dr;
        vol = 4.0 * pi / 3.0 * (hi * hi * hi - lo * lo * lo);
    } else if (ob.kind == 1) {
        const double lo = ob.r - ob.dr, hi = ob.r + ob.dr;
        vol = (hi * hi * hi - lo * lo * lo) / 3.0 * (cos(ob.th - ob.dth) - cos(ob.th + ob.dth))
              * 2.0 * ob.dph;
    } else {
        vol = 2.0 * ob.dr;
    }
    const int ie = k / ob.nt;
    const double e0 = ob.e_lo * pow(ob.e_hi / ob.e_lo, (double)ie / ob.ne);
    const double e1 = ob.e_lo * pow(ob.e_hi / ob.e_lo, (double)(ie + 1) / ob.ne);
    const double ec = sqrt(e0 * e1);
    const double T = ec / 938.27208816;
    const double pm = sqrt(T * (T + 2.0));
    const double v = (299792458.0 / 1.495978707e11) * pm / sqrt(1.0 + pm * pm);
    const double dtb = (ob.t_hi - ob.t_lo) / ob.nt;
    out[k] = S[b] * v / (4.0 * pi * vol * dtb * (e1 - e0));
}

cudaError_t launch_tally_out(const double* S, const double* S2, const unsigned long long* C,
                             const ObsOut& ob, int kind, double* out, cudaStream_t s)
{
    const int n = ob.ne * ob.nt;
    tally_out_kernel<<<(n + 255) / 256, 256, 0, s>>>(S, S2, C, ob, kind, out);
    return cudaGetLastError();
}

}  // namespace fte
