// The per-particle step loop of the transport kernels (Sec. 2.1, 2.4) with the
// fused occupancy tally, shared by the single-set and the ensemble kernels.
#pragma once

#include "fte_kernels.cuh"

namespace fte {

// ---------------------------------------------------------------------------
// Occupancy tally (start-of-step state, w dt per step).  A particle's consecutive
// tallied steps in one bin add up in two registers (its w dt is the same every
// step) and reach the accumulators once, when the bin changes and when the particle
// leaves the launch: the steps tallied at one time are concentrated in a few bins
// (one time bin, a few energy bins), so adding every step there would have tens of
// thousands of threads contend for a handful of addresses.  The accumulators are
// the FP64 tally in global memory (global modes) or the block's shared-memory
// histogram (shared modes); the class-resolved tally (batch means) gains the same
// sum in the particle's id class.
// ---------------------------------------------------------------------------
struct TallyRun {
    int bin;          // bin of the run of tallied steps, -1 before the first
    unsigned cnt;     // steps in it not yet added to the accumulators
};

template <int MODE>
__device__ __forceinline__ void tally_flush(const AdvanceArgs& a, float* shS, float* shS2, unsigned* shC,
                                           TallyRun& t, float wdt, uint32_t pid)
{
    if (t.cnt == 0) return;
    const double d = (double)wdt, c = (double)t.cnt;
    if (global_tally(MODE)) {
        atomicAdd(&a.gS[t.bin], d * c);
        atomicAdd(&a.gS2[t.bin], d * d * c);
        atomicAdd(&a.gC[t.bin], (unsigned long long)t.cnt);
    } else {
        atomicAdd(&shS[t.bin], (float)(d * c));
        atomicAdd(&shS2[t.bin], (float)(d * d * c));
        atomicAdd(&shC[t.bin], t.cnt);
    }
    if (a.cls) atomicAdd(a.cls + ((size_t)t.bin * FTE_NCLASS + (pid % FTE_NCLASS)), d * c);
    t.cnt = 0;
}

// One Euler-Maruyama step of Eqs. 2-4 for one particle (Sec. 2.1), with the
// background interpolated at the start-of-step position and time (Sec. 2.4).
template <bool KPERP, int DT, int MODE, int LAY>
__device__ __forceinline__ int step(const AdvanceArgs& a, const ParamsK& prm, float I, int sbin,
                                    long long n, uint32_t pid,
                                    float& x, float& y, float& z, float& mu, float& p, float w,
                                    float* shS, float* shS2, unsigned* shC, const float* sc,
                                    unsigned long long& noor, TallyRun& run)
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
    gather<KPERP, DT, LAY, global_tally(MODE)>(a.g, e, L, sc, F);
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
    if (prm.dvdt_term) {
        const float s = e.two ? a.g.inv_dt_snap : 0.f;   // dV/dt = dV/dt|_x + (V.grad) V
        const float a0 = F.dv[0] * s + G[0] * V[0] + G[1] * V[1] + G[2] * V[2];
        const float a1 = F.dv[1] * s + G[3] * V[0] + G[4] * V[1] + G[5] * V[2];
        const float a2 = F.dv[2] * s + G[6] * V[0] + G[7] * V[1] + G[8] * V[2];
        bdvdt = b0 * a0 + b1 * a1 + b2 * a2;
    }

    const float v = speed_of(p);
    const float inv_v = 1.f / v;
    float D, dD;
    dmumu(prm, I, mu, v, p, D, dD);

    const uint4 rb = philox4x32_10(make_uint4((uint32_t)n, pid, 0u, 0u),
                                   make_uint2(prm.seed, prm.set_id));
    const float amp0 = sqrtf(-2.f * logf(u01(rb.x)));
    float s1, c1;
    sincospif(2.f * u01(rb.y), &s1, &c1);
    const float dt = prm.dt;

    // Eq. 3 + Ito pitch-angle diffusion, reflecting at mu = +-1
    const float omm = 1.f - mu * mu;
    const float mudot = 0.5f * omm * (v * divb + mu * divv - 3.f * mu * bbgv - 2.f * inv_v * bdvdt);
    float mun = mu + (mudot + dD) * dt + sqrtf(2.f * D * dt) * (amp0 * c1);
    if (mun > 1.f) mun = 2.f - mun;
    if (mun < -1.f) mun = -2.f - mun;
    mun = fminf(fmaxf(mun, -1.f), 1.f);

    // Eq. 2 (V_d = 0) + cross-field diffusion kappa_perp = (v lambda_perp / 3)(I - bb)
    float ux = V[0] + mu * v * b0, uy = V[1] + mu * v * b1, uz = V[2] + mu * v * b2;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (KPERP) {
        const float kap = v * prm.lambda_perp * (1.f / 3.f);
        if (prm.kappa_drift) {
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
    const float pdot = 0.5f * (1.f - 3.f * mu * mu) * bbgv - 0.5f * omm * divv - mu * inv_v * bdvdt;
    const float pn = (prm.p_update == 0) ? p * expf(pdot * dt) : p * (1.f + pdot * dt);

    // occupancy tally of the start-of-step state
    if (a.n_obs) {
        for (int o = 0; o < a.n_obs; ++o) {
            const ObsK& ob = a.obs[o];
            bool in;
            if (ob.kind == 2) {
                in = fabsf(x - ob.r) <= ob.dr;
            } else if (ob.kind == 3) {       // ring: longitude profile at fixed r, theta
                in = fabsf(r - ob.r) <= ob.dr && fabsf(th - ob.th) <= ob.dth;
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
                const float le = logf(energy_of(p) / ob.e_lo) * ob.ne_over_lnratio;
                int it = __ldg(&ep->it[o]);     // time bin, -1 outside [t_lo, t_hi)
                if (ob.kind == 3 && it >= 0) it = min((int)(ph * ob.phi_scale), ob.nt - 1);
                if (le >= 0.f && le < (float)ob.ne && it >= 0)
                    bin = sbin + ob.off + (int)le * ob.nt + it;
                else
                    ++noor;
            }
            if (bin >= 0) {
                if (bin != run.bin) {
                    tally_flush<MODE>(a, shS, shS2, shC, run, w * dt, pid);
                    run.bin = bin;
                }
                ++run.cnt;
            }
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

// Persistent work distribution: lane 0 of the warp claims the next 32 entries of the
// work list and each lane takes one, after the warp has reconverged (every lane of a
// warp runs the same fetch loop and leaves it at the same time, so the full-warp
// barrier always completes).  A per-lane counter would let lanes that reach the fetch
// at different times (a particle absorbed early, a tally added) take entries far apart
// in the ordered list, and their loads would then touch more cache lines.
__device__ __forceinline__ unsigned long long warp_fetch(unsigned long long* counter)
{
    __syncwarp();
    unsigned long long base = 0;
    if ((threadIdx.x & 31u) == 0) base = atomicAdd(counter, 32ULL);
    return __shfl_sync(0xffffffffu, base, 0) + (threadIdx.x & 31u);
}

// Per-SM ranges of the work list: the list is cut into `slots` equal ranges (at most
// `slots`, fewer when the device has fewer SM ids) and the warps of the SM with id c
// take 32 consecutive entries of range c at a time, so that all warps resident on one
// SM - whatever their block - hold neighbouring particles of the spatially ordered list
// and share the background records in that SM's L1.  Once its range is used up, a warp
// takes entries of the following ranges, checking 32 of them per round (one lane each,
// the counters read from L2): no entry is handed out twice, since each is claimed by the
// one atomic add on its range's counter, and a warp returns `n` only after it has seen
// every range used up, so every entry is handed out.  *end receives the end of the range
// the lane's entry lies in.
__device__ __forceinline__ unsigned long long warp_fetch_sm(unsigned long long* cnt, unsigned slots,
                                                            unsigned long long n, unsigned long long* end)
{
    __syncwarp();
    const unsigned lane = threadIdx.x & 31u;
    unsigned smid, nsmid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
    const unsigned ns = nsmid == 0 ? 1u : (nsmid < slots ? nsmid : slots);
    const unsigned own = smid % ns;
    unsigned long long base = n, hi = n;
    if (lane == 0) {
        const unsigned long long lo = own * n / ns, h = (own + 1ULL) * n / ns;
        const unsigned long long got = atomicAdd(cnt + own, 32ULL);
        if (lo + got < h) { base = lo + got; hi = h; }
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    hi = __shfl_sync(0xffffffffu, hi, 0);
    for (unsigned off = 1; base == n && off < ns; off += 32) {
        bool avail = false;
        if (off + lane < ns) {
            const unsigned c = (own + off + lane) % ns;
            avail = c * n / ns + __ldcg(cnt + c) < (c + 1ULL) * n / ns;
        }
        unsigned m = __ballot_sync(0xffffffffu, avail);
        while (m != 0u && base == n) {
            const unsigned j = __ffs(m) - 1;
            m &= m - 1;
            if (lane == 0) {
                const unsigned c = (own + off + j) % ns;
                const unsigned long long lo = c * n / ns, h = (c + 1ULL) * n / ns;
                const unsigned long long got = atomicAdd(cnt + c, 32ULL);
                if (lo + got < h) { base = lo + got; hi = h; }
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            hi = __shfl_sync(0xffffffffu, hi, 0);
        }
    }
    *end = hi;
    return base == n ? n : base + lane;
}

// Set of pool entry i: the first s with i < end[s] (end holds running totals).
__device__ __forceinline__ int set_of(const unsigned long long* end, int n_sets, unsigned long long i)
{
    int lo = 0, hi = n_sets - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (i < end[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Persistent step kernel: each thread takes particles from a shared counter and
// keeps each one in registers for all steps [n_start, n_end) of the launch.
// MODE kModeSingle: one parameter set, tally in shared memory; kModeSingleGlobal:
// one parameter set, warp-merged FP64 atomics to the tally (no shared memory, so
// L1 keeps its whole capacity for the gather); kModeShared: an ensemble
// (per-set parameters and tallies, the tallies of all sets in shared memory);
// kModeGlobal: an ensemble with warp-merged FP64 atomics to the tally.
// LAY: record layout (cell or pair), compile-time.  MINB: blocks per SM the single-set
// kernel is compiled for (0: the register count ptxas chooses; 3: at most 85
// registers, 24 warps per SM, for the longer dependent-load chains of block AMR).
template <bool KPERP, int DT, int MODE, int NT, int LAY, int MINB = 0>
__global__ void __launch_bounds__(NT, single_set(MODE) ? MINB : 512 / NT) advance_kernel(const AdvanceArgs a, const BatchArgs b)
{
    extern __shared__ float sh[];
    const int nsh = global_tally(MODE) ? 0 : (MODE == kModeShared ? b.n_sets : 1) * a.nbins;
    float* shS = sh;
    float* shS2 = sh + nsh;
    unsigned* shC = reinterpret_cast<unsigned*>(sh + 2 * nsh);
    __shared__ float sc[FTE_NFIELD];      // per-field scales of 16-bit storage
    constexpr int kSets = single_set(MODE) ? 1 : FTE_MAX_SETS;
    __shared__ unsigned long long s_end[kSets];
    __shared__ SetK s_set[kSets];
    __shared__ float s_I[kSets];
    for (int q = threadIdx.x; q < 3 * nsh; q += NT) sh[q] = 0.f;
    if (DT != FTE_F32 && threadIdx.x < FTE_NFIELD) sc[threadIdx.x] = __ldg(a.g.scale + threadIdx.x);
    if (!single_set(MODE)) {
        for (int s = threadIdx.x; s < b.n_sets; s += NT) {
            s_end[s] = b.end[s];
            s_set[s] = b.set[s];
            s_I[s] = (float)__ldg(a.norm + s);
        }
    }
    __syncthreads();

    const float I0 = single_set(MODE) ? (float)__ldg(a.norm) : 0.f;
    const unsigned long long n_work = a.order ? (unsigned long long)__ldg(a.n_order) : a.n_particles;
    // A launch of one of two half-pools (on two streams) with fewer alive particles than
    // resident threads keeps only the blocks that give each thread one particle: the others
    // leave at once, so that their SM slots go to the other half's launch (a persistent block
    // holds its slot until its last warp ends).  The blocks that stay take work from one global
    // counter.  A pool launched alone keeps all blocks: there the freed slots would stay idle.
    unsigned fetch_slots = a.fetch_slots;
    if (MODE == kModeSingleGlobal && a.order && a.compact) {
        if (n_work < (unsigned long long)gridDim.x * NT) {
            fetch_slots = 0;
            if (blockIdx.x >= (n_work + NT - 1) / NT) return;
        }
    }
    unsigned long long nsteps = 0, noor = 0;
    for (;;) {
        // the warp takes 32 consecutive entries of the (spatially ordered) work list at once,
        // so that its lanes hold neighbouring particles whatever branches they took before
        unsigned long long fend = n_work;
        const unsigned long long f = fetch_slots ? warp_fetch_sm(a.fetch, fetch_slots, n_work, &fend)
                                                   : warp_fetch(a.fetch);
        if (__shfl_sync(0xffffffffu, f, 0) >= n_work) break;
        if (f >= fend) continue;
        const unsigned long long i = a.order ? (unsigned long long)__ldg(a.order + f) : f;
        if (!a.order && a.status[i] != FTE_ALIVE) continue;
        float x = a.x[i], y = a.y[i], z = a.z[i], mu = a.mu[i], p = a.p[i];
        const float w = a.w[i];
        const uint32_t pid = a.id[i];
        int st = FTE_ALIVE;
        TallyRun run{-1, 0u};
        if (single_set(MODE)) {
            for (long long n = a.n_start; n < a.n_end; ++n) {
                ++nsteps;
                st = step<KPERP, DT, MODE, LAY>(a, a.prm, I0, 0, n, pid, x, y, z, mu, p, w, shS, shS2, shC, sc, noor,
                                                run);
                if (st != FTE_ALIVE) break;
            }
        } else {
            const int s = set_of(s_end, b.n_sets, i);
            ParamsK prm = a.prm;
            prm.lambda_par = s_set[s].lambda_par;
            prm.inv_lambda_par = 1.f / s_set[s].lambda_par;
            prm.q = s_set[s].q;
            prm.H = s_set[s].H;
            prm.eps = s_set[s].eps;
            prm.seed = s_set[s].seed;
            prm.set_id = s_set[s].set_id;
            const float I = s_I[s];
            const int sbin = s * a.nbins;
            for (long long n = a.n_start; n < a.n_end; ++n) {
                ++nsteps;
                st = step<KPERP, DT, MODE, LAY>(a, prm, I, sbin, n, pid, x, y, z, mu, p, w, shS, shS2, shC, sc, noor,
                                                run);
                if (st != FTE_ALIVE) break;
            }
        }
        tally_flush<MODE>(a, shS, shS2, shC, run, w * a.prm.dt, pid);
        a.x[i] = x; a.y[i] = y; a.z[i] = z; a.mu[i] = mu; a.p[i] = p;
        if (st != FTE_ALIVE) {
            a.status[i] = (uint8_t)st;
            atomicAdd(&a.ledger_w[st], (double)w);
            atomicAdd(&a.ledger_n[st], 1ULL);
        }
    }

    __syncthreads();   // all tally updates of this block are in shared memory
    if (!global_tally(MODE)) {
        float* out = a.part + (size_t)blockIdx.x * 3 * nsh;
        for (int q = threadIdx.x; q < 3 * nsh; q += NT) out[q] = sh[q];
    }
    nsteps = warp_sum_u64(nsteps);
    noor = warp_sum_u64(noor);
    if ((threadIdx.x & 31) == 0) {
        if (nsteps) atomicAdd(&a.ledger_n[6], nsteps);
        if (noor) atomicAdd(&a.ledger_n[7], noor);
    }
}

}  // namespace fte
