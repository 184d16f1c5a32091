// Injection kernel (Sec. 2.3, Eq. 7): one thread per particle, counter-based
// draws (tag 1: pitch-angle cosine and energy; tag 2: position attempt a),
// volume-uniform positions (optionally in a band of spiral phase) with optional
// div V < 0 acceptance on the stored cell values, weight 1 or 1/r^2.
#include "fte_kernels.cuh"

namespace fte {

__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) inject_kernel(const InjectArgs a)
{
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    double wsum = 0.0;
    unsigned nok = 0, nfail = 0;
    if (i < a.n) {
        const unsigned long long idx = a.offset + i;
        const uint32_t pid = a.id_base + (uint32_t)i;
        const uint2 key = make_uint2(a.seed, a.set_id);
        const uint4 d = philox4x32_10(make_uint4(0u, pid, 1u, 0u), key);
        const float mu = a.mu_mode ? a.mu0 : u11(d.x);
        float E;
        if (a.energy == 0) {
            E = a.e0;
        } else if (fabsf(a.gamma - 1.f) < 1e-6f) {
            E = a.e1 * powf(a.e2 / a.e1, u01(d.y));
        } else {
            const float g1 = 1.f - a.gamma;
            const float lo = powf(a.e1, g1), hi = powf(a.e2, g1);
            E = powf(lo + u01(d.y) * (hi - lo), 1.f / g1);
        }
        const float T = E / kMc2;
        const float p = sqrtf(T * (T + 2.f));
        float r = a.r, th = a.th, ph = a.ph;
        bool ok = true;
        if (a.region == 1) {
            ok = false;
            const float r13 = a.r1 * a.r1 * a.r1, r23 = a.r2 * a.r2 * a.r2;
            const float c1 = cosf(a.th1), c2 = cosf(a.th2);
            for (int t = 0; t < a.max_tries && !ok; ++t) {
                const uint4 q = philox4x32_10(make_uint4((uint32_t)t, pid, 2u, 0u), key);
                r = cbrtf(r13 + u01(q.x) * (r23 - r13));
                th = acosf(c1 + u01(q.y) * (c2 - c1));
                ph = a.ph1 + u01(q.z) * (a.ph2 - a.ph1);
                if (a.spiral != 0.f) ph -= a.spiral * (r - a.spiral_rb);   // spiral phase -> longitude
                if (!a.use_divv) { ok = true; break; }
                const GridK& g = a.g;
                float phw = fmodf(ph, kTwoPi);
                if (phw < 0.f) phw += kTwoPi;
                long long ri;
                if (g.amr) {
                    int ci, cj, ck;
                    const int leaf = amr_containing(g, r, th, phw, ci, cj, ck);
                    ri = (long long)a.divv_snap * g.snap_recs +
                         (((long long)leaf * g.P + ck + 1) * g.P + cj + 1) * g.P + ci + 1;
                } else {
                    const float xr = g.radial ? logf(r / g.r_min) * g.inv_dr : (r - g.r_min) * g.inv_dr;
                    const float xt = (th - g.th_min) * g.inv_dth;
                    const float xp = phw * g.inv_dph;
                    const int ci = min(max((int)floorf(xr), 0), g.nr - 1);
                    const int cj = min(max((int)floorf(xt), 0), g.nth - 1);
                    int ck = (int)floorf(xp) % g.nph;
                    if (ck < 0) ck += g.nph;
                    ri = (long long)a.divv_snap * g.snap_recs + ((long long)ck * g.nth + cj) * g.nr + ci;
                }
                float g00, g11, g22;
                // the cell's own fields lead its record in either layout
                if (g.dtype == FTE_F32) {
                    const float* rec = g.fields + ri * (g.pair ? kPairRec : FTE_REC);
                    g00 = __ldg(rec + 6); g11 = __ldg(rec + 10); g22 = __ldg(rec + 14);
                } else {
                    // stored value times its field scale, rounded once
                    const uint32_t* rec = g.hfields + ri * ((g.pair ? kPairHRec : FTE_HREC) / 2);
                    const uint32_t w3 = __ldg(rec + 3), w5 = __ldg(rec + 5), w7 = __ldg(rec + 7);
                    const bool bf = g.dtype == FTE_BF16;
                    g00 = __fmul_rn(bf ? h_lo<FTE_BF16>(w3) : h_lo<FTE_F16>(w3), __ldg(g.scale + 6));
                    g11 = __fmul_rn(bf ? h_lo<FTE_BF16>(w5) : h_lo<FTE_F16>(w5), __ldg(g.scale + 10));
                    g22 = __fmul_rn(bf ? h_lo<FTE_BF16>(w7) : h_lo<FTE_F16>(w7), __ldg(g.scale + 14));
                }
                const float s01 = __fadd_rn(g00, g11);
                const float tr = __fadd_rn(s01, g22);
                if (tr < a.divv_max) ok = true;
            }
        }
        float sp, cp, st, ct;
        sincosf(ph, &sp, &cp);
        sincosf(th, &st, &ct);
        a.x[idx] = r * st * cp;
        a.y[idx] = r * st * sp;
        a.z[idx] = r * ct;
        a.mu[idx] = mu;
        a.p[idx] = p;
        a.id[idx] = pid;
        const float w = a.weight ? 1.f / (r * r) : 1.f;
        if (ok) {
            a.w[idx] = w;
            a.status[idx] = FTE_ALIVE;
            wsum = (double)w;
            nok = 1;
        } else {
            a.w[idx] = 0.f;
            a.status[idx] = FTE_INJ_FAIL;
            nfail = 1;
        }
    }
    wsum = warp_sum_f64(wsum);
    nok = warp_sum_u32(nok);
    nfail = warp_sum_u32(nfail);
    if ((threadIdx.x & 31) == 0) {
        if (nok) {
            atomicAdd(&a.ledger_w[0], wsum);
            atomicAdd(&a.ledger_n[0], (unsigned long long)nok);
        }
        if (nfail) atomicAdd(&a.ledger_n[5], (unsigned long long)nfail);
    }
}

cudaError_t launch_inject(const InjectArgs& a, cudaStream_t s)
{
    const unsigned long long blocks = (a.n + 255) / 256;
    if (blocks) inject_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fte
