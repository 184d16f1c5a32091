// Device-side building blocks of the focused-transport pusher (sm_103a).
//
// One thread owns one pseudo-particle and keeps its state in registers for
// every step of a launch.  Per step it locates the particle on the spherical
// grid, gathers the 8 surrounding cell records of the two bracketing snapshots
// (Sec. 2.4: trilinear interpolation of the surrounding grid values; linear in
// time between snapshots), forms the coefficients of Eqs. 3-4, draws one
// Philox4x32-10 block and applies one Euler-Maruyama step of the Ito SDEs
// (Sec. 2.1).  All arithmetic is FP32 except the per-step time table, which is
// built in FP64 by a separate kernel.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fte.h"

namespace fte {

constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;
constexpr float kCau = 2.003988804e-3f;      // speed of light, au/s
constexpr float kMc2 = 938.27208816f;        // proton rest energy, MeV
constexpr int kThreads = 256;                // threads per block of the step kernel
constexpr int kPairRec = 40;                 // floats of an FP32 pair record
constexpr int kPairHRec = 48;                // 16-bit values of a 16-bit pair record

// ---------------------------------------------------------------------------
// Kernel-side descriptions (passed by value in the kernel parameter space)
// ---------------------------------------------------------------------------
struct GridK {
    const float* fields;     // FP32: record r of snapshot s at fields[(s * snap_recs + r) * FTE_REC]
    const uint32_t* hfields; // 16-bit: record r of snapshot s at hfields[(s * snap_recs + r) * FTE_HREC / 2]
    const float* scale;      // 16-bit: per-field scales (FTE_HHDR floats)
    long long snap_recs;     // records per snapshot
    int dtype;
    int pair;                // 1: FTE_LAYOUT_PAIR records (cell k and k + 1 in one record)
    int nr, nth, nph, radial;
    float r_min, r_max, th_min, th_max;
    float cos_th_min, cos_th_max;
    float inv_dr;            // linear: nr / (r_max - r_min); log: nr / ln(r_max / r_min)
    float dr;                // linear: (r_max - r_min) / nr; log: ln(r_max / r_min) / nr
    float inv_dth, dth, inv_dph;
    float inv_dt_snap;
    // block AMR (amr > 0: number of levels); nr, nth, nph are base-level cells
    int amr, B, P, L, amr_leaves;
    int nf0, nf1, nf2;                // finest-level blocks per axis
    const int4* leaves;               // (level, bi, bj, bk)
    const int* table;                 // [nf2][nf1][nf0] leaf ids
    float inv_lnr;                    // 1 / ln(r_max / r_min) (log) or 1 / (r_max - r_min)
    float inv_thspan;
};

struct ParamsK {
    int dmumu, p_update, kappa_drift, dvdt_term;
    int use_rig;
    float lambda_par, p_ref, alpha, q, H, eps, mu_floor, lambda_perp, dt;
    uint32_t seed, set_id;
    float inv_lambda_par;      // 1 / lambda_par, so that a step divides by nothing constant
};

struct ObsK {
    int kind, ne, nt, off;
    float r, dr, th, dth, ph, dph;
    float e_lo, ne_over_lnratio;   // i_E = floor(ln(E / e_lo) * ne / ln(e_hi / e_lo))
    float phi_scale;               // ring: longitude bin = floor(phi * nt / (2 pi))
};

// Per-step entry of the time table (built in FP64 by step_table_kernel).
struct StepEntry {
    int s0, s1;              // bracketing snapshots
    float wt;                // weight of s1
    int two;                 // 1: two snapshots and dV/dt from their difference
    short it[FTE_MAX_OBS];   // time bin per observer, -1 outside [t_lo, t_hi)
};
static_assert(sizeof(StepEntry) == 32, "StepEntry layout");

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications (high words mixed into the other lanes with the round key),
// the key advanced by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// 32-bit word -> uniform in (0, 1): ((x >> 8) + 1/2) 2^-24 (25 significant bits,
// rounded to nearest in FP32).
__device__ __forceinline__ float u01(uint32_t x)
{
    return (float)(x >> 8) * (1.0f / 16777216.0f) + (0.5f / 16777216.0f);
}

// 2 u - 1 for the same word, exactly: (2 (x >> 8) + 1 - 2^24) 2^-24 has at most 24 bits.
__device__ __forceinline__ float u11(uint32_t x)
{
    return (float)((int)((x >> 8) << 1) + 1 - (1 << 24)) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------------
// Kinematics: p in m_p c; v = c p / gamma; E = m c^2 p^2 / (gamma + 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float speed_of(float p) { return kCau * p * rsqrtf(fmaf(p, p, 1.0f)); }
__device__ __forceinline__ float energy_of(float p)
{
    const float g = sqrtf(fmaf(p, p, 1.0f));
    return kMc2 * p * p / (g + 1.0f);
}

// ---------------------------------------------------------------------------
// Pitch-angle diffusion coefficient and its mu derivative (Eq. 5 and the
// quasi-linear / isotropic alternatives).  `I` is the normalisation integral.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void dmumu(const ParamsK& P, float I, float mu, float v, float p,
                                      float& D, float& dD)
{
    const float ilam = P.use_rig ? 1.f / (P.lambda_par * powf(p / P.p_ref, P.alpha)) : P.inv_lambda_par;
    const float am = fabsf(mu);
    const float sg = (mu > 0.f) ? 1.f : ((mu < 0.f) ? -1.f : 0.f);
    const float omm = 1.f - mu * mu;
    if (P.dmumu == 0) {
        const float nu = 1.5f * v * I * ilam;
        // |mu|^(q-1) and max(|mu|, mu_floor)^(q-2) from one logarithm: above the floor
        // the first is the second times |mu| (two exp2/log2 instead of two powf)
        const float pq2 = exp2f((P.q - 2.f) * log2f(fmaxf(am, P.mu_floor)));
        const float pq1 = am >= P.mu_floor ? pq2 * am : exp2f((P.q - 1.f) * log2f(am));
        const float g = pq1 + P.H;
        const float dg = (P.q - 1.f) * pq2 * sg;
        D = 0.5f * nu * omm * g;
        dD = 0.5f * nu * (-2.f * mu * g + omm * dg);
    } else if (P.dmumu == 1) {
        const float D0 = 0.75f * v * I * ilam;
        const float h = am / (1.f + am) + P.eps;
        const float dh = sg / ((1.f + am) * (1.f + am));
        D = D0 * h * omm;
        dD = D0 * (dh * omm - 2.f * mu * h);
    } else {
        const float Dc = 0.5f * v * ilam;
        D = Dc * omm;
        dD = -2.f * mu * Dc;
    }
}

// ---------------------------------------------------------------------------
// Grid location: bracketing cell centres and weights along each axis.
// Beyond the outermost centres in r and theta the field is held constant.
// ---------------------------------------------------------------------------
struct Loc {
    int i0, j0, k0, k1;
    int base[4];             // record (within a snapshot) of the lower r-neighbour of corner
                             // c = ct + 2 cp, ct/cp the upper theta/phi neighbour flags
    float fr, ft, fp;        // weights of the upper neighbour
    float dfr, dft, dfp;     // d(weight)/d(coordinate); 0 where clamped
};

// Block AMR: the leaf holding a point and the point's cell within it (interior
// indices 0..B-1 along r, theta, phi).
__device__ __forceinline__ int amr_containing(const GridK& g, float r, float th, float ph, int& ci, int& cj,
                                              int& ck)
{
    const float ur = g.radial ? logf(r / g.r_min) * g.inv_lnr : (r - g.r_min) * g.inv_lnr;
    const float ut = (th - g.th_min) * g.inv_thspan;
    const float up = ph * (1.f / kTwoPi);
    const int f0 = min(max((int)floorf(ur * (float)g.nf0), 0), g.nf0 - 1);
    const int f1 = min(max((int)floorf(ut * (float)g.nf1), 0), g.nf1 - 1);
    int f2 = (int)floorf(up * (float)g.nf2);
    if (f2 < 0) f2 += g.nf2;
    if (f2 >= g.nf2) f2 -= g.nf2;
    // the clamp keeps every address inside the arrays even for a table that was never prepared
    const int leaf = min(max(__ldg(g.table + ((long long)f2 * g.nf1 + f1) * g.nf0 + f0), 0), g.amr_leaves - 1);
    const int4 lf = __ldg(g.leaves + leaf);
    const float s = (float)(1 << lf.x);
    const float xr = (g.radial ? logf(r / g.r_min) * g.inv_dr : (r - g.r_min) * g.inv_dr) * s;
    ci = min(max((int)floorf(xr) - lf.y * g.B, 0), g.B - 1);
    cj = min(max((int)floorf((th - g.th_min) * g.inv_dth * s) - lf.z * g.B, 0), g.B - 1);
    ck = min(max((int)floorf(ph * g.inv_dph * s) - lf.w * g.B, 0), g.B - 1);
    return leaf;
}

// Block AMR: leaf from the finest-level table, then the bracketing cells on the
// leaf's padded lattice (level-l cell coordinate x = u n_l - 1/2, weights in the
// physical coordinate).  The ghost layer supplies the neighbours' values.
__device__ __forceinline__ void locate_amr(const GridK& g, float r, float th, float ph, Loc& L)
{
    const float ur = g.radial ? logf(r / g.r_min) * g.inv_lnr : (r - g.r_min) * g.inv_lnr;
    const float ut = (th - g.th_min) * g.inv_thspan;
    const float up = ph * (1.f / kTwoPi);
    const int f0 = min(max((int)floorf(ur * (float)g.nf0), 0), g.nf0 - 1);
    const int f1 = min(max((int)floorf(ut * (float)g.nf1), 0), g.nf1 - 1);
    int f2 = (int)floorf(up * (float)g.nf2);
    if (f2 < 0) f2 += g.nf2;
    if (f2 >= g.nf2) f2 -= g.nf2;
    // the clamp keeps every address inside the arrays even for a table that was never prepared
    const int leaf = min(max(__ldg(g.table + ((long long)f2 * g.nf1 + f1) * g.nf0 + f0), 0), g.amr_leaves - 1);
    const int4 lf = __ldg(g.leaves + leaf);
    const float s = (float)(1 << lf.x);
    const int B = g.B, P = g.P;
    // r
    float x = (g.radial ? logf(r / g.r_min) * g.inv_dr : (r - g.r_min) * g.inv_dr) * s - 0.5f;
    int lo = lf.y * B - 1;
    int i = min(max((int)floorf(x), lo), lo + B);
    if (g.radial) {
        const float c0 = g.r_min * expf(((float)i + 0.5f) * g.dr / s);
        const float c1 = g.r_min * expf(((float)i + 1.5f) * g.dr / s);
        L.dfr = 1.f / (c1 - c0);
        L.fr = (r - c0) * L.dfr;
    } else {
        L.fr = x - (float)i;
        L.dfr = g.inv_dr * s;
    }
    const int ii = i - lo;
    // theta
    x = (th - g.th_min) * g.inv_dth * s - 0.5f;
    lo = lf.z * B - 1;
    i = min(max((int)floorf(x), lo), lo + B);
    L.ft = x - (float)i;
    L.dft = g.inv_dth * s;
    const int jj = i - lo;
    // phi
    x = ph * g.inv_dph * s - 0.5f;
    lo = lf.w * B - 1;
    i = min(max((int)floorf(x), lo), lo + B);
    L.fp = x - (float)i;
    L.dfp = g.inv_dph * s;
    const int kk = i - lo;
    const int b0 = ((leaf * P + kk) * P + jj) * P + ii;
    L.base[0] = b0;
    L.base[1] = b0 + P;
    L.base[2] = b0 + P * P;
    L.base[3] = b0 + P * P + P;
}

__device__ __forceinline__ void locate(const GridK& g, float r, float th, float ph, Loc& L)
{
    if (g.amr) {
        locate_amr(g, r, th, ph, L);
        return;
    }
    float xi = g.radial ? logf(r / g.r_min) * g.inv_dr - 0.5f : (r - g.r_min) * g.inv_dr - 0.5f;
    if (xi < 0.f) {
        L.i0 = 0; L.fr = 0.f; L.dfr = 0.f;
    } else if (xi >= (float)(g.nr - 1)) {
        L.i0 = g.nr - 2; L.fr = 1.f; L.dfr = 0.f;
    } else {
        L.i0 = (int)xi;
        if (g.radial) {
            const float c0 = g.r_min * expf(((float)L.i0 + 0.5f) * g.dr);
            const float c1 = g.r_min * expf(((float)L.i0 + 1.5f) * g.dr);
            L.dfr = 1.f / (c1 - c0);
            L.fr = (r - c0) * L.dfr;
        } else {
            L.fr = xi - (float)L.i0;
            L.dfr = g.inv_dr;
        }
    }
    xi = (th - g.th_min) * g.inv_dth - 0.5f;
    if (xi < 0.f) {
        L.j0 = 0; L.ft = 0.f; L.dft = 0.f;
    } else if (xi >= (float)(g.nth - 1)) {
        L.j0 = g.nth - 2; L.ft = 1.f; L.dft = 0.f;
    } else {
        L.j0 = (int)xi;
        L.ft = xi - (float)L.j0;
        L.dft = g.inv_dth;
    }
    xi = ph * g.inv_dph - 0.5f;
    const float kf = floorf(xi);
    L.fp = xi - kf;
    L.dfp = g.inv_dph;
    int k0 = (int)kf;
    if (k0 < 0) k0 += g.nph;
    if (k0 >= g.nph) k0 -= g.nph;
    L.k0 = k0;
    L.k1 = (k0 + 1 == g.nph) ? 0 : k0 + 1;
    L.base[0] = (L.k0 * g.nth + L.j0) * g.nr + L.i0;
    L.base[1] = L.base[0] + g.nr;
    L.base[2] = (L.k1 * g.nth + L.j0) * g.nr + L.i0;
    L.base[3] = L.base[2] + g.nr;
}

// 32-byte read-only loads (one sector each); the address must be 32-byte aligned.
__device__ __forceinline__ void ldg8(const float* q, float* v)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
          "=f"(v[7])
        : "l"(q));
}

__device__ __forceinline__ void ldg8u(const uint32_t* q, uint32_t* v)
{
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7])
        : "l"(q));
}

// Narrower loads for the tail of a record: the L1 returns a warp's loaded bytes to
// registers at 128 bytes per data-pipe wavefront, so bytes of padding loaded cost
// as much as bytes used.  Alignment: 16 (v4), 8 (v2) or 4 bytes.
__device__ __forceinline__ void ldg4(const float* q, float* v)
{
    asm("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(q));
}

__device__ __forceinline__ void ldg2(const float* q, float* v)
{
    asm("ld.global.nc.v2.f32 {%0,%1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "l"(q));
}

__device__ __forceinline__ void ldg2u(const uint32_t* q, uint32_t* v)
{
    asm("ld.global.nc.v2.b32 {%0,%1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "l"(q));
}

__device__ __forceinline__ void ldg1u(const uint32_t* q, uint32_t* v)
{
    asm("ld.global.nc.b32 %0, [%1];" : "=r"(v[0]) : "l"(q));
}

// 16-bit storage formats: value k of a record is half k & 1 of 32-bit word k >> 1.
template <int DT>
__device__ __forceinline__ float h_lo(uint32_t w)
{
    if (DT == FTE_BF16) return __uint_as_float(w << 16);
    return __half2float(__ushort_as_half((unsigned short)(w & 0xFFFFu)));
}
template <int DT>
__device__ __forceinline__ float h_hi(uint32_t w)
{
    if (DT == FTE_BF16) return __uint_as_float(w & 0xFFFF0000u);
    return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
}
template <int DT>
__device__ __forceinline__ float h_get(const uint32_t* words, int k)
{
    return (k & 1) ? h_hi<DT>(words[k >> 1]) : h_lo<DT>(words[k >> 1]);
}

// Interpolated background at the particle (18 fields, dV/dt partial, and the
// axis derivatives of B when the cross-field drift is on).
template <bool KPERP>
struct Fields {
    float f[FTE_NFIELD];
    float dv[3];             // sum_c w_c (V_s1 - V_s0): times 1/dt_snap gives dV/dt
    float dBa[KPERP ? 9 : 1];  // dB_i / d(weight axis a), a = r, theta, phi
};

// The stored fields of the two r-neighbours of one corner pair: record `rec` and
// the next one (cell layout) or the one pair record; 16-bit values are returned
// unscaled.
// Record layout of a kernel, fixed at compile time (each kernel is built for both).
constexpr int kLayCell = 0, kLayPair = 1;

template <int DT, int LAY>
__device__ __forceinline__ void corner_pair(const GridK& g, long long rec, float* lo, float* hi)
{
    // Only the 18 stored fields of each cell are loaded, the last piece of a record
    // with a narrower load (FP32 pair: 4 x 32 + 16 bytes of 160; FP32 cell: 2 x 32 +
    // 8 of 96 per record; 16-bit pair: 2 x 32 + 8 of 96; 16-bit cell: 32 + 4 of 64).
    constexpr bool pair = LAY == kLayPair;
    static_assert(FTE_NFIELD == 18, "load pattern assumes 18 fields per cell");
    if (DT == FTE_F32) {
        if (pair) {
            float a[2 * FTE_NFIELD];
            const float* q = g.fields + rec * kPairRec;
#pragma unroll
            for (int m = 0; m < 4; ++m) ldg8(q + 8 * m, a + 8 * m);
            ldg4(q + 32, a + 32);
#pragma unroll
            for (int m = 0; m < FTE_NFIELD; ++m) { lo[m] = a[m]; hi[m] = a[FTE_NFIELD + m]; }
        } else {
            const float* q = g.fields + rec * FTE_REC;
            ldg8(q, lo);
            ldg8(q + 8, lo + 8);
            ldg2(q + 16, lo + 16);
            ldg8(q + FTE_REC, hi);
            ldg8(q + FTE_REC + 8, hi + 8);
            ldg2(q + FTE_REC + 16, hi + 16);
        }
    } else if (pair) {
        uint32_t u[FTE_NFIELD];       // 36 values in 18 words
        const uint32_t* q = g.hfields + rec * (kPairHRec / 2);
        ldg8u(q, u);
        ldg8u(q + 8, u + 8);
        ldg2u(q + 16, u + 16);
#pragma unroll
        for (int m = 0; m < FTE_NFIELD; ++m) {
            lo[m] = h_get<DT>(u, m);
            hi[m] = h_get<DT>(u, FTE_NFIELD + m);
        }
    } else {
        uint32_t u[FTE_HREC];         // two records of FTE_HREC / 2 words; 9 words used of each
        const uint32_t* q = g.hfields + rec * (FTE_HREC / 2);
        ldg8u(q, u);
        ldg1u(q + 8, u + 8);
        ldg8u(q + FTE_HREC / 2, u + FTE_HREC / 2);
        ldg1u(q + FTE_HREC / 2 + 8, u + FTE_HREC / 2 + 8);
#pragma unroll
        for (int m = 0; m < FTE_NFIELD; ++m) {
            lo[m] = h_get<DT>(u, m);
            hi[m] = h_get<DT>(u + FTE_HREC / 2, m);
        }
    }
}

// d0 = a0 * b0 + d0 and d1 = a1 * b1 + d1 in one paired FP32 FMA (each lane a fused
// multiply-add rounded once, so the results equal two fmaf calls).
__device__ __forceinline__ void fma2(float& d0, float& d1, float a0, float a1, float b0, float b1)
{
    unsigned long long d, a, b, c;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b0), "f"(b1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(d0), "f"(d1));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d));
}

// Trilinear (space) x linear (time) interpolation: for each snapshot and each
// of the 4 (theta, phi) corners, the two r-neighbours are one contiguous block
// (pair layout: one record; 144 of its bytes loaded in FP32, 72 in 16-bit).  For 16-bit
// storage the sums run over the stored values and the per-field scales `sc`
// are applied once at the end.
// PAIRED: accumulate with paired FMAs (the step kernels with the global tally; the
// adjoint kernels, at their register bound, measured faster with scalar FMAs; both
// round identically).
template <bool KPERP, int DT, int LAY, bool PAIRED = false>
__device__ __forceinline__ void gather(const GridK& g, const StepEntry& e, const Loc& L,
                                       const float* sc, Fields<KPERP>& F)
{
#pragma unroll
    for (int m = 0; m < FTE_NFIELD; ++m) F.f[m] = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) F.dv[m] = 0.f;
    if (KPERP) {
#pragma unroll
        for (int m = 0; m < 9; ++m) F.dBa[m] = 0.f;
    }
    const int ns = e.two ? 2 : 1;
    for (int s = 0; s < ns; ++s) {
        const int snap = s ? e.s1 : e.s0;
        const float ws = e.two ? (s ? e.wt : 1.f - e.wt) : 1.f;
        const float sgn = s ? 1.f : -1.f;
        // V of this snapshot, spatially interpolated: it enters F (weighted by ws) and
        // the snapshot difference for dV/dt, from one set of accumulators
        float vs[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int ct = c & 1, cp = c >> 1;
            const float wt_ = ct ? L.ft : 1.f - L.ft;
            const float wp_ = cp ? L.fp : 1.f - L.fp;
            const float wjk = wt_ * wp_;
            const long long rec = (long long)snap * g.snap_recs + L.base[c];
            float lo[FTE_NFIELD], hi[FTE_NFIELD];
            corner_pair<DT, LAY>(g, rec, lo, hi);
            const float c0 = (1.f - L.fr) * wjk, c1 = L.fr * wjk;
            const float w0 = ws * c0, w1 = ws * c1;
            // acc = w0 lo + (w1 hi + acc) per field, two fields per paired FMA along the
            // record's field pairs: (B_x, B_y), (B_z, V_x), (V_y, V_z), then the gradients;
            // V goes to this snapshot's vs with the spatial weights c0, c1 alone
            if (PAIRED) {
                fma2(F.f[0], F.f[1], w1, w1, hi[0], hi[1]);
                fma2(F.f[0], F.f[1], w0, w0, lo[0], lo[1]);
                fma2(F.f[2], vs[0], w1, c1, hi[2], hi[3]);
                fma2(F.f[2], vs[0], w0, c0, lo[2], lo[3]);
                fma2(vs[1], vs[2], c1, c1, hi[4], hi[5]);
                fma2(vs[1], vs[2], c0, c0, lo[4], lo[5]);
#pragma unroll
                for (int m = 6; m < FTE_NFIELD; m += 2) {
                    fma2(F.f[m], F.f[m + 1], w1, w1, hi[m], hi[m + 1]);
                    fma2(F.f[m], F.f[m + 1], w0, w0, lo[m], lo[m + 1]);
                }
            } else {
#pragma unroll
                for (int m = 0; m < FTE_NFIELD; ++m) {
                    if (m >= 3 && m < 6) continue;
                    F.f[m] = fmaf(w0, lo[m], fmaf(w1, hi[m], F.f[m]));
                }
#pragma unroll
                for (int m = 0; m < 3; ++m) vs[m] = fmaf(c0, lo[3 + m], fmaf(c1, hi[3 + m], vs[m]));
            }
            if (KPERP) {
                const float er = L.dfr * wjk;                          // d w / d r
                const float et = (ct ? 1.f : -1.f) * L.dft * wp_;      // d w / d theta (x w_r)
                const float ep = (cp ? 1.f : -1.f) * L.dfp * wt_;      // d w / d phi   (x w_r)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float mix = (1.f - L.fr) * lo[m] + L.fr * hi[m];
                    F.dBa[3 * m + 0] += ws * er * (hi[m] - lo[m]);
                    F.dBa[3 * m + 1] += ws * et * mix;
                    F.dBa[3 * m + 2] += ws * ep * mix;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            F.f[3 + m] = fmaf(ws, vs[m], F.f[3 + m]);
            if (e.two) F.dv[m] = fmaf(sgn, vs[m], F.dv[m]);
        }
    }
    if (DT != FTE_F32) {
#pragma unroll
        for (int m = 0; m < FTE_NFIELD; ++m) F.f[m] *= sc[m];
#pragma unroll
        for (int m = 0; m < 3; ++m) F.dv[m] *= sc[3 + m];
        if (KPERP) {
#pragma unroll
            for (int m = 0; m < 9; ++m) F.dBa[m] *= sc[m / 3];
        }
    }
}

}  // namespace fte
