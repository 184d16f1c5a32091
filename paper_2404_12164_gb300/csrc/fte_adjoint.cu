// Adjoint of the transport (Sec. 2.1 steps, Sec. 2.4 interpolation): gradients
// of a smooth observable J = sum_i w_i sum_n dt K(x_n, E_n, t_n) with respect to
// the pitch-angle-diffusion parameters (lambda_par, q, H, eps), pathwise with the
// Philox noise of every step held fixed except at the steps whose pitch-angle
// Gaussian reaches mu = 0, which enter in the score (likelihood-ratio) form (see
// step_vjp), and with respect to the injection spectral index through the
// likelihood ratio of the injected energies.
//
// Forward: the run is cut into segments of K steps; every particle stores its
// state at each segment start (checkpoints).  Reverse: segment by segment from
// the last, every particle replays its segment from the checkpoint (start-of-
// step states into per-thread scratch) and walks it backwards:
// lambda_n = (dF/ds_n)^T lambda_{n+1} + w dt grad K(s_n), and the parameter
// adjoint gains (dF/dtheta)^T lambda_{n+1}; the adjoints cross segment borders
// through global memory.  Discrete decisions of a step (cell, reflection,
// clamp, absorption) are those of the replayed path.  Each launch may take the
// particles in spatial order (a counting sort by grid bucket of the positions
// the launch starts from), which changes no result.
#include "fte_step.cuh"

namespace fte {

// ---------------------------------------------------------------------------
// d/dq and d/dH (quasi-linear) or d/deps (Eq. 5) of the normalisation integral,
// same nodes as launch_norm: mu = s^3, Simpson on [0, 1] in s.
// out[0] = dI/dq, out[1] = dI/dH or dJ/deps.
// ---------------------------------------------------------------------------
constexpr int kNdInt = 16384;
constexpr int kNdThreads = 256;
constexpr int kNdBlocks = kNdInt / kNdThreads + 1;

__global__ void __launch_bounds__(kNdThreads) normd_partial_kernel(int model, double q, double H, double eps,
                                                                   double* part)
{
    __shared__ double sh[2][kNdThreads];
    const int i = blockIdx.x * kNdThreads + threadIdx.x;
    double f1 = 0.0, f2 = 0.0;
    if (model != 2 && i <= kNdInt) {
        const double u = (double)i / kNdInt;
        const double m = u * u * u;
        const double wgt = (i == 0 || i == kNdInt) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        const double jac = wgt * 3.0 * u * u * (1.0 - m * m);
        if (model == 0) {
            const double pm = m > 0.0 ? pow(m, q - 1.0) : 0.0;
            const double den = pm + H;
            f1 = m > 0.0 ? -jac * pm * log(m) / (den * den) : 0.0;
            f2 = -jac / (den * den);
        } else {
            const double den = m / (1.0 + m) + eps;
            f2 = -jac / (den * den);
        }
    }
    sh[0][threadIdx.x] = f1;
    sh[1][threadIdx.x] = f2;
    __syncthreads();
    for (int o = kNdThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh[0][0];
        part[2 * blockIdx.x + 1] = sh[1][0];
    }
}

__global__ void normd_final_kernel(const double* part, double* out)
{
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kNdBlocks; ++k) { a += part[2 * k]; b += part[2 * k + 1]; }
    out[0] = a / (3.0 * kNdInt);
    out[1] = b / (3.0 * kNdInt);
}

// ---------------------------------------------------------------------------
// Smooth observable K(r, E, t) and its gradient with respect to (x, y, z, p);
// c = (t - t_c) / sigma_t is passed in (see time_arg).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float smooth_k(const AdjK& k, float r, float p, float c, float* dKdr, float* dKdp)
{
    const float E = energy_of(p);
    const float a = (r - k.r_o) * k.inv_sr;
    const float b = logf(E * k.inv_ec) * k.inv_se;
    const float K = expf(-0.5f * (a * a + b * b + c * c));
    if (dKdr) {
        *dKdr = -K * a * k.inv_sr;
        // dE/dp = m c^2 p / sqrt(1 + p^2)
        const float dEdp = kMc2 * p * rsqrtf(fmaf(p, p, 1.f));
        *dKdp = -K * b * k.inv_se * dEdp / E;
    }
    return K;
}

// The observable's time argument at step s in FP32: c0 + s * cstep with c0 =
// (t0 - t_c) / sigma_t (FP64, rounded once); it depends on s alone, not on how
// the run is cut into launches.
__device__ __forceinline__ float time_arg(const AdjK& k, long long s)
{
    return fmaf((float)s, k.cstep, k.c0);
}

// ---------------------------------------------------------------------------
// Derivatives of D_mumu and dD_mumu/dmu (the functions `dmumu` evaluates) with
// respect to mu, v and the parameters; gth gains Dbar dD/dtheta + dDbar ddD/dtheta
// for theta = (lambda_par, q, H, eps).
// ---------------------------------------------------------------------------
constexpr float kLn2f = 0.693147180559945309f;

__device__ __forceinline__ void dmumu_vjp(const ParamsK& P, float I, float rq, float rh, float mu, float v,
                                          float Db, float dDb, float& mub, float& vb, float* gth)
{
    const float am = fabsf(mu);
    const float sg = (mu > 0.f) ? 1.f : ((mu < 0.f) ? -1.f : 0.f);
    const float omm = 1.f - mu * mu;
    float D, dD, D_mu, dD_mu, D_q = 0.f, dD_q = 0.f, D_h = 0.f, dD_h = 0.f, D_e = 0.f, dD_e = 0.f;
    if (P.dmumu == 0) {
        const float nu = 1.5f * v * I * P.inv_lambda_par;
        // the powers of |mu| from one base-2 logarithm: |mu|^(q-1), then divided by |mu|
        // (la = -inf and pq1 = 0 at mu = 0, where the terms that divide are not used)
        const float la = log2f(am);
        const float pq1 = exp2f((P.q - 1.f) * la);
        const float ia = 1.f / am;
        const float g = pq1 + P.H;
        const float amf = fmaxf(am, P.mu_floor);
        const float laf = am >= P.mu_floor ? la : log2f(amf);
        const float pf2 = am >= P.mu_floor ? pq1 * ia : exp2f((P.q - 2.f) * laf);
        const float gp = (P.q - 1.f) * pf2 * sg;
        D = 0.5f * nu * omm * g;
        dD = 0.5f * nu * (-2.f * mu * g + omm * gp);
        const float gmu = am > 0.f ? (P.q - 1.f) * (pq1 * ia) * sg : 0.f;
        const float gpmu = am > P.mu_floor ? (P.q - 1.f) * (P.q - 2.f) * (pq1 * ia * ia) : 0.f;
        D_mu = 0.5f * nu * (-2.f * mu * g + omm * gmu);
        dD_mu = 0.5f * nu * (-2.f * g - 2.f * mu * gmu - 2.f * mu * gp + omm * gpmu);
        const float gq = am > 0.f ? pq1 * (la * kLn2f) : 0.f;
        const float gpq = (pf2 + (P.q - 1.f) * pf2 * (laf * kLn2f)) * sg;
        D_q = 0.5f * nu * omm * gq + D * rq;
        dD_q = 0.5f * nu * (-2.f * mu * gq + omm * gpq) + dD * rq;
        D_h = 0.5f * nu * omm + D * rh;
        dD_h = 0.5f * nu * (-2.f * mu) + dD * rh;
    } else if (P.dmumu == 1) {
        const float D0 = 0.75f * v * I * P.inv_lambda_par;
        const float opa = 1.f + am;
        const float h = am / opa + P.eps;
        const float dh = sg / (opa * opa);
        const float ddh = am > 0.f ? -2.f / (opa * opa * opa) : 0.f;
        D = D0 * h * omm;
        dD = D0 * (dh * omm - 2.f * mu * h);
        D_mu = dD;
        dD_mu = D0 * (ddh * omm - 4.f * mu * dh - 2.f * h);
        D_e = D0 * omm + D * rh;
        dD_e = D0 * (-2.f * mu) + dD * rh;
    } else {
        const float Dc = 0.5f * v * P.inv_lambda_par;
        D = Dc * omm;
        dD = -2.f * mu * Dc;
        D_mu = dD;
        dD_mu = -2.f * Dc;
    }
    mub += Db * D_mu + dDb * dD_mu;
    vb += (Db * D + dDb * dD) / v;
    gth[0] -= (Db * D + dDb * dD) * P.inv_lambda_par;
    gth[1] += Db * D_q + dDb * dD_q;
    gth[2] += Db * D_h + dDb * dD_h;
    gth[3] += Db * D_e + dDb * dD_e;
}

// ---------------------------------------------------------------------------
// Vector-Jacobian product of one step (lambda_perp = 0): lam holds the adjoint
// of the state after step n on entry and of the state before it on return.
// Score form (win > 0): when the pitch-angle Gaussian's mean m lies within win
// widths s of a value landing at mu = 0, mu' is held instead of differentiated:
// the derivative of ln p(mu' | m, s) (p the Gaussian with its reflection images
// 2 - mu', -2 - mu'), times Gto, the observable accumulated after the step, takes
// the place of the adjoint of mu'; m and s then carry it back to the state and
// the parameters exactly as the pathwise adjoint would.
// ---------------------------------------------------------------------------
template <int DT, int LAY>
__device__ void step_vjp(const AdvanceArgs& a, float I, float rq, float rh, long long n, uint32_t pid, float x,
                         float y, float z, float mu, float p, const float* sc, float Gto, float win, float* lam,
                         float* gth)
{
    const GridK& g = a.g;
    const ParamsK& P = a.prm;
    const StepEntry* ep = a.table + (n - a.n_table0);
    StepEntry e;
    {
        const int4 h = __ldg(reinterpret_cast<const int4*>(ep));
        e.s0 = h.x; e.s1 = h.y; e.wt = __int_as_float(h.z); e.two = h.w;
    }
    const float rho2 = x * x + y * y;
    const float r = sqrtf(rho2 + z * z);
    const float rho = sqrtf(rho2);
    const float th = atan2f(rho, z);
    float ph = atan2f(y, x);
    if (ph < 0.f) ph += kTwoPi;
    Loc L;
    locate(g, r, th, ph, L);
    Fields<false> F;
    gather<false, DT, LAY>(g, e, L, sc, F);
    const float* B = F.f;
    const float* V = F.f + 3;
    const float* G = F.f + 6;
    const float* gB = F.f + 15;
    const float invB = rsqrtf(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    const float b[3] = {B[0] * invB, B[1] * invB, B[2] * invB};
    const float bgb = b[0] * gB[0] + b[1] * gB[1] + b[2] * gB[2];
    const float divb = -bgb * invB;
    const float divv = G[0] + G[4] + G[8];
    float Gb[3], bG[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Gb[i] = G[3 * i] * b[0] + G[3 * i + 1] * b[1] + G[3 * i + 2] * b[2];
        bG[i] = b[0] * G[i] + b[1] * G[3 + i] + b[2] * G[6 + i];
    }
    const float bbgv = b[0] * Gb[0] + b[1] * Gb[1] + b[2] * Gb[2];
    const float st = e.two ? g.inv_dt_snap : 0.f;
    float acc[3] = {0.f, 0.f, 0.f};
    float bdvdt = 0.f;
    if (P.dvdt_term) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
            acc[i] = F.dv[i] * st + G[3 * i] * V[0] + G[3 * i + 1] * V[1] + G[3 * i + 2] * V[2];
        bdvdt = b[0] * acc[0] + b[1] * acc[1] + b[2] * acc[2];
    }
    const float v = speed_of(p);
    const float iv = 1.f / v;      // the step and its VJP divide by v only through iv
    float D, dD;
    dmumu(P, I, mu, v, p, D, dD);
    const uint4 rb = philox4x32_10(make_uint4((uint32_t)n, pid, 0u, 0u), make_uint2(P.seed, P.set_id));
    const float amp0 = sqrtf(-2.f * logf(u01(rb.x)));
    float s1, c1;
    sincospif(2.f * u01(rb.y), &s1, &c1);
    const float zmu = amp0 * c1;
    const float dt = P.dt;
    const float omm = 1.f - mu * mu;
    const float Q = v * divb + mu * divv - 3.f * mu * bbgv - 2.f * iv * bdvdt;
    const float mudot = 0.5f * omm * Q;
    const float mu1 = mu + (mudot + dD) * dt + sqrtf(2.f * D * dt) * zmu;
    float fm = 1.f, m2 = mu1;
    if (m2 > 1.f) { m2 = 2.f - m2; fm = -fm; }
    if (m2 < -1.f) { m2 = -2.f - m2; fm = -fm; }
    if (m2 > 1.f || m2 < -1.f) fm = 0.f;
    const float pdot = 0.5f * (1.f - 3.f * mu * mu) * bbgv - 0.5f * omm * divv - mu * iv * bdvdt;
    const float ep_ = (P.p_update == 0) ? expf(pdot * dt) : 1.f + pdot * dt;

    // ---- reverse ----
    const float xnb[3] = {lam[0], lam[1], lam[2]};
    float pb = lam[4] * ep_;
    const float pdotb = (P.p_update == 0) ? lam[4] * p * ep_ * dt : lam[4] * p * dt;
    float xb[3] = {xnb[0], xnb[1], xnb[2]};
    const float ub[3] = {xnb[0] * dt, xnb[1] * dt, xnb[2] * dt};
    // adjoints of the Gaussian's mean (m1b) and of its width times dsigma/dD's z factor (zb)
    float m1b = lam[3] * fm, zb = m1b * zmu;
    if (win > 0.f && D > 0.f) {
        const float mm = mu + (mudot + dD) * dt;
        const float sg = sqrtf(2.f * D * dt);
        const float am = fabsf(mm);
        if (fminf(am, fabsf(am - 2.f)) < win * sg) {
            const float is = 1.f / sg;
            const float mc = fminf(fmaxf(m2, -1.f), 1.f);
            const float z0 = (mc - mm) * is, z1 = (2.f - mc - mm) * is, z2 = (-2.f - mc - mm) * is;
            const float e0 = z0 * z0, e1 = z1 * z1, e2 = z2 * z2;
            const float emin = fminf(e0, fminf(e1, e2));
            const float w0 = __expf(-0.5f * (e0 - emin)), w1 = __expf(-0.5f * (e1 - emin)),
                        w2 = __expf(-0.5f * (e2 - emin));
            const float gw = Gto * is / (w0 + w1 + w2);
            m1b = gw * (w0 * z0 + w1 * z1 + w2 * z2);                       // G d ln p / dm
            zb = gw * (w0 * (e0 - 1.f) + w1 * (e1 - 1.f) + w2 * (e2 - 1.f));  // G d ln p / ds
        }
    }
    float mub = m1b;
    const float mudotb = m1b * dt;
    const float dDb = m1b * dt;
    const float Db = D > 0.f ? zb * dt * rsqrtf(2.f * D * dt) : 0.f;
    // u = V + mu v b
    const float ubb = ub[0] * b[0] + ub[1] * b[1] + ub[2] * b[2];
    float Vb[3] = {ub[0], ub[1], ub[2]};
    mub += v * ubb;
    float vb = mu * ubb;
    float bb[3] = {mu * v * ub[0], mu * v * ub[1], mu * v * ub[2]};
    // pdot
    float bbgvb = 0.5f * (1.f - 3.f * mu * mu) * pdotb;
    mub += pdotb * (-3.f * mu * bbgv + mu * divv - bdvdt * iv);
    float divvb = -0.5f * omm * pdotb;
    float bdvdtb = -(mu * iv) * pdotb;
    vb += (mu * iv * iv) * bdvdt * pdotb;
    // mudot = omm Q / 2
    mub += mudotb * (-mu * Q + 0.5f * omm * (divv - 3.f * bbgv));
    const float Qb = 0.5f * omm * mudotb;
    vb += Qb * (divb + 2.f * bdvdt * (iv * iv));
    const float divbb = Qb * v;
    divvb += Qb * mu;
    bbgvb += -3.f * mu * Qb;
    bdvdtb += -(2.f * iv) * Qb;
    // D, dD/dmu
    dmumu_vjp(P, I, rq, rh, mu, v, Db, dDb, mub, vb, gth);
    // v(p)
    {
        const float ro = rsqrtf(fmaf(p, p, 1.f));
        pb += vb * kCau * (ro * ro * ro);
    }
    // background quantities -> fields
    float Fb[FTE_NFIELD], dvb[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < FTE_NFIELD; ++m) Fb[m] = 0.f;
    Fb[3] = Vb[0]; Fb[4] = Vb[1]; Fb[5] = Vb[2];
    if (P.dvdt_term) {
        const float accb[3] = {bdvdtb * b[0], bdvdtb * b[1], bdvdtb * b[2]};
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            bb[i] += bdvdtb * acc[i];
            dvb[i] = accb[i] * st;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Fb[6 + 3 * i + j] += accb[i] * V[j];
                Fb[3 + j] += accb[i] * G[3 * i + j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) Fb[6 + 3 * i + j] += bbgvb * b[i] * b[j];
        bb[i] += bbgvb * (Gb[i] + bG[i]);
    }
    Fb[6] += divvb; Fb[10] += divvb; Fb[14] += divvb;
    float invBb = -divbb * bgb;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        bb[i] += -divbb * invB * gB[i];
        Fb[15 + i] = -divbb * invB * b[i];
    }
    invBb += bb[0] * B[0] + bb[1] * B[1] + bb[2] * B[2];
    const float ib3 = invB * invB * invB;
#pragma unroll
    for (int i = 0; i < 3; ++i) Fb[i] = bb[i] * invB - invBb * ib3 * B[i];

    // interpolation: second pass over the corner records
    if (DT != FTE_F32) {
#pragma unroll
        for (int m = 0; m < FTE_NFIELD; ++m) Fb[m] *= sc[m];
#pragma unroll
        for (int m = 0; m < 3; ++m) dvb[m] *= sc[3 + m];
    }
    float frb = 0.f, ftb = 0.f, fpb = 0.f;
    const int ns = e.two ? 2 : 1;
    for (int s = 0; s < ns; ++s) {
        const int snap = s ? e.s1 : e.s0;
        const float ws = e.two ? (s ? e.wt : 1.f - e.wt) : 1.f;
        const float sgn = s ? 1.f : -1.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int ct = c & 1, cp = c >> 1;
            const float wt_ = ct ? L.ft : 1.f - L.ft;
            const float wp_ = cp ? L.fp : 1.f - L.fp;
            const long long rec = (long long)snap * g.snap_recs + L.base[c];
            float lo[FTE_NFIELD], hi[FTE_NFIELD];
            corner_pair<DT, LAY>(g, rec, lo, hi);
            float dlo = 0.f, dhi = 0.f, vlo = 0.f, vhi = 0.f;
#pragma unroll
            for (int m = 0; m < FTE_NFIELD; ++m) { dlo += Fb[m] * lo[m]; dhi += Fb[m] * hi[m]; }
#pragma unroll
            for (int m = 0; m < 3; ++m) { vlo += dvb[m] * lo[3 + m]; vhi += dvb[m] * hi[3 + m]; }
            const float tlo = ws * dlo + (e.two ? sgn * vlo : 0.f);
            const float thi = ws * dhi + (e.two ? sgn * vhi : 0.f);
            frb += wt_ * wp_ * (thi - tlo);
            const float mix = (1.f - L.fr) * tlo + L.fr * thi;
            ftb += (ct ? 1.f : -1.f) * wp_ * mix;
            fpb += (cp ? 1.f : -1.f) * wt_ * mix;
        }
    }
    const float rb_ = frb * L.dfr, thb = ftb * L.dft, phb = fpb * L.dfp;
    // (r, theta, phi) of (x, y, z)
    const float ir = 1.f / r;
    xb[0] += rb_ * x * ir;
    xb[1] += rb_ * y * ir;
    xb[2] += rb_ * z * ir;
    if (rho > 0.f) {
        const float irr = ir * ir, irho = 1.f / rho;
        xb[0] += thb * x * z * irr * irho - phb * y * irho * irho;
        xb[1] += thb * y * z * irr * irho + phb * x * irho * irho;
        xb[2] += -thb * rho * irr;
    }
    lam[0] = xb[0]; lam[1] = xb[1]; lam[2] = xb[2]; lam[3] = mub; lam[4] = pb;
}

// ---------------------------------------------------------------------------
// Forward pass, one launch per segment of K steps: each alive particle (taken
// in spatial order from a.order when reordering is on) stores its checkpoint,
// runs the segment's steps and adds its observable to J_part.
// ---------------------------------------------------------------------------
template <int DT, int LAY>
__global__ void __launch_bounds__(256) adj_forward_kernel(const AdvanceArgs a, const AdjK k)
{
    __shared__ float sc[FTE_NFIELD];
    __shared__ double red[8];
    if (DT != FTE_F32 && threadIdx.x < FTE_NFIELD) sc[threadIdx.x] = __ldg(a.g.scale + threadIdx.x);
    __syncthreads();
    const float I = (float)__ldg(a.norm);
    const unsigned long long n_work = a.order ? (unsigned long long)__ldg(a.n_order) : a.n_particles;
    const size_t n = a.n_particles;
    float* c = k.ckpt + (size_t)k.seg * 5 * n;
    double jsum = 0.0;
    unsigned long long noor = 0;
    TallyRun nrun{-1, 0u};                 // the adjoint kernels run without observers
    for (;;) {
        unsigned long long fend = n_work;
        const unsigned long long f = a.fetch_slots ? warp_fetch_sm(a.fetch, a.fetch_slots, n_work, &fend)
                                                   : warp_fetch(a.fetch);
        if (__shfl_sync(0xffffffffu, f, 0) >= n_work) break;
        if (f >= fend) continue;
        const unsigned long long i = a.order ? (unsigned long long)__ldg(a.order + f) : f;
        if (!a.order && a.status[i] != FTE_ALIVE) continue;
        float x = a.x[i], y = a.y[i], z = a.z[i], mu = a.mu[i], p = a.p[i];
        if (k.ckpt_on) { c[i] = x; c[n + i] = y; c[2 * n + i] = z; c[3 * n + i] = mu; c[4 * n + i] = p; }
        const float w = a.w[i];
        const uint32_t pid = a.id[i];
        double J = 0.0;
        int st = FTE_ALIVE;
        long long s = a.n_start;
        for (; s < a.n_end; ++s) {
            const float r = sqrtf(x * x + y * y + z * z);
            J += (double)(w * a.prm.dt * smooth_k(k, r, p, time_arg(k, s), nullptr, nullptr));
            st = step<false, DT, kModeSingle, LAY>(a, a.prm, I, 0, s, pid, x, y, z, mu, p, w, nullptr, nullptr,
                                              nullptr, sc, noor, nrun);
            if (st != FTE_ALIVE) { ++s; break; }
        }
        // steps taken since the start of the run (a.n_table0), counting the one that ended it
        k.n_dead[i] = (int)(s - a.n_table0);
        k.J_part[i] += J;
        jsum += J;
        a.x[i] = x; a.y[i] = y; a.z[i] = z; a.mu[i] = mu; a.p[i] = p;
        if (st != FTE_ALIVE) a.status[i] = (uint8_t)st;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jsum += __shfl_down_sync(0xffffffffu, jsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        if (t != 0.0) atomicAdd(k.out, t);
    }
}

// ---------------------------------------------------------------------------
// Reverse pass, in two phases per checkpoint segment, each launched chunk by chunk
// (chunk [k.c_start, k.c_end), the particles reordered before the chunk's replay):
// the replay walks the chunk forwards from the checkpoint (or from the state the
// previous chunk left in k.carry) and stores every start-of-step state at the
// particle's position f in the chunk's order; the backward phase walks the chunks
// from the last, in the same order as their replay, and runs the step VJPs over
// the stored states, carrying the adjoints between launches in k.adj.  The launch
// of the run's first chunk adds the injection-index term and reduces the gradients.
// ---------------------------------------------------------------------------
template <int DT, int LAY>
__global__ void __launch_bounds__(256) adj_replay_kernel(const AdvanceArgs a, const AdjK k)
{
    __shared__ float sc[FTE_NFIELD];
    if (DT != FTE_F32 && threadIdx.x < FTE_NFIELD) sc[threadIdx.x] = __ldg(a.g.scale + threadIdx.x);
    __syncthreads();
    const float I = (float)__ldg(a.norm);
    const unsigned long long n_work = a.order ? (unsigned long long)__ldg(a.n_order) : a.n_particles;
    const size_t n = a.n_particles;
    const long long n0 = a.n_table0 + (long long)k.seg * k.K;    // segment start
    const long long cs = k.c_start, ce = k.c_end;
    const float* c = k.ckpt + (size_t)k.seg * 5 * n;
    unsigned long long noor = 0;
    TallyRun nrun{-1, 0u};                 // the adjoint kernels run without observers
    for (;;) {
        unsigned long long fend = n_work;
        const unsigned long long f = a.fetch_slots ? warp_fetch_sm(a.fetch, a.fetch_slots, n_work, &fend)
                                                   : warp_fetch(a.fetch);
        if (__shfl_sync(0xffffffffu, f, 0) >= n_work) break;
        if (f >= fend) continue;
        const unsigned long long i = a.order ? (unsigned long long)__ldg(a.order + f) : f;
        const long long nd = k.n_dead[i];
        if (nd <= cs - a.n_table0) continue;                  // not alive at this chunk's start
        const long long e = min(n0 + (long long)k.K, a.n_table0 + nd);   // end of its steps here
        const float* src = cs == n0 ? c : k.carry;
        float x = src[i], y = src[n + i], z = src[2 * n + i], mu = src[3 * n + i], p = src[4 * n + i];
        const float w = a.w[i];
        const uint32_t pid = a.id[i];
        const long long hi = min(ce, e);
        for (long long s = cs; s < hi; ++s) {
            float* sp = k.scratch + (size_t)(s - n0) * 5 * n + f;
            sp[0] = x; sp[n] = y; sp[2 * n] = z; sp[3 * n] = mu; sp[4 * n] = p;
            if (s + 1 < e)
                step<false, DT, kModeSingle, LAY>(a, a.prm, I, 0, s, pid, x, y, z, mu, p, w, nullptr, nullptr, nullptr,
                                             sc, noor, nrun);
        }
        if (ce < e) {      // the start of the next chunk
            float* cp = k.carry + i;
            cp[0] = x; cp[n] = y; cp[2 * n] = z; cp[3 * n] = mu; cp[4 * n] = p;
        }
    }
}

template <int DT, int LAY>
__global__ void __launch_bounds__(256, 2) adj_back_kernel(const AdvanceArgs a, const AdjK k)
{
    __shared__ float sc[FTE_NFIELD];
    __shared__ double red[8][FTE_NGRAD];
    if (DT != FTE_F32 && threadIdx.x < FTE_NFIELD) sc[threadIdx.x] = __ldg(a.g.scale + threadIdx.x);
    __syncthreads();
    const double In = __ldg(a.norm);
    const float I = (float)In;
    const float rq = (float)(__ldg(k.normd) / In), rh = (float)(__ldg(k.normd + 1) / In);
    const unsigned long long n_work = a.order ? (unsigned long long)__ldg(a.n_order) : a.n_particles;
    const size_t n = a.n_particles;
    const long long n0 = a.n_table0 + (long long)k.seg * k.K;
    const long long cs = k.c_start, ce = k.c_end;
    const bool closing = k.last && cs == n0;                    // the first chunk of the run
    const float* c = k.ckpt + (size_t)k.seg * 5 * n;
    double gsum[FTE_NGRAD];
#pragma unroll
    for (int q = 0; q < FTE_NGRAD; ++q) gsum[q] = 0.0;
    for (;;) {
        unsigned long long fend = n_work;
        const unsigned long long f = a.fetch_slots ? warp_fetch_sm(a.fetch, a.fetch_slots, n_work, &fend)
                                                   : warp_fetch(a.fetch);
        if (__shfl_sync(0xffffffffu, f, 0) >= n_work) break;
        if (f >= fend) continue;
        const unsigned long long i = a.order ? (unsigned long long)__ldg(a.order + f) : f;
        const long long nd = k.n_dead[i];
        if (nd <= cs - a.n_table0) continue;
        const long long e = min(n0 + (long long)k.K, a.n_table0 + nd);
        float lam[5], gth[4];
#pragma unroll
        for (int q = 0; q < 5; ++q) lam[q] = k.adj[q * n + i];
#pragma unroll
        for (int q = 0; q < 4; ++q) gth[q] = k.adj[(5 + q) * n + i];
        float Gacc = k.adj[9 * n + i];      // observable of the steps after the current one
        const float w = a.w[i];
        const uint32_t pid = a.id[i];
        for (long long s = min(ce, e) - 1; s >= cs; --s) {
            const float* sp = k.scratch + (size_t)(s - n0) * 5 * n + f;
            const float sx = sp[0], sy = sp[n], sz = sp[2 * n], smu = sp[3 * n], spp = sp[4 * n];
            step_vjp<DT, LAY>(a, I, rq, rh, s, pid, sx, sy, sz, smu, spp, sc, Gacc, k.lr_window, lam, gth);
            // the observable's own term at the start-of-step state
            const float r = sqrtf(sx * sx + sy * sy + sz * sz);
            float dKdr, dKdp;
            const float Kv = smooth_k(k, r, spp, time_arg(k, s), &dKdr, &dKdp);
            const float fw = w * a.prm.dt;
            lam[0] += fw * dKdr * sx / r;
            lam[1] += fw * dKdr * sy / r;
            lam[2] += fw * dKdr * sz / r;
            lam[4] += fw * dKdp;
            Gacc += fw * Kv;
        }
        if (!closing) {
#pragma unroll
            for (int q = 0; q < 5; ++q) k.adj[q * n + i] = lam[q];
#pragma unroll
            for (int q = 0; q < 4; ++q) k.adj[(5 + q) * n + i] = gth[q];
            k.adj[9 * n + i] = Gacc;
            continue;
        }
        // first step of the run: injection index by the likelihood ratio of the injected energy
        float gg = 0.f;
        if (k.score_on) gg = (float)(-(log((double)energy_of(c[4 * n + i])) - k.mean_lnE) * k.J_part[i]);
        if (k.per_particle) {
            float* o = k.per_particle + i * (1 + FTE_NGRAD);
            o[0] = (float)k.J_part[i];
            o[1] = gth[0]; o[2] = gth[1]; o[3] = gth[2]; o[4] = gth[3]; o[5] = gg;
        }
        gsum[0] += gth[0]; gsum[1] += gth[1]; gsum[2] += gth[2]; gsum[3] += gth[3]; gsum[4] += gg;
    }
    if (!closing) return;
#pragma unroll
    for (int q = 0; q < FTE_NGRAD; ++q) {
        double v = gsum[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < FTE_NGRAD) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q][threadIdx.x];
        atomicAdd(k.out + 1 + threadIdx.x, t);
    }
}

template <int LAY>
static const void* fwd_fn_lay(int dtype)
{
    if (dtype == FTE_BF16) return (const void*)adj_forward_kernel<FTE_BF16, LAY>;
    if (dtype == FTE_F16) return (const void*)adj_forward_kernel<FTE_F16, LAY>;
    return (const void*)adj_forward_kernel<FTE_F32, LAY>;
}

template <int LAY>
static const void* rep_fn_lay(int dtype)
{
    if (dtype == FTE_BF16) return (const void*)adj_replay_kernel<FTE_BF16, LAY>;
    if (dtype == FTE_F16) return (const void*)adj_replay_kernel<FTE_F16, LAY>;
    return (const void*)adj_replay_kernel<FTE_F32, LAY>;
}

template <int LAY>
static const void* back_fn_lay(int dtype)
{
    if (dtype == FTE_BF16) return (const void*)adj_back_kernel<FTE_BF16, LAY>;
    if (dtype == FTE_F16) return (const void*)adj_back_kernel<FTE_F16, LAY>;
    return (const void*)adj_back_kernel<FTE_F32, LAY>;
}

// record layout fixed at compile time, as for the step kernels; kind 0 forward,
// 1 backward VJP, 2 replay
static const void* adj_fn(int kind, int dtype, int pair)
{
    if (kind == 1) return pair ? back_fn_lay<kLayPair>(dtype) : back_fn_lay<kLayCell>(dtype);
    if (kind == 2) return pair ? rep_fn_lay<kLayPair>(dtype) : rep_fn_lay<kLayCell>(dtype);
    return pair ? fwd_fn_lay<kLayPair>(dtype) : fwd_fn_lay<kLayCell>(dtype);
}

cudaError_t adjoint_blocks(int dtype, int pair, int kind, int* blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, adj_fn(kind, dtype, pair), 256, 0);
}

static cudaError_t launch_adj(int kind, const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s)
{
    void* args[] = {(void*)&a, (void*)&k};
    return cudaLaunchKernel(adj_fn(kind, a.g.dtype, a.g.pair), dim3(blocks), dim3(256), args, 0, s);
}

cudaError_t launch_adjoint_forward(const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s)
{
    return launch_adj(0, a, k, blocks, s);
}

cudaError_t launch_adjoint_replay(const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s)
{
    return launch_adj(2, a, k, blocks, s);
}

cudaError_t launch_adjoint_back(const AdvanceArgs& a, const AdjK& k, int blocks, cudaStream_t s)
{
    return launch_adj(1, a, k, blocks, s);
}

cudaError_t launch_norm_derivs(int model, double q, double H, double eps, double* out, double* part,
                               cudaStream_t s)
{
    normd_partial_kernel<<<kNdBlocks, kNdThreads, 0, s>>>(model, q, H, eps, part);
    normd_final_kernel<<<1, 1, 0, s>>>(part, out);
    return cudaGetLastError();
}

}  // namespace fte
