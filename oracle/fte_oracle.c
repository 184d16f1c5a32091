/*
 * FP64 CPU oracle of the focused-transport particle pusher.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests/, by __graft_entry__.smoke() (as the
 * checker) and by the cpu_baseline / reference legs of bench.py.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Every function below restates one part of the method of Husidic et al. (2024),
 * Sec. 2.1-2.4, in plain double precision, in the order the method states it:
 *
 *   - Eq. 2  dx/dt  = V_sw + V_d + mu v b, with V_d = 0 (Sec. 2.1)
 *   - Eq. 3  dmu/dt = (1-mu^2)/2 (v div b + mu div V - 3 mu bb:grad V - (2/v) b.dV/dt)
 *   - Eq. 4  dp/dt  = [(1-3mu^2)/2 bb:grad V - (1-mu^2)/2 div V - (mu/v) b.dV/dt] p
 *   - Eq. 5  D_mumu = D0 (|mu|/(1+|mu|) + eps)(1-mu^2), plus the quasi-linear form
 *            (nu/2)(1-mu^2)(|mu|^(q-1) + H) and the isotropic form D(1-mu^2)
 *   - Sec. 2.1: Eqs. 1-4 are integrated as Ito SDEs forward in time; here by
 *            Euler-Maruyama, with the Ito drift dD_mumu/dmu in mu, reflection at
 *            mu = +-1, and cross-field diffusion kappa_perp = (v lambda_perp/3)(I-bb)
 *            with its Ito drift div(kappa_perp)
 *   - Sec. 2.4: locate the particle on the grid, read the surrounding cell
 *            values and interpolate them trilinearly at every step; snapshots
 *            are interpolated linearly in time
 *   - Eq. 7: injection uniform in volume over the div V < 0 region with weight
 *            1/r^2, mono-energetic or a power law in energy
 *   - Sec. 2.3 / Figs. 5-8: intensities from weighted occupancy tallies
 *
 * Readings where the paper is silent (normalisation of D0 from lambda_par,
 * the mu floor of the quasi-linear drift, the momentum update, the cross-field
 * drift form, the counter-based random numbers) are stated at each function.
 *
 * Parity pins: tests/test_oracle_*.py check this file against closed forms,
 * invariants and library routines (the <mu> decay, stationary isotropy, the
 * diffusion-limit kappa_par, the Hubble-flow exact solution, the magnetic-moment
 * invariant, the diffusive-shock-acceleration index, the weight ledger,
 * interpolation of affine data, Philox known-answer vectors).  The paper's own
 * figures print no numbers, so agreement with its results is "parity unpinned".
 */
#include "fte_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- units (own definitions) ---------------------------------------------- */
static const double OR_PI = 3.14159265358979323846;
static const double OR_AU_M = 1.495978707e11;
static const double OR_C_MS = 299792458.0;
static const double OR_MC2 = 938.27208816;   /* MeV */

static double c_au(void) { return OR_C_MS / OR_AU_M; }

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --------------------- */
/* A Philox round: two 32x32->64 multiplications by the round multipliers,
   the high halves xored with the other counter words and the round key.  The
   key is advanced by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter (c0, id, tag, 0), key (seed, set_id).  tag 0: transport step c0;
   tag 1: injection draw (c0 = 0); tag 2: injection position attempt c0.
   A 32-bit word x becomes u = ((x >> 8) + 1/2) 2^-24, in (0, 1). */
void or_uniforms(uint32_t seed, uint32_t set_id, uint32_t c0, uint32_t id, uint32_t tag,
                 double u[4])
{
    uint32_t ctr[4] = {c0, id, tag, 0u}, key[2] = {seed, set_id}, x[4];
    or_philox4x32_10(ctr, key, x);
    for (int i = 0; i < 4; ++i) u[i] = ((double)(x[i] >> 8) + 0.5) * (1.0 / 16777216.0);
}

/* Box-Muller: (u0, u1) -> z_mu, z_perp1; (u2, u3) -> z_perp2. */
void or_normals(uint32_t seed, uint32_t set_id, uint32_t n, uint32_t id, double z[3])
{
    double u[4];
    or_uniforms(seed, set_id, n, id, 0u, u);
    double a = sqrt(-2.0 * log(u[0]));
    double b = sqrt(-2.0 * log(u[2]));
    z[0] = a * cos(2.0 * OR_PI * u[1]);
    z[1] = a * sin(2.0 * OR_PI * u[1]);
    z[2] = b * cos(2.0 * OR_PI * u[3]);
}

/* ---- Gauss-Legendre rule (Newton iteration on P_n) ----------------------- */
#define OR_GL_N 1000
static double gl_x[OR_GL_N], gl_w[OR_GL_N];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    const int n = OR_GL_N;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = pk;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {   /* recompute derivative at the converged root */
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = pk;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        double w = 2.0 / ((1.0 - x * x) * dp * dp);
        gl_x[i] = -x; gl_w[i] = w;
        gl_x[n - 1 - i] = x; gl_w[n - 1 - i] = w;
    }
    gl_ready = 1;
}

/* Normalisation of the pitch-angle coefficient from lambda_par (Sec. 2.1: D0 is
   fixed by the rigidity and a prescribed lambda_par).  Reading: the standard
   relation lambda_par = (3v/8) int_{-1}^{1} (1-mu^2)^2 / D_mumu dmu.
     QLT:   D = (nu/2)(1-mu^2)(|mu|^(q-1)+H)  -> nu = 3 v I / (2 lambda),
            I = int_0^1 (1-mu^2)/(mu^(q-1)+H) dmu
     Eq. 5: D = D0 (|mu|/(1+|mu|)+eps)(1-mu^2) -> D0 = 3 v J / (4 lambda),
            J = int_0^1 (1-mu^2)/(mu/(1+mu)+eps) dmu
     iso:   D = D(1-mu^2) -> D = v / (2 lambda)   (returns 1)
   Integrals by Gauss-Legendre after mu = s^3 (removes the cusp at mu = 0). */
double or_norm_integral(int model, double q, double H, double eps)
{
    if (model == OR_DMUMU_ISO) return 1.0;
    gl_init();
    double sum = 0.0;
    for (int i = 0; i < OR_GL_N; ++i) {
        double s = 0.5 * (gl_x[i] + 1.0);
        double mu = s * s * s;
        double jac = 3.0 * s * s * 0.5;
        double den = (model == OR_DMUMU_QLT) ? (pow(mu, q - 1.0) + H) : (mu / (1.0 + mu) + eps);
        sum += gl_w[i] * jac * (1.0 - mu * mu) / den;
    }
    return sum;
}

static double lambda_of_p(const or_params* prm, double p)
{
    if (prm->p_ref > 0.0 && prm->alpha != 0.0) return prm->lambda_par * pow(p / prm->p_ref, prm->alpha);
    return prm->lambda_par;
}

/* D_mumu and dD_mumu/dmu (Eq. 5 and the alternatives of Sec. 2.1).  For the
   quasi-linear form the factor |mu|^(q-2) of the derivative is evaluated with
   |mu| floored at mu_floor (the derivative diverges at mu = 0 for q < 2).
   sgn(0) = 0.  out = {D, dD/dmu, scale (nu, D0 or D)}. */
static void dmumu_eval(const or_params* prm, double I, double mu, double v, double p,
                       double* D, double* dD, double* scale)
{
    double lam = lambda_of_p(prm, p);
    double am = fabs(mu);
    double sg = (mu > 0.0) ? 1.0 : ((mu < 0.0) ? -1.0 : 0.0);
    double omm = 1.0 - mu * mu;
    if (prm->dmumu == OR_DMUMU_QLT) {
        double nu = 3.0 * v * I / (2.0 * lam);
        double g = pow(am, prm->q - 1.0) + prm->H;
        double amf = am > prm->mu_floor ? am : prm->mu_floor;
        double dg = (prm->q - 1.0) * pow(amf, prm->q - 2.0) * sg;
        *D = 0.5 * nu * omm * g;
        *dD = 0.5 * nu * (-2.0 * mu * g + omm * dg);
        *scale = nu;
    } else if (prm->dmumu == OR_DMUMU_PAPER) {
        double D0 = 3.0 * v * I / (4.0 * lam);
        double h = am / (1.0 + am) + prm->eps;
        double dh = sg / ((1.0 + am) * (1.0 + am));
        *D = D0 * h * omm;
        *dD = D0 * (dh * omm - 2.0 * mu * h);
        *scale = D0;
    } else {
        double Dc = v / (2.0 * lam);
        *D = Dc * omm;
        *dD = -2.0 * mu * Dc;
        *scale = Dc;
    }
}

/* d2 D_mumu / d mu2 of dmumu_eval's forms (with the same floor on |mu|); used only
   to record where the pitch-angle map is strongly expanding. */
static double dmumu_d2(const or_params* prm, double I, double mu, double v, double p)
{
    double lam = lambda_of_p(prm, p);
    double am = fabs(mu);
    double sg = (mu > 0.0) ? 1.0 : ((mu < 0.0) ? -1.0 : 0.0);
    double omm = 1.0 - mu * mu;
    if (prm->dmumu == OR_DMUMU_QLT) {
        double nu = 3.0 * v * I / (2.0 * lam);
        double g = pow(am, prm->q - 1.0) + prm->H;
        double amf = am > prm->mu_floor ? am : prm->mu_floor;
        double dg = (prm->q - 1.0) * pow(amf, prm->q - 2.0) * sg;
        double d2g = (prm->q - 1.0) * (prm->q - 2.0) * pow(amf, prm->q - 3.0);
        return 0.5 * nu * (-2.0 * g - 4.0 * mu * dg + omm * d2g);
    } else if (prm->dmumu == OR_DMUMU_PAPER) {
        double D0 = 3.0 * v * I / (4.0 * lam);
        double h = am / (1.0 + am) + prm->eps;
        double dh = sg / ((1.0 + am) * (1.0 + am));
        double d2h = -2.0 / ((1.0 + am) * (1.0 + am) * (1.0 + am));
        return D0 * (d2h * omm - 4.0 * mu * dh - 2.0 * h);
    }
    return -2.0 * v / (2.0 * lam);
}

void or_dmumu(const or_params* prm, double mu, double v, double p, double out[3])
{
    double I = or_norm_integral(prm->dmumu, prm->q, prm->H, prm->eps);
    dmumu_eval(prm, I, mu, v, p, &out[0], &out[1], &out[2]);
}

/* ---- background evaluation (Sec. 2.4) ------------------------------------- */
typedef struct {
    double B[3], V[3], G[9], gB[3], dVdt[3], dB[9];
    double divv;
} fields_t;

typedef struct { int i0; double f; double dfdx; } axis_t;

static double r_centre(const or_background* g, int i)
{
    if (g->radial == 1) return g->r_min * exp((i + 0.5) * log(g->r_max / g->r_min) / g->nr);
    return g->r_min + (i + 0.5) * (g->r_max - g->r_min) / g->nr;
}

/* Bracketing cell centres along one axis and the weight in the physical
   coordinate; outside the outermost centres the value is held constant. */
static void grid_axes(const or_background* g, double r, double th, double ph,
                      axis_t* ar, axis_t* at, axis_t* ap, int* k1)
{
    double xi;
    if (g->radial == 1) xi = log(r / g->r_min) / (log(g->r_max / g->r_min) / g->nr) - 0.5;
    else xi = (r - g->r_min) / ((g->r_max - g->r_min) / g->nr) - 0.5;
    if (xi < 0.0) { ar->i0 = 0; ar->f = 0.0; ar->dfdx = 0.0; }
    else if (xi >= g->nr - 1) { ar->i0 = g->nr - 2; ar->f = 1.0; ar->dfdx = 0.0; }
    else {
        ar->i0 = (int)floor(xi);
        double c0 = r_centre(g, ar->i0), c1 = r_centre(g, ar->i0 + 1);
        ar->f = (r - c0) / (c1 - c0);
        ar->dfdx = 1.0 / (c1 - c0);
    }
    double dth = (g->th_max - g->th_min) / g->nth;
    xi = (th - g->th_min) / dth - 0.5;
    if (xi < 0.0) { at->i0 = 0; at->f = 0.0; at->dfdx = 0.0; }
    else if (xi >= g->nth - 1) { at->i0 = g->nth - 2; at->f = 1.0; at->dfdx = 0.0; }
    else {
        at->i0 = (int)floor(xi);
        double c0 = g->th_min + (at->i0 + 0.5) * dth;
        at->f = (th - c0) / dth;
        at->dfdx = 1.0 / dth;
    }
    double dph = 2.0 * OR_PI / g->nph;
    xi = ph / dph - 0.5;
    int k0 = (int)floor(xi);
    ap->f = xi - k0;
    ap->dfdx = 1.0 / dph;
    k0 = ((k0 % g->nph) + g->nph) % g->nph;
    ap->i0 = k0;
    *k1 = (k0 + 1) % g->nph;
}

/* Bracketing snapshots and the weight of the later one (linear in time); `two`
   says whether dV/dt gains the difference of the pair. */
static void time_bracket(const or_background* g, double t, int* s0_, int* s1_, double* wt_,
                         int* two_)
{
    int s0 = 0, s1 = 0, two = 0;
    double wt = 0.0;
    if (g->n_snap > 1) {
        double tau = (t - g->t_snap0) / g->dt_snap;
        if (g->periodic) {
            double kf = floor(tau);
            wt = tau - kf;
            long long k = (long long)kf;
            s0 = (int)(((k % g->n_snap) + g->n_snap) % g->n_snap);
            s1 = (s0 + 1) % g->n_snap;
            two = 1;
        } else if (tau < 0.0) {
            s0 = s1 = 0;
        } else if (tau >= g->n_snap - 1) {
            s0 = s1 = g->n_snap - 1;
        } else {
            double kf = floor(tau);
            s0 = (int)kf; s1 = s0 + 1; wt = tau - kf; two = 1;
        }
    }
    *s0_ = s0; *s1_ = s1; *wt_ = wt; *two_ = two;
}

/* ---- block AMR (Sec. 2.4) --------------------------------------------------
   Leaves of 2:1-balanced blocks of B^3 cells.  The value at a point is the
   trilinear interpolation (physical weights) of the containing leaf's cell
   lattice extended by one ghost cell.  The paper fetches the neighbour data a
   point near a block edge needs from the neighbouring blocks instead of storing
   ghost cells (Sec. 2.4); here each ghost value is computed on demand from the
   neighbours' interior cells:
     same level   -> the neighbour's cell;
     finer (L+1)  -> interpolation of the level-(L+1) lattice at the ghost centre;
     coarser (L-1)-> interpolation of the level-(L-1) lattice at the ghost centre;
   where a level-m lattice cell covered by finer leaves takes the interpolation of
   the level-(m+1) lattice at its centre (recursively), and one inside a coarser
   leaf takes that leaf's cell.  Outside the domain in r and theta a ghost takes
   the nearest interior cell (constant beyond the outermost centres); phi wraps. */
static int amr_L(const or_background* g) { return g->amr_levels - 1; }

static void amr_ncells(const or_background* g, int m, long n[3])
{
    n[0] = (long)g->nr << m; n[1] = (long)g->nth << m; n[2] = (long)g->nph << m;
}

static double amr_centre(const or_background* g, int m, int a, long i)
{
    long n[3];
    amr_ncells(g, m, n);
    if (a == 0) {
        if (g->radial == 1) return g->r_min * exp((i + 0.5) * log(g->r_max / g->r_min) / n[0]);
        return g->r_min + (i + 0.5) * (g->r_max - g->r_min) / n[0];
    }
    if (a == 1) return g->th_min + (i + 0.5) * (g->th_max - g->th_min) / n[1];
    return (i + 0.5) * (2.0 * OR_PI / n[2]);
}

static void amr_wrap(const or_background* g, int m, long X[3])
{
    long n[3];
    amr_ncells(g, m, n);
    if (X[0] < 0) X[0] = 0;
    if (X[0] > n[0] - 1) X[0] = n[0] - 1;
    if (X[1] < 0) X[1] = 0;
    if (X[1] > n[1] - 1) X[1] = n[1] - 1;
    X[2] = ((X[2] % n[2]) + n[2]) % n[2];
}

static int amr_cover(const or_background* g, int m, const long X[3])
{
    const int L = amr_L(g), B = g->amr_bsize;
    const long nf0 = (long)(g->nr / B) << L, nf1 = (long)(g->nth / B) << L;
    const long f0 = (X[0] << (L - m)) / B, f1 = (X[1] << (L - m)) / B, f2 = (X[2] << (L - m)) / B;
    return g->table[(f2 * nf1 + f1) * nf0 + f0];
}

static const float* amr_rec(const or_background* g, int snap, int leaf, const long X[3])
{
    const int B = g->amr_bsize, P = B + 2;
    const int32_t* lf = g->leaves + 4 * leaf;
    const long li = X[0] - (long)lf[1] * B + 1, lj = X[1] - (long)lf[2] * B + 1;
    const long lk = X[2] - (long)lf[3] * B + 1;
    const size_t idx = ((((size_t)snap * g->n_leaves + leaf) * P + lk) * P + lj) * P + li;
    return g->fields + idx * (size_t)g->rec;
}

static void amr_interp(const or_background* g, int snap, int m, const double c[3], double out[18]);

static void amr_composite(const or_background* g, int snap, int m, const long Xin[3], double out[18])
{
    long X[3] = {Xin[0], Xin[1], Xin[2]};
    amr_wrap(g, m, X);
    const int leaf = amr_cover(g, m, X);
    const int lv = g->leaves[4 * leaf];
    if (lv == m) {
        const float* q = amr_rec(g, snap, leaf, X);
        for (int f = 0; f < 18; ++f) out[f] = q[f];
    } else if (lv > m) {
        const double c[3] = {amr_centre(g, m, 0, X[0]), amr_centre(g, m, 1, X[1]), amr_centre(g, m, 2, X[2])};
        amr_interp(g, snap, m + 1, c, out);
    } else {
        const long Y[3] = {X[0] >> (m - lv), X[1] >> (m - lv), X[2] >> (m - lv)};
        const float* q = amr_rec(g, snap, leaf, Y);
        for (int f = 0; f < 18; ++f) out[f] = q[f];
    }
}

static void amr_interp(const or_background* g, int snap, int m, const double c[3], double out[18])
{
    long n[3];
    amr_ncells(g, m, n);
    long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double x;
        if (a == 0) x = (g->radial == 1) ? log(c[0] / g->r_min) / (log(g->r_max / g->r_min) / n[0]) - 0.5
                                         : (c[0] - g->r_min) / ((g->r_max - g->r_min) / n[0]) - 0.5;
        else if (a == 1) x = (c[1] - g->th_min) / ((g->th_max - g->th_min) / n[1]) - 0.5;
        else x = c[2] / (2.0 * OR_PI / n[2]) - 0.5;
        if (a < 2 && x < 0.0) { i0[a] = 0; f[a] = 0.0; }
        else if (a < 2 && x >= n[a] - 1) { i0[a] = n[a] - 2; f[a] = 1.0; }
        else {
            i0[a] = (long)floor(x);
            if (a == 0) {
                const double c0 = amr_centre(g, m, 0, i0[0]), c1 = amr_centre(g, m, 0, i0[0] + 1);
                f[a] = (c[0] - c0) / (c1 - c0);
            } else {
                f[a] = x - i0[a];
            }
        }
    }
    for (int k = 0; k < 18; ++k) out[k] = 0.0;
    for (int cc = 0; cc < 8; ++cc) {
        const int d0 = cc & 1, d1 = (cc >> 1) & 1, d2 = (cc >> 2) & 1;
        const double w = (d0 ? f[0] : 1.0 - f[0]) * (d1 ? f[1] : 1.0 - f[1]) * (d2 ? f[2] : 1.0 - f[2]);
        const long X[3] = {i0[0] + d0, i0[1] + d1, i0[2] + d2};
        double v[18];
        amr_composite(g, snap, m, X, v);
        for (int k = 0; k < 18; ++k) out[k] += w * v[k];
    }
}

/* value of the ghost cell G (global level-lv index) of a level-lv leaf */
static void amr_ghost(const or_background* g, int snap, int lv, const long Gin[3], double out[18])
{
    long G[3] = {Gin[0], Gin[1], Gin[2]};
    amr_wrap(g, lv, G);
    const int leaf = amr_cover(g, lv, G);
    const int lc = g->leaves[4 * leaf];
    if (lc == lv) {
        const float* q = amr_rec(g, snap, leaf, G);
        for (int f = 0; f < 18; ++f) out[f] = q[f];
        return;
    }
    const double c[3] = {amr_centre(g, lv, 0, G[0]), amr_centre(g, lv, 1, G[1]), amr_centre(g, lv, 2, G[2])};
    amr_interp(g, snap, lc > lv ? lv + 1 : lv - 1, c, out);
}

void or_amr_cell(const or_background* g, int snap, int leaf, int li, int lj, int lk, double out[18])
{
    const int B = g->amr_bsize;
    const int32_t* lf = g->leaves + 4 * leaf;
    const long X[3] = {(long)lf[1] * B + li - 1, (long)lf[2] * B + lj - 1, (long)lf[3] * B + lk - 1};
    if (li >= 1 && li <= B && lj >= 1 && lj <= B && lk >= 1 && lk <= B) {
        const float* q = amr_rec(g, snap, leaf, X);
        for (int k = 0; k < 18; ++k) out[k] = q[k];
        return;
    }
    amr_ghost(g, snap, lf[0], X, out);
}

/* leaf containing the point and its level-lv cell coordinates x[a] = u n - 1/2 */
static int amr_locate(const or_background* g, double r, double th, double ph, long i0[3], double f[3],
                      double dfdx[3], int* lv_out)
{
    const int L = amr_L(g), B = g->amr_bsize;
    const long nf[3] = {(long)(g->nr / B) << L, (long)(g->nth / B) << L, (long)(g->nph / B) << L};
    double u[3];
    u[0] = (g->radial == 1) ? log(r / g->r_min) / log(g->r_max / g->r_min) : (r - g->r_min) / (g->r_max - g->r_min);
    u[1] = (th - g->th_min) / (g->th_max - g->th_min);
    u[2] = ph / (2.0 * OR_PI);
    long fb[3];
    for (int a = 0; a < 3; ++a) {
        fb[a] = (long)floor(u[a] * nf[a]);
        if (fb[a] < 0) fb[a] = (a == 2) ? fb[a] + nf[a] : 0;
        if (fb[a] > nf[a] - 1) fb[a] = (a == 2) ? fb[a] - nf[a] : nf[a] - 1;
    }
    const int leaf = g->table[(fb[2] * nf[1] + fb[1]) * nf[0] + fb[0]];
    const int lv = g->leaves[4 * leaf];
    long n[3];
    amr_ncells(g, lv, n);
    for (int a = 0; a < 3; ++a) {
        double x;
        if (a == 0) x = (g->radial == 1) ? log(r / g->r_min) / (log(g->r_max / g->r_min) / n[0]) - 0.5
                                         : (r - g->r_min) / ((g->r_max - g->r_min) / n[0]) - 0.5;
        else if (a == 1) x = (th - g->th_min) / ((g->th_max - g->th_min) / n[1]) - 0.5;
        else x = ph / (2.0 * OR_PI / n[2]) - 0.5;
        long lo = (long)g->leaves[4 * leaf + 1 + a] * B - 1;       /* first padded index */
        long k = (long)floor(x);
        if (k < lo) k = lo;                                           /* rounding at the leaf edge */
        if (k > lo + B) k = lo + B;
        i0[a] = k;
        if (a == 0) {
            const double c0 = amr_centre(g, lv, 0, k), c1 = amr_centre(g, lv, 0, k + 1);
            f[a] = (r - c0) / (c1 - c0);
            dfdx[a] = 1.0 / (c1 - c0);
        } else {
            f[a] = x - k;
            dfdx[a] = (a == 1) ? n[1] / (g->th_max - g->th_min) : n[2] / (2.0 * OR_PI);
        }
    }
    *lv_out = lv;
    return leaf;
}

static void amr_fields(const or_background* g, double x, double y, double z, double t, fields_t* F)
{
    memset(F, 0, sizeof(*F));
    const double r = sqrt(x * x + y * y + z * z);
    const double rho = sqrt(x * x + y * y);
    const double th = atan2(rho, z);
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * OR_PI;
    long i0[3];
    double f[3], dfdx[3];
    int lv;
    const int leaf = amr_locate(g, r, th, ph, i0, f, dfdx, &lv);
    const int B = g->amr_bsize;
    int s0, s1, two;
    double wt;
    time_bracket(g, t, &s0, &s1, &wt, &two);
    double dBax[3][3] = {{0}};
    for (int s = 0; s < (two ? 2 : 1); ++s) {
        const int snap = (s == 0) ? s0 : s1;
        const double ws = two ? ((s == 0) ? 1.0 - wt : wt) : 1.0;
        for (int c = 0; c < 8; ++c) {
            const int cr = c & 1, ct = (c >> 1) & 1, cp = (c >> 2) & 1;
            const long X[3] = {i0[0] + cr, i0[1] + ct, i0[2] + cp};
            double q[18];
            int interior = 1;
            for (int a = 0; a < 3; ++a) {
                const long loc = X[a] - (long)g->leaves[4 * leaf + 1 + a] * B;
                if (loc < 0 || loc > B - 1) interior = 0;
            }
            if (interior) {
                const float* p = amr_rec(g, snap, leaf, X);
                for (int k = 0; k < 18; ++k) q[k] = p[k];
            } else {
                amr_ghost(g, snap, lv, X, q);
            }
            const double wr = cr ? f[0] : 1.0 - f[0];
            const double wth = ct ? f[1] : 1.0 - f[1];
            const double wp = cp ? f[2] : 1.0 - f[2];
            const double wc = wr * wth * wp;
            for (int m = 0; m < 3; ++m) F->B[m] += ws * wc * q[m];
            for (int m = 0; m < 3; ++m) F->V[m] += ws * wc * q[3 + m];
            for (int m = 0; m < 9; ++m) F->G[m] += ws * wc * q[6 + m];
            for (int m = 0; m < 3; ++m) F->gB[m] += ws * wc * q[15 + m];
            if (two)
                for (int m = 0; m < 3; ++m) F->dVdt[m] += (s == 0 ? -1.0 : 1.0) * wc * q[3 + m] / g->dt_snap;
            const double er = (cr ? 1.0 : -1.0) * dfdx[0] * wth * wp;
            const double et = wr * (ct ? 1.0 : -1.0) * dfdx[1] * wp;
            const double ep = wr * wth * (cp ? 1.0 : -1.0) * dfdx[2];
            for (int m = 0; m < 3; ++m) {
                dBax[m][0] += ws * er * q[m];
                dBax[m][1] += ws * et * q[m];
                dBax[m][2] += ws * ep * q[m];
            }
        }
    }
    const double st = sin(th), ctt = cos(th), sp = sin(ph), cpp = cos(ph);
    const double rh[3] = {st * cpp, st * sp, ctt};
    const double thh[3] = {ctt * cpp, ctt * sp, -st};
    const double phh[3] = {-sp, cpp, 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            F->dB[3 * i + j] = dBax[i][0] * rh[j] + dBax[i][1] * thh[j] / r + dBax[i][2] * phh[j] / (r * st);
    F->divv = F->G[0] + F->G[4] + F->G[8];
}

static void grid_fields(const or_background* g, double x, double y, double z, double t,
                        fields_t* F)
{
    memset(F, 0, sizeof(*F));
    double r = sqrt(x * x + y * y + z * z);
    double rho = sqrt(x * x + y * y);
    double th = atan2(rho, z);
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * OR_PI;
    axis_t ar, at, ap;
    int k1;
    grid_axes(g, r, th, ph, &ar, &at, &ap, &k1);
    int s0, s1, two;
    double wt;
    time_bracket(g, t, &s0, &s1, &wt, &two);
    double dBax[3][3] = {{0}};   /* dB_i / d(r, theta, phi) */
    const size_t rec = (size_t)g->rec;
    for (int s = 0; s < (two ? 2 : 1); ++s) {
        int snap = (s == 0) ? s0 : s1;
        double ws = two ? ((s == 0) ? 1.0 - wt : wt) : 1.0;
        for (int c = 0; c < 8; ++c) {
            int cr = c & 1, ct = (c >> 1) & 1, cp = (c >> 2) & 1;
            int i = ar.i0 + cr, j = at.i0 + ct, k = cp ? k1 : ap.i0;
            double wr = cr ? ar.f : 1.0 - ar.f;
            double wth = ct ? at.f : 1.0 - at.f;
            double wp = cp ? ap.f : 1.0 - ap.f;
            double wc = wr * wth * wp;
            const float* q = g->fields + ((((size_t)snap * g->nph + k) * g->nth + j) * g->nr + i) * rec;
            for (int m = 0; m < 3; ++m) F->B[m] += ws * wc * q[m];
            for (int m = 0; m < 3; ++m) F->V[m] += ws * wc * q[3 + m];
            for (int m = 0; m < 9; ++m) F->G[m] += ws * wc * q[6 + m];
            for (int m = 0; m < 3; ++m) F->gB[m] += ws * wc * q[15 + m];
            if (two)
                for (int m = 0; m < 3; ++m)
                    F->dVdt[m] += (s == 0 ? -1.0 : 1.0) * wc * q[3 + m] / g->dt_snap;
            double er = (cr ? 1.0 : -1.0) * ar.dfdx * wth * wp;
            double et = wr * (ct ? 1.0 : -1.0) * at.dfdx * wp;
            double ep = wr * wth * (cp ? 1.0 : -1.0) * ap.dfdx;
            for (int m = 0; m < 3; ++m) {
                dBax[m][0] += ws * er * q[m];
                dBax[m][1] += ws * et * q[m];
                dBax[m][2] += ws * ep * q[m];
            }
        }
    }
    /* d/dx_j = r_hat_j d/dr + theta_hat_j / r d/dtheta + phi_hat_j / (r sin theta) d/dphi */
    double st = sin(th), ctt = cos(th), sp = sin(ph), cpp = cos(ph);
    double rh[3] = {st * cpp, st * sp, ctt};
    double thh[3] = {ctt * cpp, ctt * sp, -st};
    double phh[3] = {-sp, cpp, 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            F->dB[3 * i + j] = dBax[i][0] * rh[j] + dBax[i][1] * thh[j] / r
                             + dBax[i][2] * phh[j] / (r * st);
    F->divv = F->G[0] + F->G[4] + F->G[8];
}

/* Analytic backgrounds used by the physics pins (all static):
   UNIFORM_B    a0 = B0: B = B0 z_hat, V = 0
   HUBBLE       a0 = alpha, a1 = B0: V = alpha x (grad V = alpha I), B = B0 z_hat
   MONOPOLE     a0 = B0: B = B0 r_hat / r^2, V = 0
   RADIAL_WIND  a0 = V0, a1 = B0: V = V0 r_hat, B = B0 r_hat / r^2
   PLANAR_SHOCK a0 = V1, a1 = V2, a2 = width w, a3 = B0, a4 = field angle from x_hat (x-y plane):
                V = V(x) x_hat, V(x) = V1 + (V2 - V1)(1 + tanh(x/w))/2, B uniform */
static void analytic_fields(const or_background* g, double x, double y, double z, fields_t* F)
{
    memset(F, 0, sizeof(*F));
    const double* a = g->a;
    double r = sqrt(x * x + y * y + z * z);
    double rh[3] = {x / r, y / r, z / r};
    switch (g->kind) {
    case OR_BG_UNIFORM_B:
        F->B[2] = a[0];
        break;
    case OR_BG_HUBBLE:
        F->V[0] = a[0] * x; F->V[1] = a[0] * y; F->V[2] = a[0] * z;
        F->G[0] = F->G[4] = F->G[8] = a[0];
        F->B[2] = a[1];
        break;
    case OR_BG_MONOPOLE:
    case OR_BG_RADIAL_WIND: {
        double B0 = (g->kind == OR_BG_MONOPOLE) ? a[0] : a[1];
        double Bm = B0 / (r * r);
        for (int i = 0; i < 3; ++i) {
            F->B[i] = Bm * rh[i];
            F->gB[i] = -2.0 * Bm / r * rh[i];
            for (int j = 0; j < 3; ++j)
                F->dB[3 * i + j] = Bm / r * ((i == j ? 1.0 : 0.0) - 3.0 * rh[i] * rh[j]);
        }
        if (g->kind == OR_BG_RADIAL_WIND) {
            for (int i = 0; i < 3; ++i) {
                F->V[i] = a[0] * rh[i];
                for (int j = 0; j < 3; ++j)
                    F->G[3 * i + j] = a[0] / r * ((i == j ? 1.0 : 0.0) - rh[i] * rh[j]);
            }
        }
        break;
    }
    case OR_BG_PLANAR_SHOCK: {
        double V1 = a[0], V2 = a[1], w = a[2];
        double th = tanh(x / w);
        F->V[0] = V1 + (V2 - V1) * 0.5 * (1.0 + th);
        F->G[0] = (V2 - V1) * 0.5 * (1.0 - th * th) / w;
        F->B[0] = a[3] * cos(a[4]);
        F->B[1] = a[3] * sin(a[4]);
        break;
    }
    default:
        break;
    }
    F->divv = F->G[0] + F->G[4] + F->G[8];
}

static void eval_fields(const or_background* g, double x, double y, double z, double t,
                        fields_t* F)
{
    if (g->kind == OR_BG_GRID && g->amr_levels > 0) amr_fields(g, x, y, z, t, F);
    else if (g->kind == OR_BG_GRID) grid_fields(g, x, y, z, t, F);
    else analytic_fields(g, x, y, z, F);
}

int or_eval_fields(const or_background* bg, double x, double y, double z, double t,
                   double out[40])
{
    fields_t F;
    eval_fields(bg, x, y, z, t, &F);
    memset(out, 0, 40 * sizeof(double));
    memcpy(out + 0, F.B, 3 * sizeof(double));
    memcpy(out + 3, F.V, 3 * sizeof(double));
    memcpy(out + 6, F.G, 9 * sizeof(double));
    memcpy(out + 15, F.gB, 3 * sizeof(double));
    memcpy(out + 18, F.dVdt, 3 * sizeof(double));
    memcpy(out + 21, F.dB, 9 * sizeof(double));
    out[30] = F.divv;
    return 0;
}

/* ---- kinematics ------------------------------------------------------------ */
/* p in m_p c: gamma = sqrt(1 + p^2), v = c p / gamma, E = m c^2 (gamma - 1)
   evaluated as m c^2 p^2 / (gamma + 1). */
static double speed(double p) { return c_au() * p / sqrt(1.0 + p * p); }
static double kinetic(double p) { return OR_MC2 * p * p / (sqrt(1.0 + p * p) + 1.0); }
static double momentum(double e) { double T = e / OR_MC2; return sqrt(T * (T + 2.0)); }

/* ---- injection (Sec. 2.3, Eq. 7) ------------------------------------------- */
static int near_integer(double xi, double tol)
{
    double d = xi - floor(xi);
    return d < tol || d > 1.0 - tol;
}

int or_inject(const or_background* bg, const or_inject_spec* sp, const uint32_t* ids,
              int64_t n, or_particle* out, double ledger_w[8], uint64_t ledger_n[8])
{
    for (int64_t i = 0; i < n; ++i) {
        or_particle* P = &out[i];
        memset(P, 0, sizeof(*P));
        P->id = ids[i];
        P->n_div = -1;
        P->n_sens = -1;
        P->status = OR_ALIVE;
        double u[4];
        or_uniforms(sp->seed, sp->set_id, 0u, P->id, 1u, u);
        P->mu = (sp->mu_mode == 1) ? sp->mu0 : 2.0 * u[0] - 1.0;
        double E;
        if (sp->energy == 0) {
            E = sp->e0;
        } else if (fabs(sp->gamma - 1.0) < 1e-12) {
            E = sp->e1 * pow(sp->e2 / sp->e1, u[1]);
        } else {
            double g1 = 1.0 - sp->gamma;
            double a = pow(sp->e1, g1), b = pow(sp->e2, g1);
            E = pow(a + u[1] * (b - a), 1.0 / g1);
        }
        P->p = momentum(E);
        double r = sp->r, th = sp->th, ph = sp->ph;
        int ok = 1;
        if (sp->region == 1) {
            ok = 0;
            for (int a = 0; a < sp->max_tries && !ok; ++a) {
                double v[4];
                or_uniforms(sp->seed, sp->set_id, (uint32_t)a, P->id, 2u, v);
                double r13 = sp->r1 * sp->r1 * sp->r1, r23 = sp->r2 * sp->r2 * sp->r2;
                r = cbrt(r13 + v[0] * (r23 - r13));
                double c1 = cos(sp->th1), c2 = cos(sp->th2);
                th = acos(c1 + v[1] * (c2 - c1));
                ph = sp->ph1 + v[2] * (sp->ph2 - sp->ph1);
                /* a band of spiral phase phi_hat = phi + spiral (r - r_b) (the region
                   criterion of Sec. 2.3 for one CIR) */
                if (sp->spiral != 0.0) ph -= sp->spiral * (r - sp->spiral_rb);
                if (!sp->use_divv || bg->kind != OR_BG_GRID) { ok = 1; break; }
                /* acceptance decided on the stored cell value of the containing
                   cell, summed in float like the device does */
                const or_background* g = bg;
                if (g->amr_levels > 0) {
                    const int L = amr_L(g), B = g->amr_bsize;
                    const long nf[3] = {(long)(g->nr / B) << L, (long)(g->nth / B) << L, (long)(g->nph / B) << L};
                    double phw = fmod(ph, 2.0 * OR_PI);
                    if (phw < 0) phw += 2.0 * OR_PI;
                    double uu[3];
                    uu[0] = (g->radial == 1) ? log(r / g->r_min) / log(g->r_max / g->r_min)
                                             : (r - g->r_min) / (g->r_max - g->r_min);
                    uu[1] = (th - g->th_min) / (g->th_max - g->th_min);
                    uu[2] = phw / (2.0 * OR_PI);
                    long fb[3];
                    for (int k = 0; k < 3; ++k) {
                        fb[k] = (long)floor(uu[k] * nf[k]);
                        if (fb[k] < 0) fb[k] = 0;
                        if (fb[k] > nf[k] - 1) fb[k] = nf[k] - 1;
                    }
                    const int leaf = g->table[(fb[2] * nf[1] + fb[1]) * nf[0] + fb[0]];
                    const int lv = g->leaves[4 * leaf];
                    long nl[3];
                    amr_ncells(g, lv, nl);
                    long X[3];
                    for (int k = 0; k < 3; ++k) {
                        const double xc = uu[k] * nl[k];
                        if (near_integer(xc, k == 0 ? 2e-4 : 1e-4)) P->flags |= 1;
                        const long lo = (long)g->leaves[4 * leaf + 1 + k] * B;
                        X[k] = (long)floor(xc);
                        if (X[k] < lo) X[k] = lo;
                        if (X[k] > lo + B - 1) X[k] = lo + B - 1;
                    }
                    const float* q = amr_rec(g, sp->divv_snap, leaf, X);
                    float s01 = q[6] + q[10];
                    float tr = s01 + q[14];
                    if (tr < (float)sp->divv_max) ok = 1;
                    continue;
                }
                double xr = (g->radial == 1) ? log(r / g->r_min) / (log(g->r_max / g->r_min) / g->nr)
                                             : (r - g->r_min) / ((g->r_max - g->r_min) / g->nr);
                double xt = (th - g->th_min) / ((g->th_max - g->th_min) / g->nth);
                double phw = fmod(ph, 2.0 * OR_PI); if (phw < 0) phw += 2.0 * OR_PI;
                double xp = phw / (2.0 * OR_PI / g->nph);
                if (near_integer(xr, 2e-4) || near_integer(xt, 1e-4) || near_integer(xp, 1e-4))
                    P->flags |= 1;
                int ci = (int)floor(xr), cj = (int)floor(xt), ck = (int)floor(xp);
                if (ci < 0) ci = 0;
                if (ci > g->nr - 1) ci = g->nr - 1;
                if (cj < 0) cj = 0;
                if (cj > g->nth - 1) cj = g->nth - 1;
                ck = ((ck % g->nph) + g->nph) % g->nph;
                int sn = sp->divv_snap;
                const float* q = g->fields + ((((size_t)sn * g->nph + ck) * g->nth + cj) * g->nr + ci) * (size_t)g->rec;
                float s01 = q[6] + q[10];
                float tr = s01 + q[14];
                if (tr < (float)sp->divv_max) ok = 1;
            }
        }
        P->x = r * sin(th) * cos(ph);
        P->y = r * sin(th) * sin(ph);
        P->z = r * cos(th);
        P->w = (sp->weight == 1) ? 1.0 / (r * r) : 1.0;
        if (!ok) {
            P->status = OR_INJ_FAIL;
            P->w = 0.0;
            ledger_n[5] += 1;
            continue;
        }
        ledger_w[0] += P->w;
        ledger_n[0] += 1;
    }
    return 0;
}

/* ---- one transport step ----------------------------------------------------- */
typedef struct {
    const or_observer* obs;
    int n_obs;
    const int64_t* off;
    double *S, *S2;
    uint64_t *C, *A;
    double* SC;                  /* optional [bin][32]: S of every bin by particle id mod 32 */
    double lw[8];
    uint64_t ln[8];
} tally_t;

static double wrap_pi(double a)
{
    a = fmod(a + OR_PI, 2.0 * OR_PI);
    if (a < 0) a += 2.0 * OR_PI;
    return a - OR_PI;
}

/* Occupancy tally of the start-of-step state: in observer o, bin (E, t) gains
   w dt (and (w dt)^2, and one count), and the bin's total for the particle's id
   class (id mod 32) gains w dt.  Events within 1e-4 (relative) of an
   energy-bin edge or of the observer's boundary are also counted in A. */
static void tally_state(tally_t* T, double x, double y, double z, double p, double w,
                        double t, double dt, uint32_t id)
{
    if (!T || T->n_obs == 0) return;
    double r = sqrt(x * x + y * y + z * z);
    double th = atan2(sqrt(x * x + y * y), z);
    double ph = atan2(y, x);
    if (ph < 0.0) ph += 2.0 * OR_PI;
    double E = kinetic(p);
    for (int o = 0; o < T->n_obs; ++o) {
        const or_observer* ob = &T->obs[o];
        int inside, amb = 0;
        if (ob->kind == 2) {
            double d = fabs(x - ob->r);
            inside = d <= ob->dr;
            if (fabs(d - ob->dr) < 1e-4 * (ob->dr > 1.0 ? ob->dr : 1.0)) amb = 1;
        } else if (ob->kind == 3) {
            /* ring |r - r_o| <= dr, |theta - th_o| <= dth: longitudinal profile, second
               bin axis = longitude (nt equal bins over [0, 2 pi)), time integrated over
               [t_lo, t_hi) */
            double d = fabs(r - ob->r), dth_ = fabs(th - ob->th);
            inside = d <= ob->dr && dth_ <= ob->dth;
            if (fabs(d - ob->dr) < 1e-4 * ob->r || fabs(dth_ - ob->dth) < 1e-4) amb = 1;
        } else {
            double d = fabs(r - ob->r);
            inside = d <= ob->dr;
            if (fabs(d - ob->dr) < 1e-4 * ob->r) amb = 1;
            if (ob->kind == 1) {
                double dt_ = fabs(th - ob->th), dp_ = fabs(wrap_pi(ph - ob->ph));
                inside = inside && dt_ <= ob->dth && dp_ <= ob->dph;
                if (fabs(dt_ - ob->dth) < 1e-4 || fabs(dp_ - ob->dph) < 1e-4) amb = 1;
            }
        }
        if (!inside && !amb) continue;
        double le = log(E / ob->e_lo) / log(ob->e_hi / ob->e_lo) * ob->ne;
        double ie_f = floor(le);
        double it_f = floor(((t - ob->t_lo) * ob->nt) / (ob->t_hi - ob->t_lo));
        if (ie_f < 0 || ie_f >= ob->ne || it_f < 0 || it_f >= ob->nt) {
            if (inside) T->ln[7] += 1;
            continue;
        }
        double step_le = log(ob->e_hi / ob->e_lo) / ob->ne;
        double fr = le - ie_f;
        if (fr * step_le < 1e-4 || (1.0 - fr) * step_le < 1e-4) amb = 1;
        if (ob->kind == 3) {            /* inside the time window: bin in longitude */
            double lp = ph * ob->nt / (2.0 * OR_PI);
            it_f = floor(lp);
            if (it_f >= ob->nt) it_f = ob->nt - 1;
            double fp = lp - it_f;
            double wbin = 2.0 * OR_PI / ob->nt;
            if (fp * wbin < 1e-4 || (1.0 - fp) * wbin < 1e-4) amb = 1;
        }
        int64_t b = T->off[o] + (int64_t)ie_f * ob->nt + (int64_t)it_f;
        if (inside) {
            double wd = w * dt;
            T->S[b] += wd;
            T->S2[b] += wd * wd;
            T->C[b] += 1;
            if (T->SC) T->SC[b * 32 + (int)(id % 32u)] += wd;
        }
        if (amb) T->A[b] += 1;
    }
}

/* Advance particle P by one step from step index n.  Returns the new status.
   hold (optional): the pitch-angle cosine after the step is *hold instead of the
   Euler-Maruyama draw (the score form of the gradient holds it; everything else
   of the step is unchanged).  ms (optional): receives the mean mu + (mudot +
   dD/dmu) dt and the width sqrt(2 D dt) of the Gaussian pitch-angle increment. */
static int step_core(const or_background* bg, const or_params* prm, double I,
                     or_particle* P, int64_t n, tally_t* T, double* terms,
                     const double* hold, double* ms)
{
    const double dt = prm->dt;
    const double t = prm->t0 + (double)n * dt;
    double x = P->x, y = P->y, z = P->z, mu = P->mu, p = P->p;
    fields_t F;
    eval_fields(bg, x, y, z, t, &F);

    /* derived background quantities (Eqs. 3, 4) */
    double Bm = sqrt(F.B[0] * F.B[0] + F.B[1] * F.B[1] + F.B[2] * F.B[2]);
    double b[3] = {F.B[0] / Bm, F.B[1] / Bm, F.B[2] / Bm};
    double divb = -(b[0] * F.gB[0] + b[1] * F.gB[1] + b[2] * F.gB[2]) / Bm;  /* = 1/L */
    double divv = F.G[0] + F.G[4] + F.G[8];
    double bbgv = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) bbgv += b[i] * b[j] * F.G[3 * i + j];
    double dvdt[3];
    for (int i = 0; i < 3; ++i) {
        dvdt[i] = F.dVdt[i];
        for (int j = 0; j < 3; ++j) dvdt[i] += F.V[j] * F.G[3 * i + j];  /* (V.grad)V */
    }
    double bdvdt = prm->dvdt_term ? (b[0] * dvdt[0] + b[1] * dvdt[1] + b[2] * dvdt[2]) : 0.0;

    double v = speed(p);
    double D, dD, scale;
    dmumu_eval(prm, I, mu, v, p, &D, &dD, &scale);
    double zn[3];
    or_normals(prm->seed, prm->set_id, (uint32_t)n, P->id, zn);

    /* Eq. 3 and the Ito pitch-angle step */
    double omm = 1.0 - mu * mu;
    double mudot = 0.5 * omm * (v * divb + mu * divv - 3.0 * mu * bbgv - (2.0 / v) * bdvdt);
    double m_mean = mu + (mudot + dD) * dt;
    double sig = sqrt(2.0 * D * dt);
    if (ms) { ms[0] = m_mean; ms[1] = sig; }
    double mu_new = hold ? *hold : m_mean + sig * zn[0];
    int ev = 0;
    if (mu_new > 1.0 || mu_new < -1.0) ev = 1;           /* reflection */
    if (mu_new > 1.0) mu_new = 2.0 - mu_new;
    if (mu_new < -1.0) mu_new = -2.0 - mu_new;
    if (mu_new > 1.0) mu_new = 1.0;
    if (mu_new < -1.0) mu_new = -1.0;
    if (mu * mu_new <= 0.0) ev = 1;                      /* mu changes sign */
    if (prm->shock_divv > 0.0 && fabs(divv) > prm->shock_divv) ev = 1;
    if (P->n_sens < 0) {
        /* derivative of the pitch-angle update with respect to mu, fields held fixed:
           1 + dt (d mudot/dmu + d2D/dmu2) + z sqrt(2 dt) d sqrt(D)/dmu (bookkeeping) */
        double d2D = dmumu_d2(prm, I, mu, v, p);
        double dq = divv - 3.0 * bbgv;
        double dmudot = 0.5 * (-2.0 * mu * (v * divb + mu * divv - 3.0 * mu * bbgv - (2.0 / v) * bdvdt)
                               + omm * dq);
        double jac = 1.0 + (dmudot + d2D) * dt + (D > 0.0 ? zn[0] * sqrt(2.0 * dt) * dD / (2.0 * sqrt(D)) : 0.0);
        double L = P->amp_log + log(fabs(jac) > 1e-300 ? fabs(jac) : 1e-300);
        P->amp_log = L > 0.0 ? L : 0.0;
        if (P->amp_log > log(100.0)) P->n_sens = (int32_t)n;
    }

    /* Eq. 2 with cross-field diffusion kappa_perp = (v lambda_perp / 3)(I - bb) */
    double kap = v * prm->lambda_perp / 3.0;
    double u_perp[3] = {0, 0, 0}, noise[3] = {0, 0, 0};
    if (kap > 0.0) {
        if (prm->kappa_drift) {
            /* div(kappa_perp) = -kappa [(div b) b + (b.grad) b], with
               (b.grad) b = [(b.grad)B - b (b.(b.grad)B)] / |B| */
            double bgB[3];
            for (int i = 0; i < 3; ++i)
                bgB[i] = F.dB[3 * i + 0] * b[0] + F.dB[3 * i + 1] * b[1] + F.dB[3 * i + 2] * b[2];
            double par = b[0] * bgB[0] + b[1] * bgB[1] + b[2] * bgB[2];
            for (int i = 0; i < 3; ++i) {
                double curv = (bgB[i] - b[i] * par) / Bm;
                u_perp[i] = -kap * (divb * b[i] + curv);
            }
        }
        double e1[3], e2[3];
        double cz = sqrt(b[1] * b[1] + b[0] * b[0]);      /* |b x z_hat| */
        if (fabs(cz - 0.1) < 1e-5) ev = 1;
        if (cz >= 0.1) { e1[0] = b[1] / cz; e1[1] = -b[0] / cz; e1[2] = 0.0; }
        else {
            double cx = sqrt(b[2] * b[2] + b[1] * b[1]);  /* |b x x_hat| */
            e1[0] = 0.0; e1[1] = b[2] / cx; e1[2] = -b[1] / cx;
        }
        e2[0] = b[1] * e1[2] - b[2] * e1[1];
        e2[1] = b[2] * e1[0] - b[0] * e1[2];
        e2[2] = b[0] * e1[1] - b[1] * e1[0];
        double amp = sqrt(2.0 * kap * dt);
        for (int i = 0; i < 3; ++i) noise[i] = amp * (zn[1] * e1[i] + zn[2] * e2[i]);
    }
    double xn[3];
    double xo[3] = {x, y, z};
    for (int i = 0; i < 3; ++i)
        xn[i] = xo[i] + (F.V[i] + mu * v * b[i] + u_perp[i]) * dt + noise[i];

    /* Eq. 4 */
    double pdot_p = 0.5 * (1.0 - 3.0 * mu * mu) * bbgv - 0.5 * omm * divv - (mu / v) * bdvdt;
    double p_new = prm->p_update == 0 ? p * exp(pdot_p * dt) : p * (1.0 + pdot_p * dt);

    if (terms) {
        double* o = terms;
        o[0] = v; o[1] = sqrt(1.0 + p * p); o[2] = D; o[3] = dD; o[4] = mudot; o[5] = pdot_p;
        o[6] = divb; o[7] = divv; o[8] = bbgv; o[9] = bdvdt;
        o[10] = b[0]; o[11] = b[1]; o[12] = b[2];
        o[13] = F.V[0]; o[14] = F.V[1]; o[15] = F.V[2];
        o[16] = zn[0]; o[17] = zn[1]; o[18] = zn[2];
        o[19] = kap; o[20] = u_perp[0]; o[21] = u_perp[1]; o[22] = u_perp[2];
        o[23] = xn[0]; o[24] = xn[1]; o[25] = xn[2];
        o[26] = mu_new; o[27] = p_new; o[28] = kinetic(p); o[29] = scale;
        o[30] = t; o[31] = ev;
        return P->status;
    }

    /* tally the start-of-step state */
    tally_state(T, x, y, z, p, P->w, t, dt, P->id);

    P->x = xn[0]; P->y = xn[1]; P->z = xn[2];
    P->mu = mu_new; P->p = p_new;

    int st = OR_ALIVE;
    if (!isfinite(xn[0]) || !isfinite(xn[1]) || !isfinite(xn[2]) || !isfinite(mu_new) ||
        !isfinite(p_new)) {
        st = OR_NAN; ev = 1;
    } else if (bg->domain == OR_DOM_SPHERE) {
        double rmin = bg->dom[0], rmax = bg->dom[1], tmin = bg->dom[2], tmax = bg->dom[3];
        double rn = sqrt(xn[0] * xn[0] + xn[1] * xn[1] + xn[2] * xn[2]);
        double thn = atan2(sqrt(xn[0] * xn[0] + xn[1] * xn[1]), xn[2]);
        if (fabs(rn - rmin) < 1e-5 * rmin || fabs(rn - rmax) < 1e-5 * rmax ||
            fabs(thn - tmin) < 1e-5 || fabs(thn - tmax) < 1e-5) ev = 1;
        if (rn < rmin) st = OR_ABS_INNER;
        else if (rn > rmax) st = OR_ABS_OUTER;
        else if (thn < tmin || thn > tmax) st = OR_ABS_THETA;
    } else if (bg->domain == OR_DOM_SLAB_X) {
        double a = bg->dom[0], c = bg->dom[1];
        if (fabs(xn[0] - a) < 1e-5 * (fabs(a) > 1 ? fabs(a) : 1) ||
            fabs(xn[0] - c) < 1e-5 * (fabs(c) > 1 ? fabs(c) : 1)) ev = 1;
        if (xn[0] < a) st = OR_ABS_INNER;
        else if (xn[0] > c) st = OR_ABS_OUTER;
    }
    if (ev && P->n_div < 0) P->n_div = n;
    P->status = st;
    if (st != OR_ALIVE && T) {
        T->lw[st] += P->w;
        T->ln[st] += 1;
    }
    return st;
}

static int step_one(const or_background* bg, const or_params* prm, double I,
                    or_particle* P, int64_t n, tally_t* T, double* terms)
{
    return step_core(bg, prm, I, P, n, T, terms, NULL, NULL);
}

int or_step_terms(const or_background* bg, const or_params* prm, const or_particle* p,
                  int64_t n, double out[32])
{
    or_particle q = *p;
    double I = or_norm_integral(prm->dmumu, prm->q, prm->H, prm->eps);
    step_one(bg, prm, I, &q, n, NULL, out);
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int or_advance(const or_background* bg, const or_params* prm, const or_observer* obs,
               int n_obs, or_particle* P, int64_t n, int64_t n_start, int64_t n_end,
               double* S, double* S2, uint64_t* C, uint64_t* A, double* SC, double ledger_w[8],
               uint64_t ledger_n[8], int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    int64_t off[64 + 1];
    if (n_obs > 64) return -1;
    off[0] = 0;
    for (int o = 0; o < n_obs; ++o) off[o + 1] = off[o] + (int64_t)obs[o].ne * obs[o].nt;
    const int64_t nb = off[n_obs];
    const double I = or_norm_integral(prm->dmumu, prm->q, prm->H, prm->eps);

    double* tS = (double*)calloc((size_t)n_threads * (nb > 0 ? nb : 1), sizeof(double));
    double* tS2 = (double*)calloc((size_t)n_threads * (nb > 0 ? nb : 1), sizeof(double));
    uint64_t* tC = (uint64_t*)calloc((size_t)n_threads * (nb > 0 ? nb : 1), sizeof(uint64_t));
    uint64_t* tA = (uint64_t*)calloc((size_t)n_threads * (nb > 0 ? nb : 1), sizeof(uint64_t));
    double* tSC = (double*)calloc((size_t)n_threads * (nb > 0 ? nb : 1) * 32, sizeof(double));
    tally_t* tt = (tally_t*)calloc((size_t)n_threads, sizeof(tally_t));
    if (!tS || !tS2 || !tC || !tA || !tSC || !tt) return -2;
    for (int k = 0; k < n_threads; ++k) {
        tt[k].obs = obs; tt[k].n_obs = n_obs; tt[k].off = off;
        tt[k].S = tS + (size_t)k * nb; tt[k].S2 = tS2 + (size_t)k * nb;
        tt[k].C = tC + (size_t)k * nb; tt[k].A = tA + (size_t)k * nb;
        tt[k].SC = tSC + (size_t)k * (nb > 0 ? nb : 1) * 32;
    }
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        tally_t* T = &tt[tid];
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < n; ++i) {
            or_particle* q = &P[i];
            if (q->status != OR_ALIVE) continue;
            for (int64_t s = n_start; s < n_end; ++s) {
                T->ln[6] += 1;
                if (step_one(bg, prm, I, q, s, T, NULL) != OR_ALIVE) break;
            }
        }
    }
    for (int k = 0; k < n_threads; ++k) {
        for (int64_t b = 0; b < nb; ++b) {
            S[b] += tt[k].S[b]; S2[b] += tt[k].S2[b]; C[b] += tt[k].C[b]; A[b] += tt[k].A[b];
        }
        for (int m = 0; m < 8; ++m) { ledger_w[m] += tt[k].lw[m]; ledger_n[m] += tt[k].ln[m]; }
        if (SC)
            for (int64_t b = 0; b < nb * 32; ++b) SC[b] += tt[k].SC[b];
    }
    free(tS); free(tS2); free(tC); free(tA); free(tSC); free(tt);
    return 0;
}

/* Smooth observable whose parameter gradients fit transport parameters to
   intensities: every alive step of particle i adds w dt K(start-of-step state)
   to J[i], K = exp(-(r - r_o)^2 / (2 s_r^2)) exp(-ln(E / E_c)^2 / (2 s_E^2))
   exp(-(t - t_c)^2 / (2 s_t^2)); the particles are advanced as by or_advance
   (no tally, no ledger). */
static double smooth_kernel(const or_smooth_obs* K, double x, double y, double z, double p, double t)
{
    const double r = sqrt(x * x + y * y + z * z);
    const double le = log(kinetic(p) / K->e_c);
    const double a = (r - K->r_o) / K->sigma_r, b = le / K->sigma_lnE, c = (t - K->t_c) / K->sigma_t;
    return exp(-0.5 * a * a) * exp(-0.5 * b * b) * exp(-0.5 * c * c);
}

int or_observe(const or_background* bg, const or_params* prm, const or_smooth_obs* K, or_particle* P,
               int64_t n, int64_t n_start, int64_t n_end, double* J, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    const double I = or_norm_integral(prm->dmumu, prm->q, prm->H, prm->eps);
#ifdef _OPENMP
#pragma omp parallel for num_threads(n_threads) schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        or_particle* q = &P[i];
        double acc = 0.0;
        for (int64_t s = n_start; s < n_end && q->status == OR_ALIVE; ++s) {
            const double t = prm->t0 + (double)s * prm->dt;
            acc += q->w * prm->dt * smooth_kernel(K, q->x, q->y, q->z, q->p, t);
            if (step_one(bg, prm, I, q, s, NULL, NULL) != OR_ALIVE) break;
        }
        J[i] = acc;
    }
    return 0;
}

/* Density of the pitch-angle cosine after one step (Sec. 2.1: the Ito step adds a
   Gaussian increment of mean (mudot + dD/dmu) dt and variance 2 D dt; a draw beyond
   mu = +-1 is reflected back into [-1, 1]): the unreflected value y ~ N(m, s^2)
   lands at mu1 from y = mu1, 2 - mu1 or -2 - mu1.  Returns the log of the sum of
   the three Gaussian densities without the constant -ln(2 pi)/2. */
double or_mu_logpdf(double mu1, double m, double s)
{
    const double y[3] = {mu1, 2.0 - mu1, -2.0 - mu1};
    double e[3], emax = -INFINITY;
    for (int j = 0; j < 3; ++j) {
        const double z = (y[j] - m) / s;
        e[j] = -0.5 * z * z;
        if (e[j] > emax) emax = e[j];
    }
    double sum = 0.0;
    for (int j = 0; j < 3; ++j) sum += exp(e[j] - emax);
    return emax + log(sum) - log(s);
}

/* Gradient of the smooth observable (or_observe) with respect to the pitch-angle
   parameters, in the score (likelihood-ratio) form for the steps where the jump of
   Eq. 5's dD/dmu at mu = 0, or the singular quasi-linear drift, makes the
   Euler-Maruyama map discontinuous, and pathwise elsewhere.
   A step n is "gated" when the Gaussian increment's mean m lies within `window`
   widths s of a value that lands at mu = 0 (m = 0, or m = +-2 through the
   reflection): min(|m|, ||m| - 2|) < window s.  For a perturbed parameter theta', the path
   is recomputed with the noise of every other step held and, at every gated step,
   with the base path's mu_{n+1} held, while the observable's terms after step n are
   weighted by p(mu_{n+1} | state_n(theta'), theta') / p(mu_{n+1} | state_n, theta).
   Its expectation equals E[J(theta')] for every theta', so its derivative at theta
   (central differences, step rel * theta_j) estimates dE[J]/dtheta_j without bias.
   window = 0: no gated steps (the derivative of the realised path).
   which: bit j requests parameter j = lambda_par, q, H, eps; G[i * 4 + j].
   flags[i]: bit 0 a gate decision within 1e-4 (relative) of |m| = window s;
             bit 1 a step starting within 1e-5 of mu = 0 (where the map jumps);
             bit 2 a perturbed path ended at another step than the base path.
   P is advanced in place along the base path, as by or_observe. */
int or_observe_lr(const or_background* bg, const or_params* prm, const or_smooth_obs* K, double window,
                  or_particle* P, int64_t n, int64_t n_start, int64_t n_end, int which, double rel,
                  double* J, double* G, int32_t* flags, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_end < n_start) return 1;
    const int64_t ns = n_end - n_start;
    const double I = or_norm_integral(prm->dmumu, prm->q, prm->H, prm->eps);
    int rc = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
        signed char* gate = (signed char*)malloc((size_t)(ns > 0 ? ns : 1));
        double* hold = (double*)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1));
        double* lp = (double*)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1));
        if (!gate || !hold || !lp) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = 2;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < n; ++i) {
            if (!gate || !hold || !lp) continue;
            const or_particle p0 = P[i];
            or_particle q = p0;
            int32_t fl = 0;
            double acc = 0.0, ms[2];
            int64_t s_end = n_end;
            for (int64_t s = n_start; s < n_end && q.status == OR_ALIVE; ++s) {
                const double t = prm->t0 + (double)s * prm->dt;
                acc += q.w * prm->dt * smooth_kernel(K, q.x, q.y, q.z, q.p, t);
                if (fabs(q.mu) < 1e-5) fl |= 2;
                const int st = step_core(bg, prm, I, &q, s, NULL, NULL, NULL, ms);
                /* distance of the mean from the nearest unreflected value that lands at mu = 0 */
                const double am = fabs(ms[0]), d0 = fmin(am, fabs(am - 2.0));
                const double lim = window * ms[1];
                const int g = d0 < lim;
                if (window > 0.0 && fabs(d0 - lim) <= 1e-4 * lim) fl |= 1;
                gate[s - n_start] = (signed char)g;
                hold[s - n_start] = q.mu;
                lp[s - n_start] = g ? or_mu_logpdf(q.mu, ms[0], ms[1]) : 0.0;
                if (st != OR_ALIVE) { s_end = s + 1; break; }
            }
            J[i] = acc;
            for (int j = 0; j < 4; ++j) {
                if (!(which & (1 << j))) { G[i * 4 + j] = 0.0; continue; }
                double psi[2];
                for (int sg = 0; sg < 2; ++sg) {
                    or_params pp = *prm;
                    double* th = j == 0 ? &pp.lambda_par : j == 1 ? &pp.q : j == 2 ? &pp.H : &pp.eps;
                    const double d = rel * *th;
                    *th += sg ? -d : d;
                    const double Ip = or_norm_integral(pp.dmumu, pp.q, pp.H, pp.eps);
                    or_particle r = p0;
                    double sum = 0.0, logw = 0.0;
                    int64_t e = n_end;
                    for (int64_t s = n_start; s < s_end && r.status == OR_ALIVE; ++s) {
                        const double t = pp.t0 + (double)s * pp.dt;
                        sum += r.w * pp.dt * smooth_kernel(K, r.x, r.y, r.z, r.p, t) * exp(logw);
                        const int g = gate[s - n_start];
                        const int st = step_core(bg, &pp, Ip, &r, s, NULL, NULL, g ? &hold[s - n_start] : NULL, ms);
                        if (g) logw += or_mu_logpdf(hold[s - n_start], ms[0], ms[1]) - lp[s - n_start];
                        if (st != OR_ALIVE) { e = s + 1; break; }
                    }
                    /* the perturbed path must end where the base path ends */
                    if ((r.status != OR_ALIVE) != (q.status != OR_ALIVE) || e != s_end) fl |= 4;
                    psi[sg] = sum;
                }
                const double th0 = j == 0 ? prm->lambda_par : j == 1 ? prm->q : j == 2 ? prm->H : prm->eps;
                G[i * 4 + j] = (psi[0] - psi[1]) / (2.0 * rel * th0);
            }
            flags[i] = fl;
            P[i] = q;
        }
        free(gate);
        free(hold);
        free(lp);
    }
    return rc;
}

/* Intensity from the occupancy sum (Eq. 7 with j = p^2 f): S / dt_bin is the
   mean weight inside the observer volume during the bin; per unit volume and
   energy, times v / (4 pi), gives the differential intensity
   j = S v(E_c) / (4 pi V_obs dt_bin dE), E_c the geometric bin centre. */
void or_intensity(const or_observer* ob, const double* S, double* J)
{
    double vol;
    if (ob->kind == 0) {
        double a = ob->r - ob->dr, b = ob->r + ob->dr;
        vol = 4.0 * OR_PI / 3.0 * (b * b * b - a * a * a);
    } else if (ob->kind == 1) {
        double a = ob->r - ob->dr, b = ob->r + ob->dr;
        vol = (b * b * b - a * a * a) / 3.0 * (cos(ob->th - ob->dth) - cos(ob->th + ob->dth))
              * 2.0 * ob->dph;
    } else if (ob->kind == 3) {
        double a = ob->r - ob->dr, b = ob->r + ob->dr;
        vol = (b * b * b - a * a * a) / 3.0 * (cos(ob->th - ob->dth) - cos(ob->th + ob->dth))
              * 2.0 * OR_PI / ob->nt;
    } else {
        vol = 2.0 * ob->dr;
    }
    /* ring: every longitude bin integrates the whole time window */
    double dtb = ob->kind == 3 ? ob->t_hi - ob->t_lo : (ob->t_hi - ob->t_lo) / ob->nt;
    for (int e = 0; e < ob->ne; ++e) {
        double e0 = ob->e_lo * pow(ob->e_hi / ob->e_lo, (double)e / ob->ne);
        double e1 = ob->e_lo * pow(ob->e_hi / ob->e_lo, (double)(e + 1) / ob->ne);
        double ec = sqrt(e0 * e1);
        double v = speed(momentum(ec));
        for (int k = 0; k < ob->nt; ++k)
            J[e * ob->nt + k] = S[e * ob->nt + k] * v / (4.0 * OR_PI * vol * dtb * (e1 - e0));
    }
}
