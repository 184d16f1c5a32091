/*
 * FP64 CPU oracle of the focused-transport particle pusher.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, direct restatement of the
 * method in double precision, used by the tests, by the self-check in
 * __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.  The product
 * path (the CUDA library) never calls, links or includes anything here, and
 * nothing here includes the library's headers.
 *
 * Method (Husidic et al. 2024, Sec. 2.1): the focused transport equation (Eq. 1)
 * with the coefficients of Eqs. 2-4 is integrated as Ito SDEs forward in time
 * for independent pseudo-particles through a gridded, time-interpolated
 * background (Sec. 2.4), with pitch-angle diffusion D_mumu (Eq. 5 or the
 * quasi-linear form), optional cross-field diffusion (lambda_perp, Sec. 2.1),
 * injection per Eq. 7 and weighted occupancy tallies.
 *
 * Units: au, s, nT, MeV; momentum p in units of m_p c.
 */
#ifndef FTE_ORACLE_H
#define FTE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BG_GRID = 0, OR_BG_UNIFORM_B = 1, OR_BG_HUBBLE = 2, OR_BG_MONOPOLE = 3,
       OR_BG_RADIAL_WIND = 4, OR_BG_PLANAR_SHOCK = 5 };
enum { OR_DOM_SPHERE = 0, OR_DOM_SLAB_X = 1, OR_DOM_NONE = 2 };
enum { OR_DMUMU_QLT = 0, OR_DMUMU_PAPER = 1, OR_DMUMU_ISO = 2 };
enum { OR_ALIVE = 0, OR_ABS_INNER = 1, OR_ABS_OUTER = 2, OR_ABS_THETA = 3, OR_NAN = 4,
       OR_INJ_FAIL = 5 };
/* ledger slots: 0 injected, 1..4 by status, 5 failed injections (count),
   6 alive particle-steps (count), 7 tally events outside the E/t range (count) */

typedef struct {
    int32_t kind, domain;
    double a[8];                 /* analytic parameters, per kind (see fte_oracle.c) */
    double dom[4];               /* SPHERE: r_min r_max th_min th_max; SLAB_X: x_min x_max */
    int32_t nr, nth, nph, radial;     /* GRID: cells; radial 0 linear, 1 log */
    int32_t n_snap, periodic, rec, pad;
    double r_min, r_max, th_min, th_max, t_snap0, dt_snap;
    const float* fields;         /* uniform: [n_snap][nph][nth][nr][rec];
                                    AMR: [n_snap][n_leaves][B+2][B+2][B+2][rec], ghosts unused */
    /* block AMR (amr_levels > 0): nr, nth, nph are the base-level cell counts */
    int32_t amr_levels, amr_bsize, n_leaves, pad2;
    const int32_t* leaves;       /* [n_leaves][4]: level, bi, bj, bk (block index at its level) */
    const int32_t* table;        /* [nph/B 2^L][nth/B 2^L][nr/B 2^L]: leaf covering each finest block */
} or_background;

typedef struct {
    int32_t dmumu, p_update, kappa_drift, dvdt_term;  /* p_update 0 exponential, 1 Euler */
    double lambda_par, p_ref, alpha, q, H, eps, mu_floor, lambda_perp;
    double dt, t0;
    uint32_t seed, set_id;
    double shock_divv;           /* |div V| above which a step is a divergence event (0: off) */
} or_params;

typedef struct {
    int32_t region, energy, weight, mu_mode; /* region 0 point 1 box; energy 0 mono 1 power law;
                                                weight 0 unit 1 r^-2; mu 0 isotropic 1 fixed */
    double r, th, ph;
    double r1, r2, th1, th2, ph1, ph2;
    int32_t use_divv, divv_snap, max_tries, pad;
    double divv_max;
    double e0, e1, e2, gamma, mu0;
    uint32_t seed, set_id;
    double spiral, spiral_rb;    /* box: ph1..ph2 bound the spiral phase phi + spiral (r - spiral_rb) */
} or_inject_spec;

typedef struct {
    int32_t kind, ne, nt, pad;   /* kind 0 shell, 1 box, 2 slab |x - r| <= dr, 3 ring
                                    (|r - r_o| <= dr, |theta - th| <= dth; nt longitude bins,
                                    time integrated over [t_lo, t_hi)) */
    double r, dr, th, dth, ph, dph, e_lo, e_hi, t_lo, t_hi;
} or_observer;

typedef struct {
    double x, y, z, mu, p, w;
    int64_t n_div;               /* first step with a divergence event, -1 if none yet */
    uint32_t id;
    int32_t status;
    int32_t flags;               /* bit 0: injection decision within rounding of a threshold/edge */
    int32_t n_sens;              /* first step at which a difference in mu made at an earlier
                                    step has been amplified more than 100-fold by the pitch-angle
                                    map (fields held fixed), -1 if none: from there FP32 and
                                    FP64 rounding grow apart although both compute the same map
                                    (bookkeeping only) */
    double amp_log;              /* max over earlier steps k of sum_{j>=k} ln|d mu_{j+1}/d mu_j|,
                                    i.e. L_n = max(0, L_{n-1} + ln|d mu'/d mu|) */
} or_particle;

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_uniforms(uint32_t seed, uint32_t set_id, uint32_t c0, uint32_t id, uint32_t tag,
                 double u[4]);
void or_normals(uint32_t seed, uint32_t set_id, uint32_t n, uint32_t id, double z[3]);
double or_norm_integral(int model, double q, double H, double eps);
void or_dmumu(const or_params* prm, double mu, double v, double p, double out[3]);
int or_eval_fields(const or_background* bg, double x, double y, double z, double t,
                   double out[40]);
int or_inject(const or_background* bg, const or_inject_spec* spec, const uint32_t* ids,
              int64_t n, or_particle* out, double ledger_w[8], uint64_t ledger_n[8]);
/* SC (optional, [bin][32]): the tally S of every bin by particle id mod 32 */
int or_advance(const or_background* bg, const or_params* prm, const or_observer* obs,
               int n_obs, or_particle* P, int64_t n, int64_t n_start, int64_t n_end,
               double* S, double* S2, uint64_t* C, uint64_t* A, double* SC, double ledger_w[8],
               uint64_t ledger_n[8], int n_threads);
int or_step_terms(const or_background* bg, const or_params* prm, const or_particle* p,
                  int64_t n, double out[32]);
void or_intensity(const or_observer* obs, const double* S, double* J);
/* smooth observable for parameter gradients: J[i] = sum over alive steps of
   w dt exp(-(r-r_o)^2/(2 sigma_r^2)) exp(-ln(E/e_c)^2/(2 sigma_lnE^2)) exp(-(t-t_c)^2/(2 sigma_t^2)) */
typedef struct {
    double r_o, sigma_r, e_c, sigma_lnE, t_c, sigma_t;
} or_smooth_obs;
int or_observe(const or_background* bg, const or_params* prm, const or_smooth_obs* K, or_particle* P,
               int64_t n, int64_t n_start, int64_t n_end, double* J, int n_threads);
/* log density (without -ln(2 pi)/2) of the pitch-angle cosine mu1 after a step whose
   Gaussian increment has mean m and width s, reflected at mu = +-1 (images 2 - mu1,
   -2 - mu1) */
double or_mu_logpdf(double mu1, double m, double s);
/* hybrid pathwise / score gradient of or_observe's J with respect to the pitch-angle
   parameters (bit j of `which`: lambda_par, q, H, eps; G[i*4+j]); steps whose Gaussian
   increment has its mean within `window` widths of mu = 0 enter by the likelihood
   ratio of the held mu_{n+1}; see fte_oracle.c for flags */
int or_observe_lr(const or_background* bg, const or_params* prm, const or_smooth_obs* K, double window,
                  or_particle* P, int64_t n, int64_t n_start, int64_t n_end, int which, double rel,
                  double* J, double* G, int32_t* flags, int n_threads);
/* value of padded cell (li, lj, lk) of an AMR leaf (interior cells: the stored record;
   ghost cells: the neighbour value the method defines), fields 0..17 */
void or_amr_cell(const or_background* bg, int snap, int leaf, int li, int lj, int lk, double out[18]);
int or_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
