// Block-AMR set-up (Sec. 2.4, Fig. 4): the finest-level lookup table, the
// tiling / 2:1 nesting check, and the ghost layer of every leaf.
//
// The paper reads the neighbouring blocks' data whenever a particle sits near a
// block edge (same level, parent level or child level).  Here that case
// analysis runs once per snapshot, on the device, and its result is stored as a
// one-cell ghost layer around each leaf, so that the per-step gather reads one
// contiguous padded block whatever the neighbours are.
#include "fte_kernels.cuh"

namespace fte {

struct AmrK {
    const float* f;          // FP32 records [snap][leaf][P][P][P][FTE_REC]
    float* fw;               // same array, written (ghost layer)
    long long snap_recs;
    int n_leaves, B, P, L, n_snap;
    int nr, nth, nph;        // base-level cells
    int nf0, nf1, nf2;
    const int4* leaves;
    const int* table;
    int radial;
    double r_min, r_max, th_min, th_max;
};

__device__ __forceinline__ long long amr_n(const AmrK& a, int m, int axis)
{
    const long long n = axis == 0 ? a.nr : (axis == 1 ? a.nth : a.nph);
    return n << m;
}

// cell-centre coordinate of global level-m index i along an axis
__device__ double amr_centre(const AmrK& a, int m, int axis, long long i)
{
    const double n = (double)amr_n(a, m, axis);
    if (axis == 0) {
        if (a.radial) return a.r_min * exp((i + 0.5) * log(a.r_max / a.r_min) / n);
        return a.r_min + (i + 0.5) * (a.r_max - a.r_min) / n;
    }
    if (axis == 1) return a.th_min + (i + 0.5) * (a.th_max - a.th_min) / n;
    return (i + 0.5) * (2.0 * 3.141592653589793 / n);
}

// clamp into the domain in r and theta, wrap phi
__device__ __forceinline__ void amr_fold(const AmrK& a, int m, long long X[3])
{
    const long long n0 = amr_n(a, m, 0), n1 = amr_n(a, m, 1), n2 = amr_n(a, m, 2);
    X[0] = X[0] < 0 ? 0 : (X[0] > n0 - 1 ? n0 - 1 : X[0]);
    X[1] = X[1] < 0 ? 0 : (X[1] > n1 - 1 ? n1 - 1 : X[1]);
    X[2] = ((X[2] % n2) + n2) % n2;
}

__device__ __forceinline__ int amr_leaf_of(const AmrK& a, int m, const long long X[3])
{
    const long long f0 = (X[0] << (a.L - m)) / a.B, f1 = (X[1] << (a.L - m)) / a.B;
    const long long f2 = (X[2] << (a.L - m)) / a.B;
    return a.table[(f2 * a.nf1 + f1) * a.nf0 + f0];
}

// interior record of `leaf` holding its own-level cell X
__device__ __forceinline__ const float* amr_cell(const AmrK& a, int snap, int leaf, const long long X[3])
{
    const int4 lf = a.leaves[leaf];
    const long long li = X[0] - (long long)lf.y * a.B + 1, lj = X[1] - (long long)lf.z * a.B + 1;
    const long long lk = X[2] - (long long)lf.w * a.B + 1;
    const long long r = (long long)snap * a.snap_recs + (((long long)leaf * a.P + lk) * a.P + lj) * a.P + li;
    return a.f + r * FTE_REC;
}

template <int D>
__device__ __noinline__ void amr_lattice_at(const AmrK& a, int snap, int m, const double c[3], double out[FTE_NFIELD]);

// value of level-m lattice cell X: the cell itself if a level-m leaf holds it,
// the finer lattice interpolated at its centre if finer leaves cover it, the
// containing cell of a coarser leaf otherwise
template <int D>
__device__ void amr_lattice_cell(const AmrK& a, int snap, int m, const long long Xin[3], double out[FTE_NFIELD])
{
    long long X[3] = {Xin[0], Xin[1], Xin[2]};
    amr_fold(a, m, X);
    const int leaf = amr_leaf_of(a, m, X);
    const int lv = a.leaves[leaf].x;
    if constexpr (D > 0) {
        if (lv > m) {
            const double c[3] = {amr_centre(a, m, 0, X[0]), amr_centre(a, m, 1, X[1]), amr_centre(a, m, 2, X[2])};
            amr_lattice_at<D - 1>(a, snap, m + 1, c, out);
            return;
        }
    }
    long long Y[3] = {X[0], X[1], X[2]};
    if (lv < m) {
        Y[0] >>= (m - lv); Y[1] >>= (m - lv); Y[2] >>= (m - lv);
    }
    const float* q = amr_cell(a, snap, leaf, Y);
#pragma unroll
    for (int k = 0; k < FTE_NFIELD; ++k) out[k] = q[k];
}

// trilinear interpolation (physical weights) of the level-m lattice at point c,
// held constant beyond the outermost centres in r and theta, periodic in phi
template <int D>
__device__ __noinline__ void amr_lattice_at(const AmrK& a, int snap, int m, const double c[3], double out[FTE_NFIELD])
{
    long long i0[3];
    double f[3];
    for (int ax = 0; ax < 3; ++ax) {
        const double n = (double)amr_n(a, m, ax);
        double x;
        if (ax == 0) x = a.radial ? log(c[0] / a.r_min) / (log(a.r_max / a.r_min) / n) - 0.5
                                  : (c[0] - a.r_min) / ((a.r_max - a.r_min) / n) - 0.5;
        else if (ax == 1) x = (c[1] - a.th_min) / ((a.th_max - a.th_min) / n) - 0.5;
        else x = c[2] / (2.0 * 3.141592653589793 / n) - 0.5;
        if (ax < 2 && x < 0.0) { i0[ax] = 0; f[ax] = 0.0; }
        else if (ax < 2 && x >= n - 1.0) { i0[ax] = (long long)n - 2; f[ax] = 1.0; }
        else {
            i0[ax] = (long long)floor(x);
            if (ax == 0) {
                const double c0 = amr_centre(a, m, 0, i0[0]), c1 = amr_centre(a, m, 0, i0[0] + 1);
                f[ax] = (c[0] - c0) / (c1 - c0);
            } else {
                f[ax] = x - (double)i0[ax];
            }
        }
    }
    for (int k = 0; k < FTE_NFIELD; ++k) out[k] = 0.0;
    for (int cc = 0; cc < 8; ++cc) {
        const int d0 = cc & 1, d1 = (cc >> 1) & 1, d2 = cc >> 2;
        const double w = (d0 ? f[0] : 1.0 - f[0]) * (d1 ? f[1] : 1.0 - f[1]) * (d2 ? f[2] : 1.0 - f[2]);
        const long long X[3] = {i0[0] + d0, i0[1] + d1, i0[2] + d2};
        double v[FTE_NFIELD];
        amr_lattice_cell<D>(a, snap, m, X, v);
        for (int k = 0; k < FTE_NFIELD; ++k) out[k] += w * v[k];
    }
}

// one thread per (snapshot, leaf, padded cell); interior cells are left alone
__global__ void __launch_bounds__(128) ghost_kernel(const AmrK a)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long P3 = (long long)a.P * a.P * a.P;
    if (t >= (long long)a.n_snap * a.n_leaves * P3) return;
    const int snap = (int)(t / ((long long)a.n_leaves * P3));
    const long long rem = t - (long long)snap * a.n_leaves * P3;
    const int leaf = (int)(rem / P3);
    const int cell = (int)(rem - (long long)leaf * P3);
    const int li = cell % a.P, lj = (cell / a.P) % a.P, lk = cell / (a.P * a.P);
    const bool interior = li >= 1 && li <= a.B && lj >= 1 && lj <= a.B && lk >= 1 && lk <= a.B;
    if (interior) return;
    const int4 lf = a.leaves[leaf];
    const int lv = lf.x;
    long long G[3] = {(long long)lf.y * a.B + li - 1, (long long)lf.z * a.B + lj - 1,
                      (long long)lf.w * a.B + lk - 1};
    amr_fold(a, lv, G);
    const int src = amr_leaf_of(a, lv, G);
    const int lc = a.leaves[src].x;
    double v[FTE_NFIELD];
    if (lc == lv) {
        const float* q = amr_cell(a, snap, src, G);
        for (int k = 0; k < FTE_NFIELD; ++k) v[k] = q[k];
    } else {
        const double c[3] = {amr_centre(a, lv, 0, G[0]), amr_centre(a, lv, 1, G[1]), amr_centre(a, lv, 2, G[2])};
        amr_lattice_at<4>(a, snap, lc > lv ? lv + 1 : lv - 1, c, v);
    }
    float* o = a.fw + ((long long)snap * a.snap_recs + (long long)leaf * P3 + cell) * FTE_REC;
    for (int k = 0; k < FTE_NFIELD; ++k) o[k] = (float)v[k];
    for (int k = FTE_NFIELD; k < FTE_REC; ++k) o[k] = 0.f;
}

// table fill: one thread per leaf writes the finest positions it covers;
// counts malformed leaves and overlaps
__global__ void table_kernel(const int4* leaves, int n_leaves, int L, int nb0, int nb1, int nb2, int nf0,
                             int nf1, int* table, unsigned* status)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_leaves) return;
    const int4 lf = leaves[n];
    if (lf.x < 0 || lf.x > L || lf.y < 0 || lf.y >= (nb0 << lf.x) || lf.z < 0 || lf.z >= (nb1 << lf.x) ||
        lf.w < 0 || lf.w >= (nb2 << lf.x)) {
        atomicAdd(status + 0, 1u);
        return;
    }
    const int s = 1 << (L - lf.x);
    for (int c = 0; c < s; ++c)
        for (int b = 0; b < s; ++b)
            for (int q = 0; q < s; ++q) {
                const long long idx = ((long long)(lf.w * s + c) * nf1 + (lf.z * s + b)) * nf0 + (lf.y * s + q);
                if (atomicExch(table + idx, n) != -1) atomicAdd(status + 1, 1u);
            }
}

// coverage and 2:1 nesting over faces, edges and corners (phi periodic)
__global__ void nesting_kernel(const int4* leaves, const int* table, int nf0, int nf1, int nf2, unsigned* status)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nf0 * nf1 * nf2) return;
    const int i = (int)(t % nf0), j = (int)((t / nf0) % nf1), k = (int)(t / ((long long)nf0 * nf1));
    const int me = table[t];
    if (me < 0) { atomicAdd(status + 2, 1u); return; }
    const int lv = leaves[me].x;
    for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                const int ii = i + di, jj = j + dj;
                if (ii < 0 || ii >= nf0 || jj < 0 || jj >= nf1) continue;
                const int kk = ((k + dk) % nf2 + nf2) % nf2;
                const int o = table[((long long)kk * nf1 + jj) * nf0 + ii];
                if (o >= 0 && abs(leaves[o].x - lv) > 1) atomicAdd(status + 3, 1u);
            }
}

cudaError_t launch_amr_table(const GridK& g, int* table, unsigned* status, cudaStream_t s)
{
    const long long nt = (long long)g.nf0 * g.nf1 * g.nf2;
    cudaError_t e = cudaMemsetAsync(table, 0xFF, (size_t)nt * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(status, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    table_kernel<<<(unsigned)((g.amr_leaves + 127) / 128), 128, 0, s>>>(
        g.leaves, g.amr_leaves, g.L, g.nr / g.B, g.nth / g.B, g.nph / g.B, g.nf0, g.nf1, table, status);
    nesting_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g.leaves, table, g.nf0, g.nf1, g.nf2, status);
    return cudaGetLastError();
}

cudaError_t launch_amr_ghosts(const GridK& g, int n_snap, double r_min, double r_max, double th_min,
                              double th_max, cudaStream_t s)
{
    AmrK a;
    a.f = g.fields;
    a.fw = const_cast<float*>(g.fields);
    a.snap_recs = g.snap_recs;
    a.n_leaves = g.amr_leaves;
    a.B = g.B; a.P = g.P; a.L = g.L; a.n_snap = n_snap;
    a.nr = g.nr; a.nth = g.nth; a.nph = g.nph;
    a.nf0 = g.nf0; a.nf1 = g.nf1; a.nf2 = g.nf2;
    a.leaves = g.leaves;
    a.table = g.table;
    a.radial = g.radial;
    a.r_min = r_min; a.r_max = r_max; a.th_min = th_min; a.th_max = th_max;
    const long long n = (long long)n_snap * g.amr_leaves * g.P * g.P * g.P;
    ghost_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fte
