// Spatial ordering of the alive particles: a counting sort by grid bucket (the
// lower corner of the interpolation stencil, radial index in pairs, and the sign
// of mu), so
// that consecutive entries of the order list - and so the lanes of a warp - read
// the same cache lines of the background.  Dead particles are left out, which
// also compacts the work list.  Performance only: each particle's trajectory does not depend on the order.
#include "fte_kernels.cuh"

namespace fte {


// Bucket of a point: the lower corner (i0, j0, k0) of its interpolation stencil -
// the first of the records the step gathers - with i0 taken in pairs, so that the
// particles of one bucket read the same corner records (a bucket by the cell
// holding the point would mix up to 3 x 2 x 2 different stencils).  The index
// arithmetic follows locate / locate_amr.
__device__ __forceinline__ int bucket_of(const GridK& g, float x, float y, float z)
{
    const float rho2 = x * x + y * y;
    const float r = sqrtf(rho2 + z * z);
    const float th = atan2f(sqrtf(rho2), z);
    float ph = atan2f(y, x);
    if (ph < 0.f) ph += kTwoPi;
    const float xr = g.radial ? logf(r / g.r_min) * g.inv_dr : (r - g.r_min) * g.inv_dr;
    const float xt = (th - g.th_min) * g.inv_dth;
    const float xp = ph * g.inv_dph;
    if (g.amr) {      // AMR: leaf, then the stencil corner on its padded lattice (0 .. B)
        const float ur = g.radial ? logf(r / g.r_min) * g.inv_lnr : (r - g.r_min) * g.inv_lnr;
        const float ut = (th - g.th_min) * g.inv_thspan;
        const float up = ph * (1.f / kTwoPi);
        const int f0 = min(max((int)floorf(ur * (float)g.nf0), 0), g.nf0 - 1);
        const int f1 = min(max((int)floorf(ut * (float)g.nf1), 0), g.nf1 - 1);
        int f2 = (int)floorf(up * (float)g.nf2);
        if (f2 < 0) f2 += g.nf2;
        if (f2 >= g.nf2) f2 -= g.nf2;
        const int leaf = min(max(__ldg(g.table + ((long long)f2 * g.nf1 + f1) * g.nf0 + f0), 0), g.amr_leaves - 1);
        const int4 lf = __ldg(g.leaves + leaf);
        const float s = (float)(1 << lf.x);
        const int B = g.B;
        const int ii = min(max((int)floorf(xr * s - 0.5f) - (lf.y * B - 1), 0), B);
        const int jj = min(max((int)floorf(xt * s - 0.5f) - (lf.z * B - 1), 0), B);
        const int kk = min(max((int)floorf(xp * s - 0.5f) - (lf.w * B - 1), 0), B);
        return ((leaf * (B + 1) + kk) * (B + 1) + jj) * ((B + 2) >> 1) + (ii >> 1);
    }
    const int i = min(max((int)floorf(xr - 0.5f), 0), g.nr - 2);
    const int j = min(max((int)floorf(xt - 0.5f), 0), g.nth - 2);
    int k = (int)floorf(xp - 0.5f);
    if (k < 0) k += g.nph;
    k = min(max(k, 0), g.nph - 1);
    const int nrb = (g.nr + 1) >> 1;
    return (k * g.nth + j) * nrb + (i >> 1);
}

// Within a bucket the particles are grouped by the sign of the pitch-angle cosine
// (kMuBins equal bins of mu): particles moving the same way along the field stay
// together for longer (mu changes on the scattering time, many reorderings apart),
// so the lanes of a warp keep sharing records through the launch.  Two bins
// measured best: four halve the particles per bucket for a smaller gain.
constexpr int kMuBins = 2;

__global__ void __launch_bounds__(256) key_kernel(const SortArgs a)
{
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int key = -1, rank = 0;
    if (a.steps ? a.steps[i] > a.steps_min : a.status[i] == FTE_ALIVE) {
        int mb = 0;
        if (a.mu) mb = min(max((int)((a.mu[i] + 1.f) * (0.5f * kMuBins)), 0), kMuBins - 1);
        key = bucket_of(a.g, a.x[i], a.y[i], a.z[i]) * kMuBins + mb;
        rank = (int)atomicAdd(a.hist + key, 1u);
    }
    a.key[i] = key;
    a.rank[i] = rank;
}

// three-phase exclusive scan of hist[0..nb) into hist, total into hist[nb]
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* sh, unsigned* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const unsigned warp_off = wid ? sh[wid - 1] : 0u;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) tile_sum_kernel(const unsigned* hist, int nb, unsigned* tiles)
{
    __shared__ unsigned sh[32];
    const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    unsigned s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < nb) s += hist[base + q];
    unsigned total;
    block_exclusive_scan(s, sh, &total);
    if (threadIdx.x == 0) tiles[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) tile_offsets_kernel(unsigned* tiles, int ntiles)
{
    // one block: exclusive scan of the tile sums, in chunks of blockDim.x
    __shared__ unsigned sh[32];
    unsigned carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += kScanThreads) {
        const int t = b0 + threadIdx.x;
        const unsigned v = t < ntiles ? tiles[t] : 0u;
        unsigned total;
        const unsigned ex = block_exclusive_scan(v, sh, &total);
        if (t < ntiles) tiles[t] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tiles[ntiles] = carry;
}

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(unsigned* hist, int nb, const unsigned* tiles,
                                                                 int ntiles)
{
    __shared__ unsigned sh[32];
    const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    unsigned v[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = (base + q < nb) ? hist[base + q] : 0u;
        s += v[q];
    }
    unsigned total;
    unsigned run = tiles[blockIdx.x] + block_exclusive_scan(s, sh, &total);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < nb) hist[base + q] = run;
        run += v[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) hist[nb] = tiles[ntiles];
}

__global__ void __launch_bounds__(256) scatter_kernel(const SortArgs a)
{
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int key = a.key[i];
    if (key >= 0) a.order[a.hist[key] + (unsigned)a.rank[i]] = (uint32_t)i;
}

int sort_buckets(const GridK& g)
{
    if (g.amr) return g.amr_leaves * (g.B + 1) * (g.B + 1) * ((g.B + 2) >> 1) * kMuBins;
    return g.nph * g.nth * ((g.nr + 1) >> 1) * kMuBins;
}

size_t sort_scratch_bytes(const GridK& g, unsigned long long n)
{
    const long long nb = sort_buckets(g);
    const long long ntiles = (nb + kScanTile - 1) / kScanTile;
    size_t b = 0;
    b += ((size_t)(nb + 1) * 4 + 255) & ~(size_t)255;        // hist / offsets
    b += ((size_t)(ntiles + 1) * 4 + 255) & ~(size_t)255;    // tile sums
    b += 3 * (((size_t)n * 4 + 255) & ~(size_t)255);         // key, rank, order
    return b;
}

void sort_carve(const GridK& g, unsigned long long n, char* p, SortArgs* a)
{
    const long long nb = sort_buckets(g);
    const long long ntiles = (nb + kScanTile - 1) / kScanTile;
    a->hist = (unsigned*)p; p += ((size_t)(nb + 1) * 4 + 255) & ~(size_t)255;
    a->tiles = (unsigned*)p; p += ((size_t)(ntiles + 1) * 4 + 255) & ~(size_t)255;
    a->key = (int*)p; p += ((size_t)n * 4 + 255) & ~(size_t)255;
    a->rank = (int*)p; p += ((size_t)n * 4 + 255) & ~(size_t)255;
    a->order = (uint32_t*)p;
    a->nb = (int)nb;
    a->ntiles = (int)ntiles;
}

cudaError_t launch_sort(const SortArgs& a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.hist, 0, (size_t)(a.nb + 1) * 4, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((a.n + 255) / 256);
    if (blocks) key_kernel<<<blocks, 256, 0, s>>>(a);
    tile_sum_kernel<<<a.ntiles, kScanThreads, 0, s>>>(a.hist, a.nb, a.tiles);
    tile_offsets_kernel<<<1, kScanThreads, 0, s>>>(a.tiles, a.ntiles);
    tile_scan_kernel<<<a.ntiles, kScanThreads, 0, s>>>(a.hist, a.nb, a.tiles, a.ntiles);
    if (blocks) scatter_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fte
