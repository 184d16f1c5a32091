// Measurement aids (not steps of the method): random 32-byte sector reads from
// one buffer, the read bandwidth of the memory level that holds it (L2 when it
// fits); and the transport kernel's record loads from an L1-resident buffer, the
// ceiling of a gather served by L1.
#include <stdint.h>

#include "fte_kernels.cuh"

namespace fte {

// Each warp walks consecutive records of an L1-resident buffer; lane l reads record
// k + l % spread with the transport kernel's instructions (ld.global.nc.v8 x 2 + v2
// per 96-byte record, 72 bytes of fields).  The loads are volatile, so none is
// dropped; one value per load is summed to keep a dependency on each.
__global__ void __launch_bounds__(256) probe_l1_kernel(const float* __restrict__ buf, unsigned nrec, int records,
                                                       int spread, float* out)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned span = nrec - 32u;                   // walk start so that k + lane offset < nrec
    unsigned k = (warp * 7u) % span;
    const unsigned off = lane % (unsigned)spread;
    float acc = 0.f;
    for (int i = 0; i < records; ++i) {
        const float* q = buf + (size_t)(k + off) * FTE_REC;
        float a[8], b[8], c0, c1;
        asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]),
                       "=f"(a[7])
                     : "l"(q));
        asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(b[0]), "=f"(b[1]), "=f"(b[2]), "=f"(b[3]), "=f"(b[4]), "=f"(b[5]), "=f"(b[6]),
                       "=f"(b[7])
                     : "l"(q + 8));
        asm volatile("ld.global.nc.v2.f32 {%0,%1}, [%2];" : "=f"(c0), "=f"(c1) : "l"(q + 16));
        acc += a[0] + b[0] + c0;
        k = (k + 1u == span) ? 0u : k + 1u;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_probe_l1(const float* buf, unsigned nrec, int threads, int records, int spread, float* out,
                            cudaStream_t s)
{
    probe_l1_kernel<<<(threads + 255) / 256, 256, 0, s>>>(buf, nrec, records, spread, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) probe_kernel(const float* __restrict__ buf, unsigned long long nsec,
                                                    int loads, float* out)
{
    uint32_t s = 0x9E3779B9u ^ (uint32_t)(blockIdx.x * blockDim.x + threadIdx.x) * 0x85EBCA6Bu;
    float acc = 0.f;
    for (int l = 0; l < loads; ++l) {
        s ^= s << 13; s ^= s >> 17; s ^= s << 5;           // xorshift32
        const unsigned long long sec = (unsigned long long)s % nsec;
        float v[8];
        asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                       "=f"(v[6]), "=f"(v[7])
                     : "l"(buf + sec * 8));
        acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_probe(const float* buf, unsigned long long nsec, int threads, int loads, float* out,
                         cudaStream_t s)
{
    probe_kernel<<<(threads + 255) / 256, 256, 0, s>>>(buf, nsec, loads, out);
    return cudaGetLastError();
}

}  // namespace fte
