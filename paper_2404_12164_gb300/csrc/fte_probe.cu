// Measurement helper: random 32-byte sector reads from one buffer, to measure
// the read bandwidth of the memory level that holds it (L2 when it fits).
#include <stdint.h>

#include "fte_kernels.cuh"

namespace fte {

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
