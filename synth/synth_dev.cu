// Device implementation of the seeded input generators declared in synth.h.
// Same definitions as synth_host.c; written separately so that neither the
// oracle nor the product library needs the other's code.
#include <cuda_runtime.h>
#include "synth.h"

namespace {

constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ULL;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long draw(unsigned long long seed,
                                                   unsigned long long i)
{
    return mix64(seed + (i + 1) * kGamma);
}

__global__ void rmat_kernel(synth_rmat p, unsigned long long e0,
                            unsigned long long count, uint32_t* __restrict__ src,
                            uint32_t* __restrict__ dst, uint32_t* __restrict__ w,
                            unsigned long long seed_w)
{
    const unsigned k = p.scale;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         t < count; t += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long e = e0 + t;
        unsigned long long s = 0, d = 0, r64 = 0;
        for (unsigned l = 0; l < k; ++l) {
            if ((l & 1) == 0) r64 = draw(p.seed, e * 16 + (l >> 1));
            unsigned r = (l & 1) ? (unsigned)(r64 >> 32) : (unsigned)r64;
            unsigned long long sb, db;
            if (r < p.tA)        { sb = 0; db = 0; }
            else if (r < p.tAB)  { sb = 0; db = 1; }
            else if (r < p.tABC) { sb = 1; db = 0; }
            else                 { sb = 1; db = 1; }
            s |= sb << (k - 1 - l);
            d |= db << (k - 1 - l);
        }
        src[t] = (uint32_t)s;
        dst[t] = (uint32_t)d;
        if (w) {
            unsigned long long key = (s << 32) | d;
            w[t] = 1u + (uint32_t)(draw(seed_w, key) % 255u);
        }
    }
}

}  // namespace

extern "C" int synth_rmat_device(const synth_rmat* p, uint64_t e0, uint64_t count,
                                 uint32_t* src, uint32_t* dst, uint32_t* w,
                                 uint64_t seed_w, void* stream)
{
    if (count == 0) return 0;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long blocks = (count + 255) / 256;
    unsigned long long cap = (unsigned long long)sms * 16;
    if (blocks > cap) blocks = cap;
    rmat_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        *p, e0, count, src, dst, w, seed_w);
    return (int)cudaGetLastError();
}
