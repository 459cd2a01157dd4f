/* Host implementation of the seeded input generators declared in synth.h. */
#include "synth.h"

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_draw(uint64_t seed, uint64_t i)
{
    return mix64(seed + (i + 1) * GAMMA);
}

void synth_rmat_host(const synth_rmat* p, uint64_t e0, uint64_t count,
                     uint32_t* src, uint32_t* dst)
{
    const uint32_t k = p->scale;
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < (int64_t)count; ++t) {
        uint64_t e = e0 + (uint64_t)t;
        uint64_t s = 0, d = 0, r64 = 0;
        for (uint32_t l = 0; l < k; ++l) {
            if ((l & 1) == 0) r64 = synth_draw(p->seed, e * 16 + (l >> 1));
            uint32_t r = (l & 1) ? (uint32_t)(r64 >> 32) : (uint32_t)r64;
            uint64_t sb, db;
            if (r < p->tA)        { sb = 0; db = 0; }
            else if (r < p->tAB)  { sb = 0; db = 1; }
            else if (r < p->tABC) { sb = 1; db = 0; }
            else                  { sb = 1; db = 1; }
            s |= sb << (k - 1 - l);
            d |= db << (k - 1 - l);
        }
        src[t] = (uint32_t)s;
        dst[t] = (uint32_t)d;
    }
}

void synth_weights_host(uint64_t seed_w, uint64_t count, const uint32_t* src,
                        const uint32_t* dst, uint32_t* w)
{
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < (int64_t)count; ++t) {
        uint64_t key = ((uint64_t)src[t] << 32) | dst[t];
        w[t] = 1u + (uint32_t)(synth_draw(seed_w, key) % 255u);
    }
}
