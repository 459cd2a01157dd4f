/*
 * synth.h -- seeded synthetic inputs shared by the oracle and the CUDA path.
 *
 * This module generates raw R-MAT edge lists, edge weights and query sources.
 * It holds none of the graph method's arithmetic: no CSR/CSC build, no dedupe,
 * no relaxation. Both consumers (oracle/ and the product library) build their
 * own graph structures from the raw edges it produces.
 *
 * Random numbers: one counter-based generator, the splitmix64 stream of
 * Steele, Lea and Flood ("Fast splittable pseudorandom number generators",
 * OOPSLA 2014; public-domain reference code by S. Vigna). The stream seeded
 * with `seed` has increment GAMMA = 0x9E3779B97F4A7C15 and its i-th output
 * (0-based) is  mix64(seed + (i + 1) * GAMMA)  with
 *   mix64(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
 *             z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
 * Host (synth_host.c) and device (synth_dev.cu) each implement it from this
 * definition; tests check the two produce identical edge lists.
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004), as used for the paper's
 * RMAT-k graphs (2^k vertices, 2^(k+4) edges, evaluation section, Table 2):
 * edge e at scale k chooses, at each level l = 0..k-1 (most significant bit
 * first), one quadrant of the adjacency matrix from a 32-bit uniform r:
 *   r < tA -> (src bit, dst bit) = (0,0);  r < tAB -> (0,1);
 *   r < tABC -> (1,0);  else (1,1).
 * r for level l is half of the 64-bit draw with counter e*16 + (l >> 1):
 * the low 32 bits for even l, the high 32 bits for odd l. Thresholds are
 * floor(a*2^32), floor((a+b)*2^32), floor((a+b+c)*2^32). No noise and no
 * vertex relabelling: vertex 0 is the largest hub. Self-loops and duplicate
 * edges are emitted as drawn; removing them is the consumer's job.
 *
 * Weights: w(u,v) = 1 + (draw(seed_w, (u << 32) | v) mod 255), in [1,255].
 * A weight depends only on the endpoints, so duplicates carry equal weights
 * and any storage order (CSR, CSC) sees the same value.
 */
#ifndef SYNTH_H
#define SYNTH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct synth_rmat {
    uint32_t scale;      /* vertices n = 2^scale, scale <= 32            */
    uint64_t m;          /* number of raw edges to draw                  */
    uint32_t tA, tAB, tABC; /* cumulative quadrant thresholds, see above */
    uint64_t seed;       /* stream seed for the quadrant draws           */
} synth_rmat;

/* i-th output of the splitmix64 stream seeded with `seed`. */
uint64_t synth_draw(uint64_t seed, uint64_t i);

/* Host generator: edges [e0, e0+count) into src/dst (caller-owned host
 * arrays of `count` entries). Uses all host threads (OpenMP). */
void synth_rmat_host(const synth_rmat* p, uint64_t e0, uint64_t count,
                     uint32_t* src, uint32_t* dst);

/* Host weights for `count` endpoint pairs. */
void synth_weights_host(uint64_t seed_w, uint64_t count, const uint32_t* src,
                        const uint32_t* dst, uint32_t* w);

/* Device generator (synth_dev.cu): same edges into device arrays; `w` may be
 * NULL, else receives the weights for seed_w. `stream` is a cudaStream_t.
 * Returns 0, or a CUDA error code. */
int synth_rmat_device(const synth_rmat* p, uint64_t e0, uint64_t count,
                      uint32_t* src, uint32_t* dst, uint32_t* w,
                      uint64_t seed_w, void* stream);

#ifdef __cplusplus
}
#endif
#endif
