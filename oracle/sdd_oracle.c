/*
 * CPU oracle for the stochastic domain decomposition (SDD) mesh generator.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load this library.  The CUDA library never calls it and shares no
 * code with it (no headers, helpers, tables or constants).
 *
 * What is here, each written plainly from the paper and the published definitions:
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *     SC'11): the counter-based generator both sides draw from (the paper only asks for
 *     N(0,1) samples, Sec. 3.4).
 *   - Box-Muller normals from two uniforms.
 *   - Bilinear interpolation of the monitor and its gradient (Sec. 3.4) and Keys (1981)
 *     cubic-convolution ("bi-cubic", Sec. 3.4) interpolation of the previous mesh.
 *   - One Euler-Maruyama path (Eq. 7) of the SDE of Eq. (5b), with the boundary test of
 *     Sec. 3.4 (endpoint outside the unit square, or a Brownian-bridge crossing between
 *     substeps after Jansons & Lythe) and the value the path contributes to Eq. (5a)
 *     (Dirichlet) or Eq. (6) (periodic).
 *   - Sequential estimator sums over paths (the arithmetic mean of Sec. 3.4).
 *
 * The path code lives in oracle_paths_body.h and is compiled twice below, once with
 * REAL = double (suffix _f64) and once with REAL = float (suffix _f32), so the FP32
 * variant performs every path operation in single precision.  Build with
 * -ffp-contract=off so no multiply-add is fused behind the source's back on any host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al. 2011).  One round maps (c0, c1, c2, c3) with key (k0, k1) to
 *   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
 * (0x9E3779B9, 0xBB67AE85) between rounds.  Ten rounds.
 * ------------------------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* n independent draws: ctr is n x 4, key is n x 2, out is n x 4. */
void oracle_philox_batch(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i)
        oracle_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing of the single-core baseline). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------------------ */
#define CAT2_(a, b) a##_##b
#define CAT2(a, b) CAT2_(a, b)

#define REAL double
#define SFX f64
#define REAL_IS_FLOAT 0
#include "oracle_paths_body.h"
#undef REAL
#undef SFX
#undef REAL_IS_FLOAT

#define REAL float
#define SFX f32
#define REAL_IS_FLOAT 1
#include "oracle_paths_body.h"
#undef REAL
#undef SFX
#undef REAL_IS_FLOAT
