/*
 * Oracle-internal counter-based generator (test infrastructure only).
 *
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state after i+1 advances is
 * seed + (i+1)*GAMMA, and the output is that state passed through the 64-bit
 * finaliser "variant 13" of D. Stafford's MurmurHash3 mix study.  Evaluating
 * output i directly from (seed, i) makes the generator counter-based.
 *
 * The CUDA path implements the same published generator on its own; the two
 * share no source.
 */
#ifndef ORACLE_SM64_H
#define ORACLE_SM64_H
#include <stdint.h>

static inline uint64_t orc_sm64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform double in [0,1): the top 53 bits scaled by 2^-53. */
static inline double orc_u01(uint64_t seed, uint64_t i)
{
    return (double)(orc_sm64_at(seed, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* Index in [0,n) by Lemire's multiply-shift on the 64-bit output. */
static inline uint32_t orc_index(uint64_t seed, uint64_t i, uint32_t n)
{
    unsigned __int128 p = (unsigned __int128)orc_sm64_at(seed, i) * (unsigned __int128)n;
    return (uint32_t)(p >> 64);
}

#endif
