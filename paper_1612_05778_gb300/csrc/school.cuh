// school.cuh -- the schoolbook family's tile: one output coefficient
// c_k = sum_{i+j=k} a_i b_j by direct limb products (the definition of §1
// computed as written), for any block size.  Thread q owns output column q
// (limb position q of c_k) and sums, over the terms (i, k - i), the low
// words of the 64-bit limb products a_i[u] b_j[q-u] and the high words of
// a_i[u] b_j[q-1-u], positive and negative terms apart, in 64-bit
// accumulators: every column receives at most 2 min(na, nb) min(La, Lb)
// words below 2^32 (the planner keeps this count at most 2^30, so both
// sums stay below 2^62).  Then one thread carries the signed column sums
// into 32-bit limbs and writes sign and magnitude.  The tile of k also
// checks the bit bound of a_k and b_k, so every input is checked once.
// Shared memory: school_smem(P) bytes at smem.
#pragma once
#include <stdint.h>

#include "ipm_internal.h"

namespace ipm {

__device__ __forceinline__ void school_tile(const KParams &P, int64_t k, const uint32_t *__restrict__ a,
                                            const uint8_t *__restrict__ an, const uint32_t *__restrict__ b,
                                            const uint8_t *__restrict__ bn, uint32_t *__restrict__ c,
                                            uint8_t *__restrict__ cn, unsigned char *smem) {
    long long *col = reinterpret_cast<long long *>(smem);  // La + Lb + 1 signed column sums, then limbs
    const int la = P.la, lb = P.lb, lc = P.lc;
    const int ncol = la + lb;
    if (threadIdx.x == 0) {
        if (k < P.na) {
            const int top = (int)P.bits_a - 32 * (la - 1);
            if (top < 32 && (a[k * la + la - 1] >> top) != 0u) atomicOr(P.err, ERRBIT_BOUND);
        }
        if (k < P.nb) {
            const int top = (int)P.bits_b - 32 * (lb - 1);
            if (top < 32 && (b[k * lb + lb - 1] >> top) != 0u) atomicOr(P.err, ERRBIT_BOUND);
        }
    }
    const int64_t i0 = k - (P.nb - 1) > 0 ? k - (P.nb - 1) : 0;
    const int64_t i1 = k < P.na - 1 ? k : P.na - 1;
    for (int q = threadIdx.x; q <= ncol; q += blockDim.x) {
        unsigned long long pos = 0ull, neg = 0ull;
        // low words: u + v = q; high words: u + v = q - 1
        const int ulo0 = q - (lb - 1) > 0 ? q - (lb - 1) : 0, ulo1 = q < la - 1 ? q : la - 1;
        const int uhi0 = q - lb > 0 ? q - lb : 0, uhi1 = q - 1 < la - 1 ? q - 1 : la - 1;
        for (int64_t i = i0; i <= i1; ++i) {
            const int64_t j = k - i;
            const uint32_t *ai = a + i * la;
            const uint32_t *bj = b + j * lb;
            unsigned long long s = 0ull;
            for (int u = ulo0; u <= ulo1; ++u) s += (uint32_t)((unsigned long long)ai[u] * bj[q - u]);
            for (int u = uhi0; u <= uhi1; ++u) s += (uint32_t)(((unsigned long long)ai[u] * bj[q - 1 - u]) >> 32);
            if ((an[i] != 0) != (bn[j] != 0))
                neg += s;
            else
                pos += s;
        }
        col[q] = (long long)(pos - neg);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // two's complement limbs of sum_q col[q] 2^(32 q)
        uint32_t *limb = reinterpret_cast<uint32_t *>(col + ncol + 1);
        long long carry = 0;
        for (int q = 0; q <= ncol; ++q) {
            const long long t = col[q] + carry;
            carry = t >> 32;  // arithmetic shift: floor division
            limb[q] = (uint32_t)t;
        }
        const bool negative = carry < 0;
        uint32_t *out = c + k * lc;
        uint32_t any = 0u, borrow = 1u;
        for (int q = 0; q < lc; ++q) {
            uint32_t w = limb[q];
            if (negative) {  // magnitude = two's complement negation
                w = ~w + borrow;
                borrow = (borrow && w == 0u) ? 1u : 0u;
            }
            out[q] = w;
            any |= w;
        }
        cn[k] = (uint8_t)(negative && any != 0u);
    }
    __syncthreads();
}

}  // namespace ipm
