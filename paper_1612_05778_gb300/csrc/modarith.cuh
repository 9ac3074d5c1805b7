// modarith.cuh -- word-size prime-field arithmetic for 2^29 < p < 2^30.
//
// Values travel in [0, 2p) between butterflies (lazy reduction).
//  * shoup(): V. Shoup's multiplication by a constant w with the
//    precomputed quotient w' = floor(w 2^32 / p) (as in NTL's MulModPrecon
//    and D. Harvey, "Faster arithmetic for number-theoretic transforms",
//    J. Symb. Comp. 60, 2014): for any 32-bit x it returns x*w mod p up to
//    one extra p, i.e. a value in [0, 2p).
//  * montmul(): P. Montgomery's REDC ("Modular multiplication without
//    trial division", Math. Comp. 44, 1985) with R = 2^32: a*b*R^{-1} mod p
//    in [0, 2p) for a, b in [0, 2p) (needs 4p^2 < pR, true for p < 2^30).
//  * Butterflies: Gentleman-Sande (DIF, forward) and Cooley-Tukey (DIT,
//    inverse), both keeping [0, 2p).
#pragma once
#include <stdint.h>

namespace ipm {

// [0, 2m) -> [0, m): unsigned min picks x - m exactly when x >= m.
__device__ __forceinline__ uint32_t red(uint32_t x, uint32_t m) { return min(x, x - m); }

__device__ __forceinline__ uint32_t shoup(uint32_t x, uint2 w, uint32_t p) {
    const uint32_t q = __umulhi(x, w.y);
    return x * w.x - q * p;
}

__device__ __forceinline__ uint32_t montmul(uint32_t a, uint32_t b, uint32_t p, uint32_t mont) {
    const uint32_t lo = a * b;
    const uint32_t hi = __umulhi(a, b);
    const uint32_t m = lo * mont;
    const uint32_t mh = __umulhi(m, p);
    // (a*b + m*p) / 2^32: the low words sum to 0 mod 2^32, with a carry
    // exactly when lo != 0.
    return hi + mh + (lo != 0u);
}

// Forward (DIF) butterfly: (x, y) -> (x + y, (x - y) w), inputs in [0, 2p).
__device__ __forceinline__ void bf_dif(uint32_t &x, uint32_t &y, uint2 w, uint32_t p, uint32_t p2) {
    const uint32_t s = red(x + y, p2);
    const uint32_t d = x - y + p2;
    y = shoup(d, w, p);
    x = s;
}

// Inverse (DIT) butterfly: (x, y) -> (x + y w, x - y w), inputs in [0, 2p).
__device__ __forceinline__ void bf_dit(uint32_t &x, uint32_t &y, uint2 w, uint32_t p, uint32_t p2) {
    const uint32_t t = shoup(y, w, p);
    const uint32_t s = red(x + t, p2);
    const uint32_t d = red(x - t + p2, p2);
    x = s;
    y = d;
}

// ---------------------------------------------------------------------------
// Radix-2 stages over a shared-memory tile.  A twiddle table of order
// T = 2^logT holds (omega_T^e, Shoup quotient); a stage of half-size h uses
// omega_{2h}^k = omega_T^{k T / (2h)}.
// ---------------------------------------------------------------------------

// nt transforms of length 2^logL along contiguous elements; transform i
// starts at s + i*tstride.  Forward (DIF): natural order in, bit-reversed out.
__device__ __forceinline__ void dif_rows(uint32_t *s, int nt, int tstride, int logL,
                                         const uint2 *__restrict__ tw, int logT, uint32_t p,
                                         uint32_t p2) {
    if (logL == 0) return;
    const int halfm = (1 << (logL - 1)) - 1;
    const int total = nt << (logL - 1);
    for (int logh = logL - 1; logh >= 0; --logh) {
        const int h = 1 << logh;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int tr = b >> (logL - 1);
            const int k = b & halfm;
            const int kk = k & (h - 1);
            const int i0 = ((k >> logh) << (logh + 1)) + kk;
            uint32_t *x = s + tr * tstride;
            const uint2 w = tw[kk << (logT - logh - 1)];
            uint32_t u = x[i0], v = x[i0 + h];
            bf_dif(u, v, w, p, p2);
            x[i0] = u;
            x[i0 + h] = v;
        }
        __syncthreads();
    }
}

// Inverse (DIT): bit-reversed order in, natural order out (unnormalised).
__device__ __forceinline__ void dit_rows(uint32_t *s, int nt, int tstride, int logL,
                                         const uint2 *__restrict__ tw, int logT, uint32_t p,
                                         uint32_t p2) {
    if (logL == 0) return;
    const int halfm = (1 << (logL - 1)) - 1;
    const int total = nt << (logL - 1);
    for (int logh = 0; logh < logL; ++logh) {
        const int h = 1 << logh;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int tr = b >> (logL - 1);
            const int k = b & halfm;
            const int kk = k & (h - 1);
            const int i0 = ((k >> logh) << (logh + 1)) + kk;
            uint32_t *x = s + tr * tstride;
            const uint2 w = tw[kk << (logT - logh - 1)];
            uint32_t u = x[i0], v = x[i0 + h];
            bf_dit(u, v, w, p, p2);
            x[i0] = u;
            x[i0 + h] = v;
        }
        __syncthreads();
    }
}

// 2^logC columns of length 2^logL; column c is s[c + i*pitch], i < 2^logL.
// Consecutive threads take consecutive columns (conflict-free rows).
__device__ __forceinline__ void dif_cols(uint32_t *s, int logC, int pitch, int logL,
                                         const uint2 *__restrict__ tw, int logT, uint32_t p,
                                         uint32_t p2) {
    if (logL == 0) return;
    const int cm = (1 << logC) - 1;
    const int total = 1 << (logC + logL - 1);
    for (int logh = logL - 1; logh >= 0; --logh) {
        const int h = 1 << logh;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int c = b & cm;
            const int k = b >> logC;
            const int kk = k & (h - 1);
            const int i0 = ((k >> logh) << (logh + 1)) + kk;
            const uint2 w = tw[kk << (logT - logh - 1)];
            uint32_t *x0 = s + c + i0 * pitch;
            uint32_t *x1 = x0 + h * pitch;
            uint32_t u = *x0, v = *x1;
            bf_dif(u, v, w, p, p2);
            *x0 = u;
            *x1 = v;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void dit_cols(uint32_t *s, int logC, int pitch, int logL,
                                         const uint2 *__restrict__ tw, int logT, uint32_t p,
                                         uint32_t p2) {
    if (logL == 0) return;
    const int cm = (1 << logC) - 1;
    const int total = 1 << (logC + logL - 1);
    for (int logh = 0; logh < logL; ++logh) {
        const int h = 1 << logh;
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int c = b & cm;
            const int k = b >> logC;
            const int kk = k & (h - 1);
            const int i0 = ((k >> logh) << (logh + 1)) + kk;
            const uint2 w = tw[kk << (logT - logh - 1)];
            uint32_t *x0 = s + c + i0 * pitch;
            uint32_t *x1 = x0 + h * pitch;
            uint32_t u = *x0, v = *x1;
            bf_dit(u, v, w, p, p2);
            *x0 = u;
            *x1 = v;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, int bits) {
    return bits ? (__brev(x) >> (32 - bits)) : 0u;
}

}  // namespace ipm
