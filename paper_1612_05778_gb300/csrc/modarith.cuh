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

// Montgomery REDC of a 64-bit V < p 2^32: V 2^-32 mod p in [0, 2p).
__device__ __forceinline__ uint32_t redc64(uint64_t V, uint32_t p, uint32_t mont) {
    const uint32_t lo = (uint32_t)V, hi = (uint32_t)(V >> 32);
    const uint32_t m = lo * mont;
    return hi + __umulhi(m, p) + (lo != 0u);
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

// Asynchronous 4-byte global -> shared copies (LDGSTS, sm_80+): the data
// land in shared memory without passing through registers, so a thread can
// issue a whole tile's loads and work on other data while they fly.
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
// 8-byte asynchronous copy (both addresses 8-byte aligned).
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
// 16-byte copy through L2 only (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, int bits) {
    return bits ? (__brev(x) >> (32 - bits)) : 0u;
}

}  // namespace ipm
