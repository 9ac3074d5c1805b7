// ipm_kron.cu -- Kronecker balancing (§3, the footnote on balancing: when
// the coefficient size N is small against d log d, Kronecker substitution
// re-shapes the pair before the method runs).
//
// s consecutive coefficients of a are packed into one coefficient of
//   A'(z) = sum_k A'_k z^k,   A'_k = sum_{u<s} a_{ks+u} 2^{uw}
// (likewise b), with slot width w = bits_a + bits_b + ceil(log2 min(na, nb))
// + 1.  The packed product C' = A'B' is computed by the transform path, and
//   C'_k = sum_{t<2s-1} D_{k,t} 2^{tw},
//   D_{k,t} = sum_{i+j=k} sum_{u+v=t} a_{is+u} b_{js+v}.
// Each D_{k,t} is a partial sum of the terms of c_{ks+t}, so
// |D_{k,t}| <= min(na, nb) (2^bits_a - 1)(2^bits_b - 1) < 2^(w-1): the D
// are the unique balanced base-2^w digits of C'_k, and
//   c_m = D_{k,t} + D_{k-1,t+s}   for m = ks + t, t < s
// (the second term is absent for t = s - 1).  Slots are at most 128 bits,
// so every D and c_m fits four 32-bit words.
//
// Kernels: one warp per packed coefficient.  Packing places the s
// magnitudes in disjoint bit ranges (w > bits), summing the positive terms
// into P and the negative ones into Q, and writes |P - Q| and its sign.
// Unpacking reads w-bit fields of |C'_k| (lane t: field t), finds the
// balanced-digit carries with one ballot carry-lookahead, and adds the two
// digits that make each c_m.
#include <cuda_runtime.h>

#include "ipm_internal.h"

namespace ipm {
namespace {

constexpr int KRON_THREADS = 256;

// 32 bits of the magnitude x[0..l) starting at bit offset o; bits outside
// [0, 32 l) read as 0 (o may be negative).
__device__ __forceinline__ uint32_t bits32(const uint32_t *x, int l, int64_t o) {
    if (o <= -32 || o >= (int64_t)l * 32) return 0u;
    if (o < 0) return x[0] << (int)(-o);
    const int q = (int)(o >> 5), sh = (int)(o & 31);
    const uint32_t lo = x[q];
    const uint32_t hi = q + 1 < l ? x[q + 1] : 0u;
    return sh ? (lo >> sh) | (hi << (32 - sh)) : lo;
}

// Carry into each lane of a ripple chain where lane j generates a carry
// (bit j of g) or passes its incoming carry on (bit j of p, disjoint from
// g), with `cin` entering lane 0: the sum g + (g|p) + cin carries exactly
// like the chain.  Returns the per-lane carries; *cout gets the carry out of
// lane 31.
__device__ __forceinline__ uint32_t lookahead(uint32_t g, uint32_t p, uint32_t cin, uint32_t *cout) {
    const uint64_t x = (uint64_t)(g | p);
    const uint64_t sum = (uint64_t)g + x + cin;
    if (cout) *cout = (uint32_t)(sum >> 32) & 1u;
    return (uint32_t)(sum ^ x ^ (uint64_t)g);
}

struct PackArgs {
    const uint32_t *x;   // original limbs, n x l
    const uint8_t *xn;   // original signs
    int64_t n;
    int32_t l;
    uint32_t bits;
    uint32_t *y;         // packed limbs, n2 x l2
    uint8_t *yn;         // packed signs
    int64_t n2;
    int32_t l2;
    int32_t s, w;
    int *err;
};

// Limb `q` of P (positive terms) and Q (negative terms) of packed
// coefficient k: the terms u whose bit range [uw, uw + bits) meets limb q.
__device__ __forceinline__ void pack_limb(const PackArgs &A, int64_t k, int q, uint32_t negmask, uint32_t &P,
                                          uint32_t &Q) {
    P = Q = 0u;
    const int64_t lo = 32 * (int64_t)q;
    int u0 = (int)((lo - (int64_t)A.bits + A.w) / A.w);  // ceil((lo - bits + 1) / w) for lo >= bits
    if (lo < (int64_t)A.bits) u0 = 0;
    int u1 = (int)((lo + 31) / A.w);
    if (u1 > A.s - 1) u1 = A.s - 1;
    for (int u = u0; u <= u1; ++u) {
        const int64_t i = k * A.s + u;
        if (i >= A.n) break;
        const uint32_t v = bits32(A.x + i * A.l, A.l, lo - (int64_t)u * A.w);
        if ((negmask >> u) & 1u)
            Q |= v;
        else
            P |= v;
    }
}

__global__ void __launch_bounds__(KRON_THREADS) k_kron_pack(const PackArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * (KRON_THREADS / 32) + (threadIdx.x >> 5);
    if (k >= A.n2) return;  // the whole warp leaves together
    bool neg = false;
    if (lane < A.s) {
        const int64_t i = k * A.s + lane;
        if (i < A.n) {
            neg = A.xn[i] != 0;
            const int top_bits = (int)A.bits - 32 * (A.l - 1);  // 1..32
            if (top_bits < 32 && (A.x[i * A.l + A.l - 1] >> top_bits) != 0u) atomicOr(A.err, ERRBIT_BOUND);
        }
    }
    const uint32_t negmask = __ballot_sync(0xffffffffu, neg);
    uint32_t *out = A.y + k * A.l2;
    // sign of P - Q: the highest limb where P and Q differ
    int sign = -1;  // -1: P = Q
    for (int c0 = ((A.l2 - 1) >> 5) << 5; c0 >= 0 && sign < 0; c0 -= 32) {
        uint32_t P = 0u, Q = 0u;
        if (c0 + lane < A.l2) pack_limb(A, k, c0 + lane, negmask, P, Q);
        const uint32_t diff = __ballot_sync(0xffffffffu, P != Q);
        if (diff) {
            const int top = 31 - __clz((int)diff);
            sign = __shfl_sync(0xffffffffu, P < Q ? 1 : 0, top);
        }
    }
    if (sign < 0) {  // zero
        for (int q = lane; q < A.l2; q += 32) out[q] = 0u;
        if (lane == 0) A.yn[k] = 0;
        return;
    }
    // |P - Q| = X - Z with X the larger: subtraction with borrow lookahead
    uint32_t borrow = 0u;
    for (int c0 = 0; c0 < A.l2; c0 += 32) {
        uint32_t P = 0u, Q = 0u;
        if (c0 + lane < A.l2) pack_limb(A, k, c0 + lane, negmask, P, Q);
        const uint32_t X = sign ? Q : P, Z = sign ? P : Q;
        const uint32_t g = __ballot_sync(0xffffffffu, X < Z);
        const uint32_t p = __ballot_sync(0xffffffffu, X == Z);
        uint32_t cout;
        const uint32_t bin = lookahead(g, p, borrow, &cout);
        borrow = cout;
        if (c0 + lane < A.l2) out[c0 + lane] = X - Z - ((bin >> lane) & 1u);
    }
    if (lane == 0) A.yn[k] = (uint8_t)sign;
}

struct UnpackArgs {
    const uint32_t *y;   // packed product limbs, n2 x l2
    const uint8_t *yn;
    int64_t n2;
    int32_t l2;
    uint32_t *c;         // output limbs, nc x lc (lc <= 4)
    uint8_t *cn;
    int64_t nc;
    int32_t lc;
    int32_t s, w;
};

// Lane t's balanced digit D_{k,t} of packed coefficient k (zero for k
// outside [0, n2) and for t >= 2s - 1), as a 128-bit two's complement value.
__device__ __forceinline__ void digit(const UnpackArgs &U, int64_t k, int lane, uint32_t (&d)[4]) {
    const bool live = k >= 0 && k < U.n2;  // warp-uniform
    const bool active = live && lane < 2 * U.s - 1;
    uint32_t f[4] = {0u, 0u, 0u, 0u};
    bool neg = false;
    if (active) {
        const uint32_t *row = U.y + k * U.l2;
        const int64_t o = (int64_t)lane * U.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int lo = 32 * j;
            if (lo >= U.w) break;
            uint32_t v = bits32(row, U.l2, o + lo);
            if (U.w - lo < 32) v &= (1u << (U.w - lo)) - 1u;
            f[j] = v;
        }
        neg = U.yn[k] != 0;
    }
    // digit rule on the unsigned fields: e = f + carry; e >= 2^(w-1) gives
    // the digit e - 2^w and a carry.  Generate: f >= 2^(w-1); propagate:
    // f = 2^(w-1) - 1.
    const int hb = U.w - 1;
    const bool high = (f[hb >> 5] >> (hb & 31)) & 1u;
    bool below_all_ones = true;  // bits 0 .. w-2 all set
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int lo = 32 * j;
        if (lo >= hb) break;
        const int nb = hb - lo < 32 ? hb - lo : 32;
        const uint32_t mask = nb == 32 ? 0xffffffffu : (1u << nb) - 1u;
        if ((f[j] & mask) != mask) below_all_ones = false;
    }
    const uint32_t g = __ballot_sync(0xffffffffu, active && high);
    const uint32_t p = __ballot_sync(0xffffffffu, active && !high && below_all_ones);
    const uint32_t cin = (lookahead(g, p, 0u, nullptr) >> lane) & 1u;
    // e = f + cin (mod 2^w), sign-extended from bit w-1
    uint32_t carry = cin;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t t = f[j] + carry;
        carry = (carry && t == 0u) ? 1u : 0u;
        d[j] = t;
    }
    const bool dneg = (d[hb >> 5] >> (hb & 31)) & 1u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int lo = 32 * j;
        if (lo + 31 <= hb) continue;  // entirely below the sign bit
        const uint32_t keep = hb - lo >= 0 ? (hb - lo == 31 ? 0xffffffffu : (2u << (hb - lo)) - 1u) : 0u;
        d[j] = dneg ? (d[j] | ~keep) : (d[j] & keep);
    }
    if (!active) d[0] = d[1] = d[2] = d[3] = 0u;
    if (neg) {  // the digits of -|C'_k| are the negated digits of |C'_k|
        uint32_t c1 = 1u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = ~d[j] + c1;
            c1 = (c1 && t == 0u) ? 1u : 0u;
            d[j] = t;
        }
    }
}

__global__ void __launch_bounds__(KRON_THREADS) k_kron_unpack(const UnpackArgs U) {
    const int lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * (KRON_THREADS / 32) + (threadIdx.x >> 5);
    if (k > U.n2) return;  // warps for k = 0 .. n2 (the last one holds the top of C'_{n2-1})
    uint32_t dk[4], dp[4];
    digit(U, k, lane, dk);
    digit(U, k - 1, lane, dp);
    // lane t < s: c_{ks+t} = D_{k,t} + D_{k-1,t+s} (lane t+s of the previous
    // coefficient's digits; lane 2s-1 holds zero)
    const int src = lane + U.s < 32 ? lane + U.s : 31;
    uint32_t e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = __shfl_sync(0xffffffffu, dp[j], src);
    const int64_t m = k * U.s + lane;
    if (lane >= U.s || m >= U.nc) return;
    uint32_t v[4], carry = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint64_t t = (uint64_t)dk[j] + e[j] + carry;
        v[j] = (uint32_t)t;
        carry = (uint32_t)(t >> 32);
    }
    const bool neg = (v[3] >> 31) & 1u;
    if (neg) {
        uint32_t c1 = 1u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t t = ~v[j] + c1;
            c1 = (c1 && t == 0u) ? 1u : 0u;
            v[j] = t;
        }
    }
    uint32_t *row = U.c + m * U.lc;
    for (int j = 0; j < U.lc; ++j) row[j] = v[j];
    U.cn[m] = (uint8_t)(neg && (v[0] | v[1] | v[2] | v[3]) != 0u);
}

}  // namespace

int launch_kron_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    const KronPlan &kr = sp.kr;
    const KParams &kp = sp.kp;  // the packed product
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *a2 = kp.Z + kr.off_a, *b2 = kp.Z + kr.off_b, *c2 = kp.Z + kr.off_c;
    uint8_t *an2 = reinterpret_cast<uint8_t *>(kp.Z + kr.off_an);
    uint8_t *bn2 = reinterpret_cast<uint8_t *>(kp.Z + kr.off_bn);
    uint8_t *cn2 = reinterpret_cast<uint8_t *>(kp.Z + kr.off_cn);
    const int wpb = KRON_THREADS / 32;
    PackArgs pa{a, an, kr.na, kr.la, kr.bits_a, a2, an2, kp.na, kp.la, kr.s, kr.w, kp.err};
    k_kron_pack<<<(unsigned)((kp.na + wpb - 1) / wpb), KRON_THREADS, 0, st>>>(pa);
    PackArgs pb{b, bn, kr.nb, kr.lb, kr.bits_b, b2, bn2, kp.nb, kp.lb, kr.s, kr.w, kp.err};
    k_kron_pack<<<(unsigned)((kp.nb + wpb - 1) / wpb), KRON_THREADS, 0, st>>>(pb);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) return -1;
    if (launch_transform_product(sp, a2, an2, b2, bn2, c2, cn2, stream)) return -1;
    UnpackArgs ua{c2, cn2, kp.nc, kp.lc, c, cn, kr.nc, kr.lc, kr.s, kr.w};
    k_kron_unpack<<<(unsigned)((kp.nc + 1 + wpb - 1) / wpb), KRON_THREADS, 0, st>>>(ua);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
