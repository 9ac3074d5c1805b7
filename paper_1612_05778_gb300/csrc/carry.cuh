// carry.cuh -- warp-wide carry propagation of signed multi-limb sums
// (Kronecker-substitution unpacking, Karatsuba evaluation and combination).
#pragma once
#include <stdint.h>

namespace ipm {

// Warp-wide carrying of a signed multi-limb sum, 32 limbs per call, low
// chunks first.  Lane value P (|P| < 2^40) is the contribution to limb
// q = q0 + lane of X = sum_q P_q 2^(32 q).  Writing P_q = t_q + 2^32 h_q,
// adding h_(q-1) to t_q leaves t'_q + 2^32 g_q with g_q in {-1, 0, 1};
// the +1 and -1 carries one limb up are then resolved as an addition and
// a subtraction by ballot carry-lookahead (33-bit integer addition of the
// generate and propagate masks).  Returns limb q of X modulo 2^(32 n), two's
// complement; `state` carries (h, g, carry, borrow) between chunks.
struct CarryState {
    int h = 0, g = 0;
    unsigned cplus = 0, cminus = 0;
};

__device__ __forceinline__ unsigned carry_lookahead(unsigned gen, unsigned prop, unsigned *cio) {
    const uint64_t s = (uint64_t)gen + (uint64_t)(gen | prop) + *cio;
    *cio = (unsigned)(s >> 32);
    return (unsigned)s ^ prop;
}

__device__ __forceinline__ uint32_t carry_chunk(int64_t P, bool act, CarryState &st) {
    const int lane = threadIdx.x & 31;
    const int h = act ? (int)(P >> 32) : 0;
    int hprev = __shfl_up_sync(0xffffffffu, h, 1);
    if (lane == 0) hprev = st.h;
    const int64_t sum = (act ? (int64_t)(uint32_t)P : 0) + hprev;
    const uint32_t tq = (uint32_t)sum;
    const int g = (int)(sum >> 32);
    int gprev = __shfl_up_sync(0xffffffffu, g, 1);
    if (lane == 0) gprev = st.g;
    st.h = __shfl_sync(0xffffffffu, h, 31);
    st.g = __shfl_sync(0xffffffffu, g, 31);
    const uint32_t gp = gprev == 1 ? 1u : 0u;
    const unsigned cm = carry_lookahead(__ballot_sync(0xffffffffu, gp && tq == 0xffffffffu),
                                     __ballot_sync(0xffffffffu, tq + gp == 0xffffffffu), &st.cplus);
    const uint32_t u = tq + gp + ((cm >> lane) & 1u);
    const uint32_t gm = gprev == -1 ? 1u : 0u;
    const unsigned bm = carry_lookahead(__ballot_sync(0xffffffffu, gm && u == 0u),
                                     __ballot_sync(0xffffffffu, u == gm), &st.cminus);
    return u - gm - ((bm >> lane) & 1u);
}

// One warp writes X = sum_q P(q) 2^(32 q) (P(q): the signed column sum of
// limb q, |P(q)| < 2^40, zero for q > hi) in sign-magnitude form with lo
// limbs; hi >= lo is a limb that holds X's sign.  Returns false when |X|
// is not below 2^(32 lo): limbs lo .. hi must all be that sign, and the
// low limbs not all zero when it is negative.  lo = 0 checks X = 0.
template <class ColumnSum>
__device__ __forceinline__ bool warp_sum_to_sign_magnitude(const ColumnSum &P, int hi, uint32_t *out,
                                                           uint8_t *out_neg, int lo) {
    const int lane = threadIdx.x & 31;
    CarryState st;
    uint32_t sign_word = 0;
    int first_nz = -1;
    bool all_zero = true, all_ones = true;
    for (int q0 = 0; q0 <= hi; q0 += 32) {
        const int q = q0 + lane;
        const bool act = q <= hi;
        const uint32_t v = carry_chunk(act ? P(q) : 0, act, st);
        if (q < lo) out[q] = v;
        if (q == hi) sign_word = v;
        if (act && q >= lo) {
            all_zero = all_zero && v == 0u;
            all_ones = all_ones && v == 0xffffffffu;
        }
        const unsigned nz = __ballot_sync(0xffffffffu, act && q < lo && v != 0u);
        if (nz && first_nz < 0) first_nz = q0 + __ffs(nz) - 1;
    }
    sign_word = __reduce_or_sync(0xffffffffu, sign_word);
    const bool negative = sign_word == 0xffffffffu;
    // -2^(32 lo) would read as all-zero limbs with a negative sign: too large
    const bool ok = __all_sync(0xffffffffu, negative ? all_ones : all_zero) && !(negative && first_nz < 0);
    if (lane == 0 && lo > 0) *out_neg = (negative && first_nz >= 0) ? 1 : 0;
    if (negative && first_nz >= 0) {  // magnitude: zero below f, -x at f, ~x above
        __syncwarp();
        for (int q = first_nz + lane; q < lo; q += 32) {
            const uint32_t v = out[q];
            out[q] = q == first_nz ? 0u - v : ~v;
        }
    }
    __syncwarp();
    return ok;
}

// The same for a sum of nt signed terms (term i: li[i] magnitude limbs at
// x[i], negative when neg[i]); at most 16 terms, so the sign is settled by
// limb max(lo, max li + 1).
__device__ __forceinline__ bool warp_signed_sum(const uint32_t *const *x, const int *li, const uint8_t *neg, int nt,
                                                uint32_t *out, uint8_t *out_neg, int lo) {
    int hi = lo;
    for (int i = 0; i < nt; ++i) hi = max(hi, li[i] + 1);
    auto column = [&](int q) {
        int64_t P = 0;
        for (int i = 0; i < nt; ++i)
            if (q < li[i]) {
                const int64_t v = (int64_t)x[i][q];
                P += neg[i] ? -v : v;
            }
        return P;
    };
    return warp_sum_to_sign_magnitude(column, hi, out, out_neg, lo);
}

}  // namespace ipm
