// ipm_ks.cu -- Kronecker substitution (KS) on the GPU: the polynomial
// product read off one integer product, the comparison method KS_s of §1
// and §4 (there with GMP's integer multiplication), here with the
// integer product done by this library's own transform path.
//
//   A = a(2^s) = sum_t a_t 2^(s t),  B = b(2^s),  C = A B = sum_t c_t 2^(s t)
//
// Slots of s = 32 w bits with w = Lc + 3 limbs, Lc the output stride
// (|c_t| < 2^(32 Lc)).  Because every a_t has its own slot and the upper
// limbs of a slot are zero, A written limb by limb is a sequence of signed
// 32-bit digits d_k = +-(limb k mod w of a_(k/w)): A = sum_k d_k 2^(32 k),
// which is a polynomial with 32-bit sign-magnitude coefficients in the
// library's own operand format (k_ks_pack, a gather).  Its product with
// B's digit polynomial, D(z) = sum_k e_k z^k with |e_k| < min(nA, nB) 2^64
// (three limbs), is the integer C evaluated at z = 2^32 before carrying.
//
// Unpacking (no carry chain across slots): let V_t = sum_(j<w) e_(wt+j)
// 2^(32 j) (the part of the sum that starts in slot t), L_t = V_t mod 2^s
// and H_t = floor(V_t / 2^s) (|H_t| < 2^62).  Then C = sum_t (L_t +
// H_(t-1)) 2^(s t), and with g_t the borrow into slot t,
//     c_t = L_t + H_(t-1) + g_t - 2^s g_(t+1).
// |c_t| < 2^(32 Lc) = 2^(s - 96) and |H_(t-1) + g_t| < 2^63 place
// L_t + H_(t-1) + g_t within 2^(s-2) of 0 or of 2^s, so g_(t+1) is the top
// bit of L_t (bit s-1 of V_t): every slot is decided from V_t and V_(t-1)
// alone.  k_ks_slots computes (L_t, H_t, g_(t+1)) for every slot, one warp
// each; k_ks_unpack forms c_t and converts it to sign-magnitude, one warp
// each, and checks that the slot past the last coefficient is zero.
#include <cuda_runtime.h>

#include <algorithm>

#include "carry.cuh"
#include "ipm_internal.h"

namespace ipm {

namespace {

// Signed value of limb l of product digit k (le limbs each, sign byte).
__device__ __forceinline__ int64_t signed_limb(const uint32_t *e, const uint8_t *en, int le, int64_t k, int l) {
    const int64_t v = (int64_t)e[(size_t)k * le + l];
    return en[k] ? -v : v;
}

}  // namespace

// Digit polynomial of one operand: coefficient k = limb (k mod w) of
// x_(k / w) with x's sign (0 for k mod w >= L).  Also reports inputs above
// their bit bound.
__global__ void k_ks_pack(const uint32_t *__restrict__ x, const uint8_t *__restrict__ xn, int64_t n, int L,
                          uint32_t bits, int w, uint32_t *__restrict__ d, uint8_t *__restrict__ dn, int *err) {
    const int64_t total = n * (int64_t)w;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / w;
        const int j = (int)(k - i * w);
        uint32_t v = 0;
        if (j < L) {
            v = x[(size_t)i * L + j];
            if (j == L - 1 && (bits & 31u) && (v >> (bits & 31u))) atomicOr(err, ERRBIT_BOUND);
        }
        d[k] = v;
        dn[k] = (j < L && v) ? xn[i] : 0;
    }
}

// One warp per slot t <= nc: V_t from the product digits e_(wt .. wt+w-1)
// (ne of them in all, le <= 3 limbs each), then L_t (w limbs) to Lbuf, H_t
// to Hbuf and the top bit of L_t to gbuf.
__global__ void k_ks_slots(const uint32_t *__restrict__ e, const uint8_t *__restrict__ en, int64_t ne, int le, int w,
                           int64_t nslots, uint32_t *__restrict__ Lbuf, int64_t *__restrict__ Hbuf,
                           uint8_t *__restrict__ gbuf) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < nslots; t += nwarps) {
        const int64_t k0 = t * w;
        CarryState st;
        uint32_t hl[3] = {0u, 0u, 0u};  // limbs w, w+1, w+2 of V_t
        uint32_t top = 0;               // limb w-1
        for (int q0 = 0; q0 < w + 3; q0 += 32) {
            const int q = q0 + lane;
            const bool act = q < w + 3;
            int64_t P = 0;
            if (act) {
                for (int l = 0; l < le; ++l) {
                    const int j = q - l;  // digit e_(k0 + j) contributes its limb l
                    if (j >= 0 && j < w && k0 + j < ne) P += signed_limb(e, en, le, k0 + j, l);
                }
            }
            const uint32_t v = carry_chunk(P, act, st);
            if (q < w) Lbuf[(size_t)t * w + q] = v;
            if (q == w - 1) top = v;
            for (int l = 0; l < 3; ++l)
                if (q == w + l) hl[l] = v;
        }
        // gather the lanes' pieces (each written by exactly one lane)
        top = __reduce_or_sync(0xffffffffu, top);
        for (int l = 0; l < 3; ++l) hl[l] = __reduce_or_sync(0xffffffffu, hl[l]);
        if (lane == 0) {
            Hbuf[t] = (int64_t)(((uint64_t)hl[1] << 32) | hl[0]);  // |H_t| < 2^62: limb w+2 is the sign
            gbuf[t] = (uint8_t)(top >> 31);
        }
    }
}

// One warp per output coefficient t < nc (and the check slot t = nc):
// c_t = L_t + H_(t-1) + g_t - 2^s g_(t+1), to sign-magnitude in lc limbs.
__global__ void k_ks_unpack(const uint32_t *__restrict__ Lbuf, const int64_t *__restrict__ Hbuf,
                            const uint8_t *__restrict__ gbuf, int w, int64_t nc, int lc, uint32_t *__restrict__ c,
                            uint8_t *__restrict__ cn, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t <= nc; t += nwarps) {
        // D = H_(t-1) + g_t, the part of slot t that comes from below
        const int64_t D = t > 0 ? Hbuf[t - 1] + (int64_t)gbuf[t - 1] : 0;
        const uint32_t gnext = gbuf[t];  // g_(t+1) = top bit of L_t
        CarryState st;
        uint32_t sign_word = 0;
        int first_nz = -1;
        // limbs lc .. w (limb w: the carries out of the slot minus g_(t+1))
        // must all be 0 or all be ones: the sign extension of a value that
        // fits lc limbs
        bool all_zero = true, all_ones = true;
        uint32_t *crow = t < nc ? c + (size_t)t * lc : nullptr;
        for (int q0 = 0; q0 <= w; q0 += 32) {
            const int q = q0 + lane;
            const bool act = q <= w;
            int64_t P = 0;
            if (act) {
                if (q < w) P = (int64_t)Lbuf[(size_t)t * w + q];
                if (q == 0) P += (int64_t)(uint32_t)D;
                if (q == 1) P += D >> 32;
                if (q == w) P -= (int64_t)gnext;
            }
            const uint32_t v = carry_chunk(P, act, st);
            if (q == w) sign_word = v;
            if (crow && q < lc) crow[q] = v;
            if (act && q >= lc) {
                all_zero = all_zero && v == 0u;
                all_ones = all_ones && v == 0xffffffffu;
            }
            const unsigned nz = __ballot_sync(0xffffffffu, act && q < lc && v != 0u);
            if (nz && first_nz < 0) first_nz = q0 + __ffs(nz) - 1;
        }
        sign_word = __reduce_or_sync(0xffffffffu, sign_word);
        const bool negative = sign_word == 0xffffffffu;
        const bool ext_ok = __all_sync(0xffffffffu, negative ? all_ones : all_zero);
        if (t == nc) {  // the slot past the last coefficient must be zero
            if (lane == 0 && (sign_word != 0u || first_nz >= 0 || !ext_ok)) atomicOr(err, ERRBIT_INTERNAL);
            continue;
        }
        if (lane == 0) {
            if (!ext_ok) atomicOr(err, ERRBIT_INTERNAL);
            cn[t] = (negative && first_nz >= 0) ? 1 : 0;
        }
        if (negative && first_nz >= 0) {
            __syncwarp();
            for (int q = first_nz + lane; q < lc; q += 32) {
                const uint32_t v = crow[q];
                crow[q] = q == first_nz ? 0u - v : ~v;
            }
        }
    }
}

int launch_ks_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                      const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const KsPlan &k = sp.ks;
    const KParams &kp = sp.kp;  // the digit product
    uint32_t *Z = kp.Z;
    uint32_t *da = Z + k.off_a, *db = Z + k.off_b, *de = Z + k.off_c;
    uint8_t *dan = reinterpret_cast<uint8_t *>(Z + k.off_an), *dbn = reinterpret_cast<uint8_t *>(Z + k.off_bn);
    uint8_t *den = reinterpret_cast<uint8_t *>(Z + k.off_cn);
    uint32_t *Lbuf = Z + k.off_L;
    int64_t *Hbuf = reinterpret_cast<int64_t *>(Z + k.off_H);
    uint8_t *gbuf = reinterpret_cast<uint8_t *>(Z + k.off_g);
    const unsigned pb = 1216, pt = 256;
    k_ks_pack<<<pb, pt, 0, s>>>(a, an, k.na, k.la, k.bits_a, k.w, da, dan, kp.err);
    k_ks_pack<<<pb, pt, 0, s>>>(b, bn, k.nb, k.lb, k.bits_b, k.w, db, dbn, kp.err);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) return -1;
    if (launch_transform_product(sp, da, dan, db, dbn, de, den, stream)) return -1;
    const int64_t nslots = k.nc + 1;
    const unsigned wb = (unsigned)std::min<int64_t>((nslots + 7) / 8, 1216 * 8);
    k_ks_slots<<<wb, 256, 0, s>>>(de, den, kp.nc, kp.lc, k.w, nslots, Lbuf, Hbuf, gbuf);
    k_ks_unpack<<<wb, 256, 0, s>>>(Lbuf, Hbuf, gbuf, k.w, k.nc, k.lc, c, cn, kp.err);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
