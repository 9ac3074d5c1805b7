// ipm_bigp.cu -- the big-prime form of the method (§3.1, §4's concluding
// remarks): the cyclic and negacyclic convolutions of §2.1 computed modulo
// ONE generalized Fermat prime instead of several machine-word primes and
// Chinese remaindering.
//
// The prime is the first of the paper's table of generalized Fermat primes:
//     p = r^2 + 1,  r = 2^63 + 2^53 = 1025 * 2^53,  p ~ 2^126,  2^106 | p - 1,
// so Z/p has roots of unity of every power-of-two order up to 2^106 and a
// product is exact when p > 4H (§1), H the largest |c_ij|.
//
// Arithmetic in Z/p (elements as integers in [0, p), two 64-bit words).  The
// generalized Fermat form makes reduction a fold: write x = x1 r + x0 with
// 0 <= x0 < r (x1 <= r); since r^2 = -1 (mod p),
//     x y = x0 y0 - x1 y1 + (x0 y1 + x1 y0) r  (mod p),
// and with x0 y1 + x1 y0 = B1 r + B0 (B0 < r) the middle term is
// B0 r - B1: four 64 x 64-bit products, one more split by r and a few
// additions -- no double-length reduction.  Division by r is a shift by 53
// and a division of a 75-bit number by the constant 1025.  r itself is a
// primitive 4th root of unity (multiplication by it: x r = x0 r - x1).
//
// The path (§2): balanced base-2^M digits of |a_i| (the carry rule of
// BivariateRepresentation, negated for negative a_i: any digits with
// |d| <= 2^(M-1) represent the same polynomial), the twist by theta^j
// (theta a primitive 2K-th root) on the negacyclic half, 2-D transforms
// (length K along x on both halves, length Y along y) as radix-2 stages,
// the pointwise product, the inverse transforms, the scale (Y K)^-1, the
// untwist and the halvings c_ij = (c-_ij + c+_ij)/2, c_i,j+K = (c-_ij -
// c+_ij)/2 (§2.2), the centred lift to (-p/2, p/2), and the recombination
// c_i = sum_j c_ij 2^(M j) (one warp per coefficient, exact carries).
// Simple kernels (one radix-2 stage per launch): the variant is for small
// products, as the measured answer to what one big prime costs on this GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "carry.cuh"
#include "ipm_internal.h"

namespace ipm {

typedef unsigned __int128 u128;
typedef __int128 s128;

namespace bp {

constexpr uint64_t R = (1ull << 63) + (1ull << 53);  // 1025 * 2^53
__host__ __device__ constexpr u128 prime() { return (u128)R * R + 1; }

// x = q r + m, 0 <= m < r, for x < 2^128 (q < 2^66)
__host__ __device__ inline void divmod_r(u128 x, u128 &q, uint64_t &m) {
    const u128 t = x >> 53;                    // < 2^75
    const uint64_t hi = (uint64_t)(t >> 32), lo = (uint64_t)t & 0xffffffffu;
    const uint64_t qh = hi / 1025, rh = hi - qh * 1025;
    const uint64_t ql = ((rh << 32) | lo) / 1025;
    q = ((u128)qh << 32) + ql;                 // floor(t / 1025) = floor(x / r)
    m = (uint64_t)(x - q * (u128)R);
}

__host__ __device__ inline u128 reduce_once(u128 x) { return x >= prime() ? x - prime() : x; }
__host__ __device__ inline u128 add(u128 x, u128 y) { return reduce_once(x + y); }
__host__ __device__ inline u128 sub(u128 x, u128 y) { return x >= y ? x - y : x + prime() - y; }

__host__ __device__ inline u128 mul(u128 x, u128 y) {
    u128 x1, y1;
    uint64_t x0, y0;
    divmod_r(x, x1, x0);
    divmod_r(y, y1, y0);
    const uint64_t a1 = (uint64_t)x1, b1 = (uint64_t)y1;  // <= r < 2^64
    const u128 A0 = (u128)x0 * y0, A2 = (u128)a1 * b1;   // < 2^127 each
    const u128 B = (u128)x0 * b1 + (u128)a1 * y0;        // < 2 r (r + 1) < 2^128
    u128 Bq;
    uint64_t B0;
    divmod_r(B, Bq, B0);
    // x y = A0 - A2 + B0 r - Bq (mod p); A0 + B0 r < 2 p, A2 + Bq < p + 2^66
    const u128 T = reduce_once(A0 + (u128)B0 * R);
    const u128 U = reduce_once(A2 + Bq);
    return sub(T, U);
}

__host__ __device__ inline u128 pw(u128 b, u128 e) {
    u128 r = 1;
    while (e) {
        if (e & 1) r = mul(r, b);
        b = mul(b, b);
        e >>= 1;
    }
    return r;
}

// a primitive 2^k-th root of unity: 3 is a quadratic non-residue mod p
inline u128 root(int k) { return pw(3, (prime() - 1) >> k); }
inline u128 inverse(u128 x) { return pw(x, prime() - 2); }

}  // namespace bp

namespace {

__device__ __forceinline__ u128 ld(const u128 *p) { return *p; }

// Balanced digits of |x_i| (base 2^M, K digits), negated for negative x_i;
// row i, columns [0, K): d_ij mod p; [K, 2K): theta^j d_ij.  One thread per
// coefficient; rows >= n are left as set by the caller (zero).
__global__ void k_bp_split(const uint32_t *__restrict__ x, const uint8_t *__restrict__ xn, int64_t n, int L,
                           uint32_t bits, int K, int M, const u128 *__restrict__ theta, u128 *__restrict__ X,
                           int *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t *row = x + (size_t)i * L;
        if ((bits & 31u) && (row[L - 1] >> (bits & 31u))) atomicOr(err, ERRBIT_BOUND);
        const bool neg = xn[i] != 0;
        const uint64_t mmask = M == 64 ? ~0ull : (1ull << M) - 1, half = 1ull << (M - 1);
        u128 *out = X + (size_t)i * 2 * K;
        uint64_t carry = 0;
        for (int j = 0; j < K; ++j) {
            const int64_t bit = (int64_t)M * j;
            const int l0 = (int)(bit >> 5), sh = (int)(bit & 31);
            u128 w = 0;
            for (int k = 0; k < 4; ++k)
                if (l0 + k < L) w |= (u128)row[l0 + k] << (32 * k);
            const uint64_t u = (uint64_t)(w >> sh) & mmask;
            const u128 t = (u128)u + carry;
            s128 d;
            if (j < K - 1) {
                carry = t >= half ? 1 : 0;
                d = carry ? (s128)t - ((s128)1 << M) : (s128)t;
            } else {
                d = (s128)t;  // the top digit absorbs the carry (|d| <= 2^(M-1))
            }
            if (neg) d = -d;
            const u128 v = d < 0 ? bp::prime() - (u128)(-d) : (u128)d;
            out[j] = v;
            out[K + j] = bp::mul(v, ld(theta + j));
        }
    }
}

// One radix-2 stage on every transform: transform t starts at
// (t % tm) ta + (t / tm) tb, element n at + n es; length 2^logL; butterflies
// at distance h; tw = omega_L^e (e < L/2) or its inverse.  forward: DIF
// (x + y, (x - y) w), natural in, bit-reversed out; else DIT (x + y w,
// x - y w), bit-reversed in, natural out.
__global__ void k_bp_stage(u128 *__restrict__ X, int64_t nt, int64_t tm, int64_t ta, int64_t tb, int64_t es,
                           int logL, int64_t h, const u128 *__restrict__ tw, int forward) {
    const int64_t per = (int64_t)1 << (logL - 1);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nt * per;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = g / per, b = g - t * per;
        const int64_t j = b % h, blk = b / h;
        u128 *base = X + (t % tm) * ta + (t / tm) * tb;
        u128 *px = base + (blk * 2 * h + j) * es, *py = px + h * es;
        const u128 w = ld(tw + j * (per / h));  // omega_L^(j L / 2h)
        const u128 x = *px, y = *py;
        if (forward) {
            *px = bp::add(x, y);
            *py = bp::mul(bp::sub(x, y), w);
        } else {
            const u128 yw = bp::mul(y, w);
            *px = bp::add(x, yw);
            *py = bp::sub(x, yw);
        }
    }
}

__global__ void k_bp_pointwise(u128 *__restrict__ A, const u128 *__restrict__ B, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        A[e] = bp::mul(A[e], B[e]);
}

// Rows i < nc: scale, untwist and the halvings of §2.2 (in place).
__global__ void k_bp_recover(u128 *__restrict__ X, int64_t nc, int K, const u128 *__restrict__ untw, u128 scale,
                             u128 half) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * K;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / K;
        const int j = (int)(e - i * K);
        u128 *row = X + (size_t)i * 2 * K;
        const u128 u = bp::mul(row[j], scale);        // c-_ij
        const u128 v = bp::mul(row[K + j], untw[j]);  // c+_ij (untw = scale theta^-j)
        row[j] = bp::mul(bp::add(u, v), half);
        row[K + j] = bp::mul(bp::sub(u, v), half);
    }
}

// Centred lift of residue v: v - p when 2 v > p.
__device__ __forceinline__ s128 lift(u128 v) { return v > (bp::prime() >> 1) ? (s128)v - (s128)bp::prime() : (s128)v; }

// c_i = sum_(j < 2K) c_ij 2^(M j), one warp per coefficient.  Term j
// starts at limb Q_j = floor(M j / 32); shifted left by M j mod 32 it
// spans five words of which the lower four are unsigned and the fifth is
// the signed top word; limb q sums the words landing on it.
__global__ void k_bp_recombine(const u128 *__restrict__ X, int64_t nc, int K, int M, uint32_t *__restrict__ c,
                               uint8_t *__restrict__ cn, int lc, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int twoK = 2 * K;
    for (int64_t i = warp; i < nc; i += nwarps) {
        const u128 *row = X + (size_t)i * twoK;
        auto column = [&](int q) {
            int64_t P = 0;
            const int jlo = q >= 4 ? (32 * (q - 4) + M - 1) / M : 0;  // Q_j >= q - 4
            int jhi = (32 * q + 31) / M;                               // Q_j <= q
            if (jhi > twoK - 1) jhi = twoK - 1;
            for (int j = jlo; j <= jhi; ++j) {
                const int64_t bit = (int64_t)M * j;
                const int Q = (int)(bit >> 5), sh = (int)(bit & 31), k = q - Q;
                if (k < 0 || k > 4) continue;
                const s128 v = lift(row[j]);
                const uint32_t w[5] = {(uint32_t)v, (uint32_t)((u128)v >> 32), (uint32_t)((u128)v >> 64),
                                       (uint32_t)((u128)v >> 96), v < 0 ? 0xffffffffu : 0u};
                const uint32_t lo = k > 0 ? w[k - 1] : 0u;
                const uint32_t word = sh ? __funnelshift_l(lo, w[k], sh) : w[k];
                P += k < 4 ? (int64_t)word : (int64_t)(int32_t)word;
            }
            return P;
        };
        if (!warp_sum_to_sign_magnitude(column, lc + 5, c + (size_t)i * lc, cn + i, lc) && lane == 0)
            atomicOr(err, ERRBIT_INTERNAL);
    }
}

}  // namespace

// Tables of a plan (host): theta^j and scale theta^-j (j < K), omega_K^(+-e)
// (e < K/2, omega_K = theta^2), omega_Y^(+-e) (e < Y/2), as 128-bit words
// (two 64-bit words, low first) in the order of BigpPlan's offsets; also
// the scalars.
void bigp_tables(BigpPlan &b, std::vector<uint64_t> &words) {
    std::vector<u128> out;
    const int K = b.K;
    const int64_t Y = b.Y;
    const u128 theta = bp::root(b.logK + 1);
    const u128 theta_i = bp::inverse(theta);
    const u128 wK = bp::mul(theta, theta), wK_i = bp::mul(theta_i, theta_i);
    const u128 wY = bp::root(b.logY), wY_i = bp::inverse(wY);
    const u128 scale = bp::inverse(bp::mul((u128)Y % bp::prime(), (u128)K));
    b.scale_lo = (uint64_t)scale;
    b.scale_hi = (uint64_t)(scale >> 64);
    const u128 half = (bp::prime() + 1) / 2;
    b.half_lo = (uint64_t)half;
    b.half_hi = (uint64_t)(half >> 64);
    out.assign(b.table_entries, 0);
    u128 t = 1, ti = scale;
    for (int j = 0; j < K; ++j) {
        out[b.tab_theta + j] = t;
        out[b.tab_untw + j] = ti;
        t = bp::mul(t, theta);
        ti = bp::mul(ti, theta_i);
    }
    u128 f = 1, fi = 1;
    for (int e = 0; e < K / 2; ++e) {
        out[b.tab_wk + e] = f;
        out[b.tab_wk_i + e] = fi;
        f = bp::mul(f, wK);
        fi = bp::mul(fi, wK_i);
    }
    f = 1;
    fi = 1;
    for (int64_t e = 0; e < Y / 2; ++e) {
        out[b.tab_wy + e] = f;
        out[b.tab_wy_i + e] = fi;
        f = bp::mul(f, wY);
        fi = bp::mul(fi, wY_i);
    }
    words.resize(2 * out.size());
    for (size_t e = 0; e < out.size(); ++e) {
        words[2 * e] = (uint64_t)out[e];
        words[2 * e + 1] = (uint64_t)(out[e] >> 64);
    }
}

// Does 4 H < p hold, H = min(na, nb) K 2^(2M - 2)?
bool bigp_bound_ok(int64_t mn, int K, int M) {
    // 4H = mn K 2^(2M): compare bit lengths first, then exactly
    const int bits_mnK = 64 - __builtin_clzll((unsigned long long)((uint64_t)mn * (uint64_t)K));
    if (bits_mnK + 2 * M > 127) return false;
    const u128 four_h = (u128)((uint64_t)mn * (uint64_t)K) << (2 * M);
    return four_h < bp::prime();
}

namespace {

unsigned grid_for(int64_t n, int per_block = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, 152 * 16));
}

int run_stages(u128 *X, int64_t nt, int64_t tm, int64_t ta, int64_t tb, int64_t es, int logL, const u128 *tw,
               bool forward, cudaStream_t s) {
    if (logL < 1) return 0;
    const int64_t L = (int64_t)1 << logL;
    for (int i = 0; i < logL; ++i) {
        const int64_t h = forward ? L >> (i + 1) : (int64_t)1 << i;
        k_bp_stage<<<grid_for(nt * (L / 2)), 256, 0, s>>>(X, nt, tm, ta, tb, es, logL, h, tw, forward ? 1 : 0);
        note_launches(1);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

}  // namespace

int launch_bigp_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const BigpPlan &P = sp.bp;
    int *err = sp.kp.err;
    u128 *base = reinterpret_cast<u128 *>(sp.kp.Z);  // 16-byte aligned
    u128 *XA = base + P.off_xa, *XB = base + P.off_xb;
    const u128 *tab = reinterpret_cast<const u128 *>(P.dtab);  // built by the plan (bigp_tables)
    const int64_t n = P.Y * 2 * P.K;
    if (cudaMemsetAsync(XA, 0, (size_t)n * sizeof(u128), s) != cudaSuccess) return -1;
    if (cudaMemsetAsync(XB, 0, (size_t)n * sizeof(u128), s) != cudaSuccess) return -1;
    k_bp_split<<<grid_for(P.na), 256, 0, s>>>(a, an, P.na, P.la, P.bits_a, P.K, P.M, tab + P.tab_theta, XA, err);
    k_bp_split<<<grid_for(P.nb), 256, 0, s>>>(b, bn, P.nb, P.lb, P.bits_b, P.K, P.M, tab + P.tab_theta, XB, err);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) return -1;
    const int64_t twoK = 2 * P.K;
    for (u128 *X : {XA, XB}) {
        if (run_stages(X, 2 * P.Y, 2, P.K, twoK, 1, P.logK, tab + P.tab_wk, true, s)) return -1;     // x
        if (run_stages(X, twoK, twoK, 1, 0, twoK, P.logY, tab + P.tab_wy, true, s)) return -1;       // y
    }
    k_bp_pointwise<<<grid_for(n), 256, 0, s>>>(XA, XB, n);
    note_launches(1);
    if (run_stages(XA, twoK, twoK, 1, 0, twoK, P.logY, tab + P.tab_wy_i, false, s)) return -1;
    if (run_stages(XA, 2 * P.Y, 2, P.K, twoK, 1, P.logK, tab + P.tab_wk_i, false, s)) return -1;
    const u128 scale = ((u128)P.scale_hi << 64) | P.scale_lo, half = ((u128)P.half_hi << 64) | P.half_lo;
    k_bp_recover<<<grid_for(P.nc * P.K), 256, 0, s>>>(XA, P.nc, P.K, tab + P.tab_untw, scale, half);
    k_bp_recombine<<<grid_for(P.nc * 32), 256, 0, s>>>(XA, P.nc, P.K, P.M, c, cn, P.lc, err);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
