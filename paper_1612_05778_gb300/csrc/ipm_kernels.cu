// ipm_kernels.cu -- the three passes of one product c = a*b.
//
// Index conventions.  y-transform length Y = Y1*Y2 >= nc; a y index is
// i = i1 + Y1*i2 (i1 < Y1, i2 < Y2).  The forward y transform is the
// four-step split of a length-Y DFT: a length-Y2 DFT over i2 for every i1
// (step A), the twiddle omega_Y^{i1*k2} (step B), then a length-Y1 DFT over
// i1 for every k2 (step C).  x runs over 2K columns: columns [0, K) carry
// the cyclic convolution (C^-, mod x^K - 1) and [K, 2K) the negacyclic one
// (C^+, mod x^K + 1) after the twist x -> theta x (§2.1).
//
//  k_forward  (grid Y1 x 2 operands): split into balanced digits (§2,
//             BivariateRepresentation), residues mod p_t, twist, x-DFT of
//             both halves, y step A + step B; writes Z[t][op][k2][i1][2K].
//  k_middle   (grid 2K/S x Y2 x r): y step C for A and B, pointwise
//             product, inverse step C; writes the product back over A.
//  k_inverse  (grid Y1): inverse step B + A, inverse x-DFTs, untwist and
//             the halvings c_{i,j} = (c^- + c^+)/2, c_{i,j+K} = (c^- - c^+)/2
//             (§2.2 step 3 per digit), CRT over the primes (§4), then
//             c_i = sum_j c_{i,j} 2^{Mj} with full carry propagation and
//             conversion to sign-magnitude.
#include <cuda_runtime.h>
#include <atomic>

#include "ipm_internal.h"
#include "modarith.cuh"

namespace ipm {

static std::atomic<int64_t> g_launches{0};
int64_t launches_so_far() { return g_launches.load(); }

// ---------------------------------------------------------------------------
// Pass 1
// ---------------------------------------------------------------------------

// Limb l of the N-bit two's complement of a sign-magnitude coefficient
// (row: L magnitude limbs; f: index of its lowest non-zero limb).
__device__ __forceinline__ uint32_t twos_limb(const uint32_t *__restrict__ row, int L, bool neg,
                                              int f, int l) {
    const uint32_t v = l < L ? __ldg(row + l) : 0u;
    if (!neg) return v;
    if (l < f) return 0u;
    return l == f ? 0u - v : ~v;
}

__global__ void __launch_bounds__(THREADS_FWD)
k_forward(const __grid_constant__ KParams P, const uint32_t *__restrict__ a,
          const uint8_t *__restrict__ an, const uint32_t *__restrict__ b,
          const uint8_t *__restrict__ bn) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int op = blockIdx.y;
    const int64_t i1 = blockIdx.x;
    const uint32_t *X = op ? b : a;
    const uint8_t *Xn = op ? bn : an;
    const int64_t nX = op ? P.nb : P.na;
    const int L = op ? P.lb : P.la;
    const uint32_t bits = op ? P.bits_b : P.bits_a;
    const int K = P.K, logK = P.logK, M = P.M;
    const int Y2 = (int)P.Y2;
    const int twoK = 2 * K;
    int64_t *dig = reinterpret_cast<int64_t *>(smem);            // [Y2][K]
    uint32_t *tile = reinterpret_cast<uint32_t *>(dig + (size_t)Y2 * K);  // [Y2][2K]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint64_t mmask = (1ull << M) - 1;
    const uint64_t halfM = 1ull << (M - 1);

    // 1. Balanced base-2^M digits of every row (one warp per row).  Digits
    //    j < K-1 follow the carry rule t = u_j + carry, digit = t - 2^M and
    //    carry 1 when t >= 2^(M-1); the top digit is the signed top field
    //    plus the carry.  The carry chain is resolved with ballots: with
    //    generate g_j = [u_j >= 2^(M-1)] and propagate q_j = [u_j = 2^(M-1)-1]
    //    the carries into every digit are (g + (g|q)) xor q (carry-lookahead
    //    by integer addition), 32 digits per ballot word.
    for (int i2 = warp; i2 < Y2; i2 += nw) {
        const int64_t i = i1 + P.Y1 * (int64_t)i2;
        int64_t *drow = dig + (size_t)i2 * K;
        if (i >= nX) {
            for (int j = lane; j < K; j += 32) drow[j] = 0;
            continue;
        }
        const uint32_t *row = X + (size_t)i * L;
        int f = L;
        for (int c0 = 0; c0 < L; c0 += 32) {
            const int l = c0 + lane;
            const uint32_t v = l < L ? __ldg(row + l) : 0u;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0u);
            if (m && f == L) f = c0 + __ffs(m) - 1;
        }
        if (lane == 0 && (bits & 31u) && (__ldg(row + L - 1) >> (bits & 31u)))
            atomicOr(P.err, ERRBIT_BOUND);
        const bool neg = Xn[i] != 0 && f < L;
        unsigned carry_in = 0;
        for (int j0 = 0; j0 < K; j0 += 32) {
            const int j = j0 + lane;
            uint64_t u = 0;
            if (j < K) {
                const int64_t bit = (int64_t)M * j;
                const int l0 = (int)(bit >> 5), sh = (int)(bit & 31);
                const uint64_t lo = (uint64_t)twos_limb(row, L, neg, f, l0) |
                                    ((uint64_t)twos_limb(row, L, neg, f, l0 + 1) << 32);
                uint64_t v = lo;
                if (sh) v = (lo >> sh) | ((uint64_t)twos_limb(row, L, neg, f, l0 + 2) << (64 - sh));
                u = v & mmask;
            }
            const bool inner = j < K - 1;
            const unsigned g = __ballot_sync(0xffffffffu, inner && u >= halfM);
            const unsigned q = __ballot_sync(0xffffffffu, inner && u == halfM - 1);
            const uint64_t s = (uint64_t)g + (uint64_t)(g | q) + carry_in;
            const unsigned cm = (unsigned)s ^ q;
            carry_in = (unsigned)(s >> 32);
            if (j < K) {
                const uint64_t c = (cm >> lane) & 1u;
                int64_t d;
                if (inner) {
                    const uint64_t t = u + c;
                    d = t >= halfM ? (int64_t)t - (int64_t)(1ull << M) : (int64_t)t;
                } else {
                    d = (u >= halfM ? (int64_t)u - (int64_t)(1ull << M) : (int64_t)u) + (int64_t)c;
                }
                drow[j] = d;
            }
        }
    }
    __syncthreads();

    const int64_t Y1 = P.Y1;
    for (int t = 0; t < P.r; ++t) {
        const PrimeConst &pc = P.pc[t];
        const uint32_t p = pc.p, p2 = pc.p2;
        const uint2 one = make_uint2(1u, pc.one_s), c32 = make_uint2(pc.c32, pc.c32_s);
        // 2. residues (cyclic half) and twisted residues theta^j a_ij (negacyclic half)
        for (int e = threadIdx.x; e < Y2 * K; e += blockDim.x) {
            const int i2 = e >> logK, j = e & (K - 1);
            const int64_t d = dig[e];
            const uint64_t ad = d < 0 ? (uint64_t)(-d) : (uint64_t)d;
            uint32_t r = shoup((uint32_t)(ad >> 32), c32, p) + shoup((uint32_t)ad, one, p);
            r = red(red(r, p2), p);
            if (d < 0 && r) r = p - r;
            uint32_t *trow = tile + (size_t)i2 * twoK;
            trow[j] = r;
            trow[K + j] = shoup(r, pc.tx_f[j], p);
        }
        __syncthreads();
        // 3. x-DFTs of length K on both halves of every row (omega_K = theta^2)
        dif_rows(tile, 2 * Y2, K, logK, pc.tx_f, logK + 1, p, p2);
        // 4. y step A: length-Y2 DFT down every column
        dif_cols(tile, logK + 1, twoK, P.logY2, pc.ty_f, P.logY, p, p2);
        // 5. step B twiddle, full reduction, store rows (k2, i1)
        uint32_t *Zt = P.Z + (size_t)(t * 2 + op) * (size_t)P.Y * twoK;
        for (int e = threadIdx.x; e < Y2 * twoK; e += blockDim.x) {
            const int pos = e >> (logK + 1), col = e & (twoK - 1);
            const uint32_t k2 = bitrev((uint32_t)pos, P.logY2);
            const uint2 w = pc.ty_f[(size_t)i1 * k2];
            const uint32_t v = red(shoup(tile[e], w, p), p);
            Zt[((size_t)pos * Y1 + i1) * twoK + col] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Pass 2
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(THREADS_MID) k_middle(const __grid_constant__ KParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int cs = blockIdx.x, pos = blockIdx.y, t = blockIdx.z;
    const int S = P.S, logS = P.logS;
    const int twoK = 2 * P.K;
    const int Y1 = (int)P.Y1;
    uint32_t *A = reinterpret_cast<uint32_t *>(smem);  // [Y1][S]
    uint32_t *B = A + (size_t)Y1 * S;                   // [Y1][S]
    const PrimeConst &pc = P.pc[t];
    const uint32_t p = pc.p, p2 = pc.p2;
    uint32_t *ZA = P.Z + (size_t)(t * 2 + 0) * (size_t)P.Y * twoK;
    const uint32_t *ZB = P.Z + (size_t)(t * 2 + 1) * (size_t)P.Y * twoK;
    const size_t base = (size_t)pos * Y1 * twoK + (size_t)cs * S;
    for (int e = threadIdx.x; e < Y1 * S; e += blockDim.x) {
        const int i1 = e >> logS, c = e & (S - 1);
        const size_t g = base + (size_t)i1 * twoK + c;
        A[e] = ZA[g];
        B[e] = ZB[g];
    }
    __syncthreads();
    // y step C (omega_Y1 = omega_Y^Y2) on A and B
    dif_cols(A, logS, S, P.logY1, pc.ty_f, P.logY, p, p2);
    dif_cols(B, logS, S, P.logY1, pc.ty_f, P.logY, p, p2);
    // pointwise product in Montgomery form: A*B*2^-32 (the 2^32 is put back
    // by the scale factor of the inverse pass)
    for (int e = threadIdx.x; e < Y1 * S; e += blockDim.x) A[e] = montmul(A[e], B[e], p, pc.mont);
    __syncthreads();
    dit_cols(A, logS, S, P.logY1, pc.ty_i, P.logY, p, p2);
    for (int e = threadIdx.x; e < Y1 * S; e += blockDim.x) {
        const int i1 = e >> logS, c = e & (S - 1);
        ZA[base + (size_t)i1 * twoK + c] = red(A[e], p);
    }
}

// ---------------------------------------------------------------------------
// Pass 3
// ---------------------------------------------------------------------------

// Carry-in function of one limb: cin in {-1,0,1} -> carry out in {-1,0,1},
// packed as three 2-bit fields (value + 1) at bits 0, 2, 4 for cin = -1, 0, 1.
__device__ __forceinline__ int fn_apply(unsigned code, int c) {
    return (int)((code >> (2 * (c + 1))) & 3u) - 1;
}
__device__ __forceinline__ unsigned fn_compose(unsigned outer, unsigned inner) {
    unsigned r = 0;
#pragma unroll
    for (int c = -1; c <= 1; ++c) r |= (unsigned)(fn_apply(outer, fn_apply(inner, c)) + 1) << (2 * (c + 1));
    return r;
}
constexpr unsigned FN_IDENTITY = 0u | (1u << 2) | (2u << 4);

// Sum of the contributions to limb q of sum_j V_j 2^{Mj}, where V_j is an
// r-word two's-complement value at V[w * wstride + j] (mod 2^(32(lc+1))).
// V_j 2^sh is read as r unsigned words plus one signed top word.
__device__ __forceinline__ int64_t limb_sum(const uint32_t *V, size_t wstride, int q, int M, int r,
                                            int twoK) {
    if (q < 0) return 0;
    int jlo = q - r <= 0 ? 0 : (32 * (q - r) + M - 1) / M;
    int jhi = (32 * q + 31) / M;
    if (jhi > twoK - 1) jhi = twoK - 1;
    int64_t acc = 0;
    for (int j = jlo; j <= jhi; ++j) {
        const int e = M * j;
        const int k = q - (e >> 5), sh = e & 31;
        if (k < 0 || k > r) continue;
        if (k < r) {
            const uint32_t hi = V[(size_t)k * wstride + j];
            const uint32_t lo = k > 0 ? V[(size_t)(k - 1) * wstride + j] : 0u;
            acc += (int64_t)(sh ? __funnelshift_l(lo, hi, sh) : hi);
        } else {
            const int32_t top = (int32_t)V[(size_t)(r - 1) * wstride + j];
            acc += (int64_t)(sh ? (top >> (32 - sh)) : (top < 0 ? -1 : 0));
        }
    }
    return acc;
}

__global__ void __launch_bounds__(THREADS_INV)
k_inverse(const __grid_constant__ KParams P, uint32_t *__restrict__ c, uint8_t *__restrict__ cn) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t i1 = blockIdx.x;
    const int K = P.K, logK = P.logK, twoK = 2 * K, r = P.r, M = P.M;
    const int Y2 = (int)P.Y2;
    const int64_t Y1 = P.Y1;
    const size_t plane = (size_t)Y2 * twoK;
    uint32_t *R = reinterpret_cast<uint32_t *>(smem);  // [r][Y2][2K]
    const int lc1 = P.lc + 1;
    const size_t stage_bytes = stage_bytes_per_warp(P.lc);
    unsigned char *stage_base = smem + (size_t)r * plane * 4;

    for (int t = 0; t < r; ++t) {
        const PrimeConst &pc = P.pc[t];
        const uint32_t p = pc.p, p2 = pc.p2;
        uint32_t *Rt = R + (size_t)t * plane;
        const uint32_t *Zt = P.Z + (size_t)(t * 2) * (size_t)P.Y * twoK;
        for (int e = threadIdx.x; e < Y2 * twoK; e += blockDim.x) {
            const int pos = e >> (logK + 1), col = e & (twoK - 1);
            const uint32_t k2 = bitrev((uint32_t)pos, P.logY2);
            const uint32_t v = Zt[((size_t)pos * Y1 + i1) * twoK + col];
            Rt[e] = shoup(v, pc.ty_i[(size_t)i1 * k2], p);
        }
        __syncthreads();
        dit_cols(Rt, logK + 1, twoK, P.logY2, pc.ty_i, P.logY, p, p2);
        dit_rows(Rt, 2 * Y2, K, logK, pc.tx_i, logK + 1, p, p2);
        const uint2 sc = make_uint2(pc.scale, pc.scale_s);
        for (int e = threadIdx.x; e < Y2 * K; e += blockDim.x) {
            const int i2 = e >> logK, j = e & (K - 1);
            uint32_t *row = Rt + (size_t)i2 * twoK;
            const uint32_t u = shoup(row[j], sc, p);
            const uint32_t v = shoup(row[K + j], pc.untw[j], p);
            row[j] = red(red(u + v, p2), p);
            row[K + j] = red(red(u - v + p2, p2), p);
        }
        __syncthreads();
    }

    // CRT (Garner's mixed radix), centred lift to (-m/2, m/2), r-word
    // two's complement written back over the residues (word w in plane w).
    for (int e = threadIdx.x; e < (int)plane; e += blockDim.x) {
        uint32_t v[RMAX];
        v[0] = R[e];
        for (int t = 1; t < r; ++t) {
            const uint32_t pt = P.pc[t].p;
            uint32_t y = R[(size_t)t * plane + e];
            for (int s = 0; s < t; ++s) {
                const uint32_t vs = red(v[s], pt);  // v_s < 2^30 < 2 p_t
                y = red(shoup(y + pt - vs, make_uint2(P.ginv[t][s], P.ginv_s[t][s]), pt), pt);
            }
            v[t] = y;
        }
        uint32_t X[RMAX];
#pragma unroll
        for (int w = 0; w < RMAX; ++w) X[w] = 0;
        X[0] = v[r - 1];
        for (int t = r - 2; t >= 0; --t) {
            uint64_t carry = v[t];
            const uint32_t pt = P.pc[t].p;
            for (int w = 0; w < r; ++w) {
                const uint64_t z = (uint64_t)X[w] * pt + carry;
                X[w] = (uint32_t)z;
                carry = z >> 32;
            }
        }
        // 2X >= m  <=>  X > (m-1)/2 (m is odd)  ->  X - m
        uint32_t borrow = 0;
        for (int w = 0; w < r; ++w) {
            const uint32_t x2 = (X[w] << 1) | (w ? (X[w - 1] >> 31) : 0u);
            const uint64_t d = (uint64_t)x2 - P.m_words[w] - borrow;
            borrow = (uint32_t)(d >> 63);
        }
        if (!borrow) {
            uint32_t bb = 0;
            for (int w = 0; w < r; ++w) {
                const uint64_t d = (uint64_t)X[w] - P.m_words[w] - bb;
                X[w] = (uint32_t)d;
                bb = (uint32_t)(d >> 63);
            }
        }
        for (int w = 0; w < r; ++w) R[(size_t)w * plane + e] = X[w];
    }
    __syncthreads();

    // Recombination c_i = sum_{j<2K} c_{i,j} 2^{Mj}, one warp per row,
    // computed modulo 2^(32(lc+1)); the top limb is the sign word.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t *st = reinterpret_cast<uint32_t *>(stage_base + (size_t)warp * stage_bytes);
    int8_t *gg = reinterpret_cast<int8_t *>(st + lc1);
    const int per = (lc1 + 31) / 32;
    const int qb = lane * per, qe = min(qb + per, lc1);
    for (int i2 = warp; i2 < Y2; i2 += nw) {
        const int64_t i = i1 + Y1 * (int64_t)i2;
        if (i >= P.nc) continue;
        const uint32_t *V = R + (size_t)i2 * twoK;
        // phases 1-2: limb sums -> (t', g) with carries g in {-1,0,1}
        int64_t hprev = qb < lc1 ? (limb_sum(V, plane, qb - 1, M, r, twoK) >> 32) : 0;
        unsigned F = FN_IDENTITY;
        for (int q = qb; q < qe; ++q) {
            const int64_t Pq = limb_sum(V, plane, q, M, r, twoK);
            const int64_t s = (int64_t)(uint32_t)Pq + hprev;
            hprev = Pq >> 32;
            const uint32_t tq = (uint32_t)s;
            const int g = (int)(s >> 32);
            st[q] = tq;
            gg[q] = (int8_t)g;
            const unsigned f = (unsigned)(g + (tq == 0u ? -1 : 0) + 1) | ((unsigned)(g + 1) << 2) |
                               ((unsigned)(g + (tq == 0xffffffffu ? 1 : 0) + 1) << 4);
            F = fn_compose(f, F);
        }
        // phase 3: warp scan of the carry functions
        unsigned inc = F;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc = fn_compose(inc, o);
        }
        unsigned ex = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) ex = FN_IDENTITY;
        int cin = fn_apply(ex, 0);
        for (int q = qb; q < qe; ++q) {
            const uint32_t tq = st[q];
            const int g = gg[q];
            const int cout = g + ((tq == 0xffffffffu && cin == 1) ? 1 : 0) + ((tq == 0u && cin == -1) ? -1 : 0);
            st[q] = tq + (uint32_t)cin;
            cin = cout;
        }
        __syncwarp();
        const uint32_t top = st[lc1 - 1];
        const bool negative = top == 0xffffffffu;
        if (lane == 0 && top != 0u && !negative) atomicOr(P.err, ERRBIT_INTERNAL);
        if (negative) {
            // magnitude = -value over lc limbs: zero below the lowest non-zero
            // limb f, -x at f, ~x above
            int myf = 0x7fffffff;
            for (int q = qb; q < min(qe, lc1 - 1); ++q)
                if (st[q] != 0u) { myf = q; break; }
            const unsigned m = __ballot_sync(0xffffffffu, myf != 0x7fffffff);
            const int f = m ? __shfl_sync(0xffffffffu, myf, __ffs(m) - 1) : lc1;
            for (int q = qb; q < min(qe, lc1 - 1); ++q) {
                if (q == f) st[q] = 0u - st[q];
                else if (q > f) st[q] = ~st[q];
            }
        }
        __syncwarp();
        uint32_t *crow = c + (size_t)i * P.lc;
        for (int q = lane; q < P.lc; q += 32) crow[q] = st[q];
        if (lane == 0) cn[i] = negative ? 1 : 0;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

int set_kernel_attributes() {
    cudaError_t e1 = cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_FWD_MAX);
    cudaError_t e2 = cudaFuncSetAttribute(k_middle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_MID_MAX);
    cudaError_t e3 = cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)SMEM_INV_MAX);
    return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess) ? 0 : -1;
}

int launch_forward(const KParams &kp, size_t smem, const uint32_t *a, const uint8_t *an,
                   const uint32_t *b, const uint8_t *bn, void *stream) {
    dim3 grid((unsigned)kp.Y1, 2, 1);
    k_forward<<<grid, THREADS_FWD, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_middle(const KParams &kp, size_t smem, void *stream) {
    dim3 grid((unsigned)(2 * kp.K / kp.S), (unsigned)kp.Y2, (unsigned)kp.r);
    k_middle<<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_inverse(const KParams &kp, size_t smem, uint32_t *c, uint8_t *cn, void *stream) {
    dim3 grid((unsigned)kp.Y1, 1, 1);
    k_inverse<<<grid, THREADS_INV, smem, (cudaStream_t)stream>>>(kp, c, cn);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
