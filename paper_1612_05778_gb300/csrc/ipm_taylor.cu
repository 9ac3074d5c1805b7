// ipm_taylor.cu -- Taylor shift by one, g(x) = f(x + 1), on top of the
// exact product.
//
// The paper's application (§1: real root isolation) shifts polynomials with
// a divide-and-conquer Taylor shift (Algorithm E of J. von zur Gathen and
// J. Gerhard, "Fast algorithms for Taylor shifts and certain difference
// equations", ISSAC 1997) whose cost is that of its polynomial products.
// With n' = 2^m >= n coefficients (f padded with zeros) and
// f = f_lo + x^(n'/2) f_hi,
//     f(x + 1) = f_lo(x + 1) + (x + 1)^(n'/2) f_hi(x + 1),
// done bottom-up: at level l (blocks of b = 2^l coefficients, each already
// shifted) every pair of adjacent blocks (lo, hi) becomes
// lo + (x + 1)^b hi, a block of 2b.  All pairs of one level are one
// product: with H(x) = sum_j hi_j(x) x^(2bj) (the hi blocks moved onto the
// lo positions, zeros in between), (x + 1)^b H(x) holds every
// (x + 1)^b hi_j, of degree 2b - 1, in its own block [2bj, 2bj + 2b).
// The binomial polynomial (x + 1)^b is the square of (x + 1)^(b/2); the
// plan computes all of them once (they do not depend on f).
//
// Bounds: a shifted block of B coefficients below 2^bits in magnitude has
// |coefficient k| <= (2^bits - 1) C(B, k + 1) < 2^(bits + B), and
// C(b, k) < 2^b for b >= 1.  Every intermediate is stored at the stride of
// its bound; a non-zero limb beyond it sets ERRBIT_INTERNAL.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ipm_internal.h"

namespace ipm {
namespace {

// dst row i (i < nd) = src row i + shift when blk == 0 or i mod 2blk < blk
// (and that row exists), else zero; limb strides dL and sL (limbs of src
// beyond dL must be zero).  bound > 0: every source row must be below
// 2^bound (ERRBIT_BOUND otherwise).  One thread per destination limb.
__global__ void k_taylor_rows(uint32_t *__restrict__ dst, uint8_t *__restrict__ dneg, int dL,
                              const uint32_t *__restrict__ src, const uint8_t *__restrict__ sneg, int sL,
                              int64_t ns, int64_t nd, int64_t shift, int64_t blk, uint32_t bound, int *err) {
    const int64_t total = nd * dL;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / dL;
        const int q = (int)(e - i * dL);
        const int64_t j = i + shift;
        const bool take = j < ns && (blk == 0 || (i & (2 * blk - 1)) < blk);
        dst[e] = take && q < sL ? src[j * sL + q] : 0u;
        if (q == 0) dneg[i] = take ? sneg[j] : 0;
        if (take && q == dL - 1)
            for (int r = dL; r < sL; ++r)
                if (src[j * sL + r]) atomicOr(err, ERRBIT_INTERNAL);
        if (take && bound && q == 0 && (bound & 31u) && (src[j * sL + (sL - 1)] >> (bound & 31u)))
            atomicOr(err, ERRBIT_BOUND);
    }
}

// (x + 1): two coefficients equal to 1, stride L.
__global__ void k_taylor_xplus1(uint32_t *b, uint8_t *bneg, int L) {
    for (int q = threadIdx.x; q < 2 * L; q += blockDim.x) b[q] = (q % L) == 0 ? 1u : 0u;
    if (threadIdx.x < 2) bneg[threadIdx.x] = 0;
}

// Carries (or borrows) into each lane of a 32-limb chunk from generate and
// propagate bits (disjoint) and the chunk's carry-in; *cio becomes the
// carry out.
__device__ __forceinline__ unsigned chain(unsigned gen, unsigned prop, unsigned *cio) {
    const uint64_t s = (uint64_t)gen + (uint64_t)(gen | prop) + *cio;
    *cio = (unsigned)(s >> 32);
    return (unsigned)s ^ prop;
}

// D_i = P_i + (i mod 2blk < blk ? S_i : 0) for i < nd, sign-magnitude, one
// warp per row: equal signs add the magnitudes, opposite signs subtract the
// smaller from the larger (found from the highest differing limb); both
// with ballot carry-lookahead over 32 limbs per step.  Zero is stored as +0.
__global__ void k_taylor_add(const uint32_t *__restrict__ P, const uint8_t *__restrict__ Pn, int LP,
                             const uint32_t *__restrict__ S, const uint8_t *__restrict__ Sn, int LS, int64_t blk,
                             uint32_t *__restrict__ D, uint8_t *__restrict__ Dn, int LD, int64_t nd, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int Lm = max(LP, LS);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < nd; i += warps) {
        const uint32_t *x = P + i * LP;
        const bool use_s = (i & (2 * blk - 1)) < blk;
        const uint32_t *y = S + i * LS;
        const int Ly = use_s ? LS : 0;
        const bool sx = Pn[i] != 0, sy = use_s && Sn[i] != 0;
        // opposite signs: which magnitude is larger (highest differing limb)
        bool x_big = true, equal = false;
        const bool sub = Ly > 0 && sx != sy;
        if (sub) {
            int top = -1;
            for (int q0 = ((Lm - 1) & ~31); q0 >= 0 && top < 0; q0 -= 32) {
                const int q = q0 + lane;
                const uint32_t a = q < LP ? x[q] : 0u, b = q < Ly ? y[q] : 0u;
                const unsigned d = __ballot_sync(0xffffffffu, a != b);
                if (d) {
                    top = q0 + 31 - __clz(d);
                    const int src = top & 31;
                    const unsigned gt = __ballot_sync(0xffffffffu, a > b);
                    x_big = (gt >> src) & 1u;
                }
            }
            equal = top < 0;
        }
        const uint32_t *u = x_big ? x : y;  // the larger magnitude when subtracting
        const uint32_t *v = x_big ? y : x;
        const int Lu = x_big ? LP : Ly, Lv = x_big ? Ly : LP;
        unsigned cio = 0;
        bool nonzero = false;
        for (int q0 = 0; q0 < Lm; q0 += 32) {
            const int q = q0 + lane;
            uint32_t r;
            if (!sub) {
                const uint32_t a = q < LP ? x[q] : 0u, b = q < Ly ? y[q] : 0u;
                const uint32_t s = a + b;
                const unsigned cm = chain(__ballot_sync(0xffffffffu, s < a), __ballot_sync(0xffffffffu, s == 0xffffffffu),
                                          &cio);
                r = s + ((cm >> lane) & 1u);
            } else {
                const uint32_t a = q < Lu ? u[q] : 0u, b = q < Lv ? v[q] : 0u;
                const uint32_t d = a - b;
                const unsigned bm = chain(__ballot_sync(0xffffffffu, a < b), __ballot_sync(0xffffffffu, a == b), &cio);
                r = d - ((bm >> lane) & 1u);
            }
            if (q < LD) D[i * LD + q] = r;
            else if (q < Lm && r) atomicOr(err, ERRBIT_INTERNAL);
            if (__ballot_sync(0xffffffffu, q < Lm && r != 0u)) nonzero = true;
        }
        if (!sub && cio) atomicOr(err, ERRBIT_INTERNAL);  // a carry out of the top limb
        for (int q = Lm + lane; q < LD; q += 32) D[i * LD + q] = 0u;
        if (lane == 0) Dn[i] = (nonzero && !equal) ? (uint8_t)(sub ? (x_big ? sx : sy) : (sx || sy)) : 0;
    }
}

// ---- the first levels in shared memory ----------------------------------------
//
// Levels 0..5 (blocks of up to TB = 64 coefficients) of every 64-block in
// one kernel: a CUDA block holds its 64 coefficients as W-limb two's
// complement values (W covers bits + 64 magnitude bits and the sign) and
// runs the same recursion with additions only: at level b, T = the hi
// blocks moved onto the lo positions, b steps T_k <- T_k + T_(k-1) inside
// each 2b-window (a multiplication by x + 1 each), then A_k = T_k + lo_k.
// One warp per coefficient row, ballot carry-lookahead over 32 limbs.
constexpr int TB = 64;
constexpr int TB_THREADS = 256;

// dst = src + (b ? b : 0), W limbs, two's complement (mod 2^(32 W)).
__device__ __forceinline__ void warp_add_rows(uint32_t *dst, const uint32_t *a, const uint32_t *b, int W) {
    const int lane = threadIdx.x & 31;
    unsigned cio = 0;
    for (int q0 = 0; q0 < W; q0 += 32) {
        const int q = q0 + lane;
        const uint32_t x = q < W ? a[q] : 0u, y = (b && q < W) ? b[q] : 0u;
        const uint32_t sum = x + y;
        const unsigned cm = chain(__ballot_sync(0xffffffffu, sum < x), __ballot_sync(0xffffffffu, sum == 0xffffffffu),
                                  &cio);
        if (q < W) dst[q] = sum + ((cm >> lane) & 1u);
    }
}

__global__ void __launch_bounds__(TB_THREADS) k_taylor_base(const uint32_t *__restrict__ f,
                                                          const uint8_t *__restrict__ fn, int lf, int64_t n,
                                                          uint32_t bits, int W, uint32_t *__restrict__ S,
                                                          uint8_t *__restrict__ Sn, int LS, int *err) {
    extern __shared__ uint32_t sm[];
    uint32_t *A = sm, *T = sm + TB * W, *U = sm + 2 * TB * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = TB_THREADS / 32;
    const int64_t base = (int64_t)blockIdx.x * TB;
    // load: sign-magnitude -> two's complement (-x = ~x + 1)
    for (int k = warp; k < TB; k += nw) {
        const int64_t i = base + k;
        const bool have = i < n;
        const bool neg = have && fn[i] != 0;
        unsigned cio = neg ? 1u : 0u;
        for (int q0 = 0; q0 < W; q0 += 32) {
            const int q = q0 + lane;
            uint32_t x = (have && q < lf) ? f[i * lf + q] : 0u;
            if (q == lf - 1 && (bits & 31u) && (x >> (bits & 31u))) atomicOr(err, ERRBIT_BOUND);
            if (neg) x = ~x;
            const unsigned cm = chain(0u, __ballot_sync(0xffffffffu, x == 0xffffffffu), &cio);
            if (q < W) A[k * W + q] = x + ((cm >> lane) & 1u);
        }
    }
    __syncthreads();
    for (int b = 1; b < TB; b <<= 1) {
        const int w2 = 2 * b;
        for (int k = warp; k < TB; k += nw)  // T: hi moved down, zeros above
            for (int q = lane; q < W; q += 32) T[k * W + q] = (k & (w2 - 1)) < b ? A[(k + b) * W + q] : 0u;
        __syncthreads();
        for (int step = 0; step < b; ++step) {  // T <- (x + 1) T inside each window
            for (int k = warp; k < TB; k += nw) {
                if ((k & (w2 - 1)) == 0)
                    for (int q = lane; q < W; q += 32) U[k * W + q] = T[k * W + q];
                else
                    warp_add_rows(U + k * W, T + k * W, T + (k - 1) * W, W);
            }
            __syncthreads();
            uint32_t *x = T;
            T = U;
            U = x;
        }
        for (int k = warp; k < TB; k += nw)  // A = T + lo
            warp_add_rows(A + k * W, T + k * W, (k & (w2 - 1)) < b ? A + k * W : nullptr, W);
        __syncthreads();
    }
    // store: two's complement -> sign-magnitude at stride LS
    for (int k = warp; k < TB; k += nw) {
        const int64_t i = base + k;
        const bool neg = (A[k * W + W - 1] >> 31) != 0;
        unsigned cio = neg ? 1u : 0u;
        bool nonzero = false;
        for (int q0 = 0; q0 < W; q0 += 32) {
            const int q = q0 + lane;
            uint32_t x = q < W ? A[k * W + q] : 0u;
            if (neg) x = ~x;
            const unsigned cm = chain(0u, __ballot_sync(0xffffffffu, x == 0xffffffffu), &cio);
            const uint32_t r = x + ((cm >> lane) & 1u);
            if (q < LS) S[i * LS + q] = r;
            else if (q < W && r) atomicOr(err, ERRBIT_INTERNAL);
            if (__ballot_sync(0xffffffffu, q < W && r != 0u)) nonzero = true;
        }
        for (int q = W + lane; q < LS; q += 32) S[i * LS + q] = 0u;
        if (lane == 0) Sn[i] = (neg && nonzero) ? 1 : 0;
    }
}

int grid_for(int64_t work, int per_block) {
    const int64_t b = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

int ceil_div32(int64_t bits) { return (int)((bits + 31) / 32); }

}  // namespace
}  // namespace ipm

using namespace ipm;

struct ipm_taylor_s {
    int64_t n = 0, n2 = 0;  // coefficients, padded to a power of two
    uint32_t bits = 0;
    int m = 0;              // levels
    uint32_t flags = 0;
    int32_t lg = 0;         // output limb stride
    std::vector<ipm_plan_t> square;  // square[l]: (x+1)^(2^(l-1)) squared (l >= 1); plan time only
    std::vector<ipm_plan_t> level;   // level[l]: (x+1)^b times H
    std::vector<int32_t> ls;         // ls[l]: stride of the level-l state (bound bits + 2^l)
    std::vector<int32_t> lp;         // lp[l]: stride of the level-l product
    std::vector<int32_t> lq;         // lq[l]: stride of the level-l square
    std::vector<void *> mem;
    uint32_t *S[2] = {nullptr, nullptr}, *H = nullptr, *P = nullptr, *Q = nullptr;
    uint8_t *Sn[2] = {nullptr, nullptr}, *Hn = nullptr, *Pn = nullptr, *Qn = nullptr;
    // levels 0..5 in shared memory (k_taylor_base) when the plan has more
    // levels and 3 TB W words fit a block
    bool base = false;
    int base_w = 0;
    // (x + 1)^(2^l) of every level l, computed once by the plan (they do not
    // depend on f): b + 1 coefficients at stride ceil(b / 32), 16-byte aligned
    std::vector<uint32_t *> Bl;
    std::vector<uint8_t *> Bln;
    int *err = nullptr;
};

namespace {

void free_taylor(ipm_taylor_s *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    for (auto p : t->square)
        if (p) ipm_destroy(p);
    for (auto p : t->level)
        if (p) ipm_destroy(p);
    for (void *p : t->mem) cudaFree(p);
    delete t;
}

template <class T>
ipm_status dalloc(ipm_taylor_s *t, T **out, size_t count) {
    void *d = nullptr;
    const cudaError_t e = cudaMalloc(&d, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? IPM_ERR_NOMEM : IPM_ERR_CUDA;
    t->mem.push_back(d);
    *out = (T *)d;
    return IPM_OK;
}

}  // namespace

extern "C" ipm_status ipm_taylor_plan(ipm_taylor_t *out, int64_t deg, uint32_t bits, uint32_t flags) {
    if (!out || deg < 0 || bits < 1) return IPM_ERR_ARG;
    *out = nullptr;
    auto *t = new (std::nothrow) ipm_taylor_s;
    if (!t) return IPM_ERR_NOMEM;
    t->n = deg + 1;
    t->bits = bits;
    t->flags = flags;
    t->n2 = 1;
    while (t->n2 < t->n) {
        t->n2 <<= 1;
        ++t->m;
    }
    // the top level multiplies coefficients of bits + n2/2 bits
    if ((int64_t)bits + t->n2 / 2 > 65536 || t->n > (1ll << 20)) {
        delete t;
        return IPM_ERR_UNSUPPORTED;
    }
    t->lg = ceil_div32((int64_t)bits + t->n);
    const uint32_t inner = flags & (IPM_COSTMODEL | IPM_TENSOR_STAGES);
    ipm_status st;
    int32_t lsmax = ceil_div32((int64_t)bits + t->n2), lpmax = 1, lqmax = 1;
    for (int l = 0; l < t->m; ++l) {
        const int64_t b = 1ll << l;
        t->ls.push_back(ceil_div32((int64_t)bits + b));
        if (l >= 1) {  // (x+1)^b = ((x+1)^(b/2))^2
            ipm_shape sh{b / 2, b / 2, (uint32_t)(b / 2), (uint32_t)(b / 2)};
            ipm_plan_t p = nullptr;
            if ((st = ipm_plan(&p, &sh, 1, inner)) != IPM_OK) { free_taylor(t); return st; }
            t->square.push_back(p);
            ipm_plan_info I;
            ipm_get_info(p, 0, &I);
            t->lq.push_back(I.lc);
            lqmax = std::max(lqmax, I.lc);
        } else {
            t->square.push_back(nullptr);
            t->lq.push_back(0);
        }
        // (x+1)^b (b+1 coefficients < 2^b) times H (n2 - b coefficients < 2^(bits+b));
        // short binomials (b <= 32) by the schoolbook family where its limits
        // allow (b + 1 terms per output coefficient), unless the learned
        // dispatch chooses
        ipm_shape sh{b, t->n2 - b - 1, (uint32_t)b, (uint32_t)(bits + b)};
        ipm_plan_t p = nullptr;
        st = IPM_ERR_ARG;
        if (!(inner & IPM_COSTMODEL) && b <= 32) {
            ipm_params school{};
            school.school = 1;
            st = ipm_plan_ex(&p, &sh, 1, inner, &school);
        }
        if (st != IPM_OK && (st = ipm_plan(&p, &sh, 1, inner)) != IPM_OK) { free_taylor(t); return st; }
        t->level.push_back(p);
        ipm_plan_info I;
        ipm_get_info(p, 0, &I);
        t->lp.push_back(I.lc);
        lpmax = std::max(lpmax, I.lc);
    }
    const size_t n2 = (size_t)t->n2;
    if ((st = dalloc(t, &t->S[0], n2 * lsmax)) || (st = dalloc(t, &t->S[1], n2 * lsmax)) ||
        (st = dalloc(t, &t->Sn[0], n2)) || (st = dalloc(t, &t->Sn[1], n2)) ||
        (st = dalloc(t, &t->H, n2 * lsmax)) || (st = dalloc(t, &t->Hn, n2)) ||
        (st = dalloc(t, &t->P, n2 * lpmax)) || (st = dalloc(t, &t->Pn, n2)) ||
        (st = dalloc(t, &t->Q, (n2 / 2 + 1) * lqmax)) || (st = dalloc(t, &t->Qn, n2 / 2 + 2)) ||
        (st = dalloc(t, &t->err, 4))) {
        free_taylor(t);
        return st;
    }
    if (cudaMemset(t->err, 0, sizeof(int)) != cudaSuccess) { free_taylor(t); return IPM_ERR_CUDA; }
    t->base_w = ceil_div32((int64_t)bits + TB + 1);
    const size_t base_smem = (size_t)3 * TB * t->base_w * sizeof(uint32_t);
    if (t->m > 6 && base_smem <= 200 * 1024) {
        if (cudaFuncSetAttribute(k_taylor_base, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)base_smem) !=
            cudaSuccess) {
            free_taylor(t);
            return IPM_ERR_CUDA;
        }
        t->base = true;
    }
    // the binomial polynomials, once: (x + 1), then squarings (the square
    // plans are not needed afterwards and are freed)
    if (t->m > 0) {
        size_t words = 0;
        for (int l = 0; l < t->m; ++l) {
            const int64_t b = 1ll << l;
            words += ((size_t)(b + 1) * ceil_div32(b) + 3) & ~(size_t)3;
        }
        uint32_t *arena = nullptr;
        uint8_t *arena_n = nullptr;
        if ((st = dalloc(t, &arena, words)) || (st = dalloc(t, &arena_n, (size_t)t->n2 + t->m))) {
            free_taylor(t);
            return st;
        }
        size_t off = 0, off_n = 0;
        for (int l = 0; l < t->m; ++l) {
            const int64_t b = 1ll << l;
            t->Bl.push_back(arena + off);
            t->Bln.push_back(arena_n + off_n);
            off += ((size_t)(b + 1) * ceil_div32(b) + 3) & ~(size_t)3;
            off_n += (size_t)b + 1;
        }
        k_taylor_xplus1<<<1, 64>>>(t->Bl[0], t->Bln[0], 1);
        note_launches(1);
        for (int l = 1; l < t->m; ++l) {
            const int64_t b = 1ll << l;
            const int lbin = ceil_div32(b);
            if ((st = ipm_mul(t->square[l], t->Bl[l - 1], t->Bln[l - 1], t->Bl[l - 1], t->Bln[l - 1], t->Q, t->Qn,
                              nullptr)) != IPM_OK) {
                free_taylor(t);
                return st;
            }
            k_taylor_rows<<<grid_for((b + 1) * lbin, 256), 256>>>(t->Bl[l], t->Bln[l], lbin, t->Q, t->Qn, t->lq[l],
                                                                  b + 1, b + 1, 0, 0, 0u, t->err);
            note_launches(1);
        }
        if (cudaStreamSynchronize(nullptr) != cudaSuccess) { free_taylor(t); return IPM_ERR_CUDA; }
        for (auto &p : t->square)
            if (p) {
                const ipm_status sst = ipm_sync(p, nullptr);
                ipm_destroy(p);
                p = nullptr;
                if (sst != IPM_OK) { free_taylor(t); return sst; }
            }
        int h = 0;
        if (cudaMemcpy(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || h) {
            free_taylor(t);
            return IPM_ERR_CUDA;
        }
    }
    *out = t;
    return IPM_OK;
}

extern "C" ipm_status ipm_taylor_limbs(ipm_taylor_t t, int32_t *limbs) {
    if (!t || !limbs) return IPM_ERR_ARG;
    *limbs = t->lg;
    return IPM_OK;
}

extern "C" ipm_status ipm_taylor_shift(ipm_taylor_t t, const uint32_t *f, const uint8_t *f_neg, uint32_t *g,
                                       uint8_t *g_neg, ipm_stream_t stream) {
    if (!t || !f || !f_neg || !g || !g_neg) return IPM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int lf = ceil_div32(t->bits);
    const int64_t n2 = t->n2;
    auto launched = [&](int k) {
        note_launches(k);
        return cudaGetLastError() == cudaSuccess;
    };
    if (t->m == 0) {  // one coefficient: g = f (the addition of nothing normalises -0)
        k_taylor_rows<<<1, 256, 0, s>>>(t->S[0], t->Sn[0], lf, f, f_neg, lf, 1, 1, 0, 0, t->bits, t->err);
        k_taylor_add<<<1, 32, 0, s>>>(t->S[0], t->Sn[0], lf, t->S[0], t->Sn[0], lf, 0, g, g_neg, t->lg, 1, t->err);
        if (!launched(2)) return IPM_ERR_CUDA;
        return (t->flags & IPM_SYNC) ? ipm_taylor_sync(t, stream) : IPM_OK;
    }
    int cur = 0, l0 = 0;
    if (t->base) {
        // levels 0..5 in shared memory: the level-6 state, and (x + 1)^64
        const size_t smem = (size_t)3 * TB * t->base_w * sizeof(uint32_t);
        k_taylor_base<<<(unsigned)(n2 / TB), TB_THREADS, smem, s>>>(f, f_neg, lf, t->n, t->bits, t->base_w, t->S[0],
                                                                     t->Sn[0], t->ls[6], t->err);
        if (!launched(1)) return IPM_ERR_CUDA;
        l0 = 6;
    } else {
        // level-0 state: f at its stride, rows n.. zero
        k_taylor_rows<<<grid_for(n2 * t->ls[0], 256), 256, 0, s>>>(t->S[0], t->Sn[0], t->ls[0], f, f_neg, lf, t->n,
                                                                   n2, 0, 0, t->bits, t->err);
        if (!launched(1)) return IPM_ERR_CUDA;
    }
    for (int l = l0; l < t->m; ++l) {
        const int64_t b = 1ll << l;
        // H: the hi blocks moved onto the lo positions
        const int L = t->ls[l];
        k_taylor_rows<<<grid_for((n2 - b) * L, 256), 256, 0, s>>>(t->H, t->Hn, L, t->S[cur], t->Sn[cur], L, n2,
                                                                  n2 - b, b, b, 0u, t->err);
        if (!launched(1)) return IPM_ERR_CUDA;
        ipm_status st = ipm_mul(t->level[l], t->Bl[l], t->Bln[l], t->H, t->Hn, t->P, t->Pn, stream);
        if (st != IPM_OK) return st;
        // the new state: the product plus the lo blocks
        const bool last = l + 1 == t->m;
        uint32_t *D = last ? g : t->S[cur ^ 1];
        uint8_t *Dn = last ? g_neg : t->Sn[cur ^ 1];
        const int LD = last ? t->lg : t->ls[l + 1];
        const int64_t nd = last ? t->n : n2;
        k_taylor_add<<<grid_for(nd * 32, 256), 256, 0, s>>>(t->P, t->Pn, t->lp[l], t->S[cur], t->Sn[cur], L, b, D,
                                                            Dn, LD, nd, t->err);
        if (!launched(1)) return IPM_ERR_CUDA;
        cur ^= 1;
    }
    if (t->flags & IPM_SYNC) return ipm_taylor_sync(t, stream);
    return IPM_OK;
}

extern "C" ipm_status ipm_taylor_sync(ipm_taylor_t t, ipm_stream_t stream) {
    if (!t) return IPM_ERR_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return IPM_ERR_CUDA;
    ipm_status worst = IPM_OK;
    for (auto p : t->square)
        if (p) {
            const ipm_status st = ipm_sync(p, stream);
            if (st != IPM_OK && worst == IPM_OK) worst = st;
        }
    for (auto p : t->level) {
        const ipm_status st = ipm_sync(p, stream);
        if (st != IPM_OK && worst == IPM_OK) worst = st;
    }
    int h = 0;
    if (cudaMemcpy(&h, t->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return IPM_ERR_CUDA;
    if (h) {
        cudaMemset(t->err, 0, sizeof(int));
        if (h & ERRBIT_BOUND) return IPM_ERR_BOUND;
        if (worst == IPM_OK) worst = IPM_ERR_CUDA;
    }
    return worst;
}

extern "C" ipm_status ipm_taylor_destroy(ipm_taylor_t t) {
    free_taylor(t);
    return IPM_OK;
}
