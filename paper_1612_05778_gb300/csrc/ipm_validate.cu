// ipm_validate.cu -- a randomised check of a finished product on the GPU:
// c(t) = a(t) b(t) modulo the Mersenne prime q = 2^61 - 1 at a random point
// t.  A wrong c (any changed limb or sign) passes with probability at most
// deg(c) / q (a non-zero polynomial of degree D has at most D roots mod q):
// below 2^-40 for every supported shape.  The paper has no counterpart; the
// plain definition c_k = sum a_i b_{k-i} (§1) is what it checks.
//
// One warp per coefficient row: lane l adds limb_l 2^(32 l mod 61) (2^61 = 1
// mod q; a multiplication by a power of two is a 61-bit rotation), the warp
// sums, the sign is applied and the value weighted by t^i (t^i advanced by
// t^W for the warp's next row, W the number of warps; the first powers come
// from one thread per block); the per-block sums land in `part`, and one
// final block compares.
#include <cuda_runtime.h>

#include <algorithm>

#include "ipm_internal.h"

namespace ipm {
namespace {

constexpr uint64_t Q61 = (1ull << 61) - 1;

__host__ __device__ __forceinline__ uint64_t red61(uint64_t x) {  // x < 2^64 -> [0, q)
    x = (x & Q61) + (x >> 61);
    return x >= Q61 ? x - Q61 : x;
}
__device__ __forceinline__ uint64_t mul61(uint64_t a, uint64_t b) {  // a, b < 2^61
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    return red61((lo & Q61) + ((hi << 3) | (lo >> 61)));
}
__device__ __forceinline__ uint64_t add61(uint64_t a, uint64_t b) { return red61(a + b); }
// x 2^e mod q for x < 2^61, 0 <= e < 61: a 61-bit rotation (2^61 = 1 mod q).
__device__ __forceinline__ uint64_t rot61(uint64_t x, int e) {
    return e ? ((x << e) & Q61) | (x >> (61 - e)) : x;
}
__device__ uint64_t pow61(uint64_t t, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = mul61(r, t);
        t = mul61(t, t);
        e >>= 1;
    }
    return r;
}

__global__ void __launch_bounds__(VAL_THREADS) k_val_partial(const uint32_t *__restrict__ x,
                                                             const uint8_t *__restrict__ xn, int64_t n, int L,
                                                             uint64_t t, uint64_t *__restrict__ part) {
    constexpr int NW = VAL_THREADS / 32;
    __shared__ uint64_t wsum[NW], tpow[NW + 1];  // t^(first row of warp w); t^W
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * NW;
    const int64_t row0 = (int64_t)blockIdx.x * NW + warp;
    // the powers once per block (64-bit modular products are slow: one
    // thread's chain instead of one per warp)
    if (threadIdx.x == 0) {
        uint64_t p = pow61(t, (uint64_t)blockIdx.x * NW);
        for (int w = 0; w < NW; ++w) {
            tpow[w] = p;
            p = mul61(p, t);
        }
        tpow[NW] = pow61(t, (uint64_t)W);
    }
    __syncthreads();
    uint64_t acc = 0;  // lane 0's
    if (row0 < n) {
        uint64_t tp = tpow[warp];
        const uint64_t tW = tpow[NW];
        const int e0 = (32 * lane) % 61;  // limb l = lane + 32k has weight 2^(32 l) = 2^(e0 + 48k mod 61)
        for (int64_t i = row0; i < n; i += W) {
            const uint32_t *r = x + i * L;
            uint64_t v = 0;
            int e = e0;
            for (int l0 = lane; l0 < L; l0 += 8 * 32) {
                // eight rotated limbs (each < 2^61) sum below 2^64: one reduction
                uint64_t s8 = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int l = l0 + 32 * u;
                    if (l < L) s8 += rot61(r[l], e);
                    e += 48;
                    if (e >= 61) e -= 61;
                }
                v = add61(v, red61(s8));
            }
            for (int o = 16; o; o >>= 1) v = add61(v, __shfl_down_sync(0xffffffffu, v, o));
            if (lane == 0) {
                if (xn[i] && v) v = Q61 - v;
                acc = add61(acc, mul61(v, tp));
                tp = mul61(tp, tW);
            }
        }
    }
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t s = 0;
        for (int w = 0; w < NW; ++w) s = add61(s, wsum[w]);
        part[blockIdx.x] = s;
    }
}

// Batched check, pass 1: one warp per item, Horner over its rows from the
// top (acc = acc t + row value), then the weight t^row0.
__global__ void __launch_bounds__(VAL_THREADS) k_valb_partial(const ValItem *__restrict__ items, int64_t nitems,
                                                              const ipm_operands *__restrict__ ops, uint64_t t,
                                                              uint64_t *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (VAL_THREADS / 32);
    for (int64_t w = (int64_t)blockIdx.x * (VAL_THREADS / 32) + (threadIdx.x >> 5); w < nitems; w += warps) {
        const ValItem it = items[w];
        const ipm_operands &o = ops[it.product];
        const uint32_t *x = it.operand == 0 ? o.a : it.operand == 1 ? o.b : o.c;
        const uint8_t *xn = it.operand == 0 ? o.a_neg : it.operand == 1 ? o.b_neg : o.c_neg;
        const int L = it.limbs;
        const int e0 = (32 * lane) % 61;
        uint64_t acc = 0;  // lane 0's
        for (int j = it.rows - 1; j >= 0; --j) {
            const int64_t i = it.row0 + j;
            const uint32_t *r = x + i * L;
            uint64_t v = 0;
            int e = e0;
            for (int l0 = lane; l0 < L; l0 += 8 * 32) {
                uint64_t s8 = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int l = l0 + 32 * u;
                    if (l < L) s8 += rot61(r[l], e);
                    e += 48;
                    if (e >= 61) e -= 61;
                }
                v = add61(v, red61(s8));
            }
            for (int off = 16; off; off >>= 1) v = add61(v, __shfl_down_sync(0xffffffffu, v, off));
            if (lane == 0) {
                if (xn[i] && v) v = Q61 - v;
                acc = add61(mul61(acc, t), v);
            }
        }
        if (lane == 0) part[w] = mul61(acc, it.t_row0);
    }
}

// Batched check, pass 2: one thread per product sums its items.
__global__ void k_valb_final(const int64_t *__restrict__ first, int32_t n, const uint64_t *__restrict__ part,
                             int *err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint64_t s[3];
        for (int o = 0; o < 3; ++o) {
            uint64_t acc = 0;
            for (int64_t k = first[3 * i + o]; k < first[3 * i + o + 1]; ++k) acc = add61(acc, part[k]);
            s[o] = acc;
        }
        if (mul61(s[0], s[1]) != s[2]) atomicOr(err, ERRBIT_MISMATCH);
    }
}

// part: [3][VAL_BLOCKS] sums of a(t), b(t), c(t); sets ERRBIT_MISMATCH in
// *err when a(t) b(t) != c(t) mod q.
__global__ void __launch_bounds__(VAL_THREADS) k_val_final(const uint64_t *__restrict__ part, int *err) {
    __shared__ uint64_t sum[3][VAL_THREADS];
    for (int k = 0; k < 3; ++k) {
        uint64_t s = 0;
        for (int b = threadIdx.x; b < VAL_BLOCKS; b += VAL_THREADS) s = add61(s, part[k * VAL_BLOCKS + b]);
        sum[k][threadIdx.x] = s;
    }
    __syncthreads();
    for (int h = VAL_THREADS / 2; h >= 1; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 3; ++k) sum[k][threadIdx.x] = add61(sum[k][threadIdx.x], sum[k][threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && mul61(sum[0][0], sum[1][0]) != sum[2][0]) atomicOr(err, ERRBIT_MISMATCH);
}

uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

}  // namespace

uint64_t pow61_host(uint64_t t, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = red61((uint64_t)(((unsigned __int128)r * t) % Q61));
        t = (uint64_t)(((unsigned __int128)t * t) % Q61);
        e >>= 1;
    }
    return r;
}

int launch_validate_batch(const ValBatch &vb, const ipm_operands *ops, int *err, void *stream) {
    if (vb.nitems == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t blocks = std::min<int64_t>((vb.nitems + VAL_THREADS / 32 - 1) / (VAL_THREADS / 32), 152 * 64);
    k_valb_partial<<<(unsigned)blocks, VAL_THREADS, 0, s>>>(vb.items, vb.nitems, ops, vb.t, vb.part);
    k_valb_final<<<(vb.nproducts + 255) / 256, 256, 0, s>>>(vb.first, vb.nproducts, vb.part, err);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

uint64_t validation_point(uint64_t seed) {
    return 2 + red61(splitmix64(seed)) % (Q61 - 3);  // t in [2, q - 2]
}

int launch_validate(const ipm_plan_info &I, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                    const uint8_t *bn, const uint32_t *c, const uint8_t *cn, uint64_t t, uint64_t *part, int *err,
                    void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    k_val_partial<<<VAL_BLOCKS, VAL_THREADS, 0, s>>>(a, an, I.na, I.la, t, part);
    k_val_partial<<<VAL_BLOCKS, VAL_THREADS, 0, s>>>(b, bn, I.nb, I.lb, t, part + VAL_BLOCKS);
    k_val_partial<<<VAL_BLOCKS, VAL_THREADS, 0, s>>>(c, cn, I.nc, I.lc, t, part + 2 * VAL_BLOCKS);
    k_val_final<<<1, VAL_THREADS, 0, s>>>(part, err);
    note_launches(4);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm

extern "C" ipm_status ipm_validate(const ipm_shape *shape, const uint32_t *a, const uint8_t *a_neg,
                                   const uint32_t *b, const uint8_t *b_neg, const uint32_t *c,
                                   const uint8_t *c_neg, uint64_t seed, ipm_stream_t stream) {
    if (!shape || !a || !a_neg || !b || !b_neg || !c || !c_neg) return IPM_ERR_ARG;
    ipm_plan_info I;
    ipm_status st = ipm_choose(shape, nullptr, &I);  // the layout (strides) only
    if (st != IPM_OK) return st;
    void *d = nullptr;
    if (cudaMalloc(&d, 3 * ipm::VAL_BLOCKS * sizeof(uint64_t) + 16) != cudaSuccess) return IPM_ERR_NOMEM;
    uint64_t *part = (uint64_t *)d;
    int *err = (int *)(part + 3 * ipm::VAL_BLOCKS);
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    bool ok = cudaMemsetAsync(err, 0, sizeof(int), s) == cudaSuccess &&
              ipm::launch_validate(I, a, a_neg, b, b_neg, c, c_neg, ipm::validation_point(seed), part, err,
                                   stream) == 0 &&
              cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
              cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(d);
    if (!ok) return IPM_ERR_CUDA;
    return (h & ipm::ERRBIT_MISMATCH) ? IPM_ERR_MISMATCH : IPM_OK;
}
