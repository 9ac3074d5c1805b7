// ntt_stages.cuh -- register-resident radix-R transform stages on
// shared-memory tiles (R = 2, 4, 8, 16).
//
// A length-L transform is split into stages of radix R_1, R_2, ... (the
// four-step factorisation applied recursively).  At a stage of radix R the
// data are L/Lc independent sub-blocks of length Lc; with L' = Lc/R, thread
// group (block, n1) gathers x_m = block[n1 + L' m] (m < R) into registers,
// runs an R-point DFT there as radix-2 Gentleman-Sande butterflies with the
// constants omega_R^j (held in registers), multiplies output k2 by
// omega_Lc^{n1 k2}, and scatters it back.  The result is the same
// bit-reversed-order DFT the plain radix-2 DIF gives, with one table
// twiddle per element per stage instead of one per butterfly.  The inverse
// stage is the exact mirror (inverse twiddle, then an R-point DIT DFT with
// omega_R^{-1}), so forward followed by inverse is L times the identity.
//
// Element n of transform t lives at s[(t % tm) * ta + (t / tm) * tb + n * es]
// (two-level transform index: e.g. row and half of a tile).  Consecutive
// threads take consecutive t, so with an odd row pitch the gathers of a
// warp hit distinct banks.
#pragma once
#include <stdint.h>

#include "modarith.cuh"

namespace ipm {

__host__ __device__ constexpr int clog2(int x) { return x <= 1 ? 0 : 1 + clog2(x / 2); }

template <int R>
struct Roots {
    uint2 w[R / 2 > 0 ? R / 2 : 1];  // omega_R^{+-j}, j < R/2
};

// Where a stage's twiddles come from (the SM template argument of the
// stage functions):
//   TW_GLOBAL (0): omega_T^e, e < T, in global memory (non-coherent cache);
//   TW_SHARED (1): the same table in shared memory;
//   TW_STAGE  (2): a per-stage block in shared memory for a stage of
//     sub-block length Lc = R L': entry m L' + n1 holds the twiddle
//     omega_Lc^{n1 brev(m)} of output (forward) or input (inverse) m of
//     group n1, and entries Lc .. Lc + R/2 - 1 the roots omega_R^j.  A
//     warp's groups have consecutive n1, so its twiddle reads are
//     consecutive entries (no bank conflicts) at addresses that need no
//     multiplication; logT passes log2 Lc.
constexpr int TW_GLOBAL = 0, TW_SHARED = 1, TW_STAGE = 2;

template <int SM>
__device__ __forceinline__ uint2 tload(const uint2 *p) {
    if constexpr (SM != TW_GLOBAL)
        return *p;
    else
        return __ldg(p);
}

template <int R, int SM>
__device__ __forceinline__ void load_roots(Roots<R> &rt, const uint2 *__restrict__ tab, int logT) {
    constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
#pragma unroll
    for (int j = 0; j < R / 2; ++j)
        rt.w[j] = SM == TW_STAGE ? tab[(1u << logT) + j] : tload<SM>(tab + ((uint32_t)j << (logT - LR)));
}

template <int R>
__host__ __device__ constexpr int brev_c(int m) {
    int r = 0;
    for (int b = 1, rb = R >> 1; b < R; b <<= 1, rb >>= 1)
        if (m & b) r |= rb;
    return r;
}

// (x, y) -> (x + y, x - y) with unit twiddle, values in [0, 2p).
__device__ __forceinline__ void bf_unit(uint32_t &x, uint32_t &y, uint32_t p2) {
    const uint32_t s = red(x + y, p2);
    const uint32_t d = red(x - y + p2, p2);
    x = s;
    y = d;
}

// In-register DFT, natural order in, bit-reversed order out.
template <int R>
__device__ __forceinline__ void dft_dif(uint32_t (&x)[R], const Roots<R> &rt, uint32_t p, uint32_t p2) {
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                if (k == 0)
                    bf_unit(x[b], x[b + h], p2);
                else
                    bf_dif(x[b + k], x[b + k + h], rt.w[k * (R / (2 * h))], p, p2);
            }
        }
    }
}

// dft_dif for inputs whose upper half x[R/2..R) is zero: the first level
// reduces to x[k + R/2] = x[k] omega_R^k.
template <int R>
__device__ __forceinline__ void dft_dif_hz(uint32_t (&x)[R], const Roots<R> &rt, uint32_t p, uint32_t p2) {
    x[R / 2] = x[0];
#pragma unroll
    for (int k = 1; k < R / 2; ++k) x[k + R / 2] = shoup(x[k], rt.w[k], p);
#pragma unroll
    for (int h = R / 4; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                if (k == 0)
                    bf_unit(x[b], x[b + h], p2);
                else
                    bf_dif(x[b + k], x[b + k + h], rt.w[k * (R / (2 * h))], p, p2);
            }
        }
    }
}

// dft_dif followed by the stage twiddle of every output m >= 1, with the
// twiddle folded into the last butterfly level: the unreduced sum and
// difference of a unit butterfly (x + y and x - y + 2p, both < 4p < 2^32)
// go straight into Shoup's multiplication, which accepts any 32-bit input
// and returns [0, 2p) -- two reductions fewer per twiddled output.
// HZ: the upper half of the inputs is zero (as dft_dif_hz).
template <int R, bool HZ>
__device__ __forceinline__ void dft_dif_tw(uint32_t (&x)[R], const Roots<R> &rt, const uint2 (&w)[R], uint32_t p,
                                           uint32_t p2) {
    if constexpr (R == 2) {
        if (HZ) {
            x[1] = shoup(x[0], w[1], p);  // (x0, 0) -> (x0, x0 w1)
        } else {
            const uint32_t s = x[0] + x[1], d = x[0] - x[1] + p2;
            x[0] = red(s, p2);
            x[1] = shoup(d, w[1], p);
        }
    } else {
        int h0 = R / 2;
        if (HZ) {
            x[R / 2] = x[0];
#pragma unroll
            for (int k = 1; k < R / 2; ++k) x[k + R / 2] = shoup(x[k], rt.w[k], p);
            h0 = R / 4;
        }
#pragma unroll
        for (int h = R / 2; h >= 2; h >>= 1) {
            if (h > h0) continue;
#pragma unroll
            for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    if (k == 0)
                        bf_unit(x[b], x[b + h], p2);
                    else
                        bf_dif(x[b + k], x[b + k + h], rt.w[k * (R / (2 * h))], p, p2);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < R; b += 2) {
            const uint32_t s = x[b] + x[b + 1], d = x[b] - x[b + 1] + p2;
            x[b] = b == 0 ? red(s, p2) : shoup(s, w[b], p);
            x[b + 1] = shoup(d, w[b + 1], p);
        }
    }
}

// In-register inverse DFT (roots omega_R^{-j}), bit-reversed in, natural
// out, inputs and outputs in [0, 2p).  Harvey's lazy Cooley-Tukey
// butterflies (D. Harvey, J. Symb. Comp. 60, 2014): between levels the
// values may reach [0, 4p); a butterfly brings only its x input back to
// [0, 2p) (the Shoup product of y accepts any 32-bit input), then forms
// x + t and x - t + 2p without reducing them.  The first level's inputs are
// already in [0, 2p) and its twiddles are 1, so it needs no reduction.
template <int R>
__device__ __forceinline__ void dft_dit(uint32_t (&x)[R], const Roots<R> &rt, uint32_t p, uint32_t p2) {
#pragma unroll
    for (int b = 0; b < R; b += 2) {
        const uint32_t s = x[b] + x[b + 1], d = x[b] - x[b + 1] + p2;
        x[b] = s;
        x[b + 1] = d;
    }
#pragma unroll
    for (int h = 2; h < R; h <<= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int k = 0; k < h; ++k) {
                const uint32_t xa = red(x[b + k], p2);
                const uint32_t t = k == 0 ? red(x[b + k + h], p2)
                                          : shoup(x[b + k + h], rt.w[k * (R / (2 * h))], p);
                x[b + k] = xa + t;
                x[b + k + h] = xa - t + p2;
            }
        }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) x[m] = red(x[m], p2);
}

struct TileMap {
    uint32_t *s;
    int T;       // number of transforms
    int tm;      // transforms per first-level group
    int ta, tb;  // strides of t % tm and t / tm
    int es;      // element stride
    int rot;     // log2 T for tiles of T < 32 transforms at row pitch T + 1, else 0 (see rotate_rows)
    // Padded rows: 0, or log2 P for a tile that leaves one empty element
    // slot after every P elements, so element n lives at slot n + n / P.
    // With P the radix of the transform's last stage, the last stage's
    // groups (P consecutive elements each, P apart) land on distinct banks
    // even at a dense row pitch (P + 1 slots per P elements); every earlier
    // stage's stride L' is a multiple of P, so its elements stay evenly
    // spaced (L' + L'/P slots apart).
    int pl = 0;
};

// Slot of element n in a padded tile (see TileMap::pl).
__device__ __forceinline__ int padded(const TileMap &M, int n) { return M.pl ? n + (n >> M.pl) : n; }

// With T < 32 transforms at row pitch T + 1, a warp's gathers touch 32 / T
// rows; rows T apart land on disjoint banks ((T + 1) T j = 0 mod T, and the
// 32 / T offsets are distinct mod 32 for T = 2..16), consecutive rows do
// not.  So in stages whose groups have at least 32 consecutive n1, the low
// five bits of the group index are transposed (32 / T x T -> T x 32 / T)
// before n1 is taken from them: a permutation of the groups, not of the
// work.
__device__ __forceinline__ int rotate_rows(int rest, int logT) {
    const int logr = 5 - logT;
    const int j = rest & ((1 << logr) - 1);
    const int k = (rest >> logr) & ((1 << logT) - 1);
    return (rest & ~31) | (j << logT) | k;
}

__device__ __forceinline__ int ilog2_if_pow2(int x) {
    return (x & (x - 1)) ? -1 : 31 - __clz(x);
}

// Splits g into (t, rest) = (g % T, g / T) and returns the base address of
// transform t; shifts when T and tm are powers of two.
__device__ __forceinline__ uint32_t *group_base(const TileMap &m, int lT, int ltm, int g, int &rest) {
    int t;
    if (lT >= 0) {
        t = g & (m.T - 1);
        rest = g >> lT;
    } else {
        t = g % m.T;
        rest = g / m.T;
    }
    const int t0 = ltm >= 0 ? (t & (m.tm - 1)) : t % m.tm;
    const int t1 = ltm >= 0 ? (t >> ltm) : t / m.tm;
    return m.s + t0 * m.ta + t1 * m.tb;
}

// One forward stage of radix R at sub-block length Lc = 2^logLc (L = 2^logL).
// tw: table of omega_T^e (T = 2^logT), T a multiple of L.
// HZ: the second half of every group's inputs is zero (not read).
// Where a stage's outputs go: back to the tile (the default), or, for the
// last stage of a transform, to any destination put(address in the tile,
// transform t, element n, value) chooses.
struct TileOut {
    __device__ __forceinline__ void put(uint32_t *a, int, int, uint32_t v) const { *a = v; }
};

template <int R, int SM, bool HZ = false, class Out = TileOut>
__device__ __forceinline__ void stage_dif(const TileMap &M, int logL, int logLc,
                                          const uint2 *__restrict__ tw, int logT, uint32_t p,
                                          uint32_t p2, const Out &out = Out()) {
    constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    Roots<R> rt;
    load_roots<R, SM>(rt, tw, logT);
    const int logLp = logLc - LR;
    const int Lp = 1 << logLp;
    const int total = M.T << (logL - LR);
    const int tsh = logT - logLc;
    const int lT = ilog2_if_pow2(M.T), ltm = ilog2_if_pow2(M.tm);
    const int st = padded(M, Lp) * M.es;
    const bool rot = M.rot && logLp >= 5;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        int rest;
        uint32_t *tb = group_base(M, lT, ltm, g, rest);
        if (rot) rest = rotate_rows(rest, M.rot);
        const int n1 = rest & (Lp - 1);
        const int blk = rest >> logLp;
        uint32_t *base = tb + padded(M, (blk << logLc) + n1) * M.es;
        uint32_t x[R];
        if (Lp > 1) {
            // twiddles omega_Lc^{n1 k2} first: their latency hides behind the
            // DFT; entry n1 k2 2^tsh of the table is step * k2 for a per-group step
            const uint2 *wb = tw;
            const uint32_t step = (uint32_t)n1 << tsh;
            uint2 w[R];
            w[0] = make_uint2(1u, 0u);  // unused: output 0 carries no twiddle
#pragma unroll
            for (int m = 1; m < R; ++m)
                w[m] = SM == TW_STAGE ? wb[m * Lp + n1] : tload<SM>(wb + step * (uint32_t)brev_c<R>(m));
#pragma unroll
            for (int m = 0; m < (HZ ? R / 2 : R); ++m) x[m] = base[m * st];
            dft_dif_tw<R, HZ>(x, rt, w, p, p2);
        } else {  // last stage: every twiddle is 1
#pragma unroll
            for (int m = 0; m < (HZ ? R / 2 : R); ++m) x[m] = base[m * st];
            if (HZ)
                dft_dif_hz<R>(x, rt, p, p2);
            else
                dft_dif<R>(x, rt, p, p2);
        }
        const int t = lT >= 0 ? (g & (M.T - 1)) : g % M.T;
        const int n0 = (blk << logLc) + n1;
#pragma unroll
        for (int m = 0; m < R; ++m) out.put(base + m * st, t, n0 + m * Lp, x[m]);
    }
    __syncthreads();
}

// Where a stage's inputs come from: the tile (the default), or, for the
// first stage of an inverse transform, any value get(address in the tile,
// transform t, element n) makes of the tile's entry.
struct TileIn {
    __device__ __forceinline__ uint32_t get(const uint32_t *a, int, int) const { return *a; }
};

template <int R, int SM, class In = TileIn, class Out = TileOut>
__device__ __forceinline__ void stage_dit(const TileMap &M, int logL, int logLc,
                                          const uint2 *__restrict__ tw, int logT, uint32_t p,
                                          uint32_t p2, const In &in = In(), const Out &out = Out()) {
    constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    Roots<R> rt;
    load_roots<R, SM>(rt, tw, logT);
    const int logLp = logLc - LR;
    const int Lp = 1 << logLp;
    const int total = M.T << (logL - LR);
    const int tsh = logT - logLc;
    const int lT = ilog2_if_pow2(M.T), ltm = ilog2_if_pow2(M.tm);
    const int st = padded(M, Lp) * M.es;
    const bool rot = M.rot && logLp >= 5;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        int rest;
        uint32_t *tb = group_base(M, lT, ltm, g, rest);
        if (rot) rest = rotate_rows(rest, M.rot);
        const int n1 = rest & (Lp - 1);
        const int blk = rest >> logLp;
        uint32_t *base = tb + padded(M, (blk << logLc) + n1) * M.es;
        uint32_t x[R];
        if (Lp > 1) {
            const uint32_t step = (uint32_t)n1 << tsh;
            uint2 w[R];
#pragma unroll
            for (int m = 1; m < R; ++m)
                w[m] = SM == TW_STAGE ? tw[m * Lp + n1] : tload<SM>(tw + step * (uint32_t)brev_c<R>(m));
#pragma unroll
            for (int m = 0; m < R; ++m) x[m] = base[m * st];
#pragma unroll
            for (int m = 1; m < R; ++m) x[m] = shoup(x[m], w[m], p);
        } else {  // first inverse stage: every twiddle is 1
            const int t = lT >= 0 ? (g & (M.T - 1)) : g % M.T;
            const int n0 = blk << logLc;
#pragma unroll
            for (int m = 0; m < R; ++m) x[m] = in.get(base + m * st, t, n0 + m);
        }
        dft_dit<R>(x, rt, p, p2);
        const int t = lT >= 0 ? (g & (M.T - 1)) : g % M.T;
        const int n0 = (blk << logLc) + n1;
#pragma unroll
        for (int m = 0; m < R; ++m) out.put(base + m * st, t, n0 + m * Lp, x[m]);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Radix-16 stages on the INT8 tensor cores (IPM_TENSOR_STAGES).
//
// A radix-16 DFT over Z/p is the product of a 16 x 16 matrix E (powers of
// omega_16; rows in the order the stage leaves its outputs: forward
// E[m][k] = omega^{brev(m) k}, inverse E[n][m] = omega^{-n brev(m)}) with
// each input vector x.  Split every input word into bytes,
// x_k = sum_s x_k^(s) 2^(8s), and every constant C[j][k][s] =
// E[j][k] 2^(8s) 2^32 mod p into bytes as well, C = sum_l C^(l) 2^(8l).
// Then
//     V_j = sum_l 2^(8l) D_l[j],  D_l[j] = sum_{k,s} C^(l)[j][k][s] x_k^(s),
// is congruent to 2^32 sum_k E[j][k] x_k modulo p, and every D_l is the
// product of a 16 x 64 byte matrix with the 64 bytes of x: an unsigned
// 8-bit matrix product with 32-bit accumulation, exact because
// D_l <= 64 * 255^2 < 2^22.  So V < 2^46 < p 2^32, and one Montgomery
// reduction returns sum_k E[j][k] x_k mod p in [0, 2p): the same residue
// the register stage computes, with no rounding anywhere.
//
// mma.sync m16n8k32 .u8: a warp multiplies 8 vectors at once.  Lane
// (g, q) = (lane / 4, lane % 4) supplies, as its B fragment, words
// x_{q + 4i} (i < 4) of vector g read straight from the tile -- the bytes
// of a little-endian word are the K-dimension entries 4k + s in order --
// and receives D_l[j] of vectors 2q, 2q + 1 for rows j = g, g + 8.  The A
// fragments (the byte slices C^(l)) are precomputed per prime and
// direction: word ((l * 32 + lane) * 8 + c * 4 + i) of a 1024-word table
// is register i of K-chunk c (inputs 8c .. 8c + 7) of slice l.
// ---------------------------------------------------------------------------

struct NoTc {
    static constexpr bool on = false;
};
// The fragment tables of one prime (forward and inverse matrix) and
// -p^{-1} mod 2^32.
struct TcOn {
    static constexpr bool on = true;
    const uint32_t *fwd, *inv;
    uint32_t mont;
};

__device__ __forceinline__ void mma_u8_m16n8k32(uint32_t (&d)[4], uint4 a, uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// Group g of a stage: its first element's address, transform t, and n1.
struct StageGroup {
    uint32_t *base;
    int t, n0, n1;  // n0: index of the group's first element in transform t
};
__device__ __forceinline__ StageGroup stage_group(const TileMap &M, int lT, int ltm, bool rot, int logLp, int logLc,
                                                  int g) {
    int rest;
    uint32_t *tb = group_base(M, lT, ltm, g, rest);
    if (rot) rest = rotate_rows(rest, M.rot);
    const int n1 = rest & ((1 << logLp) - 1);
    const int blk = rest >> logLp;
    StageGroup G;
    G.base = tb + padded(M, (blk << logLc) + n1) * M.es;
    G.t = lT >= 0 ? (g & (M.T - 1)) : g % M.T;
    G.n0 = (blk << logLc) + n1;
    G.n1 = n1;
    return G;
}

// One radix-16 stage (the same groups, twiddles and output order as
// stage_dif<16> when FWD, stage_dit<16> otherwise) on the tensor cores.
// HZ: inputs 8..15 of every group are zero (forward only): one K-chunk.
template <bool FWD, bool HZ, int SM, class In = TileIn, class Out = TileOut>
__device__ __forceinline__ void stage_tc16(const TileMap &M, int logL, int logLc, const uint2 *__restrict__ tw,
                                           int logT, uint32_t p, const TcOn &tc, const In &in = In(),
                                           const Out &out = Out()) {
    const int logLp = logLc - 4;
    const int Lp = 1 << logLp;
    const int total = M.T << (logL - 4);
    const int tsh = logT - logLc;
    const int lT = ilog2_if_pow2(M.T), ltm = ilog2_if_pow2(M.tm);
    const int st = padded(M, Lp) * M.es;
    const bool rot = M.rot && logLp >= 5;
    const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const uint4 *fr = reinterpret_cast<const uint4 *>(FWD ? tc.fwd : tc.inv) + 2 * lane;
    for (int g0 = (int)(threadIdx.x >> 5) * 8; g0 < total; g0 += (int)(blockDim.x >> 5) * 8) {
        uint32_t b[4] = {0u, 0u, 0u, 0u};
        if (g0 + gq < total) {
            const StageGroup G = stage_group(M, lT, ltm, rot, logLp, logLc, g0 + gq);
            const uint32_t step = (uint32_t)G.n1 << tsh;
#pragma unroll
            for (int i = 0; i < (HZ ? 2 : 4); ++i) {
                const int k = tq + 4 * i;
                if (FWD)
                    b[i] = G.base[k * st];
                else if (Lp > 1)  // inverse: the twiddle omega_Lc^{-n1 brev(k)} first
                    b[i] = shoup(G.base[k * st],
                                 SM == TW_STAGE ? tw[k * Lp + G.n1] : tload<SM>(tw + step * bitrev((uint32_t)k, 4)),
                                 p);
                else
                    b[i] = in.get(G.base + k * st, G.t, G.n0 + k);
            }
        }
        uint32_t d[4][4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            d[l][0] = d[l][1] = d[l][2] = d[l][3] = 0u;
            mma_u8_m16n8k32(d[l], __ldg(fr + 64 * l), b[0], b[1]);
            if (!HZ) mma_u8_m16n8k32(d[l], __ldg(fr + 64 * l + 1), b[2], b[3]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int g = g0 + 2 * tq + h;
            if (g >= total) continue;
            const StageGroup G = stage_group(M, lT, ltm, rot, logLp, logLc, g);
            const uint32_t step = (uint32_t)G.n1 << tsh;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int m = gq + 8 * u, e = 2 * u + h;
                const uint32_t lo = d[0][e] + (d[1][e] << 8);  // < 2^31
                const uint32_t hi = d[2][e] + (d[3][e] << 8);
                uint32_t v = redc64((uint64_t)hi * 65536u + lo, p, tc.mont);
                if (FWD && Lp > 1)
                    v = shoup(v, SM == TW_STAGE ? tw[m * Lp + G.n1] : tload<SM>(tw + step * bitrev((uint32_t)m, 4)),
                              p);
                out.put(G.base + m * st, G.t, G.n0 + m * Lp, v);
            }
        }
    }
    __syncthreads();
}

// Radix sequence: logL is split into ceil(logL/4) stages of at most 4 bits
// (radix 16), as even as possible, the larger stages first.
__device__ __forceinline__ void stage_split(int logL, int &nst, int &base, int &extra) {
    nst = (logL + 3) / 4;
    base = nst ? logL / nst : 0;
    extra = nst ? logL % nst : 0;
}

template <bool FWD, int SM, class TC = NoTc>
__device__ __forceinline__ void run_stage(int b, const TileMap &M, int logL, int logLc,
                                          const uint2 *__restrict__ tw, int logT, uint32_t p,
                                          uint32_t p2, bool hz = false, const TC &tc = TC()) {
    if constexpr (TC::on) {
        if (b == 4) {
            if (FWD && hz)
                stage_tc16<true, true, SM>(M, logL, logLc, tw, logT, p, tc);
            else
                stage_tc16<FWD, false, SM>(M, logL, logLc, tw, logT, p, tc);
            return;
        }
    }
    if (FWD && hz) {
        switch (b) {
            case 1: stage_dif<2, SM, true>(M, logL, logLc, tw, logT, p, p2); return;
            case 2: stage_dif<4, SM, true>(M, logL, logLc, tw, logT, p, p2); return;
            case 3: stage_dif<8, SM, true>(M, logL, logLc, tw, logT, p, p2); return;
            default: stage_dif<16, SM, true>(M, logL, logLc, tw, logT, p, p2); return;
        }
    }
    switch (b) {
        case 1: FWD ? stage_dif<2, SM>(M, logL, logLc, tw, logT, p, p2) : stage_dit<2, SM>(M, logL, logLc, tw, logT, p, p2); break;
        case 2: FWD ? stage_dif<4, SM>(M, logL, logLc, tw, logT, p, p2) : stage_dit<4, SM>(M, logL, logLc, tw, logT, p, p2); break;
        case 3: FWD ? stage_dif<8, SM>(M, logL, logLc, tw, logT, p, p2) : stage_dit<8, SM>(M, logL, logLc, tw, logT, p, p2); break;
        default: FWD ? stage_dif<16, SM>(M, logL, logLc, tw, logT, p, p2) : stage_dit<16, SM>(M, logL, logLc, tw, logT, p, p2); break;
    }
}

// The last stage of a forward transform, radix 2^b, writing through out.
template <bool SM, class Out, class TC = NoTc>
__device__ __forceinline__ void last_stage_out(int b, bool hz, const TileMap &M, int logL, int logLc,
                                               const uint2 *__restrict__ tw, int logT, uint32_t p, uint32_t p2,
                                               const Out &out, const TC &tc = TC()) {
    if constexpr (TC::on) {
        if (b == 4) {
            if (hz)
                stage_tc16<true, true, SM>(M, logL, logLc, tw, logT, p, tc, TileIn(), out);
            else
                stage_tc16<true, false, SM>(M, logL, logLc, tw, logT, p, tc, TileIn(), out);
            return;
        }
    }
    if (hz) {
        switch (b) {
            case 1: stage_dif<2, SM, true>(M, logL, logLc, tw, logT, p, p2, out); return;
            case 2: stage_dif<4, SM, true>(M, logL, logLc, tw, logT, p, p2, out); return;
            case 3: stage_dif<8, SM, true>(M, logL, logLc, tw, logT, p, p2, out); return;
            default: stage_dif<16, SM, true>(M, logL, logLc, tw, logT, p, p2, out); return;
        }
    }
    switch (b) {
        case 1: stage_dif<2, SM, false>(M, logL, logLc, tw, logT, p, p2, out); return;
        case 2: stage_dif<4, SM, false>(M, logL, logLc, tw, logT, p, p2, out); return;
        case 3: stage_dif<8, SM, false>(M, logL, logLc, tw, logT, p, p2, out); return;
        default: stage_dif<16, SM, false>(M, logL, logLc, tw, logT, p, p2, out); return;
    }
}

// ntt_forward whose last stage hands every output to out.put instead of
// writing it back to the tile (a length-1 transform hands over its input).
template <bool SM = false, class Out, class TC = NoTc>
__device__ __forceinline__ void ntt_forward_out(const TileMap &M, int logL, const uint2 *__restrict__ tw,
                                                int logT, uint32_t p, uint32_t p2, bool upper_zero,
                                                const Out &out, const TC &tc = TC()) {
    int nst, base, extra;
    stage_split(logL, nst, base, extra);
    if (nst == 0) {
        for (int t = threadIdx.x; t < M.T; t += blockDim.x) {
            uint32_t *a = M.s + (t % M.tm) * M.ta + (t / M.tm) * M.tb;
            out.put(a, t, 0, *a);
        }
        __syncthreads();
        return;
    }
    int logLc = logL;
    for (int i = 0; i + 1 < nst; ++i) {
        const int b = base + (i < extra ? 1 : 0);
        run_stage<true, SM>(b, M, logL, logLc, tw, logT, p, p2, upper_zero && i == 0, tc);
        logLc -= b;
    }
    last_stage_out<SM>(base + (nst - 1 < extra ? 1 : 0), upper_zero && nst == 1, M, logL, logLc, tw, logT, p, p2,
                       out, tc);
}

// Full forward transform of length 2^logL on every transform of the map
// (natural order in, bit-reversed order out).  Values in [0, 2p).
// upper_zero: the second half of every transform's input is zero and is
// not read (the zero padding of an acyclic convolution).
template <bool SM = false, class TC = NoTc>
__device__ __forceinline__ void ntt_forward(const TileMap &M, int logL, const uint2 *__restrict__ tw,
                                            int logT, uint32_t p, uint32_t p2, bool upper_zero = false,
                                            const TC &tc = TC()) {
    int nst, base, extra;
    stage_split(logL, nst, base, extra);
    int logLc = logL;
    for (int i = 0; i < nst; ++i) {
        const int b = base + (i < extra ? 1 : 0);
        run_stage<true, SM>(b, M, logL, logLc, tw, logT, p, p2, upper_zero && i == 0, tc);
        logLc -= b;
    }
}

// The middle of a convolution in one register pass: the last forward stage
// (radix R, L' = 1) of A and of B, the pointwise product A*B*2^-32
// (Montgomery), and the first inverse stage, for each group of R
// consecutive elements; the product is written over A.
template <int R, int SM>
__device__ __forceinline__ void stage_fused_pointwise(const TileMap &MA, const TileMap &MB, int logL,
                                                      const uint2 *__restrict__ twf,
                                                      const uint2 *__restrict__ twi, int logT,
                                                      uint32_t p, uint32_t p2, uint32_t mont) {
    constexpr int LR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
    Roots<R> rf, ri;
    load_roots<R, SM>(rf, twf, logT);
    load_roots<R, SM>(ri, twi, logT);
    const int total = MA.T << (logL - LR);
    const int lT = ilog2_if_pow2(MA.T), ltm = ilog2_if_pow2(MA.tm);
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        int blk;
        // group_base sets blk: the offsets are added in separate statements
        uint32_t *ba = group_base(MA, lT, ltm, g, blk);
        ba += padded(MA, blk << LR) * MA.es;
        uint32_t *bb = group_base(MB, lT, ltm, g, blk);
        bb += padded(MB, blk << LR) * MB.es;
        uint32_t xa[R], xb[R];
#pragma unroll
        for (int m = 0; m < R; ++m) {
            xa[m] = ba[m * MA.es];
            xb[m] = bb[m * MB.es];
        }
        dft_dif<R>(xa, rf, p, p2);
        dft_dif<R>(xb, rf, p, p2);
#pragma unroll
        for (int m = 0; m < R; ++m) xa[m] = montmul(xa[m], xb[m], p, mont);
        dft_dit<R>(xa, ri, p, p2);
#pragma unroll
        for (int m = 0; m < R; ++m) ba[m * MA.es] = xa[m];
    }
    __syncthreads();
}

// Convolution core on two sets of transforms: forward A and B (all but the
// last stage each; A may be run before B's data are ready -- wait_b is
// called in between), the fused last/pointwise/first-inverse stage, then
// the remaining inverse stages on A.
//
// Twiddles.  COMPACT = false: every stage reads omega_T^{+-e} from twf /
// twi (T = 2^logT, a multiple of 2^logL), stage i at stride T / Lc_i;
// SM says whether that table is in shared memory.  COMPACT = true: twf
// points at one block per stage in shared memory, back to back (stage_block
// gives the layout): stage i's forward entries in the TW_STAGE layout
// (Lc_i twiddles, then R_i root slots), then its inverse entries (twi and
// logT are unused).
//
// The last inverse stage hands its outputs to out.put; the return value says
// whether it did (false when the transform has fewer than two stages: the
// results are then in MA's tile).
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};
// step(pass, i) runs after register stage i of the forward transform of A
// (pass 0) or B (pass 1), and after every inverse stage i > 0 (pass 2, i
// counting down): a caller may issue copies there.
struct NoStep {
    __device__ __forceinline__ void operator()(int, int) const {}
};

// after_fused() runs once B's tile is no longer read (after the pointwise
// stage and its barrier), before the inverse stages: a caller may start
// refilling B's memory there.
template <bool SM, bool COMPACT, typename WaitB, class Out = TileOut, class TC = NoTc, class Hook = NoHook,
          class Step = NoStep>
__device__ __forceinline__ bool ntt_convolve(const TileMap &MA, const TileMap &MB, int logL,
                                             const uint2 *__restrict__ twf, const uint2 *__restrict__ twi,
                                             int logT, uint32_t p, uint32_t p2, uint32_t mont, WaitB wait_b,
                                             const Out &out = Out(), const TC &tc = TC(),
                                             const Hook &after_fused = Hook(), const Step &step = Step()) {
    constexpr int MODE = COMPACT ? TW_STAGE : SM ? TW_SHARED : TW_GLOBAL;
    int nst, base, extra;
    stage_split(logL, nst, base, extra);
    if (nst == 0) {  // length 1: the product of the single values
        wait_b();
        for (int t = threadIdx.x; t < MA.T; t += blockDim.x) {
            int rest;
            uint32_t *a = group_base(MA, ilog2_if_pow2(MA.T), ilog2_if_pow2(MA.tm), t, rest);
            uint32_t *b = group_base(MB, ilog2_if_pow2(MB.T), ilog2_if_pow2(MB.tm), t, rest);
            *a = montmul(*a, *b, p, mont);
        }
        __syncthreads();
        after_fused();
        return false;
    }
    // stage at block offset toff (radix 2^b, sub-block length 2^logLc):
    // tables (tf, ti, lg); a stage block holds 2 (Lc + R) entries
    auto tables = [&](int toff, int logLc, int b, const uint2 *&tf, const uint2 *&ti, int &lg) {
        if (COMPACT) {
            tf = twf + toff;
            ti = tf + (1 << logLc) + (1 << b);
            lg = logLc;
        } else {
            tf = twf;
            ti = twi;
            lg = logT;
        }
    };
    const uint2 *tf, *ti;
    int lg;
    for (int pass = 0; pass < 2; ++pass) {
        const TileMap &M = pass ? MB : MA;
        if (pass) wait_b();
        int logLc = logL, toff = 0;
        for (int i = 0; i + 1 < nst; ++i) {
            const int b = base + (i < extra ? 1 : 0);
            tables(toff, logLc, b, tf, ti, lg);
            run_stage<true, MODE>(b, M, logL, logLc, tf, lg, p, p2, false, tc);
            step(pass, i);
            toff += 2 * ((1 << logLc) + (1 << b));
            logLc -= b;
        }
    }
    // the last stage (length 2^blast); its block follows the earlier ones
    const int blast = base + (nst - 1 < extra ? 1 : 0);
    int toff = 0;
    {
        int logLc = logL;
        for (int i = 0; i + 1 < nst; ++i) {
            const int b = base + (i < extra ? 1 : 0);
            toff += 2 * ((1 << logLc) + (1 << b));
            logLc -= b;
        }
    }
    tables(toff, blast, blast, tf, ti, lg);
    switch (blast) {
        case 1: stage_fused_pointwise<2, MODE>(MA, MB, logL, tf, ti, lg, p, p2, mont); break;
        case 2: stage_fused_pointwise<4, MODE>(MA, MB, logL, tf, ti, lg, p, p2, mont); break;
        case 3: stage_fused_pointwise<8, MODE>(MA, MB, logL, tf, ti, lg, p, p2, mont); break;
        default: stage_fused_pointwise<16, MODE>(MA, MB, logL, tf, ti, lg, p, p2, mont); break;
    }
    after_fused();
    int logLc = blast;
    for (int i = nst - 2; i >= 0; --i) {
        const int b = base + (i < extra ? 1 : 0);
        logLc += b;
        toff -= 2 * ((1 << logLc) + (1 << b));  // stage i's block precedes stage i+1's
        tables(toff, logLc, b, tf, ti, lg);
        if (i > 0) {
            run_stage<false, MODE>(b, MA, logL, logLc, ti, lg, p, p2, false, tc);
            step(2, i);
        } else {  // the last inverse stage
            const TileIn in;
            if constexpr (TC::on) {
                if (b == 4) {
                    stage_tc16<false, false, MODE>(MA, logL, logLc, ti, lg, p, tc, in, out);
                    continue;
                }
            }
            switch (b) {
                case 1: stage_dit<2, MODE>(MA, logL, logLc, ti, lg, p, p2, in, out); break;
                case 2: stage_dit<4, MODE>(MA, logL, logLc, ti, lg, p, p2, in, out); break;
                case 3: stage_dit<8, MODE>(MA, logL, logLc, ti, lg, p, p2, in, out); break;
                default: stage_dit<16, MODE>(MA, logL, logLc, ti, lg, p, p2, in, out); break;
            }
        }
    }
    return nst >= 2;
}

// Inverse of ntt_forward up to the factor 2^logL (tw: inverse table): the
// forward stages replayed backwards.
template <bool SM = false, class TC = NoTc>
__device__ __forceinline__ void ntt_inverse(const TileMap &M, int logL, const uint2 *__restrict__ tw,
                                            int logT, uint32_t p, uint32_t p2, const TC &tc = TC()) {
    int nst, base, extra;
    stage_split(logL, nst, base, extra);
    int logLc = 0;
    for (int i = nst - 1; i >= 0; --i) {
        const int b = base + (i < extra ? 1 : 0);
        logLc += b;
        run_stage<false, SM>(b, M, logL, logLc, tw, logT, p, p2, false, tc);
    }
}

// ntt_inverse whose first stage reads every input through in.get (a
// length-1 transform writes in.get of its input back to the tile).
template <bool SM = false, class In, class TC = NoTc>
__device__ __forceinline__ void ntt_inverse_in(const TileMap &M, int logL, const uint2 *__restrict__ tw,
                                               int logT, uint32_t p, uint32_t p2, const In &in,
                                               const TC &tc = TC()) {
    int nst, base, extra;
    stage_split(logL, nst, base, extra);
    if (nst == 0) {
        for (int t = threadIdx.x; t < M.T; t += blockDim.x) {
            uint32_t *a = M.s + (t % M.tm) * M.ta + (t / M.tm) * M.tb;
            *a = in.get(a, t, 0);
        }
        __syncthreads();
        return;
    }
    int logLc = 0;
    for (int i = nst - 1; i >= 0; --i) {
        const int b = base + (i < extra ? 1 : 0);
        logLc += b;
        if (i == nst - 1) {  // the first inverse stage (every twiddle is 1)
            if constexpr (TC::on) {
                if (b == 4) {
                    stage_tc16<false, false, SM>(M, logL, logLc, tw, logT, p, tc, in);
                    continue;
                }
            }
            switch (b) {
                case 1: stage_dit<2, SM>(M, logL, logLc, tw, logT, p, p2, in); break;
                case 2: stage_dit<4, SM>(M, logL, logLc, tw, logT, p, p2, in); break;
                case 3: stage_dit<8, SM>(M, logL, logLc, tw, logT, p, p2, in); break;
                default: stage_dit<16, SM>(M, logL, logLc, tw, logT, p, p2, in); break;
            }
        } else {
            run_stage<false, SM>(b, M, logL, logLc, tw, logT, p, p2, false, tc);
        }
    }
}

}  // namespace ipm
