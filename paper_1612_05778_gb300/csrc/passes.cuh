// passes.cuh -- the tile functions of the three passes of one product
// (and the outer pass of split plans), shared by the integer-stage
// kernels (ipm_kernels.cu) and the tensor-core-stage kernels
// (ipm_kernels_tc.cu).  Index conventions are those of ipm_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include "ipm_internal.h"
#include "modarith.cuh"
#include "ntt_stages.cuh"

namespace ipm {

// The tensor-core stage tables of prime t (TcOn), or nothing (NoTc): tile
// functions templated on TC run every radix-16 stage on the INT8 tensor
// cores when TC = TcOn.
__device__ __forceinline__ void tc_prime(NoTc &, const KParams &, int) {}
__device__ __forceinline__ void tc_prime(TcOn &tc, const KParams &P, int t) {
    tc.fwd = P.tcfrag + (size_t)t * TC_FRAG_WORDS;
    tc.inv = tc.fwd + TC_FRAG_WORDS / 2;
    tc.mont = P.pc[t].mont;
}

// ---------------------------------------------------------------------------
// Pass 1
// ---------------------------------------------------------------------------

// Pass 1's output: step-B twiddle of row pos, full reduction, store to row
// (pos, i1) of the workspace.
struct FwdStore {
    uint32_t *Zt;
    const uint2 *tw_rows;
    size_t i1, Y1;
    int twoK;
    uint32_t p;
    __device__ __forceinline__ void put(uint32_t *, int col, int pos, uint32_t v) const {
        Zt[((size_t)pos * Y1 + i1) * twoK + col] = red(shoup(v, tw_rows[pos], p), p);
    }
};

// Pass 1 on one tile: rows i = i1 + Y1*i2 (i2 < Y2) of operand op.
template <class TC, int CK = 0, int CLY2 = 0, int CM = 0>
__device__ __forceinline__ void fwd_tile(const KParams &P, int64_t i1, int op,
                                         const uint32_t *__restrict__ a, const uint8_t *__restrict__ an,
                                         const uint32_t *__restrict__ b, const uint8_t *__restrict__ bn) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t *X = op ? b : a;
    const uint8_t *Xn = op ? bn : an;
    const int64_t nX = op ? P.nb : P.na;
    const int L = op ? P.lb : P.la;
    const uint32_t bits = op ? P.bits_b : P.bits_a;
    // CK, CLY2, CM > 0: the plan's K, log2 Y2 and M as compile-time
    // constants (the launcher checks that they match): strides, stage
    // radices and digit positions fold into the instructions
    const int K = CK ? CK : P.K, logK = CK ? clog2(CK) : P.logK, M = CM ? CM : P.M;
    const int logY2 = CLY2 ? CLY2 : P.logY2;
    const int Y2 = 1 << logY2;
    const int twoK = 2 * K;
    const int pitch = twoK + 1;  // odd row pitch: column walks hit distinct banks
    int64_t *dig = reinterpret_cast<int64_t *>(smem);            // [Y2][K]
    // two sets of per-prime tables (prime t in set t & 1, the next prime's
    // copied while this one is transformed): theta^j (j < K), omega_Y^{i1
    // k2(pos)} (pos < Y2), omega_K^e = theta^2e (e < K), omega_Y2^e (e < Y2)
    uint2 *tw_sets = reinterpret_cast<uint2 *>(dig + (size_t)Y2 * K);
    const int set_len = 2 * (K + Y2);
    uint8_t *signs = reinterpret_cast<uint8_t *>(tw_sets + 2 * set_len);  // sign of row i2
    uint32_t *tile = reinterpret_cast<uint32_t *>(signs + ((Y2 + 15) & ~15));  // [Y2][pitch]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint64_t mmask = (1ull << M) - 1;
    const uint64_t halfM = 1ull << (M - 1);
    auto prefetch_tables = [&](int t) {
        const PrimeConst &pq = P.pc[t];
        uint2 *set = tw_sets + (t & 1) * set_len;
        for (int j = threadIdx.x; j < K; j += blockDim.x) {
            cp_async8(set + j, pq.tx_f + j);
            cp_async8(set + K + Y2 + j, pq.tx_f + 2 * j);
        }
        for (int q = threadIdx.x; q < Y2; q += blockDim.x) {
            cp_async8(set + K + q, pq.ty_f + (size_t)i1 * bitrev((uint32_t)q, logY2));
            cp_async8(set + 2 * K + Y2 + q, pq.ty_f + ((size_t)q << (P.logY - logY2)));
        }
        cp_async_commit();
    };

    // 1. Balanced base-2^M digits of every row (one warp per row).  Digits
    //    j < K-1 follow the carry rule t = u_j + carry, digit = t - 2^M and
    //    carry 1 when t >= 2^(M-1); the top digit is the signed top field
    //    plus the carry.  The carry chain is resolved with ballots: with
    //    generate g_j = [u_j >= 2^(M-1)] and propagate q_j = [u_j = 2^(M-1)-1]
    //    the carries into every digit are (g + (g|q)) xor q (carry-lookahead
    //    by integer addition), 32 digits per ballot word.
    // rows i2 < nr hold coefficients (i = i1 + Y1*i2 < nX); the rest are the
    // zero padding of the acyclic y-convolution
    const int64_t Y1 = P.Y1;
    const int nr = i1 < nX ? (int)min((int64_t)Y2, (nX - i1 + Y1 - 1) / Y1) : 0;
    // 0. stage the magnitude limbs of the non-zero rows (L <= 2K < pitch, so
    //    row i2 fits at tile + i2 * pitch), all loads in flight at once
    for (int e = threadIdx.x; e < nr * L; e += blockDim.x) {
        const int i2 = e / L, l = e - i2 * L;
        cp_async4(tile + (size_t)i2 * pitch + l, X + (size_t)(i1 + Y1 * i2) * L + l);
    }
    cp_async_commit();
    prefetch_tables(0);  // the first prime's tables fly during the digit split
    for (int i2 = threadIdx.x; i2 < nr; i2 += blockDim.x) signs[i2] = Xn[i1 + Y1 * i2];
    cp_async_wait<1>();  // the limbs
    __syncthreads();
    for (int i2 = warp; i2 < Y2; i2 += nw) {
        int64_t *drow = dig + (size_t)i2 * K;
        if (i2 >= nr) {
            for (int j = lane; j < K; j += 32) drow[j] = 0;
            continue;
        }
        uint32_t *row = tile + (size_t)i2 * pitch;
        int f = L;
        for (int c0 = 0; c0 < L; c0 += 32) {
            const int l = c0 + lane;
            const uint32_t v = l < L ? row[l] : 0u;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0u);
            if (m && f == L) f = c0 + __ffs(m) - 1;
        }
        if (lane == 0 && (bits & 31u) && (row[L - 1] >> (bits & 31u)))
            atomicOr(P.err, ERRBIT_BOUND);
        const bool neg = signs[i2] != 0 && f < L;
        // N-bit two's complement in place: zero below the lowest non-zero
        // limb f, -x at f, ~x above; limbs beyond L are the sign extension
        if (neg)
            for (int l = lane; l < L; l += 32) {
                const uint32_t v = row[l];
                row[l] = l < f ? 0u : (l == f ? 0u - v : ~v);
            }
        __syncwarp();
        const uint32_t ext = neg ? 0xffffffffu : 0u;
        unsigned carry_in = 0;
        for (int j0 = 0; j0 < K; j0 += 32) {
            const int j = j0 + lane;
            uint64_t u = 0;
            if (j < K) {
                const int64_t bit = (int64_t)M * j;
                const int l0 = (int)(bit >> 5), sh = (int)(bit & 31);
                const uint64_t lo = (uint64_t)(l0 < L ? row[l0] : ext) |
                                    ((uint64_t)(l0 + 1 < L ? row[l0 + 1] : ext) << 32);
                uint64_t v = lo >> sh;
                if (sh + M > 64) v |= (uint64_t)(l0 + 2 < L ? row[l0 + 2] : ext) << (64 - sh);
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

    for (int t = 0; t < P.r; ++t) {
        const PrimeConst &pc = P.pc[t];
        const uint32_t p = pc.p, p2 = pc.p2;
        const uint2 one = make_uint2(1u, pc.one_s), c32 = make_uint2(pc.c32, pc.c32_s);
        TC tc{};
        tc_prime(tc, P, t);
        // this prime's tables in shared memory (the transforms' twiddles are
        // read by every warp as broadcasts, whatever their stride); the next
        // prime's are copied meanwhile
        if (t + 1 < P.r) {
            prefetch_tables(t + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const uint2 *tw_twist = tw_sets + (t & 1) * set_len;
        const uint2 *tw_rows = tw_twist + K;
        const uint2 *tw_x = tw_rows + Y2;
        const uint2 *tw_y = tw_x + K;
        // 2. residues (cyclic half) and twisted residues theta^j a_ij (negacyclic half)
        for (int e = threadIdx.x; e < nr * K; e += blockDim.x) {
            const int i2 = e >> logK, j = e & (K - 1);
            const int64_t d = dig[e];
            const uint64_t ad = d < 0 ? (uint64_t)(-d) : (uint64_t)d;
            uint32_t r = shoup((uint32_t)(ad >> 32), c32, p) + shoup((uint32_t)ad, one, p);
            r = red(red(r, p2), p);
            if (d < 0 && r) r = p - r;
            uint32_t *trow = tile + (size_t)i2 * pitch;
            trow[j] = r;
            trow[K + j] = shoup(r, tw_twist[j], p);
        }
        // rows nr.. are zero padding; when they cover the upper half the first
        // y stage does not read that half at all
        const bool upper_zero = Y2 >= 2 && 2 * nr <= Y2;
        const int zlim = upper_zero ? Y2 / 2 : Y2;
        for (int e = threadIdx.x; e < (zlim - nr) * twoK; e += blockDim.x) {
            const int i2 = nr + (e >> (logK + 1)), col = e & (twoK - 1);
            tile[(size_t)i2 * pitch + col] = 0u;
        }
        __syncthreads();
        // 3. x-DFTs of length K on both halves of the non-zero rows (omega_K = theta^2)
        if (CLY2 && nr == Y2 / 2) {  // the usual tile (half the rows hold coefficients): constant map
            const TileMap xm{tile, Y2, Y2 / 2, pitch, K, 1};
            ntt_forward<true>(xm, logK, tw_x, logK, p, p2, false, tc);
        } else if (nr > 0) {
            const TileMap xm{tile, 2 * nr, nr, pitch, K, 1};
            ntt_forward<true>(xm, logK, tw_x, logK, p, p2, false, tc);
        }
        // 4. y step A: length-Y2 DFT down every column; its last stage applies
        //    the step-B twiddle omega_Y^{i1 k2} of row pos, reduces fully and
        //    stores row (k2, i1) -- a warp's 32 consecutive columns per row
        const TileMap ym{tile, twoK, twoK, 1, 0, pitch};
        const FwdStore out{P.Z + (size_t)(t * 2 + op) * (size_t)P.Y * twoK, tw_rows, (size_t)i1, (size_t)Y1, twoK, p};
        ntt_forward_out<true>(ym, logY2, tw_y, logY2, p, p2, upper_zero, out, tc);
    }
}

// ---------------------------------------------------------------------------
// Pass 2
// ---------------------------------------------------------------------------

__device__ __forceinline__ const uint2 *pc_tables_f(const KParams &P, int t) { return P.pc[t].t1_f; }
__device__ __forceinline__ const uint2 *pc_tables_i(const KParams &P, int t) { return P.pc[t].t1_i; }

// Pass 2's output: the product of column c, row i1 of a slice, fully
// reduced, to the workspace.
struct MidStore {
    uint32_t *Zs;  // the slice's first word
    int twoK;
    uint32_t p;
    __device__ __forceinline__ void put(uint32_t *, int c, int i1, uint32_t v) const {
        Zs[(size_t)i1 * twoK + c] = red(v, p);
    }
};

// The middle pass's twiddles for prime t in shared memory, one block per
// register stage of the length-Y1a column transform (ntt_stages.cuh,
// stage_blocks, TW_STAGE): for a stage of radix R and sub-block length
// Lc = R L', entry m L' + n1 = omega_Lc^{n1 brev(m)} and, after the Lc
// entries, the roots omega_R^j (j < R/2), forward then inverse; taken from
// the omega_Y1^{+-e} tables (omega_Lc = omega_Y1^{Y1 / Lc}) by asynchronous
// copies the caller commits.
__device__ __forceinline__ void copy_stage_tables(const KParams &P, int t, uint2 *tab) {
    const PrimeConst &pc = P.pc[t];
    int nst, sbase, sextra;
    stage_split(P.logY1a, nst, sbase, sextra);
    int logLc = P.logY1a, toff = 0;
    for (int i = 0; i < nst; ++i) {
        const int b = sbase + (i < sextra ? 1 : 0);
        const int logLp = logLc - b, sh = P.logY1 - logLc;
        const int Lc = 1 << logLc, R = 1 << b;
        uint2 *F = tab + toff;
        uint2 *I = F + Lc + R;
        toff += 2 * (Lc + R);
        for (int idx = threadIdx.x; idx < Lc + R / 2; idx += blockDim.x) {
            size_t e;
            if (idx < Lc)
                e = (size_t)(idx & ((1 << logLp) - 1)) * bitrev((uint32_t)(idx >> logLp), b);
            else
                e = (size_t)(idx - Lc) << logLp;  // root omega_R^j = omega_Lc^(j L')
            cp_async8(F + idx, pc.t1_f + (e << sh));
            cp_async8(I + idx, pc.t1_i + (e << sh));
        }
        logLc -= b;
    }
}

// Pass 2 on one tile: columns [cs S, cs S + S) of the rows (pos, i1), prime t,
// for i1 = Y1a pb + i1a, i1a < Y1a (without a split Y1a = Y1 and pb = 0).
// SMTW: the omega_Y1 tables, and for every later stage a compact table of
// its own sub-block length, are copied to shared memory (else every stage
// reads the omega_Y1 tables in global memory through the non-coherent
// cache).
// COH: the workspace was written by other blocks of the same launch (the
// persistent batch kernel), so it is read through L2 only: 16-byte copies
// (cp.async.cg) or plain L2 loads, never an L1-allocating copy.
template <bool SMTW, class TC, bool COH = false>
__device__ __forceinline__ void mid_tile(const KParams &P, int cs, int pos, int pb, int t) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int S = P.S, logS = P.logS;
    const int twoK = 2 * P.K;
    const int Y1 = (int)P.Y1a;  // this tile's column length
    const PrimeConst &pc = P.pc[t];
    // SMTW: per-stage twiddle blocks (copy_stage_tables), then the tiles
    uint2 *tab = reinterpret_cast<uint2 *>(smem);
    int offs[8];
    const size_t tab_entries = (size_t)stage_blocks(P.logY1a, offs);
    // Tile layout.  S < 32 (a warp spans several rows): rows of S words at
    // pitch S, one empty row after every R rows, R the radix of the column
    // transform's last stage (TileMap::pl) -- every stage's warp accesses
    // hit distinct banks and each row is 16-byte aligned for S >= 4.
    // S >= 32: rows at pitch S, unpadded (a warp's accesses are whole rows).
    const int pl = mid_pad_log(P.logY1a, S);
    const int pitch = mid_pitch(S, pl);
    const int rows = pl ? Y1 + (Y1 >> pl) : Y1;
    uint32_t *A = reinterpret_cast<uint32_t *>(SMTW ? (void *)(tab + tab_entries) : (void *)smem);
    uint32_t *B = A + (size_t)rows * pitch + 16;  // shifted 16 banks
    const uint32_t p = pc.p, p2 = pc.p2;
    uint32_t *ZA = P.Z + (size_t)(t * 2 + 0) * (size_t)P.Y * twoK;
    const uint32_t *ZB = P.Z + (size_t)(t * 2 + 1) * (size_t)P.Y * twoK;
    const size_t base = ((size_t)pos * P.Y1 + (size_t)P.Y1a * pb) * twoK + (size_t)cs * S;
    const TileMap tmp{A, S, S, 1, 0, pitch, 0, pl};
    if (SMTW) copy_stage_tables(P, t, tab);  // copied asynchronously with A's slice
    // A's slice, then B's, as two asynchronous copy groups: B is still in
    // flight while A is transformed.  Rows of S words: 16-byte copies when
    // both ends of every row are 16-byte aligned -- pitch S with S a
    // multiple of 4; row starts in global memory are multiples of 4 words
    // from a 16-byte aligned slab -- else 4-byte copies.
    const bool copy16 = pitch == S && S % 4 == 0;
    auto fill = [&](uint32_t *T, const uint32_t *Z) {
        if (copy16) {
            const int logS4 = logS - 2;
            for (int e = threadIdx.x; e < Y1 * (S >> 2); e += blockDim.x) {
                const int i1 = e >> logS4, c4 = (e & ((S >> 2) - 1)) << 2;
                cp_async16(T + (size_t)padded(tmp, i1) * pitch + c4, Z + base + (size_t)i1 * twoK + c4);
            }
        } else {
            for (int e = threadIdx.x; e < Y1 * S; e += blockDim.x) {
                const int i1 = e >> logS, c = e & (S - 1);
                uint32_t *dst = T + (size_t)padded(tmp, i1) * pitch + c;
                const uint32_t *src = Z + base + (size_t)i1 * twoK + c;
                if (COH)
                    *dst = __ldcg(src);
                else
                    cp_async4(dst, src);
            }
        }
        cp_async_commit();
    };
    fill(A, ZA);
    fill(B, ZB);
    cp_async_wait<1>();
    __syncthreads();
    // y step C (omega_Y1 = omega_Y^Y2) on the S columns of A and of B (B's
    // copies finish while A is transformed), the pointwise product in
    // Montgomery form A*B*2^-32 (the 2^32 is put back by the scale factor of
    // the inverse pass) and the inverse step C, written over A
    const TileMap am{A, S, S, 1, 0, pitch, 0, pl};
    const TileMap bm{B, S, S, 1, 0, pitch, 0, pl};
    // the last inverse stage stores its outputs, fully reduced, to the
    // workspace (rows i1, columns c of this slice)
    const MidStore out{ZA + base, twoK, p};
    TC tc{};
    tc_prime(tc, P, t);
    const bool stored = ntt_convolve<SMTW, SMTW>(am, bm, P.logY1a, SMTW ? tab : pc_tables_f(P, t), pc_tables_i(P, t),
                                                 P.logY1, p, p2, pc.mont, [] {
        cp_async_wait<0>();
        __syncthreads();
    }, out, tc);
    if (stored) return;
    for (int e = threadIdx.x; e < Y1 * S; e += blockDim.x) {
        const int i1 = e >> logS, c = e & (S - 1);
        ZA[base + (size_t)i1 * twoK + c] = red(A[(size_t)padded(tmp, i1) * pitch + c], p);
    }
}

// Pass 2, persistent form for one product: block b runs the tiles b,
// b + gridDim.x, ... of the tile list ordered prime-slowest (tile T: prime
// T / (ncs Y2 Y1b), then pos, pb and the column slice), so a block loads
// each prime's twiddle tables once rather than once per tile.  Two tile
// buffers alternate roles: when the pointwise stage of tile i has consumed
// its second operand, the first operand of tile i+1 starts copying into
// that buffer while tile i's inverse stages run; when tile i's results are
// stored, tile i+1's second operand starts copying into the other buffer
// while tile i+1's first operand is transformed.  Same shared memory as
// mid_tile, same arithmetic and results.
template <bool SMTW, int CS = 0, int CLOG = 0, int CK = 0>
__device__ __forceinline__ void mid_tiles(const KParams &P) {
    extern __shared__ __align__(16) unsigned char smem[];
    // CS, CLOG, CK > 0: the plan's S, log2 Y1a and K as compile-time
    // constants (the launcher checks that they match), so that every
    // stride and stage radix below folds into the instructions
    const int S = CS ? CS : P.S, logS = CS ? clog2(CS) : P.logS;
    const int logY1a = CLOG ? CLOG : P.logY1a;
    const int logY1 = CLOG && P.Y1b == 1 ? CLOG : P.logY1;
    const int twoK = 2 * (CK ? CK : P.K);
    const int Y1 = 1 << logY1a;
    uint2 *tab = reinterpret_cast<uint2 *>(smem);
    int offs[8];
    const size_t tab_entries = (size_t)stage_blocks(logY1a, offs);
    const int pl = mid_pad_log(logY1a, S);
    const int pitch = mid_pitch(S, pl);
    const int rows = pl ? Y1 + (Y1 >> pl) : Y1;
    uint32_t *X = reinterpret_cast<uint32_t *>(SMTW ? (void *)(tab + tab_entries) : (void *)smem);
    uint32_t *Ybuf = X + (size_t)rows * pitch + 16;
    const TileMap tmp{X, S, S, 1, 0, pitch, 0, pl};
    const bool copy16 = pitch == S && S % 4 == 0;
    const int ncs = twoK >> logS;
    const int per_t = ncs * (int)P.Y2 * (int)P.Y1b;
    const int ntiles = per_t * P.r;

    struct Tile {
        int t;
        size_t base;
    };
    auto tile_of = [&](int T) {
        Tile u;
        u.t = T / per_t;
        int rem = T - u.t * per_t;
        const int cs = rem % ncs;
        rem /= ncs;
        const int pb = rem & ((int)P.Y1b - 1), pos = rem >> P.logY1b;
        u.base = ((size_t)pos * P.Y1 + (size_t)P.Y1a * pb) * twoK + (size_t)cs * S;
        return u;
    };
    auto slab = [&](int t, int op) { return P.Z + (size_t)(t * 2 + op) * (size_t)P.Y * twoK; };
    // rows [r0, r1) of an operand slice into a tile buffer
    auto fill_rows = [&](uint32_t *T, const uint32_t *Z, size_t base, int r0, int r1) {
        if (copy16) {
            const int logS4 = logS - 2;
            for (int e = threadIdx.x + (r0 << logS4); e < (r1 << logS4); e += blockDim.x) {
                const int i1 = e >> logS4, c4 = (e & ((S >> 2) - 1)) << 2;
                cp_async16(T + (size_t)padded(tmp, i1) * pitch + c4, Z + base + (size_t)i1 * twoK + c4);
            }
        } else {
            for (int e = threadIdx.x + (r0 << logS); e < (r1 << logS); e += blockDim.x) {
                const int i1 = e >> logS, c = e & (S - 1);
                cp_async4(T + (size_t)padded(tmp, i1) * pitch + c, Z + base + (size_t)i1 * twoK + c);
            }
        }
    };
    auto fill = [&](uint32_t *T, const uint32_t *Z, size_t base) { fill_rows(T, Z, base, 0, Y1); };
    // With three or more register stages each operand copy is issued in two
    // halves at different stage boundaries (first operand: after the
    // pointwise stage and after the first inverse stage; second operand: at
    // the end of the previous tile and after the first stage of this one),
    // so that no single point floods the load queue while the stages wait.
    int nst_c, sbase_c, sextra_c;
    stage_split(logY1a, nst_c, sbase_c, sextra_c);
    const bool halves = nst_c >= 3;
    const int half = Y1 >> 1;
    bool b_second_half = false;  // this tile's second operand: rows [half, Y1) not yet requested
    auto load_tables = [&](int t) { copy_stage_tables(P, t, tab); };

    int T = blockIdx.x;
    if (T >= ntiles) return;
    Tile cur = tile_of(T);
    uint32_t *Pb = X, *Qb = Ybuf;
    // prologue: tables and the first operand, then the second operand
    if (SMTW) load_tables(cur.t);
    fill(Pb, slab(cur.t, 0), cur.base);
    cp_async_commit();
    fill(Qb, slab(cur.t, 1), cur.base);
    cp_async_commit();
    for (;;) {
        const int Tn = T + (int)gridDim.x;
        const bool has_next = Tn < ntiles;
        const Tile nxt = tile_of(has_next ? Tn : T);
        const PrimeConst &pc = P.pc[cur.t];
        const uint32_t p = pc.p, p2 = pc.p2;
        cp_async_wait<1>();  // this tile's first operand (and tables); its second may still fly
        __syncthreads();
        const TileMap am{Pb, S, S, 1, 0, pitch, 0, pl};
        const TileMap bm{Qb, S, S, 1, 0, pitch, 0, pl};
        uint32_t *ZA = slab(cur.t, 0);
        const MidStore out{ZA + cur.base, twoK, p};
        uint32_t *q_next = Qb;
        const bool stored = ntt_convolve<SMTW, SMTW>(
            am, bm, logY1a, SMTW ? tab : pc_tables_f(P, cur.t), pc_tables_i(P, cur.t), logY1, p, p2, pc.mont,
            [] {
                cp_async_wait<0>();
                __syncthreads();
            },
            out, NoTc(),
            [&] {
                if (has_next) {  // the second operand is consumed: next tile's first operand into it
                    fill_rows(q_next, slab(nxt.t, 0), nxt.base, 0, halves ? half : Y1);
                    cp_async_commit();
                }
            },
            [&](int pass, int i) {
                if (pass == 0 && i == 0 && b_second_half) {
                    fill_rows(Qb, slab(cur.t, 1), cur.base, half, Y1);
                    cp_async_commit();
                    b_second_half = false;
                }
                if (pass == 2 && i == nst_c - 2 && halves && has_next) {
                    fill_rows(q_next, slab(nxt.t, 0), nxt.base, half, Y1);
                    cp_async_commit();
                }
            });
        if (!stored) {
            for (int e = threadIdx.x; e < Y1 * S; e += blockDim.x) {
                const int i1 = e >> logS, c = e & (S - 1);
                ZA[cur.base + (size_t)i1 * twoK + c] = red(Pb[(size_t)padded(tmp, i1) * pitch + c], p);
            }
            __syncthreads();
        }
        if (!has_next) break;
        if (SMTW && nxt.t != cur.t) {  // the old tables are no longer read
            load_tables(nxt.t);
            cp_async_commit();
        }
        // next tile's second operand into the freed buffer (its first half when halved)
        fill_rows(Pb, slab(nxt.t, 1), nxt.base, 0, halves ? half : Y1);
        cp_async_commit();
        b_second_half = halves;
        uint32_t *tmpb = Pb;
        Pb = Qb;
        Qb = tmpb;
        T = Tn;
        cur = nxt;
    }
}

// Outer pass of a split middle transform, on one tile: the Y1b rows
// (pos, i1a + Y1a i1b), i1b < Y1b, of prime t and operand op, restricted to
// the W consecutive words [w0, w0 + W) of the flattened (i1a, column) index
// (a tile may span several i1a).  Forward: a length-Y1b DFT down every word
// column, then the twiddle omega_Y1^{i1a k1b}.  Inverse: the twiddle's
// inverse, then the inverse DFT.  Rows are copied with 16-byte cp.async
// (W, 2K and every row start are multiples of four words).
template <bool FWD, class TC>
__device__ __forceinline__ void outer_tile(const KParams &P, int pos, size_t w0, int t, int op) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = P.S2, logW = P.logS2;
    const int twoK = 2 * P.K, log2K = P.logK + 1;
    const int Y1b = (int)P.Y1b, logY1b = P.logY1b;
    uint32_t *T = reinterpret_cast<uint32_t *>(smem);  // [Y1b][W]
    const PrimeConst &pc = P.pc[t];
    const uint32_t p = pc.p, p2 = pc.p2;
    uint32_t *Zt = P.Z + (size_t)(t * 2 + op) * (size_t)P.Y * twoK;
    const size_t base = (size_t)pos * P.Y1 * twoK + w0;
    const size_t rstride = (size_t)P.Y1a * twoK;
    const int W4 = W >> 2, logW4 = logW - 2;
    for (int e = threadIdx.x; e < Y1b * W4; e += blockDim.x) {
        const int ib = e >> logW4, c4 = e & (W4 - 1);
        cp_async16(T + ib * W + 4 * c4, Zt + base + ib * rstride + 4 * c4);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // twiddle omega_Y1^{+-i1a bitrev(ib)} of element (ib, c)
    const uint2 *tab = FWD ? pc.t1_f : pc.t1_i;
    auto tw = [&](int ib, int c) {
        const uint32_t i1a = (uint32_t)((w0 + (size_t)c) >> log2K);
        return __ldg(tab + i1a * bitrev((uint32_t)ib, logY1b));
    };
    const TileMap m{T, W, W, 1, 0, W};  // W transforms of length Y1b, consecutive threads on consecutive words
    TC tc{};
    tc_prime(tc, P, t);
    // four consecutive words share i1a (w0 and 2K are multiples of 4): one
    // twiddle per four words
    if (FWD) {
        ntt_forward(m, logY1b, pc.t1_f, P.logY1, p, p2, false, tc);
    } else {
        for (int e = threadIdx.x; e < Y1b * W4; e += blockDim.x) {
            const int ib = e >> logW4, c4 = e & (W4 - 1);
            const uint2 w = tw(ib, 4 * c4);
            uint4 v = *reinterpret_cast<const uint4 *>(T + ib * W + 4 * c4);
            v.x = shoup(v.x, w, p);
            v.y = shoup(v.y, w, p);
            v.z = shoup(v.z, w, p);
            v.w = shoup(v.w, w, p);
            *reinterpret_cast<uint4 *>(T + ib * W + 4 * c4) = v;
        }
        __syncthreads();
        ntt_inverse(m, logY1b, pc.t1_i, P.logY1, p, p2, tc);
    }
    for (int e = threadIdx.x; e < Y1b * W4; e += blockDim.x) {
        const int ib = e >> logW4, c4 = e & (W4 - 1);
        uint4 v = *reinterpret_cast<const uint4 *>(T + ib * W + 4 * c4);
        if (FWD) {
            const uint2 w = tw(ib, 4 * c4);
            v.x = red(shoup(v.x, w, p), p);
            v.y = red(shoup(v.y, w, p), p);
            v.z = red(shoup(v.z, w, p), p);
            v.w = red(shoup(v.w, w, p), p);
        } else {
            v.x = red(v.x, p);
            v.y = red(v.y, p);
            v.z = red(v.z, p);
            v.w = red(v.w, p);
        }
        *reinterpret_cast<uint4 *>(Zt + base + ib * rstride + 4 * c4) = v;
    }
}

// ---------------------------------------------------------------------------
// Pass 3
// ---------------------------------------------------------------------------

// Recombination tables.  Limb q of sum_j V_j 2^{Mj} receives word k of the
// value V_j 2^{(Mj) mod 32} (r unsigned words and one signed top word, k =
// 0..r) from every column j whose first limb floor(Mj/32) is q - k.  For
// M >= 32 at most one column has a given first limb, so limb q's sources
// are one column per k (or none): packed as 16-bit column indices, 0xffff
// for none, eight slots per limb.  For M < 32 the general range form is
// used: columns jlo .. jlo+count-1, packed as jlo | count << 16.
__device__ __forceinline__ uint4 limb_sources(int q, int M, int r, int twoK) {
    uint32_t slot[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) slot[k] = 0xffffu;
    for (int k = 0; k <= r && k < 8; ++k) {
        const int Q = q - k;  // first limb of the source column
        if (Q < 0) break;
        const int j = (32 * Q + M - 1) / M;  // smallest j with Mj >= 32Q
        if (j < twoK && M * j < 32 * (Q + 1)) slot[k] = (uint32_t)j;
    }
    return make_uint4(slot[0] | slot[1] << 16, slot[2] | slot[3] << 16, slot[4] | slot[5] << 16,
                      slot[6] | slot[7] << 16);
}

__device__ __forceinline__ uint32_t contrib_range(int q, int M, int r, int twoK) {
    const int jlo = q - r <= 0 ? 0 : (32 * (q - r) + M - 1) / M;
    int jhi = (32 * q + 31) / M;
    if (jhi > twoK - 1) jhi = twoK - 1;
    const int cnt = jhi >= jlo ? jhi - jlo + 1 : 0;
    return (uint32_t)jlo | ((uint32_t)cnt << 16);
}

// Word k of V_j 2^sh: unsigned for k < r, the signed top word for k = r.
template <int RR>
__device__ __forceinline__ int64_t shifted_word(const uint32_t *V, int plane, int j, int k, int sh) {
    if (k < RR) {
        const uint32_t hi = V[k * plane + j];
        const uint32_t lo = k > 0 ? V[(k - 1) * plane + j] : 0u;
        return (int64_t)(sh ? __funnelshift_l(lo, hi, sh) : hi);
    }
    const int32_t top = (int32_t)V[(RR - 1) * plane + j];
    return (int64_t)(sh ? (top >> (32 - sh)) : (top >> 31));
}

// Sum of the contributions to limb q (M >= 32: table form, unrolled).
template <int RR>
__device__ __forceinline__ int64_t limb_sum_tab(const uint32_t *V, int plane, int M, uint4 src) {
    const uint32_t w[4] = {src.x, src.y, src.z, src.w};
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k <= RR; ++k) {
        const uint32_t j = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
        if (j != 0xffffu) acc += shifted_word<RR>(V, plane, (int)j, k, (int)((M * j) & 31));
    }
    return acc;
}

// Sum of the contributions to limb q (any M: range form).
template <int RR>
__device__ __forceinline__ int64_t limb_sum_rng(const uint32_t *V, int plane, int q, int M,
                                                uint32_t range) {
    const int jlo = (int)(range & 0xffffu), cnt = (int)(range >> 16);
    int e = M * jlo;
    int64_t acc = 0;
    for (int n = 0; n < cnt; ++n, e += M) {
        const int k = q - (e >> 5);
        if (k >= 0 && k <= RR) acc += shifted_word<RR>(V, plane, jlo + n, k, e & 31);
    }
    return acc;
}

// Carries into each lane of a 32-limb chunk from per-lane generate and
// propagate bits (disjoint) and the chunk's carry-in: carry-lookahead by
// one 33-bit addition.  Returns the carry mask; *cio becomes the carry out.
__device__ __forceinline__ unsigned lookahead(unsigned gen, unsigned prop, unsigned *cio) {
    const uint64_t s = (uint64_t)gen + (uint64_t)(gen | prop) + *cio;
    *cio = (unsigned)(s >> 32);
    return (unsigned)s ^ prop;
}

// CRT over RR primes (Garner's mixed radix) for every (row < nro, column)
// of the tile, centred lift to (-m/2, m/2), written back as an RR-word
// two's-complement value (word w in plane w).
template <int RR>
__device__ __forceinline__ void crt_tile(const KParams &P, uint32_t *R, size_t plane, int pitch,
                                         int nro, int logK) {
    const int twoK = 2 << logK;
    uint32_t pr[RR];
    uint2 gi[RR][RR];
#pragma unroll
    for (int t = 0; t < RR; ++t) {
        pr[t] = P.pc[t].p;
#pragma unroll
        for (int s = 0; s < t; ++s) gi[t][s] = make_uint2(P.ginv[t][s], P.ginv_s[t][s]);
    }
    for (int e2 = threadIdx.x; e2 < nro * twoK; e2 += blockDim.x) {
        const int e = (e2 >> (logK + 1)) * pitch + (e2 & (twoK - 1));
        uint32_t v[RR];
#pragma unroll
        for (int t = 0; t < RR; ++t) v[t] = R[(size_t)t * plane + e];
#pragma unroll
        for (int t = 1; t < RR; ++t) {
            uint32_t y = v[t];
#pragma unroll
            for (int s = 0; s < t; ++s) {
                const uint32_t vs = red(v[s], pr[t]);  // v_s < 2^30 < 2 p_t
                y = red(shoup(y + pr[t] - vs, gi[t][s], pr[t]), pr[t]);
            }
            v[t] = y;
        }
        // X = v0 + p0 (v1 + p1 (v2 + ...))
        uint32_t X[RR];
#pragma unroll
        for (int w = 0; w < RR; ++w) X[w] = 0;
        X[0] = v[RR - 1];
#pragma unroll
        for (int t = RR - 2; t >= 0; --t) {
            uint64_t carry = v[t];
#pragma unroll
            for (int w = 0; w < RR; ++w) {
                const uint64_t z = (uint64_t)X[w] * pr[t] + carry;
                X[w] = (uint32_t)z;
                carry = z >> 32;
            }
        }
        // 2X >= m  <=>  X > (m-1)/2 (m is odd)  ->  X - m
        uint32_t borrow = 0;
#pragma unroll
        for (int w = 0; w < RR; ++w) {
            const uint32_t x2 = (X[w] << 1) | (w ? (X[w - 1] >> 31) : 0u);
            const uint64_t d = (uint64_t)x2 - P.m_words[w] - borrow;
            borrow = (uint32_t)(d >> 63);
        }
        if (!borrow) {
            uint32_t bb = 0;
#pragma unroll
            for (int w = 0; w < RR; ++w) {
                const uint64_t d = (uint64_t)X[w] - P.m_words[w] - bb;
                X[w] = (uint32_t)d;
                bb = (uint32_t)(d >> 63);
            }
        }
#pragma unroll
        for (int w = 0; w < RR; ++w) R[(size_t)w * plane + e] = X[w];
    }
}

// Recombination c_i = sum_{j<2K} c_{i,j} 2^{Mj}, one warp per row, limbs
// 0..lc computed modulo 2^(32(lc+1)) (limb lc is the sign word), 32 limbs
// per step.  Each lane sums the pieces landing on its limb (a signed 64-bit
// P_q = t_q + 2^32 h_q).  Adding h_{q-1} to t_q leaves t'_q and a carry g_q
// in {-1, 0, 1}; the value is then sum t'_q 2^{32q} + sum_{g=1} 2^{32(q+1)}
// - sum_{g=-1} 2^{32(q+1)}, resolved as one addition and one subtraction,
// each by ballot carry-lookahead.  Limbs go straight to the output in two's
// complement; a negative row is then turned into its magnitude in place (it
// is still in L2): zero below the lowest non-zero limb f, -x at f, ~x above.
template <int RR, int CM = 0>
__device__ __forceinline__ void recombine_rows(const KParams &P, const uint32_t *R, int plane, int pitch,
                                               const uint4 *sources, int nro, int64_t i1,
                                               uint32_t *__restrict__ c, uint8_t *__restrict__ cn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int lc1 = P.lc + 1, M = CM ? CM : P.M;
    const bool tab = M >= 32;
    for (int i2 = warp; i2 < nro; i2 += nw) {
        const int64_t i = i1 + P.Y1 * (int64_t)i2;
        const uint32_t *V = R + i2 * pitch;
        uint32_t *crow = c + (size_t)i * P.lc;
        int h_last = 0;  // h of the previous chunk's last limb
        int g_last = 0;  // g of the previous chunk's last limb
        unsigned cplus = 0, cminus = 0;
        int first_nz = lc1;  // lowest non-zero limb below the sign word
        uint32_t top = 0;
        for (int q0 = 0; q0 < lc1; q0 += 32) {
            const int q = q0 + lane;
            const bool act = q < lc1;
            int64_t Pq = 0;
            if (act) {
                const uint4 src = sources[q];
                Pq = tab ? limb_sum_tab<RR>(V, plane, M, src) : limb_sum_rng<RR>(V, plane, q, M, src.x);
            }
            const int h = (int)(Pq >> 32);  // |h| < 2^8
            int hprev = __shfl_up_sync(0xffffffffu, h, 1);
            if (lane == 0) hprev = h_last;
            const int64_t sum = (int64_t)(uint32_t)Pq + hprev;
            const uint32_t tq = (uint32_t)sum;
            const int g = (int)(sum >> 32);
            int gprev = __shfl_up_sync(0xffffffffu, g, 1);
            if (lane == 0) gprev = g_last;
            h_last = __shfl_sync(0xffffffffu, h, 31);
            g_last = __shfl_sync(0xffffffffu, g, 31);
            // + 1 at every limb whose lower neighbour carried +1
            const uint32_t gp = gprev == 1 ? 1u : 0u;
            const unsigned cm = lookahead(__ballot_sync(0xffffffffu, act && gp && tq == 0xffffffffu),
                                          __ballot_sync(0xffffffffu, act && tq + gp == 0xffffffffu), &cplus);
            const uint32_t u = tq + gp + ((cm >> lane) & 1u);
            // - 1 at every limb whose lower neighbour carried -1
            const uint32_t gm = gprev == -1 ? 1u : 0u;
            const unsigned bm = lookahead(__ballot_sync(0xffffffffu, act && gm && u == 0u),
                                          __ballot_sync(0xffffffffu, act && u == gm), &cminus);
            const uint32_t v = u - gm - ((bm >> lane) & 1u);
            if (q < lc1 - 1) crow[q] = v;
            if (q == lc1 - 1) top = v;
            const unsigned nz = __ballot_sync(0xffffffffu, q < lc1 - 1 && v != 0u);
            if (nz && first_nz == lc1) first_nz = q0 + __ffs(nz) - 1;
        }
        top = __shfl_sync(0xffffffffu, top, (lc1 - 1) & 31);
        const bool negative = top == 0xffffffffu;
        if (lane == 0) {
            if (top != 0u && !negative) atomicOr(P.err, ERRBIT_INTERNAL);
            cn[i] = negative ? 1 : 0;
        }
        if (negative) {
            __syncwarp();  // the warp's own limb stores are visible to all its lanes
            for (int q = first_nz + lane; q < P.lc; q += 32) {
                const uint32_t v = crow[q];
                crow[q] = q == first_nz ? 0u - v : ~v;
            }
        }
    }
}

// Pass 3's input: the step-B inverse twiddle of row pos, in [0, 2p).
struct RowTwiddle {
    const uint2 *tw_rows;
    uint32_t p;
    __device__ __forceinline__ uint32_t get(const uint32_t *a, int, int pos) const {
        return shoup(*a, tw_rows[pos], p);
    }
};

// Pass 3 on one tile: output rows i = i1 + Y1*i2 (i2 < Y2).
// COH: as for mid_tile (the rows were written by other blocks of the same
// launch): plain L2 loads instead of L1-allocating asynchronous copies.
template <class TC, bool COH = false, int CK = 0, int CLY2 = 0, int CM = 0>
__device__ __forceinline__ void inv_tile(const KParams &P, int64_t i1, uint32_t *__restrict__ c,
                                         uint8_t *__restrict__ cn) {
    extern __shared__ __align__(16) unsigned char smem[];
    // CK, CLY2, CM > 0: K, log2 Y2 and M as compile-time constants (as fwd_tile)
    const int K = CK ? CK : P.K, logK = CK ? clog2(CK) : P.logK, twoK = 2 * K, r = P.r, M = CM ? CM : P.M;
    const int logY2 = CLY2 ? CLY2 : P.logY2;
    const int Y2 = 1 << logY2;
    const int64_t Y1 = P.Y1;
    const int pitch = twoK + 1;  // odd row pitch
    const size_t plane = (size_t)Y2 * pitch;
    uint32_t *R = reinterpret_cast<uint32_t *>(smem);  // [r][Y2][pitch]
    const int lc1 = P.lc + 1;
    uint4 *sources = reinterpret_cast<uint4 *>(smem + (((size_t)r * plane * 4 + 15) & ~(size_t)15));  // [lc1]
    // per-prime tables, copied with the prime's rows: omega_Y^{-i1 k2(pos)}
    // (pos < Y2), omega_K^{-e} (e < K), omega_Y2^{-e} (e < Y2)
    uint2 *tw_sets = reinterpret_cast<uint2 *>(sources + lc1);
    const int set_len = 2 * Y2 + K;
    for (int q = threadIdx.x; q < lc1; q += blockDim.x)
        sources[q] = M >= 32 ? limb_sources(q, M, r, twoK) : make_uint4(contrib_range(q, M, r, twoK), 0, 0, 0);

    // rows i2 < nro are output coefficients (i = i1 + Y1*i2 < nc)
    const int nro = i1 < P.nc ? (int)min((int64_t)Y2, (P.nc - i1 + Y1 - 1) / Y1) : 0;
    // every prime's rows (k2, i1) requested at once, one copy group per prime
    for (int t = 0; t < r; ++t) {
        const uint32_t *Zt = P.Z + (size_t)(t * 2) * (size_t)P.Y * twoK;
        for (int e = threadIdx.x; e < Y2 * twoK; e += blockDim.x) {
            const int pos = e >> (logK + 1), col = e & (twoK - 1);
            uint32_t *dst = R + (size_t)t * plane + (size_t)pos * pitch + col;
            const uint32_t *src = Zt + ((size_t)pos * Y1 + i1) * twoK + col;
            if (COH)
                *dst = __ldcg(src);
            else
                cp_async4(dst, src);
        }
        const PrimeConst &pq = P.pc[t];
        uint2 *set = tw_sets + t * set_len;
        for (int q = threadIdx.x; q < Y2; q += blockDim.x) {
            cp_async8(set + q, pq.ty_i + (size_t)i1 * bitrev((uint32_t)q, logY2));
            cp_async8(set + Y2 + K + q, pq.ty_i + ((size_t)q << (P.logY - logY2)));
        }
        for (int j = threadIdx.x; j < K; j += blockDim.x) cp_async8(set + Y2 + j, pq.tx_i + 2 * j);
        cp_async_commit();
    }
    for (int t = 0; t < r; ++t) {
        const PrimeConst &pc = P.pc[t];
        const uint32_t p = pc.p, p2 = pc.p2;
        uint32_t *Rt = R + (size_t)t * plane;
        // wait for prime t's group (groups complete in order)
        switch (r - 1 - t) {
            case 0: cp_async_wait<0>(); break;
            case 1: cp_async_wait<1>(); break;
            case 2: cp_async_wait<2>(); break;
            case 3: cp_async_wait<3>(); break;
            case 4: cp_async_wait<4>(); break;
            default: cp_async_wait<5>(); break;
        }
        __syncthreads();
        const uint2 *tw_rows = tw_sets + t * set_len;
        const uint2 *tw_x = tw_rows + Y2;
        const uint2 *tw_y = tw_x + K;
        const uint2 *tw_untw = pc.untw;  // read once per element, contiguously
        TC tc{};
        tc_prime(tc, P, t);
        // inverse y step A; its first stage applies the step-B twiddle
        // omega_Y^{-i1 k2} of row pos as it loads
        const TileMap ym{Rt, twoK, twoK, 1, 0, pitch};
        ntt_inverse_in<true>(ym, logY2, tw_y, logY2, p, p2, RowTwiddle{tw_rows, p}, tc);
        if (CLY2 && nro == Y2) {  // every row is an output row: constant map
            const TileMap xm{Rt, 2 * Y2, Y2, pitch, K, 1};
            ntt_inverse<true>(xm, logK, tw_x, logK, p, p2, tc);
        } else if (nro > 0) {
            const TileMap xm{Rt, 2 * nro, nro, pitch, K, 1};
            ntt_inverse<true>(xm, logK, tw_x, logK, p, p2, tc);
        }
        const uint2 sc = make_uint2(pc.scale, pc.scale_s);
        for (int e = threadIdx.x; e < nro * K; e += blockDim.x) {
            const int i2 = e >> logK, j = e & (K - 1);
            uint32_t *row = Rt + (size_t)i2 * pitch;
            const uint32_t u = shoup(row[j], sc, p);
            const uint32_t v = shoup(row[K + j], tw_untw[j], p);
            row[j] = red(red(u + v, p2), p);
            row[K + j] = red(red(u - v + p2, p2), p);
        }
        __syncthreads();
    }

    switch (r) {
        case 1: crt_tile<1>(P, R, plane, pitch, nro, logK); break;
        case 2: crt_tile<2>(P, R, plane, pitch, nro, logK); break;
        case 3: crt_tile<3>(P, R, plane, pitch, nro, logK); break;
        case 4: crt_tile<4>(P, R, plane, pitch, nro, logK); break;
        case 5: crt_tile<5>(P, R, plane, pitch, nro, logK); break;
        default: crt_tile<6>(P, R, plane, pitch, nro, logK); break;
    }
    __syncthreads();

    // Recombination c_i = sum_{j<2K} c_{i,j} 2^{Mj}, one warp per row, limbs
    // 0..lc computed modulo 2^(32(lc+1)) (limb lc is the sign word), 32 limbs
    // per step.  Each lane sums the pieces landing on its limb (a signed
    // 64-bit P_q); P_q = t_q + 2^32 h_q.  Adding h_{q-1} to t_q leaves t'_q and
    // a carry g_q in {-1, 0, 1}; the value is then sum t'_q 2^{32q} +
    // sum_{g=1} 2^{32(q+1)} - sum_{g=-1} 2^{32(q+1)}, resolved as one
    // addition and one subtraction, each by ballot carry-lookahead.  Limbs go
    // straight to the output in two's complement; a negative row is then
    // turned into its magnitude in place (it is still in L2): zero below the
    // lowest non-zero limb f, -x at f, ~x above.
    switch (r) {
        case 1: recombine_rows<1, CM>(P, R, (int)plane, pitch, sources, nro, i1, c, cn); break;
        case 2: recombine_rows<2, CM>(P, R, (int)plane, pitch, sources, nro, i1, c, cn); break;
        case 3: recombine_rows<3, CM>(P, R, (int)plane, pitch, sources, nro, i1, c, cn); break;
        case 4: recombine_rows<4, CM>(P, R, (int)plane, pitch, sources, nro, i1, c, cn); break;
        case 5: recombine_rows<5, CM>(P, R, (int)plane, pitch, sources, nro, i1, c, cn); break;
        default: recombine_rows<6, CM>(P, R, (int)plane, pitch, sources, nro, i1, c, cn); break;
    }
}

}  // namespace ipm
