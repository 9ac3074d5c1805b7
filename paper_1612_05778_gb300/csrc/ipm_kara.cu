// ipm_kara.cu -- the Karatsuba family: L levels of Karatsuba's
// three-product recursion over y (A. Karatsuba, Yu. Ofman, 1962; §1 lists
// it among the plain methods the paper improves on), with the schoolbook
// kernel at the leaves.
//
// Both operands are padded with zero coefficients to n2 = m 2^L.  A node
// of length len splits each operand into its lower and upper halves
// (x = x0 + y^(len/2) x1); its three children are (a0, b0), (a1, b1) and
// (a0 + a1, b0 + b1), numbered 0, 1, 2, so the leaf with base-3 digits
// j_1 .. j_L (top level first) has operand coefficients
//     A_leaf[i] = sum of a_(i + sum_d c_d n2 / 2^d) over c_d in S(j_d),
// S(0) = {0}, S(1) = {1}, S(2) = {0, 1}: up to 2^L input coefficients,
// |A_leaf[i]| < 2^(bits_a + L).  The 3^L leaf products of m x m
// coefficients run in one schoolbook launch.  Going up, a node's product
// is P0 + y^h (PS - P0 - P1) + y^(2h) P1 from its children's products
// P0 = a0 b0, P1 = a1 b1, PS = (a0 + a1)(b0 + b1), h = len/2: coefficient
//     c_k = P0_k + PS_(k-h) - P0_(k-h) - P1_(k-h) + P1_(k-2h),
// one warp per coefficient, carried exactly (carry.cuh).  The root's
// product is written to c; its coefficients beyond na + nb - 1 (the
// padding) must be zero, and every intermediate must fit its stride
// (otherwise ERRBIT_INTERNAL).
#include <cuda_runtime.h>

#include <algorithm>

#include "carry.cuh"
#include "ipm_internal.h"

namespace ipm {

namespace {

constexpr int KARA_THREADS = 256;

// Leaf operands of one input x (n coefficients of L limbs, the rest zero
// padding up to n2): one warp per (leaf, i).
__global__ void k_kara_eval(const uint32_t *__restrict__ x, const uint8_t *__restrict__ xn, int64_t n, int L,
                            uint32_t bits, int levels, int64_t n2, int64_t m, int Lleaf, uint32_t *__restrict__ out,
                            uint8_t *__restrict__ outn, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t leaves = 1;
    for (int d = 0; d < levels; ++d) leaves *= 3;
    for (int64_t it = warp; it < leaves * m; it += nwarps) {
        const int64_t leaf = it / m, i = it - leaf * m;
        // base-3 digits of the leaf, top level first
        int digit[8];
        {
            int64_t v = leaf;
            for (int d = levels - 1; d >= 0; --d) {
                digit[d] = (int)(v % 3);
                v /= 3;
            }
        }
        const uint32_t *ptr[16];
        int li[16];
        uint8_t ng[16];
        int nt = 0;
        // every combination of the halves the digits allow
        const int ntwo = [&] {
            int c = 0;
            for (int d = 0; d < levels; ++d) c += digit[d] == 2;
            return c;
        }();
        for (int combo = 0; combo < (1 << ntwo); ++combo) {
            int64_t pos = i;
            int bit = 0;
            for (int d = 0; d < levels; ++d) {
                const int64_t half = n2 >> (d + 1);
                int c = digit[d];
                if (c == 2) c = (combo >> bit++) & 1;
                pos += c * half;
            }
            if (pos < n) {
                ptr[nt] = x + (size_t)pos * L;
                li[nt] = L;
                ng[nt] = xn[pos];
                ++nt;
            }
        }
        // an input above its bit bound is reported by the one leaf with
        // digits 0 and 1 only that takes it alone (those leaves cover every
        // position once)
        if (ntwo == 0 && nt == 1 && lane == 0 && (bits & 31u) && (ptr[0][L - 1] >> (bits & 31u)))
            atomicOr(err, ERRBIT_BOUND);
        if (!warp_signed_sum(ptr, li, ng, nt, out + (size_t)it * Lleaf, outn + it, Lleaf) && lane == 0)
            atomicOr(err, ERRBIT_INTERNAL);
    }
}

// Node products at depth d from their children's: one warp per (node, k).
// children: 3^(d+1) products of 2h - 1 coefficients (stride ls limbs);
// out: 3^d products of 4h - 1 coefficients (stride lo limbs), of which the
// first nkeep are written (the rest must be zero).
__global__ void k_kara_combine(const uint32_t *__restrict__ ch, const uint8_t *__restrict__ chn, int64_t nodes,
                               int64_t h, int ls, uint32_t *__restrict__ out, uint8_t *__restrict__ outn, int lo,
                               int64_t nkeep, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t clen = 2 * h - 1, olen = 4 * h - 1;
    for (int64_t it = warp; it < nodes * olen; it += nwarps) {
        const int64_t node = it / olen, k = it - node * olen;
        const int64_t c0 = 3 * node, c1 = c0 + 1, cs = c0 + 2;  // P0, P1, PS
        const uint32_t *ptr[5];
        int li[5];
        uint8_t ng[5];
        int nt = 0;
        auto term = [&](int64_t child, int64_t idx, bool minus) {
            if (idx < 0 || idx >= clen) return;
            const int64_t at = child * clen + idx;
            ptr[nt] = ch + (size_t)at * ls;
            li[nt] = ls;
            ng[nt] = (uint8_t)((chn[at] != 0) != minus);
            ++nt;
        };
        term(c0, k, false);
        term(cs, k - h, false);
        term(c0, k - h, true);
        term(c1, k - h, true);
        term(c1, k - 2 * h, false);
        if (k < nkeep) {
            const int64_t o = node * nkeep + k;
            if (!warp_signed_sum(ptr, li, ng, nt, out + (size_t)o * lo, outn + o, lo) && lane == 0)
                atomicOr(err, ERRBIT_INTERNAL);
        } else {  // padding of the root product: must be zero (fits zero limbs)
            uint8_t unused;
            if (!warp_signed_sum(ptr, li, ng, nt, nullptr, &unused, 0) && lane == 0) atomicOr(err, ERRBIT_INTERNAL);
        }
    }
}

}  // namespace

int launch_kara_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const KaraPlan &k = sp.ka;
    uint32_t *Z = sp.kp.Z;
    int *err = sp.kp.err;
    const int64_t m = k.m;
    int64_t leaves = 1;
    for (int d = 0; d < k.levels; ++d) leaves *= 3;
    uint32_t *A = Z + k.off_a, *B = Z + k.off_b;
    uint8_t *An = reinterpret_cast<uint8_t *>(Z + k.off_an), *Bn = reinterpret_cast<uint8_t *>(Z + k.off_bn);
    const unsigned eb = (unsigned)std::min<int64_t>((leaves * m + 7) / 8, 1216 * 8);
    k_kara_eval<<<eb, KARA_THREADS, 0, s>>>(a, an, k.na, k.la, k.bits_a, k.levels, k.n2, m, k.lla, A, An, err);
    k_kara_eval<<<eb, KARA_THREADS, 0, s>>>(b, bn, k.nb, k.lb, k.bits_b, k.levels, k.n2, m, k.llb, B, Bn, err);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) return -1;
    // leaf products into level L's buffer
    uint32_t *lev = Z + k.off_lev[k.levels];
    uint8_t *levn = reinterpret_cast<uint8_t *>(Z + k.off_levn[k.levels]);
    if (launch_school_batch(sp.kp, A, An, B, Bn, lev, levn, leaves, stream)) return -1;
    // combine upward
    int64_t nodes = leaves;
    for (int d = k.levels - 1; d >= 0; --d) {
        nodes /= 3;
        const int64_t len = k.n2 >> d, h = len / 2;
        const uint32_t *ch = Z + k.off_lev[d + 1];
        const uint8_t *chn = reinterpret_cast<const uint8_t *>(Z + k.off_levn[d + 1]);
        uint32_t *out = d ? Z + k.off_lev[d] : c;
        uint8_t *outn = d ? reinterpret_cast<uint8_t *>(Z + k.off_levn[d]) : cn;
        const int lo = d ? k.lci : k.lc;
        const int64_t nkeep = d ? 2 * len - 1 : k.nc;
        const unsigned cb = (unsigned)std::min<int64_t>((nodes * (2 * len - 1) + 7) / 8, 1216 * 8);
        k_kara_combine<<<cb, KARA_THREADS, 0, s>>>(ch, chn, nodes, h, k.lci, out, outn, lo, nkeep, err);
        note_launches(1);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

}  // namespace ipm
