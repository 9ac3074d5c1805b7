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
#include <algorithm>
#include <atomic>

#include "ipm_internal.h"
#include "modarith.cuh"
#include "ntt_stages.cuh"
#include "ipm_mid256.h"
#include "passes.cuh"

namespace ipm {

static std::atomic<int64_t> g_launches{0};
int64_t launches_so_far() { return g_launches.load(); }
void note_launches(int n) { g_launches.fetch_add(n); }

// ---------------------------------------------------------------------------
// Kernels.  Single product: the plan's constants are a __grid_constant__
// parameter and the grid is the tile grid.  Batched: one launch covers the
// tiles of many products; block b reads (product, tile) = items[b] and that
// product's constants and operand pointers from device arrays.
// Forward/inverse come in two block sizes: THREADS_FWD / THREADS_INV for
// tiles that leave room for several blocks per SM, 1024 for tiles that fill
// an SM.
// ---------------------------------------------------------------------------

template <int NT, int CK = 0, int CLY2 = 0, int CM = 0>
__global__ void __launch_bounds__(NT, NT == THREADS_FWD ? 3 : 1)
k_forward(const __grid_constant__ KParams P, const uint32_t *__restrict__ a, const uint8_t *__restrict__ an,
          const uint32_t *__restrict__ b, const uint8_t *__restrict__ bn) {
    fwd_tile<NoTc, CK, CLY2, CM>(P, blockIdx.x, blockIdx.y, a, an, b, bn);
}

// persistent: one block per SM walks the tile list (passes.cuh, mid_tiles)
template <bool SMTW, int CS = 0, int CLOG = 0, int CK = 0>
__global__ void __launch_bounds__(THREADS_MID, 1) k_middle(const __grid_constant__ KParams P) {
    mid_tiles<SMTW, CS, CLOG, CK>(P);
}

// grid: x = pos * (Y1a 2K / W) + word block; y = 2t + op forward (both
// operands), y = t inverse (the product, held in operand A's slab)
template <bool FWD>
__global__ void __launch_bounds__(THREADS_OUTER) k_outer(const __grid_constant__ KParams P) {
    const int lnb = P.logY1a + P.logK + 1 - P.logS2;  // word blocks per row: Y1a 2K / W
    const size_t wb = blockIdx.x & ((1u << lnb) - 1);
    const int pos = (int)(blockIdx.x >> lnb);
    const int t = FWD ? (int)(blockIdx.y >> 1) : (int)blockIdx.y;
    const int op = FWD ? (int)(blockIdx.y & 1) : 0;
    outer_tile<FWD, NoTc>(P, pos, wb << P.logS2, t, op);
}

template <int NT, int CK = 0, int CLY2 = 0, int CM = 0>
__global__ void __launch_bounds__(NT, NT == THREADS_INV ? 2 : 1)
k_inverse(const __grid_constant__ KParams P, uint32_t *__restrict__ c, uint8_t *__restrict__ cn) {
    inv_tile<NoTc, false, CK, CLY2, CM>(P, blockIdx.x, c, cn);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == THREADS_FWD ? 3 : 1)
kb_forward(const KParams *__restrict__ Ps, const ipm_operands *__restrict__ ops, const uint2 *__restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const KParams &P = Ps[it.x];
    const ipm_operands o = ops[P.batch_index];
    const int op = (int64_t)it.y >= P.Y1 ? 1 : 0;
    fwd_tile<NoTc>(P, (int64_t)it.y - (op ? P.Y1 : 0), op, o.a, o.a_neg, o.b, o.b_neg);
}

template <bool SMTW>
__global__ void __launch_bounds__(THREADS_MID, 1)
kb_middle(const KParams *__restrict__ Ps, const uint2 *__restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const KParams &P = Ps[it.x];
    const int ncs = 2 * P.K / P.S;
    const int cs = (int)(it.y % (uint32_t)ncs);
    const int rest = (int)(it.y / (uint32_t)ncs);  // (t, pos) of an unsplit plan
    mid_tile<SMTW, NoTc>(P, cs, rest % (int)P.Y2, 0, rest / (int)P.Y2);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == THREADS_INV ? 2 : 1)
kb_inverse(const KParams *__restrict__ Ps, const ipm_operands *__restrict__ ops, const uint2 *__restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const KParams &P = Ps[it.x];
    const ipm_operands o = ops[P.batch_index];
    inv_tile<NoTc>(P, it.y, o.c, o.c_neg);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

int set_kernel_attributes() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_forward<THREADS_FWD>, SMEM_FWD_MAX);
    set((const void *)k_forward<THREADS_FWD, 32, 7, 33>, SMEM_FWD_MAX);
    set((const void *)k_forward<THREADS_FWD, 128, 5, 33>, SMEM_FWD_MAX);
    set((const void *)k_forward<THREADS_FWD, 128, 5, 17>, SMEM_FWD_MAX);
    set((const void *)k_forward<1024>, SMEM_FWD_MAX);
    set((const void *)k_middle<true>, SMEM_MID_MAX);
    set((const void *)k_middle<false>, SMEM_MID_MAX);
    set((const void *)k_middle<true, 4, 12, 32>, SMEM_MID_MAX);
    set((const void *)k_middle<true, 8, 11, 128>, SMEM_MID_MAX);
    set((const void *)k_middle<true, 16, 10, 128>, SMEM_MID_MAX);
    set((const void *)k_inverse<THREADS_INV>, SMEM_INV_MAX);
    set((const void *)k_inverse<THREADS_INV, 32, 7, 33>, SMEM_INV_MAX);
    set((const void *)k_inverse<THREADS_INV, 128, 5, 33>, SMEM_INV_MAX);
    set((const void *)k_inverse<THREADS_INV, 128, 5, 17>, SMEM_INV_MAX);
    set((const void *)k_inverse<1024>, SMEM_INV_MAX);
    set((const void *)k_outer<true>, SMEM_MID_MAX);
    set((const void *)k_outer<false>, SMEM_MID_MAX);
    set((const void *)kb_forward<THREADS_FWD>, SMEM_FWD_MAX);
    set((const void *)kb_forward<1024>, SMEM_FWD_MAX);
    set((const void *)kb_middle<true>, SMEM_MID_MAX);
    set((const void *)kb_middle<false>, SMEM_MID_MAX);
    set((const void *)kb_inverse<THREADS_INV>, SMEM_INV_MAX);
    set((const void *)kb_inverse<1024>, SMEM_INV_MAX);
    if (e == cudaSuccess && set_kernel_attributes_tc()) return -1;
    if (e == cudaSuccess && set_kernel_attributes_mid256()) return -1;
    if (e == cudaSuccess && set_kernel_attributes_batch()) return -1;
    return e == cudaSuccess ? 0 : -1;
}

int launch_batch(const BatchLaunch &bl, const ipm_operands *ops, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (bl.items[0] && bl.fwd_small && bl.nruns > 0) {
        // runs of one (K, log2 Y2): compiled kernels where there is one
        for (int k = 0; k < bl.nruns; ++k) {
            const BatchRun &r = bl.runs[k];
            if (!r.nf) continue;
            const int rc = r.K ? launch_batch_run(true, r.K, r.logY2, bl.params, ops, bl.items[0] + r.f0, r.nf,
                                                  bl.smem[0], stream)
                               : 1;
            if (rc < 0) return -1;
            if (rc == 1) {
                kb_forward<THREADS_FWD><<<r.nf, THREADS_FWD, bl.smem[0], s>>>(bl.params, ops, bl.items[0] + r.f0);
                g_launches.fetch_add(1);
                if (cudaGetLastError() != cudaSuccess) return -1;
            }
        }
    } else if (bl.items[0]) {
        if (bl.fwd_small)
            kb_forward<THREADS_FWD><<<bl.nitems[0], THREADS_FWD, bl.smem[0], s>>>(bl.params, ops, bl.items[0]);
        else
            kb_forward<1024><<<bl.nitems[0], 1024, bl.smem[0], s>>>(bl.params, ops, bl.items[0]);
        g_launches.fetch_add(1);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    if (bl.items[1]) {
        if (bl.mid_tables)
            kb_middle<true><<<bl.nitems[1], THREADS_MID, bl.smem[1], s>>>(bl.params, bl.items[1]);
        else
            kb_middle<false><<<bl.nitems[1], THREADS_MID, bl.smem[1], s>>>(bl.params, bl.items[1]);
        g_launches.fetch_add(1);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    if (bl.items[2] && bl.inv_small && bl.nruns > 0) {
        for (int k = 0; k < bl.nruns; ++k) {
            const BatchRun &r = bl.runs[k];
            if (!r.ni) continue;
            const int rc = r.K ? launch_batch_run(false, r.K, r.logY2, bl.params, ops, bl.items[2] + r.i0, r.ni,
                                                  bl.smem[2], stream)
                               : 1;
            if (rc < 0) return -1;
            if (rc == 1) {
                kb_inverse<THREADS_INV><<<r.ni, THREADS_INV, bl.smem[2], s>>>(bl.params, ops, bl.items[2] + r.i0);
                g_launches.fetch_add(1);
                if (cudaGetLastError() != cudaSuccess) return -1;
            }
        }
    } else if (bl.items[2]) {
        if (bl.inv_small)
            kb_inverse<THREADS_INV><<<bl.nitems[2], THREADS_INV, bl.smem[2], s>>>(bl.params, ops, bl.items[2]);
        else
            kb_inverse<1024><<<bl.nitems[2], 1024, bl.smem[2], s>>>(bl.params, ops, bl.items[2]);
        g_launches.fetch_add(1);
        if (cudaGetLastError() != cudaSuccess) return -1;
    }
    return 0;
}

int launch_forward(const KParams &kp, size_t smem, const uint32_t *a, const uint8_t *an,
                   const uint32_t *b, const uint8_t *bn, void *stream) {
    if (kp.tcfrag) return launch_forward_tc(kp, smem, a, an, b, bn, stream);
    dim3 grid((unsigned)kp.Y1, 2, 1);
    if (smem <= SMEM_FWD_3PERSM && kp.K == 32 && kp.logY2 == 7 && kp.M == 33)
        k_forward<THREADS_FWD, 32, 7, 33><<<grid, THREADS_FWD, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    else if (smem <= SMEM_FWD_3PERSM && kp.K == 128 && kp.logY2 == 5 && kp.M == 33)
        k_forward<THREADS_FWD, 128, 5, 33><<<grid, THREADS_FWD, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    else if (smem <= SMEM_FWD_3PERSM && kp.K == 128 && kp.logY2 == 5 && kp.M == 17)
        k_forward<THREADS_FWD, 128, 5, 17><<<grid, THREADS_FWD, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    else if (smem <= SMEM_FWD_3PERSM)
        k_forward<THREADS_FWD><<<grid, THREADS_FWD, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    else
        k_forward<1024><<<grid, 1024, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_outer(const KParams &kp, size_t smem, bool forward, void *stream) {
    if (kp.tcfrag) return launch_outer_tc(kp, smem, forward, stream);
    dim3 grid((unsigned)(kp.Y2 * (kp.Y1a * 2 * kp.K / kp.S2)), (unsigned)(forward ? 2 * kp.r : kp.r), 1);
    if (forward)
        k_outer<true><<<grid, THREADS_OUTER, smem, (cudaStream_t)stream>>>(kp);
    else
        k_outer<false><<<grid, THREADS_OUTER, smem, (cudaStream_t)stream>>>(kp);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int sm_count() {
    static int counts[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!counts[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        counts[dev] = n;
    }
    return counts[dev];
}

int middle_tiles(const KParams &kp) { return (int)(2 * kp.K / kp.S * kp.Y2 * kp.Y1b * kp.r); }

int launch_middle(const KParams &kp, size_t smem, void *stream) {
    if (kp.tcfrag) return launch_middle_tc(kp, smem, stream);
    // tiles small enough for two blocks per SM run in 256-thread blocks
    if (smem <= MID256_SMEM_MAX) return launch_middle256(kp, smem, stream);
    const unsigned grid = (unsigned)std::min(middle_tiles(kp), sm_count());
    // compile-time tile shapes (with the tables in shared memory the column
    // length log2 Y1a is the only length the stages use, split plan or not)
    const bool tsm = kp.mid_tables_in_smem != 0;
    if (tsm && kp.S == 4 && kp.logY1a == 12 && kp.K == 32)
        k_middle<true, 4, 12, 32><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    else if (tsm && kp.S == 8 && kp.logY1a == 11 && kp.K == 128)
        k_middle<true, 8, 11, 128><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    else if (tsm && kp.S == 16 && kp.logY1a == 10 && kp.K == 128)
        k_middle<true, 16, 10, 128><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    else if (kp.mid_tables_in_smem)
        k_middle<true><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    else
        k_middle<false><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_inverse(const KParams &kp, size_t smem, uint32_t *c, uint8_t *cn, void *stream) {
    if (kp.tcfrag) return launch_inverse_tc(kp, smem, c, cn, stream);
    dim3 grid((unsigned)kp.Y1, 1, 1);
    if (smem <= SMEM_INV_2PERSM && kp.K == 32 && kp.logY2 == 7 && kp.M == 33)
        k_inverse<THREADS_INV, 32, 7, 33><<<grid, THREADS_INV, smem, (cudaStream_t)stream>>>(kp, c, cn);
    else if (smem <= SMEM_INV_2PERSM && kp.K == 128 && kp.logY2 == 5 && kp.M == 33)
        k_inverse<THREADS_INV, 128, 5, 33><<<grid, THREADS_INV, smem, (cudaStream_t)stream>>>(kp, c, cn);
    else if (smem <= SMEM_INV_2PERSM && kp.K == 128 && kp.logY2 == 5 && kp.M == 17)
        k_inverse<THREADS_INV, 128, 5, 17><<<grid, THREADS_INV, smem, (cudaStream_t)stream>>>(kp, c, cn);
    else if (smem <= SMEM_INV_2PERSM)
        k_inverse<THREADS_INV><<<grid, THREADS_INV, smem, (cudaStream_t)stream>>>(kp, c, cn);
    else
        k_inverse<1024><<<grid, 1024, smem, (cudaStream_t)stream>>>(kp, c, cn);
    g_launches.fetch_add(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                   const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    if (sp.school) return launch_school(sp, a, an, b, bn, c, cn, stream);
    if (sp.ka.levels) return launch_kara_product(sp, a, an, b, bn, c, cn, stream);
    if (sp.bp.on) return launch_bigp_product(sp, a, an, b, bn, c, cn, stream);
    if (sp.kr.s > 1) return launch_kron_product(sp, a, an, b, bn, c, cn, stream);
    if (sp.ks.on) return launch_ks_product(sp, a, an, b, bn, c, cn, stream);
    return launch_transform_product(sp, a, an, b, bn, c, cn, stream);
}

int launch_transform_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                             const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    const KParams &kp = sp.kp;
    if (launch_forward(kp, sp.smem_fwd, a, an, b, bn, stream)) return -1;
    if (kp.Y1b > 1 && launch_outer(kp, sp.smem_outer, true, stream)) return -1;
    if (launch_middle(kp, sp.smem_mid, stream)) return -1;
    if (kp.Y1b > 1 && launch_outer(kp, sp.smem_outer, false, stream)) return -1;
    return launch_inverse(kp, sp.smem_inv, c, cn, stream);
}

}  // namespace ipm
