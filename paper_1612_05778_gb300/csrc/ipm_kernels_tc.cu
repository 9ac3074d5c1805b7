// ipm_kernels_tc.cu -- the passes of one product with every radix-16
// transform stage on the INT8 tensor cores (plan flag IPM_TENSOR_STAGES):
// the tile functions of passes.cuh instantiated with TC = TcOn.  Stages
// of other radices, the fused pointwise stage, digits, CRT and
// recombination are those of the integer path, so both paths compute the
// same exact product.  Batched launches (kb_*) keep the integer stages.
#include <cuda_runtime.h>

#include "ipm_internal.h"
#include "passes.cuh"

namespace ipm {

template <int NT>
__global__ void __launch_bounds__(NT, NT == THREADS_FWD ? 3 : 1)
k_forward_tc(const __grid_constant__ KParams P, const uint32_t *__restrict__ a, const uint8_t *__restrict__ an,
             const uint32_t *__restrict__ b, const uint8_t *__restrict__ bn) {
    fwd_tile<TcOn>(P, blockIdx.x, blockIdx.y, a, an, b, bn);
}

template <bool SMTW>
__global__ void __launch_bounds__(THREADS_MID, 1) k_middle_tc(const __grid_constant__ KParams P) {
    mid_tile<SMTW, TcOn>(P, blockIdx.x, blockIdx.y >> P.logY1b, blockIdx.y & (P.Y1b - 1), blockIdx.z);
}

template <bool FWD>
__global__ void __launch_bounds__(THREADS_OUTER) k_outer_tc(const __grid_constant__ KParams P) {
    const int lnb = P.logY1a + P.logK + 1 - P.logS2;
    const size_t wb = blockIdx.x & ((1u << lnb) - 1);
    const int pos = (int)(blockIdx.x >> lnb);
    const int t = FWD ? (int)(blockIdx.y >> 1) : (int)blockIdx.y;
    const int op = FWD ? (int)(blockIdx.y & 1) : 0;
    outer_tile<FWD, TcOn>(P, pos, wb << P.logS2, t, op);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == THREADS_INV ? 2 : 1)
k_inverse_tc(const __grid_constant__ KParams P, uint32_t *__restrict__ c, uint8_t *__restrict__ cn) {
    inv_tile<TcOn>(P, blockIdx.x, c, cn);
}

int set_kernel_attributes_tc() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_forward_tc<THREADS_FWD>, SMEM_FWD_MAX);
    set((const void *)k_forward_tc<1024>, SMEM_FWD_MAX);
    set((const void *)k_middle_tc<true>, SMEM_MID_MAX);
    set((const void *)k_middle_tc<false>, SMEM_MID_MAX);
    set((const void *)k_inverse_tc<THREADS_INV>, SMEM_INV_MAX);
    set((const void *)k_inverse_tc<1024>, SMEM_INV_MAX);
    set((const void *)k_outer_tc<true>, SMEM_MID_MAX);
    set((const void *)k_outer_tc<false>, SMEM_MID_MAX);
    return e == cudaSuccess ? 0 : -1;
}

// Grids and block sizes as in ipm_kernels.cu.
int launch_forward_tc(const KParams &kp, size_t smem, const uint32_t *a, const uint8_t *an,
                      const uint32_t *b, const uint8_t *bn, void *stream) {
    dim3 grid((unsigned)kp.Y1, 2, 1);
    if (smem <= SMEM_FWD_3PERSM)
        k_forward_tc<THREADS_FWD><<<grid, THREADS_FWD, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    else
        k_forward_tc<1024><<<grid, 1024, smem, (cudaStream_t)stream>>>(kp, a, an, b, bn);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_outer_tc(const KParams &kp, size_t smem, bool forward, void *stream) {
    dim3 grid((unsigned)(kp.Y2 * (kp.Y1a * 2 * kp.K / kp.S2)), (unsigned)(forward ? 2 * kp.r : kp.r), 1);
    if (forward)
        k_outer_tc<true><<<grid, THREADS_OUTER, smem, (cudaStream_t)stream>>>(kp);
    else
        k_outer_tc<false><<<grid, THREADS_OUTER, smem, (cudaStream_t)stream>>>(kp);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_middle_tc(const KParams &kp, size_t smem, void *stream) {
    dim3 grid((unsigned)(2 * kp.K / kp.S), (unsigned)(kp.Y2 * kp.Y1b), (unsigned)kp.r);
    if (kp.mid_tables_in_smem)
        k_middle_tc<true><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    else
        k_middle_tc<false><<<grid, THREADS_MID, smem, (cudaStream_t)stream>>>(kp);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_inverse_tc(const KParams &kp, size_t smem, uint32_t *c, uint8_t *cn, void *stream) {
    dim3 grid((unsigned)kp.Y1, 1, 1);
    if (smem <= SMEM_INV_2PERSM)
        k_inverse_tc<THREADS_INV><<<grid, THREADS_INV, smem, (cudaStream_t)stream>>>(kp, c, cn);
    else
        k_inverse_tc<1024><<<grid, 1024, smem, (cudaStream_t)stream>>>(kp, c, cn);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
