// ipm_kernels_batch.cu -- batched forward and inverse passes compiled for
// fixed (K, log2 Y2): the tile functions (passes.cuh) then fold their
// strides and stage radices as the single-product instantiations do.  A
// batched launch group orders its forward and inverse items by (K, log2 Y2)
// (ipm_api.cu, build_batch) and launches each run of one shape through the
// matching kernel here, the other runs through the generic kb_forward /
// kb_inverse.  The pairs are those that carry most of the transform points
// of uneven batches under the learned dispatch (K = 16 .. 128, Y2 = 32 ..
// 128).  Every block checks that its product has the kernel's shape and
// otherwise only flags ERRBIT_INTERNAL: a scheduling mistake cannot make a
// tile of one shape run with another shape's strides.
#include <cuda_runtime.h>

#include "ipm_internal.h"
#include "passes.cuh"

namespace ipm {

namespace {

template <int NT, int CK, int CLY2>
__global__ void __launch_bounds__(NT, NT == THREADS_FWD ? 3 : 1)
kb_forward_c(const KParams *__restrict__ Ps, const ipm_operands *__restrict__ ops, const uint2 *__restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const KParams &P = Ps[it.x];
    if (P.K != CK || P.logY2 != CLY2) {
        if (threadIdx.x == 0) atomicOr(P.err, ERRBIT_INTERNAL);
        return;
    }
    const ipm_operands o = ops[P.batch_index];
    const int op = (int64_t)it.y >= P.Y1 ? 1 : 0;
    fwd_tile<NoTc, CK, CLY2>(P, (int64_t)it.y - (op ? P.Y1 : 0), op, o.a, o.a_neg, o.b, o.b_neg);
}

template <int NT, int CK, int CLY2>
__global__ void __launch_bounds__(NT, NT == THREADS_INV ? 2 : 1)
kb_inverse_c(const KParams *__restrict__ Ps, const ipm_operands *__restrict__ ops, const uint2 *__restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const KParams &P = Ps[it.x];
    if (P.K != CK || P.logY2 != CLY2) {
        if (threadIdx.x == 0) atomicOr(P.err, ERRBIT_INTERNAL);
        return;
    }
    const ipm_operands o = ops[P.batch_index];
    inv_tile<NoTc, false, CK, CLY2>(P, it.y, o.c, o.c_neg);
}

// The instantiated (K, log2 Y2) pairs, one list for the dispatch below and
// the attribute setup.
#define IPM_BATCH_SHAPES(X) \
    X(64, 5)                \
    X(64, 6)                \
    X(128, 5)               \
    X(32, 5)                \
    X(32, 6)                \
    X(32, 7)                \
    X(16, 7)                \
    X(16, 6)

}  // namespace

bool batch_shape_compiled(int K, int logY2) {
#define IPM_X(k, l) \
    if (K == k && logY2 == l) return true;
    IPM_BATCH_SHAPES(IPM_X)
#undef IPM_X
    return false;
}

int set_kernel_attributes_batch() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
#define IPM_X(k, l)                                                   \
    set((const void *)kb_forward_c<THREADS_FWD, k, l>, SMEM_FWD_MAX); \
    set((const void *)kb_inverse_c<THREADS_INV, k, l>, SMEM_INV_MAX);
    IPM_BATCH_SHAPES(IPM_X)
#undef IPM_X
    return e == cudaSuccess ? 0 : -1;
}

// One run of items of shape (K, log2 Y2): the forward pass (fwd = true, the
// three-blocks-per-SM shape) or the inverse pass (the two-blocks-per-SM
// shape).  Returns 1 when no kernel is compiled for the shape (the caller
// launches the generic one), -1 on a launch error.
int launch_batch_run(bool fwd, int K, int logY2, const KParams *params, const ipm_operands *ops,
                     const uint2 *items, unsigned n, size_t smem, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
#define IPM_X(k, l)                                                                           \
    if (K == k && logY2 == l) {                                                               \
        if (fwd)                                                                              \
            kb_forward_c<THREADS_FWD, k, l><<<n, THREADS_FWD, smem, s>>>(params, ops, items); \
        else                                                                                  \
            kb_inverse_c<THREADS_INV, k, l><<<n, THREADS_INV, smem, s>>>(params, ops, items); \
        note_launches(1);                                                                     \
        return cudaGetLastError() == cudaSuccess ? 0 : -1;                                    \
    }
    IPM_BATCH_SHAPES(IPM_X)
#undef IPM_X
    return 1;
}

}  // namespace ipm
