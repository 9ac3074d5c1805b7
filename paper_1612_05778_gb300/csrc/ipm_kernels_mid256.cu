// ipm_kernels_mid256.cu -- the middle pass in blocks of 256 threads, two
// per SM, for products (and batch groups) whose middle tiles fit two
// blocks' shared memory.  Same tile function as k_middle / kb_middle
// (passes.cuh); two independent blocks per SM overlap one block's tile
// copies with the other block's transforms (measured on a 1024-row,
// 8-column tile: 0.433 ms against 0.520 ms for one 512-thread block per SM).
#include <cuda_runtime.h>

#include <algorithm>

#include "ipm_internal.h"
#include "ipm_mid256.h"
#include "passes.cuh"

namespace ipm {

namespace {
constexpr int THREADS_MID2 = 256;
}

template <bool SMTW>
__global__ void __launch_bounds__(THREADS_MID2, 2)
kb_middle256(const KParams *__restrict__ Ps, const uint2 *__restrict__ items) {
    const uint2 it = items[blockIdx.x];
    const KParams &P = Ps[it.x];
    const int ncs = 2 * P.K / P.S;
    const int cs = (int)(it.y % (uint32_t)ncs);
    const int rest = (int)(it.y / (uint32_t)ncs);  // (t, pos) of an unsplit plan
    mid_tile<SMTW, NoTc>(P, cs, rest % (int)P.Y2, 0, rest / (int)P.Y2);
}

// single product, persistent: two blocks per SM walk the tile list
// (passes.cuh, mid_tiles)
template <bool SMTW>
__global__ void __launch_bounds__(THREADS_MID2, 2) k_middle256(const __grid_constant__ KParams P) {
    mid_tiles<SMTW>(P);
}

int set_kernel_attributes_mid256() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MID256_SMEM_MAX);
    };
    set((const void *)kb_middle256<true>);
    set((const void *)kb_middle256<false>);
    set((const void *)k_middle256<true>);
    set((const void *)k_middle256<false>);
    return e == cudaSuccess ? 0 : -1;
}

int launch_middle256(const KParams &kp, size_t smem, void *stream) {
    const unsigned grid = (unsigned)std::min(middle_tiles(kp), 2 * sm_count());
    if (kp.mid_tables_in_smem)
        k_middle256<true><<<grid, THREADS_MID2, smem, (cudaStream_t)stream>>>(kp);
    else
        k_middle256<false><<<grid, THREADS_MID2, smem, (cudaStream_t)stream>>>(kp);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_batch_middle256(const BatchLaunch &bl, void *stream) {
    if (!bl.items[1]) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (bl.mid_tables)
        kb_middle256<true><<<bl.nitems[1], THREADS_MID2, bl.smem[1], s>>>(bl.params, bl.items[1]);
    else
        kb_middle256<false><<<bl.nitems[1], THREADS_MID2, bl.smem[1], s>>>(bl.params, bl.items[1]);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// A group may take the 256-thread middle when its largest tile fits two
// blocks per SM (the tile function works with any block size).
bool mid256_ok(const KParams &, size_t smem_mid) { return smem_mid <= MID256_SMEM_MAX; }

}  // namespace ipm
