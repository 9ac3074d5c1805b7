// ipm_persist.cu -- a batched call as ONE persistent launch over a device
// work queue (plan flag IPM_PERSISTENT).  The paper multiplies one pair at a
// time; this is the batch form of its three steps per product (§2.4's
// parallel loops become tiles of a shared queue).
//
// Work list.  Every product of the batch (those of the three-pass transform
// path, and schoolbook products) becomes segments of items (product, phase,
// tile): phase 0 the forward tiles (or a schoolbook product's output
// coefficients), phase 1 the middle tiles, phase 2 the inverse tiles.
// Products are cut into windows of at most PERSIST_WINDOW_WORDS of
// workspace, and the segments are ordered as a software pipeline over the
// windows: step s holds window s's forward tiles, window s-1's middle tiles
// and window s-2's inverse tiles, so a tile's inputs were produced a step
// earlier (rarely still in flight) and, windows being small, are often
// still in L2.
//
// Queue and dependencies.  Blocks take items in list order, PERSIST_CHUNK
// tiles of one segment per atomic increment (the next chunk is reserved while
// the current one runs); an item of phase f > 0 of product p may start once all phase
// f-1 tiles of p are done: a per-product counter that each finished tile
// increments after a memory fence, which the waiting block polls (volatile
// reads, __nanosleep between polls).  No deadlock: a block only waits for
// items taken earlier by running blocks, whose own waits concern still
// earlier items.  Every wait has a limit in clock cycles; when it runs out
// the block sets ERRBIT_TIMEOUT in the error word and a shared abort flag,
// and every block returns at its next item or poll, so the launch always
// ends and the context stays usable; the call then reports IPM_ERR_TIMEOUT.
//
// Coherence.  L1 is not kept coherent between SMs within a launch.  The
// middle tiles read the forward output through L2 only (their COH form),
// so no SM holds a line of a product's workspace from before the middle
// pass overwrites it (middle slices share 32-byte sectors, so an
// L1-allocating read could pull in a neighbouring slice that another SM
// overwrites later); the inverse tiles then read final data and keep their
// asynchronous, L1-allocating copies.  Forward tiles read only the inputs.
//
// Block shape.  Batches whose every tile fits 113 KB of shared memory run
// 256-thread blocks, two per SM; others 512-thread blocks, one per SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ipm_internal.h"
#include "passes.cuh"
#include "school.cuh"

namespace ipm {

namespace {


// The segment holding queue index idx, searched forward from segment `from`
// (a block's indices only grow): one probe when idx is still in `from`'s
// segment, else a galloping search.  seg[s].start is in chunk units.
__device__ __forceinline__ int find_segment(const PersistSeg *__restrict__ seg, int nseg, int64_t idx, int from) {
    int lo = from;
    if (lo + 1 >= nseg || seg[lo + 1].start > idx) return lo;
    int step = 1, hi = lo + 1;
    while (hi < nseg && seg[hi].start <= idx) {
        lo = hi;
        step <<= 1;
        hi = lo + step;
    }
    if (hi > nseg) hi = nseg;
    // seg[lo].start <= idx < seg[hi].start (or hi = nseg)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (seg[mid].start <= idx)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1)
k_batch_persistent(const KParams *__restrict__ Ps, const ipm_operands *__restrict__ ops,
                   const PersistSeg *__restrict__ seg, int nseg, int64_t nitems, const int *__restrict__ need,
                   PersistControl *ctl, int *done_all, long long wait_cycles) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_idx;
    __shared__ int s_seg, s_go;
    int64_t next = 0;  // thread 0: the chunk reserved while the current one runs
    int from = 0;      // thread 0: segment of the previous chunk
    if (threadIdx.x == 0) next = (int64_t)atomicAdd(&ctl->head, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            const bool aborted = *(volatile int *)&ctl->abort != 0;
            const int64_t idx = aborted ? nitems : next;
            if (idx < nitems) {
                from = find_segment(seg, nseg, idx, from);
                next = (int64_t)atomicAdd(&ctl->head, 1ull);  // reserve the next chunk now
            }
            s_idx = idx;
            s_seg = from;
        }
        __syncthreads();
        const int64_t idx = s_idx;
        if (idx >= nitems) return;
        const PersistSeg S = seg[s_seg];
        const int p = S.product, f = S.phase;
        const int64_t t0 = (idx - S.start) * PERSIST_CHUNK;
        const int64_t t1 = min(t0 + PERSIST_CHUNK, (int64_t)S.tiles);
        const KParams &P = Ps[p];
        // wait for the previous phase of this product
        if (threadIdx.x == 0) {
            int go = 1;
            if (f > 0) {
                const volatile int *done = done_all + 3 * p + f - 1;
                const int target = need[3 * p + f - 1];
                const long long c0 = clock64();
                while (*done < target) {
                    if (*(volatile int *)&ctl->abort) {
                        go = 0;
                        break;
                    }
                    if (clock64() - c0 > wait_cycles) {
                        atomicOr(P.err, ERRBIT_TIMEOUT);
                        atomicExch(&ctl->abort, 1);
                        go = 0;
                        break;
                    }
                    __nanosleep(256);
                }
                __threadfence();
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) return;
        const ipm_operands o = ops[P.batch_index];
        for (int64_t tile = t0; tile < t1; ++tile) {
            if (P.K == 0) {  // schoolbook product: tile = output coefficient
                school_tile(P, tile, o.a, o.a_neg, o.b, o.b_neg, o.c, o.c_neg, smem);
            } else if (f == 0) {
                const int op = tile >= P.Y1 ? 1 : 0;
                fwd_tile<NoTc>(P, tile - (op ? P.Y1 : 0), op, o.a, o.a_neg, o.b, o.b_neg);
            } else if (f == 1) {
                const int ncs = 2 * P.K / P.S;
                const int cs = (int)(tile % ncs), rest = (int)(tile / ncs);
                if (P.mid_tables_in_smem)
                    mid_tile<true, NoTc, true>(P, cs, rest % (int)P.Y2, 0, rest / (int)P.Y2);
                else
                    mid_tile<false, NoTc, true>(P, cs, rest % (int)P.Y2, 0, rest / (int)P.Y2);
            } else {
                inv_tile<NoTc>(P, tile, o.c, o.c_neg);
            }
            __syncthreads();  // the next tile reuses the shared memory
        }
        // publish: every thread's stores before the counter moves
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done_all + 3 * p + f, (int)(t1 - t0));
    }
}

}  // namespace

// Segments of a batch: products in order, cut into windows, ordered as the
// three-stage pipeline over windows.  need[3 p + f]: phase f's tile count.
void persist_schedule(const std::vector<ShapePlan> &shapes, const std::vector<int> &members,
                      std::vector<PersistSeg> &segs, std::vector<int> &need, int64_t &nitems) {
    need.assign(3 * shapes.size(), 0);
    std::vector<std::vector<int>> windows;
    std::vector<int> cur;
    size_t words = 0;
    for (int i : members) {
        const size_t z = (shapes[(size_t)i].z_words + 63) & ~(size_t)63;
        if (!cur.empty() && words + z > PERSIST_WINDOW_WORDS) {
            windows.push_back(cur);
            cur.clear();
            words = 0;
        }
        cur.push_back(i);
        words += z;
    }
    if (!cur.empty()) windows.push_back(cur);
    for (int i : members) {
        const ShapePlan &sp = shapes[(size_t)i];
        const KParams &kp = sp.kp;
        if (sp.school) {
            need[3 * i] = (int)kp.nc;
        } else {
            need[3 * i] = (int)(2 * kp.Y1);
            need[3 * i + 1] = (int)((2 * kp.K / kp.S) * kp.Y2 * kp.r);
            need[3 * i + 2] = (int)kp.Y1;
        }
    }
    segs.clear();
    int64_t at = 0;
    const int nw = (int)windows.size();
    for (int step = 0; step < nw + 2; ++step)
        for (int f = 0; f < 3; ++f) {
            const int w = step - f;
            if (w < 0 || w >= nw) continue;
            for (int i : windows[(size_t)w]) {
                const int n = need[3 * i + f];
                if (n == 0) continue;
                segs.push_back(PersistSeg{at, i, f, n, 0});
                at += (n + PERSIST_CHUNK - 1) / PERSIST_CHUNK;  // queue entries are chunks of tiles
            }
        }
    nitems = at;
}

// 256-thread blocks when every tile fits two blocks' shared memory per SM.
int persist_threads(size_t smem) { return smem <= PERSIST_SMEM_SMALL ? 256 : 512; }

int persist_blocks(size_t smem) {
    int per_sm = 0;
    const cudaError_t e = persist_threads(smem) == 256
                              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<256>, 256, smem)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_persistent<512>, 512, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * sm_count();
}

int set_kernel_attributes_persist() {
    cudaError_t e = cudaFuncSetAttribute((const void *)k_batch_persistent<256>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PERSIST_SMEM_SMALL);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)k_batch_persistent<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PERSIST_SMEM_MAX);
    return e == cudaSuccess ? 0 : -1;
}

int launch_persistent(const PersistLaunch &pl, const ipm_operands *ops, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(pl.ctl, 0, pl.ctl_bytes, s) != cudaSuccess) return -1;
    if (persist_threads(pl.smem) == 256)
        k_batch_persistent<256><<<pl.blocks, 256, pl.smem, s>>>(pl.params, ops, pl.segs, pl.nseg, pl.nitems, pl.need,
                                                               pl.ctl, pl.done, pl.wait_cycles);
    else
        k_batch_persistent<512><<<pl.blocks, 512, pl.smem, s>>>(pl.params, ops, pl.segs, pl.nseg, pl.nitems, pl.need,
                                                               pl.ctl, pl.done, pl.wait_cycles);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
