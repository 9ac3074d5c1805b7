// ipm_noalloc.cu -- ipm_mul_noalloc: a product that allocates no memory.
//
// Who needs it: callers that must not allocate device memory while they
// run -- services with latency limits that forbid allocator calls
// (cudaMalloc can synchronise the device and take milliseconds), and
// plugins whose host application owns every allocation and gives the
// plugin only the input and output buffers.
//
// How: the error word, the twiddle tables and the transform workspace of
// one product live in one file-scope device array of fixed size,
// IPM_NOALLOC_SCRATCH_BYTES.  Every GPU that loads this library holds that
// array until the process exits.  The kernels are the same three passes
// ipm_mul launches; only where their scratch comes from differs.
//
// Rules (also in include/ipm.h):
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (host code may not use the symbol itself: on the
//    host it names a stand-in, not device memory) and sets the kernels'
//    shared-memory limits.  Make that first call before any stream capture.
//  * All calls share the array, which keeps the previous call's contents.
//    The error word is cleared and the tables rewritten on every call; the
//    workspace is fully written before it is read.  Calls are serialised
//    by g_lock, held until the call's stream has finished, so two calls
//    never overlap on the GPU.
//  * The call waits for its stream and returns the product's device status.
#include <cuda_runtime.h>

#include <mutex>

#include "ipm_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[IPM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices] = {};   // device address per device
std::mutex g_lock;  // held through the whole call: the host table buffer and the device array

// Host staging for the tables: the largest table set that can fit the
// device array.  Static storage, so no allocation happens at call time.
constexpr size_t kMaxTableEntries = IPM_NOALLOC_SCRATCH_BYTES / sizeof(uint2);
uint2 g_host_tables[kMaxTableEntries];

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

ipm_status setup_device(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return IPM_ERR_UNSUPPORTED;
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) return IPM_ERR_CUDA;
        if (ipm::set_kernel_attributes()) return IPM_ERR_CUDA;
        g_scratch_dev[dev] = (unsigned char *)ptr;
    }
    *out = g_scratch_dev[dev];
    return IPM_OK;
}

}  // namespace

extern "C" ipm_status ipm_mul_noalloc(const ipm_shape *shape, const uint32_t *a,
                                      const uint8_t *a_neg, const uint32_t *b,
                                      const uint8_t *b_neg, uint32_t *c, uint8_t *c_neg,
                                      ipm_stream_t stream) {
    if (!shape || !a || !a_neg || !b || !b_neg || !c || !c_neg) return IPM_ERR_ARG;
    if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15u) return IPM_ERR_ARG;
    ipm::ShapePlan sp;
    ipm_status st = ipm::choose_plan(*shape, nullptr, sp);
    if (st != IPM_OK) return st;
    const size_t err_bytes = 256;
    const size_t tab_entries = (size_t)sp.kp.r * sp.table_words;
    const size_t tab_bytes = up256(tab_entries * sizeof(uint2));
    const size_t z_bytes = sp.z_words * sizeof(uint32_t);
    if (err_bytes + tab_bytes + z_bytes > IPM_NOALLOC_SCRATCH_BYTES || tab_entries > kMaxTableEntries)
        return IPM_ERR_UNSUPPORTED;  // the product needs more than the static scratch

    std::lock_guard<std::mutex> guard(g_lock);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IPM_ERR_CUDA;
    unsigned char *base = nullptr;
    st = setup_device(dev, &base);
    if (st != IPM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = (int *)base;
    uint2 *dtab = (uint2 *)(base + err_bytes);
    uint32_t *Z = (uint32_t *)(base + err_bytes + tab_bytes);

    ipm::build_tables(sp, g_host_tables);  // also fills the scalar constants
    // pageable source: the copy has left g_host_tables when this returns
    if (cudaMemcpyAsync(dtab, g_host_tables, tab_entries * sizeof(uint2), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return IPM_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return IPM_ERR_CUDA;
    const ipm::TableLayout L = ipm::table_layout(sp.kp.Y, sp.kp.Y1, sp.kp.K);
    for (int t = 0; t < sp.kp.r; ++t) {
        const uint2 *blk = dtab + (size_t)t * L.total;
        sp.kp.pc[t].ty_f = blk + L.ty_f;
        sp.kp.pc[t].ty_i = blk + L.ty_i;
        sp.kp.pc[t].t1_f = blk + L.t1_f;
        sp.kp.pc[t].t1_i = blk + L.t1_i;
        sp.kp.pc[t].tx_f = blk + L.tx_f;
        sp.kp.pc[t].tx_i = blk + L.tx_i;
        sp.kp.pc[t].untw = blk + L.untw;
    }
    sp.kp.Z = Z;
    sp.kp.err = err;
    if (ipm::launch_product(sp, a, a_neg, b, b_neg, c, c_neg, stream)) return IPM_ERR_CUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return IPM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return IPM_ERR_CUDA;
    if (h & ipm::ERRBIT_BOUND) return IPM_ERR_BOUND;
    if (h) return IPM_ERR_CUDA;
    return IPM_OK;
}
