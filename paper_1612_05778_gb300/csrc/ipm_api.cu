// ipm_api.cu -- the C ABI of include/ipm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "ipm_internal.h"
#include "ipm_mid256.h"

using namespace ipm;

struct ipm_plan_s {
    int device = 0;
    uint32_t flags = 0;
    std::vector<ShapePlan> shapes;
    std::vector<void *> allocations;  // device allocations owned by the plan
    uint32_t *Z = nullptr;            // shared workspace (largest shape)
    int *err = nullptr;               // device error word
    // ipm_mul_host staging (allocated on first use)
    unsigned char *io = nullptr;
    size_t io_bytes = 0;
    // batched calls (n > 1): groups of products launched together
    std::vector<BatchLaunch> batch;
    std::vector<char> batch_mid256;   // per group: middle pass in 256-thread blocks, two per SM
    ipm_operands *d_ops = nullptr;    // operand pointers of the current call
    // IPM_GRAPH: the grouped launches captured once into a CUDA graph
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_kernels = 0;
    // IPM_VALIDATE: partial sums of the evaluation check, and a call counter
    // that gives every check its own point
    uint64_t *val_part = nullptr;
    uint64_t val_calls = 0;
    ValBatch vb;  // batched calls: the work list of their check (fixed point)
    // IPM_PERSISTENT: one persistent launch over a device work queue
    bool persistent = false;
    PersistLaunch pl{};
    std::vector<int> need_host;       // tiles per (product, phase), as built
    int *need_dev = nullptr;
    int hold = -1;                    // ipm_debug_hold: product whose forward phase cannot complete
    // per-pass profiling events (ipm_set_profiling)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool profiling = false;
    bool profiled_once = false;
};

namespace {

ipm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return IPM_OK;
    if (e == cudaErrorMemoryAllocation) return IPM_ERR_NOMEM;
    return IPM_ERR_CUDA;
}

void free_plan(ipm_plan_s *p) {
    if (!p) return;
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    for (void *ptr : p->allocations) cudaFree(ptr);
    delete p;
}

bool aligned16(const void *ptr) { return ((uintptr_t)ptr & 15u) == 0; }

ipm_status run_product(ipm_plan_s *plan, const ShapePlan &sp, const uint32_t *a, const uint8_t *an,
                       const uint32_t *b, const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    if (!a || !an || !b || !bn || !c || !cn) return IPM_ERR_ARG;
    if (!aligned16(a) || !aligned16(b) || !aligned16(c)) return IPM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool prof = plan->profiling;
    // (packed, substituted and schoolbook plans are timed as one phase)
    if (!prof || sp.kr.s > 1 || sp.school || sp.ks.on || sp.ka.levels || sp.bp.on)
        return launch_product(sp, a, an, b, bn, c, cn, stream) ? IPM_ERR_CUDA : IPM_OK;
    // profiled: events around the three passes (a split plan's outer
    // passes count with the middle one)
    const KParams &kp = sp.kp;
    if (cudaEventRecord(plan->ev[0], s) != cudaSuccess) return IPM_ERR_CUDA;
    if (launch_forward(kp, sp.smem_fwd, a, an, b, bn, stream)) return IPM_ERR_CUDA;
    if (cudaEventRecord(plan->ev[1], s) != cudaSuccess) return IPM_ERR_CUDA;
    if (kp.Y1b > 1 && launch_outer(kp, sp.smem_outer, true, stream)) return IPM_ERR_CUDA;
    if (launch_middle(kp, sp.smem_mid, stream)) return IPM_ERR_CUDA;
    if (kp.Y1b > 1 && launch_outer(kp, sp.smem_outer, false, stream)) return IPM_ERR_CUDA;
    if (cudaEventRecord(plan->ev[2], s) != cudaSuccess) return IPM_ERR_CUDA;
    if (launch_inverse(kp, sp.smem_inv, c, cn, stream)) return IPM_ERR_CUDA;
    if (cudaEventRecord(plan->ev[3], s) != cudaSuccess) return IPM_ERR_CUDA;
    if (prof) plan->profiled_once = true;
    return IPM_OK;
}

// One product, then (IPM_VALIDATE) its randomised check at a fresh point.
ipm_status run_one(ipm_plan_s *plan, const ShapePlan &sp, const uint32_t *a, const uint8_t *an,
                   const uint32_t *b, const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream) {
    const ipm_status st = run_product(plan, sp, a, an, b, bn, c, cn, stream);
    if (st != IPM_OK || !(plan->flags & IPM_VALIDATE)) return st;
    const uint64_t t = validation_point(0x1612057780000000ull + plan->val_calls++);
    return launch_validate(sp.info, a, an, b, bn, c, cn, t, plan->val_part, plan->err, stream) ? IPM_ERR_CUDA
                                                                                                : IPM_OK;
}

ipm_status read_error(ipm_plan_s *plan, void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    int h = 0;
    e = cudaMemcpy(&h, plan->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (h) {
        e = cudaMemset(plan->err, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_status(e);
        if (h & ERRBIT_BOUND) return IPM_ERR_BOUND;
        if (h & ERRBIT_MISMATCH) return IPM_ERR_MISMATCH;
        if (h & ERRBIT_TIMEOUT) return IPM_ERR_TIMEOUT;
        return IPM_ERR_CUDA;
    }
    return IPM_OK;
}


// ---- batched schedule ------------------------------------------------------

// Products of one batched group run concurrently, each in its own slice of
// the workspace; a group is closed when the next product would take the
// group's workspace past this size (4 GiB), so memory stays bounded.
constexpr size_t kBatchWorkspaceWords = (size_t)1 << 30;

struct VariantKey {
    bool fwd_small, mid_tables, inv_small, mid256;
    bool operator<(const VariantKey &o) const {
        return std::tie(fwd_small, mid_tables, inv_small, mid256) <
               std::tie(o.fwd_small, o.mid_tables, o.inv_small, o.mid256);
    }
};

// mid256: the product's middle tiles can run as 256-thread blocks, two per
// SM (ipm_kernels_mid256.cu); such products are grouped apart so that one
// large tile does not keep a whole group on the 512-thread blocks
VariantKey variant_of(const ShapePlan &sp) {
    return VariantKey{sp.smem_fwd <= SMEM_FWD_3PERSM, sp.kp.mid_tables_in_smem != 0,
                      sp.smem_inv <= SMEM_INV_2PERSM, mid256_ok(sp.kp, sp.smem_mid)};
}

// Groups of shape indices: same kernel variants, bounded workspace,
// largest products first (they bound the group's run time).
std::vector<std::vector<int>> batch_groups(const std::vector<ShapePlan> &shapes) {
    std::map<VariantKey, std::vector<int>> by_variant;
    for (int i = 0; i < (int)shapes.size(); ++i)
        if (!runs_alone(shapes[(size_t)i])) by_variant[variant_of(shapes[(size_t)i])].push_back(i);
    std::vector<std::vector<int>> groups;
    for (auto &kv : by_variant) {
        auto &v = kv.second;
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
            return shapes[(size_t)x].z_words > shapes[(size_t)y].z_words;
        });
        std::vector<int> cur;
        size_t words = 0;
        for (int i : v) {
            const size_t z = shapes[(size_t)i].z_words;
            if (!cur.empty() && words + z > kBatchWorkspaceWords) {
                groups.push_back(cur);
                cur.clear();
                words = 0;
            }
            cur.push_back(i);
            words += z;
        }
        if (!cur.empty()) groups.push_back(cur);
    }
    return groups;
}

size_t batch_workspace_words(const std::vector<ShapePlan> &shapes) {
    size_t most = 0;
    for (const auto &g : batch_groups(shapes)) {
        size_t w = 0;
        for (int i : g) w += (shapes[(size_t)i].z_words + 63) & ~(size_t)63;
        most = std::max(most, w);
    }
    return most;
}

// IPM_GRAPH: record the grouped launches of a batched call once, on a
// plan-owned stream, into a CUDA graph.  Every kernel of the graph reads the
// operand pointers from the plan's device table (d_ops), which each call
// refreshes before launching the graph, so the graph stays valid for any
// operands.  Products that run alone are launched outside the graph.
// One group's three passes: the middle one in 256-thread blocks when the
// group qualifies (batch_mid256), else all three by launch_batch.
int launch_group(ipm_plan_s *plan, size_t g, void *stream) {
    const BatchLaunch &bl = plan->batch[g];
    if (!plan->batch_mid256[g]) return launch_batch(bl, plan->d_ops, stream);
    BatchLaunch fwd = bl, inv = bl;
    fwd.items[1] = fwd.items[2] = nullptr;
    inv.items[0] = inv.items[1] = nullptr;
    if (launch_batch(fwd, plan->d_ops, stream)) return -1;
    if (launch_batch_middle256(bl, stream)) return -1;
    return launch_batch(inv, plan->d_ops, stream);
}

ipm_status capture_batch(ipm_plan_s *plan) {
    cudaError_t ce;
    if (!plan->capture_stream) {
        ce = cudaStreamCreateWithFlags(&plan->capture_stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return cuda_status(ce);
    }
    const int64_t before = launches_so_far();
    ce = cudaStreamBeginCapture(plan->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_status(ce);
    bool failed = false;
    if (plan->persistent) {
        if (launch_persistent(plan->pl, plan->d_ops, plan->capture_stream)) failed = true;
    } else {
        for (size_t g = 0; g < plan->batch.size(); ++g)
            if (launch_group(plan, g, plan->capture_stream)) failed = true;
    }
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(plan->capture_stream, &g);
    const int captured = (int)(launches_so_far() - before);
    note_launches(-captured);  // recorded, not run
    if (failed || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return failed ? IPM_ERR_CUDA : cuda_status(ce);
    }
    ce = cudaGraphInstantiate(&plan->graph_exec, g, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(g);
        plan->graph_exec = nullptr;
        return cuda_status(ce);
    }
    plan->graph = g;
    plan->graph_kernels = captured;
    return IPM_OK;
}

// IPM_VALIDATE on a batched plan: items of up to VAL_ROWS rows of every
// operand of every product, each weighted by t^row0 for the plan's point t.
ipm_status build_val_batch(ipm_plan_s *plan) {
    const auto &shapes = plan->shapes;
    const uint64_t t = validation_point(0x5eed000000000000ull ^ (uint64_t)shapes.size());
    const uint64_t tR = pow61_host(t, VAL_ROWS);
    std::vector<ValItem> items;
    std::vector<int64_t> first;
    for (size_t i = 0; i < shapes.size(); ++i) {
        const ipm_plan_info &I = shapes[i].info;
        const int64_t rows[3] = {I.na, I.nb, I.nc};
        const int32_t limbs[3] = {I.la, I.lb, I.lc};
        for (int o = 0; o < 3; ++o) {
            first.push_back((int64_t)items.size());
            uint64_t w = 1;  // t^row0
            for (int64_t r0 = 0; r0 < rows[o]; r0 += VAL_ROWS) {
                ValItem it{};
                it.product = (int32_t)i;
                it.operand = o;
                it.row0 = r0;
                it.rows = (int32_t)std::min<int64_t>(VAL_ROWS, rows[o] - r0);
                it.limbs = limbs[o];
                it.t_row0 = w;
                items.push_back(it);
                w = (uint64_t)(((unsigned __int128)w * tR) % (((uint64_t)1 << 61) - 1));
            }
        }
    }
    first.push_back((int64_t)items.size());
    cudaError_t ce;
    void *d = nullptr;
    if ((ce = cudaMalloc(&d, items.size() * sizeof(ValItem))) != cudaSuccess) return cuda_status(ce);
    plan->allocations.push_back(d);
    if ((ce = cudaMemcpy(d, items.data(), items.size() * sizeof(ValItem), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_status(ce);
    plan->vb.items = (const ValItem *)d;
    if ((ce = cudaMalloc(&d, first.size() * sizeof(int64_t))) != cudaSuccess) return cuda_status(ce);
    plan->allocations.push_back(d);
    if ((ce = cudaMemcpy(d, first.data(), first.size() * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_status(ce);
    plan->vb.first = (const int64_t *)d;
    if ((ce = cudaMalloc(&d, items.size() * sizeof(uint64_t))) != cudaSuccess) return cuda_status(ce);
    plan->allocations.push_back(d);
    plan->vb.part = (uint64_t *)d;
    plan->vb.nitems = (int64_t)items.size();
    plan->vb.nproducts = (int32_t)shapes.size();
    plan->vb.t = t;
    return IPM_OK;
}

ipm_status build_batch(ipm_plan_s *plan) {
    const auto &shapes = plan->shapes;
    cudaError_t ce;
    void *d = nullptr;
    ce = cudaMalloc(&d, shapes.size() * sizeof(ipm_operands));
    if (ce != cudaSuccess) return cuda_status(ce);
    plan->allocations.push_back(d);
    plan->d_ops = (ipm_operands *)d;
    for (const auto &g : batch_groups(shapes)) {
        std::vector<KParams> params;
        std::vector<uint2> items[3];
        BatchLaunch bl{};
        const VariantKey vk = variant_of(shapes[(size_t)g[0]]);
        bl.fwd_small = vk.fwd_small;
        bl.mid_tables = vk.mid_tables;
        bl.inv_small = vk.inv_small;
        size_t zoff = 0;
        for (int i : g) {
            const ShapePlan &sp = shapes[(size_t)i];
            KParams kp = sp.kp;
            kp.Z = plan->Z + zoff;
            kp.batch_index = i;
            zoff += (sp.z_words + 63) & ~(size_t)63;
            const uint32_t pi = (uint32_t)params.size();
            params.push_back(kp);
            for (uint32_t t = 0; t < (uint32_t)(2 * kp.Y1); ++t) items[0].push_back(make_uint2(pi, t));
            const uint32_t nmid = (uint32_t)((2 * kp.K / kp.S) * kp.Y2 * kp.r);
            for (uint32_t t = 0; t < nmid; ++t) items[1].push_back(make_uint2(pi, t));
            for (uint32_t t = 0; t < (uint32_t)kp.Y1; ++t) items[2].push_back(make_uint2(pi, t));
            bl.smem[0] = std::max(bl.smem[0], sp.smem_fwd);
            bl.smem[1] = std::max(bl.smem[1], sp.smem_mid);
            bl.smem[2] = std::max(bl.smem[2], sp.smem_inv);
        }
        // forward and inverse items ordered by the (K, log2 Y2) of their
        // product: one run per shape with a compiled kernel
        // (ipm_kernels_batch.cu), the other shapes in one generic run
        auto key_of = [&](uint32_t pi) -> int64_t {
            const KParams &k = params[pi];
            return batch_shape_compiled(k.K, k.logY2) ? (((int64_t)k.K << 8) | k.logY2) : 0;
        };
        for (int p : {0, 2})
            std::stable_sort(items[p].begin(), items[p].end(),
                             [&](const uint2 &x, const uint2 &y) { return key_of(x.x) < key_of(y.x); });
        bl.nruns = 0;
        for (size_t a = 0, c = 0; a < items[0].size() || c < items[2].size();) {
            const int64_t kf = a < items[0].size() ? key_of(items[0][a].x) : INT64_MAX;
            const int64_t ki = c < items[2].size() ? key_of(items[2][c].x) : INT64_MAX;
            const int64_t k = std::min(kf, ki);
            BatchRun r{};
            r.K = (int32_t)(k >> 8);
            r.logY2 = (int32_t)(k & 255);
            r.f0 = (unsigned)a;
            while (a < items[0].size() && key_of(items[0][a].x) == k) ++a;
            r.nf = (unsigned)(a - r.f0);
            r.i0 = (unsigned)c;
            while (c < items[2].size() && key_of(items[2][c].x) == k) ++c;
            r.ni = (unsigned)(c - r.i0);
            if (bl.nruns == BATCH_RUNS_MAX) {  // more shapes than runs: one generic launch per pass
                bl.nruns = 0;
                break;
            }
            bl.runs[bl.nruns++] = r;
        }
        ce = cudaMalloc(&d, params.size() * sizeof(KParams));
        if (ce != cudaSuccess) return cuda_status(ce);
        plan->allocations.push_back(d);
        if ((ce = cudaMemcpy(d, params.data(), params.size() * sizeof(KParams), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_status(ce);
        bl.params = (const KParams *)d;
        for (int p = 0; p < 3; ++p) {
            ce = cudaMalloc(&d, items[p].size() * sizeof(uint2));
            if (ce != cudaSuccess) return cuda_status(ce);
            plan->allocations.push_back(d);
            if ((ce = cudaMemcpy(d, items[p].data(), items[p].size() * sizeof(uint2), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return cuda_status(ce);
            bl.items[p] = (const uint2 *)d;
            bl.nitems[p] = (unsigned)items[p].size();
        }
        plan->batch.push_back(bl);
        bool m256 = true;
        for (int i : g) m256 = m256 && mid256_ok(shapes[(size_t)i].kp, bl.smem[1]);
        plan->batch_mid256.push_back(m256 ? 1 : 0);
    }
    return IPM_OK;
}

// IPM_PERSISTENT: the work list of every product the persistent kernel
// runs (three-pass transform products and schoolbook products; the others
// still run one by one), each transform product in its own workspace
// slice, all of them at once.  Leaves plan->persistent false when a tile
// needs more shared memory than the persistent kernel can take.
ipm_status build_persistent(ipm_plan_s *plan) {
    const auto &shapes = plan->shapes;
    std::vector<int> members;
    size_t words = 0, smem = 0;
    for (int i = 0; i < (int)shapes.size(); ++i) {
        const ShapePlan &sp = shapes[(size_t)i];
        if (runs_alone(sp) && !sp.school) continue;
        members.push_back(i);
        if (sp.school) {
            smem = std::max(smem, school_smem(sp.kp));
        } else {
            words += (sp.z_words + 63) & ~(size_t)63;
            smem = std::max({smem, sp.smem_fwd, sp.smem_mid, sp.smem_inv});
        }
    }
    if (members.empty() || smem > PERSIST_SMEM_MAX) return IPM_OK;
    cudaError_t ce;
    void *d = nullptr;
    ce = cudaMalloc(&d, std::max<size_t>(words, 64) * sizeof(uint32_t));
    if (ce != cudaSuccess) return cuda_status(ce);
    plan->allocations.push_back(d);
    uint32_t *Zp = (uint32_t *)d;
    std::vector<KParams> params(shapes.size());
    size_t zoff = 0;
    for (int i : members) {
        KParams kp = shapes[(size_t)i].kp;
        kp.batch_index = i;
        if (!shapes[(size_t)i].school) {
            kp.Z = Zp + zoff;
            zoff += (shapes[(size_t)i].z_words + 63) & ~(size_t)63;
        }
        params[(size_t)i] = kp;
    }
    std::vector<PersistSeg> segs;
    int64_t nitems = 0;
    persist_schedule(shapes, members, segs, plan->need_host, nitems);
    auto upload = [&](const void *src, size_t bytes, void **dst) {
        if ((ce = cudaMalloc(dst, bytes)) != cudaSuccess) return false;
        plan->allocations.push_back(*dst);
        return (ce = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice)) == cudaSuccess;
    };
    if (!upload(params.data(), params.size() * sizeof(KParams), &d)) return cuda_status(ce);
    plan->pl.params = (const KParams *)d;
    if (!upload(segs.data(), segs.size() * sizeof(PersistSeg), &d)) return cuda_status(ce);
    plan->pl.segs = (const PersistSeg *)d;
    if (!upload(plan->need_host.data(), plan->need_host.size() * sizeof(int), &d)) return cuda_status(ce);
    plan->need_dev = (int *)d;
    plan->pl.need = plan->need_dev;
    const size_t ctl_bytes = sizeof(PersistControl) + 3 * shapes.size() * sizeof(int);
    if ((ce = cudaMalloc(&d, ctl_bytes)) != cudaSuccess) return cuda_status(ce);
    plan->allocations.push_back(d);
    plan->pl.ctl = (PersistControl *)d;
    plan->pl.done = (int *)((char *)d + sizeof(PersistControl));
    plan->pl.ctl_bytes = ctl_bytes;
    plan->pl.nseg = (int)segs.size();
    plan->pl.nitems = nitems;
    plan->pl.smem = smem;
    if (set_kernel_attributes_persist()) return IPM_ERR_CUDA;
    plan->pl.blocks = (unsigned)persist_blocks(smem);
    plan->pl.wait_cycles = (long long)(PERSIST_WAIT_US_DEFAULT * 2070);  // at most 2070 cycles per microsecond
    plan->persistent = true;
    return IPM_OK;
}

}  // namespace

extern "C" {

ipm_status ipm_plan_ex(ipm_plan_t *out, const ipm_shape *shapes, int32_t n, uint32_t flags,
                       const ipm_params *params) {
    if (!out) return IPM_ERR_ARG;
    *out = nullptr;
    if (!shapes || n < 1) return IPM_ERR_ARG;
    ipm_plan_s *plan = new (std::nothrow) ipm_plan_s();
    if (!plan) return IPM_ERR_NOMEM;
    plan->flags = flags;
    cudaError_t ce = cudaGetDevice(&plan->device);
    if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
    if (set_kernel_attributes() || set_kernel_attributes_mid256()) { free_plan(plan); return IPM_ERR_CUDA; }
    plan->shapes.resize((size_t)n);
    size_t zmax = 0;
    std::vector<ipm_params> learned;
    if ((flags & IPM_COSTMODEL) && !params) {
        learned.resize((size_t)n);
        std::vector<int32_t> src((size_t)n);
        ipm_status st = dispatch_params(shapes, n, learned.data(), src.data());
        if (st != IPM_OK) { free_plan(plan); return st; }
    }
    for (int32_t i = 0; i < n; ++i) {
        ipm_status st = choose_plan(shapes[i], learned.empty() ? params : &learned[(size_t)i],
                                    plan->shapes[(size_t)i]);
        if (st != IPM_OK) { free_plan(plan); return st; }
        zmax = std::max(zmax, plan->shapes[(size_t)i].z_words);
    }
    // Tables are shared between shapes with the same (Y, Y1, K, r): the
    // primes are always the r largest of the table, so these fix every entry.
    std::map<std::tuple<int64_t, int64_t, int32_t, int32_t>, const uint2 *> cache;
    for (auto &sp : plan->shapes) {
        if (sp.school || sp.ka.levels) continue;  // no transform tables
        if (sp.bp.on) {  // the big prime's own tables
            std::vector<uint64_t> words;
            bigp_tables(sp.bp, words);
            void *d = nullptr;
            ce = cudaMalloc(&d, words.size() * sizeof(uint64_t));
            if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
            plan->allocations.push_back(d);
            ce = cudaMemcpy(d, words.data(), words.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
            sp.bp.dtab = d;
            continue;
        }
        auto key = std::make_tuple(sp.kp.Y, sp.kp.Y1, sp.kp.K, sp.kp.r);
        std::vector<uint2> host((size_t)sp.kp.r * sp.table_words);
        build_tables(sp, host.data());  // also fills the scalar constants
        const uint2 *dtab = nullptr;
        auto it = cache.find(key);
        if (it != cache.end()) {
            dtab = it->second;
        } else {
            void *d = nullptr;
            ce = cudaMalloc(&d, host.size() * sizeof(uint2));
            if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
            plan->allocations.push_back(d);
            ce = cudaMemcpy(d, host.data(), host.size() * sizeof(uint2), cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
            dtab = (const uint2 *)d;
            cache[key] = dtab;
        }
        const TableLayout L = table_layout(sp.kp.Y, sp.kp.Y1, sp.kp.K);
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
    }
    // IPM_TENSOR_STAGES: the radix-16 fragment tables, one set for every
    // shape (prime t is the same for every shape: the r largest of the table)
    if (flags & IPM_TENSOR_STAGES) {
        const ShapePlan *wide = nullptr;
        for (auto &sp : plan->shapes)
            if (!sp.school && !sp.ka.levels && !sp.bp.on && (!wide || sp.kp.r > wide->kp.r)) wide = &sp;
        if (wide) {
            for (auto &sp : plan->shapes)
                for (int t = 0; !sp.school && !sp.ka.levels && !sp.bp.on && t < sp.kp.r; ++t)
                    if (sp.info.primes[t] != wide->info.primes[t]) { free_plan(plan); return IPM_ERR_UNSUPPORTED; }
            std::vector<uint32_t> frag((size_t)wide->kp.r * TC_FRAG_WORDS);
            build_tc_fragments(wide->info.primes, wide->kp.r, frag.data());
            void *d = nullptr;
            ce = cudaMalloc(&d, frag.size() * sizeof(uint32_t));
            if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
            plan->allocations.push_back(d);
            ce = cudaMemcpy(d, frag.data(), frag.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
            if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
            for (auto &sp : plan->shapes)
                if (!sp.school && !sp.ka.levels && !sp.bp.on) sp.kp.tcfrag = (const uint32_t *)d;
        }
    }
    // batched calls run a group's products at once: the workspace holds the
    // largest group (groups are cut at kBatchWorkspaceWords or one product)
    if (n > 1) zmax = std::max(zmax, batch_workspace_words(plan->shapes));
    zmax = std::max<size_t>(zmax, 64);  // schoolbook-only plans need none
    void *d = nullptr;
    ce = cudaMalloc(&d, zmax * sizeof(uint32_t));
    if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
    plan->allocations.push_back(d);
    plan->Z = (uint32_t *)d;
    ce = cudaMalloc(&d, 16);
    if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
    plan->allocations.push_back(d);
    plan->err = (int *)d;
    ce = cudaMemset(plan->err, 0, 16);
    if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
    for (auto &sp : plan->shapes) {
        sp.kp.Z = plan->Z;
        sp.kp.err = plan->err;
    }
    if (flags & IPM_VALIDATE) {
        ce = cudaMalloc(&d, 3 * VAL_BLOCKS * sizeof(uint64_t));
        if (ce != cudaSuccess) { free_plan(plan); return cuda_status(ce); }
        plan->allocations.push_back(d);
        plan->val_part = (uint64_t *)d;
    }
    if (n > 1) {
        ipm_status st = build_batch(plan);
        if (st == IPM_OK && (flags & IPM_PERSISTENT)) st = build_persistent(plan);
        if (st == IPM_OK && (flags & IPM_VALIDATE)) st = build_val_batch(plan);
        if (st != IPM_OK) { free_plan(plan); return st; }
    }
    *out = plan;
    return IPM_OK;
}

ipm_status ipm_plan(ipm_plan_t *out, const ipm_shape *shapes, int32_t n, uint32_t flags) {
    return ipm_plan_ex(out, shapes, n, flags, nullptr);
}

ipm_status ipm_get_info(ipm_plan_t plan, int32_t index, ipm_plan_info *out) {
    if (!plan || !out || index < 0 || (size_t)index >= plan->shapes.size()) return IPM_ERR_ARG;
    *out = plan->shapes[(size_t)index].info;
    return IPM_OK;
}

ipm_status ipm_mul(ipm_plan_t plan, const uint32_t *a, const uint8_t *a_neg, const uint32_t *b,
                   const uint8_t *b_neg, uint32_t *c, uint8_t *c_neg, ipm_stream_t stream) {
    if (!plan || plan->shapes.size() != 1) return IPM_ERR_ARG;
    ipm_status st = run_one(plan, plan->shapes[0], a, a_neg, b, b_neg, c, c_neg, stream);
    if (st != IPM_OK) return st;
    if (plan->flags & IPM_SYNC) return read_error(plan, stream);
    return IPM_OK;
}

ipm_status ipm_mul_host_async(ipm_plan_t plan, const uint32_t *a, const uint8_t *a_neg, const uint32_t *b,
                              const uint8_t *b_neg, uint32_t *c, uint8_t *c_neg, ipm_stream_t stream) {
    if (!plan || plan->shapes.size() != 1) return IPM_ERR_ARG;
    if (!a || !a_neg || !b || !b_neg || !c || !c_neg) return IPM_ERR_ARG;
    const ipm_plan_info &I = plan->shapes[0].info;
    auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t ba = (size_t)I.na * I.la * 4, bb = (size_t)I.nb * I.lb * 4, bc = (size_t)I.nc * I.lc * 4;
    const size_t oa = 0, oan = oa + up16(ba), ob = oan + up16((size_t)I.na), obn = ob + up16(bb),
                 oc = obn + up16((size_t)I.nb), ocn = oc + up16(bc), total = ocn + up16((size_t)I.nc);
    if (!plan->io) {
        void *d = nullptr;
        cudaError_t ce = cudaMalloc(&d, total);
        if (ce != cudaSuccess) return cuda_status(ce);
        plan->allocations.push_back(d);
        plan->io = (unsigned char *)d;
        plan->io_bytes = total;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *io = plan->io;
    cudaError_t ce;
    if ((ce = cudaMemcpyAsync(io + oa, a, ba, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(ce);
    if ((ce = cudaMemcpyAsync(io + oan, a_neg, (size_t)I.na, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(ce);
    if ((ce = cudaMemcpyAsync(io + ob, b, bb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(ce);
    if ((ce = cudaMemcpyAsync(io + obn, b_neg, (size_t)I.nb, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(ce);
    ipm_status st = run_one(plan, plan->shapes[0], (const uint32_t *)(io + oa), io + oan,
                            (const uint32_t *)(io + ob), io + obn, (uint32_t *)(io + oc), io + ocn, stream);
    if (st != IPM_OK) return st;
    if ((ce = cudaMemcpyAsync(c, io + oc, bc, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_status(ce);
    if ((ce = cudaMemcpyAsync(c_neg, io + ocn, (size_t)I.nc, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_status(ce);
    return IPM_OK;
}

ipm_status ipm_mul_host(ipm_plan_t plan, const uint32_t *a, const uint8_t *a_neg, const uint32_t *b,
                        const uint8_t *b_neg, uint32_t *c, uint8_t *c_neg, ipm_stream_t stream) {
    const ipm_status st = ipm_mul_host_async(plan, a, a_neg, b, b_neg, c, c_neg, stream);
    if (st != IPM_OK) return st;
    return read_error(plan, stream);
}

ipm_status ipm_mul_batched(ipm_plan_t plan, const ipm_operands *ops, int32_t n, ipm_stream_t stream) {
    if (!plan || !ops || n < 1 || (size_t)n != plan->shapes.size()) return IPM_ERR_ARG;
    for (int32_t i = 0; i < n; ++i) {
        const ipm_operands &o = ops[i];
        if (!o.a || !o.a_neg || !o.b || !o.b_neg || !o.c || !o.c_neg) return IPM_ERR_ARG;
        if (!aligned16(o.a) || !aligned16(o.b) || !aligned16(o.c)) return IPM_ERR_ARG;
    }
    if (n == 1) {
        const ipm_operands &o = ops[0];
        ipm_status st = run_one(plan, plan->shapes[0], o.a, o.a_neg, o.b, o.b_neg, o.c, o.c_neg, stream);
        if (st != IPM_OK) return st;
    } else {
        // operand pointers to the device (a pageable copy: the host array may
        // be reused as soon as this call returns)
        cudaError_t ce = cudaMemcpyAsync(plan->d_ops, ops, (size_t)n * sizeof(ipm_operands),
                                         cudaMemcpyHostToDevice, (cudaStream_t)stream);
        if (ce != cudaSuccess) return cuda_status(ce);
        if (plan->flags & IPM_GRAPH) {
            if (!plan->graph_exec) {
                ipm_status st = capture_batch(plan);
                if (st != IPM_OK) return st;
            }
            ce = cudaGraphLaunch(plan->graph_exec, (cudaStream_t)stream);
            if (ce != cudaSuccess) return cuda_status(ce);
            note_launches(plan->graph_kernels);
        } else if (plan->persistent) {
            if (launch_persistent(plan->pl, plan->d_ops, stream)) return IPM_ERR_CUDA;
        } else {
            for (size_t g = 0; g < plan->batch.size(); ++g)
                if (launch_group(plan, g, stream)) return IPM_ERR_CUDA;
        }
        // products whose middle transform is split or whose operands are
        // packed (and, without the persistent launch, schoolbook products)
        // run one after another
        for (int32_t i = 0; i < n; ++i) {
            const ShapePlan &sp = plan->shapes[(size_t)i];
            if (!runs_alone(sp) || (plan->persistent && sp.school)) continue;
            const ipm_operands &o = ops[i];
            if (launch_product(sp, o.a, o.a_neg, o.b, o.b_neg, o.c, o.c_neg, stream)) return IPM_ERR_CUDA;
        }
        if ((plan->flags & IPM_VALIDATE) && launch_validate_batch(plan->vb, plan->d_ops, plan->err, stream))
            return IPM_ERR_CUDA;
    }
    if (plan->flags & IPM_SYNC) return read_error(plan, stream);
    return IPM_OK;
}

ipm_status ipm_sync(ipm_plan_t plan, ipm_stream_t stream) {
    if (!plan) return IPM_ERR_ARG;
    return read_error(plan, stream);
}

ipm_status ipm_set_wait_limit(ipm_plan_t plan, uint64_t microseconds) {
    if (!plan || microseconds == 0 || microseconds > 600000000ull) return IPM_ERR_ARG;
    if (!plan->persistent) return IPM_ERR_UNSUPPORTED;
    plan->pl.wait_cycles = (long long)(microseconds * 2070);
    if (plan->graph_exec) {  // the recorded launch carries the old limit: record again on the next call
        cudaGraphExecDestroy(plan->graph_exec);
        cudaGraphDestroy(plan->graph);
        plan->graph_exec = nullptr;
        plan->graph = nullptr;
    }
    return IPM_OK;
}

ipm_status ipm_debug_hold(ipm_plan_t plan, int32_t product) {
    if (!plan || product < -1 || product >= (int32_t)plan->shapes.size()) return IPM_ERR_ARG;
    if (!plan->persistent) return IPM_ERR_UNSUPPORTED;
    std::vector<int> need = plan->need_host;
    if (product >= 0) {
        if (need[3 * (size_t)product] == 0) return IPM_ERR_ARG;  // not run by the persistent kernel
        need[3 * (size_t)product] += 1;  // one forward tile more than exist: never complete
    }
    cudaError_t ce = cudaMemcpy(plan->need_dev, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_status(ce);
    plan->hold = product;
    return IPM_OK;
}

ipm_status ipm_destroy(ipm_plan_t plan) {
    if (!plan) return IPM_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return IPM_OK;
}

ipm_status ipm_set_profiling(ipm_plan_t plan, int32_t enable) {
    if (!plan) return IPM_ERR_ARG;
    if (enable && !plan->ev[0]) {
        for (auto &e : plan->ev) {
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) return cuda_status(ce);
        }
    }
    plan->profiling = enable != 0;
    return IPM_OK;
}

ipm_status ipm_phase_ms(ipm_plan_t plan, float *ms, int32_t n) {
    if (!plan || !ms || n < 0 || !plan->ev[0] || !plan->profiled_once) return IPM_ERR_ARG;
    cudaError_t ce = cudaEventSynchronize(plan->ev[3]);
    if (ce != cudaSuccess) return cuda_status(ce);
    for (int32_t i = 0; i < n && i < 3; ++i) {
        ce = cudaEventElapsedTime(&ms[i], plan->ev[i], plan->ev[i + 1]);
        if (ce != cudaSuccess) return cuda_status(ce);
    }
    return IPM_OK;
}

const char *ipm_strerror(ipm_status s) {
    switch (s) {
        case IPM_OK: return "ok";
        case IPM_ERR_ARG: return "invalid argument";
        case IPM_ERR_BOUND: return "input coefficient exceeds its bit bound";
        case IPM_ERR_NOMEM: return "out of memory";
        case IPM_ERR_CUDA: return "CUDA error";
        case IPM_ERR_TIMEOUT: return "device wait timed out";
        case IPM_ERR_UNSUPPORTED: return "shape not supported";
        case IPM_ERR_MISMATCH: return "product failed its randomised check";
    }
    return "unknown status";
}

int64_t ipm_launch_count(void) { return launches_so_far(); }

}  // extern "C"
