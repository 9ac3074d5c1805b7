// ipm_mlp.cu -- the learned cost model: a small multilayer perceptron that
// maps a candidate plan's features (IPM_FEATURES numbers, ipm_candidates) to
// its predicted log run time, trained on autotuning sweep timings.
//
// Network: IPM_FEATURES -> 32 (ReLU) -> 32 (ReLU) -> 1, on standardised
// features and targets.  Model layout (floats, IPM_MLP_FLOATS in total):
//   [0,F) feature means, [F,2F) inverse standard deviations,
//   2F target mean, 2F+1 target standard deviation,
//   then W1[32][F], b1[32], W2[32][32], b2[32], w3[32], b3.
//
// Kernels: k_mlp_grad (one thread per sample: forward, backward, gradients
// summed per block in shared memory then into global memory), k_mlp_adam
// (Adam step, D. Kingma and J. Ba, "Adam: A method for stochastic
// optimization", ICLR 2015), k_mlp_predict (forward).  Training is full
// batch; float atomic sums make the last bits of a trained model depend on
// scheduling, while every plan the model can choose computes the same exact
// product.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ipm_internal.h"

namespace {

constexpr int F = IPM_FEATURES;
constexpr int H = 32;
constexpr int NPARAM = H * F + H + H * H + H + H + 1;
constexpr int HEAD = 2 * F + 2;
static_assert(NPARAM == IPM_MLP_PARAMS && HEAD + NPARAM == IPM_MLP_FLOATS, "model layout");

struct Net {
    const float *W1, *b1, *W2, *b2, *w3, *b3;
};
__host__ __device__ inline Net net_of(const float *p) {
    Net n;
    n.W1 = p;
    n.b1 = n.W1 + H * F;
    n.W2 = n.b1 + H;
    n.b2 = n.W2 + H * H;
    n.w3 = n.b2 + H;
    n.b3 = n.w3 + H;
    return n;
}

// Forward of one standardised sample; keeps the activations for backward.
__device__ inline float forward(const Net &n, const float *x, float *h1, float *h2) {
    for (int i = 0; i < H; ++i) {
        float s = n.b1[i];
        for (int k = 0; k < F; ++k) s += n.W1[i * F + k] * x[k];
        h1[i] = s > 0.f ? s : 0.f;
    }
    for (int i = 0; i < H; ++i) {
        float s = n.b2[i];
        for (int k = 0; k < H; ++k) s += n.W2[i * H + k] * h1[k];
        h2[i] = s > 0.f ? s : 0.f;
    }
    float o = n.b3[0];
    for (int k = 0; k < H; ++k) o += n.w3[k] * h2[k];
    return o;
}

__device__ inline void standardise(const float *model, const float *raw, float *x) {
    for (int k = 0; k < F; ++k) x[k] = (raw[k] - model[k]) * model[F + k];
}

__device__ inline float warp_sum(float v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over samples of the squared error 1/2 (o - t)^2 (o the output, t the
// standardised target) and its gradient with respect to every parameter.
// One thread per sample; each parameter's contributions are summed across
// the warp with shuffles, across the block in shared memory and across
// blocks with global atomics.  Threads past n contribute zero.
__global__ void __launch_bounds__(128) k_mlp_grad(const float *__restrict__ model, const float *__restrict__ X,
                                                   const float *__restrict__ y, int n, float *__restrict__ grad,
                                                   float *__restrict__ loss) {
    __shared__ float g[NPARAM + 1];
    for (int i = threadIdx.x; i <= NPARAM; i += blockDim.x) g[i] = 0.f;
    __syncthreads();
    const Net net = net_of(model + HEAD);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const bool lane0 = (threadIdx.x & 31) == 0;
    float x[F], h1[H], h2[H], d1[H], d2[H];
    float d = 0.f;
    if (s < n) {
        standardise(model, X + (size_t)s * F, x);
        const float o = forward(net, x, h1, h2);
        d = o - (y[s] - model[2 * F]) / model[2 * F + 1];
    } else {
        for (int k = 0; k < F; ++k) x[k] = 0.f;
        for (int k = 0; k < H; ++k) h1[k] = h2[k] = 0.f;
    }
    // backward: d2 = dL/d(layer-2 pre-activation), d1 = dL/d(layer-1 pre-activation)
    for (int k = 0; k < H; ++k) d2[k] = h2[k] > 0.f ? d * net.w3[k] : 0.f;
    for (int k = 0; k < H; ++k) {
        float t = 0.f;
        for (int i = 0; i < H; ++i) t += d2[i] * net.W2[i * H + k];
        d1[k] = h1[k] > 0.f ? t : 0.f;
    }
    auto acc = [&](int idx, float v) {
        v = warp_sum(v);
        if (lane0) atomicAdd(&g[idx], v);
    };
    const int oW1 = 0, ob1 = H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, ow3 = ob2 + H, ob3 = ow3 + H;
    acc(NPARAM, 0.5f * d * d);
    acc(ob3, d);
    for (int k = 0; k < H; ++k) acc(ow3 + k, d * h2[k]);
    for (int i = 0; i < H; ++i) {
        acc(ob2 + i, d2[i]);
        for (int k = 0; k < H; ++k) acc(oW2 + i * H + k, d2[i] * h1[k]);
    }
    for (int i = 0; i < H; ++i) {
        acc(ob1 + i, d1[i]);
        for (int k = 0; k < F; ++k) acc(oW1 + i * F + k, d1[i] * x[k]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) atomicAdd(&grad[i], g[i]);
    if (threadIdx.x == 0) atomicAdd(loss, g[NPARAM]);
}

__global__ void k_mlp_adam(float *__restrict__ params, const float *__restrict__ grad, float *__restrict__ m,
                           float *__restrict__ v, float scale, float lr, float b1, float b2, float c1,
                           float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i] * scale;
    m[i] = b1 * m[i] + (1.f - b1) * g;
    v[i] = b2 * v[i] + (1.f - b2) * g * g;
    params[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + 1e-8f);
}

__global__ void k_mlp_predict(const float *__restrict__ model, const float *__restrict__ X, int n,
                              float *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const Net net = net_of(model + HEAD);
    float x[F], h1[H], h2[H];
    standardise(model, X + (size_t)s * F, x);
    out[s] = forward(net, x, h1, h2) * model[2 * F + 1] + model[2 * F];
}

// splitmix64 (S. Vigna): the initial weights are a function of the seed.
uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t bytes) { return cudaMalloc(&p, bytes) == cudaSuccess; }
    float *f() const { return (float *)p; }
};

std::mutex g_model_lock;
std::vector<float> g_model;  // ipm_set_cost_model

ipm_status st_of(cudaError_t e) { return e == cudaSuccess ? IPM_OK : (e == cudaErrorMemoryAllocation ? IPM_ERR_NOMEM : IPM_ERR_CUDA); }

}  // namespace

extern "C" ipm_status ipm_mlp_grad(const float *model, const float *X, const float *y, int32_t n, float *grad,
                                   float *loss) {
    if (!model || !X || !y || !grad || !loss || n < 1) return IPM_ERR_ARG;
    DevBuf dm, dX, dy, dg, dl;
    if (!dm.alloc(IPM_MLP_FLOATS * 4) || !dX.alloc((size_t)n * F * 4) || !dy.alloc((size_t)n * 4) ||
        !dg.alloc(NPARAM * 4) || !dl.alloc(4))
        return IPM_ERR_NOMEM;
    cudaError_t e;
    if ((e = cudaMemcpy(dm.p, model, IPM_MLP_FLOATS * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(dX.p, X, (size_t)n * F * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(dy.p, y, (size_t)n * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    cudaMemset(dg.p, 0, NPARAM * 4);
    cudaMemset(dl.p, 0, 4);
    k_mlp_grad<<<(n + 127) / 128, 128>>>(dm.f(), dX.f(), dy.f(), n, dg.f(), dl.f());
    if ((e = cudaGetLastError()) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(grad, dg.p, NPARAM * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(loss, dl.p, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return st_of(e);
    return IPM_OK;
}

extern "C" ipm_status ipm_mlp_train(const float *X, const float *y, int32_t n, int32_t epochs, float lr,
                                    uint64_t seed, float *model, float *final_loss) {
    if (!X || !y || !model || n < 2 || epochs < 0) return IPM_ERR_ARG;
    std::vector<float> m(IPM_MLP_FLOATS, 0.f);
    // standardisation of features and targets
    for (int k = 0; k < F; ++k) {
        double s = 0, s2 = 0;
        for (int i = 0; i < n; ++i) s += X[(size_t)i * F + k];
        const double mean = s / n;
        for (int i = 0; i < n; ++i) s2 += (X[(size_t)i * F + k] - mean) * (X[(size_t)i * F + k] - mean);
        const double sd = std::sqrt(s2 / n);
        m[k] = (float)mean;
        m[F + k] = sd > 1e-6 ? (float)(1.0 / sd) : 0.f;
    }
    double s = 0, s2 = 0;
    for (int i = 0; i < n; ++i) s += y[i];
    const double ym = s / n;
    for (int i = 0; i < n; ++i) s2 += (y[i] - ym) * (y[i] - ym);
    m[2 * F] = (float)ym;
    m[2 * F + 1] = (float)std::max(std::sqrt(s2 / n), 1e-6);
    // Glorot-uniform weights, zero biases
    uint64_t st = seed;
    auto uni = [&](float a) { return a * (2.0f * (float)((splitmix64(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0f); };
    float *p = m.data() + HEAD;
    const float a1 = std::sqrt(6.0f / (F + H)), a2 = std::sqrt(6.0f / (2 * H)), a3 = std::sqrt(6.0f / (H + 1));
    for (int i = 0; i < H * F; ++i) p[i] = uni(a1);
    for (int i = 0; i < H * H; ++i) p[H * F + H + i] = uni(a2);
    for (int i = 0; i < H; ++i) p[H * F + H + H * H + H + i] = uni(a3);
    DevBuf dm, dX, dy, dg, dl, dmom, dvel;
    if (!dm.alloc(IPM_MLP_FLOATS * 4) || !dX.alloc((size_t)n * F * 4) || !dy.alloc((size_t)n * 4) ||
        !dg.alloc(NPARAM * 4) || !dl.alloc(4) || !dmom.alloc(NPARAM * 4) || !dvel.alloc(NPARAM * 4))
        return IPM_ERR_NOMEM;
    cudaError_t e;
    if ((e = cudaMemcpy(dm.p, m.data(), IPM_MLP_FLOATS * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(dX.p, X, (size_t)n * F * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(dy.p, y, (size_t)n * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    cudaMemset(dmom.p, 0, NPARAM * 4);
    cudaMemset(dvel.p, 0, NPARAM * 4);
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f, c2 = 1.f;
    for (int ep = 0; ep < epochs; ++ep) {
        cudaMemsetAsync(dg.p, 0, NPARAM * 4);
        cudaMemsetAsync(dl.p, 0, 4);
        k_mlp_grad<<<(n + 127) / 128, 128>>>(dm.f(), dX.f(), dy.f(), n, dg.f(), dl.f());
        c1 *= b1;
        c2 *= b2;
        k_mlp_adam<<<(NPARAM + 255) / 256, 256>>>(dm.f() + HEAD, dg.f(), dmom.f(), dvel.f(), 1.0f / n, lr, b1, b2,
                                                  1.f - c1, 1.f - c2);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(model, dm.p, IPM_MLP_FLOATS * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return st_of(e);
    if (final_loss) {
        float l = 0;
        cudaMemset(dg.p, 0, NPARAM * 4);
        cudaMemset(dl.p, 0, 4);
        k_mlp_grad<<<(n + 127) / 128, 128>>>(dm.f(), dX.f(), dy.f(), n, dg.f(), dl.f());
        if ((e = cudaMemcpy(&l, dl.p, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return st_of(e);
        *final_loss = l / n;
    }
    return IPM_OK;
}

extern "C" ipm_status ipm_mlp_predict(const float *model, const float *X, int32_t n, float *out) {
    if (!model || !X || !out || n < 0) return IPM_ERR_ARG;
    if (n == 0) return IPM_OK;
    DevBuf dm, dX, dout;
    if (!dm.alloc(IPM_MLP_FLOATS * 4) || !dX.alloc((size_t)n * F * 4) || !dout.alloc((size_t)n * 4))
        return IPM_ERR_NOMEM;
    cudaError_t e;
    if ((e = cudaMemcpy(dm.p, model, IPM_MLP_FLOATS * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(dX.p, X, (size_t)n * F * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return st_of(e);
    k_mlp_predict<<<(n + 127) / 128, 128>>>(dm.f(), dX.f(), n, dout.f());
    if ((e = cudaGetLastError()) != cudaSuccess) return st_of(e);
    if ((e = cudaMemcpy(out, dout.p, (size_t)n * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return st_of(e);
    return IPM_OK;
}

extern "C" ipm_status ipm_set_cost_model(const float *model, int32_t nfloats) {
    std::lock_guard<std::mutex> g(g_model_lock);
    if (!model) {
        g_model.clear();
        return IPM_OK;
    }
    if (nfloats != IPM_MLP_FLOATS) return IPM_ERR_ARG;
    g_model.assign(model, model + nfloats);
    return IPM_OK;
}

namespace {

std::mutex g_tuned_lock;
std::map<std::tuple<int64_t, int64_t, uint32_t, uint32_t>, ipm_params> g_tuned;  // ipm_set_tuned

std::tuple<int64_t, int64_t, uint32_t, uint32_t> key_of(const ipm_shape &s) {
    return std::make_tuple(s.deg_a, s.deg_b, s.bits_a, s.bits_b);
}

}  // namespace

extern "C" ipm_status ipm_set_tuned(const ipm_shape *shapes, const ipm_params *params, int32_t n) {
    if (n < 0 || (n > 0 && (!shapes || !params))) return IPM_ERR_ARG;
    std::map<std::tuple<int64_t, int64_t, uint32_t, uint32_t>, ipm_params> t;
    for (int32_t i = 0; i < n; ++i) {
        ipm::ShapePlan sp;
        const ipm_status st = ipm::choose_plan(shapes[i], &params[i], sp);
        if (st != IPM_OK) return st;
        t[key_of(shapes[i])] = params[i];
    }
    std::lock_guard<std::mutex> g(g_tuned_lock);
    g_tuned.swap(t);
    return IPM_OK;
}

namespace ipm {

// Dispatch for n shapes: the measured best of the tuning table where the
// shape is in it, else the candidate with the smallest predicted time under
// the installed model (all shapes' candidates in one prediction launch),
// else the analytic planner.  src[i]: 0 planner, 1 table, 2 model.
ipm_status dispatch_params(const ipm_shape *shapes, int32_t n, ipm_params *out, int32_t *src) {
    std::vector<float> model;
    {
        std::lock_guard<std::mutex> g(g_model_lock);
        model = g_model;
    }
    std::vector<int32_t> first((size_t)n + 1, 0);
    std::vector<ipm_candidate> cand;
    {
        std::lock_guard<std::mutex> g(g_tuned_lock);
        for (int32_t i = 0; i < n; ++i) {
            out[i] = ipm_params{};
            src[i] = 0;
            first[(size_t)i] = (int32_t)cand.size();
            auto it = g_tuned.find(key_of(shapes[i]));
            if (it != g_tuned.end()) {
                out[i] = it->second;
                src[i] = 1;
                continue;
            }
            if (model.empty()) continue;
            const int32_t m = ipm_candidates(&shapes[i], nullptr, 0);
            if (m <= 0) continue;  // the planner reports the shape's error
            const size_t at = cand.size();
            cand.resize(at + (size_t)m);
            ipm_candidates(&shapes[i], cand.data() + at, m);
            const float batch = (float)std::log2((double)std::min<int32_t>(n, 16));
            for (size_t j = at; j < cand.size(); ++j) cand[j].features[F - 1] = batch;
        }
        first[(size_t)n] = (int32_t)cand.size();
    }
    if (cand.empty()) return IPM_OK;
    const int32_t total = (int32_t)cand.size();
    std::vector<float> X((size_t)total * F), pred((size_t)total);
    for (int32_t j = 0; j < total; ++j) std::memcpy(&X[(size_t)j * F], cand[(size_t)j].features, F * sizeof(float));
    const ipm_status st = ipm_mlp_predict(model.data(), X.data(), total, pred.data());
    if (st != IPM_OK) return st;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t b = first[(size_t)i], e = first[(size_t)i + 1];
        if (src[i] == 1 || b == e) continue;
        int32_t best = b;
        for (int32_t j = b + 1; j < e; ++j)
            if (pred[(size_t)j] < pred[(size_t)best]) best = j;
        out[i] = cand[(size_t)best].params;
        src[i] = 2;
    }
    return IPM_OK;
}

}  // namespace ipm

extern "C" ipm_status ipm_dispatch(const ipm_shape *shape, ipm_params *out, int32_t *source) {
    if (!shape || !out) return IPM_ERR_ARG;
    int32_t src = 0;
    const ipm_status st = ipm::dispatch_params(shape, 1, out, &src);
    if (source) *source = src;
    return st;
}
