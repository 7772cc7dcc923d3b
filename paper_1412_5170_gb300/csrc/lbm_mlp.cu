// lbm_mlp.cu -- the learned warm start's network: a tanh multilayer
// perceptron (inputs T/Tc, tau, A, K, radius -> density profile samples)
// trained and evaluated by hand-written FP32 kernels (forward, backward,
// Adam).  Inputs and outputs are standardised inside the model with affine
// scalings set by the caller.  Parameters are flattened layer by layer as
// [W (out x in, row-major), b], hidden layers first, then the linear output.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"

namespace {

constexpr int TS = 16;   // GEMM tile

enum Epi : int { EPI_NONE = 0, EPI_BIAS_TANH = 1, EPI_BIAS = 2, EPI_TANH_BACK = 3 };

// C[m, n] = sum_k A(m, k) B(k, n), A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn],
// with an epilogue: + bias[n] then tanh; + bias[n]; or times (1 - P[m, n]^2)
// (backpropagation through tanh, P the layer output).  Fixed summation order.
template <int EPI>
__global__ void __launch_bounds__(TS * TS)
k_gemm(const float* __restrict__ A, int sam, int sak, const float* __restrict__ B, int sbk, int sbn,
       float* __restrict__ C, int M, int N, int K, const float* __restrict__ bias, const float* __restrict__ P)
{
    __shared__ float sa[TS][TS + 1], sb[TS][TS + 1];
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    const int m = blockIdx.y * TS + ty, n = blockIdx.x * TS + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TS) {
        const int ka = k0 + tx, kb = k0 + ty;
        const int am = blockIdx.y * TS + ty, bn = blockIdx.x * TS + tx;
        sa[ty][tx] = (am < M && ka < K) ? A[(size_t)am * sam + (size_t)ka * sak] : 0.f;
        sb[ty][tx] = (kb < K && bn < N) ? B[(size_t)kb * sbk + (size_t)bn * sbn] : 0.f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TS; ++kk) acc = fmaf(sa[ty][kk], sb[kk][tx], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        if (EPI == EPI_BIAS_TANH) acc = tanhf(acc + bias[n]);
        else if (EPI == EPI_BIAS) acc = acc + bias[n];
        else if (EPI == EPI_TANH_BACK) { const float p = P[(size_t)m * N + n]; acc *= (1.f - p * p); }
        C[(size_t)m * N + n] = acc;
    }
}

// (x - mean) / std per column.
__global__ void k_standardize(const float* __restrict__ X, float* __restrict__ Y, int n, int d,
                              const float* __restrict__ mean, const float* __restrict__ sd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * d) Y[i] = (X[i] - mean[i % d]) / sd[i % d];
}

__global__ void k_destandardize(float* __restrict__ Y, int n, int d, const float* __restrict__ mean,
                                const float* __restrict__ sd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n * d) Y[i] = Y[i] * sd[i % d] + mean[i % d];
}

// Output delta of the MSE loss in standardised units, d loss / d out =
// 2 (out - t) / (n m), t = (y - mean)/std, and per-row squared error sums.
__global__ void k_loss_delta(const float* __restrict__ out, const float* __restrict__ Y, float* __restrict__ delta,
                             float* __restrict__ row_loss, int n, int m, const float* __restrict__ mean,
                             const float* __restrict__ sd)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float s = 0.f;
    const float inv = 2.f / (float(n) * float(m));
    for (int j = 0; j < m; ++j) {
        const float t = (Y[(size_t)r * m + j] - mean[j]) / sd[j];
        const float d = out[(size_t)r * m + j] - t;
        delta[(size_t)r * m + j] = inv * d;
        s += d * d;
    }
    row_loss[r] = s;
}

// Column sums of delta (bias gradient), fixed order.
__global__ void k_colsum(const float* __restrict__ delta, float* __restrict__ g, int n, int m)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float s = 0.f;
    for (int r = 0; r < n; ++r) s += delta[(size_t)r * m + j];
    g[j] = s;
}

// Adam (Kingma & Ba) with bias correction.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

uint64_t splitmix(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct lbm_ws {
    std::vector<int> sizes;          // n_in, hidden..., n_out
    std::vector<size_t> woff, boff;  // parameter offsets per layer
    size_t np = 0;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    float *xm = nullptr, *xs = nullptr, *ym = nullptr, *ys = nullptr;   // device scalings
    long long t = 0;                 // Adam steps taken
    cudaStream_t stream = nullptr;
    // per-batch buffers
    int cap = 0;
    std::vector<float*> acts;        // [L+1] activations (acts[0] = standardised input)
    float *delta0 = nullptr, *delta1 = nullptr, *rowloss = nullptr, *X = nullptr, *Y = nullptr;
};

namespace {

int ok(cudaError_t e)
{
    if (e == cudaSuccess) return LBM_OK;
    std::fprintf(stderr, "liblbm (mlp): CUDA error %s\n", cudaGetErrorString(e));
    return LBM_E_CUDA;
}
#define W_CUDA(call)                  \
    do {                              \
        int s_ = ok(call);            \
        if (s_ != LBM_OK) return s_;  \
    } while (0)

int nlayers(const lbm_ws* w) { return (int)w->sizes.size() - 1; }
int widest(const lbm_ws* w)
{
    int m = 0;
    for (int s : w->sizes) m = s > m ? s : m;
    return m;
}

int ensure(lbm_ws* w, int n)
{
    if (n <= w->cap) return LBM_OK;
    for (float* p : w->acts) cudaFree(p);
    cudaFree(w->delta0);
    cudaFree(w->delta1);
    cudaFree(w->rowloss);
    cudaFree(w->X);
    cudaFree(w->Y);
    w->acts.assign(nlayers(w) + 1, nullptr);
    for (int l = 0; l <= nlayers(w); ++l) W_CUDA(cudaMalloc(&w->acts[l], sizeof(float) * n * w->sizes[l]));
    W_CUDA(cudaMalloc(&w->delta0, sizeof(float) * n * widest(w)));
    W_CUDA(cudaMalloc(&w->delta1, sizeof(float) * n * widest(w)));
    W_CUDA(cudaMalloc(&w->rowloss, sizeof(float) * n));
    W_CUDA(cudaMalloc(&w->X, sizeof(float) * n * w->sizes.front()));
    W_CUDA(cudaMalloc(&w->Y, sizeof(float) * n * w->sizes.back()));
    w->cap = n;
    return LBM_OK;
}

dim3 tiles(int M, int N) { return dim3((N + TS - 1) / TS, (M + TS - 1) / TS); }

// Forward pass of n rows already in w->X (raw inputs); output (standardised) in acts[L].
int forward(lbm_ws* w, int n)
{
    const int d = w->sizes.front();
    k_standardize<<<(n * d + 255) / 256, 256, 0, w->stream>>>(w->X, w->acts[0], n, d, w->xm, w->xs);
    const int L = nlayers(w);
    for (int l = 0; l < L; ++l) {
        const int in = w->sizes[l], out = w->sizes[l + 1];
        const float* Wl = w->params + w->woff[l];
        const float* bl = w->params + w->boff[l];
        if (l < L - 1)
            k_gemm<EPI_BIAS_TANH><<<tiles(n, out), TS * TS, 0, w->stream>>>(w->acts[l], in, 1, Wl, 1, in, w->acts[l + 1],
                                                                             n, out, in, bl, nullptr);
        else
            k_gemm<EPI_BIAS><<<tiles(n, out), TS * TS, 0, w->stream>>>(w->acts[l], in, 1, Wl, 1, in, w->acts[l + 1], n,
                                                                        out, in, bl, nullptr);
    }
    return ok(cudaGetLastError());
}

// Backward pass for n rows with targets in w->Y: gradient into w->grads, row losses into w->rowloss.
int backward(lbm_ws* w, int n)
{
    const int L = nlayers(w);
    const int m = w->sizes.back();
    k_loss_delta<<<(n + 127) / 128, 128, 0, w->stream>>>(w->acts[L], w->Y, w->delta0, w->rowloss, n, m, w->ym, w->ys);
    float* delta = w->delta0;
    float* other = w->delta1;
    for (int l = L - 1; l >= 0; --l) {
        const int in = w->sizes[l], out = w->sizes[l + 1];
        // gW[o, i] = sum_b delta[b, o] acts_l[b, i]
        k_gemm<EPI_NONE><<<tiles(out, in), TS * TS, 0, w->stream>>>(delta, 1, out, w->acts[l], in, 1,
                                                                    w->grads + w->woff[l], out, in, n, nullptr, nullptr);
        k_colsum<<<(out + 127) / 128, 128, 0, w->stream>>>(delta, w->grads + w->boff[l], n, out);
        if (l > 0) {
            // delta_prev[b, i] = (sum_o delta[b, o] W[o, i]) (1 - acts_l[b, i]^2)
            k_gemm<EPI_TANH_BACK><<<tiles(n, in), TS * TS, 0, w->stream>>>(delta, out, 1, w->params + w->woff[l], in, 1,
                                                                           other, n, in, out, nullptr, w->acts[l]);
            float* t = delta;
            delta = other;
            other = t;
        }
    }
    return ok(cudaGetLastError());
}

}  // namespace

extern "C" {

int lbm_ws_create(const lbm_ws_cfg* cfg, lbm_ws** out)
{
    if (!cfg || !out || cfg->n_in < 1 || cfg->n_out < 1 || cfg->n_hidden < 1 || cfg->hidden_layers < 1 ||
        cfg->hidden_layers > 16)
        return LBM_E_INVALID;
    *out = nullptr;
    lbm_ws* w = new (std::nothrow) lbm_ws();
    if (!w) return LBM_E_INVALID;
    w->sizes.push_back(cfg->n_in);
    for (int i = 0; i < cfg->hidden_layers; ++i) w->sizes.push_back(cfg->n_hidden);
    w->sizes.push_back(cfg->n_out);
    size_t p = 0;
    for (int l = 0; l < nlayers(w); ++l) {
        w->woff.push_back(p);
        p += (size_t)w->sizes[l + 1] * w->sizes[l];
        w->boff.push_back(p);
        p += w->sizes[l + 1];
    }
    w->np = p;
    // Glorot-uniform weights from SplitMix64(seed, index), zero biases.
    std::vector<float> h(p, 0.f);
    for (int l = 0; l < nlayers(w); ++l) {
        const double lim = std::sqrt(6.0 / (w->sizes[l] + w->sizes[l + 1]));
        for (size_t i = 0; i < (size_t)w->sizes[l + 1] * w->sizes[l]; ++i) {
            const double xi = double(splitmix(cfg->seed ^ (w->woff[l] + i)) >> 11) * (1.0 / 9007199254740992.0);
            h[w->woff[l] + i] = float(lim * (2.0 * xi - 1.0));
        }
    }
    std::vector<float> one_in(cfg->n_in, 1.f), zero_in(cfg->n_in, 0.f), one_out(cfg->n_out, 1.f),
        zero_out(cfg->n_out, 0.f);
    cudaError_t e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&w->params, sizeof(float) * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->grads, sizeof(float) * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->m1, sizeof(float) * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->m2, sizeof(float) * p);
    if (e == cudaSuccess) e = cudaMalloc(&w->xm, sizeof(float) * cfg->n_in);
    if (e == cudaSuccess) e = cudaMalloc(&w->xs, sizeof(float) * cfg->n_in);
    if (e == cudaSuccess) e = cudaMalloc(&w->ym, sizeof(float) * cfg->n_out);
    if (e == cudaSuccess) e = cudaMalloc(&w->ys, sizeof(float) * cfg->n_out);
    if (e == cudaSuccess) e = cudaMemcpy(w->params, h.data(), sizeof(float) * p, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(w->m1, 0, sizeof(float) * p);
    if (e == cudaSuccess) e = cudaMemset(w->m2, 0, sizeof(float) * p);
    if (e == cudaSuccess) e = cudaMemcpy(w->xm, zero_in.data(), sizeof(float) * cfg->n_in, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->xs, one_in.data(), sizeof(float) * cfg->n_in, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->ym, zero_out.data(), sizeof(float) * cfg->n_out, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w->ys, one_out.data(), sizeof(float) * cfg->n_out, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lbm_ws_destroy(w);
        return ok(e);
    }
    *out = w;
    return LBM_OK;
}

void lbm_ws_destroy(lbm_ws* w)
{
    if (!w) return;
    if (w->stream) cudaStreamSynchronize(w->stream);
    for (float* p : {w->params, w->grads, w->m1, w->m2, w->xm, w->xs, w->ym, w->ys, w->delta0, w->delta1,
                     w->rowloss, w->X, w->Y})
        cudaFree(p);
    for (float* p : w->acts) cudaFree(p);
    if (w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

int lbm_ws_num_params(lbm_ws* w, int64_t* n)
{
    if (!w || !n) return LBM_E_INVALID;
    *n = (int64_t)w->np;
    return LBM_OK;
}

int lbm_ws_set_scaling(lbm_ws* w, const float* x_mean, const float* x_std, const float* y_mean, const float* y_std)
{
    if (!w || !x_mean || !x_std || !y_mean || !y_std) return LBM_E_INVALID;
    const int d = w->sizes.front(), m = w->sizes.back();
    for (int i = 0; i < d; ++i)
        if (!(x_std[i] > 0)) return LBM_E_INVALID;
    for (int i = 0; i < m; ++i)
        if (!(y_std[i] > 0)) return LBM_E_INVALID;
    W_CUDA(cudaMemcpy(w->xm, x_mean, sizeof(float) * d, cudaMemcpyHostToDevice));
    W_CUDA(cudaMemcpy(w->xs, x_std, sizeof(float) * d, cudaMemcpyHostToDevice));
    W_CUDA(cudaMemcpy(w->ym, y_mean, sizeof(float) * m, cudaMemcpyHostToDevice));
    W_CUDA(cudaMemcpy(w->ys, y_std, sizeof(float) * m, cudaMemcpyHostToDevice));
    return LBM_OK;
}

int lbm_ws_get_params(lbm_ws* w, float* host)
{
    if (!w || !host) return LBM_E_INVALID;
    W_CUDA(cudaMemcpy(host, w->params, sizeof(float) * w->np, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int lbm_ws_set_params(lbm_ws* w, const float* host)
{
    if (!w || !host) return LBM_E_INVALID;
    W_CUDA(cudaMemcpy(w->params, host, sizeof(float) * w->np, cudaMemcpyHostToDevice));
    w->t = 0;
    W_CUDA(cudaMemset(w->m1, 0, sizeof(float) * w->np));
    W_CUDA(cudaMemset(w->m2, 0, sizeof(float) * w->np));
    return LBM_OK;
}

int lbm_ws_loss_grad(lbm_ws* w, const float* X_host, const float* Y_host, int n, float* loss, float* grad_host)
{
    if (!w || !X_host || !Y_host || n < 1) return LBM_E_INVALID;
    int s = ensure(w, n);
    if (s != LBM_OK) return s;
    W_CUDA(cudaMemcpyAsync(w->X, X_host, sizeof(float) * n * w->sizes.front(), cudaMemcpyHostToDevice, w->stream));
    W_CUDA(cudaMemcpyAsync(w->Y, Y_host, sizeof(float) * n * w->sizes.back(), cudaMemcpyHostToDevice, w->stream));
    if ((s = forward(w, n)) != LBM_OK) return s;
    if ((s = backward(w, n)) != LBM_OK) return s;
    std::vector<float> rl(n);
    W_CUDA(cudaMemcpyAsync(rl.data(), w->rowloss, sizeof(float) * n, cudaMemcpyDeviceToHost, w->stream));
    if (grad_host) W_CUDA(cudaMemcpyAsync(grad_host, w->grads, sizeof(float) * w->np, cudaMemcpyDeviceToHost, w->stream));
    W_CUDA(cudaStreamSynchronize(w->stream));
    double tot = 0;
    for (float v : rl) tot += v;
    if (loss) *loss = float(tot / (double(n) * w->sizes.back()));
    return LBM_OK;
}

int lbm_ws_train(lbm_ws* w, const float* X_host, const float* Y_host, int n, int epochs, int batch, float lr,
                 uint64_t seed, float* final_loss)
{
    if (!w || !X_host || !Y_host || n < 1 || epochs < 0 || batch < 1 || !(lr > 0)) return LBM_E_INVALID;
    const int d = w->sizes.front(), m = w->sizes.back();
    batch = batch > n ? n : batch;
    int s = ensure(w, batch);
    if (s != LBM_OK) return s;
    float *dX = nullptr, *dY = nullptr;
    W_CUDA(cudaMalloc(&dX, sizeof(float) * n * d));
    W_CUDA(cudaMalloc(&dY, sizeof(float) * n * m));
    std::vector<int> perm(n);
    std::vector<float> hx((size_t)n * d), hy((size_t)n * m);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs && s == LBM_OK; ++ep) {
        // deterministic per-epoch shuffle (Fisher-Yates on SplitMix64 draws)
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = n - 1; i > 0; --i) {
            const int j = int(splitmix(seed ^ ((uint64_t)ep << 32) ^ (uint64_t)i) % (uint64_t)(i + 1));
            const int t = perm[i];
            perm[i] = perm[j];
            perm[j] = t;
        }
        for (int i = 0; i < n; ++i) {
            std::memcpy(&hx[(size_t)i * d], X_host + (size_t)perm[i] * d, sizeof(float) * d);
            std::memcpy(&hy[(size_t)i * m], Y_host + (size_t)perm[i] * m, sizeof(float) * m);
        }
        if ((s = ok(cudaMemcpyAsync(dX, hx.data(), sizeof(float) * n * d, cudaMemcpyHostToDevice, w->stream))) != LBM_OK) break;
        if ((s = ok(cudaMemcpyAsync(dY, hy.data(), sizeof(float) * n * m, cudaMemcpyHostToDevice, w->stream))) != LBM_OK) break;
        for (int b0 = 0; b0 < n && s == LBM_OK; b0 += batch) {
            const int nb = (n - b0 < batch) ? n - b0 : batch;
            cudaMemcpyAsync(w->X, dX + (size_t)b0 * d, sizeof(float) * nb * d, cudaMemcpyDeviceToDevice, w->stream);
            cudaMemcpyAsync(w->Y, dY + (size_t)b0 * m, sizeof(float) * nb * m, cudaMemcpyDeviceToDevice, w->stream);
            if ((s = forward(w, nb)) != LBM_OK) break;
            if ((s = backward(w, nb)) != LBM_OK) break;
            ++w->t;
            const float c1 = 1.f - std::pow(b1, float(w->t)), c2 = 1.f - std::pow(b2, float(w->t));
            k_adam<<<(int(w->np) + 255) / 256, 256, 0, w->stream>>>(w->params, w->grads, w->m1, w->m2, int(w->np), lr,
                                                                   b1, b2, eps, c1, c2);
            s = ok(cudaGetLastError());
        }
        cudaStreamSynchronize(w->stream);   // hx/hy are refilled next epoch
    }
    if (s == LBM_OK && final_loss)   // loss over the whole training set with the final parameters
        s = lbm_ws_loss_grad(w, X_host, Y_host, n, final_loss, nullptr);
    cudaFree(dX);
    cudaFree(dY);
    return s;
}

int lbm_ws_predict(lbm_ws* w, const float* X_host, int n, float* Y_host)
{
    if (!w || !X_host || !Y_host || n < 1) return LBM_E_INVALID;
    int s = ensure(w, n);
    if (s != LBM_OK) return s;
    const int d = w->sizes.front(), m = w->sizes.back();
    W_CUDA(cudaMemcpyAsync(w->X, X_host, sizeof(float) * n * d, cudaMemcpyHostToDevice, w->stream));
    if ((s = forward(w, n)) != LBM_OK) return s;
    float* outp = w->acts[nlayers(w)];
    k_destandardize<<<(n * m + 255) / 256, 256, 0, w->stream>>>(outp, n, m, w->ym, w->ys);
    W_CUDA(cudaGetLastError());
    W_CUDA(cudaMemcpyAsync(Y_host, outp, sizeof(float) * n * m, cudaMemcpyDeviceToHost, w->stream));
    W_CUDA(cudaStreamSynchronize(w->stream));
    return LBM_OK;
}

}  // extern "C"
