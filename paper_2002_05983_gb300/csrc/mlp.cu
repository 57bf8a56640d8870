// Cost model of the schedule tuner: a small multilayer perceptron
// (features -> H -> H -> 1, ReLU) trained on measured schedule timings, with
// hand-written CUDA kernels for the forward pass, the backward pass of the
// mean-squared error and the Adam update.  Everything is FP32; the problem
// is tiny (a few thousand rows, H = 64), so each kernel is a plain
// one-thread-per-output loop.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "stencil.h"

struct stencil_model {
    int nf = 0, h = 0;
    // parameters, flat on the device: W1[nf*h] b1[h] W2[h*h] b2[h] w3[h] b3[1]
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int np = 0;
    int step = 0;
    // activations / scratch for the current batch
    float *x = nullptr, *y = nullptr, *a1 = nullptr, *a2 = nullptr, *out = nullptr;
    float *d1 = nullptr, *d2 = nullptr, *d3 = nullptr, *loss = nullptr;
    int cap = 0;
    float fmean[STENCIL_NFEAT] = {}, fstd[STENCIL_NFEAT] = {};
    float ymean = 0.f, ystd = 1.f;
    bool normed = false;
};

namespace {

thread_local int g_mlp_err = 0;

int fail(cudaError_t e)
{
    g_mlp_err = static_cast<int>(e);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? STENCIL_ERR_OOM : STENCIL_ERR_CUDA;
}
#define MK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return fail(e_);   \
    } while (0)

// Z[n][o] = act(sum_i A[n][i] W[i][o] + b[o])
__global__ void dense_fwd(const float *A, const float *W, const float *b, float *Z, int n, int in,
                          int out, int relu)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * out) return;
    const int r = idx / out, o = idx % out;
    float acc = b[o];
    for (int i = 0; i < in; ++i) acc = fmaf(A[r * in + i], W[i * out + o], acc);
    Z[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// d3[n] = 2 (out - y) / n and the loss sum((out - y)^2) / n
__global__ void mse_grad(const float *out, const float *y, float *d3, float *loss, int n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float e = out[r] - y[r];
    d3[r] = 2.f * e / n;
    atomicAdd(loss, e * e / n);
}

// gW[i][o] = sum_r A[r][i] D[r][o];  gb[o] = sum_r D[r][o]  (gb may be null)
__global__ void weight_grad(const float *A, const float *D, float *gW, float *gb, int n, int in, int out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < in * out) {
        const int i = idx / out, o = idx % out;
        float acc = 0.f;
        for (int r = 0; r < n; ++r) acc = fmaf(A[r * in + i], D[r * out + o], acc);
        gW[idx] = acc;
    } else if (gb && idx < in * out + out) {
        const int o = idx - in * out;
        float acc = 0.f;
        for (int r = 0; r < n; ++r) acc += D[r * out + o];
        gb[o] = acc;
    }
}

// Dprev[r][i] = (sum_o D[r][o] W[i][o]) * (Aprev[r][i] > 0)
__global__ void back_prop(const float *D, const float *W, const float *Aprev, float *Dprev, int n, int in,
                          int out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * in) return;
    const int r = idx / in, i = idx % in;
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc = fmaf(D[r * out + o], W[i * out + o], acc);
    Dprev[idx] = Aprev[idx] > 0.f ? acc : 0.f;
}

__global__ void adam(float *p, const float *g, float *m, float *v, int np, float lr, float b1, float b2,
                     float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

unsigned cdiv(long a, int b) { return static_cast<unsigned>((a + b - 1) / b); }

int ensure_batch(stencil_model *md, int n)
{
    if (n <= md->cap) return 0;
    float **bufs[] = {&md->x, &md->y, &md->a1, &md->a2, &md->out, &md->d1, &md->d2, &md->d3};
    for (float **b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    const size_t nf = md->nf, h = md->h;
    MK(cudaMalloc(&md->x, n * nf * sizeof(float)));
    MK(cudaMalloc(&md->y, n * sizeof(float)));
    MK(cudaMalloc(&md->a1, n * h * sizeof(float)));
    MK(cudaMalloc(&md->a2, n * h * sizeof(float)));
    MK(cudaMalloc(&md->out, n * sizeof(float)));
    MK(cudaMalloc(&md->d1, n * h * sizeof(float)));
    MK(cudaMalloc(&md->d2, n * h * sizeof(float)));
    MK(cudaMalloc(&md->d3, n * sizeof(float)));
    md->cap = n;
    return 0;
}

// parameter offsets
struct Off {
    int W1, b1, W2, b2, w3, b3, n;
};
Off offsets(int nf, int h)
{
    Off o;
    o.W1 = 0;
    o.b1 = o.W1 + nf * h;
    o.W2 = o.b1 + h;
    o.b2 = o.W2 + h * h;
    o.w3 = o.b2 + h;
    o.b3 = o.w3 + h;
    o.n = o.b3 + 1;
    return o;
}

void forward(stencil_model *md, int n, cudaStream_t st)
{
    const Off o = offsets(md->nf, md->h);
    const int h = md->h;
    dense_fwd<<<cdiv(long(n) * h, 256), 256, 0, st>>>(md->x, md->p + o.W1, md->p + o.b1, md->a1, n, md->nf, h, 1);
    dense_fwd<<<cdiv(long(n) * h, 256), 256, 0, st>>>(md->a1, md->p + o.W2, md->p + o.b2, md->a2, n, h, h, 1);
    dense_fwd<<<cdiv(n, 256), 256, 0, st>>>(md->a2, md->p + o.w3, md->p + o.b3, md->out, n, h, 1, 0);
}

void backward(stencil_model *md, int n, cudaStream_t st)
{
    const Off o = offsets(md->nf, md->h);
    const int h = md->h, nf = md->nf;
    cudaMemsetAsync(md->loss, 0, sizeof(float), st);
    mse_grad<<<cdiv(n, 256), 256, 0, st>>>(md->out, md->y, md->d3, md->loss, n);
    weight_grad<<<cdiv(h + 1, 256), 256, 0, st>>>(md->a2, md->d3, md->g + o.w3, md->g + o.b3, n, h, 1);
    back_prop<<<cdiv(long(n) * h, 256), 256, 0, st>>>(md->d3, md->p + o.w3, md->a2, md->d2, n, h, 1);
    weight_grad<<<cdiv(h * h + h, 256), 256, 0, st>>>(md->a1, md->d2, md->g + o.W2, md->g + o.b2, n, h, h);
    back_prop<<<cdiv(long(n) * h, 256), 256, 0, st>>>(md->d2, md->p + o.W2, md->a1, md->d1, n, h, h);
    weight_grad<<<cdiv(nf * h + h, 256), 256, 0, st>>>(md->x, md->d1, md->g + o.W1, md->g + o.b1, n, nf, h);
}

// normalised copy of features / targets to the device
int upload(stencil_model *md, const float *X, const float *y, int n, cudaStream_t st)
{
    std::vector<float> xs(static_cast<size_t>(n) * md->nf);
    for (int r = 0; r < n; ++r)
        for (int f = 0; f < md->nf; ++f)
            xs[static_cast<size_t>(r) * md->nf + f] = (X[static_cast<size_t>(r) * md->nf + f] - md->fmean[f]) / md->fstd[f];
    MK(cudaMemcpyAsync(md->x, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    if (y) {
        std::vector<float> ys(n);
        for (int r = 0; r < n; ++r) ys[r] = (y[r] - md->ymean) / md->ystd;
        MK(cudaMemcpyAsync(md->y, ys.data(), ys.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    }
    MK(cudaStreamSynchronize(st));
    return 0;
}

}  // namespace

extern "C" {

int stencil_model_create(stencil_model_handle *out, int n_features, int hidden, int seed)
{
    if (!out || n_features < 1 || n_features > STENCIL_NFEAT || hidden < 1 || hidden > 256)
        return STENCIL_ERR_INVALID_ARG;
    *out = nullptr;
    stencil_model *md = new (std::nothrow) stencil_model;
    if (!md) return STENCIL_ERR_OOM;
    md->nf = n_features;
    md->h = hidden;
    const Off o = offsets(n_features, hidden);
    md->np = o.n;
    for (int f = 0; f < STENCIL_NFEAT; ++f) md->fstd[f] = 1.f;
    // He initialisation from a fixed-seed LCG (reproducible, host side)
    std::vector<float> p(o.n, 0.f);
    uint64_t s = 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(seed);
    auto unif = [&]() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return static_cast<float>((s >> 40) * (1.0 / 16777216.0));
    };
    auto fill = [&](int off, int count, int fan_in) {
        const float a = std::sqrt(6.f / fan_in);
        for (int i = 0; i < count; ++i) p[off + i] = (2.f * unif() - 1.f) * a;
    };
    fill(o.W1, n_features * hidden, n_features);
    fill(o.W2, hidden * hidden, hidden);
    fill(o.w3, hidden, hidden);
    int rc = 0;
    auto alloc = [&](float **d) {
        if (cudaMalloc(d, o.n * sizeof(float)) != cudaSuccess) return false;
        return cudaMemset(*d, 0, o.n * sizeof(float)) == cudaSuccess;
    };
    if (!alloc(&md->p) || !alloc(&md->g) || !alloc(&md->m) || !alloc(&md->v) ||
        cudaMalloc(&md->loss, sizeof(float)) != cudaSuccess ||
        cudaMemcpy(md->p, p.data(), o.n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = STENCIL_ERR_OOM;
    if (rc) {
        stencil_model_destroy(md);
        return rc;
    }
    *out = md;
    return STENCIL_OK;
}

int stencil_model_destroy(stencil_model_handle md)
{
    if (!md) return STENCIL_OK;
    float *bufs[] = {md->p, md->g, md->m, md->v, md->x, md->y, md->a1, md->a2, md->out, md->d1, md->d2, md->d3, md->loss};
    for (float *b : bufs)
        if (b) cudaFree(b);
    delete md;
    return STENCIL_OK;
}

int stencil_model_params(stencil_model_handle md, float *host, int count, int set)
{
    if (!md || !host) return STENCIL_ERR_INVALID_ARG;
    if (count != md->np) return md->np;
    if (set) {
        MK(cudaMemcpy(md->p, host, count * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        MK(cudaMemcpy(host, md->p, count * sizeof(float), cudaMemcpyDeviceToHost));
    }
    return STENCIL_OK;
}

int stencil_model_normalization(stencil_model_handle md, const float *fmean, const float *fstd, float ymean,
                                float ystd)
{
    if (!md || !fmean || !fstd || !(ystd > 0.f)) return STENCIL_ERR_INVALID_ARG;
    for (int f = 0; f < md->nf; ++f) {
        if (!(fstd[f] > 0.f)) return STENCIL_ERR_INVALID_ARG;
        md->fmean[f] = fmean[f];
        md->fstd[f] = fstd[f];
    }
    md->ymean = ymean;
    md->ystd = ystd;
    md->normed = true;
    return STENCIL_OK;
}

int stencil_model_grad(stencil_model_handle md, const float *X, const float *y, int n, float *loss, float *grad)
{
    if (!md || !X || !y || n < 1) return STENCIL_ERR_INVALID_ARG;
    int rc = ensure_batch(md, n);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    rc = upload(md, X, y, n, st);
    if (rc) return rc;
    forward(md, n, st);
    backward(md, n, st);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(st));
    if (loss) MK(cudaMemcpy(loss, md->loss, sizeof(float), cudaMemcpyDeviceToHost));
    if (grad) MK(cudaMemcpy(grad, md->g, md->np * sizeof(float), cudaMemcpyDeviceToHost));
    return STENCIL_OK;
}

int stencil_model_train(stencil_model_handle md, const float *X, const float *y, int n, int epochs, float lr,
                        float *final_loss)
{
    if (!md || !X || !y || n < 2 || epochs < 1 || !(lr > 0.f)) return STENCIL_ERR_INVALID_ARG;
    if (!md->normed) {
        // standardise features and targets on this training set
        for (int f = 0; f < md->nf; ++f) {
            double s = 0, s2 = 0;
            for (int r = 0; r < n; ++r) {
                const double v = X[static_cast<size_t>(r) * md->nf + f];
                s += v;
                s2 += v * v;
            }
            const double mu = s / n, var = s2 / n - mu * mu;
            md->fmean[f] = static_cast<float>(mu);
            md->fstd[f] = var > 1e-12 ? static_cast<float>(std::sqrt(var)) : 1.f;
        }
        double s = 0, s2 = 0;
        for (int r = 0; r < n; ++r) {
            s += y[r];
            s2 += static_cast<double>(y[r]) * y[r];
        }
        const double mu = s / n, var = s2 / n - mu * mu;
        md->ymean = static_cast<float>(mu);
        md->ystd = var > 1e-12 ? static_cast<float>(std::sqrt(var)) : 1.f;
        md->normed = true;
    }
    int rc = ensure_batch(md, n);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    rc = upload(md, X, y, n, st);
    if (rc) return rc;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int e = 0; e < epochs; ++e) {
        forward(md, n, st);
        backward(md, n, st);
        ++md->step;
        const float c1 = 1.f - std::pow(b1, static_cast<float>(md->step));
        const float c2 = 1.f - std::pow(b2, static_cast<float>(md->step));
        adam<<<cdiv(md->np, 256), 256, 0, st>>>(md->p, md->g, md->m, md->v, md->np, lr, b1, b2, 1e-8f, c1, c2);
    }
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(st));
    if (final_loss) {
        forward(md, n, st);
        backward(md, n, st);
        MK(cudaStreamSynchronize(st));
        MK(cudaMemcpy(final_loss, md->loss, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return STENCIL_OK;
}

int stencil_model_predict(stencil_model_handle md, const float *X, float *y, int n)
{
    if (!md || !X || !y || n < 1) return STENCIL_ERR_INVALID_ARG;
    int rc = ensure_batch(md, n);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    rc = upload(md, X, nullptr, n, st);
    if (rc) return rc;
    forward(md, n, st);
    MK(cudaGetLastError());
    MK(cudaStreamSynchronize(st));
    MK(cudaMemcpy(y, md->out, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (int r = 0; r < n; ++r) y[r] = y[r] * md->ystd + md->ymean;
    return STENCIL_OK;
}

}  // extern "C"
