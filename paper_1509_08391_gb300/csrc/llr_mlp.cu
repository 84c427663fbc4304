// llr_mlp.cu -- the learned warm start of the Robbins-Monro iteration: a
// 3 -> 64 -> 64 -> 64 -> 1 GELU multilayer perceptron mapping
// (1/V, E/6V, dE/6V), V = L^4, to the slope a, with hand-written FP32
// forward, backward and Adam kernels.  1/V is the volume feature because the
// finite-volume corrections of a_k are O(1/V) (appendix, eq. (A.12)).
//
// The paper's a_k are intrinsic quantities (Sec. 2.2, eq. (2.5); appendix,
// eqs. (A.11)-(A.13)), so a map learned on small volumes can predict the
// slopes of larger ones, and Sec. 2.4 only asks the initial a to be close.
//
// Layout: one float array of parameters, W1 (3x64, row-major [in][out]),
// b1 (64), W2 (64x64), b2, W3 (64x64), b3, W4 (64x1), b4 (1).  Activations
// are [sample][feature].  Layers are small, so each kernel is a plain
// thread-per-output dot product (no tensor cores: a 64-wide layer is not a
// contraction worth them), and the sums over samples are done in a fixed
// order (no atomics), so training is deterministic.  One training epoch
// (features are fixed) is ~13 launches; the host captures it once in a CUDA
// graph and replays it.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/llr.h"
#include "llr_internal.h"

namespace {

constexpr int kW = 64;      // hidden width
constexpr int kIn = 3;      // features
constexpr int kNParams = kIn * kW + kW + 2 * (kW * kW + kW) + kW + 1;   // 8641
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kW, kOffW2 = kOffB1 + kW,
              kOffB2 = kOffW2 + kW * kW, kOffW3 = kOffB2 + kW, kOffB3 = kOffW3 + kW * kW,
              kOffW4 = kOffB3 + kW, kOffB4 = kOffW4 + kW;

__device__ __forceinline__ float gelu(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Raw features (1/V, E/6V, dE/6V) standardised with mean / std.
__global__ void features_kernel(int n, const double *L, const double *e, const double *d,
                                const double *mean, const double *std, float *X)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const double L2 = L[s] * L[s];
        const double r[3] = {1.0 / (L2 * L2), e[s], d[s]};
        for (int k = 0; k < 3; ++k) X[s * 3 + k] = (float)((r[k] - mean[k]) / std[k]);
    }
}

// Mean and population standard deviation of the raw features (one CTA).
__global__ void feature_stats_kernel(int n, const double *L, const double *e, const double *d,
                                     double *mean, double *std)
{
    __shared__ double red[3][256];
    const int t = threadIdx.x;
    double s1[3] = {0, 0, 0};
    for (int s = t; s < n; s += 256) {
        const double L2 = L[s] * L[s];
        s1[0] += 1.0 / (L2 * L2);
        s1[1] += e[s];
        s1[2] += d[s];
    }
    for (int k = 0; k < 3; ++k) red[k][t] = s1[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < 3; ++k) red[k][t] += red[k][t + o];
        __syncthreads();
    }
    double m[3];
    for (int k = 0; k < 3; ++k) m[k] = red[k][0] / n;
    __syncthreads();
    double s2[3] = {0, 0, 0};
    for (int s = t; s < n; s += 256) {
        const double L2 = L[s] * L[s];
        const double r[3] = {1.0 / (L2 * L2), e[s], d[s]};
        for (int k = 0; k < 3; ++k) s2[k] += (r[k] - m[k]) * (r[k] - m[k]);
    }
    for (int k = 0; k < 3; ++k) red[k][t] = s2[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < 3; ++k) red[k][t] += red[k][t + o];
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 3; ++k) {
            mean[k] = m[k];
            const double sd = sqrt(red[k][0] / n);
            std[k] = sd > 0.0 ? sd : 1.0;
        }
}

// Z[s][j] = b[j] + sum_i H[s][i] W[i][j];  A = gelu(Z) (or Z for the output).
__global__ void linear_fwd_kernel(int n, int in_dim, int out_dim, const float *H, const float *W,
                                  const float *b, float *Z, float *A, int act)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * out_dim) return;
    const int s = idx / out_dim, j = idx - s * out_dim;
    float z = b[j];
    for (int i = 0; i < in_dim; ++i) z = fmaf(H[s * in_dim + i], W[i * out_dim + j], z);
    Z[idx] = z;
    A[idx] = act ? gelu(z) : z;
}

// dY = 2 (y - t) / n and the loss mean (y - t)^2 (one CTA reduces the loss).
__global__ void loss_grad_kernel(int n, const float *Y, const double *T, float *dY, double *loss)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int s = threadIdx.x; s < n; s += 256) {
        const double r = (double)Y[s] - T[s];
        dY[s] = (float)(2.0 * r / n);
        acc += r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = red[0] / n;
}

// dZin[s][i] = (sum_j dZ[s][j] W[i][j]) * gelu'(Zin[s][i]).
__global__ void linear_bwd_data_kernel(int n, int in_dim, int out_dim, const float *dZ,
                                       const float *W, const float *Zin, float *dZin)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * in_dim) return;
    const int s = idx / in_dim, i = idx - s * in_dim;
    float g = 0.0f;
    for (int j = 0; j < out_dim; ++j) g = fmaf(dZ[s * out_dim + j], W[i * out_dim + j], g);
    dZin[idx] = g * gelu_grad(Zin[idx]);
}

// gW[i][j] = sum_s H[s][i] dZ[s][j]; gb[j] = sum_s dZ[s][j] (thread per output,
// samples summed in order).
__global__ void linear_bwd_weight_kernel(int n, int in_dim, int out_dim, const float *H,
                                         const float *dZ, float *gW, float *gb)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = in_dim * out_dim;
    if (idx < nw) {
        const int i = idx / out_dim, j = idx - i * out_dim;
        float g = 0.0f;
        for (int s = 0; s < n; ++s) g = fmaf(H[s * in_dim + i], dZ[s * out_dim + j], g);
        gW[idx] = g;
    } else if (idx < nw + out_dim) {
        const int j = idx - nw;
        float g = 0.0f;
        for (int s = 0; s < n; ++s) g += dZ[s * out_dim + j];
        gb[j] = g;
    }
}

// Adam (Kingma & Ba 2015) with bias correction; step count in *t.
__global__ void adam_kernel(int np, float *P, const float *G, float *M, float *V,
                            const int *t, float lr, float b1, float b2, float eps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float c1 = 1.0f - powf(b1, (float)*t);
    const float c2 = 1.0f - powf(b2, (float)*t);
    const float g = G[k];
    const float m = b1 * M[k] + (1.0f - b1) * g;
    const float v = b2 * V[k] + (1.0f - b2) * g * g;
    M[k] = m;
    V[k] = v;
    P[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void step_count_kernel(int *t)
{
    *t += 1;
}

__global__ void to_double_kernel(int n, const float *a, double *b)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) b[k] = (double)a[k];
}

// Initial weights: normal(0, 1/sqrt(fan_in)) from Philox (Box-Muller), zero biases.
__global__ void init_params_kernel(float *P, uint32_t k0, uint32_t k1)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNParams) return;
    int fan = 0;
    if (k < kOffB1) fan = kIn;
    else if (k >= kOffW2 && k < kOffB2) fan = kW;
    else if (k >= kOffW3 && k < kOffB3) fan = kW;
    else if (k >= kOffW4 && k < kOffB4) fan = kW;
    if (fan == 0) {
        P[k] = 0.0f;
        return;
    }
    const llr::U4 w = llr::philox4x32_10((uint32_t)k, 0u, 0x4D4Cu, 0u, k0, k1);
    const float u1 = llr::u01(w.x), u2 = llr::u01(w.y);
    const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    P[k] = z / sqrtf((float)fan);
}

struct Buffers {
    int n = 0;
    float *X = nullptr, *Z = nullptr, *A = nullptr, *dZ = nullptr, *Y = nullptr, *dY = nullptr;
    double *T = nullptr, *raw = nullptr, *loss = nullptr;
};

}  // namespace

struct llr_mlp {
    cudaStream_t stream = nullptr;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    int *t = nullptr;
    double *norm = nullptr;   // mean[3], std[3]
    Buffers buf;
    cudaGraphExec_t graph = nullptr;
    int graph_n = -1;
    float graph_lr = 0.0f;
};

namespace {

int fail(int code, const std::string &msg)
{
    return llr::set_last_error(code, msg.c_str());
}

#define MLP_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(LLR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

unsigned blocks(long long n, int t = 256)
{
    return (unsigned)((n + t - 1) / t);
}

int ensure_buffers(llr_mlp *h, int n)
{
    if (h->buf.n >= n) return LLR_OK;
    Buffers &b = h->buf;
    cudaFree(b.X); cudaFree(b.Z); cudaFree(b.A); cudaFree(b.dZ); cudaFree(b.Y); cudaFree(b.dY);
    cudaFree(b.T); cudaFree(b.raw); cudaFree(b.loss);
    b = Buffers();
    MLP_CUDA(cudaMalloc(&b.X, sizeof(float) * 3 * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.Z, sizeof(float) * 3 * kW * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.A, sizeof(float) * 3 * kW * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.dZ, sizeof(float) * 3 * kW * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.Y, sizeof(float) * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.dY, sizeof(float) * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.T, sizeof(double) * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.raw, sizeof(double) * 4 * (size_t)n));
    MLP_CUDA(cudaMalloc(&b.loss, sizeof(double)));
    b.n = n;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_n = -1;
    }
    return LLR_OK;
}

int upload_inputs(llr_mlp *h, int n, const double *L, const double *e, const double *d)
{
    double *r = h->buf.raw;
    MLP_CUDA(cudaMemcpyAsync(r, L, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    MLP_CUDA(cudaMemcpyAsync(r + n, e, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    MLP_CUDA(cudaMemcpyAsync(r + 2 * n, d, sizeof(double) * n, cudaMemcpyHostToDevice,
                             h->stream));
    return LLR_OK;
}

void enqueue_features(llr_mlp *h, int n)
{
    const double *r = h->buf.raw;
    features_kernel<<<blocks(n), 256, 0, h->stream>>>(n, r, r + n, r + 2 * n, h->norm,
                                                      h->norm + 3, h->buf.X);
}

// Forward pass on the standardised features in buf.X; output in buf.Y.
void enqueue_forward(llr_mlp *h, int n)
{
    Buffers &b = h->buf;
    const size_t L1 = 0, L2 = (size_t)kW * n, L3 = 2 * (size_t)kW * n;
    linear_fwd_kernel<<<blocks((long long)n * kW), 256, 0, h->stream>>>(
        n, kIn, kW, b.X, h->P + kOffW1, h->P + kOffB1, b.Z + L1, b.A + L1, 1);
    linear_fwd_kernel<<<blocks((long long)n * kW), 256, 0, h->stream>>>(
        n, kW, kW, b.A + L1, h->P + kOffW2, h->P + kOffB2, b.Z + L2, b.A + L2, 1);
    linear_fwd_kernel<<<blocks((long long)n * kW), 256, 0, h->stream>>>(
        n, kW, kW, b.A + L2, h->P + kOffW3, h->P + kOffB3, b.Z + L3, b.A + L3, 1);
    linear_fwd_kernel<<<blocks(n), 256, 0, h->stream>>>(n, kW, 1, b.A + L3, h->P + kOffW4,
                                                       h->P + kOffB4, b.dY, b.Y, 0);
}

// Loss, gradients into h->G (forward must have run).
void enqueue_backward(llr_mlp *h, int n)
{
    Buffers &b = h->buf;
    const size_t L1 = 0, L2 = (size_t)kW * n, L3 = 2 * (size_t)kW * n;
    loss_grad_kernel<<<1, 256, 0, h->stream>>>(n, b.Y, b.T, b.dY, b.loss);
    linear_bwd_weight_kernel<<<blocks(kW + 1), 256, 0, h->stream>>>(
        n, kW, 1, b.A + L3, b.dY, h->G + kOffW4, h->G + kOffB4);
    linear_bwd_data_kernel<<<blocks((long long)n * kW), 256, 0, h->stream>>>(
        n, kW, 1, b.dY, h->P + kOffW4, b.Z + L3, b.dZ + L3);
    linear_bwd_weight_kernel<<<blocks(kW * kW + kW), 256, 0, h->stream>>>(
        n, kW, kW, b.A + L2, b.dZ + L3, h->G + kOffW3, h->G + kOffB3);
    linear_bwd_data_kernel<<<blocks((long long)n * kW), 256, 0, h->stream>>>(
        n, kW, kW, b.dZ + L3, h->P + kOffW3, b.Z + L2, b.dZ + L2);
    linear_bwd_weight_kernel<<<blocks(kW * kW + kW), 256, 0, h->stream>>>(
        n, kW, kW, b.A + L1, b.dZ + L2, h->G + kOffW2, h->G + kOffB2);
    linear_bwd_data_kernel<<<blocks((long long)n * kW), 256, 0, h->stream>>>(
        n, kW, kW, b.dZ + L2, h->P + kOffW2, b.Z + L1, b.dZ + L1);
    linear_bwd_weight_kernel<<<blocks(kIn * kW + kW), 256, 0, h->stream>>>(
        n, kIn, kW, b.X, b.dZ + L1, h->G + kOffW1, h->G + kOffB1);
}

void enqueue_epoch(llr_mlp *h, int n, float lr)
{
    enqueue_forward(h, n);
    enqueue_backward(h, n);
    step_count_kernel<<<1, 1, 0, h->stream>>>(h->t);
    adam_kernel<<<blocks(kNParams), 256, 0, h->stream>>>(kNParams, h->P, h->G, h->M, h->V, h->t,
                                                         lr, 0.9f, 0.999f, 1e-8f);
}

}  // namespace

extern "C" {

int llr_mlp_create(llr_mlp_handle *out, uint64_t seed, void *cuda_stream)
{
    if (!out) return fail(LLR_ERR_ARG, "null handle pointer");
    *out = nullptr;
    llr_mlp *h = new llr_mlp();
    h->stream = (cudaStream_t)cuda_stream;
    *out = h;
    MLP_CUDA(cudaMalloc(&h->P, sizeof(float) * kNParams));
    MLP_CUDA(cudaMalloc(&h->G, sizeof(float) * kNParams));
    MLP_CUDA(cudaMalloc(&h->M, sizeof(float) * kNParams));
    MLP_CUDA(cudaMalloc(&h->V, sizeof(float) * kNParams));
    MLP_CUDA(cudaMalloc(&h->t, sizeof(int)));
    MLP_CUDA(cudaMalloc(&h->norm, sizeof(double) * 6));
    MLP_CUDA(cudaMemsetAsync(h->G, 0, sizeof(float) * kNParams, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->M, 0, sizeof(float) * kNParams, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->V, 0, sizeof(float) * kNParams, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->t, 0, sizeof(int), h->stream));
    const double init_norm[6] = {0, 0, 0, 1, 1, 1};
    MLP_CUDA(cudaMemcpy(h->norm, init_norm, sizeof(init_norm), cudaMemcpyHostToDevice));
    init_params_kernel<<<blocks(kNParams), 256, 0, h->stream>>>(h->P, (uint32_t)seed,
                                                                (uint32_t)(seed >> 32));
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_mlp_num_params(void)
{
    return kNParams;
}

int llr_mlp_get_params(llr_mlp_handle h, float *out)
{
    if (!h || !out) return fail(LLR_ERR_ARG, "null argument");
    MLP_CUDA(cudaMemcpyAsync(out, h->P, sizeof(float) * kNParams, cudaMemcpyDeviceToHost,
                             h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_mlp_set_params(llr_mlp_handle h, const float *in)
{
    if (!h || !in) return fail(LLR_ERR_ARG, "null argument");
    MLP_CUDA(cudaMemcpyAsync(h->P, in, sizeof(float) * kNParams, cudaMemcpyHostToDevice,
                             h->stream));
    MLP_CUDA(cudaMemsetAsync(h->M, 0, sizeof(float) * kNParams, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->V, 0, sizeof(float) * kNParams, h->stream));
    MLP_CUDA(cudaMemsetAsync(h->t, 0, sizeof(int), h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_mlp_set_norm(llr_mlp_handle h, const double *mean, const double *std)
{
    if (!h || !mean || !std) return fail(LLR_ERR_ARG, "null argument");
    for (int k = 0; k < 3; ++k)
        if (!(std[k] > 0.0) || !std::isfinite(mean[k]))
            return fail(LLR_ERR_ARG, "std must be positive and mean finite");
    const double v[6] = {mean[0], mean[1], mean[2], std[0], std[1], std[2]};
    MLP_CUDA(cudaMemcpyAsync(h->norm, v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_mlp_get_norm(llr_mlp_handle h, double *mean, double *std)
{
    if (!h || !mean || !std) return fail(LLR_ERR_ARG, "null argument");
    double v[6];
    MLP_CUDA(cudaMemcpyAsync(v, h->norm, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 3; ++k) {
        mean[k] = v[k];
        std[k] = v[3 + k];
    }
    return LLR_OK;
}

static int check_inputs(int n, const double *L, const double *e, const double *d)
{
    if (n < 1 || !L || !e || !d) return fail(LLR_ERR_ARG, "need n >= 1 and input arrays");
    for (int s = 0; s < n; ++s)
        if (!(L[s] > 0.0) || !std::isfinite(e[s]) || !std::isfinite(d[s]))
            return fail(LLR_ERR_ARG, "inputs must be finite with L > 0");
    return LLR_OK;
}

int llr_mlp_predict(llr_mlp_handle h, int n, const double *L, const double *e6v,
                    const double *dE6v, double *a_out)
{
    if (!h || !a_out) return fail(LLR_ERR_ARG, "null argument");
    if (int r = check_inputs(n, L, e6v, dE6v)) return r;
    if (int r = ensure_buffers(h, n)) return r;
    if (int r = upload_inputs(h, n, L, e6v, dE6v)) return r;
    enqueue_features(h, n);
    enqueue_forward(h, n);
    to_double_kernel<<<blocks(n), 256, 0, h->stream>>>(n, h->buf.Y, h->buf.T);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaMemcpyAsync(a_out, h->buf.T, sizeof(double) * n, cudaMemcpyDeviceToHost,
                             h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_mlp_grad(llr_mlp_handle h, int n, const double *L, const double *e6v,
                 const double *dE6v, const double *a_target, float *grad_out, double *loss_out)
{
    if (!h || !a_target || !grad_out) return fail(LLR_ERR_ARG, "null argument");
    if (int r = check_inputs(n, L, e6v, dE6v)) return r;
    if (int r = ensure_buffers(h, n)) return r;
    if (int r = upload_inputs(h, n, L, e6v, dE6v)) return r;
    MLP_CUDA(cudaMemcpyAsync(h->buf.T, a_target, sizeof(double) * n, cudaMemcpyHostToDevice,
                             h->stream));
    enqueue_features(h, n);
    enqueue_forward(h, n);
    enqueue_backward(h, n);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaMemcpyAsync(grad_out, h->G, sizeof(float) * kNParams, cudaMemcpyDeviceToHost,
                             h->stream));
    double loss = 0.0;
    MLP_CUDA(cudaMemcpyAsync(&loss, h->buf.loss, sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    if (loss_out) *loss_out = loss;
    return LLR_OK;
}

int llr_mlp_fit(llr_mlp_handle h, int n, const double *L, const double *e6v, const double *dE6v,
                const double *a_target, int epochs, double lr, int standardise,
                double *loss_out)
{
    if (!h || !a_target) return fail(LLR_ERR_ARG, "null argument");
    if (epochs < 0 || !(lr > 0.0)) return fail(LLR_ERR_ARG, "epochs >= 0 and lr > 0");
    if (int r = check_inputs(n, L, e6v, dE6v)) return r;
    if (int r = ensure_buffers(h, n)) return r;
    if (int r = upload_inputs(h, n, L, e6v, dE6v)) return r;
    MLP_CUDA(cudaMemcpyAsync(h->buf.T, a_target, sizeof(double) * n, cudaMemcpyHostToDevice,
                             h->stream));
    const double *r = h->buf.raw;
    if (standardise)
        feature_stats_kernel<<<1, 256, 0, h->stream>>>(n, r, r + n, r + 2 * n, h->norm,
                                                       h->norm + 3);
    enqueue_features(h, n);
    MLP_CUDA(cudaGetLastError());
    // one epoch captured once as a CUDA graph, replayed `epochs` times
    if (!h->graph || h->graph_n != n || h->graph_lr != (float)lr) {
        if (h->graph) cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        cudaStream_t cap = h->stream;
        bool own = false;
        if (!cap) {
            MLP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            own = true;
            MLP_CUDA(cudaDeviceSynchronize());
        }
        cudaStream_t keep = h->stream;
        h->stream = cap;
        cudaGraph_t g;
        MLP_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        enqueue_epoch(h, n, (float)lr);
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        h->stream = keep;
        if (own) cudaStreamDestroy(cap);
        MLP_CUDA(ce);
        ce = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        MLP_CUDA(ce);
        h->graph_n = n;
        h->graph_lr = (float)lr;
    }
    for (int ep = 0; ep < epochs; ++ep) MLP_CUDA(cudaGraphLaunch(h->graph, h->stream));
    // loss of the final parameters
    enqueue_forward(h, n);
    loss_grad_kernel<<<1, 256, 0, h->stream>>>(n, h->buf.Y, h->buf.T, h->buf.dY, h->buf.loss);
    MLP_CUDA(cudaGetLastError());
    double loss = 0.0;
    MLP_CUDA(cudaMemcpyAsync(&loss, h->buf.loss, sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    if (loss_out) *loss_out = loss;
    return LLR_OK;
}

int llr_mlp_destroy(llr_mlp_handle h)
{
    if (!h) return LLR_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->graph) cudaGraphExecDestroy(h->graph);
    Buffers &b = h->buf;
    cudaFree(b.X); cudaFree(b.Z); cudaFree(b.A); cudaFree(b.dZ); cudaFree(b.Y); cudaFree(b.dY);
    cudaFree(b.T); cudaFree(b.raw); cudaFree(b.loss);
    cudaFree(h->P); cudaFree(h->G); cudaFree(h->M); cudaFree(h->V); cudaFree(h->t);
    cudaFree(h->norm);
    delete h;
    return LLR_OK;
}

}  // extern "C"
