// Multilayer perceptron of the tolerance predictor: initialization,
// input standardization, forward pass, mean-squared-error backpropagation
// and Adam, as hand-written kernels (float32).
//
// Network: x [NFEAT] -> xn = (x - mu) / max(sd, 0.05) ->
// h1 = relu(W1 xn + b1) [H] -> h2 = relu(W2 h1 + b2) [H] -> y = w3 . h2 + b3,
// relu'(0) = 0.  Parameters (float): W1 [H, IN] row-major, b1, W2 [H, H], b2,
// w3, b3 (trainable), then mu [IN], sd [IN].  Loss (1/B) sum_b (y_b - t_b)^2.
// The paper has no predictor; this network serves ratio-targeted
// compression (mgard_compress_to_ratio), where the bin-width bound itself
// is never changed.
#include <cmath>

#include "multilevel.cuh"
#include "predictor.cuh"

namespace mgb {

namespace {

constexpr int IN = MGARD_NFEAT;
constexpr int H = MGARD_MLP_HIDDEN;
constexpr int O_W1 = 0;
constexpr int O_B1 = O_W1 + H * IN;
constexpr int O_W2 = O_B1 + H;
constexpr int O_B2 = O_W2 + H * H;
constexpr int O_W3 = O_B2 + H;
constexpr int O_B3 = O_W3 + H;
constexpr int O_MU = O_B3 + 1;
constexpr int O_SD = O_MU + IN;
static_assert(O_MU == MGARD_MLP_NTRAIN, "trainable parameter count");
static_assert(O_SD + IN == MGARD_MLP_NPARAM, "parameter count");

// splitmix64 (Steele, Lea and Flood 2014): a counter-based generator
__device__ inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// He-uniform weights U(-sqrt(6 / fan_in), sqrt(6 / fan_in)), zero biases,
// mu = 0, sd = 1.
__global__ void k_mlp_init(float* p, uint64_t seed) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MGARD_MLP_NPARAM;
         k += gridDim.x * blockDim.x) {
        const double u = (double)(splitmix64(seed * 0x100000001B3ull + (uint64_t)k) >> 11) *
                         (1.0 / 9007199254740992.0);   // [0, 1)
        float v = 0.f;
        if (k < O_B1) v = (float)((2.0 * u - 1.0) * sqrt(6.0 / IN));
        else if (k >= O_W2 && k < O_B2) v = (float)((2.0 * u - 1.0) * sqrt(6.0 / H));
        else if (k >= O_W3 && k < O_B3) v = (float)((2.0 * u - 1.0) * sqrt(6.0 / H));
        else if (k >= O_SD) v = 1.f;
        p[k] = v;
    }
}

// mu, sd: per-input mean and population standard deviation over the batch
// (double accumulation, fixed order).
__global__ void k_mlp_norm(float* p, const float* __restrict__ x, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= IN) return;
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < B; ++b) {
        const double v = x[(size_t)b * IN + i];
        s += v;
        s2 += v * v;
    }
    const double m = s / B;
    p[O_MU + i] = (float)m;
    p[O_SD + i] = (float)sqrt(fmax(s2 / B - m * m, 0.0));
}

// One block of H threads per sample: forward pass, and with `t` the
// backward pass down to the per-sample deltas.
struct Acts {
    float* xn;   // [B, IN]
    float* h1;   // [B, H]
    float* h2;   // [B, H]
    float* d1;   // [B, H]   dL/dz1
    float* d2;   // [B, H]   dL/dz2
    float* dy;   // [B]
    float* e2;   // [B]      squared error
};

__global__ void __launch_bounds__(H) k_mlp_sample(const float* __restrict__ p,
                                                  const float* __restrict__ x,
                                                  const float* __restrict__ t, int B,
                                                  float* __restrict__ y, Acts a) {
    __shared__ float xn[IN];
    __shared__ float h1s[H], d2s[H];
    __shared__ float red[H / 32];
    const int b = blockIdx.x, j = threadIdx.x, lane = j & 31, warp = j >> 5;
    if (b >= B) return;
    for (int i = j; i < IN; i += H) {
        // the floor keeps inputs that barely vary in training from turning
        // small differences into large standardized values
        const float sd = fmaxf(p[O_SD + i], 0.05f);
        xn[i] = (x[(size_t)b * IN + i] - p[O_MU + i]) / sd;
    }
    __syncthreads();
    float z1 = p[O_B1 + j];
    for (int i = 0; i < IN; ++i) z1 += p[O_W1 + j * IN + i] * xn[i];
    const float h1 = fmaxf(z1, 0.f);
    h1s[j] = h1;
    __syncthreads();
    float z2 = p[O_B2 + j];
    for (int k = 0; k < H; ++k) z2 += p[O_W2 + j * H + k] * h1s[k];
    const float h2 = fmaxf(z2, 0.f);
    float c = p[O_W3 + j] * h2;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) red[warp] = c;
    __syncthreads();
    float yv = p[O_B3];
    for (int w = 0; w < H / 32; ++w) yv += red[w];
    if (j == 0 && y) y[b] = yv;
    if (!t) return;
    const float e = yv - t[b];
    const float dy = 2.f * e / (float)B;
    const float d2 = z2 > 0.f ? dy * p[O_W3 + j] : 0.f;
    d2s[j] = d2;
    __syncthreads();
    float g = 0.f;
    for (int k = 0; k < H; ++k) g += d2s[k] * p[O_W2 + k * H + j];
    const float d1 = z1 > 0.f ? g : 0.f;
    for (int i = j; i < IN; i += H) a.xn[(size_t)b * IN + i] = xn[i];
    a.h1[(size_t)b * H + j] = h1;
    a.h2[(size_t)b * H + j] = h2;
    a.d1[(size_t)b * H + j] = d1;
    a.d2[(size_t)b * H + j] = d2;
    if (j == 0) {
        a.dy[b] = dy;
        a.e2[b] = e * e;
    }
}

// Gradient of every trainable parameter: one thread per entry, sum over
// the batch in sample order.  Thread MGARD_MLP_NTRAIN writes the loss.
__global__ void k_mlp_wgrad(Acts a, int B, float* __restrict__ g, float* __restrict__ loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > MGARD_MLP_NTRAIN) return;
    float s = 0.f;
    if (k < O_B1) {
        const int j = k / IN, i = k - j * IN;
        for (int b = 0; b < B; ++b) s += a.d1[(size_t)b * H + j] * a.xn[(size_t)b * IN + i];
    } else if (k < O_W2) {
        const int j = k - O_B1;
        for (int b = 0; b < B; ++b) s += a.d1[(size_t)b * H + j];
    } else if (k < O_B2) {
        const int j = (k - O_W2) / H, i = (k - O_W2) - j * H;
        for (int b = 0; b < B; ++b) s += a.d2[(size_t)b * H + j] * a.h1[(size_t)b * H + i];
    } else if (k < O_W3) {
        const int j = k - O_B2;
        for (int b = 0; b < B; ++b) s += a.d2[(size_t)b * H + j];
    } else if (k < O_B3) {
        const int j = k - O_W3;
        for (int b = 0; b < B; ++b) s += a.dy[b] * a.h2[(size_t)b * H + j];
    } else if (k == O_B3) {
        for (int b = 0; b < B; ++b) s += a.dy[b];
    } else {   // the loss
        double l = 0.0;
        for (int b = 0; b < B; ++b) l += a.e2[b];
        if (loss) *loss = (float)(l / B);
        return;
    }
    g[k] = s;
}

// Adam with bias correction on the first n entries.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

struct ActBufs {
    DevBuf buf;
    Acts a;
    mgard_status alloc(int B, cudaStream_t st) {
        const size_t f = (size_t)B * IN + 4 * (size_t)B * H + 2 * (size_t)B;
        MGB_TRY(buf.alloc(f * sizeof(float), st));
        float* q = buf.as<float>();
        a.xn = q;
        a.h1 = a.xn + (size_t)B * IN;
        a.h2 = a.h1 + (size_t)B * H;
        a.d1 = a.h2 + (size_t)B * H;
        a.d2 = a.d1 + (size_t)B * H;
        a.dy = a.d2 + (size_t)B * H;
        a.e2 = a.dy + B;
        return MGARD_OK;
    }
};

}  // namespace

mgard_status mlp_forward(const float* params, const float* x, int B, float* y, cudaStream_t st) {
    if (B <= 0) return MGARD_OK;
    MGB_LAUNCH("k_mlp_sample", st, k_mlp_sample<<<B, H, 0, st>>>(params, x, nullptr, B, y, Acts{}));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

}  // namespace mgb

using namespace mgb;

extern "C" {

mgard_status mgard_mlp_init(float* params, uint64_t seed, void* stream) {
    if (!params) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    MGB_LAUNCH("k_mlp_init", st, k_mlp_init<<<grid_for(MGARD_MLP_NPARAM, 256), 256, 0, st>>>(params, seed));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status mgard_mlp_set_norm(float* params, const float* x, int B, void* stream) {
    if (!params || !x || B <= 0) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    MGB_LAUNCH("k_mlp_norm", st, k_mlp_norm<<<(IN + 127) / 128, 128, 0, st>>>(params, x, B));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status mgard_mlp_forward(const float* params, const float* x, int B, float* y, void* stream) {
    if (!params || (B > 0 && (!x || !y)) || B < 0) return MGARD_EINVAL;
    return mlp_forward(params, x, B, y, (cudaStream_t)stream);
}

mgard_status mgard_mlp_loss_grad(const float* params, const float* x, const float* t, int B,
                                 float* grad, float* loss, void* stream) {
    if (!params || !x || !t || !grad || B <= 0) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ActBufs ab;
    MGB_TRY(ab.alloc(B, st));
    MGB_LAUNCH("k_mlp_sample", st, k_mlp_sample<<<B, H, 0, st>>>(params, x, t, B, nullptr, ab.a));
    MGB_LAUNCH("k_mlp_wgrad", st, k_mlp_wgrad<<<(MGARD_MLP_NTRAIN + 1 + 255) / 256, 256, 0, st>>>(ab.a, B, grad, loss));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status mgard_adam_step(float* params, const float* grad, float* m, float* v, int n,
                             float lr, float beta1, float beta2, float eps, int t, void* stream) {
    if (!params || !grad || !m || !v || n < 0 || t < 1) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const float c1 = (float)(1.0 - std::pow((double)beta1, t));
    const float c2 = (float)(1.0 - std::pow((double)beta2, t));
    MGB_LAUNCH("k_adam", st, k_adam<<<grid_for(n, 256), 256, 0, st>>>(params, grad, m, v, n, lr, beta1, beta2, eps, c1, c2));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status mgard_mlp_train(float* params, float* m, float* v, const float* x, const float* t,
                             int B, int steps, int t0, float lr, float* losses, void* stream) {
    if (!params || !m || !v || !x || !t || B <= 0 || steps < 0 || t0 < 0) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    ActBufs ab;
    MGB_TRY(ab.alloc(B, st));
    DevBuf g;
    MGB_TRY(g.alloc(MGARD_MLP_NTRAIN * sizeof(float), st));
    for (int k = 0; k < steps; ++k) {
        MGB_LAUNCH("k_mlp_sample", st, k_mlp_sample<<<B, H, 0, st>>>(params, x, t, B, nullptr, ab.a));
        MGB_LAUNCH("k_mlp_wgrad", st, k_mlp_wgrad<<<(MGARD_MLP_NTRAIN + 1 + 255) / 256, 256, 0, st>>>(
                                          ab.a, B, g.as<float>(), losses ? losses + k : nullptr));
        MGB_TRY(mgard_adam_step(params, g.as<float>(), m, v, MGARD_MLP_NTRAIN, lr, 0.9f, 0.999f,
                                1e-8f, t0 + k + 1, stream));
    }
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

}  // extern "C"
