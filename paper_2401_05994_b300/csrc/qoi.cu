// Error control of linear quantities of interest (paper: "Software design",
// guarantees on quantities derived from the data; "Application impact",
// plasma physics).
//
// A linear QoI Q(v) = sum_p g_p v_p has the representer r in V_L with
// M_L r = g, so Q(e) = <r, e>_{L2}.  Splitting both over the orthogonal
// level spaces (Q_l - Q_{l-1}) V_L and applying Cauchy-Schwarz gives
// |Q(e)| <= ||r||_{-s} ||e||_s, where ||r||_{-s} is the s-norm with -s.  A
// QoI tolerance tau_Q therefore becomes the s-norm tolerance
// tau_Q / ||Q||_{-s}; for s = infinity the dual norm is ||g||_1.
//
// Device work: the representer solve (one FP64 tridiagonal solve per line
// along every active axis, one thread per line), the level energies of r
// (the FP64 decomposition), and deterministic FP64 dot products.
#include <cmath>
#include <vector>

#include "../../include/mgard_b300.h"
#include "multilevel.cuh"

namespace mgb {

namespace {

constexpr int DOT_BLOCKS = 296;
constexpr int DOT_THREADS = 256;

bool on_device(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Forward-elimination factors of the 1D mass matrix of the unit-spacing grid
// with n nodes (diagonal 1/3 at the ends, 2/3 inside; off-diagonals 1/6):
// inv[i] = 1 / (b_i - a_i cp[i-1]), cp[i] = c_i inv[i].
void mass_factors(int64_t n, double* cp, double* inv) {
    double prev = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double b = (i == 0 || i == n - 1) ? 1.0 / 3.0 : 2.0 / 3.0;
        const double a = i == 0 ? 0.0 : 1.0 / 6.0;
        const double c = i == n - 1 ? 0.0 : 1.0 / 6.0;
        inv[i] = 1.0 / (b - a * prev);
        cp[i] = c * inv[i];
        prev = cp[i];
    }
}

// Thomas solve of M x = d along one axis of extent n whose consecutive nodes
// are S apart, in place, one thread per line (the lines of a strided axis
// are adjacent in memory, so a warp's accesses coalesce).
__global__ void k_mass_solve(double* __restrict__ x, int64_t lines, int64_t n, int64_t S,
                             const double* __restrict__ cp, const double* __restrict__ inv) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= lines) return;
    double* p = x + (t / S) * S * n + t % S;
    double prev = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double y = (p[i * S] - (1.0 / 6.0) * prev) * inv[i];
        p[i * S] = y;
        prev = y;
    }
    double next = 0.0;
    for (int64_t i = n - 1; i >= 0; --i) {
        const double v = p[i * S] - cp[i] * next;
        p[i * S] = v;
        next = v;
    }
}

// Partial sums of g_p u_p (u null: |g_p|), FP64, one per block in a fixed
// order; non-finite weights or values set ST_NONFINITE.
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) k_qoi_dot(const T* __restrict__ u,
                                                         const double* __restrict__ g, int64_t n,
                                                         double* __restrict__ part,
                                                         unsigned* status) {
    __shared__ double red[DOT_THREADS];
    double acc = 0.0;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double w = g[i];
        const double v = u ? (double)u[i] : 1.0;
        if (!isfinite(w) || !isfinite(v)) bad = true;
        acc += u ? w * v : fabs(w);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = DOT_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <typename T>
mgard_status qoi_dot(const T* u, const double* g, int64_t n, double* out, cudaStream_t st) {
    DevBuf part, stat;
    MGB_TRY(part.alloc(DOT_BLOCKS * sizeof(double), st));
    MGB_TRY(stat.alloc(sizeof(unsigned), st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(unsigned), st));
    MGB_LAUNCH("k_qoi_dot", st,
               k_qoi_dot<T><<<DOT_BLOCKS, DOT_THREADS, 0, st>>>(u, g, n, part.as<double>(),
                                                                stat.as<unsigned>()));
    MGB_CUDA(cudaGetLastError());
    double h[DOT_BLOCKS];
    unsigned hs = 0;
    MGB_CUDA(cudaMemcpyAsync(h, part.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaMemcpyAsync(&hs, stat.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    if (hs & ST_NONFINITE) {
        set_error("QoI weights or field hold NaN or Inf");
        return MGARD_ENONFINITE;
    }
    double s = 0.0;
    for (int i = 0; i < DOT_BLOCKS; ++i) s += h[i];
    *out = s;
    return MGARD_OK;
}

// r = M_L^{-1} r in place on the squeezed grid of plan p.
mgard_status representer_solve(const Plan& p, double* r, cudaStream_t st) {
    const int64_t N = p.total();
    for (int a = 4 - p.D; a < 4; ++a) {
        const int64_t n = p.n4[a];
        int64_t S = 1;
        for (int k = a + 1; k < 4; ++k) S *= p.n4[k];
        std::vector<double> h(2 * n);
        mass_factors(n, h.data(), h.data() + n);
        DevBuf f;
        MGB_TRY(f.alloc(2 * n * sizeof(double), st));
        MGB_CUDA(cudaMemcpyAsync(f.p, h.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice, st));
        const int64_t lines = N / n;
        const int threads = 128;
        MGB_LAUNCH("k_mass_solve", st,
                   k_mass_solve<<<(unsigned)((lines + threads - 1) / threads), threads, 0, st>>>(
                       r, lines, n, S, f.as<double>(), f.as<double>() + n));
        MGB_CUDA(cudaGetLastError());
        // the factors' buffer is released stream-ordered after the launch
    }
    return MGARD_OK;
}

mgard_status qoi_norm_impl(const Plan& p, const double* g, double s, double* out,
                           cudaStream_t st) {
    const int64_t N = p.total();
    double l1 = 0.0;
    MGB_TRY(qoi_dot<double>(nullptr, g, N, &l1, st));   // also rejects non-finite weights
    if (std::isinf(s)) {
        *out = l1;
        return MGARD_OK;
    }
    if (p.D == 0) {   // one node: the value itself
        *out = l1;
        return MGARD_OK;
    }
    DevBuf r;
    MGB_TRY(r.alloc(N * sizeof(double), st));
    MGB_CUDA(cudaMemcpyAsync(r.p, g, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MGB_TRY(representer_solve(p, r.as<double>(), st));
    Pyramid<double> py;
    MGB_TRY(py.alloc(p, st));
    std::vector<double> E(p.L + 1, 0.0);
    MGB_TRY(decompose_pyramid<double>(p, r.as<double>(), r.as<double>(), py, st, E.data()));
    // ||r||_{-s}^2 = E_0 + sum_l 4^{-s l} (E_l - E_{l-1}), increments clamped at 0
    double total = E[0];
    for (int l = 1; l <= p.L; ++l) total += std::pow(4.0, -s * (double)l) * std::max(E[l] - E[l - 1], 0.0);
    *out = std::sqrt(std::max(total, 0.0));
    return MGARD_OK;
}

mgard_status check_weights(const double* g, const char* what) {
    if (!g || !on_device(g)) {
        set_error(std::string(what) + ": weights must be device memory");
        return MGARD_EINVAL;
    }
    return MGARD_OK;
}

}  // namespace

}  // namespace mgb

using namespace mgb;

extern "C" mgard_status mgard_qoi_representer(const double* g, int ndim, const int64_t* shape,
                                              double* r, void* stream) {
    MGB_TRY(check_weights(g, "qoi_representer"));
    if (!r || !on_device(r)) {
        set_error("qoi_representer: r must be device memory");
        return MGARD_EINVAL;
    }
    const Plan* p = nullptr;
    MGB_TRY(get_plan(ndim, shape, -1, &p));
    cudaStream_t st = (cudaStream_t)stream;
    double l1 = 0.0;
    MGB_TRY(qoi_dot<double>(nullptr, g, p->total(), &l1, st));
    if (r != g)
        MGB_CUDA(cudaMemcpyAsync(r, g, p->total() * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return representer_solve(*p, r, st);
}

extern "C" mgard_status mgard_qoi_norm(const double* g, int ndim, const int64_t* shape,
                                       int max_levels, double s, double* norm, void* stream) {
    MGB_TRY(check_weights(g, "qoi_norm"));
    if (!norm || std::isnan(s) || s < 0.0) {
        set_error("qoi_norm: s must be >= 0 or INFINITY");
        return MGARD_EINVAL;
    }
    const Plan* p = nullptr;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    return qoi_norm_impl(*p, g, s, norm, (cudaStream_t)stream);
}

extern "C" mgard_status mgard_qoi_value(const void* field, const double* g, int ndim,
                                        const int64_t* shape, mgard_dtype dtype, double* value,
                                        void* stream) {
    MGB_TRY(check_weights(g, "qoi_value"));
    if (!field || !value || !on_device(field)) {
        set_error("qoi_value: field must be device memory");
        return MGARD_EINVAL;
    }
    if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_EDTYPE;
    const Plan* p = nullptr;
    MGB_TRY(get_plan(ndim, shape, -1, &p, false));
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MGARD_F32) return qoi_dot<float>((const float*)field, g, p->total(), value, st);
    return qoi_dot<double>((const double*)field, g, p->total(), value, st);
}

extern "C" mgard_status mgard_compress_qoi(const void* field, int ndim, const int64_t* shape,
                                           mgard_dtype dtype, const double* g, double tol_qoi,
                                           double s, void** out, size_t* out_bytes,
                                           int out_preallocated, double* tol_used, void* stream) {
    MGB_TRY(check_weights(g, "compress_qoi"));
    if (!(tol_qoi > 0.0) || !std::isfinite(tol_qoi) || std::isnan(s) || s < 0.0) {
        set_error("compress_qoi: tol_qoi must be positive and finite, s >= 0 or INFINITY");
        return MGARD_EINVAL;
    }
    double nq = 0.0;
    MGB_TRY(mgard_qoi_norm(g, ndim, shape, -1, s, &nq, stream));
    if (!(nq > 0.0)) {
        set_error("compress_qoi: the QoI is zero on every field");
        return MGARD_EINVAL;
    }
    const double tol = tol_qoi / nq;
    if (!std::isfinite(tol)) {
        set_error("compress_qoi: tolerance overflows");
        return MGARD_EINVAL;
    }
    if (tol_used) *tol_used = tol;
    return mgard_compress(field, ndim, shape, dtype, tol, s, MGARD_ABS, out, out_bytes,
                          out_preallocated, stream);
}
