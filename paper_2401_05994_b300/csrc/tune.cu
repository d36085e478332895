// Autotuner of the row kernels' launch shapes (mgard_autotune).
//
// For every level of a shape and every row kernel (coefficients, fill,
// restriction along x, restriction along y/z, quantization,
// dequantization) the tuner times each launch shape -- 2, 4, 8 or 16 elements
// per lane per batch, grids sized for 4, 8 or 16 resident blocks per SM, and
// for the coefficient and fill kernels rows staged in shared memory or not --
// on workspace buffers holding a decomposed synthetic field, and keeps the
// fastest in the shape's plan.  Launch shapes change only how rows are
// spread over warps, never the arithmetic, so every choice gives the same
// bits.  The paper has no tuner; its GPU kernels fix their tile shapes.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pipeline.cuh"
#include "quantize.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

// A smooth field plus a hashed perturbation (values only steer the
// quantizer's escape rate; timing is what matters here).
template <typename T>
__global__ void k_tune_fill(T* u, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const double noise = ((double)(h & 0xFFFF) / 65536.0 - 0.5) * 1e-2;
        u[i] = (T)(sin(1e-3 * (double)i) + noise);
    }
}

const int U_CAND[] = {2, 4, 8, 16};
const int B_CAND[] = {4, 8, 16};
const char* KIND_NAME[RK_COUNT] = {"coeff", "fill", "restrict_x", "restrict_rows", "quantize",
                                   "dequantize"};

template <typename T>
mgard_status tune_impl(const Plan& p, cudaStream_t st, std::string& rep) {
    const int64_t N = p.total();
    const int L = p.L;
    Pyramid<T> py;
    MGB_TRY(py.alloc(p, st));
    DevBuf in, top, sym, esc, hist, stat, wdev;
    MGB_TRY(in.alloc(N * sizeof(T), st));
    MGB_TRY(top.alloc(N * sizeof(T), st));
    MGB_TRY(sym.alloc(N * sizeof(uint16_t), st));
    MGB_TRY(esc.alloc(N * sizeof(int32_t), st));
    MGB_TRY(hist.alloc(DICT * sizeof(unsigned long long), st));
    MGB_TRY(stat.alloc(sizeof(unsigned), st));
    MGB_TRY(wdev.alloc((L + 1) * sizeof(double), st));
    MGB_LAUNCH("k_tune_fill", st, k_tune_fill<T><<<grid_for(N, 256, 148LL * 16), 256, 0, st>>>(in.as<T>(), N));
    MGB_CUDA(cudaGetLastError());
    MGB_TRY(decompose_pyramid<T>(p, in.as<T>(), top.as<T>(), py, st, nullptr));
    std::vector<double> w(L + 1);
    bin_widths(p, 1e-3, INFINITY, w.data());
    MGB_CUDA(cudaMemcpyAsync(wdev.p, w.data(), (L + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    MGB_CUDA(cudaMemsetAsync(hist.p, 0, DICT * sizeof(unsigned long long), st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(unsigned), st));
    cudaEvent_t e0, e1;
    MGB_CUDA(cudaEventCreate(&e0));
    MGB_CUDA(cudaEventCreate(&e1));
    auto run = [&](int l, int kind) -> mgard_status {
        T* lvl = l == L ? top.as<T>() : py.lv[l];
        switch (kind) {
            case RK_COEFF:   // the coefficients go to `top` (large enough for any level)
                return rows3_coeff<T>(p, l, l == L ? in.as<T>() : py.lv[l], top.as<T>(),
                                      py.lv[l - 1], st);
            case RK_FILL: return rows3_fill<T>(p, l, lvl, py.lv[l - 1], lvl, st);
            case RK_RX:
            case RK_RROWS:
                return correct_coarse<T>(p, l, lvl, py.lv[l - 1], py.temp0.p, py.temp1.p, T(0), st);
            case RK_QUANT:
                return rows3_quantize<T>(p, l, lvl, wdev.as<double>() + l, sym.as<uint16_t>(),
                                         esc.as<int32_t>(), hist.as<unsigned long long>(),
                                         stat.as<unsigned>(), st);
            default:
                return rows3_dequantize<T>(p, l, sym.as<uint16_t>(), esc.as<int32_t>(), w[l], lvl, st);
        }
    };
    mgard_status err = MGARD_OK;
    for (int l = L; l >= 0 && err == MGARD_OK; --l) {
        for (int kind = 0; kind < RK_COUNT && err == MGARD_OK; ++kind) {
            if (l == 0 && kind != RK_QUANT && kind != RK_DEQUANT) continue;
            RowCfg& slot = p.tune[l][kind];
            const RowCfg keep = slot;
            float best = 1e30f, base = 0.f;
            RowCfg pick = keep;
            const int nstage = (kind == RK_COEFF || kind == RK_FILL) ? 2 : 1;
            for (int ui = -1; ui < 4 && err == MGARD_OK; ++ui) {
                for (int bs = 0; bs < 3 * nstage && err == MGARD_OK; ++bs) {
                    const int bi = bs % 3;
                    if (ui < 0 && bs > 0) break;   // ui = -1: the built-in choice
                    RowCfg c;
                    c.u = ui < 0 ? 0 : U_CAND[ui];
                    c.bpsm = ui < 0 ? 0 : B_CAND[bi];
                    c.stage = (ui < 0 || nstage == 1) ? -1 : 1 - bs / 3;
                    slot = c;
                    if ((err = run(l, kind)) != MGARD_OK) break;   // warm-up
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < 3 && err == MGARD_OK; ++r) err = run(l, kind);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) err = MGARD_ECUDA;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= 3.f;
                    if (ui < 0) base = ms;
                    if (ms < best) {
                        best = ms;
                        pick = c;
                    }
                }
            }
            slot = err == MGARD_OK ? pick : keep;
            char line[160];
            std::snprintf(line, sizeof(line),
                          "level %d %-13s u=%d blocks/SM=%d stage=%d %.4f ms (built-in %.4f ms)\n",
                          l, KIND_NAME[kind], pick.u, pick.bpsm, pick.stage, best, base);
            rep += line;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MGB_CUDA(cudaStreamSynchronize(st));
    return err;
}

std::mutex g_tune_mu;

}  // namespace

mgard_status autotune_plan(const Plan& p, mgard_dtype dtype, cudaStream_t st, std::string* report) {
    std::string rep;
    if (!rows3_ok(p) || p.L == 0) {
        if (report) *report = "nothing to tune: the shape runs on the generic kernels\n";
        return MGARD_OK;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const mgard_status e = dtype == MGARD_F64 ? tune_impl<double>(p, st, rep)
                                              : tune_impl<float>(p, st, rep);
    if (report) *report = rep;
    return e;
}

}  // namespace mgb

using namespace mgb;

extern "C" mgard_status mgard_autotune(int ndim, const int64_t* shape, mgard_dtype dtype,
                                       char* report, size_t report_cap, void* stream) {
    if (dtype != MGARD_F32 && dtype != MGARD_F64) {
        set_error("dtype must be MGARD_F32 or MGARD_F64");
        return MGARD_EDTYPE;
    }
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, -1, &p));
    std::string rep;
    MGB_TRY(autotune_plan(*p, dtype, (cudaStream_t)stream, &rep));
    if (report && report_cap) {
        const size_t k = rep.size() < report_cap - 1 ? rep.size() : report_cap - 1;
        std::memcpy(report, rep.data(), k);
        report[k] = 0;
    }
    return MGARD_OK;
}
