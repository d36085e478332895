// C ABI (include/mgard_b300.h): argument checks, workspace, buffer-location
// detection and the self-describing format (include/mgard_format.h).
//
// Paper, "APIs": the high-level calls take the data, shape, dtype, tau, s
// and the bound type (Listing 1), detect where the buffers live and move
// data as needed; the low-level calls expose each step with device
// asynchrony.  Pipelines here:
//   compress:   [norm] -> decompose -> widths -> quantize+histogram ->
//               codebook -> count/scan -> pack -> header
//   decompress: header checks -> tables -> decode -> dequantize -> recompose
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/mgard_format.h"
#include "huffman.cuh"
#include "multilevel.cuh"
#include "pipeline.cuh"
#include "quantize.cuh"
#include "region.cuh"

namespace mgb {

namespace {
thread_local std::string g_last_error;

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}


mgard_status check_dtype(mgard_dtype d) {
    if (d != MGARD_F32 && d != MGARD_F64) {
        set_error("dtype must be MGARD_F32 or MGARD_F64");
        return MGARD_EDTYPE;
    }
    return MGARD_OK;
}


double s_norm_from_levels(const std::vector<double>& E, double s) {
    double total = E[0];
    for (size_t l = 1; l < E.size(); ++l) total += std::pow(4.0, s * (double)l) * std::max(E[l] - E[l - 1], 0.0);
    return std::sqrt(std::max(total, 0.0));
}

// ---------------------------------------------------------------------------
template <typename T>
mgard_status norm_impl(const Plan& p, const T* data, double s, double* out, cudaStream_t st) {
    const int64_t N = p.total();
    if (std::isinf(s)) {
        unsigned status = 0;
        MGB_TRY(max_abs<T>(data, nullptr, N, out, &status, st));
        return status_to_error(status);
    }
    unsigned status = 0;
    double dummy;
    MGB_TRY(max_abs<T>(data, nullptr, N, &dummy, &status, st));
    MGB_TRY(status_to_error(status));
    Pyramid<T> py;
    MGB_TRY(py.alloc(p, st));
    DevBuf top;
    MGB_TRY(top.alloc(N * sizeof(T), st));
    std::vector<double> E(p.L + 1, 0.0);
    MGB_TRY(decompose_pyramid<T>(p, data, top.as<T>(), py, st, E.data()));
    *out = s_norm_from_levels(E, s);
    return MGARD_OK;
}

// With `rh` the output is the region header (inner_bytes filled in here)
// followed by the buffer, whose coefficients are scaled by `rs`.
template <typename T>
mgard_status compress_impl(const Plan& p, const void* field, bool field_dev, mgard_dtype dtype,
                           int ndim, const int64_t* shape, double tol, double s,
                           mgard_tolmode mode, void** out, size_t* out_bytes, int prealloc,
                           cudaStream_t st, const RegionScale* rs = nullptr,
                           mgard_region_header* rh = nullptr) {
    const size_t pre = rh ? MGARD_REGION_INNER : 0;
    const int64_t N = p.total();
    const uint64_t nchunks = ((uint64_t)N + CHUNK - 1) / CHUNK;
    const Sections fx = layout(p.L, nchunks, 0, 0);
    if (prealloc && (!out || !*out || !out_bytes)) {
        set_error("preallocated output missing");
        return MGARD_EINVAL;
    }
    DevBuf inbuf;
    const T* din = (const T*)field;
    if (!field_dev) {
        MGB_TRY(inbuf.alloc(N * sizeof(T), st));
        MGB_CUDA(cudaMemcpyAsync(inbuf.p, field, N * sizeof(T), cudaMemcpyHostToDevice, st));
        din = inbuf.as<T>();
    }
    CompressWork<T> w;
    MGB_TRY(w.alloc(p, st));
    DevBuf metab, scratch;
    MGB_TRY(metab.alloc(sizeof(CompressMeta), st));
    // a 16-byte aligned device buffer of the caller is written in place;
    // anything else goes through a scratch buffer of the worst-case size
    const bool direct = prealloc && is_device_ptr(*out) && ((uintptr_t)*out & 15) == 0 &&
                        *out_bytes >= pre + fx.outliers;
    char* dd;
    uint64_t cap;
    if (direct) {
        dd = (char*)*out + pre;
        cap = *out_bytes - pre;
    } else {
        cap = layout(p.L, nchunks, (uint64_t)N, (uint64_t)N + nchunks).total;
        MGB_TRY(scratch.alloc(cap, st));
        dd = scratch.as<char>();
    }
    const mgard_header h0 = header_template(p, dtype, ndim, shape, tol, s, mode);
    MGB_TRY(compress_core<T>(p, din, h0, tol, s, mode, dd, cap, w, metab.as<CompressMeta>(), st, rs));
    CompressMeta m;
    MGB_CUDA(cudaMemcpyAsync(&m, metab.p, sizeof(m), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    MGB_TRY(status_to_error(m.status & ~(unsigned)ST_CAPACITY));
    if (m.status & ST_CAPACITY) {
        *out_bytes = pre + m.total;
        set_error("preallocated output too small");
        return MGARD_ECAPACITY;
    }
    const size_t total = pre + m.total;
    if (rh) rh->inner_bytes = m.total;
    if (direct) {
        if (rh) {
            MGB_CUDA(cudaMemcpyAsync(*out, rh, sizeof(*rh), cudaMemcpyHostToDevice, st));
            MGB_CUDA(cudaMemsetAsync((char*)*out + sizeof(*rh), 0, pre - sizeof(*rh), st));
            MGB_CUDA(cudaStreamSynchronize(st));
        }
        *out_bytes = total;
        return MGARD_OK;
    }
    char* dst;
    if (prealloc) {
        if (*out_bytes < total) {
            *out_bytes = total;
            set_error("preallocated output too small");
            return MGARD_ECAPACITY;
        }
        dst = (char*)*out;
    } else if (field_dev) {
        void* q = nullptr;
        count_device_alloc();
        cudaError_t e = cudaMalloc(&q, total);
        if (e != cudaSuccess) {
            set_error(std::string("output allocation: ") + cudaGetErrorString(e));
            return MGARD_ENOMEM;
        }
        dst = (char*)q;
    } else {
        dst = (char*)std::malloc(total);
        if (!dst) {
            set_error("host output allocation failed");
            return MGARD_ENOMEM;
        }
    }
    if (rh) {
        char head[MGARD_REGION_INNER] = {};
        std::memcpy(head, rh, sizeof(*rh));
        MGB_CUDA(cudaMemcpyAsync(dst, head, pre, cudaMemcpyDefault, st));
    }
    MGB_CUDA(cudaMemcpyAsync(dst + pre, dd, m.total, cudaMemcpyDefault, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    *out = dst;
    *out_bytes = total;
    return MGARD_OK;
}

mgard_status read_header(const void* in, size_t in_bytes, bool in_dev, mgard_header* h,
                         std::vector<double>* widths, cudaStream_t st) {
    if (!in || in_bytes < sizeof(mgard_header)) {
        set_error("compressed buffer too small");
        return MGARD_ECORRUPT;
    }
    // a device buffer's header and widths (which follow it) come over in
    // one copy and one synchronization
    constexpr size_t HEAD = 768;   // header + widths of up to 64 levels
    static_assert(sizeof(mgard_header) <= HEAD, "the header fits the first copy");
    alignas(16) char head[HEAD];
    const size_t got = std::min(in_bytes, HEAD);
    if (in_dev) {
        MGB_CUDA(cudaMemcpyAsync(head, in, got, cudaMemcpyDeviceToHost, st));
        MGB_CUDA(cudaStreamSynchronize(st));
    } else {
        std::memcpy(head, in, got);
    }
    std::memcpy(h, head, sizeof(*h));
    MGB_TRY(check_header(*h, in_bytes));
    widths->resize(h->nlevels + 1);
    const size_t wbytes = 8 * (size_t)(h->nlevels + 1);
    if (h->off_widths + wbytes <= got)
        std::memcpy(widths->data(), head + h->off_widths, wbytes);
    else if (in_dev)
        MGB_CUDA(cudaMemcpy(widths->data(), (const char*)in + h->off_widths, wbytes,
                            cudaMemcpyDeviceToHost));
    else
        std::memcpy(widths->data(), (const char*)in + h->off_widths, wbytes);
    if (!widths_valid(widths->data(), (int)h->nlevels)) {
        set_error("corrupt header: bin width");
        return MGARD_ECORRUPT;
    }
    return MGARD_OK;
}

template <typename T>
mgard_status decompress_impl(const Plan& p, const mgard_header& h, const std::vector<double>& w,
                             const char* din, void** field, bool out_dev, void* dst,
                             cudaStream_t st, const RegionScale* rs) {
    const int64_t N = p.total();
    DevBuf stage, stat;
    T* dout = (T*)dst;
    if (!out_dev) {
        MGB_TRY(stage.alloc(N * sizeof(T), st));
        dout = stage.as<T>();
    }
    DecompressWork<T> work;
    MGB_TRY(work.alloc(p, st));
    MGB_TRY(stat.alloc(sizeof(unsigned), st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(unsigned), st));
    MGB_TRY(decompress_core<T>(p, h, w.data(), din, dout, work, stat.as<unsigned>(), st, rs));
    unsigned status = 0;
    MGB_CUDA(cudaMemcpyAsync(&status, stat.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    MGB_TRY(status_to_error(status));
    if (!out_dev) {
        MGB_CUDA(cudaMemcpyAsync(dst, dout, N * sizeof(T), cudaMemcpyDeviceToHost, st));
        MGB_CUDA(cudaStreamSynchronize(st));
    }
    *field = dst;
    return MGARD_OK;
}

// Decompress an ordinary buffer (device or host), optionally with region
// scaling of its coefficients.
mgard_status decompress_buffer(const void* in, size_t in_bytes, bool in_dev, void** field,
                               int prealloc, cudaStream_t st, const RegionScale* rs) {
    mgard_header h;
    std::vector<double> w;
    MGB_TRY(read_header(in, in_bytes, in_dev, &h, &w, st));
    const Plan* p;
    MGB_TRY(get_plan((int)h.ndim, h.shape, -1, &p));
    if (p->L != (int)h.nlevels) {
        set_error("corrupt header: level count");
        return MGARD_ECORRUPT;
    }
    const size_t nbytes = (size_t)p->total() * ((h.dtype == MGARD_F64) ? 8 : 4);
    // device image of the compressed buffer
    DevBuf inbuf;
    const char* din = (const char*)in;
    if (!in_dev) {
        MGB_TRY(inbuf.alloc(h.total_bytes, st));
        MGB_CUDA(cudaMemcpyAsync(inbuf.p, in, h.total_bytes, cudaMemcpyHostToDevice, st));
        din = inbuf.as<char>();
    }
    void* dst;
    bool out_dev;
    if (prealloc) {
        if (!*field) {
            set_error("preallocated output missing");
            return MGARD_EINVAL;
        }
        dst = *field;
        out_dev = is_device_ptr(dst);
    } else {
        out_dev = in_dev;
        if (out_dev) {
            count_device_alloc();
            cudaError_t e = cudaMalloc(&dst, nbytes);
            if (e != cudaSuccess) {
                set_error(std::string("output allocation: ") + cudaGetErrorString(e));
                return MGARD_ENOMEM;
            }
        } else {
            dst = std::malloc(nbytes);
            if (!dst) return MGARD_ENOMEM;
        }
    }
    mgard_status r;
    if (h.dtype == MGARD_F32) r = decompress_impl<float>(*p, h, w, din, field, out_dev, dst, st, rs);
    else r = decompress_impl<double>(*p, h, w, din, field, out_dev, dst, st, rs);
    if (r != MGARD_OK && !prealloc) mgard_free(dst);
    return r;
}


bool region_magic(const void* in, size_t in_bytes, bool in_dev, cudaStream_t st) {
    char m[8] = {};
    if (in_bytes < 8) return false;
    if (in_dev) {
        if (cudaMemcpyAsync(m, in, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    } else {
        std::memcpy(m, in, 8);
    }
    return std::memcmp(m, MGARD_REGION_MAGIC, 8) == 0;
}

// The region header of a buffer, checked, and the boxes as mgard_region.
mgard_status read_region_header(const void* in, size_t in_bytes, bool in_dev,
                                mgard_region_header* rh, mgard_region* boxes, cudaStream_t st) {
    if (in_bytes < MGARD_REGION_INNER) {
        set_error("region buffer too small");
        return MGARD_ECORRUPT;
    }
    if (in_dev) {
        MGB_CUDA(cudaMemcpyAsync(rh, in, sizeof(*rh), cudaMemcpyDeviceToHost, st));
        MGB_CUDA(cudaStreamSynchronize(st));
    } else {
        std::memcpy(rh, in, sizeof(*rh));
    }
    if (std::memcmp(rh->magic, MGARD_REGION_MAGIC, 8) != 0 || rh->version != MGARD_REGION_VERSION ||
        rh->nregions > MGARD_REGION_SLOTS || rh->rho < 0 || rh->rho > Plan::RHO_MAX ||
        rh->inner_bytes > in_bytes - MGARD_REGION_INNER || !(rh->tol > 0.0) ||
        !std::isfinite(rh->tol)) {
        set_error("corrupt region header");
        return MGARD_ECORRUPT;
    }
    for (uint32_t r = 0; r < rh->nregions; ++r) {
        for (int a = 0; a < 4; ++a) {
            boxes[r].lo[a] = rh->box[r].lo[a];
            boxes[r].hi[a] = rh->box[r].hi[a];
        }
        boxes[r].tol = rh->box[r].tol;
    }
    return MGARD_OK;
}

mgard_status decompress_regions(const void* in, size_t in_bytes, bool in_dev, void** field,
                                int prealloc, cudaStream_t st) {
    mgard_region_header rh;
    mgard_region boxes[MGARD_REGION_SLOTS];
    MGB_TRY(read_region_header(in, in_bytes, in_dev, &rh, boxes, st));
    const char* inner = (const char*)in + MGARD_REGION_INNER;
    mgard_header h;
    std::vector<double> w;
    MGB_TRY(read_header(inner, rh.inner_bytes, in_dev, &h, &w, st));
    const Plan* p;
    MGB_TRY(get_plan((int)h.ndim, h.shape, -1, &p));
    RegionScale rs;
    if (region_table(*p, (int)h.ndim, h.shape, rh.rho, rh.k, boxes, (int)rh.nregions, &rs) != MGARD_OK) {
        set_error("corrupt region header: boxes");
        return MGARD_ECORRUPT;
    }
    return decompress_buffer(inner, rh.inner_bytes, in_dev, field, prealloc, st, &rs);
}

}  // namespace

mgard_status status_to_error(unsigned st) {
    if (st & ST_TIMEOUT) {
        set_error("a bounded device wait (tensor-copy barrier) gave up");
        return MGARD_ETIMEOUT;
    }
    if (st & ST_NONFINITE) {
        set_error("input holds NaN or Inf");
        return MGARD_ENONFINITE;
    }
    if (st & ST_RANGE) {
        set_error("tolerance too small: a quantized value exceeds the 32-bit range");
        return MGARD_ERANGE;
    }
    if (st & ST_CORRUPT) {
        set_error("compressed stream is corrupt");
        return MGARD_ECORRUPT;
    }
    if (st & ST_NOCODE) {
        set_error("a symbol has no Huffman code");
        return MGARD_EINVAL;
    }
    return MGARD_OK;
}

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {
std::atomic<uint64_t> g_device_allocs{0};
}
void count_device_alloc() { g_device_allocs.fetch_add(1, std::memory_order_relaxed); }

}  // namespace mgb

using namespace mgb;

extern "C" {

const char* mgard_strerror(mgard_status s) {
    switch (s) {
        case MGARD_OK: return "ok";
        case MGARD_EINVAL: return "invalid argument";
        case MGARD_ESHAPE: return "invalid shape";
        case MGARD_EDTYPE: return "invalid dtype";
        case MGARD_ENONFINITE: return "non-finite input";
        case MGARD_ENOMEM: return "out of memory";
        case MGARD_ECUDA: return "CUDA error";
        case MGARD_ECORRUPT: return "corrupt compressed buffer";
        case MGARD_EBOUND: return "error bound violated";
        case MGARD_ETIMEOUT: return "device wait timed out";
        case MGARD_ECAPACITY: return "output capacity too small";
        case MGARD_ERANGE: return "tolerance too small for 32-bit quantization";
    }
    return "unknown status";
}

const char* mgard_last_error(void) { return g_last_error.c_str(); }

uint64_t mgard_device_allocations(void) {
    return mgb::g_device_allocs.load(std::memory_order_relaxed);
}

uint32_t mgard_version(void) { return 0x010000u; }

mgard_status mgard_levels(int ndim, const int64_t* shape, int max_levels, int* nlevels) {
    int64_t n4[4];
    int D;
    MGB_TRY(squeeze_shape(ndim, shape, n4, &D));
    if (!nlevels) return MGARD_EINVAL;
    *nlevels = level_count(n4, D, max_levels);
    return MGARD_OK;
}

mgard_status mgard_decompose(void* data, int ndim, const int64_t* shape, mgard_dtype dtype,
                             int max_levels, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!data) return MGARD_EINVAL;
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MGARD_F32) {
        Pyramid<float> py;
        MGB_TRY(py.alloc(*p, st));
        MGB_TRY(decompose_pyramid<float>(*p, (float*)data, (float*)data, py, st, nullptr));
        MGB_TRY(scatter_levels<float>(*p, py, (float*)data, st));
    } else {
        Pyramid<double> py;
        MGB_TRY(py.alloc(*p, st));
        MGB_TRY(decompose_pyramid<double>(*p, (double*)data, (double*)data, py, st, nullptr));
        MGB_TRY(scatter_levels<double>(*p, py, (double*)data, st));
    }
    return MGARD_OK;
}

mgard_status mgard_recompose(void* data, int ndim, const int64_t* shape, mgard_dtype dtype,
                             int max_levels, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!data) return MGARD_EINVAL;
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MGARD_F32) {
        Pyramid<float> py;
        MGB_TRY(py.alloc(*p, st));
        MGB_TRY(gather_levels<float>(*p, (float*)data, py, st));
        MGB_TRY(recompose_pyramid<float>(*p, (float*)data, (float*)data, py, st));
    } else {
        Pyramid<double> py;
        MGB_TRY(py.alloc(*p, st));
        MGB_TRY(gather_levels<double>(*p, (double*)data, py, st));
        MGB_TRY(recompose_pyramid<double>(*p, (double*)data, (double*)data, py, st));
    }
    return MGARD_OK;
}

mgard_status mgard_bin_widths(int ndim, const int64_t* shape, int max_levels, double tol_abs,
                              double s, double* widths, int* nlevels) {
    if (!widths || !(tol_abs > 0.0) || !std::isfinite(tol_abs) || std::isnan(s) || s < 0.0) {
        set_error("tol_abs must be positive and finite, s >= 0 or INFINITY");
        return MGARD_EINVAL;
    }
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p, false));
    bin_widths(*p, tol_abs, s, widths);
    if (nlevels) *nlevels = p->L;
    return MGARD_OK;
}

mgard_status mgard_norm(const void* data, int ndim, const int64_t* shape, mgard_dtype dtype,
                        int max_levels, double s, double* out, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!data || !out || std::isnan(s) || s < 0.0) return MGARD_EINVAL;
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MGARD_F32) return norm_impl<float>(*p, (const float*)data, s, out, st);
    return norm_impl<double>(*p, (const double*)data, s, out, st);
}

mgard_status mgard_error_norm(const void* a, const void* b, int ndim, const int64_t* shape,
                              mgard_dtype dtype, int max_levels, double s, double* out,
                              void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!a || !b || !out || std::isnan(s) || s < 0.0) return MGARD_EINVAL;
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = p->total();
    unsigned status = 0;
    if (std::isinf(s)) {
        if (dtype == MGARD_F32) MGB_TRY(max_abs<float>((const float*)a, (const float*)b, N, out, &status, st));
        else MGB_TRY(max_abs<double>((const double*)a, (const double*)b, N, out, &status, st));
        return status_to_error(status);
    }
    DevBuf y;
    MGB_TRY(y.alloc(N * sizeof(double), st));
    if (dtype == MGARD_F32) MGB_TRY(difference<float>((const float*)a, (const float*)b, y.as<double>(), N, st));
    else MGB_TRY(difference<double>((const double*)a, (const double*)b, y.as<double>(), N, st));
    return norm_impl<double>(*p, y.as<double>(), s, out, st);
}

mgard_status mgard_quantize(const void* coeffs, int ndim, const int64_t* shape, mgard_dtype dtype,
                            int max_levels, const double* widths, uint16_t* symbols,
                            int32_t* escapes, uint64_t* hist, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!coeffs || !widths || !symbols || !escapes || !hist) return MGARD_EINVAL;
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    for (int l = 0; l <= p->L; ++l)
        if (!(widths[l] > 0.0) || !std::isfinite(widths[l])) {
            set_error("bin widths must be positive and finite");
            return MGARD_EINVAL;
        }
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf stat, wdev;
    MGB_TRY(stat.alloc(sizeof(unsigned), st));
    MGB_TRY(wdev.alloc(sizeof(double) * (p->L + 1), st));
    MGB_CUDA(cudaMemcpyAsync(wdev.p, widths, sizeof(double) * (p->L + 1), cudaMemcpyHostToDevice, st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(unsigned), st));
    MGB_CUDA(cudaMemsetAsync(hist, 0, DICT * sizeof(uint64_t), st));
    for (int l = 0; l <= p->L; ++l) {
        const double* wl = wdev.as<double>() + l;
        if (dtype == MGARD_F32)
            MGB_TRY(quantize_level<float>(*p, l, (const float*)coeffs, true, wl, symbols,
                                          escapes, (unsigned long long*)hist, stat.as<unsigned>(), st));
        else
            MGB_TRY(quantize_level<double>(*p, l, (const double*)coeffs, true, wl, symbols,
                                           escapes, (unsigned long long*)hist, stat.as<unsigned>(), st));
    }
    unsigned status = 0;
    MGB_CUDA(cudaMemcpyAsync(&status, stat.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    return status_to_error(status);
}

mgard_status mgard_dequantize(const uint16_t* symbols, const int32_t* escapes, int ndim,
                              const int64_t* shape, mgard_dtype dtype, int max_levels,
                              const double* widths, void* coeffs, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!coeffs || !widths || !symbols || !escapes) return MGARD_EINVAL;
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, max_levels, &p));
    cudaStream_t st = (cudaStream_t)stream;
    for (int l = 0; l <= p->L; ++l) {
        if (dtype == MGARD_F32)
            MGB_TRY(dequantize_level<float>(*p, l, symbols, escapes, true, widths[l], (float*)coeffs, st));
        else
            MGB_TRY(dequantize_level<double>(*p, l, symbols, escapes, true, widths[l], (double*)coeffs, st));
    }
    return MGARD_OK;
}

mgard_status mgard_huffman_codebook(const uint64_t* hist, uint8_t* lengths, uint32_t* codes,
                                    void* stream) {
    if (!hist || !lengths || !codes) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    MGB_TRY(huffman_codebook((const unsigned long long*)hist, lengths, codes, st));
    DevBuf dt;
    MGB_TRY(dt.alloc(sizeof(DecodeTables), st));
    MGB_TRY(huffman_tables(lengths, codes, dt.as<DecodeTables>(), st));
    return MGARD_OK;
}

mgard_status mgard_huffman_encode(const uint16_t* symbols, uint64_t n, const uint8_t* lengths,
                                  const int32_t* escapes, uint32_t* words, uint64_t words_cap,
                                  uint64_t* word_off, uint64_t* esc_off, uint16_t* sub_off,
                                  int32_t* outliers, uint64_t outliers_cap, uint64_t* nwords,
                                  uint64_t* noutliers, void* stream) {
    if ((!symbols && n) || !lengths || !nwords || !noutliers ||
        (n && (!word_off || !esc_off || !sub_off)))
        return MGARD_EINVAL;
    if (((uintptr_t)symbols & 15) != 0) {
        set_error("symbols must be 16-byte aligned");
        return MGARD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf totals, stat, codes, dt;
    MGB_TRY(totals.alloc(16, st));
    MGB_TRY(stat.alloc(4, st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, 4, st));
    MGB_TRY(huffman_count(symbols, n, lengths, word_off, esc_off, totals.as<unsigned long long>(),
                          stat.as<unsigned>(), st));
    unsigned long long tot[2];
    unsigned status = 0;
    MGB_CUDA(cudaMemcpyAsync(tot, totals.p, 16, cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaMemcpyAsync(&status, stat.p, 4, cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    *nwords = tot[0];
    *noutliers = tot[1];
    MGB_TRY(status_to_error(status));
    if (tot[0] > words_cap || tot[1] > outliers_cap) {
        set_error("encode capacity too small");
        return MGARD_ECAPACITY;
    }
    MGB_TRY(codes.alloc(DICT * 4, st));
    MGB_TRY(dt.alloc(sizeof(DecodeTables), st));
    MGB_TRY(huffman_tables(lengths, codes.as<uint32_t>(), dt.as<DecodeTables>(), st));
    MGB_TRY(huffman_pack(symbols, n, lengths, codes.as<uint32_t>(), word_off, esc_off, escapes,
                         words, sub_off, outliers, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    return MGARD_OK;
}

mgard_status mgard_huffman_decode(const uint32_t* words, uint64_t nwords, const uint64_t* word_off,
                                  const uint64_t* esc_off, const uint16_t* sub_off,
                                  const uint8_t* lengths, uint64_t n, const int32_t* outliers,
                                  uint64_t noutliers, uint16_t* symbols, int32_t* escapes,
                                  void* stream) {
    if (!lengths || (n && (!words || !word_off || !esc_off || !sub_off || !symbols || !escapes)))
        return MGARD_EINVAL;
    if (((uintptr_t)symbols & 15) != 0) {
        set_error("symbols must be 16-byte aligned");
        return MGARD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf codes, dt, stat;
    MGB_TRY(codes.alloc(DICT * 4, st));
    MGB_TRY(dt.alloc(sizeof(DecodeTables), st));
    MGB_TRY(stat.alloc(4, st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, 4, st));
    MGB_TRY(huffman_tables(lengths, codes.as<uint32_t>(), dt.as<DecodeTables>(), st));
    MGB_TRY(huffman_decode(words, nwords, word_off, sub_off, dt.as<DecodeTables>(), n, outliers,
                           noutliers, esc_off, symbols, escapes, stat.as<unsigned>(), st));
    unsigned status = 0;
    MGB_CUDA(cudaMemcpyAsync(&status, stat.p, 4, cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    return status_to_error(status);
}

size_t mgard_compress_bound(int ndim, const int64_t* shape, mgard_dtype dtype) {
    int64_t n4[4];
    int D;
    if (squeeze_shape(ndim, shape, n4, &D) != MGARD_OK) return 0;
    (void)dtype;
    const uint64_t n = (uint64_t)(n4[0] * n4[1] * n4[2] * n4[3]);
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    return layout(64, nchunks, n, n + nchunks).total;
}

mgard_status mgard_compress(const void* field, int ndim, const int64_t* shape, mgard_dtype dtype,
                            double tol, double s, mgard_tolmode mode, void** out,
                            size_t* out_bytes, int out_preallocated, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!field || !out || !out_bytes) {
        set_error("null argument");
        return MGARD_EINVAL;
    }
    if (!(tol > 0.0) || !std::isfinite(tol) || std::isnan(s) || s < 0.0 ||
        (mode != MGARD_ABS && mode != MGARD_REL)) {
        set_error("tol must be positive and finite, s >= 0 or INFINITY, mode ABS or REL");
        return MGARD_EINVAL;
    }
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, -1, &p));
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = is_device_ptr(field);
    // device field into a device buffer: the one-field batch path, which keeps
    // the workspace and replays a captured graph when the same call repeats
    if (dev && out_preallocated && out && *out && out_bytes && is_device_ptr(*out) &&
        ((uintptr_t)*out & 15) == 0) {
        const uint64_t N = (uint64_t)p->total();
        if (*out_bytes >= layout(p->L, (N + CHUNK - 1) / CHUNK, 0, 0).outliers) {
            const void* f = field;
            const int64_t* shp = shape;
            size_t cap = *out_bytes, bytes = 0;
            mgard_status fst = MGARD_OK;
            const mgard_status r = mgard_compress_batch(1, &f, &ndim, &shp, dtype, tol, s, mode, out,
                                                        &cap, &bytes, &fst, MGARD_BATCH_REPEAT, stream);
            if (r == MGARD_OK || r == MGARD_ECAPACITY) *out_bytes = bytes;
            return r;
        }
    }
    if (dtype == MGARD_F32)
        return compress_impl<float>(*p, field, dev, dtype, ndim, shape, tol, s, mode, out, out_bytes,
                                    out_preallocated, st);
    return compress_impl<double>(*p, field, dev, dtype, ndim, shape, tol, s, mode, out, out_bytes,
                                 out_preallocated, st);
}

mgard_status mgard_decompress(const void* in, size_t in_bytes, void** field, int out_preallocated,
                              void* stream) {
    if (!in || !field) {
        set_error("null argument");
        return MGARD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool in_dev = is_device_ptr(in);
    if (!in_dev && in_bytes >= 8 && std::memcmp(in, MGARD_REGION_MAGIC, 8) == 0)
        return decompress_regions(in, in_bytes, in_dev, field, out_preallocated, st);
    if (!in_dev && is_ooc_buffer(in, in_bytes))
        return decompress_ooc(in, in_bytes, field, out_preallocated, st);
    // device buffer into a device field: the one-buffer batch path (see
    // mgard_compress); a region buffer fails its header check there
    if (in_dev && out_preallocated && *field && is_device_ptr(*field)) {
        const void* i = in;
        const size_t cap = ~size_t(0);   // the caller guarantees room for the field
        mgard_status fst = MGARD_OK;
        const mgard_status r = mgard_decompress_batch(1, &i, &in_bytes, field, &cap, &fst,
                                                      MGARD_BATCH_REPEAT, stream);
        if (r == MGARD_ECORRUPT && region_magic(in, in_bytes, in_dev, st))
            return decompress_regions(in, in_bytes, in_dev, field, out_preallocated, st);
        return r;
    }
    if (in_dev && region_magic(in, in_bytes, in_dev, st))
        return decompress_regions(in, in_bytes, in_dev, field, out_preallocated, st);
    return decompress_buffer(in, in_bytes, in_dev, field, out_preallocated, st, nullptr);
}

mgard_status mgard_compress_regions(const void* field, int ndim, const int64_t* shape,
                                    mgard_dtype dtype, double tol, const mgard_region* regions,
                                    int nregions, void** out, size_t* out_bytes,
                                    int out_preallocated, void* stream) {
    MGB_TRY(check_dtype(dtype));
    if (!field || !out || !out_bytes || (out_preallocated && !*out)) {
        set_error("null argument");
        return MGARD_EINVAL;
    }
    const Plan* p;
    MGB_TRY(get_plan(ndim, shape, -1, &p));
    mgard_region_header rh;
    std::memset(&rh, 0, sizeof(rh));
    MGB_TRY(region_params(*p, ndim, shape, tol, regions, nregions, &rh.rho, rh.k));
    RegionScale rs;
    MGB_TRY(region_table(*p, ndim, shape, rh.rho, rh.k, regions, nregions, &rs));
    std::memcpy(rh.magic, MGARD_REGION_MAGIC, 8);
    rh.version = MGARD_REGION_VERSION;
    rh.nregions = (uint32_t)nregions;
    rh.tol = tol;
    for (int r = 0; r < nregions; ++r) {
        for (int d = 0; d < ndim; ++d) {
            rh.box[r].lo[d] = regions[r].lo[d];
            rh.box[r].hi[d] = regions[r].hi[d];
        }
        rh.box[r].tol = regions[r].tol;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool dev = is_device_ptr(field);
    if (dtype == MGARD_F32)
        return compress_impl<float>(*p, field, dev, dtype, ndim, shape, tol, INFINITY, MGARD_ABS, out,
                                    out_bytes, out_preallocated, st, &rs, &rh);
    return compress_impl<double>(*p, field, dev, dtype, ndim, shape, tol, INFINITY, MGARD_ABS, out,
                                 out_bytes, out_preallocated, st, &rs, &rh);
}

mgard_status mgard_info(const void* in, size_t in_bytes, int* ndim, int64_t shape[4],
                        mgard_dtype* dtype, double* tol_abs, int* nlevels) {
    mgard_header h;
    std::vector<double> w;
    const bool in_dev = is_device_ptr(in);
    if (!in_dev && is_ooc_buffer(in, in_bytes)) {   // the field's shape, the blocks' tolerance
        mgard_ooc_header oh;
        MGB_TRY(ooc_info(in, in_bytes, &oh));
        const uint64_t first = *(const uint64_t*)((const char*)in + sizeof(oh));
        MGB_TRY(read_header((const char*)in + first, in_bytes - first, false, &h, &w, nullptr));
        if (ndim) *ndim = (int)oh.ndim;
        if (shape)
            for (int i = 0; i < 4; ++i) shape[i] = oh.shape[i];
        if (dtype) *dtype = (mgard_dtype)oh.dtype;
        if (tol_abs) *tol_abs = oh.tol_abs;
        if (nlevels) *nlevels = (int)h.nlevels;
        return MGARD_OK;
    }
    if (in && region_magic(in, in_bytes, in_dev, nullptr)) {   // the wrapped buffer's fields
        mgard_region_header rh;
        mgard_region boxes[MGARD_REGION_SLOTS];
        MGB_TRY(read_region_header(in, in_bytes, in_dev, &rh, boxes, nullptr));
        in = (const char*)in + MGARD_REGION_INNER;
        in_bytes = rh.inner_bytes;
    }
    MGB_TRY(read_header(in, in_bytes, in_dev, &h, &w, nullptr));
    if (ndim) *ndim = (int)h.ndim;
    if (shape)
        for (int i = 0; i < 4; ++i) shape[i] = h.shape[i];
    if (dtype) *dtype = (mgard_dtype)h.dtype;
    if (tol_abs) *tol_abs = h.tol_abs;
    if (nlevels) *nlevels = (int)h.nlevels;
    return MGARD_OK;
}

void mgard_free(void* p) {
    if (!p) return;
    if (is_device_ptr(p)) cudaFree(p);
    else std::free(p);
}

void mgard_release_plans(void) {
    release_batches();
    release_decompress_batches();
    release_plans();
}

}  // extern "C"
