// Refactoring for progressive retrieval (paper: "Software design", the
// refactoring pipeline; "APIs": MDRefactor / MDRequest / MDReconstruct).
//
// The field is decomposed by the compressor's own pipeline (coefficients of
// every level in level order), each level is cut into a sign plane and
// `planes` magnitude planes of its normalized integers q = floor(|c|
// 2^(planes - e)), and any prefix of a level's planes reconstructs its
// coefficients to within 2^(e - P).  On the GPU a warp takes 32 words of a
// level (1024 coefficients): for each word the 32 lanes hold 32
// coefficients, and one ballot per plane gives that plane's word; the words
// of a tile are gathered in shared memory so every plane is written with
// coalesced stores.  Decoding reverses it: the warp loads the selected
// planes' words of its tile, then each lane rebuilds its coefficient from one
// bit of every plane word.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pipeline.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

constexpr int MDR_WARPS = 8;
constexpr int MDR_MAXP = 32;
constexpr uint32_t MDR_VERSION = 1;

bool on_device(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Largest |c| of every level as the bits of a non-negative double (they
// order like the values); blockIdx.y is the level.
template <typename T>
__global__ void k_mdr_levelmax(const T* __restrict__ c, const long long* __restrict__ off,
                               unsigned long long* __restrict__ lmax) {
    const int l = blockIdx.y;
    const long long b = off[l], e = off[l + 1];
    unsigned long long m = 0;
    for (long long i = b + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < e;
         i += (long long)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(fabs((double)c[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(lmax + l, m);
}

// Planes of one level: coefficients c[0 .. n), exponent e, B planes; the
// sign plane at out[0 .. words), plane b at out[(1 + b) words ..].
template <typename T>
__global__ void __launch_bounds__(MDR_WARPS * 32) k_mdr_encode(const T* __restrict__ c, long long n,
                                                               int e, int B, uint32_t words,
                                                               uint32_t* __restrict__ out) {
    __shared__ uint32_t tile[MDR_WARPS][MDR_MAXP + 1][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t(*tw)[33] = tile[wid];
    const double scale = ldexp(1.0, B - e);
    for (long long w0 = ((long long)blockIdx.x * MDR_WARPS + wid) * 32; w0 < (long long)words;
         w0 += (long long)gridDim.x * MDR_WARPS * 32) {
        for (int k = 0; k < 32; ++k) {
            const long long i = (w0 + k) * 32 + lane;
            const double v = i < n ? (double)c[i] : 0.0;
            const uint32_t q = (uint32_t)floor(fabs(v) * scale);   // exact: < 2^B
            const uint32_t sg = __ballot_sync(0xffffffffu, v < 0.0);
            if (lane == 0) tw[0][k] = sg;
            for (int b = 0; b < B; ++b) {
                const uint32_t pw = __ballot_sync(0xffffffffu, (q >> (B - 1 - b)) & 1u);
                if (lane == (b & 31)) tw[1 + b][k] = pw;
            }
        }
        __syncwarp();
        const long long w = w0 + lane;
        if (w < (long long)words)
            for (int b = 0; b <= B; ++b) out[(long long)b * words + w] = tw[b][lane];
        __syncwarp();
    }
}

// Coefficients of one level from its first P planes (and the sign plane).
template <typename T>
__global__ void __launch_bounds__(MDR_WARPS * 32) k_mdr_decode(const uint32_t* __restrict__ in,
                                                               long long n, int e, int B, int P,
                                                               uint32_t words, T* __restrict__ c) {
    __shared__ uint32_t tile[MDR_WARPS][MDR_MAXP + 1][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t(*tw)[33] = tile[wid];
    const double unit = ldexp(1.0, e - B);
    const double half = P < B ? ldexp(1.0, B - P - 1) : 0.0;
    for (long long w0 = ((long long)blockIdx.x * MDR_WARPS + wid) * 32; w0 < (long long)words;
         w0 += (long long)gridDim.x * MDR_WARPS * 32) {
        const long long w = w0 + lane;
        for (int b = 0; b <= P; ++b) tw[b][lane] = w < (long long)words ? in[(long long)b * words + w] : 0u;
        __syncwarp();
        for (int k = 0; k < 32; ++k) {
            const long long i = (w0 + k) * 32 + lane;
            uint32_t q = 0;
            for (int b = 0; b < P; ++b) q |= ((tw[1 + b][k] >> lane) & 1u) << (B - 1 - b);
            double v = q ? ((double)q + half) * unit : 0.0;
            if ((tw[0][k] >> lane) & 1u) v = -v;
            if (i < n) c[i] = (T)v;
        }
        __syncwarp();
    }
}

size_t header_bytes() { return (sizeof(mgard_mdr_header) + 15) & ~size_t(15); }

// Level layout of a refactored buffer.
void level_layout(const Plan& p, int B, mgard_mdr_header* h) {
    uint64_t off = header_bytes();
    for (int l = 0; l <= p.L; ++l) {
        mgard_mdr_level& lv = h->level[l];
        lv.count = (uint64_t)p.count[l];
        lv.words = (uint32_t)((lv.count + 31) / 32);
        lv.offset = off;
        off += ((uint64_t)(B + 1) * lv.words * 4 + 15) & ~uint64_t(15);
        lv.weight = l == 0 ? 1.0 : p.linf_c[l];
    }
    h->total_bytes = off;
}

int grid_words(uint32_t words) {
    const int64_t per = MDR_WARPS * 32;
    return (int)std::max<int64_t>(1, std::min<int64_t>((words + per - 1) / per, 148LL * 8));
}

template <typename T>
mgard_status refactor_t(const Plan& p, const T* din, int ndim, const int64_t* shape, int B,
                        mgard_dtype dtype, char* out, size_t* out_bytes, cudaStream_t st) {
    mgard_mdr_header h;
    std::memset(&h, 0, sizeof(h));
    level_layout(p, B, &h);
    if (*out_bytes < h.total_bytes) {
        *out_bytes = h.total_bytes;
        set_error("refactor: output capacity too small");
        return MGARD_ECAPACITY;
    }
    CompressWork<T> w;
    MGB_TRY(w.alloc(p, st));
    DevBuf meta, offs, lmax;
    MGB_TRY(meta.alloc(sizeof(CompressMeta), st));
    MGB_TRY(offs.alloc(sizeof(long long) * (p.L + 2), st));
    MGB_TRY(lmax.alloc(sizeof(unsigned long long) * (p.L + 1), st));
    MGB_TRY(compress_decompose<T>(p, din, INFINITY, MGARD_ABS, w, meta.as<CompressMeta>(), st));
    const T* coeff = w.top.template as<T>();   // every level in level order
    std::vector<long long> ho(p.L + 2, 0);
    for (int l = 0; l <= p.L; ++l) ho[l + 1] = ho[l] + p.count[l];
    MGB_CUDA(cudaMemcpyAsync(offs.p, ho.data(), sizeof(long long) * (p.L + 2), cudaMemcpyHostToDevice, st));
    MGB_CUDA(cudaMemsetAsync(lmax.p, 0, sizeof(unsigned long long) * (p.L + 1), st));
    MGB_LAUNCH("k_mdr_levelmax", st, k_mdr_levelmax<T><<<dim3(148, p.L + 1), 256, 0, st>>>(
                                         coeff, offs.as<long long>(), lmax.as<unsigned long long>()));
    MGB_CUDA(cudaGetLastError());
    std::vector<unsigned long long> hm(p.L + 1);
    double parts[RED_PARTS];
    CompressMeta m;
    MGB_CUDA(cudaMemcpyAsync(hm.data(), lmax.p, sizeof(unsigned long long) * (p.L + 1), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaMemcpyAsync(parts, w.parts.p, sizeof(parts), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaMemcpyAsync(&m, meta.p, sizeof(m), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    if (m.status & ST_NONFINITE) {
        set_error("input holds NaN or Inf");
        return MGARD_ENONFINITE;
    }
    if (m.status & ST_TIMEOUT) {
        set_error("a bounded device wait (tensor-copy barrier) gave up");
        return MGARD_ETIMEOUT;
    }
    std::memcpy(h.magic, "MGARDMDR", 8);
    h.version = MDR_VERSION;
    h.dtype = (uint32_t)dtype;
    h.ndim = (uint32_t)ndim;
    h.nlevels = (uint32_t)(p.L + 1);
    h.planes = (uint32_t)B;
    for (int d = 0; d < 4; ++d) h.shape[d] = d < ndim ? shape[d] : 1;
    double umax = 0.0;
    for (double v : parts) umax = std::max(umax, v);
    h.max_abs = umax;
    for (int l = 0; l <= p.L; ++l) {
        double mx;
        std::memcpy(&mx, &hm[l], sizeof(mx));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);
        h.level[l].exponent = e;
        h.level[l].nonzero = mx > 0.0 ? 1u : 0u;
    }
    // header, then every level's planes
    MGB_CUDA(cudaMemsetAsync(out, 0, header_bytes(), st));
    MGB_CUDA(cudaMemcpyAsync(out, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    for (int l = 0; l <= p.L; ++l) {
        const mgard_mdr_level& lv = h.level[l];
        MGB_LAUNCH("k_mdr_encode", st, k_mdr_encode<T><<<grid_words(lv.words), MDR_WARPS * 32, 0, st>>>(
                                           coeff + p.offset[l], (long long)lv.count, lv.exponent, B,
                                           lv.words, (uint32_t*)(out + lv.offset)));
        MGB_CUDA(cudaGetLastError());
    }
    MGB_CUDA(cudaStreamSynchronize(st));
    *out_bytes = h.total_bytes;
    return MGARD_OK;
}

template <typename T>
mgard_status reconstruct_t(const Plan& p, const mgard_mdr_header& h, const char* in,
                           const int32_t* P, T* dout, cudaStream_t st) {
    DecompressWork<T> work;
    MGB_TRY(work.alloc(p, st));
    DevBuf stat;
    MGB_TRY(stat.alloc(sizeof(unsigned), st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(unsigned), st));
    work.py.status = stat.as<unsigned>();
    T* zs = work.zs.template as<T>();
    for (int l = 0; l <= p.L; ++l) {
        const mgard_mdr_level& lv = h.level[l];
        MGB_LAUNCH("k_mdr_decode", st, k_mdr_decode<T><<<grid_words(lv.words), MDR_WARPS * 32, 0, st>>>(
                                           (const uint32_t*)(in + lv.offset), (long long)lv.count,
                                           lv.exponent, (int)h.planes, P[l], lv.words, zs + p.offset[l]));
        MGB_CUDA(cudaGetLastError());
    }
    MGB_TRY(recompose_pyramid<T>(p, nullptr, dout, work.py, st, zs));
    unsigned status = 0;
    MGB_CUDA(cudaMemcpyAsync(&status, stat.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    if (status & ST_TIMEOUT) {
        set_error("a bounded device wait (tensor-copy barrier) gave up");
        return MGARD_ETIMEOUT;
    }
    return MGARD_OK;
}

mgard_status mdr_plan(int ndim, const int64_t* shape, const Plan** p) {
    MGB_TRY(get_plan(ndim, shape, -1, p));
    if (!rows3_ok(**p)) {
        set_error("refactoring takes grids of up to three active axes");
        return MGARD_ESHAPE;
    }
    if ((*p)->L > MGARD_MDR_MAX_LEVELS) {
        set_error("too many levels");
        return MGARD_ESHAPE;
    }
    return MGARD_OK;
}

}  // namespace

}  // namespace mgb

using namespace mgb;

extern "C" size_t mgard_refactor_bound(int ndim, const int64_t* shape, int planes) {
    const Plan* p = nullptr;
    if (planes < 1 || planes > MDR_MAXP || get_plan(ndim, shape, -1, &p, false) != MGARD_OK) return 0;
    mgard_mdr_header h;
    std::memset(&h, 0, sizeof(h));
    level_layout(*p, planes, &h);
    return (size_t)h.total_bytes;
}

extern "C" mgard_status mgard_refactor(const void* field, int ndim, const int64_t* shape,
                                       mgard_dtype dtype, int planes, void* out, size_t* out_bytes,
                                       void* stream) {
    if (!field || !out || !out_bytes || planes < 1 || planes > MDR_MAXP) {
        set_error("refactor: null pointer or planes outside 1..32");
        return MGARD_EINVAL;
    }
    if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_EDTYPE;
    if (!on_device(field) || !on_device(out) || ((uintptr_t)out & 15)) {
        set_error("refactor: field and out must be device memory, out 16-byte aligned");
        return MGARD_EINVAL;
    }
    const Plan* p = nullptr;
    MGB_TRY(mdr_plan(ndim, shape, &p));
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == MGARD_F32)
        return refactor_t<float>(*p, (const float*)field, ndim, shape, planes, dtype, (char*)out,
                                 out_bytes, st);
    return refactor_t<double>(*p, (const double*)field, ndim, shape, planes, dtype, (char*)out,
                              out_bytes, st);
}

extern "C" mgard_status mgard_request(const mgard_mdr_header* h, double tol, int32_t* P,
                                      uint64_t* bytes, double* estimate) {
    if (!h || !P || std::memcmp(h->magic, "MGARDMDR", 8) != 0 || h->version != MDR_VERSION ||
        h->nlevels < 1 || h->nlevels > MGARD_MDR_MAX_LEVELS + 1 || h->planes < 1 ||
        h->planes > (uint32_t)MDR_MAXP || !(tol >= 0)) {
        set_error("request: bad header or tolerance");
        return MGARD_EINVAL;
    }
    const int nl = (int)h->nlevels, B = (int)h->planes;
    auto bound = [&](int l, int planes) {
        return h->level[l].nonzero ? std::ldexp(1.0, h->level[l].exponent - planes) : 0.0;
    };
    auto est_of = [&]() {   // left to right in level order; each term is exact
        double e = 0.0;
        for (int l = 0; l < nl; ++l) e += h->level[l].weight * bound(l, P[l]);
        return e;
    };
    for (int l = 0; l < nl; ++l) P[l] = 0;
    double est = est_of();
    while (est > tol) {
        int best = -1;
        double best_rate = -1.0;
        for (int l = 0; l < nl; ++l) {
            if (P[l] >= B || !h->level[l].nonzero) continue;
            const double gain = h->level[l].weight * (bound(l, P[l]) - bound(l, P[l] + 1));
            const double cost = 4.0 * h->level[l].words * (P[l] == 0 ? 2 : 1);
            const double rate = gain / cost;
            if (rate > best_rate) {
                best = l;
                best_rate = rate;
            }
        }
        if (best < 0) break;
        ++P[best];
        est = est_of();
    }
    uint64_t nb = 0;
    for (int l = 0; l < nl; ++l)
        if (P[l] > 0) nb += 4ull * h->level[l].words * (uint64_t)(1 + P[l]);
    if (bytes) *bytes = nb;
    if (estimate) *estimate = est;
    if (est > tol) {
        set_error("request: the tolerance is below what every stored plane guarantees");
        return MGARD_EBOUND;
    }
    return MGARD_OK;
}

extern "C" mgard_status mgard_reconstruct(const void* refactored, const int32_t* P, void* field,
                                          void* stream) {
    if (!refactored || !P || !field) return MGARD_EINVAL;
    if (!on_device(refactored) || !on_device(field)) {
        set_error("reconstruct: buffers must be device memory");
        return MGARD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    mgard_mdr_header h;
    MGB_CUDA(cudaMemcpyAsync(&h, refactored, sizeof(h), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    if (std::memcmp(h.magic, "MGARDMDR", 8) != 0 || h.version != MDR_VERSION || h.ndim < 1 ||
        h.ndim > 4 || h.planes < 1 || h.planes > (uint32_t)MDR_MAXP ||
        (h.dtype != MGARD_F32 && h.dtype != MGARD_F64)) {
        set_error("reconstruct: not a refactored buffer");
        return MGARD_ECORRUPT;
    }
    const Plan* p = nullptr;
    MGB_TRY(mdr_plan((int)h.ndim, h.shape, &p));
    mgard_mdr_header want;
    std::memset(&want, 0, sizeof(want));
    level_layout(*p, (int)h.planes, &want);
    if (h.nlevels != (uint32_t)(p->L + 1) || h.total_bytes != want.total_bytes) {
        set_error("reconstruct: header does not match its shape");
        return MGARD_ECORRUPT;
    }
    for (int l = 0; l <= p->L; ++l) {
        if (h.level[l].offset != want.level[l].offset || h.level[l].words != want.level[l].words ||
            h.level[l].count != want.level[l].count || h.level[l].exponent < -1100 ||
            h.level[l].exponent > 1100) {
            set_error("reconstruct: level table does not match its shape");
            return MGARD_ECORRUPT;
        }
        if (P[l] < 0 || P[l] > (int32_t)h.planes) {
            set_error("reconstruct: plane count outside 0..planes");
            return MGARD_EINVAL;
        }
    }
    if (h.dtype == MGARD_F32)
        return reconstruct_t<float>(*p, h, (const char*)refactored, P, (float*)field, st);
    return reconstruct_t<double>(*p, h, (const char*)refactored, P, (double*)field, st);
}
