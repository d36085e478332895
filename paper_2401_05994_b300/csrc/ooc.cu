// Out-of-core compression (paper: "Software architecture", the out-of-core
// module that chunks arrays to fit device memory; "APIs": host or device
// buffers).
//
// A host field is cut along its first axis into blocks that are compressed
// independently (each block has its own hierarchy and keeps the L-infinity
// bound on its nodes, so the whole field keeps it).  Two streams alternate
// over the blocks: while one block is being decomposed and encoded, the next
// block's host-to-device copy and the previous block's device-to-host copy
// run on the other stream, so with pinned host memory the PCIe transfers
// overlap the kernels.  A relative tolerance takes max|u| of the whole field
// from a first streaming pass (host-to-device copies and the max-abs
// reduction, overlapped the same way).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "../../include/mgard_b300.h"
#include "pipeline.cuh"

namespace mgb {

namespace {

constexpr int NS = 2;   // streams (and buffers) in flight

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct Blocks {
    int64_t n0 = 0, plane = 0, nb = 0, q = 0, r = 0;
    int64_t begin(int64_t b) const { return b * q + std::min(b, r); }
    int64_t rows(int64_t b) const { return q + (b < r ? 1 : 0); }
};

mgard_status make_blocks(int ndim, const int64_t* shape, int64_t nblocks, Blocks* bl) {
    if (ndim < 1 || ndim > 4 || !shape || shape[0] < 1 || nblocks < 1 || nblocks > shape[0]) {
        set_error("out-of-core: 1..4 axes and 1..shape[0] blocks");
        return MGARD_EINVAL;
    }
    bl->n0 = shape[0];
    bl->plane = 1;
    for (int d = 1; d < ndim; ++d) bl->plane *= shape[d];
    bl->nb = nblocks;
    bl->q = shape[0] / nblocks;
    bl->r = shape[0] % nblocks;
    return MGARD_OK;
}

struct Streams {
    cudaStream_t s[NS] = {};
    cudaEvent_t ev[NS] = {};
    mgard_status init(cudaStream_t caller) {
        cudaEvent_t start;
        MGB_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
        MGB_CUDA(cudaEventRecord(start, caller));
        for (int i = 0; i < NS; ++i) {
            MGB_CUDA(cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking));
            MGB_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
            MGB_CUDA(cudaStreamWaitEvent(s[i], start, 0));
        }
        cudaEventDestroy(start);
        return MGARD_OK;
    }
    ~Streams() {
        for (int i = 0; i < NS; ++i) {
            if (s[i]) {
                cudaStreamSynchronize(s[i]);
                cudaStreamDestroy(s[i]);
            }
            if (ev[i]) cudaEventDestroy(ev[i]);
        }
    }
};

struct Pinned {
    void* p = nullptr;
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
    mgard_status alloc(size_t n) {
        count_device_alloc();
        MGB_CUDA(cudaMallocHost(&p, n));
        return MGARD_OK;
    }
};

int64_t block_shape(const Blocks& bl, int ndim, const int64_t* shape, int64_t b, int64_t* out) {
    out[0] = bl.rows(b);
    for (int d = 1; d < ndim; ++d) out[d] = shape[d];
    return out[0] * bl.plane;
}

// max|u| of a host field, streamed block by block.
template <typename T>
mgard_status streamed_max(const T* host, const Blocks& bl, Streams& ss, DevBuf* in, double* out) {
    DevBuf parts, stat;
    MGB_TRY(parts.alloc((size_t)bl.nb * RED_PARTS * sizeof(double), ss.s[0]));
    MGB_TRY(stat.alloc(NS * sizeof(unsigned), ss.s[0]));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, NS * sizeof(unsigned), ss.s[0]));
    MGB_CUDA(cudaEventRecord(ss.ev[0], ss.s[0]));
    MGB_CUDA(cudaStreamWaitEvent(ss.s[1], ss.ev[0], 0));
    for (int64_t b = 0; b < bl.nb; ++b) {
        const int i = (int)(b % NS);
        const int64_t n = bl.rows(b) * bl.plane;
        MGB_CUDA(cudaMemcpyAsync(in[i].p, host + bl.begin(b) * bl.plane, n * sizeof(T),
                                 cudaMemcpyHostToDevice, ss.s[i]));
        MGB_TRY(max_abs_partials<T>(in[i].as<T>(), n, parts.as<double>() + b * RED_PARTS,
                                    stat.as<unsigned>() + i, ss.s[i]));
    }
    std::vector<double> h((size_t)bl.nb * RED_PARTS);
    unsigned hs[NS];
    for (int i = 0; i < NS; ++i) MGB_CUDA(cudaStreamSynchronize(ss.s[i]));
    MGB_CUDA(cudaMemcpy(h.data(), parts.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    MGB_CUDA(cudaMemcpy(hs, stat.p, sizeof(hs), cudaMemcpyDeviceToHost));
    for (int i = 0; i < NS; ++i) MGB_TRY(status_to_error(hs[i]));
    double m = 0.0;
    for (double v : h) m = std::max(m, v);
    *out = m;
    return MGARD_OK;
}

// Per-stream workspace for the (at most two) block shapes.
template <typename W>
struct ShapeWork {
    const Plan* plan[2] = {nullptr, nullptr};
    std::unique_ptr<W> work[2][NS];
    mgard_status get(const Plan* p, int stream, cudaStream_t st, W** out) {
        for (int k = 0; k < 2; ++k) {
            if (!plan[k]) plan[k] = p;
            if (plan[k] != p) continue;
            if (!work[k][stream]) {
                work[k][stream].reset(new W());
                MGB_TRY(work[k][stream]->alloc(*p, st));
            }
            *out = work[k][stream].get();
            return MGARD_OK;
        }
        set_error("out-of-core: more than two block shapes");
        return MGARD_EINVAL;
    }
};

template <typename T>
mgard_status compress_ooc_t(const T* host, mgard_dtype dtype, int ndim, const int64_t* shape,
                            double tol, mgard_tolmode mode, const Blocks& bl, char* out,
                            size_t cap, size_t* used, cudaStream_t caller) {
    Streams ss;
    MGB_TRY(ss.init(caller));
    const int64_t maxn = (bl.q + (bl.r ? 1 : 0)) * bl.plane;
    DevBuf in[NS], dout[NS], meta[NS];
    int64_t bshape[4];
    block_shape(bl, ndim, shape, 0, bshape);
    const size_t ocap = mgard_compress_bound(ndim, bshape, dtype);
    for (int i = 0; i < NS; ++i) {
        MGB_TRY(in[i].alloc(maxn * sizeof(T), ss.s[i]));
        MGB_TRY(dout[i].alloc(ocap, ss.s[i]));
        MGB_TRY(meta[i].alloc(sizeof(CompressMeta), ss.s[i]));
    }
    double tol_abs = tol;
    if (mode == MGARD_REL) {
        double m = 0.0;
        MGB_TRY(streamed_max<T>(host, bl, ss, in, &m));
        tol_abs = tol * m;
        if (!(tol_abs > 0.0) || !std::isfinite(tol_abs)) {
            set_error("relative tolerance of a zero or non-finite field");
            return MGARD_EINVAL;
        }
    }
    const size_t head = align16(sizeof(mgard_ooc_header) + 8 * (size_t)(bl.nb + 1));
    if (cap < head) {
        *used = head;
        set_error("out-of-core output too small");
        return MGARD_ECAPACITY;
    }
    std::vector<uint64_t> offs((size_t)bl.nb + 1, 0), sizes((size_t)bl.nb, 0);
    Pinned hmeta;
    MGB_TRY(hmeta.alloc(NS * sizeof(CompressMeta)));
    CompressMeta* hm = (CompressMeta*)hmeta.p;
    ShapeWork<CompressWork<T>> sw;
    size_t off = head;
    bool short_cap = false;
    // the block compressed on stream i has its size read, then its bytes
    // copied out behind the next block's launches
    auto finish = [&](int64_t b) -> mgard_status {
        const int i = (int)(b % NS);
        MGB_CUDA(cudaEventSynchronize(ss.ev[i]));
        MGB_TRY(status_to_error(hm[i].status & ~(unsigned)ST_CAPACITY));
        const size_t sz = hm[i].total;
        offs[b] = off;
        sizes[b] = sz;
        if (!short_cap && off + sz <= cap)
            MGB_CUDA(cudaMemcpyAsync(out + off, dout[i].p, sz, cudaMemcpyDeviceToHost, ss.s[i]));
        else
            short_cap = true;
        off = align16(off + sz);
        return MGARD_OK;
    };
    for (int64_t b = 0; b < bl.nb; ++b) {
        const int i = (int)(b % NS);
        const int64_t n = block_shape(bl, ndim, shape, b, bshape);
        const Plan* p;
        MGB_TRY(get_plan(ndim, bshape, -1, &p));
        CompressWork<T>* w;
        MGB_TRY(sw.get(p, i, ss.s[i], &w));
        MGB_CUDA(cudaMemcpyAsync(in[i].p, host + bl.begin(b) * bl.plane, n * sizeof(T),
                                 cudaMemcpyHostToDevice, ss.s[i]));
        const mgard_header h0 = header_template(*p, dtype, ndim, bshape, tol_abs, INFINITY, MGARD_ABS);
        MGB_TRY(compress_core<T>(*p, in[i].as<T>(), h0, tol_abs, INFINITY, MGARD_ABS, dout[i].as<char>(),
                                 ocap, *w, meta[i].as<CompressMeta>(), ss.s[i]));
        MGB_CUDA(cudaMemcpyAsync(&hm[i], meta[i].p, sizeof(CompressMeta), cudaMemcpyDeviceToHost, ss.s[i]));
        MGB_CUDA(cudaEventRecord(ss.ev[i], ss.s[i]));
        if (b >= 1) MGB_TRY(finish(b - 1));
    }
    MGB_TRY(finish(bl.nb - 1));
    for (int i = 0; i < NS; ++i) MGB_CUDA(cudaStreamSynchronize(ss.s[i]));
    offs[bl.nb] = off;
    *used = off;
    if (short_cap) {
        set_error("out-of-core output too small");
        return MGARD_ECAPACITY;
    }
    mgard_ooc_header hh;
    std::memset(&hh, 0, sizeof(hh));
    std::memcpy(hh.magic, MGARD_OOC_MAGIC, 8);
    hh.version = MGARD_OOC_VERSION;
    hh.dtype = (uint32_t)dtype;
    hh.ndim = (uint32_t)ndim;
    hh.nblocks = (uint32_t)bl.nb;
    for (int d = 0; d < 4; ++d) hh.shape[d] = d < ndim ? shape[d] : 1;
    hh.tol = tol;
    hh.tol_abs = tol_abs;
    hh.mode = (uint32_t)mode;
    hh.total_bytes = off;
    std::memset(out, 0, head);
    std::memcpy(out, &hh, sizeof(hh));
    std::memcpy(out + sizeof(hh), offs.data(), 8 * offs.size());
    for (int64_t b = 0; b < bl.nb; ++b)   // alignment gaps, so the bytes depend on the data only
        std::memset(out + offs[b] + sizes[b], 0, offs[b + 1] - offs[b] - sizes[b]);
    return MGARD_OK;
}

mgard_status read_ooc(const char* in, size_t in_bytes, mgard_ooc_header* h, std::vector<uint64_t>* offs,
                      Blocks* bl) {
    auto bad = [](const char* why) {
        set_error(std::string("corrupt out-of-core buffer: ") + why);
        return MGARD_ECORRUPT;
    };
    if (in_bytes < sizeof(*h)) return bad("size");
    std::memcpy(h, in, sizeof(*h));
    if (std::memcmp(h->magic, MGARD_OOC_MAGIC, 8) != 0 || h->version != MGARD_OOC_VERSION)
        return bad("magic or version");
    if (h->dtype > 1 || h->ndim < 1 || h->ndim > 4 || h->nblocks < 1 || h->total_bytes > in_bytes)
        return bad("header");
    for (uint32_t d = 0; d < h->ndim; ++d)
        if (h->shape[d] < 1 || h->shape[d] > (int64_t(1) << 40)) return bad("shape");
    if ((int64_t)h->nblocks > h->shape[0]) return bad("blocks");
    if (make_blocks((int)h->ndim, h->shape, h->nblocks, bl) != MGARD_OK) return bad("blocks");
    const size_t head = align16(sizeof(*h) + 8 * ((size_t)h->nblocks + 1));
    if (head > in_bytes) return bad("offsets");
    offs->resize((size_t)h->nblocks + 1);
    std::memcpy(offs->data(), in + sizeof(*h), 8 * offs->size());
    if ((*offs)[0] != head || (*offs)[h->nblocks] != h->total_bytes) return bad("offsets");
    for (uint32_t b = 0; b < h->nblocks; ++b)
        if ((*offs)[b] > (*offs)[b + 1] || ((*offs)[b] & 15)) return bad("offsets");
    return MGARD_OK;
}

template <typename T>
mgard_status decompress_ooc_t(const char* in, const mgard_ooc_header& hh,
                              const std::vector<uint64_t>& offs, const Blocks& bl, T* field,
                              cudaStream_t caller) {
    Streams ss;
    MGB_TRY(ss.init(caller));
    const int ndim = (int)hh.ndim;
    const int64_t maxn = (bl.q + (bl.r ? 1 : 0)) * bl.plane;
    size_t maxc = 0;
    for (int64_t b = 0; b < bl.nb; ++b) maxc = std::max<size_t>(maxc, offs[b + 1] - offs[b]);
    DevBuf cin[NS], dout[NS], stat;
    for (int i = 0; i < NS; ++i) {
        MGB_TRY(cin[i].alloc(maxc, ss.s[i]));
        MGB_TRY(dout[i].alloc(maxn * sizeof(T), ss.s[i]));
    }
    MGB_TRY(stat.alloc(NS * sizeof(unsigned), ss.s[0]));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, NS * sizeof(unsigned), ss.s[0]));
    MGB_CUDA(cudaEventRecord(ss.ev[0], ss.s[0]));
    MGB_CUDA(cudaStreamWaitEvent(ss.s[1], ss.ev[0], 0));
    ShapeWork<DecompressWork<T>> sw;
    std::vector<std::vector<double>> widths((size_t)bl.nb);
    for (int64_t b = 0; b < bl.nb; ++b) {
        const int i = (int)(b % NS);
        const char* blk = in + offs[b];
        const size_t nbytes = offs[b + 1] - offs[b];
        mgard_header h;
        if (nbytes < sizeof(h)) {
            set_error("corrupt out-of-core buffer: block size");
            return MGARD_ECORRUPT;
        }
        std::memcpy(&h, blk, sizeof(h));
        MGB_TRY(check_header(h, nbytes));
        int64_t bshape[4];
        block_shape(bl, ndim, hh.shape, b, bshape);
        if ((int)h.ndim != ndim || h.dtype != hh.dtype || h.mode != MGARD_ABS || !std::isinf(h.s)) {
            set_error("corrupt out-of-core buffer: block header");
            return MGARD_ECORRUPT;
        }
        for (int d = 0; d < ndim; ++d)
            if (h.shape[d] != bshape[d]) {
                set_error("corrupt out-of-core buffer: block shape");
                return MGARD_ECORRUPT;
            }
        widths[b].resize(h.nlevels + 1);
        std::memcpy(widths[b].data(), blk + h.off_widths, 8 * (h.nlevels + 1));
        if (!widths_valid(widths[b].data(), (int)h.nlevels)) {
            set_error("corrupt out-of-core buffer: bin width");
            return MGARD_ECORRUPT;
        }
        const Plan* p;
        MGB_TRY(get_plan(ndim, bshape, -1, &p));
        if (p->L != (int)h.nlevels) {
            set_error("corrupt out-of-core buffer: level count");
            return MGARD_ECORRUPT;
        }
        DecompressWork<T>* w;
        MGB_TRY(sw.get(p, i, ss.s[i], &w));
        MGB_CUDA(cudaMemcpyAsync(cin[i].p, blk, h.total_bytes, cudaMemcpyHostToDevice, ss.s[i]));
        MGB_TRY(decompress_core<T>(*p, h, widths[b].data(), cin[i].as<char>(), dout[i].as<T>(), *w,
                                   stat.as<unsigned>() + i, ss.s[i]));
        MGB_CUDA(cudaMemcpyAsync(field + bl.begin(b) * bl.plane, dout[i].p,
                                 bl.rows(b) * bl.plane * sizeof(T), cudaMemcpyDeviceToHost, ss.s[i]));
    }
    unsigned hs[NS];
    for (int i = 0; i < NS; ++i) MGB_CUDA(cudaStreamSynchronize(ss.s[i]));
    MGB_CUDA(cudaMemcpy(hs, stat.p, sizeof(hs), cudaMemcpyDeviceToHost));
    for (int i = 0; i < NS; ++i) MGB_TRY(status_to_error(hs[i]));
    return MGARD_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace mgb

using namespace mgb;

extern "C" size_t mgard_compress_ooc_bound(int ndim, const int64_t* shape, mgard_dtype dtype,
                                           int64_t nblocks) {
    Blocks bl;
    if (make_blocks(ndim, shape, nblocks, &bl) != MGARD_OK) return 0;
    size_t total = align16(sizeof(mgard_ooc_header) + 8 * (size_t)(nblocks + 1));
    for (int64_t b = 0; b < bl.nb; ++b) {
        int64_t bs[4];
        block_shape(bl, ndim, shape, b, bs);
        total += align16(mgard_compress_bound(ndim, bs, dtype));
    }
    return total;
}

extern "C" mgard_status mgard_compress_ooc(const void* field, int ndim, const int64_t* shape,
                                           mgard_dtype dtype, double tol, mgard_tolmode mode,
                                           int64_t nblocks, void** out, size_t* out_bytes,
                                           int out_preallocated, void* stream) {
    if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_EDTYPE;
    if (!field || !out || !out_bytes || (out_preallocated && !*out) || on_device(field) ||
        (out_preallocated && on_device(*out))) {
        set_error("out-of-core: host field and host output");
        return MGARD_EINVAL;
    }
    if (!(tol > 0.0) || !std::isfinite(tol) || (mode != MGARD_ABS && mode != MGARD_REL)) {
        set_error("out-of-core: tol must be positive and finite, mode ABS or REL");
        return MGARD_EINVAL;
    }
    Blocks bl;
    MGB_TRY(make_blocks(ndim, shape, nblocks, &bl));
    char* dst = (char*)*out;
    size_t cap = *out_bytes;
    if (!out_preallocated) {
        cap = mgard_compress_ooc_bound(ndim, shape, dtype, nblocks);
        dst = (char*)std::malloc(cap);
        if (!dst) {
            set_error("host output allocation failed");
            return MGARD_ENOMEM;
        }
    }
    size_t used = 0;
    cudaStream_t st = (cudaStream_t)stream;
    const mgard_status r =
        dtype == MGARD_F32
            ? compress_ooc_t<float>((const float*)field, dtype, ndim, shape, tol, mode, bl, dst, cap, &used, st)
            : compress_ooc_t<double>((const double*)field, dtype, ndim, shape, tol, mode, bl, dst, cap, &used, st);
    if (r != MGARD_OK) {
        if (!out_preallocated) std::free(dst);
        if (r == MGARD_ECAPACITY) *out_bytes = used;
        return r;
    }
    *out = dst;
    *out_bytes = used;
    return MGARD_OK;
}

namespace mgb {

// Host entry for mgard_decompress / mgard_info on an out-of-core buffer.
bool is_ooc_buffer(const void* in, size_t in_bytes) {
    return in && in_bytes >= 8 && std::memcmp(in, MGARD_OOC_MAGIC, 8) == 0;
}

mgard_status ooc_info(const void* in, size_t in_bytes, mgard_ooc_header* h) {
    std::vector<uint64_t> offs;
    Blocks bl;
    return read_ooc((const char*)in, in_bytes, h, &offs, &bl);
}

mgard_status decompress_ooc(const void* in, size_t in_bytes, void** field, int prealloc,
                            cudaStream_t st) {
    mgard_ooc_header h;
    std::vector<uint64_t> offs;
    Blocks bl;
    MGB_TRY(read_ooc((const char*)in, in_bytes, &h, &offs, &bl));
    int64_t n = 1;
    for (uint32_t d = 0; d < h.ndim; ++d) n *= h.shape[d];
    const size_t nbytes = (size_t)n * (h.dtype == MGARD_F64 ? 8 : 4);
    void* dst = prealloc ? *field : std::malloc(nbytes);
    if (!dst) {
        set_error(prealloc ? "preallocated output missing" : "host output allocation failed");
        return prealloc ? MGARD_EINVAL : MGARD_ENOMEM;
    }
    if (on_device(dst)) {
        set_error("out-of-core buffers decompress into host memory");
        return MGARD_EINVAL;
    }
    const mgard_status r =
        h.dtype == MGARD_F32
            ? decompress_ooc_t<float>((const char*)in, h, offs, bl, (float*)dst, st)
            : decompress_ooc_t<double>((const char*)in, h, offs, bl, (double*)dst, st);
    if (r != MGARD_OK) {
        if (!prealloc) std::free(dst);
        return r;
    }
    *field = dst;
    return MGARD_OK;
}

}  // namespace mgb
