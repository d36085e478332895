// Compression pipeline without host round trips (see pipeline.cuh).
//
// Paper, "Software design" and Listing 1: a relative tolerance is scaled by
// the norm of the data, the data is decomposed, every coefficient is
// quantized with its level's bin width and the symbols are Huffman-coded
// into a self-describing buffer.  Here every step is a launch on one
// stream; the norm, widths, sizes and header are produced by small device
// kernels (k_widths, k_finalize) instead of the host.
#include <cmath>
#include <cstring>

#include "huffman.cuh"
#include "pipeline.cuh"
#include "quantize.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

constexpr int MAXLV = 64;   // levels a header may record

struct WidthArgs {
    int L;
    int rel;                      // relative tolerance: scale by the norm of the data
    int snorm;                    // finite s: the norm comes from the level energies
    int finest;                   // s = 0: the level sums telescope to E_L alone
    double tol;
    double den[MAXLV + 1];        // width denominators of every level
    double f[MAXLV + 1];          // 4^(s l)
    long long eoff[MAXLV + 2];    // ranges of the energy partial sums of every level
};

// One warp: norm of the data (relative tolerances), tol_abs and the widths.
// Norm: max|u| (L-infinity), or sqrt(E_0 + sum_l 4^(s l) max(E_l - E_{l-1}, 0))
// with E_l = u_l^T M_l u_l (s-norm; for s = 0 the sum is E_L alone).  Sums and
// maxima run in a fixed order, and every lane ends with the same value.
__global__ void k_widths(WidthArgs a, const double* __restrict__ maxparts,
                         const double* __restrict__ eparts, CompressMeta* meta,
                         double* __restrict__ w) {
    const int lane = threadIdx.x;
    double nrm = 0.0;
    if (a.rel) {
        if (!a.snorm) {
            double m = 0.0;
            for (int i = lane; i < RED_PARTS; i += 32) m = fmax(m, maxparts[i]);
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            nrm = m;
        } else if (a.finest) {   // ||u||_0^2 = E_L (the L2 norm of the interpolant)
            double e = 0.0;
            for (long long i = a.eoff[a.L] + lane; i < a.eoff[a.L + 1]; i += 32) e += eparts[i];
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            nrm = sqrt(fmax(e, 0.0));
        } else {
            double total = 0.0, prev = 0.0;
            for (int l = 0; l <= a.L; ++l) {
                double e = 0.0;
                for (long long i = a.eoff[l] + lane; i < a.eoff[l + 1]; i += 32) e += eparts[i];
                for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
                if (l == 0) total = e;
                else total += a.f[l] * fmax(e - prev, 0.0);
                prev = e;
            }
            nrm = sqrt(fmax(total, 0.0));
        }
    }
    const double tol_abs = a.rel ? (nrm > 0.0 ? a.tol * nrm : a.tol) : a.tol;
    for (int l = lane; l <= a.L; l += 32) w[l] = 2.0 * tol_abs / a.den[l] * WIDTH_MARGIN;
    if (lane == 0) meta->tol_abs = tol_abs;
}

// Status bits of an encoding pass start clear (those of the input check stay).
__global__ void k_meta_reset(CompressMeta* meta) {
    if (threadIdx.x == 0) meta->status &= (unsigned)(ST_NONFINITE | ST_TIMEOUT);
}

// Sizes and offsets that follow from the totals of the count pass; the
// header goes to the front of the buffer.
__global__ void k_finalize(mgard_header h, const unsigned long long* __restrict__ totals,
                           CompressMeta* meta, unsigned char* dd, unsigned long long cap) {
    if (threadIdx.x != 0) return;
    const unsigned long long nwords = totals[0], nout = totals[1];
    const unsigned long long off_words = (h.off_outliers + 4 * nout + 15) & ~15ull;
    const unsigned long long total = (off_words + 4 * nwords + 15) & ~15ull;
    h.tol_abs = meta->tol_abs;
    h.nwords = nwords;
    h.noutliers = nout;
    h.off_words = off_words;
    h.total_bytes = total;
    meta->nwords = nwords;
    meta->noutliers = nout;
    meta->off_words = off_words;
    meta->total = total;
    if (!dd) return;   // size only
    if (total > cap) {
        atomicOr(&meta->status, (unsigned)ST_CAPACITY);
    } else {
        // alignment gaps after the outliers and after the payload hold zeros,
        // so the whole buffer is a function of the input
        for (unsigned long long i = h.off_outliers + 4 * nout; i < off_words; ++i) dd[i] = 0;
        for (unsigned long long i = off_words + 4 * nwords; i < total; ++i) dd[i] = 0;
    }
    const unsigned char* src = reinterpret_cast<const unsigned char*>(&h);
    for (size_t i = 0; i < sizeof(h); ++i) dd[i] = src[i];
}

}  // namespace

Sections layout(int L, uint64_t nchunks, uint64_t nout, uint64_t nwords) {
    Sections s;
    size_t o = align16(sizeof(mgard_header));
    s.widths = o;
    o = align16(o + 8 * (size_t)(L + 1));
    s.lengths = o;
    o = align16(o + DICT);
    s.word_off = o;
    o = align16(o + 8 * nchunks);
    s.esc_off = o;
    o = align16(o + 8 * nchunks);
    s.sub_off = o;
    o = align16(o + 2 * SUBREC * nchunks);
    s.outliers = o;
    o = align16(o + 4 * nout);
    s.words = o;
    o = align16(o + 4 * nwords);
    s.total = o;
    return s;
}

template <typename T>
mgard_status CompressWork<T>::alloc(const Plan& p, cudaStream_t st) {
    const int64_t N = p.total();
    const uint64_t nchunks = ((uint64_t)N + CHUNK - 1) / CHUNK;
    MGB_TRY(py.alloc(p, st));
    MGB_TRY(top.alloc(N * sizeof(T), st));
    MGB_TRY(sym.alloc(N * sizeof(uint16_t), st));
    MGB_TRY(esc.alloc(N * sizeof(int32_t), st));
    MGB_TRY(hist.alloc(DICT * sizeof(unsigned long long), st));
    MGB_TRY(lengths.alloc(DICT, st));
    MGB_TRY(codes.alloc(DICT * sizeof(uint32_t), st));
    MGB_TRY(dt.alloc(sizeof(DecodeTables), st));
    MGB_TRY(offs.alloc(16 * nchunks + 16, st));
    MGB_TRY(totals.alloc(2 * sizeof(unsigned long long), st));
    MGB_TRY(parts.alloc((RED_PARTS + energy_parts_total(p)) * sizeof(double), st));
    MGB_TRY(scan.alloc(count_scratch_bytes((uint64_t)N), st));
    MGB_TRY(wdev.alloc(8 * (p.L + 1), st));
    return MGARD_OK;
}

mgard_header header_template(const Plan& p, mgard_dtype dtype, int ndim, const int64_t* shape,
                             double tol, double s, mgard_tolmode mode) {
    const uint64_t N = (uint64_t)p.total();
    const uint64_t nchunks = (N + CHUNK - 1) / CHUNK;
    const Sections fx = layout(p.L, nchunks, 0, 0);
    mgard_header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, MGARD_MAGIC, 8);
    h.version = MGARD_FORMAT_VERSION;
    h.dtype = (uint32_t)dtype;
    h.ndim = (uint32_t)ndim;
    h.nlevels = (uint32_t)p.L;
    for (int i = 0; i < 4; ++i) h.shape[i] = i < ndim ? shape[i] : 1;
    h.s = s;
    h.tol = tol;
    h.mode = (uint32_t)mode;
    h.dict = DICT;
    h.chunk = CHUNK;
    h.nsymbols = N;
    h.nchunks = nchunks;
    h.off_widths = fx.widths;
    h.off_lengths = fx.lengths;
    h.off_word_off = fx.word_off;
    h.off_esc_off = fx.esc_off;
    h.off_sub_off = fx.sub_off;
    h.off_outliers = fx.outliers;
    return h;
}

template <typename T>
mgard_status compress_decompose(const Plan& p, const T* din, double s, mgard_tolmode mode,
                                CompressWork<T>& w, CompressMeta* meta, cudaStream_t st) {
    const int64_t N = p.total();
    if (p.L > MAXLV) {
        set_error("too many levels");
        return MGARD_ESHAPE;
    }
    MGB_CUDA(cudaMemsetAsync(meta, 0, sizeof(CompressMeta), st));
    double* parts = w.parts.template as<double>();
    MGB_TRY(max_abs_partials<T>(din, N, parts, &meta->status, st));
    const bool energy = mode == MGARD_REL && !std::isinf(s);
    // s = 0: sum_l (E_l - E_{l-1}) telescopes to E_L = u^T M_L u, the energy
    // of the input itself; other s need every level's energy
    const bool finest = energy && s == 0.0;
    if (finest)
        MGB_TRY(mass_norm2_partials<T>(p, p.L, din, parts + RED_PARTS + energy_parts_offset(p, p.L), st));
    // shapes on the row kernels keep every level's coefficients in symbol
    // order in `top` (quantization then streams through it)
    T* top = w.top.template as<T>();
    w.py.status = &meta->status;
    MGB_TRY(decompose_pyramid<T>(p, din, top, w.py, st, nullptr,
                                 energy && !finest ? parts + RED_PARTS : nullptr,
                                 rows3_ok(p) ? top : nullptr));
    return MGARD_OK;
}

template <typename T>
mgard_status compress_encode_front(const Plan& p, const T* din, double tol, double s,
                                   mgard_tolmode mode, CompressWork<T>& w, CompressMeta* meta,
                                   cudaStream_t st, bool quantize) {
    const int L = p.L;
    MGB_LAUNCH("k_meta_reset", st, k_meta_reset<<<1, 32, 0, st>>>(meta));
    MGB_CUDA(cudaMemsetAsync(w.hist.p, 0, DICT * sizeof(unsigned long long), st));
    unsigned* status = &meta->status;
    double* parts = w.parts.template as<double>();
    const bool energy = mode == MGARD_REL && !std::isinf(s);
    WidthArgs a;
    std::memset(&a, 0, sizeof(a));
    a.L = L;
    a.rel = mode == MGARD_REL;
    a.snorm = energy;
    a.finest = energy && s == 0.0;
    a.tol = tol;
    width_denominators(p, s, a.den);
    for (int l = 0; l <= L; ++l) {
        a.f[l] = energy ? std::pow(4.0, s * (double)l) : 1.0;
        a.eoff[l] = energy_parts_offset(p, l);
    }
    a.eoff[L + 1] = energy_parts_total(p);
    double* widths = w.wdev.template as<double>();
    MGB_LAUNCH("k_widths", st, k_widths<<<1, 32, 0, st>>>(a, parts, parts + RED_PARTS, meta, widths));
    MGB_CUDA(cudaGetLastError());
    if (!quantize) return MGARD_OK;
    uint16_t* sym = w.sym.template as<uint16_t>();
    int32_t* esc = w.esc.template as<int32_t>();
    if (rows3_ok(p)) {
        MGB_TRY(quantize_stream<T>(p, w.top.template as<T>(), widths, sym, esc,
                                   w.hist.template as<unsigned long long>(), status, st));
    } else {
        for (int l = 0; l <= L; ++l) {
            const T* lvl = l == L ? (L ? w.top.template as<T>() : din) : w.py.lv[l];
            MGB_TRY(quantize_level<T>(p, l, lvl, false, widths + l, sym, esc,
                                      w.hist.template as<unsigned long long>(), status, st));
        }
    }
    return MGARD_OK;
}

template <typename T>
CodebookJob codebook_job(const Plan& p, CompressWork<T>& w) {
    CodebookJob j;
    j.hist = w.hist.template as<unsigned long long>();
    j.lengths = w.lengths.template as<uint8_t>();
    j.codes = w.codes.template as<uint32_t>();
    j.dt = w.dt.template as<DecodeTables>();
    j.wide = (uint64_t)p.total() >= (uint64_t(1) << 32) ? 1 : 0;
    return j;
}

template <typename T>
mgard_status compress_encode_back(const Plan& p, const mgard_header& h0, char* dd, uint64_t cap,
                                  CompressWork<T>& w, CompressMeta* meta, cudaStream_t st) {
    const int64_t N = p.total();
    const uint64_t nchunks = ((uint64_t)N + CHUNK - 1) / CHUNK;
    uint64_t* word_off = w.offs.template as<uint64_t>();
    uint64_t* esc_off = word_off + nchunks;
    MGB_TRY(huffman_count(w.sym.template as<uint16_t>(), N, w.lengths.template as<uint8_t>(), word_off,
                          esc_off, w.totals.template as<unsigned long long>(), &meta->status, st,
                          w.scan.template as<unsigned long long>()));
    MGB_LAUNCH("k_finalize", st, k_finalize<<<1, 32, 0, st>>>(
        h0, w.totals.template as<unsigned long long>(), meta, reinterpret_cast<unsigned char*>(dd), cap));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status compress_encode(const Plan& p, const T* din, const mgard_header& h0, double tol,
                             double s, mgard_tolmode mode, char* dd, uint64_t cap,
                             CompressWork<T>& w, CompressMeta* meta, cudaStream_t st) {
    MGB_TRY(compress_encode_front<T>(p, din, tol, s, mode, w, meta, st));
    const CodebookJob j = codebook_job<T>(p, w);
    MGB_TRY(huffman_codebook(j.hist, j.lengths, nullptr, st, j.wide != 0));
    MGB_TRY(huffman_tables(j.lengths, j.codes, nullptr, st));   // the encoder needs the codes only
    return compress_encode_back<T>(p, h0, dd, cap, w, meta, st);
}

template <typename T>
mgard_status compress_pack(const Plan& p, char* dd, CompressWork<T>& w, CompressMeta* meta,
                           cudaStream_t st) {
    const int64_t N = p.total();
    const uint64_t nchunks = ((uint64_t)N + CHUNK - 1) / CHUNK;
    const Sections fx = layout(p.L, nchunks, 0, 0);
    uint64_t* word_off = w.offs.template as<uint64_t>();
    uint64_t* esc_off = word_off + nchunks;
    MGB_CUDA(cudaMemcpyAsync(dd + fx.widths, w.wdev.p, 8 * (p.L + 1), cudaMemcpyDeviceToDevice, st));
    MGB_CUDA(cudaMemcpyAsync(dd + fx.lengths, w.lengths.p, DICT, cudaMemcpyDeviceToDevice, st));
    if (nchunks) {
        MGB_CUDA(cudaMemcpyAsync(dd + fx.word_off, word_off, 8 * nchunks, cudaMemcpyDeviceToDevice, st));
        MGB_CUDA(cudaMemcpyAsync(dd + fx.esc_off, esc_off, 8 * nchunks, cudaMemcpyDeviceToDevice, st));
    }
    PackGuard guard;
    guard.status = &meta->status;
    guard.words_byte_off = &meta->off_words;
    MGB_TRY(huffman_pack(w.sym.template as<uint16_t>(), N, w.lengths.template as<uint8_t>(),
                         w.codes.template as<uint32_t>(), word_off, esc_off, w.esc.template as<int32_t>(),
                         reinterpret_cast<uint32_t*>(dd), reinterpret_cast<uint16_t*>(dd + fx.sub_off),
                         reinterpret_cast<int32_t*>(dd + fx.outliers), st, guard,
                         rows3_ok(p)));   // the streaming quantizer compacts escapes per chunk
    return MGARD_OK;
}

template <typename T>
mgard_status compress_core(const Plan& p, const T* din, const mgard_header& h0, double tol,
                           double s, mgard_tolmode mode, char* dd, uint64_t cap,
                           CompressWork<T>& w, CompressMeta* meta, cudaStream_t st,
                           const RegionScale* rs, const AuxLane* aux) {
    const uint64_t N = (uint64_t)p.total();
    const Sections fx = layout(p.L, (N + CHUNK - 1) / CHUNK, 0, 0);
    if (cap < fx.outliers || ((uintptr_t)dd & 15) != 0) {
        set_error("compress_core: output buffer too small or misaligned");
        return MGARD_EINVAL;
    }
    MGB_CUDA(cudaMemsetAsync(dd, 0, fx.outliers, st));   // fixed sections, gaps included
    // the tail beside the larger levels' quantization: the decomposition
    // stops before the tail (it does so only where no level energies are
    // needed: tail_pending says whether it did)
    const int Lt = rows3_ok(p) ? tail_levels(p) : 0;
    const bool beside = aux && aux->stream && !rs && Lt >= 1 && Lt < p.L;
    w.py.defer_tail = beside;
    const mgard_status dr = compress_decompose<T>(p, din, s, mode, w, meta, st);
    w.py.defer_tail = false;
    MGB_TRY(dr);
    if (w.py.tail_pending) {
        T* top = w.top.template as<T>();
        uint16_t* sym = w.sym.template as<uint16_t>();
        int32_t* esc = w.esc.template as<int32_t>();
        unsigned long long* hist = w.hist.template as<unsigned long long>();
        const double* widths = w.wdev.template as<double>();
        // symbols [0, S) hold the tail's levels (and the start of the next
        // level, already final); S on a sub-chunk boundary
        const int64_t S = std::min<int64_t>((int64_t)N, (p.offset[Lt + 1] + SUB - 1) / SUB * SUB);
        MGB_CUDA(cudaEventRecord(aux->fork, st));
        MGB_CUDA(cudaStreamWaitEvent(aux->stream, aux->fork, 0));
        MGB_TRY(tail_decompose<T>(p, Lt, w.py, w.py.lv[Lt], top, top, aux->stream));
        MGB_TRY(decompose_finish<T>(p, w.py, top, aux->stream));
        MGB_TRY(compress_encode_front<T>(p, din, tol, s, mode, w, meta, st, false));   // widths
        MGB_CUDA(cudaEventRecord(aux->mid, st));
        MGB_TRY(quantize_stream<T>(p, top, widths, sym, esc, hist, &meta->status, st, S, -1, true));
        MGB_CUDA(cudaStreamWaitEvent(aux->stream, aux->mid, 0));
        MGB_TRY(quantize_stream<T>(p, top, widths, sym, esc, hist, &meta->status, aux->stream, 0, S));
        MGB_CUDA(cudaEventRecord(aux->join, aux->stream));
        MGB_CUDA(cudaStreamWaitEvent(st, aux->join, 0));
        const CodebookJob j = codebook_job<T>(p, w);
        MGB_TRY(huffman_codebook(j.hist, j.lengths, nullptr, st, j.wide != 0));
        MGB_TRY(huffman_tables(j.lengths, j.codes, nullptr, st));
        MGB_TRY(compress_encode_back<T>(p, h0, dd, cap, w, meta, st));
        return compress_pack<T>(p, dd, w, meta, st);
    }
    if (rs) {   // region-adaptive widths: coefficients scaled by 2^k of their node
        if (p.L < 1) {
            set_error("regions need at least one level");
            return MGARD_ESHAPE;
        }
        std::vector<T*> lv(p.L + 1);
        for (int l = 0; l < p.L; ++l) lv[l] = w.py.lv[l];
        lv[p.L] = w.top.template as<T>();
        MGB_TRY(region_scale<T>(p, *rs, rows3_ok(p) ? w.top.template as<T>() : nullptr, lv.data(), 1, st));
    }
    MGB_TRY(compress_encode<T>(p, din, h0, tol, s, mode, dd, cap, w, meta, st));
    return compress_pack<T>(p, dd, w, meta, st);
}

mgard_status check_header(const mgard_header& h, size_t in_bytes) {
    auto bad = [](const char* why) {
        set_error(std::string("corrupt header: ") + why);
        return MGARD_ECORRUPT;
    };
    if (std::memcmp(h.magic, MGARD_MAGIC, 8) != 0) return bad("magic");
    if (h.version != MGARD_FORMAT_VERSION) return bad("version");
    if (h.dtype > 1) return bad("dtype");
    if (h.ndim < 1 || h.ndim > 4) return bad("ndim");
    if (h.dict != DICT || h.chunk != CHUNK) return bad("dictionary or chunk size");
    uint64_t n = 1;
    for (uint32_t i = 0; i < h.ndim; ++i) {
        if (h.shape[i] < 1 || h.shape[i] > (int64_t(1) << 40)) return bad("shape");
        n *= (uint64_t)h.shape[i];
        if (n > (uint64_t(1) << 40)) return bad("shape");
    }
    if (n != h.nsymbols) return bad("symbol count");
    if (h.nchunks != (n + CHUNK - 1) / CHUNK) return bad("chunk count");
    if (h.nlevels > 64) return bad("levels");
    if (h.noutliers > n || h.nwords > n + h.nchunks) return bad("section sizes");
    Sections s = layout((int)h.nlevels, h.nchunks, h.noutliers, h.nwords);
    if (h.off_widths != s.widths || h.off_lengths != s.lengths || h.off_word_off != s.word_off ||
        h.off_esc_off != s.esc_off || h.off_sub_off != s.sub_off ||
        h.off_outliers != s.outliers || h.off_words != s.words ||
        h.total_bytes != s.total)
        return bad("section offsets");
    if (s.total > in_bytes) return bad("truncated buffer");
    if (!(h.tol_abs > 0.0) || !std::isfinite(h.tol_abs)) return bad("tolerance");
    return MGARD_OK;
}

bool widths_valid(const double* w, int L) {
    for (int l = 0; l <= L; ++l)
        if (!(w[l] > 0.0) || !std::isfinite(w[l])) return false;
    return true;
}

template <typename T>
mgard_status DecompressWork<T>::alloc(const Plan& p, cudaStream_t st) {
    const int64_t N = p.total();
    MGB_TRY(py.alloc(p, st));
    MGB_TRY(codes.alloc(DICT * sizeof(uint32_t), st));
    MGB_TRY(dt.alloc(sizeof(DecodeTables), st));
    MGB_TRY(grab.alloc(sizeof(unsigned long long), st));
    if (rows3_ok(p)) {   // decoded straight to coefficients in symbol order
        MGB_TRY(zs.alloc(N * sizeof(T), st));
    } else {
        MGB_TRY(sym.alloc(N * sizeof(uint16_t), st));
        MGB_TRY(esc.alloc(N * sizeof(int32_t), st));
    }
    return MGARD_OK;
}

template <typename T>
mgard_status decompress_core(const Plan& p, const mgard_header& h, const double* w,
                             const char* din, T* dout, DecompressWork<T>& work, unsigned* status,
                             cudaStream_t st, const RegionScale* rs) {
    work.py.status = status;
    const int64_t N = p.total();
    const int L = p.L;
    DecodeTables* dt = work.dt.template as<DecodeTables>();
    MGB_TRY(huffman_tables((const uint8_t*)(din + h.off_lengths), work.codes.template as<uint32_t>(),
                           dt, st));
    const uint32_t* words = (const uint32_t*)(din + h.off_words);
    const uint64_t* woff = (const uint64_t*)(din + h.off_word_off);
    const uint16_t* soff = (const uint16_t*)(din + h.off_sub_off);
    const int32_t* outl = (const int32_t*)(din + h.off_outliers);
    const uint64_t* eoff = (const uint64_t*)(din + h.off_esc_off);
    if (rows3_ok(p)) {
        // decode straight to coefficients in symbol order, recompose from there
        if (L > MAX_LEVELS) {
            set_error("too many levels");
            return MGARD_ECORRUPT;
        }
        DeqArgs dq;
        std::memset(&dq, 0, sizeof(dq));
        dq.lo = level_offsets(p);
        for (int l = 0; l <= L; ++l) {
            dq.w[l] = w[l];
            dq.wf[l] = (float)w[l];
            dq.ws[l] = split_width(w[l]);
        }
        T* zs = work.zs.template as<T>();
        MGB_TRY(huffman_decode_values<T>(words, h.nwords, woff, soff, dt, N, outl, h.noutliers, eoff,
                                         dq, zs, status, st,
                                         work.grab.template as<unsigned long long>()));
        if (rs) MGB_TRY(region_scale<T>(p, *rs, zs, nullptr, -1, st));
        return recompose_pyramid<T>(p, nullptr, dout, work.py, st, zs);
    }
    uint16_t* sym = work.sym.template as<uint16_t>();
    int32_t* esc = work.esc.template as<int32_t>();
    MGB_TRY(huffman_decode(words, h.nwords, woff, soff, dt, N, outl, h.noutliers, eoff, sym, esc,
                           status, st));
    std::vector<T*> lv(L + 1);
    for (int l = 0; l <= L; ++l) {
        lv[l] = l == L ? dout : work.py.lv[l];
        MGB_TRY(dequantize_level<T>(p, l, sym, esc, false, w[l], lv[l], st));
    }
    if (rs) MGB_TRY(region_scale<T>(p, *rs, nullptr, lv.data(), -1, st));
    MGB_TRY(recompose_pyramid<T>(p, dout, dout, work.py, st));
    return MGARD_OK;
}

template struct CompressWork<float>;
template struct CompressWork<double>;
#define INST_PHASES(T)                                                                            \
    template mgard_status compress_decompose<T>(const Plan&, const T*, double, mgard_tolmode,     \
                                                CompressWork<T>&, CompressMeta*, cudaStream_t);   \
    template mgard_status compress_encode<T>(const Plan&, const T*, const mgard_header&, double,  \
                                             double, mgard_tolmode, char*, uint64_t,              \
                                             CompressWork<T>&, CompressMeta*, cudaStream_t);      \
    template mgard_status compress_pack<T>(const Plan&, char*, CompressWork<T>&, CompressMeta*,   \
                                           cudaStream_t);                                         \
    template mgard_status compress_encode_front<T>(const Plan&, const T*, double, double,         \
                                                   mgard_tolmode, CompressWork<T>&, CompressMeta*, \
                                                   cudaStream_t, bool);                           \
    template CodebookJob codebook_job<T>(const Plan&, CompressWork<T>&);                          \
    template mgard_status compress_encode_back<T>(const Plan&, const mgard_header&, char*,        \
                                                  uint64_t, CompressWork<T>&, CompressMeta*,      \
                                                  cudaStream_t);
INST_PHASES(float)
INST_PHASES(double)
#undef INST_PHASES
template mgard_status compress_core<float>(const Plan&, const float*, const mgard_header&, double,
                                           double, mgard_tolmode, char*, uint64_t,
                                           CompressWork<float>&, CompressMeta*, cudaStream_t,
                                           const RegionScale*, const AuxLane*);
template struct DecompressWork<float>;
template struct DecompressWork<double>;
template mgard_status decompress_core<float>(const Plan&, const mgard_header&, const double*,
                                             const char*, float*, DecompressWork<float>&,
                                             unsigned*, cudaStream_t, const RegionScale*);
template mgard_status decompress_core<double>(const Plan&, const mgard_header&, const double*,
                                              const char*, double*, DecompressWork<double>&,
                                              unsigned*, cudaStream_t, const RegionScale*);
template mgard_status compress_core<double>(const Plan&, const double*, const mgard_header&, double,
                                            double, mgard_tolmode, char*, uint64_t,
                                            CompressWork<double>&, CompressMeta*, cudaStream_t,
                                            const RegionScale*, const AuxLane*);

}  // namespace mgb
