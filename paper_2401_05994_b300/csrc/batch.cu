// Batched compression of many fields (mgard_compress_batch).
//
// Each field runs the stream-ordered pipeline of pipeline.cu on one of a few
// internal streams forked from the caller's stream, so the small launches of
// one field's coarse levels overlap with the work of the others.  With
// MGARD_BATCH_GRAPH the fork, every field's launches and the join are
// captured once into a CUDA graph and replayed: the host then issues one
// graph launch per batch instead of thousands of kernel launches.  The
// graph bakes in pointers, so a captured batch is kept (with its
// workspaces) under a key of every argument and reused only for identical
// calls.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "huffman.cuh"
#include "pipeline.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

constexpr int BATCH_STREAMS = 32;
constexpr size_t BATCH_CACHE = 4;

struct BatchKey {
    int device = -1;
    int n = 0;
    int dtype = 0, mode = 0, flags = 0;
    double tol = 0, s = 0;
    cudaStream_t stream = nullptr;
    std::vector<int64_t> shapes;   // ndim followed by the extents, per field
    std::vector<const void*> fields;
    std::vector<void*> outs;
    std::vector<size_t> caps;
    bool operator==(const BatchKey& o) const {
        return device == o.device && n == o.n && dtype == o.dtype && mode == o.mode &&
               flags == o.flags && std::memcmp(&tol, &o.tol, sizeof tol) == 0 &&
               std::memcmp(&s, &o.s, sizeof s) == 0 && stream == o.stream &&
               shapes == o.shapes && fields == o.fields && outs == o.outs && caps == o.caps;
    }
};

// Internal streams of a batch: work forks from the caller's stream onto
// `side`, joins back, and graph capture happens on `origin` (the caller's
// stream may be the legacy default stream, which cannot capture).
struct Lanes {
    cudaStream_t side[BATCH_STREAMS] = {};
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, join[BATCH_STREAMS] = {};
    cudaEvent_t aux_ev[3] = {};   // fork, mid, join of a field's second stream (AuxLane)
    cudaGraphExec_t exec = nullptr;
    int runs = 0;   // calls served so far

    mgard_status init() {
        for (int s = 0; s < BATCH_STREAMS; ++s) {
            MGB_CUDA(cudaStreamCreateWithFlags(&side[s], cudaStreamNonBlocking));
            MGB_CUDA(cudaEventCreateWithFlags(&join[s], cudaEventDisableTiming));
        }
        MGB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        for (int k = 0; k < 3; ++k) MGB_CUDA(cudaEventCreateWithFlags(&aux_ev[k], cudaEventDisableTiming));
        MGB_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
        return MGARD_OK;
    }
    // A one-field run uses side[0] only: side[1] is the field's second stream.
    AuxLane aux() const {
        AuxLane a;
        a.stream = side[1];
        a.fork = aux_ev[0];
        a.mid = aux_ev[1];
        a.join = aux_ev[2];
        return a;
    }
    void destroy() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        for (int k = 0; k < BATCH_STREAMS; ++k) {
            if (join[k]) cudaEventDestroy(join[k]);
            if (side[k]) cudaStreamDestroy(side[k]);
            join[k] = nullptr;
            side[k] = nullptr;
        }
        if (fork) cudaEventDestroy(fork);
        for (int k = 0; k < 3; ++k) {
            if (aux_ev[k]) cudaEventDestroy(aux_ev[k]);
            aux_ev[k] = nullptr;
        }
        if (origin) cudaStreamDestroy(origin);
        fork = nullptr;
        origin = nullptr;
        cudaGetLastError();
    }
    // Fork from st, run body(i, stream) for every item on the side streams
    // (round robin), join back into st.
    template <typename F>
    mgard_status run(cudaStream_t st, int n, F&& body) {
        const int nside = std::min(BATCH_STREAMS, std::max(n, 1));
        MGB_CUDA(cudaEventRecord(fork, st));
        for (int s = 0; s < nside; ++s) MGB_CUDA(cudaStreamWaitEvent(side[s], fork, 0));
        for (int i = 0; i < n; ++i) MGB_TRY(body(i, side[i % nside]));
        for (int s = 0; s < nside; ++s) {
            MGB_CUDA(cudaEventRecord(join[s], side[s]));
            MGB_CUDA(cudaStreamWaitEvent(st, join[s], 0));
        }
        return MGARD_OK;
    }
    // Run through a graph captured on the first call.
    template <typename F>
    mgard_status run_graph(cudaStream_t st, int n, F&& body) {
        return run_graph_seq(st, [&](cudaStream_t s) { return run(s, n, body); });
    }
    // The same for any sequence of launches on one stream (whole(stream)).
    template <typename F>
    mgard_status run_graph_seq(cudaStream_t st, F&& whole) {
        if (!exec) {
            MGB_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
            const mgard_status e = whole(origin);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(origin, &g);
            if (e != MGARD_OK) {
                if (g) cudaGraphDestroy(g);
                return e;
            }
            MGB_CUDA(ce);
            const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            MGB_CUDA(ie);
        }
        MGB_CUDA(cudaGraphLaunch(exec, st));
        return MGARD_OK;
    }
};

struct BatchState {
    BatchKey key;
    std::vector<const Plan*> plans;
    std::vector<mgard_header> heads;
    std::vector<std::unique_ptr<CompressWork<float>>> wf;
    std::vector<std::unique_ptr<CompressWork<double>>> wd;
    CompressMeta* metas = nullptr;      // device, one per field
    CompressMeta* hmetas = nullptr;     // pinned host copy
    CodebookJob* jobs = nullptr;        // device, one per field (persistent codebook phase)
    unsigned* job_counter = nullptr;    // device
    // persistent tail phase: the fields whose small levels wait for one
    // batched launch, and that launch's job list (device) and shared memory
    std::vector<char> tail_deferred;
    void* tail_jobs = nullptr;
    int ntail = 0;
    size_t tail_smem = 0;
    unsigned* tail_counter = nullptr;
    Lanes lanes;

    ~BatchState() {
        // workspaces free themselves on side[0]; wait for that before the
        // stream goes away
        wf.clear();
        wd.clear();
        if (metas) cudaFreeAsync(metas, lanes.side[0]);
        if (jobs) cudaFreeAsync(jobs, lanes.side[0]);
        if (job_counter) cudaFreeAsync(job_counter, lanes.side[0]);
        if (tail_jobs) cudaFreeAsync(tail_jobs, lanes.side[0]);
        if (tail_counter) cudaFreeAsync(tail_counter, lanes.side[0]);
        if (lanes.side[0]) cudaStreamSynchronize(lanes.side[0]);
        lanes.destroy();
        if (hmetas) cudaFreeHost(hmetas);
        cudaGetLastError();
    }

    template <typename T>
    CompressWork<T>& work(int i);

    mgard_status init(const BatchKey& k, const int* ndims, const int64_t* const* shapes) {
        key = k;
        MGB_TRY(lanes.init());
        cudaStream_t s0 = lanes.side[0];
        count_device_alloc();
        MGB_CUDA(cudaMallocHost(&hmetas, sizeof(CompressMeta) * k.n));
        count_device_alloc();
        MGB_CUDA(cudaMallocAsync((void**)&metas, sizeof(CompressMeta) * k.n, s0));
        for (int i = 0; i < k.n; ++i) {
            const Plan* p;
            MGB_TRY(get_plan(ndims[i], shapes[i], -1, &p));
            plans.push_back(p);
            heads.push_back(header_template(*p, (mgard_dtype)k.dtype, ndims[i], shapes[i], k.tol,
                                            k.s, (mgard_tolmode)k.mode));
            if (k.dtype == MGARD_F32) {
                wf.emplace_back(new CompressWork<float>());
                MGB_TRY(wf.back()->alloc(*p, s0));
            } else {
                wd.emplace_back(new CompressWork<double>());
                MGB_TRY(wd.back()->alloc(*p, s0));
            }
        }
        if (k.flags & MGARD_BATCH_PERSISTENT) {
            std::vector<CodebookJob> hj;
            for (int i = 0; i < k.n; ++i)
                hj.push_back(k.dtype == MGARD_F32 ? codebook_job<float>(*plans[i], *wf[i])
                                                  : codebook_job<double>(*plans[i], *wd[i]));
            count_device_alloc();
            MGB_CUDA(cudaMallocAsync((void**)&jobs, sizeof(CodebookJob) * k.n, s0));
            count_device_alloc();
            MGB_CUDA(cudaMallocAsync((void**)&job_counter, sizeof(unsigned), s0));
            MGB_CUDA(cudaMemcpyAsync(jobs, hj.data(), sizeof(CodebookJob) * k.n, cudaMemcpyHostToDevice, s0));
            MGB_TRY(k.dtype == MGARD_F32 ? tail_jobs_t<float>(k, s0) : tail_jobs_t<double>(k, s0));
        }
        MGB_TRY(huffman_prepare());
        MGB_CUDA(cudaStreamSynchronize(s0));
        if (k.flags & MGARD_BATCH_AUTOTUNE) {   // each distinct shape once, before any capture
            std::vector<const Plan*> done;
            for (const Plan* p : plans) {
                if (std::find(done.begin(), done.end(), p) != done.end()) continue;
                done.push_back(p);
                MGB_TRY(autotune_plan(*p, (mgard_dtype)k.dtype, s0, nullptr));
            }
        }
        return MGARD_OK;
    }

    mgard_status field(int i, cudaStream_t ss) {
        char* dd = (char*)key.outs[i];
        const uint64_t cap = key.caps[i];
        // a single field runs its small levels beside its quantization
        const AuxLane a = lanes.aux();
        const AuxLane* ap = key.n == 1 ? &a : nullptr;
        if (key.dtype == MGARD_F32)
            return compress_core<float>(*plans[i], (const float*)key.fields[i], heads[i], key.tol,
                                        key.s, (mgard_tolmode)key.mode, dd, cap, *wf[i], metas + i, ss,
                                        nullptr, ap);
        return compress_core<double>(*plans[i], (const double*)key.fields[i], heads[i], key.tol,
                                     key.s, (mgard_tolmode)key.mode, dd, cap, *wd[i], metas + i, ss,
                                     nullptr, ap);
    }

    // The persistent form: every field's decomposition down to its
    // one-block tail (front_a); one launch for all those tails; every field's
    // level 0, widths and quantization (front_b); one launch for all
    // codebooks and tables; then every field's count pass, header and
    // payload (back).  Fields whose decomposition needs level energies
    // (finite s > 0, relative) run their tail in front_a.
    template <typename T>
    mgard_status tail_jobs_t(const BatchKey& k, cudaStream_t s0) {
        const size_t bytes = tail_args_bytes<T>();
        std::vector<char> host;
        tail_deferred.assign(k.n, 0);
        const bool energies = k.mode == MGARD_REL && !std::isinf(k.s) && k.s != 0.0;
        for (int i = 0; i < k.n; ++i) {
            const Plan& p = *plans[i];
            const int Lt = rows3_ok(p) ? tail_levels(p) : 0;
            if (!Lt || energies) continue;
            CompressWork<T>& w = work<T>(i);
            const T* level_Lt = Lt == p.L ? (const T*)k.fields[i] : w.py.lv[Lt];
            host.resize(host.size() + bytes);
            size_t smem = 0;
            MGB_TRY(tail_job<T>(p, Lt, w.py, level_Lt, w.top.template as<T>(), w.top.template as<T>(),
                                host.data() + host.size() - bytes, &smem));
            tail_smem = std::max(tail_smem, smem);
            tail_deferred[i] = 1;
            ++ntail;
        }
        if (!ntail) return MGARD_OK;
        count_device_alloc();
        MGB_CUDA(cudaMallocAsync(&tail_jobs, host.size(), s0));
        count_device_alloc();
        MGB_CUDA(cudaMallocAsync((void**)&tail_counter, sizeof(unsigned), s0));
        MGB_CUDA(cudaMemcpyAsync(tail_jobs, host.data(), host.size(), cudaMemcpyHostToDevice, s0));
        return MGARD_OK;
    }
    template <typename T>
    mgard_status front_a_t(int i, cudaStream_t ss, CompressWork<T>& w) {
        const Plan& p = *plans[i];
        const uint64_t N = (uint64_t)p.total();
        const Sections fx = layout(p.L, (N + CHUNK - 1) / CHUNK, 0, 0);
        MGB_CUDA(cudaMemsetAsync(key.outs[i], 0, fx.outliers, ss));
        w.py.defer_tail = tail_deferred[i] != 0;
        const mgard_status r = compress_decompose<T>(p, (const T*)key.fields[i], key.s,
                                                     (mgard_tolmode)key.mode, w, metas + i, ss);
        w.py.defer_tail = false;
        if (r == MGARD_OK && (w.py.tail_pending != (tail_deferred[i] != 0))) {
            set_error("batched tail: the decomposition did not stop where planned");
            return MGARD_EINVAL;
        }
        return r;
    }
    template <typename T>
    mgard_status front_b_t(int i, cudaStream_t ss, CompressWork<T>& w) {
        const Plan& p = *plans[i];
        if (tail_deferred[i]) MGB_TRY(decompose_finish<T>(p, w.py, w.top.template as<T>(), ss));
        return compress_encode_front<T>(p, (const T*)key.fields[i], key.tol, key.s,
                                        (mgard_tolmode)key.mode, w, metas + i, ss);
    }
    template <typename T>
    mgard_status back_t(int i, cudaStream_t ss, CompressWork<T>& w) {
        const Plan& p = *plans[i];
        char* dd = (char*)key.outs[i];
        MGB_TRY(compress_encode_back<T>(p, heads[i], dd, key.caps[i], w, metas + i, ss));
        return compress_pack<T>(p, dd, w, metas + i, ss);
    }
    mgard_status front_a(int i, cudaStream_t ss) {
        return key.dtype == MGARD_F32 ? front_a_t<float>(i, ss, *wf[i]) : front_a_t<double>(i, ss, *wd[i]);
    }
    mgard_status front_b(int i, cudaStream_t ss) {
        return key.dtype == MGARD_F32 ? front_b_t<float>(i, ss, *wf[i]) : front_b_t<double>(i, ss, *wd[i]);
    }
    mgard_status back(int i, cudaStream_t ss) {
        return key.dtype == MGARD_F32 ? back_t<float>(i, ss, *wf[i]) : back_t<double>(i, ss, *wd[i]);
    }
    mgard_status phased(cudaStream_t st) {
        const int n = key.n;
        MGB_TRY(lanes.run(st, n, [this](int i, cudaStream_t ss) { return front_a(i, ss); }));
        if (ntail)
            MGB_TRY(key.dtype == MGARD_F32
                        ? tail_decompose_batch<float>(tail_jobs, ntail, tail_smem, tail_counter, st)
                        : tail_decompose_batch<double>(tail_jobs, ntail, tail_smem, tail_counter, st));
        MGB_TRY(lanes.run(st, n, [this](int i, cudaStream_t ss) { return front_b(i, ss); }));
        MGB_TRY(huffman_codebook_tables_batch(jobs, n, job_counter, st));
        return lanes.run(st, n, [this](int i, cudaStream_t ss) { return back(i, ss); });
    }
};

template <>
CompressWork<float>& BatchState::work<float>(int i) {
    return *wf[i];
}
template <>
CompressWork<double>& BatchState::work<double>(int i) {
    return *wd[i];
}

// Graphs are used when asked for, or (MGARD_BATCH_REPEAT) from the second
// identical call on; never while kernel tracing is on (graph launches are not
// traced).
bool use_graph(int flags, const Lanes& lanes) {
    if (timing_on()) return false;
    return (flags & MGARD_BATCH_GRAPH) || ((flags & MGARD_BATCH_REPEAT) && lanes.runs > 0);
}

std::mutex g_batch_mu;
std::list<std::unique_ptr<BatchState>> g_batches;   // most recently used first

}  // namespace

void release_batches() {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batches.clear();
}

void release_decompress_batches();

}  // namespace mgb

using namespace mgb;

extern "C" mgard_status mgard_compress_batch(int n, const void* const* fields, const int* ndims,
                                             const int64_t* const* shapes, mgard_dtype dtype,
                                             double tol, double s, mgard_tolmode mode,
                                             void* const* outs, const size_t* caps,
                                             size_t* out_bytes, mgard_status* statuses,
                                             int flags, void* stream) {
    if (n < 0 || (n > 0 && (!fields || !ndims || !shapes || !outs || !caps || !out_bytes))) {
        set_error("null argument");
        return MGARD_EINVAL;
    }
    if (dtype != MGARD_F32 && dtype != MGARD_F64) {
        set_error("dtype must be MGARD_F32 or MGARD_F64");
        return MGARD_EDTYPE;
    }
    if (!(tol > 0.0) || !std::isfinite(tol) || std::isnan(s) || s < 0.0 ||
        (mode != MGARD_ABS && mode != MGARD_REL) ||
        (flags & ~(MGARD_BATCH_GRAPH | MGARD_BATCH_AUTOTUNE | MGARD_BATCH_REPEAT |
                   MGARD_BATCH_PERSISTENT))) {
        set_error("tol must be positive and finite, s >= 0 or INFINITY, mode ABS or REL");
        return MGARD_EINVAL;
    }
    if (n == 0) return MGARD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    BatchKey key;
    MGB_CUDA(cudaGetDevice(&key.device));
    key.n = n;
    key.dtype = (int)dtype;
    key.mode = (int)mode;
    key.flags = flags;
    key.tol = tol;
    key.s = s;
    key.stream = st;
    for (int i = 0; i < n; ++i) {
        if (!fields[i] || !outs[i] || !shapes[i] || ndims[i] < 1 || ndims[i] > 4) {
            set_error("field, output or shape missing");
            return MGARD_EINVAL;
        }
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, fields[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
            cudaPointerGetAttributes(&a, outs[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            set_error("batched compression takes device buffers only");
            return MGARD_EINVAL;
        }
        if (((uintptr_t)outs[i] & 15) != 0) {
            set_error("output buffers must be 16-byte aligned");
            return MGARD_EINVAL;
        }
        key.shapes.push_back(ndims[i]);
        for (int d = 0; d < ndims[i]; ++d) key.shapes.push_back(shapes[i][d]);
        key.fields.push_back(fields[i]);
        key.outs.push_back(outs[i]);
        key.caps.push_back(caps[i]);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchState* b = nullptr;
    for (auto it = g_batches.begin(); it != g_batches.end(); ++it)
        if ((*it)->key == key) {
            g_batches.splice(g_batches.begin(), g_batches, it);
            b = g_batches.front().get();
            break;
        }
    if (!b) {
        std::unique_ptr<BatchState> nb(new BatchState());
        MGB_TRY(nb->init(key, ndims, shapes));
        // every buffer must hold at least the fixed sections
        for (int i = 0; i < n; ++i) {
            const uint64_t N = (uint64_t)nb->plans[i]->total();
            const Sections fx = layout(nb->plans[i]->L, (N + CHUNK - 1) / CHUNK, 0, 0);
            if (caps[i] < fx.outliers) {
                out_bytes[i] = fx.outliers;
                if (statuses) statuses[i] = MGARD_ECAPACITY;
                set_error("output buffer smaller than the fixed sections");
                return MGARD_ECAPACITY;
            }
        }
        g_batches.push_front(std::move(nb));
        while (g_batches.size() > BATCH_CACHE) g_batches.pop_back();
        b = g_batches.front().get();
    }
    if (flags & MGARD_BATCH_PERSISTENT) {
        if (use_graph(flags, b->lanes))
            MGB_TRY(b->lanes.run_graph_seq(st, [b](cudaStream_t s0) { return b->phased(s0); }));
        else
            MGB_TRY(b->phased(st));
    } else {
        auto body = [b](int i, cudaStream_t ss) { return b->field(i, ss); };
        if (use_graph(flags, b->lanes)) MGB_TRY(b->lanes.run_graph(st, n, body));
        else MGB_TRY(b->lanes.run(st, n, body));
    }
    ++b->lanes.runs;
    MGB_CUDA(cudaMemcpyAsync(b->hmetas, b->metas, sizeof(CompressMeta) * n, cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    mgard_status first = MGARD_OK;
    for (int i = 0; i < n; ++i) {
        const CompressMeta& m = b->hmetas[i];
        out_bytes[i] = m.total;
        mgard_status e = MGARD_OK;
        if (m.status & ST_NONFINITE) e = MGARD_ENONFINITE;
        else if (m.status & ST_RANGE) e = MGARD_ERANGE;
        else if (m.status & ST_NOCODE) e = MGARD_EINVAL;
        else if (m.status & ST_CAPACITY) e = MGARD_ECAPACITY;
        if (statuses) statuses[i] = e;
        if (e != MGARD_OK && first == MGARD_OK) {
            first = e;
            const char* why = e == MGARD_ENONFINITE ? "input holds NaN or Inf"
                              : e == MGARD_ERANGE   ? "tolerance too small: a quantized value exceeds the 32-bit range"
                              : e == MGARD_ECAPACITY ? "output buffer too small"
                                                     : "a symbol has no Huffman code";
            set_error(n == 1 ? std::string(why)
                             : "batched compression: field " + std::to_string(i) + ": " + why);
        }
    }
    return first;
}

// ---------------------------------------------------------------------------
// Batched decompression.  The headers (and bin widths) of all buffers come
// to the host in one round trip; the rest runs as for compression: one
// stream-ordered pipeline per buffer over the internal streams, optionally
// from a captured graph.  The graph bakes in the headers' sizes and widths,
// so they are part of the cache key.
namespace mgb {
namespace {

constexpr size_t HEAD_BYTES = 768;   // header + widths of up to 64 levels

struct DecompressKey {
    int device = -1;
    int n = 0, flags = 0;
    cudaStream_t stream = nullptr;
    std::vector<const void*> ins;
    std::vector<size_t> in_bytes;
    std::vector<void*> outs;
    std::vector<size_t> caps;
    std::vector<char> heads;   // HEAD_BYTES per buffer
    bool operator==(const DecompressKey& o) const {
        return device == o.device && n == o.n && flags == o.flags && stream == o.stream &&
               ins == o.ins && in_bytes == o.in_bytes && outs == o.outs && caps == o.caps &&
               heads == o.heads;
    }
};

struct DecompressBatch {
    DecompressKey key;
    std::vector<const Plan*> plans;       // null for a buffer whose header failed
    std::vector<mgard_header> heads;
    std::vector<std::vector<double>> widths;
    std::vector<std::unique_ptr<DecompressWork<float>>> wf;
    std::vector<std::unique_ptr<DecompressWork<double>>> wd;
    std::vector<int> items;               // buffers that run
    std::vector<mgard_status> pre;        // result of the host checks, per buffer
    unsigned* stat = nullptr;             // device, one per buffer
    unsigned* hstat = nullptr;            // pinned
    // persistent tail phase (MGARD_BATCH_PERSISTENT): the buffers whose small
    // levels wait for one batched launch, its job list and shared memory
    std::vector<char> tail_deferred;
    void* tail_jobs = nullptr;
    int ntail = 0;
    size_t tail_smem = 0;
    unsigned* tail_counter = nullptr;
    Lanes lanes;

    ~DecompressBatch() {
        wf.clear();
        wd.clear();
        if (tail_jobs) cudaFreeAsync(tail_jobs, lanes.side[0]);
        if (tail_counter) cudaFreeAsync(tail_counter, lanes.side[0]);
        if (stat) cudaFreeAsync(stat, lanes.side[0]);
        if (lanes.side[0]) cudaStreamSynchronize(lanes.side[0]);
        lanes.destroy();
        if (hstat) cudaFreeHost(hstat);
        cudaGetLastError();
    }

    mgard_status item(int k, cudaStream_t ss) {
        const int i = items[k];
        const mgard_header& h = heads[i];
        MGB_CUDA(cudaMemsetAsync(stat + i, 0, sizeof(unsigned), ss));
        if (h.dtype == MGARD_F32)
            return item_t<float>(i, ss, *wf[i]);
        return item_t<double>(i, ss, *wd[i]);
    }
    template <typename T>
    mgard_status item_t(int i, cudaStream_t ss, DecompressWork<T>& w) {
        w.py.defer_tail = !tail_deferred.empty() && tail_deferred[i];
        const mgard_status r = decompress_core<T>(*plans[i], heads[i], widths[i].data(),
                                                  (const char*)key.ins[i], (T*)key.outs[i], w,
                                                  stat + i, ss);
        w.py.defer_tail = false;
        const bool deferred = !tail_deferred.empty() && tail_deferred[i];
        if (r == MGARD_OK && deferred != w.py.tail_pending) {
            set_error("batched tail: the recomposition did not stop where planned");
            return MGARD_EINVAL;
        }
        return r;
    }
    // after the batched tails: the levels above them
    template <typename T>
    mgard_status rest_t(int i, cudaStream_t ss, DecompressWork<T>& w) {
        if (tail_deferred.empty() || !tail_deferred[i]) return MGARD_OK;
        w.py.tail_done = true;
        const mgard_status r = recompose_pyramid<T>(*plans[i], nullptr, (T*)key.outs[i], w.py, ss,
                                                    w.zs.template as<T>());
        w.py.tail_done = false;
        return r;
    }
    mgard_status rest(int k, cudaStream_t ss) {
        const int i = items[k];
        return heads[i].dtype == MGARD_F32 ? rest_t<float>(i, ss, *wf[i]) : rest_t<double>(i, ss, *wd[i]);
    }
    template <typename T>
    mgard_status tail_jobs_t(cudaStream_t s0) {
        const size_t bytes = tail_args_bytes<T>();
        std::vector<char> host;
        tail_deferred.assign(plans.size(), 0);
        for (int i : items) {
            if (heads[i].dtype != (sizeof(T) == 4 ? (uint32_t)MGARD_F32 : (uint32_t)MGARD_F64)) continue;
            const Plan& p = *plans[i];
            const int Lt = rows3_ok(p) ? tail_levels(p) : 0;
            if (!Lt) continue;
            DecompressWork<T>& w = dwork<T>(i);
            T* level_Lt = Lt == p.L ? (T*)key.outs[i] : w.py.lv[Lt];
            host.resize(host.size() + bytes);
            size_t smem = 0;
            MGB_TRY(tail_job<T>(p, Lt, w.py, level_Lt, w.zs.template as<T>(), nullptr,
                                host.data() + host.size() - bytes, &smem));
            tail_smem = std::max(tail_smem, smem);
            tail_deferred[i] = 1;
            ++ntail;
        }
        if (!ntail) return MGARD_OK;
        count_device_alloc();
        MGB_CUDA(cudaMallocAsync(&tail_jobs, host.size(), s0));
        count_device_alloc();
        MGB_CUDA(cudaMallocAsync((void**)&tail_counter, sizeof(unsigned), s0));
        MGB_CUDA(cudaMemcpyAsync(tail_jobs, host.data(), host.size(), cudaMemcpyHostToDevice, s0));
        return MGARD_OK;
    }
    template <typename T>
    DecompressWork<T>& dwork(int i);
};

template <>
DecompressWork<float>& DecompressBatch::dwork<float>(int i) {
    return *wf[i];
}
template <>
DecompressWork<double>& DecompressBatch::dwork<double>(int i) {
    return *wd[i];
}

std::list<std::unique_ptr<DecompressBatch>> g_dbatches;

}  // namespace

void release_decompress_batches() {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_dbatches.clear();
}

}  // namespace mgb

extern "C" mgard_status mgard_decompress_batch(int n, const void* const* ins,
                                               const size_t* in_bytes, void* const* fields,
                                               const size_t* field_caps, mgard_status* statuses,
                                               int flags, void* stream) {
    if (n < 0 || (n > 0 && (!ins || !in_bytes || !fields || !field_caps))) {
        set_error("null argument");
        return MGARD_EINVAL;
    }
    if (flags & ~(MGARD_BATCH_GRAPH | MGARD_BATCH_REPEAT | MGARD_BATCH_PERSISTENT)) {
        set_error("unknown flags");
        return MGARD_EINVAL;
    }
    if (n == 0) return MGARD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        cudaPointerAttributes a;
        if (!ins[i] || !fields[i] || cudaPointerGetAttributes(&a, ins[i]) != cudaSuccess ||
            a.type != cudaMemoryTypeDevice || cudaPointerGetAttributes(&a, fields[i]) != cudaSuccess ||
            a.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            set_error("batched decompression takes device buffers only");
            return MGARD_EINVAL;
        }
    }
    DecompressKey key;
    MGB_CUDA(cudaGetDevice(&key.device));
    key.n = n;
    key.flags = flags;
    key.stream = st;
    key.heads.assign((size_t)n * HEAD_BYTES, 0);
    // one round trip for every header
    {
        char* pin = nullptr;
        count_device_alloc();
        MGB_CUDA(cudaMallocHost(&pin, (size_t)n * HEAD_BYTES));
        std::unique_ptr<char, cudaError_t (*)(void*)> guard(pin, cudaFreeHost);
        for (int i = 0; i < n; ++i) {
            const size_t k = std::min(in_bytes[i], HEAD_BYTES);
            if (k) MGB_CUDA(cudaMemcpyAsync(pin + i * HEAD_BYTES, ins[i], k, cudaMemcpyDeviceToHost, st));
        }
        MGB_CUDA(cudaStreamSynchronize(st));
        std::memcpy(key.heads.data(), pin, (size_t)n * HEAD_BYTES);
    }
    for (int i = 0; i < n; ++i) {
        key.ins.push_back(ins[i]);
        key.in_bytes.push_back(in_bytes[i]);
        key.outs.push_back(fields[i]);
        key.caps.push_back(field_caps[i]);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    DecompressBatch* b = nullptr;
    for (auto it = g_dbatches.begin(); it != g_dbatches.end(); ++it)
        if ((*it)->key == key) {
            g_dbatches.splice(g_dbatches.begin(), g_dbatches, it);
            b = g_dbatches.front().get();
            break;
        }
    if (!b) {
        std::vector<mgard_status> pre(n, MGARD_OK);
        std::unique_ptr<DecompressBatch> nb(new DecompressBatch());
        nb->key = key;
        MGB_TRY(nb->lanes.init());
        cudaStream_t s0 = nb->lanes.side[0];
        count_device_alloc();
        MGB_CUDA(cudaMallocHost(&nb->hstat, sizeof(unsigned) * n));
        count_device_alloc();
        MGB_CUDA(cudaMallocAsync((void**)&nb->stat, sizeof(unsigned) * n, s0));
        nb->plans.assign(n, nullptr);
        nb->heads.resize(n);
        nb->widths.resize(n);
        nb->wf.resize(n);
        nb->wd.resize(n);
        for (int i = 0; i < n; ++i) {
            mgard_header& h = nb->heads[i];
            std::memcpy(&h, key.heads.data() + i * HEAD_BYTES, sizeof(h));
            if (in_bytes[i] < sizeof(h) || check_header(h, in_bytes[i]) != MGARD_OK ||
                h.off_widths + 8 * (h.nlevels + 1) > HEAD_BYTES) {
                pre[i] = MGARD_ECORRUPT;
                continue;
            }
            nb->widths[i].resize(h.nlevels + 1);
            std::memcpy(nb->widths[i].data(), key.heads.data() + i * HEAD_BYTES + h.off_widths,
                        8 * (h.nlevels + 1));
            const Plan* p;
            if (!widths_valid(nb->widths[i].data(), (int)h.nlevels) ||
                get_plan((int)h.ndim, h.shape, -1, &p) != MGARD_OK || p->L != (int)h.nlevels) {
                pre[i] = MGARD_ECORRUPT;
                continue;
            }
            const size_t need = (size_t)p->total() * (h.dtype == MGARD_F64 ? 8 : 4);
            if (field_caps[i] < need) {
                pre[i] = MGARD_ECAPACITY;
                continue;
            }
            nb->plans[i] = p;
            if (h.dtype == MGARD_F32) {
                nb->wf[i].reset(new DecompressWork<float>());
                MGB_TRY(nb->wf[i]->alloc(*p, s0));
            } else {
                nb->wd[i].reset(new DecompressWork<double>());
                MGB_TRY(nb->wd[i]->alloc(*p, s0));
            }
            nb->items.push_back(i);
        }
        if ((flags & MGARD_BATCH_PERSISTENT) && !nb->items.empty()) {   // one dtype per batch
            const uint32_t dt = nb->heads[nb->items[0]].dtype;
            bool same = true;
            for (int i : nb->items) same = same && nb->heads[i].dtype == dt;
            if (same) MGB_TRY(dt == MGARD_F32 ? nb->tail_jobs_t<float>(s0) : nb->tail_jobs_t<double>(s0));
        }
        MGB_CUDA(cudaStreamSynchronize(s0));
        nb->pre = pre;
        g_dbatches.push_front(std::move(nb));
        while (g_dbatches.size() > BATCH_CACHE) g_dbatches.pop_back();
        b = g_dbatches.front().get();
    }
    const std::vector<mgard_status>& pre = b->pre;
    const int m = (int)b->items.size();
    auto body = [b](int k, cudaStream_t ss) { return b->item(k, ss); };
    // persistent form: every buffer decoded down to level 0, one launch for
    // all their small levels, then every buffer's larger levels
    auto phased = [b, m, body](cudaStream_t s0) -> mgard_status {
        MGB_TRY(b->lanes.run(s0, m, body));
        const uint32_t dt = b->heads[b->items[0]].dtype;
        MGB_TRY(dt == MGARD_F32
                    ? tail_recompose_batch<float>(b->tail_jobs, b->ntail, b->tail_smem, b->tail_counter, s0)
                    : tail_recompose_batch<double>(b->tail_jobs, b->ntail, b->tail_smem, b->tail_counter, s0));
        return b->lanes.run(s0, m, [b](int k, cudaStream_t ss) { return b->rest(k, ss); });
    };
    if (m && b->ntail) {
        if (use_graph(flags, b->lanes)) MGB_TRY(b->lanes.run_graph_seq(st, phased));
        else MGB_TRY(phased(st));
        ++b->lanes.runs;
        MGB_CUDA(cudaMemcpyAsync(b->hstat, b->stat, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, st));
    } else if (m) {
        if (use_graph(flags, b->lanes)) MGB_TRY(b->lanes.run_graph(st, m, body));
        else MGB_TRY(b->lanes.run(st, m, body));
        ++b->lanes.runs;
        MGB_CUDA(cudaMemcpyAsync(b->hstat, b->stat, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, st));
    }
    MGB_CUDA(cudaStreamSynchronize(st));
    mgard_status first = MGARD_OK;
    for (int i = 0; i < n; ++i) {
        mgard_status e = pre[i];
        if (e == MGARD_OK && b->plans[i] && (b->hstat[i] & ST_CORRUPT)) e = MGARD_ECORRUPT;
        if (statuses) statuses[i] = e;
        if (e != MGARD_OK && first == MGARD_OK) {
            first = e;
            // a header failure keeps the reason check_header gave (one buffer)
            if (n > 1 || b->plans[i])
                set_error("batched decompression: buffer " + std::to_string(i) +
                          (e == MGARD_ECAPACITY ? ": field buffer too small" : ": corrupt stream"));
        }
    }
    return first;
}
