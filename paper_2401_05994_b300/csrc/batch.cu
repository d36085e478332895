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

namespace mgb {

namespace {

constexpr int BATCH_STREAMS = 8;
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

struct BatchState {
    BatchKey key;
    std::vector<const Plan*> plans;
    std::vector<mgard_header> heads;
    std::vector<std::unique_ptr<CompressWork<float>>> wf;
    std::vector<std::unique_ptr<CompressWork<double>>> wd;
    CompressMeta* metas = nullptr;      // device, one per field
    CompressMeta* hmetas = nullptr;     // pinned host copy
    cudaStream_t side[BATCH_STREAMS] = {};
    cudaStream_t origin = nullptr;      // capture happens here (the caller's stream may be
                                        // the legacy default stream, which cannot capture)
    cudaEvent_t fork = nullptr, join[BATCH_STREAMS] = {};
    cudaGraphExec_t exec = nullptr;

    ~BatchState() {
        if (exec) cudaGraphExecDestroy(exec);
        // workspaces free themselves on side[0]; wait for that before the
        // stream goes away
        wf.clear();
        wd.clear();
        if (metas) cudaFreeAsync(metas, side[0]);
        if (side[0]) cudaStreamSynchronize(side[0]);
        for (int k = 0; k < BATCH_STREAMS; ++k) {
            if (join[k]) cudaEventDestroy(join[k]);
            if (side[k]) cudaStreamDestroy(side[k]);
        }
        if (fork) cudaEventDestroy(fork);
        if (origin) cudaStreamDestroy(origin);
        if (hmetas) cudaFreeHost(hmetas);
        cudaGetLastError();
    }

    mgard_status init(const BatchKey& k, const int* ndims, const int64_t* const* shapes) {
        key = k;
        for (int s = 0; s < BATCH_STREAMS; ++s) {
            MGB_CUDA(cudaStreamCreateWithFlags(&side[s], cudaStreamNonBlocking));
            MGB_CUDA(cudaEventCreateWithFlags(&join[s], cudaEventDisableTiming));
        }
        MGB_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        MGB_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
        MGB_CUDA(cudaMallocHost(&hmetas, sizeof(CompressMeta) * k.n));
        MGB_CUDA(cudaMallocAsync((void**)&metas, sizeof(CompressMeta) * k.n, side[0]));
        for (int i = 0; i < k.n; ++i) {
            const Plan* p;
            MGB_TRY(get_plan(ndims[i], shapes[i], -1, &p));
            plans.push_back(p);
            heads.push_back(header_template(*p, (mgard_dtype)k.dtype, ndims[i], shapes[i], k.tol,
                                            k.s, (mgard_tolmode)k.mode));
            if (k.dtype == MGARD_F32) {
                wf.emplace_back(new CompressWork<float>());
                MGB_TRY(wf.back()->alloc(*p, side[0]));
            } else {
                wd.emplace_back(new CompressWork<double>());
                MGB_TRY(wd.back()->alloc(*p, side[0]));
            }
        }
        MGB_TRY(huffman_prepare());
        MGB_CUDA(cudaStreamSynchronize(side[0]));
        return MGARD_OK;
    }

    // Fork from `st`, every field on a side stream, join back into `st`.
    mgard_status enqueue(cudaStream_t st) {
        const int nside = std::min(BATCH_STREAMS, std::max(key.n, 1));
        MGB_CUDA(cudaEventRecord(fork, st));
        for (int s = 0; s < nside; ++s) MGB_CUDA(cudaStreamWaitEvent(side[s], fork, 0));
        for (int i = 0; i < key.n; ++i) {
            cudaStream_t ss = side[i % nside];
            char* dd = (char*)key.outs[i];
            const uint64_t cap = key.caps[i];
            if (key.dtype == MGARD_F32)
                MGB_TRY(compress_core<float>(*plans[i], (const float*)key.fields[i], heads[i],
                                             key.tol, key.s, (mgard_tolmode)key.mode, dd, cap,
                                             *wf[i], metas + i, ss));
            else
                MGB_TRY(compress_core<double>(*plans[i], (const double*)key.fields[i], heads[i],
                                              key.tol, key.s, (mgard_tolmode)key.mode, dd, cap,
                                              *wd[i], metas + i, ss));
        }
        for (int s = 0; s < nside; ++s) {
            MGB_CUDA(cudaEventRecord(join[s], side[s]));
            MGB_CUDA(cudaStreamWaitEvent(st, join[s], 0));
        }
        return MGARD_OK;
    }

    // Capture fork, fields and join on the internal origin stream; the graph
    // is then launched on the caller's stream.
    mgard_status capture() {
        MGB_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
        const mgard_status e = enqueue(origin);
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
        return MGARD_OK;
    }
};

std::mutex g_batch_mu;
std::list<std::unique_ptr<BatchState>> g_batches;   // most recently used first

}  // namespace

void release_batches() {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batches.clear();
}

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
        (mode != MGARD_ABS && mode != MGARD_REL) || (flags & ~MGARD_BATCH_GRAPH)) {
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
    if (flags & MGARD_BATCH_GRAPH) {
        if (!b->exec) MGB_TRY(b->capture());
        MGB_CUDA(cudaGraphLaunch(b->exec, st));
    } else {
        MGB_TRY(b->enqueue(st));
    }
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
            set_error("batched compression: field " + std::to_string(i) + " failed");
        }
    }
    return first;
}
