// Optional kernel tracing: when enabled, each kernel launch of the library
// is bracketed by a pair of CUDA events recorded on its launch stream, and
// mgard_timing_report() aggregates launches and device time per kernel.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace mgb {

namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pool;
size_t g_used = 0;
volatile int g_on = 0;
}  // namespace

bool timing_on() { return g_on != 0; }

int timing_begin(const char* name, cudaStream_t st) {
    if (!g_on) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return -1;   // launches captured into a graph are not traced
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_used == g_pool.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        g_pool.push_back({a, b});
    }
    auto ev = g_pool[g_used++];
    cudaEventRecord(ev.first, st);
    g_recs.push_back({name, ev.first, ev.second});
    return (int)g_recs.size() - 1;
}

void timing_end(int slot, cudaStream_t st) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lock(g_mu);
    cudaEventRecord(g_recs[slot].b, st);
}

}  // namespace mgb

extern "C" {

void mgard_timing_enable(int on) {
    std::lock_guard<std::mutex> lock(mgb::g_mu);
    mgb::g_on = on ? 1 : 0;
}

size_t mgard_timing_report(char* buf, size_t cap) {
    using namespace mgb;
    std::lock_guard<std::mutex> lock(g_mu);
    std::map<std::string, std::pair<long, double>> agg;
    for (auto& r : g_recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        auto& e = agg[r.name];
        e.first += 1;
        e.second += ms;
    }
    std::string out;
    char line[256];
    for (auto& kv : agg) {
        std::snprintf(line, sizeof(line), "%s %ld %.6f\n", kv.first.c_str(), kv.second.first,
                      kv.second.second);
        out += line;
    }
    if (!buf) return out.size() + 1;   // size query: keep the records
    g_recs.clear();
    g_used = 0;
    if (cap) {
        size_t n = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return out.size() + 1;
}

}  // extern "C"
