// Shared definitions of the CUDA library (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mgard_b300.h"

namespace mgb {

// Last-error text, per host thread.
void set_error(const std::string& msg);
// Adds one to the count of CUDA allocations (device, pool or pinned host) the
// library has asked for; every allocation call site calls it first.
void count_device_alloc();

#define MGB_CUDA(call)                                                              \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            ::mgb::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
            return e_ == cudaErrorMemoryAllocation ? MGARD_ENOMEM : MGARD_ECUDA;    \
        }                                                                           \
    } while (0)

#define MGB_TRY(expr)                      \
    do {                                   \
        mgard_status s_ = (expr);          \
        if (s_ != MGARD_OK) return s_;     \
    } while (0)

// Kernel tracing (timing.cu): a scope that brackets the launches inside it
// with CUDA events on `st` when mgard_timing_enable(1) is in effect.
int timing_begin(const char* name, cudaStream_t st);
bool timing_on();
void timing_end(int slot, cudaStream_t st);
struct ScopedTimer {
    int slot;
    cudaStream_t st;
    ScopedTimer(const char* name, cudaStream_t s) : slot(timing_begin(name, s)), st(s) {}
    ~ScopedTimer() { timing_end(slot, st); }
};
#define MGB_CAT2(a, b) a##b
#define MGB_CAT(a, b) MGB_CAT2(a, b)
#define MGB_TIMED(name, st) ::mgb::ScopedTimer MGB_CAT(mgb_timer_, __LINE__)(name, st)
// Launch a kernel inside its own traced scope.
#define MGB_LAUNCH(name, st, ...)                  \
    do {                                           \
        ::mgb::ScopedTimer mgb_launch_timer_(name, st); \
        __VA_ARGS__;                               \
    } while (0)

constexpr int DICT = MGARD_DICT;
constexpr int RADIUS = MGARD_DICT / 2;
constexpr int CHUNK = MGARD_CHUNK;
constexpr int LMAX = MGARD_LMAX;
// float32 quantization: |q| below this many bins is decided and dequantized
// in float32 (the width margin covers its rounding); larger escapes are
// decided and dequantized in double.
constexpr int F32_EXACT = 4096;

// Escapes of F32_EXACT bins or more follow double-precision rules: the
// quotient q = rint(fl64(c / w)) and the value fl32(fl64(q * w)).  B300 runs
// FP64 at about two lanes per clock per SM, and under SIMT a warp pays for a
// lane's FP64 branch in nearly every group of symbols, so the float path
// takes these decisions in two-float arithmetic (error below 2^-45 relative)
// whenever that error bound proves the double computation rounds the same
// way, and falls back to double otherwise (well under 0.1% of typical
// escapes).  The result is the double rule's, bit for bit.
struct WidthSplit {
    float hi, lo;   // w = hi + lo + r with |r| <= 2^-48 w; hi = 0: no split (always double)
};
__host__ __device__ inline WidthSplit split_width(double w) {
    WidthSplit s{0.f, 0.f};
    if (w >= 0x1p-60 && w <= 0x1p60) {
        s.hi = (float)w;
        s.lo = (float)(w - (double)s.hi);
    }
    return s;
}

// q = rint(fl64(c / w)) for a finite float c; false when it leaves int32
// (the caller flags the range error).
__device__ inline bool quant_big(float c, WidthSplit ws, double w, int32_t& qo) {
    const float q0 = __fdiv_rn(c, ws.hi);   // hi = 0 gives +-inf: double path
    if (fabsf(q0) < 0x1p21f) {
        // t = c / w = q0 + q1 + e with |e| < 2^-23: the remainder of q0
        // against both parts of w, divided by the leading part
        const float r = __fmaf_rn(-q0, ws.hi, c);
        const float r2 = __fmaf_rn(-q0, ws.lo, r);
        const float q1 = __fdiv_rn(r2, ws.hi);
        const float k0 = rintf(q0);
        const float f = __fadd_rn(__fsub_rn(q0, k0), q1);   // q0 - k0 is exact
        const float n = rintf(f);
        const float g = __fsub_rn(f, n);                    // t - (k0 + n) = g +- 2^-22
        if (fabsf(g) < 0.5f - 0x1p-16f) {                   // no half-integer within reach
            qo = (int32_t)k0 + (int32_t)n;
            return true;
        }
    }
    const double qd = rint((double)c / w);
    if (fabs(qd) > 2147483647.0) return false;
    qo = (int32_t)qd;
    return true;
}

// fl32(fl64(q * w)).
__device__ inline float dequant_big(int32_t q, WidthSplit ws, double w) {
    if (q > -(1 << 24) && q < (1 << 24)) {
        // q * w = p0 + s + e with |e| < 2^-46 |q w| (q is exact in float)
        const float qf = (float)q;
        const float p0 = __fmul_rn(qf, ws.hi);
        const float e0 = __fmaf_rn(qf, ws.hi, -p0);
        const float s = __fmaf_rn(qf, ws.lo, e0);
        const float f = __fadd_rn(p0, s);
        // exact error of that sum (Knuth's two-sum)
        const float bb = __fsub_rn(f, p0);
        const float err = __fadd_rn(__fsub_rn(p0, __fsub_rn(f, bb)), __fsub_rn(s, bb));
        const unsigned b = __float_as_uint(f);
        const unsigned ex = (b >> 23) & 0xFFu;
        // f rounds q * w and its double rounding alike when p0 + s stays
        // 2^-16 ulp away from the midpoints f +- ulp/2 (equal spacing on
        // both sides: f not a power of two; normal range with room below)
        if (ex >= 64u && ex < 255u && (b & 0x7FFFFFu) != 0u) {
            const float lim = __uint_as_float((ex - 24u) << 23) * (1.f - 0x1p-15f);
            if (fabsf(err) < lim) return f;
        }
    }
    return (float)((double)q * w);
}

template <typename T>
__device__ inline T dequant_escape(int32_t q, T wt, WidthSplit ws, double w) {
    if (sizeof(T) == 4) {
        if (q < F32_EXACT && q > -F32_EXACT) return (T)__fmul_rn((float)q, (float)wt);
        return (T)dequant_big(q, ws, w);
    }
    return (T)((double)q * w);
}

// Levels a plan may have (a header records at most 64).
constexpr int MAX_LEVELS = 64;

// Symbol offsets of the levels in symbol order: level l holds symbols
// [off[l], off[l+1]); off[L+1] is the total.
struct LevelOffsets {
    int L;
    long long off[MAX_LEVELS + 2];
};

// Device status bits set by kernels and read back by the host.
enum : unsigned {
    ST_NONFINITE = 1u,
    ST_RANGE = 2u,
    ST_NOCODE = 4u,
    ST_CORRUPT = 8u,
    ST_CAPACITY = 16u,   // the output buffer is smaller than the compressed data
    ST_TIMEOUT = 32u,    // a bounded device wait gave up
};

// Partial statistics of one block over a level's coefficients (features of
// the tolerance predictor): sums of r = log10(max(|c|, 1e-12 a) / a) and r^2,
// and hist[k] = coefficients below exactly k of the thresholds 10^(-j/2) a,
// j = 0..FEAT_BINS-2.
constexpr int FEAT_BINS = 16;
struct FeatPart {
    double sum, sum2;
    unsigned long long hist[FEAT_BINS];
};

// Per-axis tables of one level transition (fine grid of level l, coarse
// grid of level l-1).  Pointers are device addresses; for an inactive axis
// (extent 1) they are null and the axis is treated as "always coarse".
template <typename T>
struct AxisT {
    const int* fcls;     // [m]  coarse index J >= 0, or -(J+1) for a new node between J and J+1
    const T* wl;         // [m]  interpolation weight of coarse J (new nodes)
    const T* wr;         // [m]  interpolation weight of coarse J+1 (new nodes)
    const int* cbefore;  // [m]  number of coarse positions < i
    const int* rf;       // [mc] fine position of coarse node J
    const T* rw;         // [mc*5] restriction weights on fine positions rf[J]-2 .. rf[J]+2
    const T* tsub;       // [mc] Thomas: sub-diagonal a_J
    const T* tinv;       // [mc] Thomas: 1 / (b_J - a_J c'_{J-1})
    const T* tcp;        // [mc] Thomas: c'_J
    const double* mdiag; // [m]  mass matrix of the level-l grid: diagonal
    const double* moff;  // [m]  mass matrix: M[i][i+1] (last entry 0)
    const T* mdt;        // [m]  the same two tables in T
    const T* mot;
    // Uniform parts of the tables, so row kernels need no per-element table
    // loads there: for i < ireg the interpolation weights are (1, 0) at even
    // i and (1/2, 1/2) at odd i; for coarse J in [rlo, rhi) the restriction
    // window is centred on 2J with weights rwi.
    int ireg;
    int rlo, rhi;
    T rwi[5];
};

template <typename T>
struct Level {
    int64_t n[4];    // fine shape (4D view, leading 1s)
    int64_t nc[4];   // coarse shape
    AxisT<T> ax[4];
};

// Finest-grid position of every level-l node, per axis (in-place layout).
struct LevelIndex {
    int64_t n[4];
    const int64_t* pos[4];
};

__host__ __device__ inline int64_t prod4(const int64_t* n) { return n[0] * n[1] * n[2] * n[3]; }

__device__ inline void unravel4(int64_t lin, const int64_t* n, int64_t* i) {
    i[3] = lin % n[3]; lin /= n[3];
    i[2] = lin % n[2]; lin /= n[2];
    i[1] = lin % n[1]; lin /= n[1];
    i[0] = lin;
}

__host__ __device__ inline int64_t ravel4(const int64_t* i, const int64_t* n) {
    return ((i[0] * n[1] + i[1]) * n[2] + i[2]) * n[3] + i[3];
}

// 3D launches over a 4D view without per-element integer division: threads
// of x cover axis 3, grid y covers axis 2, grid z covers axes 0 and 1
// folded; every level is a grid-stride loop, so any shape fits any grid.
#define FOR_NODES(n, i0, i1, i2, i3)                                                         \
    for (int64_t mgb_z_ = blockIdx.z; mgb_z_ < (n)[0] * (n)[1]; mgb_z_ += gridDim.z)          \
        for (int64_t i0 = mgb_z_ / (n)[1], i1 = mgb_z_ - i0 * (n)[1], i2 = blockIdx.y;        \
             i2 < (n)[2]; i2 += gridDim.y)                                                    \
            for (int64_t i3 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i3 < (n)[3];     \
                 i3 += (int64_t)gridDim.x * blockDim.x)

inline dim3 grid3(const int64_t* n, int bx, int64_t ycap = 65535, int64_t zcap = 65535) {
    int64_t gx = (n[3] + bx - 1) / bx;
    if (gx > (1LL << 30)) gx = 1LL << 30;
    int64_t gy = n[2] < ycap ? n[2] : ycap;
    int64_t nz = n[0] * n[1];
    int64_t gz = nz < zcap ? nz : zcap;
    return dim3((unsigned)(gx < 1 ? 1 : gx), (unsigned)(gy < 1 ? 1 : gy), (unsigned)(gz < 1 ? 1 : gz));
}

inline int grid_for(int64_t work, int block, int64_t cap = 148LL * 64) {
    int64_t g = (work + block - 1) / block;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace mgb
