// Level-wise linear quantization and its inverse, with a fused histogram.
//
// Paper, "Software design": every multilevel coefficient is approximated by
// an integer multiple of its level's bin width.  Symbols are laid out level
// by level (level 0 first), each level in row-major order of its grid,
// holding only the nodes new on that level.  |q| < DICT/2 maps to symbol
// q + DICT/2; larger values escape to symbol 0 with q stored aside.
#include <cstring>

#include "huffman.cuh"
#include "quantize.cuh"
#include "multilevel.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

struct QLevel {
    int64_t n[4];           // level grid shape
    int64_t tail[4];        // prod_{b > a} of the coarse extents (rank computation)
    const int* fcls[4];     // level tables (null: inactive axis or level 0)
    const int* cbefore[4];
    const int64_t* pos[4];  // finest positions (in-place layout); null for compact
    int64_t fine[4];        // finest shape (in-place layout)
    int64_t sym_off;
    int tables;             // level >= 1
};

struct NodeInfo {
    int64_t addr;
    int64_t rank;
    bool skip;
};

// Position of a level-l node among the nodes new on level l (row-major):
// its linear index minus the number of coarse-grid nodes before it.
__device__ inline NodeInfo node_info(const QLevel& q, const int64_t* i) {
    NodeInfo r;
    const int64_t lin = ravel4(i, q.n);
    r.skip = false;
    r.rank = lin;
    if (q.tables) {
        bool prefix = true;   // all axes before the current one are coarse
        int64_t cnt = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int* fc = q.fcls[a];
            if (!fc) continue;
            if (prefix) cnt += (int64_t)q.cbefore[a][i[a]] * q.tail[a];
            if (fc[i[a]] < 0) prefix = false;
        }
        r.skip = prefix;   // a node of the coarser grid
        r.rank = lin - cnt;
    }
    if (q.pos[0]) {
        int64_t g[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) g[a] = q.pos[a][i[a]];
        r.addr = ravel4(g, q.fine);
    } else {
        r.addr = lin;
    }
    return r;
}

__device__ inline void quantize_value(float c, float inv_w, WidthSplit ws, double w, int& sym,
                                      int32_t& qo, unsigned& st) {
    const float x = __fmul_rn(c, inv_w);
    const float q = rintf(x);
    if (fabsf(q) < (float)RADIUS) {   // false for NaN and +-Inf, which are tested below
        sym = (int)q + RADIUS;
        return;
    }
    sym = MGARD_ESC;
    if (!isfinite(c)) {
        st |= ST_NONFINITE;
        qo = 0;
        return;
    }
    if (fabsf(q) < (float)F32_EXACT) {
        qo = (int32_t)q;
        return;
    }
    if (!quant_big(c, ws, w, qo)) {
        st |= ST_RANGE;
        qo = 0;
    }
}

__device__ inline void quantize_value(double c, double /*inv_w*/, WidthSplit, double w, int& sym,
                                      int32_t& qo, unsigned& st) {
    if (!isfinite(c)) {
        st |= ST_NONFINITE;
        sym = MGARD_ESC;
        qo = 0;
        return;
    }
    const double q = rint(c / w);
    if (fabs(q) < (double)RADIUS) {
        sym = (int)q + RADIUS;
        return;
    }
    sym = MGARD_ESC;
    if (fabs(q) > 2147483647.0) {
        st |= ST_RANGE;
        qo = 0;
    } else {
        qo = (int32_t)q;
    }
}

constexpr int QT = 128;

template <typename T>
__global__ void __launch_bounds__(QT) k_quantize(const T* __restrict__ c, QLevel q,
                                                 const double* __restrict__ wp,
                                                 uint16_t* __restrict__ sym,
                                                 int32_t* __restrict__ esc,
                                                 unsigned long long* __restrict__ hist,
                                                 unsigned* status) {
    __shared__ unsigned sh[DICT];
    for (int k = threadIdx.x; k < DICT; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const double w = *wp;
    const T inv_w = (T)(1.0 / w);
    const WidthSplit ws = split_width(w);
    const int lane = threadIdx.x & 31;
    unsigned st = 0;
    // every loop bound is uniform across the block, so whole warps reach the
    // warp-aggregated histogram update together
    for (int64_t z = blockIdx.z; z < q.n[0] * q.n[1]; z += gridDim.z)
        for (int64_t y = blockIdx.y, i0 = z / q.n[1], i1 = z - i0 * q.n[1]; y < q.n[2];
             y += gridDim.y)
            for (int64_t xb = blockIdx.x * (int64_t)blockDim.x; xb < q.n[3];
                 xb += (int64_t)gridDim.x * blockDim.x) {
                const int64_t x = xb + threadIdx.x;
                int s = -1;
                if (x < q.n[3]) {
                    const int64_t i[4] = {i0, i1, y, x};
                    const NodeInfo ni = node_info(q, i);
                    if (!ni.skip) {
                        int32_t qo = 0;
                        quantize_value(c[ni.addr], inv_w, ws, w, s, qo, st);
                        const int64_t p = q.sym_off + ni.rank;
                        sym[p] = (uint16_t)s;
                        if (s == MGARD_ESC) esc[p] = qo;
                    }
                }
                const unsigned grp = __match_any_sync(0xffffffffu, s);
                if (s >= 0 && lane == __ffs(grp) - 1) atomicAdd(&sh[s], (unsigned)__popc(grp));
            }
    __syncthreads();
    for (int k = threadIdx.x; k < DICT; k += blockDim.x)
        if (sh[k]) atomicAdd(&hist[k], (unsigned long long)sh[k]);
    if (st) atomicOr(status, st);
}

template <typename T>
__global__ void k_dequantize(const uint16_t* __restrict__ sym, const int32_t* __restrict__ esc,
                             QLevel q, T wt, double w, T* __restrict__ c) {
    const WidthSplit ws = split_width(w);
    FOR_NODES(q.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        const NodeInfo ni = node_info(q, i);
        if (ni.skip) {
            if (!q.pos[0]) c[ni.addr] = T(0);   // compact level array: z = 0 on coarse nodes
            continue;
        }
        const int64_t p = q.sym_off + ni.rank;
        const int s = sym[p];
        T v;
        if (s == MGARD_ESC) v = dequant_escape<T>(esc[p], wt, ws, w);
        else if (sizeof(T) == 4) v = (T)__fmul_rn((float)(s - RADIUS), (float)wt);
        else v = (T)((double)(s - RADIUS) * w);
        c[ni.addr] = v;
    }
}

// Coefficient statistics of one level (predictor features; the row kernel
// k3_features computes the same on shapes of up to three axes).
template <typename T>
__global__ void __launch_bounds__(QT) k_features(const T* __restrict__ c, QLevel q,
                                                 const double* __restrict__ amax,
                                                 FeatPart* __restrict__ part) {
    __shared__ unsigned hist[FEAT_BINS];
    if (threadIdx.x < FEAT_BINS) hist[threadIdx.x] = 0;
    __syncthreads();
    const double a = *amax > 0.0 ? *amax : 1.0;
    const float inv_a = (float)(1.0 / a);
    double sum = 0.0, sum2 = 0.0;
    FOR_NODES(q.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        const NodeInfo ni = node_info(q, i);
        if (ni.skip) continue;
        const float rr = log10f(fmaxf(fabsf((float)c[ni.addr]) * inv_a, 1e-12f));
        sum += (double)rr;
        sum2 += (double)rr * (double)rr;
        atomicAdd(&hist[min(max((int)ceilf(-2.f * rr), 0), FEAT_BINS - 1)], 1u);
    }
    __shared__ double sh[2][QT];
    sh[0][threadIdx.x] = sum;
    sh[1][threadIdx.x] = sum2;
    __syncthreads();
    for (int o = QT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (threadIdx.x < FEAT_BINS) part[b].hist[threadIdx.x] = hist[threadIdx.x];
    if (threadIdx.x == 0) {
        part[b].sum = sh[0][0];
        part[b].sum2 = sh[1][0];
    }
}

// Quantization of coefficients held in symbol order (all levels in one
// pass): eight consecutive values per thread with vector loads and one
// 16-byte store of their symbols; the level of each value comes from the
// offsets (a group may straddle two levels).  Same decisions as k_quantize.
// Escape values are stored compacted per Huffman sub-chunk (256 symbols, the
// span of one warp per iteration): the r-th escape of sub-chunk s (in symbol
// order) at esc[s * 256 + r], placed by a warp scan of the lanes' counts.
constexpr int QS_THREADS = 256;
constexpr int QS_SUB = SUB;   // symbols per Huffman sub-chunk
static_assert(QS_SUB == 32 * 8, "a warp covers one sub-chunk per iteration");

template <typename T>
__global__ void __launch_bounds__(QS_THREADS, sizeof(T) == 4 ? 4 : 3) k_quantize_stream(
    const T* __restrict__ zs, int64_t n, LevelOffsets lo, const double* __restrict__ wdev,
    uint16_t* __restrict__ sym, int32_t* __restrict__ esc, unsigned long long* __restrict__ hist,
    unsigned* status, int64_t g_begin) {
    __shared__ unsigned sh[2][DICT];
    __shared__ double ws[MAX_LEVELS + 1];
    __shared__ T iws[MAX_LEVELS + 1];
    __shared__ WidthSplit wss[MAX_LEVELS + 1];
    __shared__ long long offs[MAX_LEVELS + 2];
    for (int k = threadIdx.x; k < 2 * DICT; k += QS_THREADS) (&sh[0][0])[k] = 0;
    for (int l = threadIdx.x; l <= lo.L; l += QS_THREADS) {
        ws[l] = wdev[l];
        iws[l] = (T)(1.0 / wdev[l]);
        wss[l] = split_width(wdev[l]);
    }
    for (int l = threadIdx.x; l <= lo.L + 1; l += QS_THREADS) offs[l] = lo.off[l];
    __syncthreads();
    const int L = lo.L;
    const int lane = threadIdx.x & 31;
    unsigned* my = sh[threadIdx.x & 1];
    unsigned center = 0, st = 0;
    // the eight values from i0 (zeros past the end)
    auto load8 = [&](int64_t i0, T* v) {
        if (i0 >= n) {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = T(0);
        } else if (i0 + 8 <= n) {
            if (sizeof(T) == 4) {
                const float4 a = reinterpret_cast<const float4*>(zs + i0)[0];
                const float4 b = reinterpret_cast<const float4*>(zs + i0)[1];
                v[0] = (T)a.x; v[1] = (T)a.y; v[2] = (T)a.z; v[3] = (T)a.w;
                v[4] = (T)b.x; v[5] = (T)b.y; v[6] = (T)b.z; v[7] = (T)b.w;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double2 a = reinterpret_cast<const double2*>(zs + i0)[k];
                    v[2 * k] = (T)a.x;
                    v[2 * k + 1] = (T)a.y;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = i0 + k < n ? zs[i0 + k] : T(0);
        }
    };
    const int64_t stride = (int64_t)gridDim.x * QS_THREADS;
    // a thread's groups come in increasing order, so its level only moves
    // forward: the search resumes where the previous group left it
    int lcur = 0;
    // the next group's values are loaded while this group is quantized
    T nxt[8];
    load8((g_begin + blockIdx.x * (int64_t)QS_THREADS + threadIdx.x) * 8, nxt);
    // block-uniform trip count (the escape scan needs whole warps)
    for (int64_t gb = g_begin + blockIdx.x * (int64_t)QS_THREADS; gb * 8 < n; gb += stride) {
        const int64_t g = gb + threadIdx.x;
        const int64_t i0 = g * 8;
        T v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = nxt[k];
        if ((gb + stride) * 8 < n) load8((g + stride) * 8, nxt);
        int32_t qe[8];      // escape values by slot
        unsigned emask = 0;  // slots holding escapes
        // the level of the group's first value; its width stays in registers
        // until a value crosses into the next level (rare)
        while (lcur < L && i0 >= offs[lcur + 1]) ++lcur;
        int l = lcur;
        long long lend = offs[l + 1];
        double wl = ws[l];
        T iwl = iws[l];
        WidthSplit wsl = wss[l];
        const bool full = i0 + 8 <= n;
        uint32_t packed[4] = {0, 0, 0, 0};
        // the usual group lies inside one level and inside the array
        const bool plain = full && i0 + 8 <= lend;
        if (sizeof(T) == 4 && plain) {
            // quantize_value's decisions without per-value branches: a
            // value escapes when |q| reaches RADIUS (or is NaN), and only
            // non-finite values and |q| >= 2^12 take the longer rules
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float q = rintf(__fmul_rn((float)v[k], (float)iwl));
                const float a = fabsf(q);
                const bool e = !(a < (float)RADIUS);
                int32_t qo = (int32_t)q;
                if (e && !(a < (float)F32_EXACT)) {
                    if (!isfinite((float)v[k])) {
                        st |= ST_NONFINITE;
                        qo = 0;
                    } else if (!quant_big((float)v[k], wsl, wl, qo)) {
                        st |= ST_RANGE;
                        qo = 0;
                    }
                }
                const int s = e ? (int)MGARD_ESC : (int)q + RADIUS;
                packed[k >> 1] |= (uint32_t)s << (16 * (k & 1));
                qe[k] = qo;
                emask |= (unsigned)e << k;
                if (s == RADIUS) ++center;
                else atomicAdd(&my[s], 1u);
            }
        } else
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t i = i0 + k;
            if (!plain && i >= n) break;
            if (!plain && i >= lend) {
                while (l < L && i >= offs[l + 1]) ++l;
                lend = offs[l + 1];
                wl = ws[l];
                iwl = iws[l];
                wsl = wss[l];
            }
            int s;
            int32_t qo = 0;
            quantize_value(v[k], iwl, wsl, wl, s, qo, st);
            packed[k >> 1] |= (uint32_t)s << (16 * (k & 1));
            qe[k] = qo;
            emask |= (unsigned)(s == MGARD_ESC) << k;
            if (s == RADIUS) ++center;
            else atomicAdd(&my[s], 1u);
        }
        if (full) {
            *reinterpret_cast<uint4*>(sym + i0) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        } else {
            for (int k = 0; k < 8 && i0 + k < n; ++k)
                sym[i0 + k] = (uint16_t)(packed[k >> 1] >> (16 * (k & 1)));
        }
        // place of this thread's first escape inside its sub-chunk: exclusive
        // scan over the warp
        const unsigned ne = __popc(emask);
        unsigned inc = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (emask) {
            int32_t* dst = esc + (i0 & ~(int64_t)(QS_SUB - 1)) + (inc - ne);
#pragma unroll
            for (int k = 0; k < 8; ++k)   // escapes in slot order
                if ((emask >> k) & 1u) *dst++ = qe[k];
        }
    }
    if (center) atomicAdd(&sh[0][RADIUS], center);
    __syncthreads();
    for (int k = threadIdx.x; k < DICT; k += QS_THREADS) {
        const unsigned v = sh[0][k] + sh[1][k];
        if (v) atomicAdd(&hist[k], (unsigned long long)v);
    }
    if (st) atomicOr(status, st);
}

// The same statistics over a contiguous run of coefficients (one level in
// symbol order).
constexpr int FR_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(FR_THREADS) k_features_range(const T* __restrict__ c, int64_t n,
                                                               const double* __restrict__ amax,
                                                               FeatPart* __restrict__ part) {
    __shared__ unsigned hist[FR_THREADS / 32][FEAT_BINS];
    for (int k = threadIdx.x; k < (FR_THREADS / 32) * FEAT_BINS; k += FR_THREADS) (&hist[0][0])[k] = 0;
    __syncthreads();
    const double a = *amax > 0.0 ? *amax : 1.0;
    const float inv_a = (float)(1.0 / a);
    const int warp = threadIdx.x >> 5;
    double sum = 0.0, sum2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)FR_THREADS + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * FR_THREADS) {
        const float rr = log10f(fmaxf(fabsf((float)c[i]) * inv_a, 1e-12f));
        sum += (double)rr;
        sum2 += (double)rr * (double)rr;
        atomicAdd(&hist[warp][min(max((int)ceilf(-2.f * rr), 0), FEAT_BINS - 1)], 1u);
    }
    __shared__ double sh[2][FR_THREADS];
    sh[0][threadIdx.x] = sum;
    sh[1][threadIdx.x] = sum2;
    __syncthreads();
    for (int o = FR_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < FEAT_BINS) {
        unsigned long long h = 0;
        for (int w = 0; w < FR_THREADS / 32; ++w) h += hist[w][threadIdx.x];
        part[blockIdx.x].hist[threadIdx.x] = h;
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x].sum = sh[0][0];
        part[blockIdx.x].sum2 = sh[1][0];
    }
}

int64_t range_feature_blocks(int64_t n) {
    const int64_t b = (n + 8 * FR_THREADS - 1) / (8 * FR_THREADS);
    return b < 1 ? 1 : (b > 148 * 4 ? 148 * 4 : b);
}

QLevel make_qlevel(const Plan& p, int l, bool inplace) {
    QLevel q{};
    int64_t nc[4];
    for (int a = 0; a < 4; ++a) nc[a] = l > 0 ? p.shape[l - 1][a] : p.shape[l][a];
    for (int a = 0; a < 4; ++a) {
        q.n[a] = p.shape[l][a];
        q.tail[a] = 1;
        for (int b = a + 1; b < 4; ++b) q.tail[a] *= nc[b];
        q.fine[a] = p.n4[a];
        q.pos[a] = inplace ? p.lidx[l].pos[a] : nullptr;
        if (l > 0) {
            q.fcls[a] = p.lf[l].ax[a].fcls;
            q.cbefore[a] = p.lf[l].ax[a].cbefore;
        }
    }
    q.tables = l > 0 ? 1 : 0;
    q.sym_off = p.offset[l];
    return q;
}

}  // namespace

LevelOffsets level_offsets(const Plan& p) {
    LevelOffsets lo;
    std::memset(&lo, 0, sizeof(lo));
    lo.L = p.L;
    for (int l = 0; l <= p.L; ++l) lo.off[l] = p.offset[l];
    lo.off[p.L + 1] = p.total();
    return lo;
}

template <typename T>
mgard_status quantize_stream(const Plan& p, const T* zs, const double* w, uint16_t* sym,
                             int32_t* esc, unsigned long long* hist, unsigned* status,
                             cudaStream_t st, int64_t i_begin, int64_t i_end, bool spare_sm) {
    const int64_t n = i_end < 0 ? p.total() : std::min<int64_t>(i_end, p.total());
    if (p.L > MAX_LEVELS) {
        set_error("too many levels");
        return MGARD_ESHAPE;
    }
    if (i_begin % QS_SUB != 0 || i_begin < 0) {
        set_error("quantize_stream: range must start on a sub-chunk");
        return MGARD_EINVAL;
    }
    if (i_begin >= n) return MGARD_OK;
    const int64_t groups = (n - i_begin + 8 * QS_THREADS - 1) / (8 * QS_THREADS);
    int grid = 0;
    MGB_TRY(resident_grid((const void*)k_quantize_stream<T>, QS_THREADS, 0, groups, &grid));
    if (spare_sm) {
        int per_sm = 0, sms = 0, dev = 0;
        MGB_CUDA(cudaGetDevice(&dev));
        MGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_quantize_stream<T>, QS_THREADS, 0));
        grid = std::max(1, std::min(grid, (sms - 1) * std::max(per_sm, 1)));
    }
    MGB_LAUNCH("k_quantize_stream", st, k_quantize_stream<T><<<grid, QS_THREADS, 0, st>>>(
                                            zs, n, level_offsets(p), w, sym, esc, hist, status,
                                            i_begin / 8));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}
template mgard_status quantize_stream<float>(const Plan&, const float*, const double*, uint16_t*,
                                             int32_t*, unsigned long long*, unsigned*, cudaStream_t,
                                             int64_t, int64_t, bool);
template mgard_status quantize_stream<double>(const Plan&, const double*, const double*, uint16_t*,
                                              int32_t*, unsigned long long*, unsigned*, cudaStream_t,
                                              int64_t, int64_t, bool);

int64_t feature_blocks(const Plan& p, int l) {
    if (rows3_ok(p)) return range_feature_blocks(p.count[l]);
    const QLevel q = make_qlevel(p, l, false);
    const dim3 g = grid3(q.n, QT, 32, 32);
    return (int64_t)g.x * g.y * g.z;
}

template <typename T>
mgard_status level_features(const Plan& p, int l, const T* c, const double* amax, FeatPart* part,
                            cudaStream_t st) {
    if (rows3_ok(p)) {   // c: the level's run of coefficients in symbol order
        MGB_LAUNCH("k_features_range", st, k_features_range<T><<<(int)range_feature_blocks(p.count[l]), FR_THREADS, 0, st>>>(
                                               c, p.count[l], amax, part));
        MGB_CUDA(cudaGetLastError());
        return MGARD_OK;
    }
    const QLevel q = make_qlevel(p, l, false);
    MGB_LAUNCH("k_features", st, k_features<T><<<grid3(q.n, QT, 32, 32), QT, 0, st>>>(c, q, amax, part));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}
template mgard_status level_features<float>(const Plan&, int, const float*, const double*,
                                            FeatPart*, cudaStream_t);
template mgard_status level_features<double>(const Plan&, int, const double*, const double*,
                                             FeatPart*, cudaStream_t);

template <typename T>
mgard_status quantize_level(const Plan& p, int l, const T* c, bool inplace, const double* w,
                            uint16_t* sym, int32_t* esc, unsigned long long* hist,
                            unsigned* status, cudaStream_t st) {
    if (!inplace && rows3_ok(p)) return rows3_quantize<T>(p, l, c, w, sym, esc, hist, status, st);
    QLevel q = make_qlevel(p, l, inplace);
    MGB_LAUNCH("k_quantize", st, k_quantize<T><<<grid3(q.n, QT, 32, 32), QT, 0, st>>>(c, q, w, sym, esc, hist, status));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status dequantize_level(const Plan& p, int l, const uint16_t* sym, const int32_t* esc,
                              bool inplace, double w, T* c, cudaStream_t st) {
    if (!inplace && rows3_ok(p)) return rows3_dequantize<T>(p, l, sym, esc, w, c, st);
    QLevel q = make_qlevel(p, l, inplace);
    MGB_LAUNCH("k_dequantize", st, k_dequantize<T><<<grid3(q.n, 128), 128, 0, st>>>(sym, esc, q, (T)w, w, c));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

#define INST(T)                                                                                  \
    template mgard_status quantize_level<T>(const Plan&, int, const T*, bool, const double*, uint16_t*, \
                                            int32_t*, unsigned long long*, unsigned*,            \
                                            cudaStream_t);                                       \
    template mgard_status dequantize_level<T>(const Plan&, int, const uint16_t*, const int32_t*, \
                                              bool, double, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

// -- region-adaptive widths -------------------------------------------------

namespace {

__device__ inline int region_k(const RegionLevel& rg, const int64_t* g) {
    int k = 0;
    for (int r = 0; r < rg.n; ++r) {
        bool in = true;
#pragma unroll
        for (int a = 0; a < 4; ++a) in = in && g[a] >= rg.lo[r][a] && g[a] <= rg.hi[r][a];
        if (in) k = max(k, rg.k[r]);
    }
    return k;
}

// 2^e as an exact float / double (|e| well inside the normal range).
__device__ inline float pow2(float, int e) { return __int_as_float((127 + e) << 23); }
__device__ inline double pow2(double, int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Scale the level-l coefficients (symbol order at q.sym_off + rank, or the
// compact level array) by 2^(sign k) of their node.
template <typename T>
__global__ void k_region_scale(T* __restrict__ c, QLevel q, LevelIndex li, RegionLevel rg,
                               int sign, int symbol_order) {
    FOR_NODES(q.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        const NodeInfo ni = node_info(q, i);
        if (ni.skip) continue;
        int64_t g[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) g[a] = li.pos[a][i[a]];
        const int k = region_k(rg, g);
        if (!k) continue;
        T* v = c + (symbol_order ? q.sym_off + ni.rank : ni.addr);
        *v *= pow2(T(0), sign * k);
    }
}

// k of every node of level l, written at its input-grid position.
__global__ void k_region_exponents(uint8_t* __restrict__ out, QLevel q, LevelIndex li,
                                   RegionLevel rg) {
    FOR_NODES(q.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        const NodeInfo ni = node_info(q, i);
        if (ni.skip) continue;
        int64_t g[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) g[a] = li.pos[a][i[a]];
        out[ravel4(g, q.fine)] = (uint8_t)region_k(rg, g);
    }
}

}  // namespace

template <typename T>
mgard_status region_scale(const Plan& p, const RegionScale& rs, T* zs, T* const* levels, int sign,
                          cudaStream_t st) {
    if ((int)rs.lv.size() != p.L + 1) {
        set_error("region table does not match the levels");
        return MGARD_EINVAL;
    }
    for (int l = 0; l <= p.L; ++l) {
        if (!rs.lv[l].n) continue;
        const QLevel q = make_qlevel(p, l, false);
        T* c = zs ? zs : levels[l];
        MGB_LAUNCH("k_region_scale", st, k_region_scale<T><<<grid3(q.n, 128), 128, 0, st>>>(
                                             c, q, p.lidx[l], rs.lv[l], sign, zs ? 1 : 0));
        MGB_CUDA(cudaGetLastError());
    }
    return MGARD_OK;
}
template mgard_status region_scale<float>(const Plan&, const RegionScale&, float*, float* const*,
                                          int, cudaStream_t);
template mgard_status region_scale<double>(const Plan&, const RegionScale&, double*, double* const*,
                                           int, cudaStream_t);

mgard_status region_exponents(const Plan& p, const RegionScale& rs, uint8_t* k, cudaStream_t st) {
    if ((int)rs.lv.size() != p.L + 1) {
        set_error("region table does not match the levels");
        return MGARD_EINVAL;
    }
    for (int l = 0; l <= p.L; ++l) {
        QLevel q = make_qlevel(p, l, false);
        for (int a = 0; a < 4; ++a) q.fine[a] = p.n4[a];
        MGB_LAUNCH("k_region_exponents", st, k_region_exponents<<<grid3(q.n, 128), 128, 0, st>>>(
                                                 k, q, p.lidx[l], rs.lv[l]));
        MGB_CUDA(cudaGetLastError());
    }
    return MGARD_OK;
}

}  // namespace mgb
