// Level-wise linear quantization and its inverse, with a fused histogram.
//
// Paper, "Software design": every multilevel coefficient is approximated by
// an integer multiple of its level's bin width.  Symbols are laid out level
// by level (level 0 first), each level in row-major order of its grid,
// holding only the nodes new on that level.  |q| < DICT/2 maps to symbol
// q + DICT/2; larger values escape to symbol 0 with q stored aside.
#include "quantize.cuh"
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

__device__ inline void quantize_value(float c, float inv_w, double w, int& sym, int32_t& qo,
                                      unsigned& st) {
    if (!isfinite(c)) {
        st |= ST_NONFINITE;
        sym = MGARD_ESC;
        qo = 0;
        return;
    }
    const float x = __fmul_rn(c, inv_w);
    const float q = rintf(x);
    if (fabsf(q) < (float)RADIUS) {
        sym = (int)q + RADIUS;
        return;
    }
    sym = MGARD_ESC;
    if (fabsf(q) < (float)F32_EXACT) {
        qo = (int32_t)q;
        return;
    }
    const double qd = rint((double)c / w);
    if (fabs(qd) > 2147483647.0) {
        st |= ST_RANGE;
        qo = 0;
    } else {
        qo = (int32_t)qd;
    }
}

__device__ inline void quantize_value(double c, double /*inv_w*/, double w, int& sym, int32_t& qo,
                                      unsigned& st) {
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
                        quantize_value(c[ni.addr], inv_w, w, s, qo, st);
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
        if (s == MGARD_ESC) v = dequant_escape<T>(esc[p], wt, w);
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

int64_t feature_blocks(const Plan& p, int l) {
    if (rows3_ok(p)) return rows3_feature_blocks(p, l);
    const QLevel q = make_qlevel(p, l, false);
    const dim3 g = grid3(q.n, QT, 32, 32);
    return (int64_t)g.x * g.y * g.z;
}

template <typename T>
mgard_status level_features(const Plan& p, int l, const T* c, const double* amax, FeatPart* part,
                            cudaStream_t st) {
    if (rows3_ok(p)) return rows3_features<T>(p, l, c, amax, part, st);
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

}  // namespace mgb
