// The small levels of a pyramid in one launch.
//
// Below a few thousand nodes a level's kernels are too small to fill the
// GPU, and each costs a launch.  k_tail_decompose / k_tail_recompose run
// every level l <= Lt (level_size(l) <= TAIL_NODES) in a single block of
// 1024 threads: the same steps as the per-level kernels (Section 3 of the
// paper: interpolation coefficients z = u - I u, load vector P^T M_l z by
// restriction along x, y and z, tridiagonal solves along z, y and x, and
// the correction of the coarse level), each a block-strided loop over the
// level's nodes, separated by block barriers.  Every level's nodal values
// and the scratch arrays live in shared memory (a few tens of KB); global
// memory sees the top level's values coming in, the coefficients going out
// and the pyramid's arrays written back.  Shapes are the row kernels' (axes
// 1..3 of the 4D view); an inactive axis (extent 1) is skipped.
#include <algorithm>
#include <cstring>

#include "multilevel.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

constexpr int TAIL_THREADS = 1024;

template <typename T>
struct TailArgs {
    int Lt;                               // levels 1..Lt run here
    Level<T> lv[TAIL_LEVELS + 1];         // [l] transition l -> l-1 (l >= 1)
    T* g[TAIL_LEVELS + 1];                // [l] level l's array in global memory
    int size[TAIL_LEVELS + 1];            // [l] nodes of level l
    long long off[TAIL_LEVELS + 1];       // [l] symbol offset of level l's new nodes
    T* zs;                                // coefficients in symbol order, or null:
    T* zl[TAIL_LEVELS + 1];               // [l] level l's coefficients in its own row-major array
    int su[TAIL_LEVELS + 1];              // shared-memory offsets (elements): level l's values,
    int szz, st0, st1;                    // a level's coefficients, restriction scratch
};

// Views of the shared-memory arrays.
template <typename T>
struct TailMem {
    T* u[TAIL_LEVELS + 1];
    T *zz, *t0, *t1;
};

// Position of a node among level l's new nodes (row-major order of the
// level grid without the nodes of the coarser grid).
template <typename T>
__device__ inline long long new_rank(const Level<T>& lv, int z, int y, int x) {
    const long long nx = lv.n[3], ny = lv.n[2];
    const long long ncx = lv.nc[3], ncy = lv.nc[2];
    const bool zc = !lv.ax[1].fcls || lv.ax[1].fcls[z] >= 0;
    const bool yc = !lv.ax[2].fcls || lv.ax[2].fcls[y] >= 0;
    const long long cz = lv.ax[1].cbefore ? lv.ax[1].cbefore[z] : 0;
    const long long cy = lv.ax[2].cbefore ? lv.ax[2].cbefore[y] : 0;
    const long long cx = lv.ax[3].cbefore ? lv.ax[3].cbefore[x] : 0;
    long long before = cz * ncy * ncx;
    if (zc) {
        before += cy * ncx;
        if (yc) before += cx;
    }
    return ((long long)z * ny + y) * nx + x - before;
}

// Interpolation from coarse nodes along one axis at fine index i: the
// coarse node itself (J, weight 1), or the two around a new node.
template <typename T>
struct Taps {
    int n;          // 1 or 2
    int J[2];       // coarse indices
    int F[2];       // their fine positions
    T w[2];
};
template <typename T>
__device__ inline Taps<T> taps(const AxisT<T>& ax, int i) {
    Taps<T> t;
    t.n = 1;
    t.J[0] = t.J[1] = i;
    t.F[0] = t.F[1] = i;
    t.w[0] = T(1);
    t.w[1] = T(0);
    if (!ax.fcls) return t;
    const int c = ax.fcls[i];
    if (c >= 0) {
        t.J[0] = c;
        return t;
    }
    const int left = -c - 1;
    t.n = 2;
    t.J[0] = left;
    t.J[1] = left + 1;
    t.F[0] = ax.rf[left];
    t.F[1] = ax.rf[left + 1];
    t.w[0] = ax.wl[i];
    t.w[1] = ax.wr[i];
    return t;
}

// One axis' five-tap restriction at coarse index J from `get(ip)` (fine ip).
template <typename T, typename G>
__device__ inline T restrict_at(const AxisT<T>& ax, int J, int m, G get) {
    const int f = ax.rf[J];
    T acc = T(0);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int ip = f - 2 + t;
        if (ip < 0 || ip >= m) continue;
        acc += ax.rw[J * 5 + t] * get(ip);
    }
    return acc;
}

// coarse += sign * M^{-1} P^T M z for level l (z in m.zz, row-major).
template <typename T>
__device__ void tail_correct(const TailArgs<T>& ga, const TailMem<T>& a, int l, T sign) {
    const Level<T>& lv = ga.lv[l];
    const int nz = (int)lv.n[1], ny = (int)lv.n[2], nx = (int)lv.n[3];
    const int ncz = (int)lv.nc[1], ncy = (int)lv.nc[2], ncx = (int)lv.nc[3];
    const bool az = lv.ax[1].fcls, ay = lv.ax[2].fcls, ax = lv.ax[3].fcls;
    const int tid = threadIdx.x;
    // restriction along x: t0 (nz, ny, ncx)
    for (int k = tid; k < nz * ny * ncx; k += TAIL_THREADS) {
        const int J = k % ncx, r = k / ncx;
        const T* row = a.zz + (long long)r * nx;
        a.t0[k] = ax ? restrict_at(lv.ax[3], J, nx, [&](int ip) { return row[ip]; }) : row[J];
    }
    __syncthreads();
    // along y: t1 (nz, ncy, ncx)
    for (int k = tid; k < nz * ncy * ncx; k += TAIL_THREADS) {
        const int x = k % ncx, Jy = (k / ncx) % ncy, z = k / (ncx * ncy);
        const T* col = a.t0 + (long long)z * ny * ncx + x;
        a.t1[k] = ay ? restrict_at(lv.ax[2], Jy, ny, [&](int ip) { return col[(long long)ip * ncx]; })
                     : col[(long long)Jy * ncx];
    }
    __syncthreads();
    // along z: t0 (ncz, ncy, ncx)
    for (int k = tid; k < ncz * ncy * ncx; k += TAIL_THREADS) {
        const int xy = k % (ncy * ncx), Jz = k / (ncy * ncx);
        const T* col = a.t1 + xy;
        a.t0[k] = az ? restrict_at(lv.ax[1], Jz, nz, [&](int ip) { return col[(long long)ip * ncy * ncx]; })
                     : col[(long long)Jz * ncy * ncx];
    }
    __syncthreads();
    // Thomas along one axis for the lines of `b` (m nodes, `stride` apart)
    auto thomas = [&](const AxisT<T>& axt, T* b, int m, long long stride) {
        T y = T(0);
        for (int k = 0; k < m; ++k) {
            y = (b[k * stride] - axt.tsub[k] * y) * axt.tinv[k];
            b[k * stride] = y;
        }
        T x = T(0);
        for (int k = m - 1; k >= 0; --k) {
            x = (k == m - 1) ? b[k * stride] : b[k * stride] - axt.tcp[k] * x;
            b[k * stride] = x;
        }
    };
    if (az) {
        for (int k = tid; k < ncy * ncx; k += TAIL_THREADS) thomas(lv.ax[1], a.t0 + k, ncz, (long long)ncy * ncx);
        __syncthreads();
    }
    if (ay) {
        for (int k = tid; k < ncz * ncx; k += TAIL_THREADS) {
            const int x = k % ncx, Jz = k / ncx;
            thomas(lv.ax[2], a.t0 + (long long)Jz * ncy * ncx + x, ncy, ncx);
        }
        __syncthreads();
    }
    if (ax) {
        for (int k = tid; k < ncz * ncy; k += TAIL_THREADS) thomas(lv.ax[3], a.t0 + (long long)k * ncx, ncx, 1);
        __syncthreads();
    }
    T* c = a.u[l - 1];
    for (int k = tid; k < ncz * ncy * ncx; k += TAIL_THREADS) c[k] += sign * a.t0[k];
    __syncthreads();
}

template <typename T>
__device__ inline TailMem<T> tail_mem(const TailArgs<T>& a) {
    extern __shared__ __align__(16) unsigned char tail_raw[];
    T* base = reinterpret_cast<T*>(tail_raw);
    TailMem<T> m;
    for (int l = 0; l <= TAIL_LEVELS; ++l) m.u[l] = base + a.su[l];
    m.zz = base + a.szz;
    m.t0 = base + a.st0;
    m.t1 = base + a.st1;
    return m;
}

template <typename T>
__device__ void tail_decompose_body(const TailArgs<T>& a) {
    const TailMem<T> m = tail_mem(a);
    for (int k = threadIdx.x; k < a.size[a.Lt]; k += TAIL_THREADS) m.u[a.Lt][k] = a.g[a.Lt][k];
    __syncthreads();
    for (int l = a.Lt; l >= 1; --l) {
        const Level<T>& lv = a.lv[l];
        const int nz = (int)lv.n[1], ny = (int)lv.n[2], nx = (int)lv.n[3];
        const int ncy = (int)lv.nc[2], ncx = (int)lv.nc[3];
        const T* u = m.u[l];
        T* c = m.u[l - 1];
        // coefficients z = u - I u on new nodes; coarse nodes copied down
        for (int k = threadIdx.x; k < nz * ny * nx; k += TAIL_THREADS) {
            const int x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
            const Taps<T> tz = taps(lv.ax[1], z), ty = taps(lv.ax[2], y), tx = taps(lv.ax[3], x);
            if (tz.n == 1 && ty.n == 1 && tx.n == 1) {
                c[((long long)tz.J[0] * ncy + ty.J[0]) * ncx + tx.J[0]] = u[k];
                m.zz[k] = T(0);
                continue;
            }
            T acc = T(0);
            for (int i = 0; i < tz.n; ++i)
                for (int j = 0; j < ty.n; ++j)
                    for (int h = 0; h < tx.n; ++h)
                        acc += tz.w[i] * ty.w[j] * tx.w[h] *
                               u[((long long)tz.F[i] * ny + ty.F[j]) * nx + tx.F[h]];
            const T zv = u[k] - acc;
            m.zz[k] = zv;
            if (a.zs) a.zs[a.off[l] + new_rank(lv, z, y, x)] = zv;
            else a.zl[l][k] = zv;
        }
        __syncthreads();
        tail_correct(a, m, l, T(1));
    }
    // the pyramid's arrays: every level's nodal values in symbol order (the
    // caller may take level energies from them); in place only level 0,
    // whose array is not also a coefficient array
    for (int l = 0; l < a.Lt; ++l) {
        if (!a.zs && l > 0) break;
        for (int k = threadIdx.x; k < a.size[l]; k += TAIL_THREADS) a.g[l][k] = m.u[l][k];
    }
}

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_decompose(TailArgs<T> a) {
    tail_decompose_body(a);
}

// The tails of many fields: a persistent grid whose blocks take one field
// at a time from a device counter (one atomicAdd per job, no waits between
// blocks), each job the same steps as k_tail_decompose on that field.
template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_decompose_batch(const TailArgs<T>* jobs,
                                                                       int n, unsigned* next) {
    __shared__ int job;
    for (;;) {
        if (threadIdx.x == 0) job = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int j = job;
        __syncthreads();   // every thread holds j before the next job is taken
        if (j >= n) return;
        tail_decompose_body(jobs[j]);
        __syncthreads();   // the shared arrays are reused by the next job
    }
}

template <typename T>
__device__ void tail_recompose_body(const TailArgs<T>& a) {
    const TailMem<T> m = tail_mem(a);
    for (int k = threadIdx.x; k < a.size[0]; k += TAIL_THREADS) m.u[0][k] = a.g[0][k];
    __syncthreads();
    for (int l = 1; l <= a.Lt; ++l) {
        const Level<T>& lv = a.lv[l];
        const int nz = (int)lv.n[1], ny = (int)lv.n[2], nx = (int)lv.n[3];
        const int ncy = (int)lv.nc[2], ncx = (int)lv.nc[3];
        for (int k = threadIdx.x; k < nz * ny * nx; k += TAIL_THREADS) {
            const int x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
            const bool coarse = (!lv.ax[1].fcls || lv.ax[1].fcls[z] >= 0) &&
                                (!lv.ax[2].fcls || lv.ax[2].fcls[y] >= 0) &&
                                (!lv.ax[3].fcls || lv.ax[3].fcls[x] >= 0);
            m.zz[k] = coarse ? T(0) : (a.zs ? a.zs[a.off[l] + new_rank(lv, z, y, x)] : a.zl[l][k]);
        }
        __syncthreads();
        tail_correct(a, m, l, T(-1));
        // u_l = I u_{l-1} + z
        const T* c = m.u[l - 1];
        T* u = m.u[l];
        for (int k = threadIdx.x; k < nz * ny * nx; k += TAIL_THREADS) {
            const int x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
            const Taps<T> tz = taps(lv.ax[1], z), ty = taps(lv.ax[2], y), tx = taps(lv.ax[3], x);
            T acc = T(0);
            for (int i = 0; i < tz.n; ++i)
                for (int j = 0; j < ty.n; ++j)
                    for (int h = 0; h < tx.n; ++h)
                        acc += tz.w[i] * ty.w[j] * tx.w[h] *
                               c[((long long)tz.J[i] * ncy + ty.J[j]) * ncx + tx.J[h]];
            u[k] = acc + m.zz[k];
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < a.size[a.Lt]; k += TAIL_THREADS) a.g[a.Lt][k] = m.u[a.Lt][k];
}

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_recompose(TailArgs<T> a) {
    tail_recompose_body(a);
}

// The inverse for many fields, scheduled like k_tail_decompose_batch.
template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_recompose_batch(const TailArgs<T>* jobs,
                                                                       int n, unsigned* next) {
    __shared__ int job;
    for (;;) {
        if (threadIdx.x == 0) job = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int j = job;
        __syncthreads();
        if (j >= n) return;
        tail_recompose_body(jobs[j]);
        __syncthreads();
    }
}

template <typename T>
mgard_status make_args(const Plan& p, int Lt, Pyramid<T>& py, T* top_level, T* zs, T* ztop,
                       TailArgs<T>* a, size_t* smem) {
    if (Lt < 1 || Lt > TAIL_LEVELS) {
        set_error("tail levels out of range");
        return MGARD_EINVAL;
    }
    std::memset(a, 0, sizeof(*a));
    a->Lt = Lt;
    int off = 0;
    int64_t t0max = 1, t1max = 1;
    for (int l = 0; l <= Lt; ++l) {
        a->g[l] = l == Lt ? top_level : py.lv[l];
        a->size[l] = (int)p.level_size(l);
        a->off[l] = p.offset[l];
        a->zl[l] = l == p.L ? ztop : py.lv[l];   // in-place layout: coefficients over the level
        a->su[l] = off;
        off += a->size[l];
        if (l >= 1) {
            a->lv[l] = p.level<T>(l);
            const Level<T>& lv = a->lv[l];
            t0max = std::max<int64_t>(t0max, lv.n[1] * lv.n[2] * lv.nc[3]);
            t1max = std::max<int64_t>(t1max, lv.n[1] * lv.nc[2] * lv.nc[3]);
        }
    }
    for (int l = Lt + 1; l <= TAIL_LEVELS; ++l) a->su[l] = 0;
    a->szz = off;
    off += a->size[Lt];
    a->st0 = off;
    off += (int)t0max;
    a->st1 = off;
    off += (int)t1max;
    a->zs = zs;
    *smem = (size_t)off * sizeof(T);
    return MGARD_OK;
}

}  // namespace

int tail_levels(const Plan& p) {
    int Lt = 0;
    while (Lt < p.L && Lt < TAIL_LEVELS && p.level_size(Lt + 1) <= TAIL_NODES) ++Lt;
    return Lt;
}

template <typename T>
mgard_status tail_decompose(const Plan& p, int Lt, Pyramid<T>& py, const T* level_Lt, T* zs,
                            T* top, cudaStream_t st) {
    TailArgs<T> a;
    size_t smem = 0;
    MGB_TRY(make_args<T>(p, Lt, py, const_cast<T*>(level_Lt), zs, top, &a, &smem));
    MGB_TRY(allow_dynamic_smem((const void*)k_tail_decompose<T>, smem));
    MGB_LAUNCH("k_tail_decompose", st, k_tail_decompose<T><<<1, TAIL_THREADS, smem, st>>>(a));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status tail_recompose(const Plan& p, int Lt, Pyramid<T>& py, const T* zs, const T* top,
                            T* level_Lt, cudaStream_t st) {
    TailArgs<T> a;
    size_t smem = 0;
    MGB_TRY(make_args<T>(p, Lt, py, level_Lt, const_cast<T*>(zs), const_cast<T*>(top), &a, &smem));
    MGB_TRY(allow_dynamic_smem((const void*)k_tail_recompose<T>, smem));
    MGB_LAUNCH("k_tail_recompose", st, k_tail_recompose<T><<<1, TAIL_THREADS, smem, st>>>(a));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
size_t tail_args_bytes() {
    return sizeof(TailArgs<T>);
}

template <typename T>
mgard_status tail_job(const Plan& p, int Lt, Pyramid<T>& py, const T* level_Lt, T* zs, T* top,
                      void* args, size_t* smem) {
    return make_args<T>(p, Lt, py, const_cast<T*>(level_Lt), zs, top,
                        reinterpret_cast<TailArgs<T>*>(args), smem);
}

template <typename T>
mgard_status tail_decompose_batch(const void* jobs, int n, size_t smem, unsigned* counter,
                                  cudaStream_t st) {
    if (n <= 0) return MGARD_OK;
    int dev = 0, sms = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    MGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MGB_TRY(allow_dynamic_smem((const void*)k_tail_decompose_batch<T>, smem));
    MGB_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    MGB_LAUNCH("k_tail_decompose_batch", st,
               k_tail_decompose_batch<T><<<std::min(n, sms), TAIL_THREADS, smem, st>>>(
                   reinterpret_cast<const TailArgs<T>*>(jobs), n, counter));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status tail_recompose_batch(const void* jobs, int n, size_t smem, unsigned* counter,
                                  cudaStream_t st) {
    if (n <= 0) return MGARD_OK;
    int dev = 0, sms = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    MGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MGB_TRY(allow_dynamic_smem((const void*)k_tail_recompose_batch<T>, smem));
    MGB_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    MGB_LAUNCH("k_tail_recompose_batch", st,
               k_tail_recompose_batch<T><<<std::min(n, sms), TAIL_THREADS, smem, st>>>(
                   reinterpret_cast<const TailArgs<T>*>(jobs), n, counter));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

#define INST_TAIL_BATCH(T)                                                                       \
    template size_t tail_args_bytes<T>();                                                        \
    template mgard_status tail_job<T>(const Plan&, int, Pyramid<T>&, const T*, T*, T*, void*,    \
                                      size_t*);                                                  \
    template mgard_status tail_decompose_batch<T>(const void*, int, size_t, unsigned*,           \
                                                  cudaStream_t);                                 \
    template mgard_status tail_recompose_batch<T>(const void*, int, size_t, unsigned*,           \
                                                  cudaStream_t);
INST_TAIL_BATCH(float)
INST_TAIL_BATCH(double)
#undef INST_TAIL_BATCH

template mgard_status tail_decompose<float>(const Plan&, int, Pyramid<float>&, const float*, float*,
                                            float*, cudaStream_t);
template mgard_status tail_decompose<double>(const Plan&, int, Pyramid<double>&, const double*,
                                             double*, double*, cudaStream_t);
template mgard_status tail_recompose<float>(const Plan&, int, Pyramid<float>&, const float*,
                                            const float*, float*, cudaStream_t);
template mgard_status tail_recompose<double>(const Plan&, int, Pyramid<double>&, const double*,
                                             const double*, double*, cudaStream_t);

}  // namespace mgb
