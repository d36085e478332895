// Multilevel decomposition and recomposition kernels.
//
// Paper, "Software design": u is decomposed recursively into multilevel
// coefficients over the grid hierarchy; recomposition is the inverse.
// One step from level l to l-1, on the P1 (piecewise multilinear) spaces:
//   1. coefficients  z = u_l - Pi_{l-1} u_l   (k_coeff_gather; also copies
//      the coarse nodal values into the compact level-(l-1) array)
//   2. load vector   b = P^T M_l z            (k_restrict, one axis at a time,
//      each pass shrinking that axis to the coarse extent)
//   3. coarse solve  M_{l-1} c = b             (k_solve_*, tridiagonal along
//      every axis; batched Thomas with precomputed factors)
//   4. correction    u_{l-1} = u_l|coarse + c (fused into the last solve)
// Recomposition runs 2-3 on the stored coefficients, subtracts the
// correction and refills the fine grid (k_fill).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include <cudaTypedefs.h>

#include "multilevel.cuh"
#include "rows3.cuh"
#include "tma.cuh"

namespace mgb {

namespace {

struct Shape4 {
    int64_t n[4];
};

struct Mask {
    const int* fcls[4];
    int on;
};

__host__ __device__ inline int64_t shape_prod(const Shape4& s) {
    return s.n[0] * s.n[1] * s.n[2] * s.n[3];
}

// -- step 1 -----------------------------------------------------------------
template <typename T>
__global__ void k_coeff_gather(const T* in, T* out, T* __restrict__ coarse, Level<T> lv) {
    FOR_NODES(lv.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        int64_t p0[4], p1[4], J[4];
        T w0[4], w1[4];
        int nc[4];
        bool allc = true;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int* fc = lv.ax[a].fcls;
            nc[a] = 1;
            p0[a] = p1[a] = i[a];
            w0[a] = T(1);
            w1[a] = T(0);
            J[a] = i[a];
            if (!fc) continue;
            const int c = fc[i[a]];
            if (c >= 0) {
                J[a] = c;
            } else {
                allc = false;
                const int left = -c - 1;
                p0[a] = lv.ax[a].rf[left];
                p1[a] = lv.ax[a].rf[left + 1];
                w0[a] = lv.ax[a].wl[i[a]];
                w1[a] = lv.ax[a].wr[i[a]];
                nc[a] = 2;
            }
        }
        const int64_t lin = ravel4(i, lv.n);
        const T u = in[lin];
        if (allc) {
            coarse[ravel4(J, lv.nc)] = u;
            continue;
        }
        T acc = T(0);
        for (int c0 = 0; c0 < nc[0]; ++c0)
            for (int c1 = 0; c1 < nc[1]; ++c1)
                for (int c2 = 0; c2 < nc[2]; ++c2)
                    for (int c3 = 0; c3 < nc[3]; ++c3) {
                        const int64_t q[4] = {c0 ? p1[0] : p0[0], c1 ? p1[1] : p0[1],
                                              c2 ? p1[2] : p0[2], c3 ? p1[3] : p0[3]};
                        const T w = (c0 ? w1[0] : w0[0]) * (c1 ? w1[1] : w0[1]) *
                                    (c2 ? w1[2] : w0[2]) * (c3 ? w1[3] : w0[3]);
                        acc += w * in[ravel4(q, lv.n)];
                    }
        out[lin] = u - acc;
    }
}

// -- step 2 -----------------------------------------------------------------
// Restriction along axis a; with mask.on the input is the fine grid and
// nodes of the coarse grid count as zero (z vanishes there) -- they are not
// even read, so stale values at those positions never matter.
template <typename Tin, typename Tout>
__global__ void k_restrict(const Tin* __restrict__ in, Tout* __restrict__ out, Shape4 sin, int a,
                           const int* __restrict__ rf, const Tout* __restrict__ rw, Shape4 so,
                           Mask mask) {
    FOR_NODES(so.n, o0, o1, o2, o3) {
        const int64_t o[4] = {o0, o1, o2, o3};
        bool others_coarse = true;
        if (mask.on) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (b != a && mask.fcls[b] && mask.fcls[b][o[b]] < 0) others_coarse = false;
        }
        const int64_t J = o[a];
        const int64_t f = rf[J];
        int64_t stride = 1;
        for (int b = 3; b > a; --b) stride *= sin.n[b];
        int64_t q[4] = {o[0], o[1], o[2], o[3]};
        q[a] = 0;
        const int64_t base = ravel4(q, sin.n);
        Tout acc = Tout(0);
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            const int64_t ip = f - 2 + t;
            if (ip < 0 || ip >= sin.n[a]) continue;
            const Tout w = rw[J * 5 + t];
            if (w == Tout(0)) continue;
            if (mask.on && others_coarse && mask.fcls[a][ip] >= 0) continue;
            acc += w * (Tout)in[base + ip * stride];
        }
        out[ravel4(o, so.n)] = acc;
    }
}

// -- step 3 (+4) --------------------------------------------------------------
// One thread per line along a non-contiguous axis a: lines are indexed by
// (outer, inner) with inner contiguous, so a warp reads 32 consecutive
// elements per step.  Loads are issued 8 at a time ahead of the recurrence.
template <typename Tw, typename Tdst>
__global__ void k_solve_lines(Tw* x, int64_t outer_n, int64_t m, int64_t stride,
                              const Tw* __restrict__ sub, const Tw* __restrict__ inv,
                              const Tw* __restrict__ cp, Tdst* dst, Tw sign) {
    constexpr int U = 8;
    for (int64_t outer = blockIdx.y; outer < outer_n; outer += gridDim.y)
        for (int64_t inner = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; inner < stride;
             inner += (int64_t)gridDim.x * blockDim.x) {
            Tw* base = x + outer * m * stride + inner;
            Tw y = Tw(0);
            for (int64_t k0 = 0; k0 < m; k0 += U) {
                Tw v[U];
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if (k0 + j < m) v[j] = base[(k0 + j) * stride];
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if (k0 + j < m) {
                        y = (v[j] - sub[k0 + j] * y) * inv[k0 + j];
                        v[j] = y;
                    }
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if (k0 + j < m) base[(k0 + j) * stride] = v[j];
            }
            Tdst* d = dst ? dst + outer * m * stride + inner : nullptr;
            Tw vnext = Tw(0);
            for (int64_t k1 = m; k1 > 0; k1 -= U) {
                const int64_t lo = k1 - U > 0 ? k1 - U : 0;
                Tw v[U], dv[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int64_t k = k1 - 1 - j;
                    if (k >= lo) {
                        v[j] = base[k * stride];
                        if (d) dv[j] = (Tw)d[k * stride];
                    }
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int64_t k = k1 - 1 - j;
                    if (k >= lo) {
                        vnext = (k == m - 1) ? v[j] : v[j] - cp[k] * vnext;
                        v[j] = vnext;
                    }
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int64_t k = k1 - 1 - j;
                    if (k >= lo) {
                        if (d) d[k * stride] = (Tdst)(dv[j] + sign * v[j]);
                        else base[k * stride] = v[j];
                    }
                }
            }
        }
}

// One line solved by a warp: lane j holds elements [k0, k0+E) of the line
// (k0 = jE) in v and replaces them with the solution of the tridiagonal
// system.  Both Thomas sweeps are first-order affine recurrences (y_k =
// alpha_k y_{k-1} + beta_k forward, x_k = gamma_k x_{k+1} + y_k backward),
// so each lane composes the maps of its segment, the warp scans the
// compositions with shuffles, and each lane replays its segment from the
// scanned input.  SUB/INV/CP(k) give the factors of element k0 + k.
template <typename Tw, int E, typename FS, typename FI, typename FC>
__device__ inline void warp_thomas(Tw (&v)[E], int k0, int m, int lane, FS SUB, FI INV, FC CP) {
    Tw A = Tw(1), B = Tw(0);
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if (k0 + k < m) {
            const Tw al = -SUB(k) * INV(k);
            A = al * A;
            B = al * B + v[k] * INV(k);
        }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Tw pa = __shfl_up_sync(0xffffffffu, A, o), pb = __shfl_up_sync(0xffffffffu, B, o);
        if (lane >= o) {
            B = A * pb + B;
            A = A * pa;
        }
    }
    Tw y = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) y = Tw(0);
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if (k0 + k < m) {
            y = (v[k] - SUB(k) * y) * INV(k);
            v[k] = y;
        }
    }
    A = Tw(1);
    B = Tw(0);
#pragma unroll
    for (int k = E - 1; k >= 0; --k) {
        if (k0 + k < m) {
            const Tw ga = -CP(k);
            A = ga * A;
            B = ga * B + v[k];
        }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Tw pa = __shfl_down_sync(0xffffffffu, A, o), pb = __shfl_down_sync(0xffffffffu, B, o);
        if (lane + o < 32) {
            B = A * pb + B;
            A = A * pa;
        }
    }
    Tw xx = __shfl_down_sync(0xffffffffu, B, 1);
    if (lane == 31) xx = Tw(0);
#pragma unroll
    for (int k = E - 1; k >= 0; --k) {
        if (k0 + k < m) {
            xx = v[k] - CP(k) * xx;
            v[k] = xx;
        }
    }
}

// A lane's Thomas factors for elements [k0, k0+E) of lines of m nodes, in
// registers when they are few (REG), else read from global memory.
template <typename Tw, int E, bool REG_ = (sizeof(Tw) * E <= 72)>
struct LaneFactors {
    static constexpr bool REG = REG_;
    Tw s[REG ? E : 1], i[REG ? E : 1], c[REG ? E : 1];
    const Tw *gs, *gi, *gc;
    int k0;
    __device__ LaneFactors(const Tw* sub, const Tw* inv, const Tw* cp, int k0_, int m)
        : gs(sub), gi(inv), gc(cp), k0(k0_) {
        if constexpr (REG) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int g = k0 + k;
                s[k] = g < m ? sub[g] : Tw(0);
                i[k] = g < m ? inv[g] : Tw(0);
                c[k] = g < m ? cp[g] : Tw(0);
            }
        }
    }
    __device__ Tw SUB(int k) const { if constexpr (REG) return s[k]; else return gs[k0 + k]; }
    __device__ Tw INV(int k) const { if constexpr (REG) return i[k]; else return gi[k0 + k]; }
    __device__ Tw CP(int k) const { if constexpr (REG) return c[k]; else return gc[k0 + k]; }
};

// Lines along a strided axis, 32 consecutive lines (in (outer, inner)
// order) per tile.  The block copies the tile, m rows of 32 elements each
// read as one warp access (coalesced within an outer index), into shared
// memory (row pitch 33),
// every warp solves lines of the tile with the warp-scan scheme of
// k_solve_warp (lane j owns elements [jE, jE+E) of the line; E odd, so the
// column reads are free of bank conflicts), and the block writes the tile
// back.  A lane's Thomas factors stay in registers across lines and tiles.
constexpr int ST_WARPS = 8;

template <typename Tw, typename Tdst, int E>
__global__ void __launch_bounds__(ST_WARPS * 32) k_solve_tile(Tw* x, int64_t outer_n, int m,
                                                              int64_t stride,
                                                              const Tw* __restrict__ sub,
                                                              const Tw* __restrict__ inv,
                                                              const Tw* __restrict__ cp, Tdst* dst,
                                                              Tw sign) {
    extern __shared__ __align__(16) unsigned char tile_raw[];
    Tw* t = reinterpret_cast<Tw*>(tile_raw);   // [m][33]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k0 = lane * E;
    const LaneFactors<Tw, E> F(sub, inv, cp, k0, m);
    // lines are numbered (outer, inner) row-major; a tile is 32 consecutive
    // lines, so a tile may span two outer indices but is never short
    const int64_t nlines = outer_n * stride;
    const int64_t ntiles = (nlines + 31) / 32;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t l0 = tile * 32;
        const int nl = (int)(nlines - l0 < 32 ? nlines - l0 : 32);   // lines in the tile
        const int64_t mine = l0 + (lane < nl ? lane : 0);            // this lane's line
        const int64_t outer = mine / stride, inner = mine - outer * stride;
        const int64_t off = outer * m * stride + inner;
        Tw* base = x + off;
        // asynchronous element copies: every row of the tile is in flight at once
        for (int k = wid; k < m; k += ST_WARPS) {
            Tw* dstp = &t[k * 33 + lane];
            if (lane < nl) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(dstp);
                const Tw* src = base + (int64_t)k * stride;
                if (sizeof(Tw) == 4)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
            } else {
                *dstp = Tw(0);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        for (int l = wid; l < nl; l += ST_WARPS) {
            Tw v[E];
#pragma unroll
            for (int k = 0; k < E; ++k) v[k] = k0 + k < m ? t[(k0 + k) * 33 + l] : Tw(0);
            warp_thomas<Tw, E>(v, k0, m, lane, [&](int k) { return F.SUB(k); },
                               [&](int k) { return F.INV(k); }, [&](int k) { return F.CP(k); });
#pragma unroll
            for (int k = 0; k < E; ++k)
                if (k0 + k < m) t[(k0 + k) * 33 + l] = v[k];
        }
        __syncthreads();
        if (lane < nl) {
            if (dst) {
                Tdst* d = dst + off;
                for (int k = wid; k < m; k += ST_WARPS) {
                    const int64_t i = (int64_t)k * stride;
                    d[i] = (Tdst)((Tw)d[i] + sign * t[k * 33 + lane]);
                }
            } else {
                for (int k = wid; k < m; k += ST_WARPS) base[(int64_t)k * stride] = t[k * 33 + lane];
            }
        }
        __syncthreads();   // the next tile overwrites t
    }
}

// The column solve of a restricted tile (to, mc rows of 32 columns, pitch
// 33): lane l owns column l, warp w rows [r0, r0 + cnt) in registers; the
// segment maps are folded through sA/sB (see k_restrict_solve).
template <typename Tw, int K>
__device__ inline void solve_columns(Tw* to, const Tw* sal, const Tw* sinv, const Tw* sga,
                                     Tw (*sA)[32], Tw (*sB)[32], int r0, int cnt, int lane,
                                     int wid) {
    Tw v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = j < cnt ? to[(r0 + j) * 33 + lane] : Tw(0);
    Tw A = Tw(1), B = Tw(0);   // forward map of the segment: y_in -> A y_in + B
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (j < cnt) {
            const Tw al = sal[r0 + j], w = v[j] * sinv[r0 + j];
            v[j] = w;
            A = al * A;
            B = al * B + w;
        }
    sA[wid][lane] = A;
    sB[wid][lane] = B;
    __syncthreads();
    Tw y = Tw(0);
    for (int s2 = 0; s2 < wid; ++s2) y = sA[s2][lane] * y + sB[s2][lane];
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (j < cnt) {
            y = sal[r0 + j] * y + v[j];
            v[j] = y;
        }
    A = Tw(1);   // backward map: x at the segment's end -> x at its start
    B = Tw(0);
#pragma unroll
    for (int j = K - 1; j >= 0; --j)
        if (j < cnt) {
            const Tw ga = sga[r0 + j];
            A = ga * A;
            B = ga * B + v[j];
        }
    __syncthreads();   // every thread has read the forward maps
    sA[wid][lane] = A;
    sB[wid][lane] = B;
    __syncthreads();
    Tw x = Tw(0);
    for (int s2 = ST_WARPS - 1; s2 > wid; --s2) x = sA[s2][lane] * x + sB[s2][lane];
#pragma unroll
    for (int j = K - 1; j >= 0; --j)
        if (j < cnt) {
            x = sga[r0 + j] * x + v[j];
            v[j] = x;
        }
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (j < cnt) to[(r0 + j) * 33 + lane] = v[j];
}

// Restriction and solve along one strided axis in a single pass.  The
// correction M_{l-1}^{-1} P^T M_l is a tensor product of one operator per
// axis, Mc_a^{-1} P_a^T M_a, and factors on different axes commute, so an
// axis may be restricted and solved before the next axis is restricted.
// in: (outer, m, inner), out: (outer, mc, inner).  A tile is 32 consecutive
// lines in (outer, inner) order.  In `parts` steps, the fine rows that a
// range of output rows reaches are copied into shared memory (cp.async) and
// each output row J takes the five-tap window of P_a^T M_a around fine row
// f(J) (weights rw[J*5 + t], taps outside the axis weigh 0); the restricted
// tile is then solved along its columns before the block writes it out.  The solve: lane l owns column l and warp w a
// segment of at most K rows.  Both Thomas sweeps are affine recurrences
// (y_k = al_k y_{k-1} + v_k inv_k with al_k = -a_k inv_k forward, x_k =
// -c'_k x_{k+1} + y_k backward), so each thread composes its segment's map
// in registers, the maps of the preceding (forward) or following (backward)
// segments are folded through shared memory, and each thread replays its
// segment.
template <typename Tw, int K>
__global__ void __launch_bounds__(ST_WARPS * 32) k_restrict_solve(
    const Tw* __restrict__ in, Tw* __restrict__ out, int64_t outer_n, int m, int mc,
    int64_t inner, AxisT<Tw> ax, int parts, int ti_rows) {
    extern __shared__ __align__(16) unsigned char tile_raw[];
    Tw* ti = reinterpret_cast<Tw*>(tile_raw);   // [ti_rows][33] fine rows of one part
    Tw* to = ti + (size_t)ti_rows * 33;          // [mc][33] restricted rows
    Tw* sal = to + (size_t)mc * 33;              // [mc] -a_k inv_k
    Tw* sinv = sal + mc;                         // [mc] inv_k
    Tw* sga = sinv + mc;                         // [mc] -c'_k
    __shared__ Tw sA[ST_WARPS][32], sB[ST_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < mc; k += blockDim.x) {
        sal[k] = -ax.tsub[k] * ax.tinv[k];
        sinv[k] = ax.tinv[k];
        sga[k] = -ax.tcp[k];
    }
    const int seg = (mc + ST_WARPS - 1) / ST_WARPS;   // rows per warp (<= K)
    const int r0 = wid * seg;
    const int cnt = max(0, min(seg, mc - r0));
    const Tw* __restrict__ rw = ax.rw;
    Tw wi[5];   // the window's weights where they are uniform (J in [rlo, rhi))
#pragma unroll
    for (int t = 0; t < 5; ++t) wi[t] = ax.rwi[t];
    const int64_t gstep = (int64_t)ST_WARPS * inner;             // ST_WARPS rows, elements
    const unsigned sstep = ST_WARPS * 33 * (unsigned)sizeof(Tw);  // ST_WARPS rows, bytes
    // lines are numbered (outer, inner) row-major; a tile is 32 consecutive
    // lines, so a tile may span two outer indices but is never short
    const int64_t nlines = outer_n * inner;
    const int64_t ntiles = (nlines + 31) / 32;
    // the restriction in parts of jp output rows: each part copies the fine
    // rows its windows reach, so the fine buffer holds ~2 jp rows
    const int jp = (mc + parts - 1) / parts;
    auto part_rows = [&](int J0, int* rb, int* re) {
        const int J1 = min(mc, J0 + jp);
        const int fb = J0 == mc - 1 ? m - 1 : 2 * J0;              // f(J0)
        const int fe = J1 - 1 == mc - 1 ? m - 1 : 2 * (J1 - 1);    // f(J1 - 1)
        *rb = max(0, fb - 2);                                       // fine rows [rb, re)
        *re = min(m, fe + 3);
    };
    // this lane's line of a tile, and the copy of fine rows [rb, re) of it
    auto line_of = [&](int64_t tile, int* nl, int64_t* o, int64_t* i) {
        const int64_t l0 = tile * 32;
        *nl = (int)(nlines - l0 < 32 ? nlines - l0 : 32);
        const int64_t mine = l0 + (lane < *nl ? lane : 0);
        *o = mine / inner;
        *i = mine - *o * inner;
    };
    auto copy_rows = [&](int nl, int64_t o, int64_t i, int rb, int re) {
        if (lane < nl) {
            const Tw* g = in + o * m * inner + i + (int64_t)(rb + wid) * inner;
            unsigned sa = (unsigned)__cvta_generic_to_shared(&ti[wid * 33 + lane]);
#pragma unroll 4
            for (int k = rb + wid; k < re; k += ST_WARPS, g += gstep, sa += sstep) {
                if (sizeof(Tw) == 4)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(g) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(g) : "memory");
            }
        } else {
            for (int k = rb + wid; k < re; k += ST_WARPS) ti[(k - rb) * 33 + lane] = Tw(0);
        }
    };
    bool ahead = false;   // the first part of this tile is already being copied
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int nl;
        int64_t o, i;
        line_of(tile, &nl, &o, &i);
        for (int J0 = 0; J0 < mc; J0 += jp) {
            const int J1 = min(mc, J0 + jp);
            int rb, re;
            part_rows(J0, &rb, &re);
            if (!(J0 == 0 && ahead)) copy_rows(nl, o, i, rb, re);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            for (int J = J0 + wid; J < J1; J += ST_WARPS) {
                Tw acc;
                if (J >= ax.rlo && J < ax.rhi) {   // window 2J-2 .. 2J+2, uniform weights
                    const Tw* q = &ti[(2 * J - 2 - rb) * 33 + lane];
                    acc = wi[0] * q[0];
                    acc += wi[1] * q[33];
                    acc += wi[2] * q[66];
                    acc += wi[3] * q[99];
                    acc += wi[4] * q[132];
                } else {
                    const int f = J == mc - 1 ? m - 1 : 2 * J;   // fine row under coarse row J
                    acc = Tw(0);
#pragma unroll
                    for (int t = 0; t < 5; ++t) {
                        int ip = f - 2 + t;
                        const bool ok = ip >= 0 && ip < m;
                        const Tw w = ok ? rw[J * 5 + t] : Tw(0);
                        ip = ok ? ip : f;
                        acc += w * ti[(ip - rb) * 33 + lane];
                    }
                }
                to[J * 33 + lane] = acc;
            }
            __syncthreads();   // the next part's copy overwrites the fine rows
        }
        // the fine rows are free now: the next tile's first part streams in
        // while this tile is solved and written out
        {
            const int64_t next = tile + gridDim.x;
            ahead = next < ntiles;
            if (ahead) {
                int nl2, rb, re;
                int64_t o2, i2;
                line_of(next, &nl2, &o2, &i2);
                part_rows(0, &rb, &re);
                copy_rows(nl2, o2, i2, rb, re);
            }
        }
        solve_columns<Tw, K>(to, sal, sinv, sga, sA, sB, r0, cnt, lane, wid);
        __syncthreads();
        if (lane < nl) {
            Tw* dst = out + o * mc * inner + i + (int64_t)wid * inner;
            const Tw* sp = &to[wid * 33 + lane];
#pragma unroll 4
            for (int k = wid; k < mc; k += ST_WARPS, dst += gstep, sp += ST_WARPS * 33) *dst = *sp;
        }
        __syncthreads();   // the next tile overwrites both buffers
    }
}

// The same pass with its tiles staged by the tensor-memory accelerator.  A
// tile is 32 adjacent lines of one outer index (columns i0 .. i0+31 of the
// (outer, m, inner) array; inner is padded to 16 bytes, so i0 * size is a
// multiple of 16), and each part of a tile (the fine rows of jp output rows)
// is one box of `br` rows starting two rows above the part's first centre;
// rows outside the axis and columns past `inner` arrive as zeros.  Two
// buffers alternate: while the block restricts one part, thread 0 has
// already asked for the next, so the copies run behind the arithmetic with
// no thread issuing element copies.  Each wait on a buffer's barrier gives up
// after a bounded number of polls: the block then sets ST_TIMEOUT in
// *status, waits (bounded again) for the copies it has in flight and
// returns.
constexpr uint32_t TMA_MAX_POLLS = 1u << 22;

template <typename Tw, int K>
__global__ void __launch_bounds__(ST_WARPS * 32) k_restrict_solve_tma(
    const __grid_constant__ CUtensorMap tin, Tw* __restrict__ out, int64_t outer_n, int m, int mc,
    int64_t inner, AxisT<Tw> ax, int jp, int br, unsigned* status) {
    extern __shared__ __align__(128) unsigned char tma_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)tma_raw + 127) & ~(uintptr_t)127);
    Tw* fb = reinterpret_cast<Tw*>(base);        // [2][br][32] fine rows, as the boxes land
    Tw* to = fb + 2 * (size_t)br * 32;           // [mc][33] restricted rows
    Tw* sal = to + (size_t)mc * 33;              // [mc] -a_k inv_k
    Tw* sinv = sal + mc;                         // [mc] inv_k
    Tw* sga = sinv + mc;                         // [mc] -c'_k
    uint64_t* bar = reinterpret_cast<uint64_t*>(((uintptr_t)(sga + mc) + 7) & ~(uintptr_t)7);
    __shared__ Tw sA[ST_WARPS][32], sB[ST_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < mc; k += blockDim.x) {
        sal[k] = -ax.tsub[k] * ax.tinv[k];
        sinv[k] = ax.tinv[k];
        sga[k] = -ax.tcp[k];
    }
    const int seg = (mc + ST_WARPS - 1) / ST_WARPS;   // rows per warp (<= K)
    const int r0 = wid * seg;
    const int cnt = max(0, min(seg, mc - r0));
    const Tw* __restrict__ rw = ax.rw;
    Tw wi[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) wi[t] = ax.rwi[t];
    const int parts = (mc + jp - 1) / jp;
    const int64_t tpo = (inner + 31) / 32;   // tiles per outer index
    const int64_t ntiles = outer_n * tpo;
    const uint32_t box_bytes = (uint32_t)br * 32u * (uint32_t)sizeof(Tw);
    const int64_t gstep = (int64_t)ST_WARPS * inner;
    auto centre = [&](int J) { return J == mc - 1 ? m - 1 : 2 * J; };   // fine row of coarse J
    // job q: part q % parts of the block's tile q / parts, into buffer q & 1
    auto issue = [&](int64_t q) {
        const int64_t tile = blockIdx.x + (q / parts) * (int64_t)gridDim.x;
        if (tile >= ntiles) return;
        const int p = (int)(q % parts);
        const int64_t o = tile / tpo;
        const int i0 = (int)((tile - o * tpo) * 32);
        uint64_t* b = &bar[q & 1];
        mbar_expect_tx(b, box_bytes);
        tma_load_3d(fb + (size_t)(q & 1) * br * 32, &tin, i0, centre(p * jp) - 2, (int)o, b);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        issue(0);
        issue(1);
    }
    int64_t q = 0;   // the next job to consume
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int64_t o = tile / tpo;
        const int64_t i0 = (tile - o * tpo) * 32;
        const int nl = (int)min((int64_t)32, inner - i0);   // columns inside the array
        for (int p = 0; p < parts; ++p, ++q) {
            const int J0 = p * jp, J1 = min(mc, J0 + jp);
            const int f0 = centre(J0) - 2;   // fine row of the box's first row
            const bool ok = mbar_wait(&bar[q & 1], (uint32_t)((q >> 1) & 1), TMA_MAX_POLLS);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            const Tw* ti = fb + (size_t)(q & 1) * br * 32;
            for (int J = J0 + wid; J < J1; J += ST_WARPS) {
                Tw acc;
                if (J >= ax.rlo && J < ax.rhi) {   // window 2J-2 .. 2J+2, uniform weights
                    const Tw* r = &ti[(2 * J - 2 - f0) * 32 + lane];
                    acc = wi[0] * r[0];
                    acc += wi[1] * r[32];
                    acc += wi[2] * r[64];
                    acc += wi[3] * r[96];
                    acc += wi[4] * r[128];
                } else {
                    const int f = centre(J);
                    acc = Tw(0);
#pragma unroll
                    for (int t = 0; t < 5; ++t) {
                        const int ip = f - 2 + t;   // rows outside the axis arrived as zeros
                        const Tw w = (ip >= 0 && ip < m) ? rw[J * 5 + t] : Tw(0);
                        acc += w * ti[(ip - f0) * 32 + lane];
                    }
                }
                to[J * 33 + lane] = acc;
            }
            __syncthreads();   // the buffer is free: the job two ahead streams into it
            if (threadIdx.x == 0) issue(q + 2);
        }
        if (failed) break;
        solve_columns<Tw, K>(to, sal, sinv, sga, sA, sB, r0, cnt, lane, wid);
        __syncthreads();
        if (lane < nl) {
            Tw* dst = out + o * mc * inner + i0 + lane + (int64_t)wid * inner;
            const Tw* sp = &to[wid * 33 + lane];
#pragma unroll 4
            for (int k = wid; k < mc; k += ST_WARPS, dst += gstep, sp += ST_WARPS * 33) *dst = *sp;
        }
        __syncthreads();   // the next tile overwrites the restricted rows
    }
    if (failed && threadIdx.x == 0) {
        atomicOr(status, (unsigned)ST_TIMEOUT);
        // the copies of jobs q and q + 1 may still be in flight
        for (int64_t r = q; r < q + 2; ++r) {
            const int64_t tile = blockIdx.x + (r / parts) * (int64_t)gridDim.x;
            if (tile < ntiles) mbar_wait(&bar[r & 1], (uint32_t)((r >> 1) & 1), TMA_MAX_POLLS);
        }
    }
}

// The same pass with each warp owning one segment of K coarse rows from the
// copy to the write.  Warp w's segment is coarse rows [r0, r0 + K), r0 = w K;
// its fine rows f(r0) - 2 .. f(r0) + 2 K arrive by TMA in one box of
// br = 2 K + 3 rows into the warp's own buffer, the warp restricts them
// straight into registers (lane l: column l), hands the buffer to the next
// tile's copy, solves its segment with the maps of the other segments folded
// through shared memory, and writes its rows from registers.  No restricted
// tile passes through shared memory.  Rows past the axis (the end of the last
// segment, and whole segments when K NW > mc) run through the same
// arithmetic with factors 0 (al = inv = -c' = 0), which leaves the real rows'
// results unchanged bit for bit, so no loop tests a row count.  Tiles are 32
// columns of one outer index (`tin`, boxes of 32 x br x 1); when the last
// columns of an outer index are at most four (the padded row of a 2^k + 1
// axis), they are taken from eight outer indices at once (`ttail`, boxes of
// 4 x br x 8, in shared memory as [8][br][4]: lane l reads outer l / 4,
// column l % 4), so no tile runs with 4 of its 32 lanes live.  Products of
// the segments' map slopes do not depend on the data and are taken once per
// block.  Same arithmetic, in the same order, as k_restrict_solve and
// k_restrict_solve_tma.

// Coarse row J's restriction from the rows of a box whose first row is fine
// row f0 (RP: the box's row pitch), by the tables: valid for any J.
template <typename Tw, int RP>
__device__ inline Tw restrict_row(const Tw* __restrict__ b, int J, int mc, int m, int f0,
                                  const Tw* __restrict__ rw) {
    const int f = J == mc - 1 ? m - 1 : 2 * J;
    Tw acc = Tw(0);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int ip = f - 2 + t;   // rows outside the axis arrived as zeros
        const Tw w = (ip >= 0 && ip < m) ? rw[J * 5 + t] : Tw(0);
        acc += w * b[(ip - f0) * RP];
    }
    return acc;
}

// A segment's restriction into registers: every row with the uniform window
// (rows 2j .. 2j+4 of the box), then the axis' first and last rows again by
// the tables.  The caller guarantees that rows 1 .. mc-2 are uniform.
template <typename Tw, int K, int RP>
__device__ inline void restrict_segment(const Tw* __restrict__ b, Tw (&v)[K], const Tw (&wi)[5],
                                        int r0, int mc, int m, int f0,
                                        const Tw* __restrict__ rw) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const Tw* r = b + 2 * j * RP;
        Tw acc = wi[0] * r[0];
        acc += wi[1] * r[RP];
        acc += wi[2] * r[2 * RP];
        acc += wi[3] * r[3 * RP];
        acc += wi[4] * r[4 * RP];
        v[j] = acc;
    }
    if (r0 == 0) v[0] = restrict_row<Tw, RP>(b, 0, mc, m, f0, rw);
    if (mc - 1 - r0 < K) {   // the axis' last row is this segment's row mc-1-r0
        const Tw g = restrict_row<Tw, RP>(b, mc - 1, mc, m, f0, rw);
        // a mask the compiler cannot see through, so the select stays one
        // select per register instead of an indexed store to local memory
        uint64_t hit;
        asm("mov.b64 %0, %1;" : "=l"(hit) : "l"(1ull << (mc - 1 - r0)));
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((hit >> j) & 1ull) v[j] = g;
    }
}

// Four consecutive factors of a segment's table (16-byte aligned).
__device__ inline void load4(const float* p, float (&o)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ inline void load4(const double* p, double (&o)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

template <typename Tw, int K, int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 3 : (K <= 17 ? 2 : 1)) k_restrict_solve_seg(
    const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap ttail,
    Tw* __restrict__ out, int64_t outer_n, int m, int mc, int64_t inner, AxisT<Tw> ax, int br,
    int64_t tpo, int64_t ntail, unsigned* status) {
    constexpr int KP = (K + 3) / 4 * 4;   // a segment's table entries, padded to 16 bytes
    extern __shared__ __align__(128) unsigned char seg_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)seg_raw + 127) & ~(uintptr_t)127);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Tw* box = reinterpret_cast<Tw*>(base) + (size_t)wid * br * 32;   // this warp's fine rows
    Tw* tab = reinterpret_cast<Tw*>(base) + (size_t)NW * br * 32;    // [3][NW][KP] factors
    uint64_t* bar = reinterpret_cast<uint64_t*>(tab + 3 * NW * KP);
    __shared__ Tw sBf[NW][32], sBb[NW][32], sAf[NW], sAb[NW];
    // factors per segment row: -a_J inv_J, inv_J, -c'_J; 0 past the axis
    for (int k = threadIdx.x; k < NW * KP; k += blockDim.x) {
        const int J = (k / KP) * K + k % KP;
        const bool in_seg = k % KP < K && J < mc;
        tab[k] = in_seg ? -ax.tsub[J] * ax.tinv[J] : Tw(0);
        tab[NW * KP + k] = in_seg ? ax.tinv[J] : Tw(0);
        tab[2 * NW * KP + k] = in_seg ? -ax.tcp[J] : Tw(0);
    }
    const Tw* tal = tab + wid * KP;
    const Tw* tinv = tab + NW * KP + wid * KP;
    const Tw* tga = tab + 2 * NW * KP + wid * KP;
    const int r0 = wid * K;
    const bool active = r0 < mc;   // the segment holds rows of the axis
    const int f0 = (r0 == mc - 1 ? m - 1 : 2 * r0) - 2;   // fine row of the box's first row
    Tw wi[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) wi[t] = ax.rwi[t];
    const int64_t nmain = outer_n * tpo;
    const int64_t ntiles = nmain + ntail;
    const int64_t x0 = tpo * 32;   // first column of the tail boxes
    const uint32_t box_bytes = (uint32_t)br * 32u * (uint32_t)sizeof(Tw);
    const bool owner = lane == 0 && active;   // issues and waits for this warp's copies
    auto issue = [&](int64_t tile) {
        mbar_expect_tx(&bar[wid], box_bytes);
        if (tile < nmain) {
            const int64_t o = tile / tpo;
            tma_load_3d(box, &tin, (int)((tile - o * tpo) * 32), f0, (int)o, &bar[wid]);
        } else {
            tma_load_3d(box, &ttail, (int)x0, f0, (int)((tile - nmain) * 8), &bar[wid]);
        }
    };
    if (threadIdx.x == 0) {
        for (int w = 0; w < NW; ++w) mbar_init(&bar[w]);
        mbar_fence_init();
    }
    __syncthreads();   // the barriers and the factor tables are ready
    if (lane == 0) {
        Tw A = Tw(1);
        for (int j = 0; j < K; ++j) A = tal[j] * A;
        sAf[wid] = A;
        A = Tw(1);
        for (int j = K - 1; j >= 0; --j) A = tga[j] * A;
        sAb[wid] = A;
    }
    if (owner && blockIdx.x < ntiles) issue(blockIdx.x);
    uint32_t phase = 0;
    bool failed = false, pending = owner && blockIdx.x < ntiles;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        bool ok = true;
        if (owner) ok = mbar_wait(&bar[wid], phase, TMA_MAX_POLLS);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        phase ^= 1u;
        pending = false;
        Tw v[K];
        const bool tail = tile >= nmain;
        if (!active) {
#pragma unroll
            for (int j = 0; j < K; ++j) v[j] = Tw(0);
        } else if (!tail) {
            restrict_segment<Tw, K, 32>(box + lane, v, wi, r0, mc, m, f0, ax.rw);
        } else {
            restrict_segment<Tw, K, 4>(box + (lane >> 2) * br * 4 + (lane & 3), v, wi, r0, mc, m,
                                       f0, ax.rw);
        }
        __syncwarp();   // every lane has read the box: the next tile's rows may land in it
        const int64_t next = tile + gridDim.x;
        if (owner && next < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(next);
            pending = true;
        }
        // forward sweep: y_k = al_k y_{k-1} + v_k inv_k
        Tw f4a[4], f4b[4];
        Tw B = Tw(0);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (j % 4 == 0) {
                load4(tal + j, f4a);
                load4(tinv + j, f4b);
            }
            const Tw w = v[j] * f4b[j % 4];
            v[j] = w;
            B = f4a[j % 4] * B + w;
        }
        sBf[wid][lane] = B;
        __syncthreads();
        Tw y = Tw(0);
        for (int s2 = 0; s2 < wid; ++s2) y = sAf[s2] * y + sBf[s2][lane];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (j % 4 == 0) load4(tal + j, f4a);
            y = f4a[j % 4] * y + v[j];
            v[j] = y;
        }
        // backward sweep: x_k = -c'_k x_{k+1} + y_k
        B = Tw(0);
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            if (j % 4 == 3 || j == K - 1) load4(tga + (j & ~3), f4a);
            B = f4a[j % 4] * B + v[j];
        }
        // (the forward maps have their own buffer: the next tile writes them
        // only after its first barrier, when every thread has read them)
        sBb[wid][lane] = B;
        __syncthreads();
        Tw x = Tw(0);
        for (int s2 = NW - 1; s2 > wid; --s2) x = sAb[s2] * x + sBb[s2][lane];
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            if (j % 4 == 3 || j == K - 1) load4(tga + (j & ~3), f4a);
            x = f4a[j % 4] * x + v[j];
            v[j] = x;
        }
        // write the segment's rows that lie on the axis
        int64_t o, col;
        bool live;
        if (!tail) {
            o = tile / tpo;
            col = (tile - o * tpo) * 32 + lane;
            live = col < inner;
        } else {
            o = (tile - nmain) * 8 + (lane >> 2);
            col = x0 + (lane & 3);
            live = o < outer_n && col < inner;
        }
        if (live && active) {
            Tw* dst = out + (o * mc + r0) * inner + col;
            if (r0 + K <= mc) {
#pragma unroll
                for (int j = 0; j < K; ++j) dst[(int64_t)j * inner] = v[j];
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if (r0 + j < mc) dst[(int64_t)j * inner] = v[j];
            }
        }
    }
    if (failed) {
        if (threadIdx.x == 0) atomicOr(status, (unsigned)ST_TIMEOUT);
        // the copy this warp asked for last may still be in flight
        if (owner && pending) mbar_wait(&bar[wid], phase, TMA_MAX_POLLS);
    }
}

// Lines along the contiguous axis, one warp per line held in registers: lane
// j owns elements [jE, jE+E).  Both Thomas sweeps are first-order affine
// recurrences (y_k = alpha_k y_{k-1} + beta_k forward, x_k = gamma_k
// x_{k+1} + y_k backward), so each lane composes the maps of its segment,
// the warp scans the compositions with shuffles, and each lane replays its
// segment from the scanned input.  Global traffic goes through a padded
// per-warp shared buffer so loads and stores stay coalesced.  E is odd
// (conflict-free segment reads) and the smallest with 32E >= m, so lines of
// 2^k + 1 nodes keep nearly every lane busy.  A lane's Thomas factors are
// the same for every line: they stay in registers (the widest segments read
// them through L1), and the next line's loads are issued before the current
// line is solved.
constexpr int SW_WARPS = 4;

template <typename Tw, typename Tdst, int E>
__global__ void __launch_bounds__(SW_WARPS * 32) k_solve_warp(Tw* x, int64_t lines, int m,
                                                              const Tw* __restrict__ sub,
                                                              const Tw* __restrict__ inv,
                                                              const Tw* __restrict__ cp, Tdst* dst,
                                                              Tw sign, int64_t pitch) {
    constexpr int W = E + 1;
    __shared__ Tw buf[SW_WARPS][32 * W];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Tw* sb = buf[wid];
    const int k0 = lane * E;
    const LaneFactors<Tw, E> F(sub, inv, cp, k0, m);
    const int64_t step = (int64_t)gridDim.x * SW_WARPS;
    int64_t ln = (int64_t)blockIdx.x * SW_WARPS + wid;
    // row element e = lane + 32 j (j < E, so 32E >= m covers the row)
    Tw nv[E];
    auto load_row = [&](int64_t l) {
        const Tw* row = x + l * pitch;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = lane + 32 * j;
            nv[j] = (l < lines && e < m) ? row[e] : Tw(0);
        }
    };
    load_row(ln);
    for (; ln < lines; ln += step) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = lane + 32 * j;
            sb[(e / E) * W + e % E] = nv[j];
        }
        __syncwarp();
        Tdst* d = dst ? dst + ln * m : nullptr;
        Tdst dv[E];
        if (d) {
#pragma unroll
            for (int j = 0; j < E; ++j) {
                const int e = lane + 32 * j;
                dv[j] = e < m ? d[e] : Tdst(0);
            }
        }
        load_row(ln + step);   // in flight while this line is solved
        Tw v[E];
#pragma unroll
        for (int k = 0; k < E; ++k) v[k] = sb[lane * W + k];
        warp_thomas<Tw, E>(v, k0, m, lane, [&](int k) { return F.SUB(k); },
                           [&](int k) { return F.INV(k); }, [&](int k) { return F.CP(k); });
#pragma unroll
        for (int k = 0; k < E; ++k) sb[lane * W + k] = v[k];
        __syncwarp();
        Tw* row = x + ln * pitch;
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int e = lane + 32 * j;
            if (e >= m) continue;
            const Tw r = sb[(e / E) * W + e % E];
            if (d) d[e] = (Tdst)((Tw)dv[j] + sign * r);
            else row[e] = r;
        }
        __syncwarp();
    }
}

// -- recomposition fill ------------------------------------------------------
template <typename T>
__global__ void k_fill(const T* zin, const T* __restrict__ coarse, T* out, Level<T> lv) {
    FOR_NODES(lv.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        int64_t j0[4], j1[4];
        T w0[4], w1[4];
        int nc[4];
        bool allc = true;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int* fc = lv.ax[a].fcls;
            nc[a] = 1;
            j0[a] = j1[a] = i[a];
            w0[a] = T(1);
            w1[a] = T(0);
            if (!fc) continue;
            const int c = fc[i[a]];
            if (c >= 0) {
                j0[a] = c;
            } else {
                allc = false;
                j0[a] = -c - 1;
                j1[a] = -c;
                w0[a] = lv.ax[a].wl[i[a]];
                w1[a] = lv.ax[a].wr[i[a]];
                nc[a] = 2;
            }
        }
        const int64_t lin = ravel4(i, lv.n);
        if (allc) {
            out[lin] = coarse[ravel4(j0, lv.nc)];
            continue;
        }
        T acc = T(0);
        for (int c0 = 0; c0 < nc[0]; ++c0)
            for (int c1 = 0; c1 < nc[1]; ++c1)
                for (int c2 = 0; c2 < nc[2]; ++c2)
                    for (int c3 = 0; c3 < nc[3]; ++c3) {
                        const int64_t q[4] = {c0 ? j1[0] : j0[0], c1 ? j1[1] : j0[1],
                                              c2 ? j1[2] : j0[2], c3 ? j1[3] : j0[3]};
                        const T w = (c0 ? w1[0] : w0[0]) * (c1 ? w1[1] : w0[1]) *
                                    (c2 ? w1[2] : w0[2]) * (c3 ? w1[3] : w0[3]);
                        acc += w * coarse[ravel4(q, lv.nc)];
                    }
        out[lin] = zin[lin] + acc;
    }
}

// -- layout conversion -------------------------------------------------------
template <typename T, bool kScatter>
__global__ void k_layout(T* compact, T* data, LevelIndex li, Level<T> lv, int has_tables,
                         Shape4 fine) {
    FOR_NODES(li.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        if (has_tables) {
            bool allc = true;
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (lv.ax[a].fcls && lv.ax[a].fcls[i[a]] < 0) allc = false;
            if (allc) continue;
        }
        int64_t q[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) q[a] = li.pos[a][i[a]];
        const int64_t g = ravel4(q, fine.n);
        const int64_t lin = ravel4(i, li.n);
        if (kScatter) data[g] = compact[lin];
        else compact[lin] = data[g];
    }
}

template <typename T>
__global__ void k_difference(const T* __restrict__ a, const T* __restrict__ b,
                             double* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)b[i] - (double)a[i];
}

// -- reductions --------------------------------------------------------------
constexpr int RED_BLOCKS = RED_PARTS;
constexpr int RED_THREADS = 256;

// max |a| (b == null, exact in the data's precision) or max |b - a| (in FP64).
template <typename T>
__global__ void k_maxabs(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                         double* partial, unsigned* status) {
    bool bad = false;
    double m = 0.0;
    if (!b && sizeof(T) == 4 && (reinterpret_cast<uintptr_t>(a) & 15) == 0) {
        // float input in 16-byte loads, two per iteration.  The largest
        // magnitude bit pattern orders like |v| and reaches the infinity
        // pattern exactly when some value is infinite or NaN.
        const float4* a4 = reinterpret_cast<const float4*>(a);
        const int64_t n4 = n / 4, stride = (int64_t)gridDim.x * blockDim.x;
        unsigned mb = 0;
        auto see = [&](const float4 v) {
            mb = max(mb, max(max(__float_as_uint(v.x) & 0x7FFFFFFFu, __float_as_uint(v.y) & 0x7FFFFFFFu),
                             max(__float_as_uint(v.z) & 0x7FFFFFFFu, __float_as_uint(v.w) & 0x7FFFFFFFu)));
        };
        int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        for (; i + stride < n4; i += 2 * stride) {
            const float4 v0 = a4[i], v1 = a4[i + stride];
            see(v0);
            see(v1);
        }
        if (i < n4) see(a4[i]);
        for (int64_t k = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride)
            mb = max(mb, __float_as_uint((float)a[k]) & 0x7FFFFFFFu);
        bad = mb >= 0x7F800000u;
        m = bad ? 0.0 : (double)__uint_as_float(mb);
    } else if (!b) {
        T mt = T(0);
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const T v = a[i];
            if (!isfinite(v)) bad = true;
            mt = fmax(mt, fabs(v));
        }
        m = (double)mt;
    } else {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const double v = (double)b[i] - (double)a[i];
            if (!isfinite(v)) bad = true;
            m = fmax(m, fabs(v));
        }
    }
    __shared__ double sh[RED_THREADS];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
    if (bad) atomicOr(status, ST_NONFINITE);
}

// sum_i u_i (M u)_i with the tensor mass matrix of a level (3^D stencil).
template <typename T>
__global__ void k_mass_norm(const T* __restrict__ u, Level<T> lv, double* partial) {
    double s = 0.0;
    FOR_NODES(lv.n, i0, i1, i2, i3) {
        const int64_t i[4] = {i0, i1, i2, i3};
        double f[4][3];
        int lo[4], hi[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double* md = lv.ax[a].mdiag;
            f[a][0] = f[a][2] = 0.0;
            if (!md) {
                lo[a] = hi[a] = 0;
                f[a][1] = 1.0;
                continue;
            }
            const double* mo = lv.ax[a].moff;
            lo[a] = i[a] > 0 ? -1 : 0;
            hi[a] = i[a] + 1 < lv.n[a] ? 1 : 0;
            f[a][0] = i[a] > 0 ? mo[i[a] - 1] : 0.0;
            f[a][1] = md[i[a]];
            f[a][2] = mo[i[a]];
        }
        double mu = 0.0;
        for (int o0 = lo[0]; o0 <= hi[0]; ++o0)
            for (int o1 = lo[1]; o1 <= hi[1]; ++o1)
                for (int o2 = lo[2]; o2 <= hi[2]; ++o2)
                    for (int o3 = lo[3]; o3 <= hi[3]; ++o3) {
                        const int64_t q[4] = {i[0] + o0, i[1] + o1, i[2] + o2, i[3] + o3};
                        mu += f[0][o0 + 1] * f[1][o1 + 1] * f[2][o2 + 1] * f[3][o3 + 1] *
                              (double)u[ravel4(q, lv.n)];
                    }
        s += (double)u[ravel4(i, lv.n)] * mu;
    }
    __shared__ double sh[RED_THREADS];
    const int t = threadIdx.x;
    sh[t] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    if (t == 0) partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = sh[0];
}

template <typename Tw, typename Tdst>
mgard_status solve_axis(Tw* x, Shape4 s, int a, const Tw* sub, const Tw* inv, const Tw* cp,
                        Tdst* dst, Tw sign, cudaStream_t st) {
    const int64_t m = s.n[a];
    if (a == 3) return solve_contiguous<Tw, Tdst>(x, shape_prod(s) / m, m, sub, inv, cp, dst, sign, st);
    int64_t stride = 1, outer = 1;
    for (int b = a + 1; b < 4; ++b) stride *= s.n[b];
    for (int b = 0; b < a; ++b) outer *= s.n[b];
    return solve_strided<Tw, Tdst>(x, outer, m, stride, sub, inv, cp, dst, sign, st);
}

// Steps 2-4 for one level: coarse += sign * M_{l-1}^{-1} P^T M_l z, with z
// read from the level-l array `z` (its coarse positions are ignored).
template <typename T, typename Tw>
mgard_status correct_level(const Plan& p, int l, const T* z, T* coarse, void* t0, void* t1,
                           T sign, cudaStream_t st) {
    const Level<Tw>& lw = p.level<Tw>(l);
    const Level<T>& lt = p.level<T>(l);
    Shape4 s;
    for (int a = 0; a < 4; ++a) s.n[a] = lt.n[a];
    Mask mask;
    for (int a = 0; a < 4; ++a) mask.fcls[a] = lt.ax[a].fcls;
    mask.on = 1;
    Mask nomask{};
    const void* cur = z;
    bool first = true;
    Tw* bufs[2] = {(Tw*)t0, (Tw*)t1};
    int which = 0;
    int last_axis = -1;
    for (int a = 0; a < 4; ++a) {
        if (!lt.ax[a].fcls) continue;
        Shape4 so = s;
        so.n[a] = lt.nc[a];
        Tw* out = bufs[which];
        if (first)
            MGB_LAUNCH("k_restrict", st, k_restrict<T, Tw><<<grid3(so.n, 128), 128, 0, st>>>(
                (const T*)cur, out, s, a, lw.ax[a].rf, lw.ax[a].rw, so, mask));
        else
            MGB_LAUNCH("k_restrict", st, k_restrict<Tw, Tw><<<grid3(so.n, 128), 128, 0, st>>>(
                (const Tw*)cur, out, s, a, lw.ax[a].rf, lw.ax[a].rw, so, nomask));
        MGB_CUDA(cudaGetLastError());
        first = false;
        s = so;
        cur = out;
        which ^= 1;
        last_axis = a;
    }
    if (last_axis < 0) return MGARD_OK;
    Tw* b = (Tw*)cur;
    for (int a = 0; a < 4; ++a) {
        if (!lt.ax[a].fcls) continue;
        T* dst = a == last_axis ? coarse : nullptr;
        MGB_TRY((solve_axis<Tw, T>(b, s, a, lw.ax[a].tsub, lw.ax[a].tinv, lw.ax[a].tcp, dst,
                                   (Tw)sign, st)));
    }
    return MGARD_OK;
}

template <typename T>
bool level_uses_fp64(const Plan& p, int l) {
    return sizeof(T) == 8 || p.level_size(l - 1) < FP64_SOLVE_NODES;
}

template <typename T>
mgard_status correct(const Plan& p, int l, const T* z, T* coarse, void* t0, void* t1, T sign,
                     cudaStream_t st, int64_t zoff = -1, bool x_done = false,
                     unsigned* status = nullptr) {
    const bool f64 = level_uses_fp64<T>(p, l);
    if (rows3_ok(p)) {
        if (!status) status = fallback_status();
        if (!status) return MGARD_ECUDA;
        if (f64)
            return rows3_correct<T, double>(p, l, z, coarse, t0, t1, sign, st, zoff, x_done, status);
        return rows3_correct<T, T>(p, l, z, coarse, t0, t1, sign, st, zoff, x_done, status);
    }
    if (f64) return correct_level<T, double>(p, l, z, coarse, t0, t1, sign, st);
    return correct_level<T, T>(p, l, z, coarse, t0, t1, sign, st);
}

}  // namespace

template <typename T>
mgard_status correct_coarse(const Plan& p, int l, const T* z, T* coarse, void* t0, void* t1,
                            T sign, cudaStream_t st) {
    return correct<T>(p, l, z, coarse, t0, t1, sign, st);
}
template mgard_status correct_coarse<float>(const Plan&, int, const float*, float*, void*, void*,
                                            float, cudaStream_t);
template mgard_status correct_coarse<double>(const Plan&, int, const double*, double*, void*,
                                             void*, double, cudaStream_t);

cudaMemPool_t workspace_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        pool = nullptr;
    } else {
        uint64_t keep = ~0ull;   // keep freed blocks for reuse instead of unmapping at each sync
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pools[dev] = pool;
    return pool;
}

// Opt a kernel in to `bytes` of dynamic shared memory where its current
// limit is lower (by default 48 KB minus its static shared memory), once per
// kernel, size and device.
// Status word of kernels run without a caller's status (file-scope device
// array; its device address is looked up once per device, with that device
// current).
static __device__ unsigned g_fallback_status;

unsigned* fallback_status() {
    static std::mutex mu;
    static std::map<int, unsigned*> addr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    auto it = addr.find(dev);
    if (it != addr.end()) return it->second;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fallback_status) != cudaSuccess) {
        set_error("status word: cudaGetSymbolAddress failed");
        return nullptr;
    }
    addr[dev] = (unsigned*)p;
    return (unsigned*)p;
}

mgard_status encode_tensor_map_3d(CUtensorMap* map, const void* base, int elem_bytes,
                                  const uint64_t dims[3], const uint64_t strides[2],
                                  const uint32_t box[3]) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!encode) {
            cudaDriverEntryPointQueryResult q{};
            void* fn = nullptr;
            const cudaError_t e =
                cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
                set_error("cuTensorMapEncodeTiled is not available");
                return MGARD_ECUDA;
            }
            encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        }
    }
    const cuuint64_t gd[3] = {dims[0], dims[1], dims[2]};
    const cuuint64_t gs[2] = {strides[0], strides[1]};
    const cuuint32_t bd[3] = {box[0], box[1], box[2]};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = encode(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              3, const_cast<void*>(base), gd, gs, bd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled rejected the tile map");
        return MGARD_EINVAL;
    }
    return MGARD_OK;
}

mgard_status allow_dynamic_smem(const void* kern, size_t bytes) {
    if (bytes == 0) return MGARD_OK;
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> limit;
    int dev = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit.find({kern, dev});
    if (it == limit.end()) {
        cudaFuncAttributes fa;
        MGB_CUDA(cudaFuncGetAttributes(&fa, kern));
        it = limit.emplace(std::make_pair(kern, dev), (size_t)fa.maxDynamicSharedSizeBytes).first;
    }
    if (it->second < bytes) {
        MGB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        it->second = bytes;
    }
    return MGARD_OK;
}

// A grid of persistent blocks: as many as stay resident at once (all SMs,
// the occupancy of `kern` at this block size and shared memory), at most
// `work` of them.  Launching more would leave a tail of blocks that start
// only when others finish.
mgard_status resident_grid(const void* kern, int threads, size_t smem, int64_t work, int* grid) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
    int dev = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(kern, threads, smem, dev);
    auto it = cache.find(key);
    int per = 0;
    if (it == cache.end()) {
        int sms = 0, nb = 0;
        MGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        MGB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem));
        per = std::max(1, sms * nb);
        cache[key] = per;
    } else {
        per = it->second;
    }
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>(work, per));
    return MGARD_OK;
}

template <typename Tw, typename Tdst>
mgard_status solve_strided(Tw* x, int64_t outer, int64_t m, int64_t stride, const Tw* sub,
                           const Tw* inv, const Tw* cp, Tdst* dst, Tw sign, cudaStream_t st) {
    // tiles of 32 lines in shared memory while a tile fits
    const size_t tile_bytes = (size_t)m * 33 * sizeof(Tw);
    if (stride > 1 && m <= 1056 && tile_bytes <= 200 * 1024) {
        const int64_t ntiles = (outer * stride + 31) / 32;
        bool launched = false;
        auto go = [&](auto kern) -> mgard_status {
            MGB_TRY(allow_dynamic_smem((const void*)kern, tile_bytes));
            int grid = 0;
            MGB_TRY(resident_grid((const void*)kern, ST_WARPS * 32, tile_bytes, ntiles, &grid));
            MGB_LAUNCH("k_solve_tile", st, kern<<<grid, ST_WARPS * 32, tile_bytes, st>>>(x, outer, (int)m, stride, sub, inv, cp, dst, sign));
            launched = true;
            return MGARD_OK;
        };
        if (m <= 32) MGB_TRY(go(k_solve_tile<Tw, Tdst, 1>));
        else if (m <= 96) MGB_TRY(go(k_solve_tile<Tw, Tdst, 3>));
        else if (m <= 160) MGB_TRY(go(k_solve_tile<Tw, Tdst, 5>));
        else if (m <= 288) MGB_TRY(go(k_solve_tile<Tw, Tdst, 9>));
        else if (m <= 544) MGB_TRY(go(k_solve_tile<Tw, Tdst, 17>));
        else MGB_TRY(go(k_solve_tile<Tw, Tdst, 33>));
        if (launched) {
            MGB_CUDA(cudaGetLastError());
            return MGARD_OK;
        }
    }
    const int bx = 128;
    dim3 grid((unsigned)std::min<int64_t>((stride + bx - 1) / bx, 1LL << 30),
              (unsigned)std::min<int64_t>(outer, 65535), 1);
    MGB_LAUNCH("k_solve_lines", st,
               k_solve_lines<Tw, Tdst><<<grid, bx, 0, st>>>(x, outer, m, stride, sub, inv, cp, dst,
                                                            sign));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

// The per-warp segment pass (k_restrict_solve_seg): eight warps of K coarse
// rows, K in {2, 3, 5, 9, 17, 33} the smallest with 8 K >= mc (2^k + 1 coarse
// rows fill the segments exactly), sixteen warps of 33 up to 528 rows (float;
// in double, segments of at most 17 rows); chosen when its boxes fit in
// 200 KB of shared memory and the axis' interior rows are uniform.  *done
// stays false otherwise.
template <typename Tw>
mgard_status restrict_solve_seg(const Tw* in, Tw* out, int64_t outer, int64_t m, int64_t mc,
                                int64_t inner, const AxisT<Tw>& ax, cudaStream_t st, bool* done,
                                unsigned* status) {
    // rows 1 .. mc-2 must take the uniform window (the first and last rows
    // are taken from the tables)
    if (mc > 528 || (mc > 2 && (ax.rlo > 1 || ax.rhi < mc - 1))) return MGARD_OK;
    const int nw = mc <= 264 ? 8 : 16;
    int K = 33;
    if (nw == 8)
        for (int k : {2, 3, 5, 9, 17, 33})
            if ((int64_t)k * nw >= mc) {
                K = k;
                break;
            }
    if (sizeof(Tw) == 8 && K > 17) return MGARD_OK;   // 33 doubles per thread would spill
    const int KP = (K + 3) / 4 * 4;
    const int br = 2 * K + 3;
    const size_t bytes = ((size_t)nw * br * 32 + 3 * (size_t)nw * KP) * sizeof(Tw) +
                         (size_t)nw * 8 + 128;   // barriers, 128-byte alignment slack
    if (bytes > (size_t)200 * 1024) return MGARD_OK;
    // the last columns of each outer index go to 4-wide tail boxes when there are at most four
    const int64_t rem = inner % 32;
    const bool tails = rem >= 1 && rem <= 4;
    const int64_t tpo = tails ? inner / 32 : (inner + 31) / 32;
    const int64_t ntail = tails ? (outer + 7) / 8 : 0;
    const int64_t ntiles = outer * tpo + ntail;
    CUtensorMap tin, ttail;
    const uint64_t dims[3] = {(uint64_t)inner, (uint64_t)m, (uint64_t)outer};
    const uint64_t strides[2] = {(uint64_t)inner * sizeof(Tw), (uint64_t)(m * inner) * sizeof(Tw)};
    const uint32_t box[3] = {32u, (uint32_t)br, 1u};
    const uint32_t tbox[3] = {4u, (uint32_t)br, 8u};
    if (encode_tensor_map_3d(&tin, in, (int)sizeof(Tw), dims, strides, box) != MGARD_OK ||
        encode_tensor_map_3d(&ttail, in, (int)sizeof(Tw), dims, strides, tbox) != MGARD_OK) {
        cudaGetLastError();
        return MGARD_OK;   // another form runs instead
    }
    auto go = [&](auto kern, int threads) -> mgard_status {
        MGB_TRY(allow_dynamic_smem((const void*)kern, bytes));
        int grid = 0;
        MGB_TRY(resident_grid((const void*)kern, threads, bytes, ntiles, &grid));
        MGB_LAUNCH("k_restrict_solve", st, kern<<<grid, threads, bytes, st>>>(tin, ttail, out, outer, (int)m, (int)mc, inner, ax, br, tpo, ntail, status));
        MGB_CUDA(cudaGetLastError());
        *done = true;
        return MGARD_OK;
    };
    switch (K) {
        case 2: return go(k_restrict_solve_seg<Tw, 2, 8>, 256);
        case 3: return go(k_restrict_solve_seg<Tw, 3, 8>, 256);
        case 5: return go(k_restrict_solve_seg<Tw, 5, 8>, 256);
        case 9: return go(k_restrict_solve_seg<Tw, 9, 8>, 256);
        case 17: return go(k_restrict_solve_seg<Tw, 17, 8>, 256);
        default: break;
    }
    if constexpr (sizeof(Tw) == 4) {
        if (nw == 16) return go(k_restrict_solve_seg<Tw, 33, 16>, 512);
        return go(k_restrict_solve_seg<Tw, 33, 8>, 256);
    }
    return MGARD_OK;
}

// The TMA-staged pass: the fewest parts whose box (2 jp + 5 rows, at most
// 256) and shared memory fit three blocks per SM (72 KB), else two (110 KB),
// else one (200 KB).  *done stays false when the rows are not 16-byte aligned
// or no split fits.
template <typename Tw>
mgard_status restrict_solve_tma(const Tw* in, Tw* out, int64_t outer, int64_t m, int64_t mc,
                                int64_t inner, const AxisT<Tw>& ax, cudaStream_t st, bool* done,
                                unsigned* status) {
    if (!status || (inner * (int64_t)sizeof(Tw)) % 16 != 0 || ((uintptr_t)in & 15) != 0 ||
        inner > (int64_t(1) << 31) || outer > (int64_t(1) << 31))
        return MGARD_OK;
    MGB_TRY(restrict_solve_seg<Tw>(in, out, outer, m, mc, inner, ax, st, done, status));
    if (*done) return MGARD_OK;
    auto smem_for = [&](int parts, int* jp, int* br) {
        *jp = (int)((mc + parts - 1) / parts);
        *br = 2 * *jp + 5;
        return (size_t)(2 * (size_t)*br * 32 + (size_t)mc * 33 + 3 * (size_t)mc) * sizeof(Tw) +
               32 + 128;   // barriers and their alignment, and the slack for 128-byte alignment
    };
    int parts = 0, jp = 0, br = 0;
    size_t bytes = 0;
    for (size_t budget : {(size_t)72 * 1024, (size_t)110 * 1024, (size_t)200 * 1024}) {
        for (int pt = 1; pt <= 32 && !parts; ++pt) {
            bytes = smem_for(pt, &jp, &br);
            if (br <= 256 && bytes <= budget) parts = pt;
        }
        if (parts) break;
    }
    if (!parts) return MGARD_OK;
    CUtensorMap map;
    const uint64_t dims[3] = {(uint64_t)inner, (uint64_t)m, (uint64_t)outer};
    const uint64_t strides[2] = {(uint64_t)inner * sizeof(Tw), (uint64_t)(m * inner) * sizeof(Tw)};
    const uint32_t box[3] = {32u, (uint32_t)br, 1u};
    if (encode_tensor_map_3d(&map, in, (int)sizeof(Tw), dims, strides, box) != MGARD_OK) {
        cudaGetLastError();
        return MGARD_OK;   // the cp.async form runs instead
    }
    const int64_t ntiles = outer * ((inner + 31) / 32);
    auto go = [&](auto kern) -> mgard_status {
        MGB_TRY(allow_dynamic_smem((const void*)kern, bytes));
        int grid = 0;
        MGB_TRY(resident_grid((const void*)kern, ST_WARPS * 32, bytes, ntiles, &grid));
        MGB_LAUNCH("k_restrict_solve", st, kern<<<grid, ST_WARPS * 32, bytes, st>>>(map, out, outer, (int)m, (int)mc, inner, ax, jp, br, status));
        MGB_CUDA(cudaGetLastError());
        *done = true;
        return MGARD_OK;
    };
    if (mc <= 16) return go(k_restrict_solve_tma<Tw, 2>);
    if (mc <= 32) return go(k_restrict_solve_tma<Tw, 4>);
    if (mc <= 64) return go(k_restrict_solve_tma<Tw, 8>);
    if (mc <= 136) return go(k_restrict_solve_tma<Tw, 17>);
    if (mc <= 264) return go(k_restrict_solve_tma<Tw, 33>);
    return go(k_restrict_solve_tma<Tw, 65>);
}

template <typename Tw>
mgard_status restrict_solve_strided(const Tw* in, Tw* out, int64_t outer, int64_t m, int64_t mc,
                                    int64_t inner, const AxisT<Tw>& ax, cudaStream_t st,
                                    bool* done, unsigned* status) {
    *done = false;
    if (inner >= 2 && mc <= 520) {
        MGB_TRY(restrict_solve_tma<Tw>(in, out, outer, m, mc, inner, ax, st, done, status));
        if (*done) return MGARD_OK;
    }
    // restriction parts: the fewest that bring a block's shared memory to
    // 72 KB (three blocks per SM), else to 110 KB (two), else to 200 KB
    auto smem_for = [&](int parts, int* rows) {
        const int64_t jp = (mc + parts - 1) / parts;
        *rows = (int)std::min<int64_t>(m, 2 * jp + 5);
        return ((size_t)(*rows + mc) * 33 + 3 * (size_t)mc) * sizeof(Tw);
    };
    int parts = 0, ti_rows = 0;
    size_t bytes = 0;
    for (size_t budget : {(size_t)72 * 1024, (size_t)110 * 1024, (size_t)200 * 1024}) {
        for (int pt = 1; pt <= 4 && !parts; ++pt)
            if ((bytes = smem_for(pt, &ti_rows)) <= budget) parts = pt;
        if (parts) break;
    }
    if (inner < 2 || mc > 520 || !parts) return MGARD_OK;   // separate passes
    const int64_t ntiles = (outer * inner + 31) / 32;
    auto go = [&](auto kern) -> mgard_status {
        MGB_TRY(allow_dynamic_smem((const void*)kern, bytes));
        int grid = 0;
        MGB_TRY(resident_grid((const void*)kern, ST_WARPS * 32, bytes, ntiles, &grid));
        MGB_LAUNCH("k_restrict_solve", st, kern<<<grid, ST_WARPS * 32, bytes, st>>>(in, out, outer, (int)m, (int)mc, inner, ax, parts, ti_rows));
        MGB_CUDA(cudaGetLastError());
        *done = true;
        return MGARD_OK;
    };
    // K: rows per warp segment, ceil(mc / ST_WARPS) at most
    if (mc <= 16) return go(k_restrict_solve<Tw, 2>);
    if (mc <= 32) return go(k_restrict_solve<Tw, 4>);
    if (mc <= 64) return go(k_restrict_solve<Tw, 8>);
    if (mc <= 136) return go(k_restrict_solve<Tw, 17>);
    if (mc <= 264) return go(k_restrict_solve<Tw, 33>);
    return go(k_restrict_solve<Tw, 65>);
}

template <typename Tw, typename Tdst>
mgard_status solve_contiguous(Tw* x, int64_t lines, int64_t m, const Tw* sub, const Tw* inv,
                              const Tw* cp, Tdst* dst, Tw sign, cudaStream_t st, int64_t pitch) {
    if (pitch <= 0) pitch = m;
    const int grid = (int)std::min<int64_t>((lines + SW_WARPS - 1) / SW_WARPS, 148LL * 16);
    const int bs = SW_WARPS * 32;
#define MGB_SOLVE_WARP(EV) \
    MGB_LAUNCH("k_solve_warp", st, k_solve_warp<Tw, Tdst, EV><<<grid, bs, 0, st>>>(x, lines, (int)m, sub, inv, cp, dst, sign, pitch))
    if (m <= 32) MGB_SOLVE_WARP(1);
    else if (m <= 96) MGB_SOLVE_WARP(3);
    else if (m <= 160) MGB_SOLVE_WARP(5);
    else if (m <= 288) MGB_SOLVE_WARP(9);
    else if (m <= 544) MGB_SOLVE_WARP(17);
    else {
        bool done = false;
        if constexpr (sizeof(Tw) == 4) {   // double tables of this width would pass 48 KB
            if (m <= 1056) {
                MGB_SOLVE_WARP(33);
                done = true;
            }
        }
        // long lines: one thread per line in global memory
        if (!done) {   // rx_pitch keeps lines this long dense
            if (pitch != m) {
                set_error("solve_contiguous: padded lines over 1056 nodes");
                return MGARD_EINVAL;
            }
            return solve_strided<Tw, Tdst>(x, lines, m, 1, sub, inv, cp, dst, sign, st);
        }
    }
#undef MGB_SOLVE_WARP
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status Pyramid<T>::alloc(const Plan& p, cudaStream_t st) {
    lv.assign(p.L + 1, nullptr);
    size_t total = 0;
    std::vector<size_t> off(p.L + 1, 0);
    for (int l = 0; l < p.L; ++l) {
        off[l] = total;
        total += ((size_t)p.level_size(l) * sizeof(T) + 255) & ~size_t(255);
    }
    // restriction intermediates: the generic path shrinks axes 0..3 in order,
    // the row path shrinks axes 3..0; size for the larger of every prefix
    size_t tmax = 16;
    for (int l = 1; l <= p.L; ++l) {
        const size_t el = level_uses_fp64<T>(p, l) ? 8 : sizeof(T);
        for (int dir = 0; dir < 2; ++dir) {
            int64_t s[4];
            for (int a = 0; a < 4; ++a) s[a] = p.shape[l][a];
            for (int k = 0; k < 4; ++k) {
                const int a = dir == 0 ? k : 3 - k;
                if (p.n4[a] == 1) continue;
                s[a] = p.shape[l - 1][a];
                // the row path pads its rows of the coarse x extent (rx_pitch)
                if (dir == 1 && a == 3 && rows3_ok(p))
                    s[a] = el == 8 ? rx_pitch<double>(s[a]) : rx_pitch<float>(s[a]);
                tmax = std::max(tmax, (size_t)(s[0] * s[1] * s[2] * s[3]) * el);
            }
        }
    }
    const int Lt = tail_levels(p);   // the one-block tail's scratch lives here too
    if (Lt) tmax = std::max(tmax, 2 * (size_t)p.level_size(Lt) * sizeof(T));
    MGB_TRY(store.alloc(total, st));
    MGB_TRY(temp0.alloc(tmax, st));
    MGB_TRY(temp1.alloc(tmax, st));
    for (int l = 0; l < p.L; ++l) lv[l] = (T*)((char*)store.p + off[l]);
    return MGARD_OK;
}

int64_t mass_norm_parts(const Plan& p, int l) {
    if (rows3_ok(p)) return rows3_mass_norm_blocks(p, l);
    const dim3 g = grid3(p.level<float>(l).n, RED_THREADS, 8, 74);
    return (int64_t)g.x * g.y * g.z;
}

int64_t energy_parts_total(const Plan& p) {
    int64_t t = 0;
    for (int l = 0; l <= p.L; ++l) t += mass_norm_parts(p, l);
    return t;
}

int64_t energy_parts_offset(const Plan& p, int l) {
    int64_t t = 0;
    for (int k = 0; k < l; ++k) t += mass_norm_parts(p, k);
    return t;
}

template <typename T>
mgard_status mass_norm2_partials(const Plan& p, int l, const T* u, double* part, cudaStream_t st) {
    if (rows3_ok(p)) return rows3_mass_norm<T>(p, l, u, part, st);
    const Level<T>& lv = p.level<T>(l);   // holds the mass tables of level l
    const dim3 g = grid3(lv.n, RED_THREADS, 8, 74);   // fixed grid: deterministic partial sums
    MGB_LAUNCH("k_mass_norm", st, k_mass_norm<T><<<g, RED_THREADS, 0, st>>>(u, lv, part));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status mass_norm2(const Plan& p, int l, const T* u, double* out, cudaStream_t st) {
    const size_t nb = (size_t)mass_norm_parts(p, l);
    DevBuf part;
    MGB_TRY(part.alloc(nb * sizeof(double), st));
    MGB_TRY(mass_norm2_partials<T>(p, l, u, part.as<double>(), st));
    std::vector<double> h(nb);
    MGB_CUDA(cudaMemcpyAsync(h.data(), part.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (size_t i = 0; i < nb; ++i) s += h[i];
    *out = s;
    return MGARD_OK;
}

template <typename T>
mgard_status max_abs_partials(const T* a, int64_t n, double* part, unsigned* status,
                              cudaStream_t st) {
    MGB_LAUNCH("k_maxabs", st, k_maxabs<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, nullptr, n, part, status));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status max_abs(const T* a, const T* b, int64_t n, double* out, unsigned* status,
                     cudaStream_t st) {
    DevBuf part, stat;
    MGB_TRY(part.alloc(RED_BLOCKS * sizeof(double), st));
    MGB_TRY(stat.alloc(sizeof(unsigned), st));
    MGB_CUDA(cudaMemsetAsync(stat.p, 0, sizeof(unsigned), st));
    MGB_LAUNCH("k_maxabs", st, k_maxabs<T><<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, n, part.as<double>(), stat.as<unsigned>()));
    MGB_CUDA(cudaGetLastError());
    double h[RED_BLOCKS];
    unsigned hs = 0;
    MGB_CUDA(cudaMemcpyAsync(h, part.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaMemcpyAsync(&hs, stat.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    double m = 0.0;
    for (int i = 0; i < RED_BLOCKS; ++i) m = std::max(m, h[i]);
    *out = m;
    if (status) *status = hs;
    return MGARD_OK;
}

template <typename T>
mgard_status difference(const T* a, const T* b, double* y, int64_t n, cudaStream_t st) {
    MGB_LAUNCH("k_difference", st, k_difference<T><<<grid_for(n, 256), 256, 0, st>>>(a, b, y, n));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status decompose_pyramid(const Plan& p, const T* in, T* top, Pyramid<T>& py,
                               cudaStream_t st, double* E, double* Epart, T* zs) {
    if (zs && !rows3_ok(p)) {
        set_error("symbol-order coefficients need the row kernels");
        return MGARD_EINVAL;
    }
    // small levels in one launch (row-kernel shapes).  In symbol order the
    // tail leaves every level's nodal values in the pyramid, so their
    // energies are taken afterwards; in place it overwrites them, so levels
    // with energies requested run level by level.
    const int Lt = (rows3_ok(p) && (zs || (!E && !Epart))) ? tail_levels(p) : 0;
    py.tail_pending = false;
    for (int l = p.L; l >= 1; --l) {
        const T* src = l == p.L ? in : py.lv[l];
        if (l == Lt && py.defer_tail && zs && !E && !Epart) {   // the caller runs the tail
            py.tail_pending = true;
            return MGARD_OK;
        }
        if (l == Lt) {
            MGB_TRY(tail_decompose<T>(p, Lt, py, src, zs, top, st));
            for (int k = Lt; k >= 1; --k) {   // level 0 follows below
                const T* uk = k == p.L ? in : py.lv[k];
                if (E) MGB_TRY(mass_norm2<T>(p, k, uk, &E[k], st));
                if (Epart) MGB_TRY(mass_norm2_partials<T>(p, k, uk, Epart + energy_parts_offset(p, k), st));
            }
            break;
        }
        T* dst = zs ? zs : (l == p.L ? top : py.lv[l]);
        const int64_t zoff = zs ? p.offset[l] : -1;
        if (E) MGB_TRY(mass_norm2<T>(p, l, src, &E[l], st));
        if (Epart) MGB_TRY(mass_norm2_partials<T>(p, l, src, Epart + energy_parts_offset(p, l), st));
        bool x_done = false;   // the coefficient kernel restricted along x into temp0
        if (rows3_ok(p)) {
            MGB_TRY(rows3_coeff<T>(p, l, src, dst, py.lv[l - 1], st, zoff, py.temp0.p,
                                   level_uses_fp64<T>(p, l), &x_done));
        } else {
            MGB_LAUNCH("k_coeff_gather", st,
                       k_coeff_gather<T><<<grid3(p.level<T>(l).n, 128), 128, 0, st>>>(
                           src, dst, py.lv[l - 1], p.level<T>(l)));
            MGB_CUDA(cudaGetLastError());
        }
        MGB_TRY(correct<T>(p, l, dst, py.lv[l - 1], py.temp0.p, py.temp1.p, T(1), st, zoff,
                           x_done, py.status));
    }
    const T* u0 = p.L ? py.lv[0] : in;
    if (E) MGB_TRY(mass_norm2<T>(p, 0, u0, &E[0], st));
    if (Epart) MGB_TRY(mass_norm2_partials<T>(p, 0, u0, Epart, st));
    if (zs)   // level 0 leads the symbol order
        MGB_CUDA(cudaMemcpyAsync(zs, u0, p.count[0] * sizeof(T), cudaMemcpyDeviceToDevice, st));
    return MGARD_OK;
}

template <typename T>
mgard_status decompose_finish(const Plan& p, Pyramid<T>& py, T* zs, cudaStream_t st) {
    if (zs && p.L)   // level 0 leads the symbol order
        MGB_CUDA(cudaMemcpyAsync(zs, py.lv[0], p.count[0] * sizeof(T), cudaMemcpyDeviceToDevice, st));
    py.tail_pending = false;
    return MGARD_OK;
}

template <typename T>
mgard_status recompose_pyramid(const Plan& p, const T* top, T* out, Pyramid<T>& py,
                               cudaStream_t st, const T* zs) {
    if (zs && !rows3_ok(p)) {
        set_error("symbol-order coefficients need the row kernels");
        return MGARD_EINVAL;
    }
    if (p.L == 0) {
        const T* src = zs ? zs : top;
        if (out != src)
            MGB_CUDA(cudaMemcpyAsync(out, src, p.total() * sizeof(T), cudaMemcpyDeviceToDevice, st));
        return MGARD_OK;
    }
    if (zs) MGB_CUDA(cudaMemcpyAsync(py.lv[0], zs, p.count[0] * sizeof(T), cudaMemcpyDeviceToDevice, st));
    // small levels in one launch (row-kernel shapes)
    const int Lt = rows3_ok(p) ? tail_levels(p) : 0;
    if (Lt && py.defer_tail && zs) {   // the caller runs the tail, then calls again with tail_done
        py.tail_pending = true;
        return MGARD_OK;
    }
    if (Lt && !py.tail_done) MGB_TRY(tail_recompose<T>(p, Lt, py, zs, top, Lt == p.L ? out : py.lv[Lt], st));
    py.tail_pending = false;
    for (int l = Lt + 1; l <= p.L; ++l) {
        const T* z = zs ? zs : (l == p.L ? top : py.lv[l]);
        const int64_t zoff = zs ? p.offset[l] : -1;
        T* dst = l == p.L ? out : py.lv[l];
        MGB_TRY(correct<T>(p, l, z, py.lv[l - 1], py.temp0.p, py.temp1.p, T(-1), st, zoff, false,
                           py.status));
        if (rows3_ok(p)) {
            MGB_TRY(rows3_fill<T>(p, l, z, py.lv[l - 1], dst, st, zoff));
        } else {
            MGB_LAUNCH("k_fill", st, k_fill<T><<<grid3(p.level<T>(l).n, 128), 128, 0, st>>>(
                                         z, py.lv[l - 1], dst, p.level<T>(l)));
            MGB_CUDA(cudaGetLastError());
        }
    }
    return MGARD_OK;
}

template <typename T>
mgard_status scatter_levels(const Plan& p, const Pyramid<T>& py, T* data, cudaStream_t st) {
    Shape4 fine;
    for (int a = 0; a < 4; ++a) fine.n[a] = p.n4[a];
    for (int l = 0; l < p.L; ++l) {
        MGB_LAUNCH("k_layout", st, k_layout<T, true><<<grid3(p.lidx[l].n, 128), 128, 0, st>>>(
            py.lv[l], data, p.lidx[l], p.level<T>(l), l > 0 ? 1 : 0, fine));
        MGB_CUDA(cudaGetLastError());
    }
    return MGARD_OK;
}

template <typename T>
mgard_status gather_levels(const Plan& p, const T* data, Pyramid<T>& py, cudaStream_t st) {
    Shape4 fine;
    for (int a = 0; a < 4; ++a) fine.n[a] = p.n4[a];
    for (int l = 0; l < p.L; ++l) {
        MGB_LAUNCH("k_layout", st, k_layout<T, false><<<grid3(p.lidx[l].n, 128), 128, 0, st>>>(
            py.lv[l], (T*)data, p.lidx[l], p.level<T>(l), 0, fine));
        MGB_CUDA(cudaGetLastError());
    }
    return MGARD_OK;
}

#define INST(T)                                                                               \
    template struct Pyramid<T>;                                                               \
    template mgard_status decompose_pyramid<T>(const Plan&, const T*, T*, Pyramid<T>&,         \
                                               cudaStream_t, double*, double*, T*);            \
    template mgard_status decompose_finish<T>(const Plan&, Pyramid<T>&, T*, cudaStream_t);     \
    template mgard_status max_abs_partials<T>(const T*, int64_t, double*, unsigned*,           \
                                              cudaStream_t);                                   \
    template mgard_status mass_norm2_partials<T>(const Plan&, int, const T*, double*,          \
                                                 cudaStream_t);                        \
    template mgard_status recompose_pyramid<T>(const Plan&, const T*, T*, Pyramid<T>&,         \
                                               cudaStream_t, const T*);                       \
    template mgard_status scatter_levels<T>(const Plan&, const Pyramid<T>&, T*, cudaStream_t); \
    template mgard_status gather_levels<T>(const Plan&, const T*, Pyramid<T>&, cudaStream_t);  \
    template mgard_status max_abs<T>(const T*, const T*, int64_t, double*, unsigned*,          \
                                     cudaStream_t);                                           \
    template mgard_status mass_norm2<T>(const Plan&, int, const T*, double*, cudaStream_t);    \
    template mgard_status difference<T>(const T*, const T*, double*, int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST
#define INST_SOLVE(Tw, Td)                                                                       \
    template mgard_status solve_strided<Tw, Td>(Tw*, int64_t, int64_t, int64_t, const Tw*,       \
                                                const Tw*, const Tw*, Td*, Tw, cudaStream_t);    \
    template mgard_status solve_contiguous<Tw, Td>(Tw*, int64_t, int64_t, const Tw*, const Tw*,  \
                                                   const Tw*, Td*, Tw, cudaStream_t, int64_t);
INST_SOLVE(float, float)
INST_SOLVE(double, float)
INST_SOLVE(double, double)
#undef INST_SOLVE
template mgard_status restrict_solve_strided<float>(const float*, float*, int64_t, int64_t, int64_t,
                                                    int64_t, const AxisT<float>&, cudaStream_t,
                                                    bool*, unsigned*);
template mgard_status restrict_solve_strided<double>(const double*, double*, int64_t, int64_t,
                                                     int64_t, int64_t, const AxisT<double>&,
                                                     cudaStream_t, bool*, unsigned*);

}  // namespace mgb
