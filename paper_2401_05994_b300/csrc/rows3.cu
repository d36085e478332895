// Row kernels for grids with at most three active axes (see rows3.cuh).
//
// Same mathematics as the generic 4D kernels in multilevel.cu and
// quantize.cu (paper, "Software design": coefficients, load vector,
// coarse solve, correction, level-wise quantization); only the work
// decomposition differs.
#include <algorithm>

#include <type_traits>

#include "rows3.cuh"

namespace mgb {

namespace {

constexpr int RT = 256;              // threads per block: 8 warps, one x-row per warp
constexpr int WPB = RT / 32;
constexpr int64_t ROW_BLOCKS = 148 * 16;   // the autotuner prefers 16 resident blocks per SM on large levels
// Elements per lane per batch: all loads of a batch are issued before its
// stores, so a batch covering a whole row puts the entire row in flight.
// U is chosen per launch from the row length (2, 5, 9 or 17 -> rows of up to
// 64, 160, 288, 544 elements in one batch).

inline int row_grid(int64_t rows, int bpsm = 0) {
    const int64_t cap = bpsm > 0 ? 148LL * bpsm : ROW_BLOCKS;
    return (int)std::min<int64_t>(std::max<int64_t>((rows + WPB - 1) / WPB, 1), cap);
}

// Node classes follow from the hierarchy rule (coarse = even positions plus
// the last one), so positions are arithmetic; only weights come from tables.
__device__ inline bool is_coarse(int i, int m) { return (i & 1) == 0 || i == m - 1; }
__device__ inline int coarse_index(int i, int m, int mc) { return i == m - 1 ? mc - 1 : i >> 1; }
__device__ inline int restrict_center(int J, int m, int mc) { return J == mc - 1 ? m - 1 : 2 * J; }
__device__ inline int coarse_before(int i) { return (i + 1) >> 1; }

// Row loops take 32 * U elements per pass (U per lane).  Extents of 2^k + 1
// would leave a last pass of one element that costs a full pass of latency,
// so a remainder of at most one warp width joins the pass before it: this
// pass (starting at element `base`) takes U + 1 elements per lane when the
// row ends within 32 elements after it.
__device__ inline bool absorbs_tail(int base, int n, int U) {
    return base + 32 * U < n && base + 32 * (U + 1) >= n;
}

// Elements of T that fill a multiple of 8 bytes (per-warp shared-memory rows).
template <typename T>
__host__ __device__ inline int pad8(int n) { return sizeof(T) >= 8 ? n : (n + 1) & ~1; }

// Rounding spelled out, so the staged and per-element forms of the
// interpolation (below) give the same bits whatever the compiler contracts.
__device__ inline float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ inline double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ inline float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ inline double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// The up-to-four coarse source rows of a row combined along z and y at fine
// x position xf: sum_k rw[k] rows[k][xf] over the rows in use (row 0 always).
template <typename T>
__device__ inline T combine_rows(const T* const rows[4], const T rw[4], const bool use[4], int xf) {
    T a = rmul(rw[0], rows[0][xf]);
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (use[k]) a = rfma(rw[k], rows[k][xf], a);
    return a;
}

// Interpolation along x between the combined values at the two coarse
// neighbours (for a coarse x both are the node itself, with weights 1, 0).
template <typename T>
__device__ inline T lerp_x(T wl, T rl, T wr, T rr) { return rfma(wl, rl, rmul(wr, rr)); }

// Coefficients of level l in symbol order (ZS kernels): the nodes new on the
// level, row-major, starting at symbol offset `zoff`.  Row (z, y) of the level
// grid starts at zoff + r nx minus the coarse-grid nodes before it; on a row
// whose z and y are both coarse only the odd positions are new, so its x
// lands at x - coarse_before(x).
__device__ inline int64_t zs_row_base(int64_t zoff, int64_t r, int nx, int z, int y, int nz,
                                      int ny, int ncy, int ncx) {
    const bool zc = (z & 1) == 0 || z == nz - 1;
    int64_t before = (int64_t)coarse_before(z) * ncy * ncx;
    if (zc) before += (int64_t)coarse_before(y) * ncx;
    (void)ny;
    return zoff + r * nx - before;
}

// Interpolation sources of one index along one axis (y or z).
template <typename T>
struct Src {
    int p[2];     // fine positions (decomposition) or coarse indices (fill)
    T w[2];
    int n;        // 1 = coarse node, 2 = new node
    int J;        // coarse index when n == 1
};

template <typename T>
__device__ inline Src<T> sources(const AxisT<T>& ax, int i, int m, int mc, bool coarse_idx) {
    Src<T> s;
    if (is_coarse(i, m)) {
        s.J = coarse_index(i, m, mc);
        s.p[0] = coarse_idx ? s.J : i;
        s.w[0] = T(1);
        s.n = 1;
    } else {
        const int left = (i - 1) >> 1;
        s.p[0] = coarse_idx ? left : i - 1;
        s.p[1] = coarse_idx ? left + 1 : i + 1;
        s.w[0] = ax.wl[i];
        s.w[1] = ax.wr[i];
        s.n = 2;
        s.J = -1;
    }
    return s;
}

inline int pick_u(int64_t nx) {
    // larger batches cost registers and occupancy more than they gain in
    // bytes in flight; the next row is prefetched into L2 instead
    return nx <= 64 ? 2 : 4;
}

template <int V>
struct UTag {
    static constexpr int value = V;
};

// Calls f(UTag<U>{}) with the batch size for row length nx.
template <typename F>
void with_u(int64_t nx, F&& f) {
    if (pick_u(nx) == 2) f(UTag<2>{});
    else f(UTag<4>{});
}

// Kernels that keep few values per element afford batches of 8.
template <typename F>
void with_u8(int64_t nx, F&& f) {
    if (nx <= 64) f(UTag<2>{});
    else if (nx <= 160) f(UTag<4>{});
    else f(UTag<8>{});
}

// Batch size from a tuned launch shape (2, 4, 8 or 16), else the built-in rule
// (`light`: the with_u8 rule, otherwise the with_u rule).
template <typename F>
void with_cfg(const RowCfg& c, int64_t nx, bool light, F&& f) {
    if (c.u == 2) f(UTag<2>{});
    else if (c.u == 4) f(UTag<4>{});
    else if (c.u == 8) f(UTag<8>{});
    else if (c.u == 16) f(UTag<16>{});
    else if (light) with_u8(nx, f);
    else with_u(nx, f);
}

// Ask the TMA unit to pull a row into L2 (no registers are held).  The
// instruction wants 16-byte boundaries: the start is rounded down (into the
// previous row, which always exists for a row after the first) and the end is
// rounded down too, so the range never reaches past the array.
__device__ inline void prefetch_l2(const void* p, size_t bytes) {
    const uintptr_t a = (uintptr_t)p & ~uintptr_t(15);
    const uintptr_t e = ((uintptr_t)p + bytes) & ~uintptr_t(15);
    if (e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a))
                     : "memory");
}

// Lane 0 of a warp prefetches the row the warp will process next.
#define PREFETCH_NEXT_ROW(base, r, rows, rowlen, esize)                                       \
    do {                                                                                      \
        const int64_t nr_ = (r) + (int64_t)gridDim.x * WPB;                                   \
        if ((threadIdx.x & 31) == 0 && nr_ < (rows))                                          \
            prefetch_l2((const char*)(base) + nr_ * (int64_t)(rowlen) * (esize),              \
                        (size_t)(rowlen) * (esize));                                          \
    } while (0)

// The same for rows of coefficients in symbol order (ZS kernels): the next
// row starts at zs_row_base and is at most nx long; the range is clipped to
// the level's run [zoff, zoff + count) of the array.
#define PREFETCH_NEXT_ZS_ROW(base, zoff, r, nz, ny, nx, ncz, ncy, ncx, esize)                 \
    do {                                                                                      \
        const int64_t nr_ = (r) + (int64_t)gridDim.x * WPB;                                   \
        if ((threadIdx.x & 31) == 0 && nr_ < (int64_t)(nz) * (ny)) {                          \
            const int z_ = (int)((uint32_t)nr_ / (uint32_t)(ny));                             \
            const int y_ = (int)(nr_ - (int64_t)z_ * (ny));                                   \
            const int64_t b_ = zs_row_base(zoff, nr_, nx, z_, y_, nz, ny, ncy, ncx);          \
            const int64_t end_ = (zoff) + (int64_t)(nz) * (ny) * (nx) -                        \
                                 (int64_t)(ncz) * (ncy) * (ncx);                               \
            const int64_t len_ = b_ + (nx) < end_ ? (nx) : end_ - b_;                         \
            if (len_ > 0)                                                                     \
                prefetch_l2((const char*)(base) + b_ * (esize), (size_t)len_ * (esize));      \
        }                                                                                     \
    } while (0)

#define WARP_ROWS(rows, r)                                                                    \
    for (int64_t r = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5); r < (rows);             \
         r += (int64_t)gridDim.x * WPB)

// -- coefficients (decomposition step 1) --------------------------------------
// The x restriction of one fine row at coarse index J: the five-tap window
// of P^T M_l around fine 2J (uniform weights rwi for J in [rlo, rhi), else
// the table rw[J*5 ..]), with fetch(ip) giving z at fine x = ip.  On rows of
// the coarser grid (rowc) z vanishes at coarse x positions: in the uniform
// window those are the even taps, elsewhere they are skipped.
template <typename Tout, typename F>
__device__ inline Tout restrict_row_at(int J, int nx, int ncx, bool rowc, const Tout wi[5],
                                       int rlo, int rhi, const Tout* __restrict__ rw, F fetch) {
    if (J >= rlo && J < rhi) {
        const Tout e0 = rowc ? Tout(0) : fetch(2 * J - 2);
        const Tout e1 = fetch(2 * J - 1);
        const Tout e2 = rowc ? Tout(0) : fetch(2 * J);
        const Tout e3 = fetch(2 * J + 1);
        const Tout e4 = rowc ? Tout(0) : fetch(2 * J + 2);
        Tout a = wi[0] * e0;
        a += wi[1] * e1;
        a += wi[2] * e2;
        a += wi[3] * e3;
        a += wi[4] * e4;
        return a;
    }
    const int f = restrict_center(J, nx, ncx);
    Tout acc = Tout(0);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int ip = f - 2 + t;
        if (ip < 0 || ip >= nx) continue;
        if (rowc && is_coarse(ip, nx)) continue;   // coarse node: z = 0 (not read)
        acc += rw[J * 5 + t] * fetch(ip);
    }
    return acc;
}

// STAGE: as in the fill kernel, the source rows are combined along y and z
// at the coarse x positions into a shared-memory row R first.  RX: the row's
// coefficients are also kept in shared memory (zero at coarse nodes of the
// coarser grid's rows) and restricted along x into rx (rows of ncx values in
// Tw), the first step of the coarse-grid correction.
// PAIR (with STAGE, on an odd extent whose interpolation weights are the
// uniform ones everywhere): lane p takes the node pair (2p, 2p+1), the
// coarse node and the new node after it, so parity, coarse index and
// weights are known without per-element tests; same arithmetic, same bits.
template <typename T, int U, bool ZS, bool STAGE, bool RX, typename Tw, bool PAIR>
__global__ void __launch_bounds__(RT) k3_coeff(const T* in, T* out, T* __restrict__ coarse,
                                               Level<T> lv, int64_t zoff, Tw* __restrict__ rx,
                                               AxisT<Tw> axw, int xpitch) {
    static_assert(!PAIR || STAGE, "pairs read the staged row");
    extern __shared__ __align__(16) unsigned char stage_raw[];
    const int nz = (int)lv.n[1], ny = (int)lv.n[2], nx = (int)lv.n[3];
    const int ncz = (int)lv.nc[1], ncy = (int)lv.nc[2], ncx = (int)lv.nc[3];
    const T* __restrict__ wlx = lv.ax[3].wl;
    const T* __restrict__ wrx = lv.ax[3].wr;
    const int ireg = lv.ax[3].ireg;
    const int lane = threadIdx.x & 31;
    WARP_ROWS((int64_t)nz * ny, r) {
        const int z = (int)((uint32_t)r / (uint32_t)ny), y = (int)(r - (int64_t)z * ny);
        const Src<T> sz = sources(lv.ax[1], z, nz, ncz, false);
        const Src<T> sy = sources(lv.ax[2], y, ny, ncy, false);
        // up to four source rows (z0|z1) x (y0|y1), fixed slots with warp-uniform use flags
        const bool zy2 = sy.n == 2, zz2 = sz.n == 2;
        const T* rows[4] = {in + ((int64_t)sz.p[0] * ny + sy.p[0]) * nx,
                            in + ((int64_t)sz.p[0] * ny + (zy2 ? sy.p[1] : sy.p[0])) * nx,
                            in + ((int64_t)(zz2 ? sz.p[1] : sz.p[0]) * ny + sy.p[0]) * nx,
                            in + ((int64_t)(zz2 ? sz.p[1] : sz.p[0]) * ny + (zy2 ? sy.p[1] : sy.p[0])) * nx};
        const T rw[4] = {sz.w[0] * sy.w[0], zy2 ? sz.w[0] * sy.w[1] : T(0),
                         zz2 ? sz.w[1] * sy.w[0] : T(0), (zz2 && zy2) ? sz.w[1] * sy.w[1] : T(0)};
        const bool use[4] = {true, zy2, zz2, zz2 && zy2};
        const bool rowc = sz.n == 1 && sy.n == 1;
        PREFETCH_NEXT_ROW(in, r, (int64_t)nz * ny, nx, sizeof(T));
        const T* urow = in + r * nx;
        T* orow = ZS ? out + zs_row_base(zoff, r, nx, z, y, nz, ny, ncy, ncx) : out + r * nx;
        T* crow = rowc ? coarse + ((int64_t)sz.J * ncy + sy.J) * ncx : nullptr;
        // per-warp rows padded to 8 bytes, so the coefficient pairs go to
        // shared memory as one access each
        const int ncxp = pad8<T>(ncx), nxp = pad8<T>(nx);
        T* R = reinterpret_cast<T*>(stage_raw) + (threadIdx.x >> 5) * ((STAGE ? ncxp : 0) + (RX ? nxp : 0));
        T* Z = R + (STAGE ? ncxp : 0);
        if (STAGE) {
            // coarse node J sits at fine x = 2J, the last one at nx - 1
            for (int j = lane; j < ncx; j += 32) R[j] = combine_rows(rows, rw, use, min(2 * j, nx - 1));
            __syncwarp();
        }
        if (PAIR) {
            for (int p0 = lane; p0 < ncx; p0 += 32 * U) {
                const bool tail = absorbs_tail(p0 - lane, ncx, U);
                // FULL: U pairs per lane, every one with its new node inside
                // the row and no tail, so no element is tested
                auto pass = [&](auto full_tag) {
                    constexpr bool FULL = decltype(full_tag)::value;
                    constexpr int NJ = FULL ? U : U + 1;
                    T u0[U + 1], u1[U + 1];
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {   // loads first
                        const int p = p0 + 32 * j;
                        if (!FULL && (p >= ncx || (j == U && !tail))) continue;
                        u0[j] = urow[2 * p];
                        if (FULL || p + 1 < ncx) u1[j] = urow[2 * p + 1];
                    }
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int p = p0 + 32 * j;
                        if (!FULL && (p >= ncx || (j == U && !tail))) continue;
                        const T r0 = R[p];
                        // coarse x = 2p: the interpolant is R[p] itself
                        const T a0 = lerp_x(T(1), r0, T(0), r0);
                        T c0 = T(0);
                        if (rowc) {
                            crow[p] = u0[j];
                        } else {
                            c0 = u0[j] - a0;
                            orow[2 * p] = c0;
                        }
                        if (FULL || p + 1 < ncx) {   // new x = 2p + 1 between coarse p and p + 1
                            const T c = u1[j] - lerp_x(T(0.5), r0, T(0.5), R[p + 1]);
                            orow[(ZS && rowc) ? p : 2 * p + 1] = c;
                            if (RX) {
                                if (sizeof(T) == 4)
                                    *reinterpret_cast<float2*>(Z + 2 * p) = make_float2((float)c0, (float)c);
                                else {
                                    Z[2 * p] = c0;
                                    Z[2 * p + 1] = c;
                                }
                            }
                        } else if (RX) {
                            Z[2 * p] = c0;
                        }
                    }
                };
                if (!tail && p0 - lane + 32 * U < ncx) pass(std::true_type{});
                else pass(std::false_type{});
                if (tail) break;
            }
        } else
        for (int x0 = lane; x0 < nx; x0 += 32 * U) {
            const bool tail = absorbs_tail(x0 - lane, nx, U);
            T u[U + 1], acc[U + 1];
#pragma unroll
            for (int j = 0; j < U + 1; ++j) {
                const int x = x0 + 32 * j;
                acc[j] = T(0);
                if (x >= nx || (j == U && !tail)) continue;
                u[j] = urow[x];
                // coarse x: neighbours x, x with weights (1, 0); new x: x-1, x+1
                const bool cx = is_coarse(x, nx);
                const int d = cx ? 0 : 1;
                T wl = (x & 1) ? T(0.5) : T(1), wr = (x & 1) ? T(0.5) : T(0);
                if (x >= ireg) {
                    wl = wlx[x];
                    wr = wrx[x];
                }
                if (STAGE) {
                    const int jl = cx ? coarse_index(x, nx, ncx) : (x - 1) >> 1;
                    acc[j] = lerp_x(wl, R[jl], wr, R[cx ? jl : jl + 1]);
                } else {
                    acc[j] = lerp_x(wl, combine_rows(rows, rw, use, x - d), wr,
                                    combine_rows(rows, rw, use, x + d));
                }
            }
#pragma unroll
            for (int j = 0; j < U + 1; ++j) {
                const int x = x0 + 32 * j;
                if (x >= nx || (j == U && !tail)) continue;
                if (rowc && is_coarse(x, nx)) {
                    crow[coarse_index(x, nx, ncx)] = u[j];
                    if (RX) Z[x] = T(0);
                } else {
                    const T c = u[j] - acc[j];
                    orow[(ZS && rowc) ? x - coarse_before(x) : x] = c;
                    if (RX) Z[x] = c;
                }
            }
            if (tail) break;
        }
        if (RX) {
            __syncwarp();
            Tw wi[5];
#pragma unroll
            for (int t = 0; t < 5; ++t) wi[t] = axw.rwi[t];
            Tw* xrow = rx + r * xpitch;
            for (int J = lane; J < ncx; J += 32) {
                if (sizeof(T) == 4 && sizeof(Tw) == 4 && J >= axw.rlo && J < axw.rhi) {
                    // the uniform window from two pair loads and one element (Z
                    // holds 0 at the coarse nodes of a coarse row)
                    const float2 a = *reinterpret_cast<const float2*>(Z + 2 * J - 2);
                    const float2 b = *reinterpret_cast<const float2*>(Z + 2 * J);
                    Tw acc = wi[0] * (Tw)a.x;
                    acc += wi[1] * (Tw)a.y;
                    acc += wi[2] * (Tw)b.x;
                    acc += wi[3] * (Tw)b.y;
                    acc += wi[4] * (Tw)Z[2 * J + 2];
                    xrow[J] = acc;
                } else {
                    xrow[J] = restrict_row_at<Tw>(J, nx, ncx, rowc, wi, axw.rlo, axw.rhi, axw.rw,
                                                  [&](int ip) { return (Tw)Z[ip]; });
                }
            }
        }
        if (STAGE || RX) __syncwarp();   // R and Z are rewritten by the warp's next row
    }
}

// -- recomposition fill ---------------------------------------------------------
// STAGE: the up-to-four coarse rows are first combined along y and z into
// one row R of the coarse x grid in shared memory (each coarse value loaded
// once), and the x interpolation then reads R; otherwise every element
// interpolates each coarse row itself.
template <typename T, int U, bool ZS, bool STAGE, bool PAIR>
__global__ void __launch_bounds__(RT) k3_fill(const T* zin, const T* __restrict__ coarse, T* out,
                                              Level<T> lv, int64_t zoff) {
    static_assert(!PAIR || STAGE, "pairs read the staged row");
    extern __shared__ __align__(16) unsigned char stage_raw[];
    const int nz = (int)lv.n[1], ny = (int)lv.n[2], nx = (int)lv.n[3];
    const int ncz = (int)lv.nc[1], ncy = (int)lv.nc[2], ncx = (int)lv.nc[3];
    const T* __restrict__ wlx = lv.ax[3].wl;
    const T* __restrict__ wrx = lv.ax[3].wr;
    const int ireg = lv.ax[3].ireg;
    const int lane = threadIdx.x & 31;
    WARP_ROWS((int64_t)nz * ny, r) {
        const int z = (int)((uint32_t)r / (uint32_t)ny), y = (int)(r - (int64_t)z * ny);
        const Src<T> sz = sources(lv.ax[1], z, nz, ncz, true);
        const Src<T> sy = sources(lv.ax[2], y, ny, ncy, true);
        const bool zy2 = sy.n == 2, zz2 = sz.n == 2;
        const T* rows[4] = {coarse + ((int64_t)sz.p[0] * ncy + sy.p[0]) * ncx,
                            coarse + ((int64_t)sz.p[0] * ncy + (zy2 ? sy.p[1] : sy.p[0])) * ncx,
                            coarse + ((int64_t)(zz2 ? sz.p[1] : sz.p[0]) * ncy + sy.p[0]) * ncx,
                            coarse + ((int64_t)(zz2 ? sz.p[1] : sz.p[0]) * ncy + (zy2 ? sy.p[1] : sy.p[0])) * ncx};
        const T rw[4] = {sz.w[0] * sy.w[0], zy2 ? sz.w[0] * sy.w[1] : T(0),
                         zz2 ? sz.w[1] * sy.w[0] : T(0), (zz2 && zy2) ? sz.w[1] * sy.w[1] : T(0)};
        const bool use[4] = {true, zy2, zz2, zz2 && zy2};
        const bool rowc = sz.n == 1 && sy.n == 1;
        if (ZS) PREFETCH_NEXT_ZS_ROW(zin, zoff, r, nz, ny, nx, ncz, ncy, ncx, sizeof(T));
        else PREFETCH_NEXT_ROW(zin, r, (int64_t)nz * ny, nx, sizeof(T));
        const T* zrow = ZS ? zin + zs_row_base(zoff, r, nx, z, y, nz, ny, ncy, ncx) : zin + r * nx;
        T* orow = out + r * nx;
        T* R = reinterpret_cast<T*>(stage_raw) + (threadIdx.x >> 5) * pad8<T>(ncx);
        if (STAGE) {
            for (int j = lane; j < ncx; j += 32) R[j] = combine_rows(rows, rw, use, j);
            __syncwarp();
        }
        if (PAIR) {   // lane p: coarse x = 2p and new x = 2p + 1 (see k3_coeff)
            for (int p0 = lane; p0 < ncx; p0 += 32 * U) {
                const bool tail = absorbs_tail(p0 - lane, ncx, U);
                // FULL: as in k3_coeff, no element is tested
                auto pass = [&](auto full_tag) {
                    constexpr bool FULL = decltype(full_tag)::value;
                    constexpr int NJ = FULL ? U : U + 1;
                    T z0[U + 1], z1[U + 1];
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {   // loads first
                        const int p = p0 + 32 * j;
                        if (!FULL && (p >= ncx || (j == U && !tail))) continue;
                        if (!rowc) z0[j] = zrow[2 * p];
                        if (FULL || p + 1 < ncx) z1[j] = zrow[(ZS && rowc) ? p : 2 * p + 1];
                    }
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int p = p0 + 32 * j;
                        if (!FULL && (p >= ncx || (j == U && !tail))) continue;
                        const T r0 = R[p];
                        T v0 = lerp_x(T(1), r0, T(0), r0);
                        if (!rowc) v0 += z0[j];   // z vanishes on coarse nodes of the coarse grid's rows
                        orow[2 * p] = v0;
                        if (FULL || p + 1 < ncx) orow[2 * p + 1] = lerp_x(T(0.5), r0, T(0.5), R[p + 1]) + z1[j];
                    }
                };
                if (!tail && p0 - lane + 32 * U < ncx) pass(std::true_type{});
                else pass(std::false_type{});
                if (tail) break;
            }
        } else
        for (int x0 = lane; x0 < nx; x0 += 32 * U) {
            const bool tail = absorbs_tail(x0 - lane, nx, U);
            T v[U + 1];
#pragma unroll
            for (int j = 0; j < U + 1; ++j) {
                const int x = x0 + 32 * j;
                v[j] = T(0);
                if (x >= nx || (j == U && !tail)) continue;
                // coarse x: coarse index J twice with weights (1, 0); new x: J, J+1
                const bool cx = is_coarse(x, nx);
                const int jl = cx ? coarse_index(x, nx, ncx) : (x - 1) >> 1;
                const int jr = cx ? jl : jl + 1;
                T wl = (x & 1) ? T(0.5) : T(1), wr = (x & 1) ? T(0.5) : T(0);
                if (x >= ireg) {
                    wl = wlx[x];
                    wr = wrx[x];
                }
                if (STAGE) v[j] = lerp_x(wl, R[jl], wr, R[jr]);
                else v[j] = lerp_x(wl, combine_rows(rows, rw, use, jl), wr, combine_rows(rows, rw, use, jr));
                // z vanishes on coarse nodes of the coarse grid's rows
                if (!(rowc && cx)) v[j] += zrow[(ZS && rowc) ? x - coarse_before(x) : x];
            }
#pragma unroll
            for (int j = 0; j < U + 1; ++j) {
                const int x = x0 + 32 * j;
                if (x < nx && (j < U || tail)) orow[x] = v[j];
            }
            if (tail) break;
        }
        if (STAGE) __syncwarp();   // R is rewritten by the warp's next row
    }
}

// -- restriction along x (first pass: z is zero on coarse nodes) -------------------
template <typename Tin, typename Tout, int U, bool ZS>
__global__ void __launch_bounds__(RT) k3_restrict_x(const Tin* __restrict__ in,
                                                    Tout* __restrict__ out, int nz, int ny,
                                                    int nx, int ncz, int ncy, int ncx,
                                                    AxisT<Tout> ax, int64_t zoff, int opitch) {
    const int lane = threadIdx.x & 31;
    const Tout* __restrict__ rw = ax.rw;
    const int rlo = ax.rlo, rhi = ax.rhi;
    Tout wi[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) wi[t] = ax.rwi[t];
    WARP_ROWS((int64_t)nz * ny, r) {
        const int z = (int)((uint32_t)r / (uint32_t)ny), y = (int)(r - (int64_t)z * ny);
        const bool rowc = is_coarse(z, nz) && is_coarse(y, ny);
        if (ZS) PREFETCH_NEXT_ZS_ROW(in, zoff, r, nz, ny, nx, ncz, ncy, ncx, sizeof(Tin));
        else PREFETCH_NEXT_ROW(in, r, (int64_t)nz * ny, nx, sizeof(Tin));
        const Tin* irow = ZS ? in + zs_row_base(zoff, r, nx, z, y, nz, ny, ncy, ncx) : in + r * nx;
        Tout* orow = out + r * opitch;
        // symbol order on a coarse row holds only the odd positions: ip -> (ip - 1) / 2
        const int sh = (ZS && rowc) ? 1 : 0;
        for (int J0 = lane; J0 < ncx; J0 += 32 * U) {
            const bool tail = absorbs_tail(J0 - lane, ncx, U);
            const int base = J0 - lane;
            if (!tail && base >= rlo && base + 32 * U <= rhi) {
                // every J of the pass takes the uniform window: no tests
                Tout acc[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int J = J0 + 32 * j;
                    if (sh) {   // coarse row in symbol order: only the odd taps
                        Tout a = wi[0] * Tout(0);
                        a += wi[1] * (Tout)irow[J - 1];
                        a += wi[2] * Tout(0);
                        a += wi[3] * (Tout)irow[J];
                        a += wi[4] * Tout(0);
                        acc[j] = a;
                    } else {
                        const Tout e0 = rowc ? Tout(0) : (Tout)irow[2 * J - 2];
                        const Tout e1 = (Tout)irow[2 * J - 1];
                        const Tout e2 = rowc ? Tout(0) : (Tout)irow[2 * J];
                        const Tout e3 = (Tout)irow[2 * J + 1];
                        const Tout e4 = rowc ? Tout(0) : (Tout)irow[2 * J + 2];
                        Tout a = wi[0] * e0;
                        a += wi[1] * e1;
                        a += wi[2] * e2;
                        a += wi[3] * e3;
                        a += wi[4] * e4;
                        acc[j] = a;
                    }
                }
#pragma unroll
                for (int j = 0; j < U; ++j) orow[J0 + 32 * j] = acc[j];
                continue;
            }
            Tout acc[U + 1];
#pragma unroll
            for (int j = 0; j < U + 1; ++j) {
                const int J = J0 + 32 * j;
                acc[j] = Tout(0);
                if (J >= ncx || (j == U && !tail)) continue;
                acc[j] = restrict_row_at<Tout>(J, nx, ncx, rowc, wi, rlo, rhi, rw, [&](int ip) {
                    return (Tout)irow[sh ? (ip - 1) >> 1 : ip];
                });
            }
#pragma unroll
            for (int j = 0; j < U + 1; ++j)
                if (J0 + 32 * j < ncx && (j < U || tail)) orow[J0 + 32 * j] = acc[j];
            if (tail) break;
        }
    }
}

// -- restriction along y or z: whole rows combined with per-row weights ----------
// in: (nouter, m, inner) rows of `nx` elements; out: (nouter, mc, inner).
template <typename Tin, typename Tout, int U>
__global__ void __launch_bounds__(RT) k3_restrict_rows(const Tin* __restrict__ in,
                                                       Tout* __restrict__ out, int nouter, int m,
                                                       int mc, int inner, int nx,
                                                       const Tout* __restrict__ rw, int pitch) {
    const int lane = threadIdx.x & 31;
    WARP_ROWS((int64_t)nouter * mc * inner, r) {
        const uint32_t ru = (uint32_t)r;
        const int i = (int)(ru % (uint32_t)inner);
        const uint32_t oj = ru / (uint32_t)inner;
        const int J = (int)(oj % (uint32_t)mc);
        const int o = (int)(oj / (uint32_t)mc);
        const int f = restrict_center(J, m, mc);
        // five taps in fixed slots; taps outside the axis get weight 0 and a valid row
        const Tin* src[5];
        Tout w[5];
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            int ip = f - 2 + t;
            const bool ok = ip >= 0 && ip < m;
            w[t] = ok ? rw[J * 5 + t] : Tout(0);
            ip = ok ? ip : f;
            src[t] = in + (((int64_t)o * m + ip) * inner + i) * pitch;
        }
        Tout* orow = out + r * pitch;
        for (int x0 = lane; x0 < nx; x0 += 32 * U) {
            Tout acc[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int x = x0 + 32 * j;
                acc[j] = Tout(0);
                if (x >= nx) continue;
#pragma unroll
                for (int k = 0; k < 5; ++k) acc[j] += w[k] * (Tout)src[k][x];
            }
#pragma unroll
            for (int j = 0; j < U; ++j)
                if (x0 + 32 * j < nx) orow[x0 + 32 * j] = acc[j];
        }
    }
}

// -- mass norm u^T M_l u (level energies of the s-norm) ----------------------------
// Per row (z, y): M u = Mx applied to the sum over the 3 x 3 neighbouring
// rows of Mz[z][z'] My[y][y'] row'.  The stencil runs in T; each lane sums
// its products over a row in T and adds that to a double accumulator, and
// blocks reduce in a fixed order, so the partial sums do not depend on
// timing.
template <typename T>
__device__ inline void mass_taps(const AxisT<T>& ax, int i, int m, T f[3], int p[3]) {
    if (!ax.mdiag) {   // inactive axis: identity
        f[0] = f[2] = T(0);
        f[1] = T(1);
        p[0] = p[1] = p[2] = i;
        return;
    }
    f[0] = i > 0 ? ax.mot[i - 1] : T(0);
    f[1] = ax.mdt[i];
    f[2] = i + 1 < m ? ax.mot[i] : T(0);
    p[0] = i > 0 ? i - 1 : i;
    p[1] = i;
    p[2] = i + 1 < m ? i + 1 : i;
}

// Work items: (z, a strip of MN_Y rows of y, a block of MN_X columns).
// A warp slides down its strip keeping t_y(x) = sum_a Mz[z][z_a] u[z_a][y][x]
// for rows y-1, y, y+1 in registers (three loads per row), combines them
// with the y taps, and takes the x taps from the adjacent lanes; lanes 0
// and 31 carry the columns either side of the block.
constexpr int MN_Y = 32;
constexpr int MN_X = 30;

template <typename T>
__global__ void __launch_bounds__(RT) k3_mass_norm(const T* __restrict__ u, Level<T> lv,
                                                   double* __restrict__ partial) {
    const int nz = (int)lv.n[1], ny = (int)lv.n[2], nx = (int)lv.n[3];
    const T* __restrict__ mdx = lv.ax[3].mdt;
    const T* __restrict__ mox = lv.ax[3].mot;
    const int lane = threadIdx.x & 31;
    const int nys = (ny + MN_Y - 1) / MN_Y, nxb = (nx + MN_X - 1) / MN_X;
    const int64_t items = (int64_t)nz * nys * nxb;
    double acc = 0.0;
    for (int64_t it = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5); it < items;
         it += (int64_t)gridDim.x * WPB) {
        const int xb = (int)(it % nxb);
        const int64_t rest = it / nxb;
        const int ys = (int)(rest % nys), z = (int)(rest / nys);
        const int x = xb * MN_X + lane - 1;
        const int xc = min(max(x, 0), nx - 1);   // halo columns outside the axis get weight 0
        T fz[3];
        int pz[3];
        mass_taps(lv.ax[1], z, nz, fz, pz);
        const T* z0 = u + (int64_t)pz[0] * ny * nx + xc;
        const T* z1 = u + (int64_t)pz[1] * ny * nx + xc;
        const T* z2 = u + (int64_t)pz[2] * ny * nx + xc;
        auto trow = [&](int y, T& centre) {
            const int64_t o = (int64_t)y * nx;
            const T a0 = z0[o], a1 = z1[o], a2 = z2[o];
            centre = a1;   // pz[1] = z: the row's own values
            return fz[0] * a0 + fz[1] * a1 + fz[2] * a2;
        };
        const int y0 = ys * MN_Y, y1 = min(ny, y0 + MN_Y);
        T cprev, ccur, cnext;
        T tprev = trow(y0 > 0 ? y0 - 1 : y0, cprev);
        T tcur = trow(y0, ccur);
        T racc = T(0);
        for (int y = y0; y < y1; ++y) {
            const T tnext = trow(y + 1 < ny ? y + 1 : y, cnext);
            T fy[3];
            int py[3];
            mass_taps(lv.ax[2], y, ny, fy, py);
            const T sv = fy[0] * tprev + fy[1] * tcur + fy[2] * tnext;   // zero weights at the ends
            const T sl = __shfl_up_sync(0xffffffffu, sv, 1);
            const T sr = __shfl_down_sync(0xffffffffu, sv, 1);
            if (lane >= 1 && lane <= MN_X && x < nx) {
                const T wl = x > 0 ? mox[x - 1] : T(0), wc = mdx[x], wr = x + 1 < nx ? mox[x] : T(0);
                racc += ccur * (wl * sl + wc * sv + wr * sr);
            }
            tprev = tcur;
            tcur = tnext;
            ccur = cnext;
        }
        (void)cprev;
        acc += (double)racc;
    }
    __shared__ double sh[RT];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// -- quantization ------------------------------------------------------------------
constexpr int HCOPIES = 2;

template <typename T>
__device__ inline void qvalue(T c, T inv_w, WidthSplit ws, double w, int& sym, int32_t& qo,
                              unsigned& st);

template <>
__device__ inline void qvalue<float>(float c, float inv_w, WidthSplit ws, double w, int& sym,
                                     int32_t& qo, unsigned& st) {
    const float q = rintf(__fmul_rn(c, inv_w));
    if (fabsf(q) < (float)RADIUS) {   // false for NaN and +-Inf
        sym = (int)q + RADIUS;
        return;
    }
    sym = MGARD_ESC;
    if (fabsf(q) < (float)F32_EXACT) {   // the float32 decision is exact enough here
        qo = (int32_t)q;
        return;
    }
    qo = 0;
    if (!isfinite(c)) {
        st |= ST_NONFINITE;
        return;
    }
    if (!quant_big(c, ws, w, qo)) {
        st |= ST_RANGE;
        qo = 0;
    }
}

template <>
__device__ inline void qvalue<double>(double c, double, WidthSplit, double w, int& sym,
                                      int32_t& qo, unsigned& st) {
    const double q = rint(c / w);
    if (fabs(q) < (double)RADIUS) {
        sym = (int)q + RADIUS;
        return;
    }
    sym = MGARD_ESC;
    qo = 0;
    if (!isfinite(c)) {
        st |= ST_NONFINITE;
        return;
    }
    if (fabs(q) > 2147483647.0) st |= ST_RANGE;
    else qo = (int32_t)q;
}

struct QRow {
    int nz, ny, nx;
    int ncz, ncy, ncx;
    int64_t tail_z, tail_y;       // ncy*ncx and ncx
    int64_t sym_off;
    int tables;                   // level >= 1
};

// Rank offset of a row: the number of coarse-grid nodes before its first
// node in row-major order, except those in the row itself; rowc reports that
// the row lies in the coarse grid's (z, y) prefix.
__device__ inline int64_t row_rank(const QRow& q, int z, int y, bool& rowc) {
    if (!q.tables) {
        rowc = false;
        return 0;
    }
    const bool zc = is_coarse(z, q.nz);
    int64_t cnt = (int64_t)coarse_before(z) * q.tail_z;
    if (zc) cnt += (int64_t)coarse_before(y) * q.tail_y;
    rowc = zc && is_coarse(y, q.ny);
    return cnt;
}

template <typename T, int U>
__global__ void __launch_bounds__(RT) k3_quantize(const T* __restrict__ c, QRow q,
                                                  const double* __restrict__ wp,
                                                  uint16_t* __restrict__ sym,
                                                  int32_t* __restrict__ esc,
                                                  unsigned long long* __restrict__ hist,
                                                  unsigned* status) {
    __shared__ unsigned sh[HCOPIES][DICT];
    for (int k = threadIdx.x; k < HCOPIES * DICT; k += RT) (&sh[0][0])[k] = 0;
    __syncthreads();
    const double w = *wp;
    const T inv_w = (T)(1.0 / w);
    const WidthSplit ws = split_width(w);
    unsigned* my = sh[threadIdx.x & (HCOPIES - 1)];
    unsigned center = 0;   // the most frequent symbol (q = 0) is counted in a register
    unsigned st = 0;
    const int lane = threadIdx.x & 31;
    WARP_ROWS((int64_t)q.nz * q.ny, r) {
        const int z = (int)((uint32_t)r / (uint32_t)q.ny), y = (int)(r - (int64_t)z * q.ny);
        bool rowc;
        const int64_t base = q.sym_off + r * q.nx - row_rank(q, z, y, rowc);
        PREFETCH_NEXT_ROW(c, r, (int64_t)q.nz * q.ny, q.nx, sizeof(T));
        const T* crow = c + r * q.nx;
        for (int x0 = lane; x0 < q.nx; x0 += 32 * U) {
            T v[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int x = x0 + 32 * j;
                v[j] = T(0);
                if (x < q.nx && !(rowc && is_coarse(x, q.nx))) v[j] = crow[x];
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int x = x0 + 32 * j;
                if (x >= q.nx) continue;
                int64_t p = base + x;
                if (rowc) {
                    if (is_coarse(x, q.nx)) continue;   // node of the coarser grid
                    p -= coarse_before(x);
                }
                int s;
                int32_t qo;
                qvalue<T>(v[j], inv_w, ws, w, s, qo, st);
                sym[p] = (uint16_t)s;
                if (s == MGARD_ESC) esc[p] = qo;
                if (s == RADIUS) ++center;
                else atomicAdd(&my[s], 1u);
            }
        }
    }
    if (center) atomicAdd(&sh[0][RADIUS], center);
    __syncthreads();
    for (int k = threadIdx.x; k < DICT; k += RT) {
        unsigned v = 0;
#pragma unroll
        for (int h = 0; h < HCOPIES; ++h) v += sh[h][k];
        if (v) atomicAdd(&hist[k], (unsigned long long)v);
    }
    if (st) atomicOr(status, st);
}

template <typename T, int U>
__global__ void __launch_bounds__(RT) k3_dequantize(const uint16_t* __restrict__ sym,
                                                    const int32_t* __restrict__ esc, QRow q,
                                                    T wt, double w, T* __restrict__ c) {
    const int lane = threadIdx.x & 31;
    const WidthSplit ws = split_width(w);
    WARP_ROWS((int64_t)q.nz * q.ny, r) {
        const int z = (int)((uint32_t)r / (uint32_t)q.ny), y = (int)(r - (int64_t)z * q.ny);
        bool rowc;
        const int64_t base = q.sym_off + r * q.nx - row_rank(q, z, y, rowc);
        T* crow = c + r * q.nx;
        for (int x0 = lane; x0 < q.nx; x0 += 32 * U) {
            int sv[U];
            int64_t pv[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int x = x0 + 32 * j;
                sv[j] = -1;
                if (x >= q.nx) continue;
                int64_t p = base + x;
                if (rowc) {
                    if (is_coarse(x, q.nx)) continue;   // z vanishes on the coarser grid
                    p -= coarse_before(x);
                }
                pv[j] = p;
                sv[j] = sym[p];
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int x = x0 + 32 * j;
                if (x >= q.nx) continue;
                const int s = sv[j];
                T v;
                if (s < 0) v = T(0);
                else if (s == MGARD_ESC) v = dequant_escape<T>(esc[pv[j]], wt, ws, w);
                else if (sizeof(T) == 4) v = (T)__fmul_rn((float)(s - RADIUS), (float)wt);
                else v = (T)((double)(s - RADIUS) * w);
                crow[x] = v;
            }
        }
    }
}

QRow make_qrow(const Plan& p, int l) {
    QRow q{};
    q.nz = (int)p.shape[l][1];
    q.ny = (int)p.shape[l][2];
    q.nx = (int)p.shape[l][3];
    q.tables = l > 0;
    q.sym_off = p.offset[l];
    if (l > 0) {
        q.ncz = (int)p.shape[l - 1][1];
        q.ncy = (int)p.shape[l - 1][2];
        q.ncx = (int)p.shape[l - 1][3];
        q.tail_z = (int64_t)q.ncy * q.ncx;
        q.tail_y = q.ncx;
    }
    return q;
}

// Shared memory of a staged coefficient or fill launch (one coarse x-row
// per warp), or 0 when the launch shape asks for per-element interpolation
// or the rows do not fit the default 48 KB.
template <typename T>
size_t stage_bytes(const Level<T>& lv, const RowCfg& c) {
    const size_t b = (size_t)WPB * (size_t)pad8<T>((int)lv.nc[3]) * sizeof(T);
    return c.stage != 0 && b <= 48 * 1024 ? b : 0;
}

// The pair paths of the coefficient and fill kernels: an odd extent along x
// (coarse nodes at the even x, the last one included) with the uniform
// interpolation weights everywhere.
template <typename T>
bool pair_ok(const Level<T>& lv) {
    return (lv.n[3] & 1) && lv.n[3] >= 3 && lv.ax[3].ireg >= lv.n[3];
}

}  // namespace

template <typename T>
mgard_status rows3_coeff(const Plan& p, int l, const T* in, T* out, T* coarse, cudaStream_t st,
                         int64_t zoff, void* rx, bool rx_f64, bool* fused) {
    const Level<T>& lv = p.level<T>(l);
    const RowCfg c = p.row_cfg(l, RK_COEFF);
    const int g = row_grid(lv.n[1] * lv.n[2], c.bpsm);
    const size_t sm = stage_bytes<T>(lv, c);
    // the fused x restriction keeps the row's coefficients beside the staged row
    const size_t smx = sm + (size_t)WPB * (size_t)pad8<T>((int)lv.n[3]) * sizeof(T);
    const bool fuse = rx && sm && smx <= 48 * 1024;
    const bool pair = sm && pair_ok(lv);
    if (fused) *fused = fuse;
    with_cfg(c, lv.n[3], false, [&](auto u) {
        constexpr int U = decltype(u)::value;
        const int64_t zo = zoff >= 0 ? zoff : 0;
        if (fuse) {
            auto go = [&](auto tw) {
                using Tw = decltype(tw);
                Tw* x = (Tw*)rx;
                const AxisT<Tw> ax = p.level<Tw>(l).ax[3];
                if (zoff >= 0 && pair)
                    MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, true, true, true, Tw, true><<<g, RT, smx, st>>>(in, out, coarse, lv, zo, x, ax, (int)rx_pitch<Tw>(lv.nc[3])));
                else if (zoff >= 0)
                    MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, true, true, true, Tw, false><<<g, RT, smx, st>>>(in, out, coarse, lv, zo, x, ax, (int)rx_pitch<Tw>(lv.nc[3])));
                else if (pair)
                    MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, false, true, true, Tw, true><<<g, RT, smx, st>>>(in, out, coarse, lv, zo, x, ax, (int)rx_pitch<Tw>(lv.nc[3])));
                else
                    MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, false, true, true, Tw, false><<<g, RT, smx, st>>>(in, out, coarse, lv, zo, x, ax, (int)rx_pitch<Tw>(lv.nc[3])));
            };
            if (rx_f64) go(double(0));
            else go(T(0));
            return;
        }
        const AxisT<T> none{};
        if (zoff >= 0 && pair)
            MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, true, true, false, T, true><<<g, RT, sm, st>>>(in, out, coarse, lv, zo, nullptr, none, 0));
        else if (zoff >= 0 && sm)
            MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, true, true, false, T, false><<<g, RT, sm, st>>>(in, out, coarse, lv, zo, nullptr, none, 0));
        else if (zoff >= 0)
            MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, true, false, false, T, false><<<g, RT, 0, st>>>(in, out, coarse, lv, zo, nullptr, none, 0));
        else if (pair)
            MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, false, true, false, T, true><<<g, RT, sm, st>>>(in, out, coarse, lv, 0, nullptr, none, 0));
        else if (sm)
            MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, false, true, false, T, false><<<g, RT, sm, st>>>(in, out, coarse, lv, 0, nullptr, none, 0));
        else
            MGB_LAUNCH("k3_coeff", st, k3_coeff<T, U, false, false, false, T, false><<<g, RT, 0, st>>>(in, out, coarse, lv, 0, nullptr, none, 0));
    });
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status rows3_fill(const Plan& p, int l, const T* z, const T* coarse, T* out,
                        cudaStream_t st, int64_t zoff) {
    const Level<T>& lv = p.level<T>(l);
    const RowCfg c = p.row_cfg(l, RK_FILL);
    const int g = row_grid(lv.n[1] * lv.n[2], c.bpsm);
    const size_t sm = stage_bytes<T>(lv, c);
    const bool pair = sm && pair_ok(lv);
    with_cfg(c, lv.n[3], false, [&](auto u) {
        constexpr int U = decltype(u)::value;
        if (zoff >= 0 && pair)
            MGB_LAUNCH("k3_fill", st, k3_fill<T, U, true, true, true><<<g, RT, sm, st>>>(z, coarse, out, lv, zoff));
        else if (zoff >= 0 && sm)
            MGB_LAUNCH("k3_fill", st, k3_fill<T, U, true, true, false><<<g, RT, sm, st>>>(z, coarse, out, lv, zoff));
        else if (zoff >= 0)
            MGB_LAUNCH("k3_fill", st, k3_fill<T, U, true, false, false><<<g, RT, 0, st>>>(z, coarse, out, lv, zoff));
        else if (pair)
            MGB_LAUNCH("k3_fill", st, k3_fill<T, U, false, true, true><<<g, RT, sm, st>>>(z, coarse, out, lv, 0));
        else if (sm)
            MGB_LAUNCH("k3_fill", st, k3_fill<T, U, false, true, false><<<g, RT, sm, st>>>(z, coarse, out, lv, 0));
        else
            MGB_LAUNCH("k3_fill", st, k3_fill<T, U, false, false, false><<<g, RT, 0, st>>>(z, coarse, out, lv, 0));
    });
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T, typename Tw>
mgard_status rows3_correct(const Plan& p, int l, const T* z, T* coarse, void* t0, void* t1,
                           T sign, cudaStream_t st, int64_t zoff, bool x_done, unsigned* status) {
    const Level<Tw>& lw = p.level<Tw>(l);
    const Level<T>& lt = p.level<T>(l);
    const int nz = (int)lt.n[1], ny = (int)lt.n[2], nx = (int)lt.n[3];
    const int ncz = (int)lt.nc[1], ncy = (int)lt.nc[2], ncx = (int)lt.nc[3];
    Tw* b0 = (Tw*)t0;
    Tw* b1 = (Tw*)t1;
    const int64_t P = rx_pitch<Tw>(ncx);   // row pitch of the intermediates
    // x (always active)
    const RowCfg cx = p.row_cfg(l, RK_RX), cr = p.row_cfg(l, RK_RROWS);
    const int gx = row_grid((int64_t)nz * ny, cx.bpsm);
    if (!x_done) with_cfg(cx, ncx, true, [&](auto u) {
        if (zoff >= 0)
            MGB_LAUNCH("k3_restrict_x", st, k3_restrict_x<T, Tw, decltype(u)::value, true><<<gx, RT, 0, st>>>(
                z, b0, nz, ny, nx, ncz, ncy, ncx, lw.ax[3], zoff, (int)P));
        else
            MGB_LAUNCH("k3_restrict_x", st, k3_restrict_x<T, Tw, decltype(u)::value, false><<<gx, RT, 0, st>>>(
                z, b0, nz, ny, nx, ncz, ncy, ncx, lw.ax[3], 0, (int)P));
    });
    MGB_CUDA(cudaGetLastError());
    Tw* cur = b0;
    Tw* nxt = b1;
    // y, then z: each axis restricted and, where its tiles fit, solved in the
    // same pass (the per-axis factors of the correction commute)
    bool y_solved = false, z_solved = false;
    if (lt.ax[2].fcls) {   // y: rows (z, Jy) of length ncx
        const AxisT<Tw>& a = lw.ax[2];
        MGB_TRY(restrict_solve_strided<Tw>(cur, nxt, nz, ny, ncy, P, a, st, &y_solved, status));
        if (!y_solved) {
            with_cfg(cr, ncx, true, [&](auto u) {
                MGB_LAUNCH("k3_restrict_rows", st, k3_restrict_rows<Tw, Tw, decltype(u)::value><<<row_grid((int64_t)nz * ncy, cr.bpsm), RT, 0, st>>>(
                    cur, nxt, nz, ny, ncy, 1, ncx, a.rw, (int)P));
            });
            MGB_CUDA(cudaGetLastError());
        }
        std::swap(cur, nxt);
    }
    if (lt.ax[1].fcls) {   // z: rows (Jz, y) of length ncx
        const AxisT<Tw>& a = lw.ax[1];
        MGB_TRY(restrict_solve_strided<Tw>(cur, nxt, 1, nz, ncz, (int64_t)ncy * P, a, st,
                                           &z_solved, status));
        if (!z_solved) {
            with_cfg(cr, ncx, true, [&](auto u) {
                MGB_LAUNCH("k3_restrict_rows", st, k3_restrict_rows<Tw, Tw, decltype(u)::value><<<row_grid((int64_t)ncz * ncy, cr.bpsm), RT, 0, st>>>(
                    cur, nxt, 1, nz, ncz, ncy, ncx, a.rw, (int)P));
            });
            MGB_CUDA(cudaGetLastError());
        }
        std::swap(cur, nxt);
    }
    // remaining solves: z, y (strided lines), then x (contiguous, fused correction add)
    if (lt.ax[1].fcls && !z_solved)
        MGB_TRY((solve_strided<Tw, T>(cur, 1, ncz, (int64_t)ncy * P, lw.ax[1].tsub, lw.ax[1].tinv,
                                      lw.ax[1].tcp, (T*)nullptr, (Tw)sign, st)));
    if (lt.ax[2].fcls && !y_solved)
        MGB_TRY((solve_strided<Tw, T>(cur, ncz, ncy, P, lw.ax[2].tsub, lw.ax[2].tinv,
                                      lw.ax[2].tcp, (T*)nullptr, (Tw)sign, st)));
    MGB_TRY((solve_contiguous<Tw, T>(cur, (int64_t)ncz * ncy, ncx, lw.ax[3].tsub, lw.ax[3].tinv,
                                     lw.ax[3].tcp, coarse, (Tw)sign, st, P)));
    return MGARD_OK;
}

int rows3_mass_norm_blocks(const Plan& p, int l) {
    return row_grid(p.shape[l][1] * p.shape[l][2]);
}

template <typename T>
mgard_status rows3_mass_norm(const Plan& p, int l, const T* u, double* partial, cudaStream_t st) {
    const Level<T>& lv = p.level<T>(l);
    MGB_LAUNCH("k3_mass_norm", st, k3_mass_norm<T><<<rows3_mass_norm_blocks(p, l), RT, 0, st>>>(u, lv, partial));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status rows3_quantize(const Plan& p, int l, const T* c, const double* w, uint16_t* sym,
                            int32_t* esc, unsigned long long* hist, unsigned* status,
                            cudaStream_t st) {
    const QRow q = make_qrow(p, l);
    const RowCfg cfg = p.row_cfg(l, RK_QUANT);
    with_cfg(cfg, q.nx, true, [&](auto u) {
        MGB_LAUNCH("k3_quantize", st, k3_quantize<T, decltype(u)::value><<<row_grid((int64_t)q.nz * q.ny, cfg.bpsm), RT, 0, st>>>(
            c, q, w, sym, esc, hist, status));
    });
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status rows3_dequantize(const Plan& p, int l, const uint16_t* sym, const int32_t* esc,
                              double w, T* c, cudaStream_t st) {
    const QRow q = make_qrow(p, l);
    const RowCfg cfg = p.row_cfg(l, RK_DEQUANT);
    with_cfg(cfg, q.nx, true, [&](auto u) {
        MGB_LAUNCH("k3_dequantize", st, k3_dequantize<T, decltype(u)::value><<<row_grid((int64_t)q.nz * q.ny, cfg.bpsm), RT, 0, st>>>(
            sym, esc, q, (T)w, w, c));
    });
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

#define INST(T)                                                                                  \
    template mgard_status rows3_coeff<T>(const Plan&, int, const T*, T*, T*, cudaStream_t,      \
                                         int64_t, void*, bool, bool*);                          \
    template mgard_status rows3_fill<T>(const Plan&, int, const T*, const T*, T*, cudaStream_t,  \
                                        int64_t);                                               \
    template mgard_status rows3_mass_norm<T>(const Plan&, int, const T*, double*, cudaStream_t); \
    template mgard_status rows3_quantize<T>(const Plan&, int, const T*, const double*, uint16_t*,       \
                                            int32_t*, unsigned long long*, unsigned*,            \
                                            cudaStream_t);                                       \
    template mgard_status rows3_dequantize<T>(const Plan&, int, const uint16_t*, const int32_t*, \
                                              double, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST
template mgard_status rows3_correct<float, float>(const Plan&, int, const float*, float*, void*,
                                                  void*, float, cudaStream_t, int64_t, bool,
                                                  unsigned*);
template mgard_status rows3_correct<float, double>(const Plan&, int, const float*, float*, void*,
                                                  void*, float, cudaStream_t, int64_t, bool,
                                                  unsigned*);
template mgard_status rows3_correct<double, double>(const Plan&, int, const double*, double*,
                                                    void*, void*, double, cudaStream_t, int64_t,
                                                    bool, unsigned*);

}  // namespace mgb
