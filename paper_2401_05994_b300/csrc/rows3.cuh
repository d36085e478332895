// Row kernels for grids of up to three active axes (the 4D view has
// n[0] == 1): axis 1 = z, axis 2 = y, axis 3 = x (contiguous).  A block
// walks whole x-rows; everything that depends only on (z, y) -- coarse or
// new, interpolation sources and weights, rank offsets -- is computed once
// per row, so the per-element work is a few loads and FMAs with 32-bit
// offsets inside the row.
#pragma once

#include "plan.cuh"

namespace mgb {

// True when the row kernels apply: at most three active axes and fewer than
// 2^31 nodes (row and symbol arithmetic inside a row uses 32 bits).
inline bool rows3_ok(const Plan& p) {
    return p.n4[0] == 1 && p.total() < (int64_t(1) << 31);
}

// With zoff >= 0 the level's coefficients are read from (coeff: written
// to) an array in symbol order, starting at symbol offset zoff: the nodes new
// on the level in row-major order (see zs_row_base); otherwise they sit in
// the level's own row-major array.
// With rx set, the kernel may also restrict the coefficients along x into
// rx (the first step of rows3_correct, in double when rx_f64, else in T);
// *fused reports whether it did (the launch shape needs staged rows that fit).
template <typename T>
mgard_status rows3_coeff(const Plan& p, int l, const T* in, T* out, T* coarse, cudaStream_t st,
                         int64_t zoff = -1, void* rx = nullptr, bool rx_f64 = false,
                         bool* fused = nullptr);
template <typename T>
mgard_status rows3_fill(const Plan& p, int l, const T* z, const T* coarse, T* out,
                        cudaStream_t st, int64_t zoff = -1);
// coarse += sign * M_{l-1}^{-1} P^T M_l z (restriction x, y, z; solves z, y, x)
// x_done: t0 already holds the restriction along x (from rows3_coeff).
template <typename T, typename Tw>
mgard_status rows3_correct(const Plan& p, int l, const T* z, T* coarse, void* t0, void* t1,
                           T sign, cudaStream_t st, int64_t zoff = -1, bool x_done = false,
                           unsigned* status = nullptr);
template <typename T>
mgard_status rows3_quantize(const Plan& p, int l, const T* c, const double* w, uint16_t* sym,
                            int32_t* esc, unsigned long long* hist, unsigned* status,
                            cudaStream_t st);
template <typename T>
mgard_status rows3_dequantize(const Plan& p, int l, const uint16_t* sym, const int32_t* esc,
                              double w, T* c, cudaStream_t st);

// Partial sums (rows3_mass_norm_blocks of them) of u^T M_l u.
int rows3_mass_norm_blocks(const Plan& p, int l);
template <typename T>
mgard_status rows3_mass_norm(const Plan& p, int l, const T* u, double* partial, cudaStream_t st);

// Row pitch (elements of Tw) of the restriction intermediates of the row
// kernels: rows of ncx values padded to a 16-byte multiple, so the strided
// passes can stage tiles with tensor copies.  Lines longer than the
// contiguous warp solver takes (1056 float, 544 double nodes) keep ncx:
// their solves run one thread per line on dense lines.
template <typename Tw>
inline int64_t rx_pitch(int64_t ncx) {
    const int64_t q = 16 / (int64_t)sizeof(Tw);
    const int64_t warp_max = sizeof(Tw) == 4 ? 1056 : 544;
    return ncx > warp_max ? ncx : (ncx + q - 1) / q * q;
}

// Solvers shared with the generic path (multilevel.cu).
template <typename Tw, typename Tdst>
mgard_status solve_strided(Tw* x, int64_t outer, int64_t m, int64_t stride, const Tw* sub,
                           const Tw* inv, const Tw* cp, Tdst* dst, Tw sign, cudaStream_t st);
template <typename Tw, typename Tdst>
mgard_status solve_contiguous(Tw* x, int64_t lines, int64_t m, const Tw* sub, const Tw* inv,
                              const Tw* cp, Tdst* dst, Tw sign, cudaStream_t st,
                              int64_t pitch = 0);
// Restriction along a strided axis (in: (outer, m, inner) -> out: (outer,
// mc, inner), the axis' weights rw[J*5 + t] on fine rows f(J)-2 .. f(J)+2,
// uniform rwi inside [rlo, rhi)) followed by the tridiagonal solve along it
// (the axis' Thomas factors), in one pass over shared-memory tiles, staged
// by tensor copies when the rows are 16-byte aligned (ST_TIMEOUT into
// *status if a copy never lands).  *done is false (and nothing runs) when a
// tile would not fit.
template <typename Tw>
mgard_status restrict_solve_strided(const Tw* in, Tw* out, int64_t outer, int64_t m, int64_t mc,
                                    int64_t inner, const AxisT<Tw>& ax, cudaStream_t st,
                                    bool* done, unsigned* status = nullptr);

}  // namespace mgb
