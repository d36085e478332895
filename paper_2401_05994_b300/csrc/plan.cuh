// Per-shape tables ("plan"): the node hierarchy, interpolation, restriction
// and tridiagonal factors of every level, and the constants of the error
// estimators.  Built once per (shape, levels) on the host in FP64 and kept
// in device memory.
#pragma once

#include <array>
#include <memory>
#include <vector>

#include "common.cuh"

namespace mgb {

// Launch shape of a row kernel: elements per lane per batch (2, 4 or 8) and
// resident blocks per SM the grid is sized for; 0 = the built-in choice.
enum RowKind { RK_COEFF = 0, RK_FILL, RK_RX, RK_RROWS, RK_QUANT, RK_DEQUANT, RK_COUNT };
struct RowCfg {
    int u = 0;
    int bpsm = 0;
    int stage = -1;   // coefficient and fill kernels: 0 interpolate per element, 1 stage in
                      // shared memory, -1 the built-in choice (stage where the rows fit)
};

struct Plan {
    int D = 0;                       // active axes
    int L = 0;                       // levels above level 0
    int64_t n4[4] = {1, 1, 1, 1};    // squeezed shape in the 4D view
    std::vector<std::array<int64_t, 4>> shape;   // [l] level-l shape, l = 0..L
    std::vector<int64_t> offset;     // [l] symbol offset of level l
    std::vector<int64_t> count;      // [l] symbols of level l (new nodes)
    std::vector<double> K;           // [l] correction norm (l >= 1)
    // region-adaptive bounds: per level and axis of the 4D view, the row-sum
    // norm of the 1D correction operator (their product is K[l]; 1 on
    // inactive axes), its far-field row sums tails[l][a * (RHO_MAX + 1) + rho]
    // (entries more than rho level-l nodes from the row's coarse node), and
    // the largest spacing of the level-l nodes in input-grid units
    static constexpr int RHO_MAX = 48;
    // the L-infinity width: per level and axis, the row classes of B = P C
    // (rows[l][a][0] at coarse nodes, [1] at new nodes), and c_l, the bound
    // of the largest row sum of I_new - P C_l they give (l >= 1); the width
    // is 2 tau / (1 + sum_l c_l)
    struct RowClass {
        double tmax, tcmin, bmin, bmax, absbmin;
    };
    std::vector<std::array<std::array<RowClass, 2>, 4>> rows;
    std::vector<double> linf_c;
    std::vector<std::array<double, 4>> Kax;
    std::vector<std::vector<double>> tails;
    std::vector<std::array<int64_t, 4>> hmax;
    std::vector<double> mu;          // [l] Gershgorin bound of the level mass matrix
    std::vector<Level<float>> lf;    // [l] tables of level l (transition l -> l-1 for l >= 1)
    std::vector<Level<double>> ld;
    std::vector<LevelIndex> lidx;    // [l] finest positions of level-l nodes
    void* dbuf = nullptr;
    // launch shapes chosen by the autotuner, per level and row kernel (set by
    // autotune_plan; every choice gives bit-identical results)
    mutable std::vector<std::array<RowCfg, RK_COUNT>> tune;
    RowCfg row_cfg(int l, int kind) const {
        return l >= 0 && l < (int)tune.size() ? tune[l][kind] : RowCfg();
    }
    int64_t total() const { return n4[0] * n4[1] * n4[2] * n4[3]; }
    int64_t level_size(int l) const { return shape[l][0] * shape[l][1] * shape[l][2] * shape[l][3]; }
    template <typename T> const Level<T>& level(int l) const;
    ~Plan();
};

template <> inline const Level<float>& Plan::level<float>(int l) const { return lf[l]; }
template <> inline const Level<double>& Plan::level<double>(int l) const { return ld[l]; }

// Validate a shape and compute the squeezed 4D view; MGARD_ESHAPE on error.
mgard_status squeeze_shape(int ndim, const int64_t* shape, int64_t n4[4], int* D);
// Number of levels for a squeezed shape.
int level_count(const int64_t n4[4], int D, int max_levels);
// Cached plan (built on first use; device tables on the current device).
// With device = false only the host-side members (shapes, offsets, K, mu)
// are filled and nothing touches the GPU.
mgard_status get_plan(int ndim, const int64_t* shape, int max_levels, const Plan** out,
                      bool device = true);
// Bin widths (host) from a plan: w[l] = 2 tol_abs / den[l] * WIDTH_MARGIN,
// with den[l] from width_denominators (the same expression is evaluated on
// the device when tol_abs is only known there).
constexpr double WIDTH_MARGIN = 1.0 - 1.0 / 256.0;
void width_denominators(const Plan& p, double s, double* den);
void bin_widths(const Plan& p, double tol_abs, double s, double* w);
void release_plans();

}  // namespace mgb
