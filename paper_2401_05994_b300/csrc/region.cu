// Region-adaptive L-infinity bounds (paper: "Application impact", Earth and
// cosmological science: tighter errors kept in chosen regions).
//
// The error that level-l coefficient errors cause at a point p is reached
// through the corners of p's level-l cell, the corners of their
// level-(l-1) cells and the correction operator C_l = M_{l-1}^{-1} P^T M_l,
// whose rows decay geometrically away from their coarse node.  Splitting
// every row into the entries within rho level-l nodes of its coarse node
// and a far-field tail bounds the error at p by the widths of the nodes
// within a level-dependent distance of p plus the background width times
// T_l(rho) = sum_d t_{l,d}(rho) prod_{e != d} S_{l,e} (S the axis row-sum
// norms, t the far-field row sums; the plan tabulates both).  A box with
// tolerance tau_r therefore gets the width w_bg 2^-k_r on every node within
// its level's dilation (m_0 = H_0, m_l = (rho + 1) H_l + H_{l-1}, H the
// largest node spacing of a level), with
//   rho: the smallest radius with tau sum_l T_l(rho) / den <= min tau_r / 8,
//   k_r: the smallest k with 2^-k tau <= tau_r - tau sum_l T_l(rho) / den,
// den = 1 + sum_l c_l as for the uniform L-infinity width (c_l bounds the
// row sums of a level's whole error operator, so it also bounds the part
// of a row inside the dilation).
#include <algorithm>
#include <cmath>

#include "region.cuh"

namespace mgb {

namespace {

constexpr int K_MAX = 60;

// Box of region r in the plan's 4D view (squeezed axes right-aligned).
mgard_status view_box(const Plan& p, int ndim, const int64_t* shape, const mgard_region& r,
                      int64_t lo[4], int64_t hi[4]) {
    for (int a = 0; a < 4; ++a) lo[a] = hi[a] = 0;
    int a = 4 - p.D;
    for (int d = 0; d < ndim; ++d) {
        if (r.lo[d] < 0 || r.hi[d] < r.lo[d] || r.hi[d] >= shape[d]) {
            set_error("region box outside the field or empty");
            return MGARD_EINVAL;
        }
        if (shape[d] == 1) continue;
        lo[a] = r.lo[d];
        hi[a] = r.hi[d];
        ++a;
    }
    return MGARD_OK;
}

}  // namespace

mgard_status region_params(const Plan& p, int ndim, const int64_t* shape, double tol,
                           const mgard_region* rg, int n, int* rho, int32_t* k) {
    if (n < 0 || n > REGION_MAX || (n && !rg) || !(tol > 0.0) || !std::isfinite(tol)) {
        set_error("regions: 0..8 boxes and a positive finite tolerance");
        return MGARD_EINVAL;
    }
    if (p.L < 1) {
        set_error("regions need at least one level");
        return MGARD_ESHAPE;
    }
    double tmin = tol;
    for (int r = 0; r < n; ++r) {
        int64_t lo[4], hi[4];
        MGB_TRY(view_box(p, ndim, shape, rg[r], lo, hi));
        if (!(rg[r].tol > 0.0) || !(rg[r].tol <= tol)) {
            set_error("a region's tolerance must lie in (0, tol]");
            return MGARD_EINVAL;
        }
        tmin = std::min(tmin, rg[r].tol);
    }
    double den = 1.0;   // the uniform L-infinity constant 1 + sum_l c_l
    for (int l = 1; l <= p.L; ++l) den += p.linf_c[l];
    constexpr int R1 = Plan::RHO_MAX + 1;
    auto tail_sum = [&](int c) {
        double total = 0.0;
        for (int l = 1; l <= p.L; ++l) {
            double T = 0.0;
            for (int a = 4 - p.D; a < 4; ++a) {
                double other = 1.0;
                for (int b = 4 - p.D; b < 4; ++b)
                    if (b != a) other *= p.Kax[l][b];
                T += p.tails[l][a * R1 + c] * other;
            }
            total += T;
        }
        return total;
    };
    int best = -1;
    for (int c = 0; c < R1; ++c)
        if (tol * tail_sum(c) / den <= tmin / 8.0) {
            best = c;
            break;
        }
    if (best < 0) {
        set_error("region tolerances too small against the background tolerance");
        return MGARD_EINVAL;
    }
    const double far = tol * tail_sum(best) / den;
    for (int r = 0; r < n; ++r) {
        int e = 0;
        while (std::ldexp(tol, -e) > rg[r].tol - far) {
            if (++e > K_MAX) {
                set_error("region tolerance too small against the background tolerance");
                return MGARD_EINVAL;
            }
        }
        k[r] = e;
    }
    *rho = best;
    return MGARD_OK;
}

mgard_status region_table(const Plan& p, int ndim, const int64_t* shape, int rho, const int32_t* k,
                          const mgard_region* rg, int n, RegionScale* out) {
    if (n < 0 || n > REGION_MAX || rho < 0 || rho > Plan::RHO_MAX || p.L < 1) {
        set_error("region table: bad count, radius or levels");
        return MGARD_EINVAL;
    }
    out->lv.assign(p.L + 1, RegionLevel{});
    for (int r = 0; r < n; ++r) {
        if (k[r] < 0 || k[r] > K_MAX) {
            set_error("region table: width exponent out of range");
            return MGARD_EINVAL;
        }
        int64_t lo[4], hi[4];
        MGB_TRY(view_box(p, ndim, shape, rg[r], lo, hi));
        for (int l = 0; l <= p.L; ++l) {
            RegionLevel& L = out->lv[l];
            L.k[L.n] = k[r];
            for (int a = 0; a < 4; ++a) {
                const int64_t m = l == 0 ? p.hmax[0][a]
                                         : (int64_t)(rho + 1) * p.hmax[l][a] + p.hmax[l - 1][a];
                L.lo[L.n][a] = lo[a] - m;
                L.hi[L.n][a] = hi[a] + m;
            }
            ++L.n;
        }
    }
    return MGARD_OK;
}

}  // namespace mgb

using namespace mgb;

extern "C" mgard_status mgard_region_plan(int ndim, const int64_t* shape, double tol,
                                          const mgard_region* regions, int nregions, int* rho,
                                          int32_t* k) {
    if (!rho || (nregions && !k)) {
        set_error("region_plan: null output");
        return MGARD_EINVAL;
    }
    const Plan* p = nullptr;
    MGB_TRY(get_plan(ndim, shape, -1, &p, false));
    return region_params(*p, ndim, shape, tol, regions, nregions, rho, k);
}

extern "C" mgard_status mgard_region_exponents(int ndim, const int64_t* shape, double tol,
                                               const mgard_region* regions, int nregions,
                                               uint8_t* k, void* stream) {
    if (!k) {
        set_error("region_exponents: null output");
        return MGARD_EINVAL;
    }
    const Plan* p = nullptr;
    MGB_TRY(get_plan(ndim, shape, -1, &p));
    int rho = 0;
    int32_t kr[REGION_MAX] = {};
    MGB_TRY(region_params(*p, ndim, shape, tol, regions, nregions, &rho, kr));
    RegionScale rs;
    MGB_TRY(region_table(*p, ndim, shape, rho, kr, regions, nregions, &rs));
    cudaStream_t st = (cudaStream_t)stream;
    MGB_TRY(region_exponents(*p, rs, k, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    return MGARD_OK;
}
