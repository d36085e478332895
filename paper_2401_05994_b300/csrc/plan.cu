// Host construction of the per-shape tables (see plan.cuh).
//
// Hierarchy (paper, "Software design": decomposition over a multigrid
// hierarchy; the coarsening rule for non-dyadic extents is this build's):
// along an axis the coarser level keeps the even positions plus the last
// one; coordinates are finest-grid indices.  Operators are the standard P1
// ones on those coordinates: interpolation weights from the coordinates,
// mass matrix M_ii = (h_{i-1}+h_i)/3, M_{i,i+1} = h_i/6, restriction
// R = P^T M, and the Thomas factorization of the coarse mass matrix.
#include <algorithm>
#include <cmath>
#include <limits>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "plan.cuh"

namespace mgb {

namespace {

std::vector<int64_t> coarse_positions(int64_t m) {
    std::vector<int64_t> p;
    for (int64_t i = 0; i < m; i += 2) p.push_back(i);
    if (p.back() != m - 1) p.push_back(m - 1);
    return p;
}

int axis_levels(int64_t n) {
    int c = 0;
    int64_t m = n;
    while (m > 2) {
        m = m / 2 + 1;
        ++c;
    }
    return c;
}

struct Blob {
    std::vector<char> bytes;
    template <typename T>
    size_t add(const std::vector<T>& v) {
        size_t off = (bytes.size() + 255) & ~size_t(255);
        bytes.resize(off + v.size() * sizeof(T) + 16);
        if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

// Thomas factors of the tridiagonal mass matrix on coordinates xc.
void thomas(const std::vector<double>& xc, std::vector<double>& sub, std::vector<double>& inv,
            std::vector<double>& cp) {
    size_t mc = xc.size();
    sub.assign(mc, 0.0);
    inv.assign(mc, 0.0);
    cp.assign(mc, 0.0);
    double prev_cp = 0.0;
    for (size_t J = 0; J < mc; ++J) {
        double hl = J > 0 ? xc[J] - xc[J - 1] : 0.0;
        double hr = J + 1 < mc ? xc[J + 1] - xc[J] : 0.0;
        double a = hl / 6.0, b = (hl + hr) / 3.0, c = hr / 6.0;
        double den = b - a * prev_cp;
        sub[J] = a;
        inv[J] = 1.0 / den;
        cp[J] = c * inv[J];
        prev_cp = cp[J];
    }
}

// Solve M_c g = e_J restricted to the index window [lo, hi] (exact when the
// window is the whole axis; otherwise the truncation error decays
// geometrically with the distance to the window edge).
void unit_solve(const std::vector<double>& xc, int64_t J, int64_t lo, int64_t hi,
                std::vector<double>& g) {
    int64_t n = hi - lo + 1;
    std::vector<double> c(n), d(n);
    double pc = 0.0, pd = 0.0;
    const int64_t mc = (int64_t)xc.size();
    for (int64_t k = 0; k < n; ++k) {
        int64_t K = lo + k;
        double hl = K > 0 ? xc[K] - xc[K - 1] : 0.0;
        double hr = K + 1 < mc ? xc[K + 1] - xc[K] : 0.0;
        double a = (K > lo) ? hl / 6.0 : 0.0;
        double b = (hl + hr) / 3.0;
        double cc = (K < hi) ? hr / 6.0 : 0.0;
        double den = b - a * pc;
        c[k] = cc / den;
        d[k] = ((K == J ? 1.0 : 0.0) - a * pd) / den;
        pc = c[k];
        pd = d[k];
    }
    g.assign(n, 0.0);
    g[n - 1] = d[n - 1];
    for (int64_t k = n - 2; k >= 0; --k) g[k] = d[k] - c[k] * g[k + 1];
}

// ||M_c^{-1} R||_inf for one axis of one level transition.  Every row is
// evaluated exactly for axes of up to 2048 coarse nodes; longer axes
// evaluate the rows near both ends and one interior row (interior rows of a
// uniform spacing are identical) with a +-300 window.
// With `tail` (RHO_MAX + 1 entries) also the largest row sum of the entries
// more than rho level-l nodes from the row's coarse node, for every rho.
double correction_norm(const std::vector<double>& xc, const std::vector<int64_t>& rf,
                       const std::vector<double>& rw, int64_t m, double* tail = nullptr) {
    int64_t mc = (int64_t)xc.size();
    std::vector<int64_t> rows;
    const int64_t W = 300;
    bool full = mc <= 2048;
    if (full) {
        for (int64_t J = 0; J < mc; ++J) rows.push_back(J);
    } else {
        for (int64_t J = 0; J < 2 * W; ++J) rows.push_back(J);
        rows.push_back(mc / 2);
        for (int64_t J = mc - 2 * W; J < mc; ++J) rows.push_back(J);
    }
    double best = 0.0;
    std::vector<double> g, row;
    for (int64_t J : rows) {
        int64_t lo = full ? 0 : std::max<int64_t>(0, J - W);
        int64_t hi = full ? mc - 1 : std::min<int64_t>(mc - 1, J + W);
        unit_solve(xc, J, lo, hi, g);
        int64_t flo = std::max<int64_t>(0, rf[lo] - 2), fhi = std::min<int64_t>(m - 1, rf[hi] + 2);
        row.assign(fhi - flo + 1, 0.0);
        for (int64_t K = lo; K <= hi; ++K)
            for (int t = 0; t < 5; ++t) {
                int64_t i = rf[K] - 2 + t;
                if (i < flo || i > fhi) continue;
                row[i - flo] += g[K - lo] * rw[K * 5 + t];
            }
        double sum = 0.0;
        for (double v : row) sum += std::fabs(v);
        best = std::max(best, sum);
        if (tail) {
            double by[Plan::RHO_MAX + 2] = {};
            for (int64_t i = flo; i <= fhi; ++i) {
                const int64_t d = std::min<int64_t>(std::llabs(i - rf[J]), Plan::RHO_MAX + 1);
                by[d] += std::fabs(row[i - flo]);
            }
            double far = 0.0;   // entries farther than rho
            for (int rho = Plan::RHO_MAX; rho >= 0; --rho) {
                far += by[rho + 1];
                tail[rho] = std::max(tail[rho], far);
            }
        }
    }
    return best;
}

// Row classes of B = P C on one axis of a level transition (C the axis
// correction operator M_c^{-1} P^T M, rows of the level-l grid): for the
// rows at coarse nodes (k = 0) and at new nodes (k = 1) the largest row sum
// T = sum_i |B(q, i)|, the smallest sum Tc over the coarse columns, and the
// range of the diagonal b = B(q, q) and of |b|.  Rows of C come from unit
// solves as in correction_norm (whole axis up to 2048 coarse nodes, a +-300
// window beyond); a new row combines its two coarse neighbours' rows with
// the interpolation weights.
void axis_row_classes(const std::vector<double>& xc, const std::vector<int64_t>& rf,
                      const std::vector<double>& rw, int64_t m, const std::vector<int>& fcls,
                      const std::vector<double>& wl, const std::vector<double>& wr,
                      Plan::RowClass cls[2]) {
    const int64_t mc = (int64_t)xc.size();
    const int64_t W = 300;
    const bool full = mc <= 2048;
    for (int k = 0; k < 2; ++k) {
        cls[k].tmax = 0.0;
        cls[k].tcmin = std::numeric_limits<double>::infinity();
        cls[k].bmin = std::numeric_limits<double>::infinity();
        cls[k].bmax = -std::numeric_limits<double>::infinity();
        cls[k].absbmin = std::numeric_limits<double>::infinity();
    }
    // row J of C over the fine index range [lo, hi]
    struct Row {
        int64_t lo = 0, hi = -1;
        std::vector<double> v;
        double at(int64_t i) const { return i >= lo && i <= hi ? v[i - lo] : 0.0; }
    };
    auto make_row = [&](int64_t J, Row& r) {
        const int64_t lo = full ? 0 : std::max<int64_t>(0, J - W);
        const int64_t hi = full ? mc - 1 : std::min<int64_t>(mc - 1, J + W);
        std::vector<double> g;
        unit_solve(xc, J, lo, hi, g);
        r.lo = std::max<int64_t>(0, rf[lo] - 2);
        r.hi = std::min<int64_t>(m - 1, rf[hi] + 2);
        r.v.assign(r.hi - r.lo + 1, 0.0);
        for (int64_t K = lo; K <= hi; ++K)
            for (int t = 0; t < 5; ++t) {
                const int64_t i = rf[K] - 2 + t;
                if (i < r.lo || i > r.hi) continue;
                r.v[i - r.lo] += g[K - lo] * rw[K * 5 + t];
            }
    };
    auto account = [&](int k, int64_t q, double a, double b_, const Row& r0, const Row* r1) {
        // B(q, :) = a r0 + b_ r1
        const int64_t lo = r1 ? std::min(r0.lo, r1->lo) : r0.lo;
        const int64_t hi = r1 ? std::max(r0.hi, r1->hi) : r0.hi;
        double T = 0.0, Tc = 0.0;
        for (int64_t i = lo; i <= hi; ++i) {
            const double v = std::fabs(a * r0.at(i) + (r1 ? b_ * r1->at(i) : 0.0));
            T += v;
            if (fcls[i] >= 0) Tc += v;
        }
        const double d = a * r0.at(q) + (r1 ? b_ * r1->at(q) : 0.0);
        Plan::RowClass& c = cls[k];
        c.tmax = std::max(c.tmax, T);
        c.tcmin = std::min(c.tcmin, Tc);
        c.bmin = std::min(c.bmin, d);
        c.bmax = std::max(c.bmax, d);
        c.absbmin = std::min(c.absbmin, std::fabs(d));
    };
    Row prev, cur;
    for (int64_t J = 0; J < mc; ++J) {
        make_row(J, cur);
        account(0, rf[J], 1.0, 0.0, cur, nullptr);
        if (J > 0)   // the new nodes between coarse J-1 and J
            for (int64_t q = rf[J - 1] + 1; q < rf[J]; ++q) account(1, q, wl[q], wr[q], prev, &cur);
        std::swap(prev, cur);
    }
}

// c_l of the L-infinity width: an upper bound of the largest row sum
// max_q sum_{i new} |A(q, i)| of A = I_new - P C on the level-l grid.  For a
// row q with per-axis values T, Tc, b the sum is
// prod T - prod Tc + [q new] (|1 - prod b| - prod |b|); over each of the
// 2^D classes of rows (which axes are coarse) the axis extremes bound it.
double linf_level_constant(const Plan& p, int l) {
    const int D = p.D;
    double best = 0.0;
    for (int mask = 0; mask < (1 << D); ++mask) {   // bit set: new on that axis
        double tmax = 1.0, tcmin = 1.0, lo = 1.0, hi = 1.0, absb = 1.0;
        for (int k = 0; k < D; ++k) {
            const Plan::RowClass& c = p.rows[l][4 - D + k][(mask >> k) & 1];
            tmax *= c.tmax;
            tcmin *= c.tcmin;
            const double cand[4] = {lo * c.bmin, lo * c.bmax, hi * c.bmin, hi * c.bmax};
            lo = std::min(std::min(cand[0], cand[1]), std::min(cand[2], cand[3]));
            hi = std::max(std::max(cand[0], cand[1]), std::max(cand[2], cand[3]));
            absb *= c.absbmin;
        }
        double v = tmax - tcmin;
        if (mask) v += std::max(std::fabs(1.0 - lo), std::fabs(1.0 - hi)) - absb;
        best = std::max(best, v);
    }
    return best;
}

template <typename T>
std::vector<T> cast(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

std::mutex g_mutex;
std::map<std::tuple<int, int, int64_t, int64_t, int64_t, int64_t>, std::unique_ptr<Plan>> g_plans;

}  // namespace

Plan::~Plan() {
    if (dbuf) cudaFree(dbuf);
}

mgard_status squeeze_shape(int ndim, const int64_t* shape, int64_t n4[4], int* D) {
    if (ndim < 1 || ndim > 4 || !shape) {
        set_error("ndim must be 1..4");
        return MGARD_ESHAPE;
    }
    int64_t sq[4];
    int k = 0;
    for (int i = 0; i < ndim; ++i) {
        if (shape[i] < 1) {
            set_error("every extent must be >= 1");
            return MGARD_ESHAPE;
        }
        if (shape[i] > 1) sq[k++] = shape[i];
    }
    for (int i = 0; i < 4; ++i) n4[i] = 1;
    for (int i = 0; i < k; ++i) n4[4 - k + i] = sq[i];
    *D = k;
    return MGARD_OK;
}

int level_count(const int64_t n4[4], int D, int max_levels) {
    if (D == 0) return 0;
    int L = 1 << 30;
    for (int a = 4 - D; a < 4; ++a) L = std::min(L, axis_levels(n4[a]));
    if (max_levels >= 0) L = std::min(L, max_levels);
    return L;
}

static mgard_status build_plan(const int64_t n4[4], int D, int L, Plan& p, bool device) {
    p.D = D;
    p.L = L;
    for (int a = 0; a < 4; ++a) p.n4[a] = n4[a];
    // finest positions of level-l nodes per axis
    std::vector<std::array<std::vector<int64_t>, 4>> idx(L + 1);
    for (int a = 0; a < 4; ++a) {
        std::vector<int64_t> v(n4[a]);
        for (int64_t i = 0; i < n4[a]; ++i) v[i] = i;
        idx[L][a] = v;
    }
    for (int l = L; l >= 1; --l)
        for (int a = 0; a < 4; ++a) {
            if (n4[a] == 1) {
                idx[l - 1][a] = idx[l][a];
                continue;
            }
            auto cp = coarse_positions((int64_t)idx[l][a].size());
            std::vector<int64_t> v;
            for (auto c : cp) v.push_back(idx[l][a][c]);
            idx[l - 1][a] = v;
        }
    p.shape.resize(L + 1);
    for (int l = 0; l <= L; ++l)
        for (int a = 0; a < 4; ++a) p.shape[l][a] = (int64_t)idx[l][a].size();
    p.count.resize(L + 1);
    p.offset.resize(L + 1);
    int64_t off = 0;
    for (int l = 0; l <= L; ++l) {
        int64_t n = p.level_size(l);
        p.count[l] = l == 0 ? n : n - p.level_size(l - 1);
        p.offset[l] = off;
        off += p.count[l];
    }
    p.K.assign(L + 1, 1.0);
    p.Kax.assign(L + 1, {1.0, 1.0, 1.0, 1.0});
    p.tails.assign(L + 1, std::vector<double>(4 * (Plan::RHO_MAX + 1), 0.0));
    p.hmax.assign(L + 1, {0, 0, 0, 0});
    p.rows.assign(L + 1, {});
    p.linf_c.assign(L + 1, 0.0);
    for (int l = 0; l <= L; ++l)
        for (int a = 0; a < 4; ++a)
            for (size_t i = 1; i < idx[l][a].size(); ++i)
                p.hmax[l][a] = std::max(p.hmax[l][a], idx[l][a][i] - idx[l][a][i - 1]);
    p.mu.assign(L + 1, 1.0);
    p.tune.assign(L + 1, std::array<RowCfg, RK_COUNT>());

    Blob blob;
    struct AxisOff {
        size_t fcls, wlf, wrf, wld, wrd, cbefore, rf, rwf, rwd, subf, invf, cpf, subd, invd, cpd,
            mdiag, moff, mdiagf, mofff;
        bool active;
        int ireg = 0, rlo = 0, rhi = 0;
        double rwi[5] = {0, 0, 0, 0, 0};
    };
    std::vector<std::array<AxisOff, 4>> aoff(L + 1);
    std::vector<std::array<size_t, 4>> ioff(L + 1);
    for (int l = 0; l <= L; ++l) {
        for (int a = 0; a < 4; ++a) {
            ioff[l][a] = blob.add(idx[l][a]);
            AxisOff& o = aoff[l][a];
            o.active = n4[a] > 1;
            if (!o.active) continue;
            std::vector<double> x(idx[l][a].begin(), idx[l][a].end());
            int64_t m = (int64_t)x.size();
            // mass matrix of level l (norms) and its Gershgorin bound
            std::vector<double> mdiag(m, 0.0), moff(m, 0.0);
            double gmax = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double hl = i > 0 ? x[i] - x[i - 1] : 0.0;
                double hr = i + 1 < m ? x[i + 1] - x[i] : 0.0;
                mdiag[i] = (hl + hr) / 3.0;
                moff[i] = hr / 6.0;
                gmax = std::max(gmax, (hl + hr) / 2.0);
            }
            p.mu[l] *= gmax;
            o.mdiag = blob.add(mdiag);
            o.moff = blob.add(moff);
            o.mdiagf = blob.add(cast<float>(mdiag));
            o.mofff = blob.add(cast<float>(moff));
            if (l == 0) continue;
            auto cp = coarse_positions(m);
            int64_t mc = (int64_t)cp.size();
            std::vector<int> fcls(m), cbefore(m);
            // coarse nodes carry the weights (1, 0) so interpolation can be
            // evaluated without branching: u(i) = 1 * u(i) + 0 * u(i)
            std::vector<double> wl(m, 1.0), wr(m, 0.0);
            int64_t J = 0;
            for (int64_t i = 0; i < m; ++i) {
                cbefore[i] = (int)J;
                if (J < mc && cp[J] == i) {
                    fcls[i] = (int)J;
                    ++J;
                } else {
                    int64_t left = J - 1;   // coarse neighbours left, left+1
                    double xa = x[cp[left]], xb = x[cp[left + 1]], xi = x[i];
                    fcls[i] = -(int)(left + 1);
                    wl[i] = (xb - xi) / (xb - xa);
                    wr[i] = (xi - xa) / (xb - xa);
                }
            }
            // restriction R = P^T M on fine positions rf[J]-2 .. rf[J]+2
            std::vector<int64_t> rf(cp.begin(), cp.end());
            std::vector<double> rw(mc * 5, 0.0);
            for (int64_t k = 0; k < m; ++k) {
                int64_t Js[2];
                double Ps[2];
                int np;
                if (fcls[k] >= 0) {
                    Js[0] = fcls[k]; Ps[0] = 1.0; np = 1;
                } else {
                    int64_t left = -fcls[k] - 1;
                    Js[0] = left; Ps[0] = wl[k];
                    Js[1] = left + 1; Ps[1] = wr[k];
                    np = 2;
                }
                for (int q = 0; q < np; ++q)
                    for (int64_t i = k - 1; i <= k + 1; ++i) {
                        if (i < 0 || i >= m) continue;
                        double Mki = (i == k) ? mdiag[k] : (i == k + 1 ? moff[k] : moff[i]);
                        int64_t t = i - rf[Js[q]] + 2;
                        rw[Js[q] * 5 + t] += Ps[q] * Mki;
                    }
            }
            std::vector<double> xc(mc);
            for (int64_t c = 0; c < mc; ++c) xc[c] = x[cp[c]];
            std::vector<double> sub, inv, tcp;
            thomas(xc, sub, inv, tcp);
            p.Kax[l][a] = correction_norm(xc, rf, rw, m, p.tails[l].data() + a * (Plan::RHO_MAX + 1));
            p.K[l] *= p.Kax[l][a];
            axis_row_classes(xc, rf, rw, m, fcls, wl, wr, p.rows[l][a].data());
            std::vector<int> rfi(rf.begin(), rf.end());
            o.fcls = blob.add(fcls);
            o.cbefore = blob.add(cbefore);
            o.wlf = blob.add(cast<float>(wl));
            o.wrf = blob.add(cast<float>(wr));
            o.wld = blob.add(wl);
            o.wrd = blob.add(wr);
            o.rf = blob.add(rfi);
            o.rwf = blob.add(cast<float>(rw));
            o.rwd = blob.add(rw);
            // uniform stretches (checked entry by entry, so the row kernels'
            // arithmetic weights equal the tables exactly)
            int64_t ireg = 0;
            while (ireg < m && wl[ireg] == ((ireg & 1) ? 0.5 : 1.0) &&
                   wr[ireg] == ((ireg & 1) ? 0.5 : 0.0))
                ++ireg;
            o.ireg = (int)ireg;
            o.rlo = o.rhi = 0;
            if (mc > 2 && rf[1] == 2) {
                int64_t hi = 1;
                while (hi < mc && rf[hi] == 2 * hi && 2 * hi + 2 < m &&
                       std::equal(rw.begin() + hi * 5, rw.begin() + hi * 5 + 5, rw.begin() + 5))
                    ++hi;
                o.rlo = 1;
                o.rhi = (int)hi;
                for (int t = 0; t < 5; ++t) o.rwi[t] = rw[5 + t];
            }
            o.subf = blob.add(cast<float>(sub));
            o.invf = blob.add(cast<float>(inv));
            o.cpf = blob.add(cast<float>(tcp));
            o.subd = blob.add(sub);
            o.invd = blob.add(inv);
            o.cpd = blob.add(tcp);
        }
    }
    for (int l = 1; l <= L; ++l) p.linf_c[l] = linf_level_constant(p, l);
    if (!device) return MGARD_OK;
    count_device_alloc();
    cudaError_t e = cudaMalloc(&p.dbuf, blob.bytes.size());
    if (e != cudaSuccess) {
        set_error(std::string("plan tables: ") + cudaGetErrorString(e));
        return MGARD_ENOMEM;
    }
    e = cudaMemcpy(p.dbuf, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error(std::string("plan tables: ") + cudaGetErrorString(e));
        return MGARD_ECUDA;
    }
    char* base = (char*)p.dbuf;
    p.lf.resize(L + 1);
    p.ld.resize(L + 1);
    p.lidx.resize(L + 1);
    for (int l = 0; l <= L; ++l) {
        LevelIndex& li = p.lidx[l];
        for (int a = 0; a < 4; ++a) {
            li.n[a] = p.shape[l][a];
            li.pos[a] = (const int64_t*)(base + ioff[l][a]);
        }
        Level<float>& F = p.lf[l];
        Level<double>& G = p.ld[l];
        std::memset(&F, 0, sizeof(F));
        std::memset(&G, 0, sizeof(G));
        for (int a = 0; a < 4; ++a) {
            F.n[a] = G.n[a] = p.shape[l][a];
            F.nc[a] = G.nc[a] = l > 0 ? p.shape[l - 1][a] : p.shape[l][a];
            const AxisOff& o = aoff[l][a];
            if (!o.active) continue;
            F.ax[a].mdiag = G.ax[a].mdiag = (const double*)(base + o.mdiag);
            F.ax[a].moff = G.ax[a].moff = (const double*)(base + o.moff);
            F.ax[a].mdt = (const float*)(base + o.mdiagf);
            F.ax[a].mot = (const float*)(base + o.mofff);
            G.ax[a].mdt = (const double*)(base + o.mdiag);
            G.ax[a].mot = (const double*)(base + o.moff);
            if (l == 0) continue;
            F.ax[a].fcls = G.ax[a].fcls = (const int*)(base + o.fcls);
            F.ax[a].cbefore = G.ax[a].cbefore = (const int*)(base + o.cbefore);
            F.ax[a].rf = G.ax[a].rf = (const int*)(base + o.rf);
            F.ax[a].wl = (const float*)(base + o.wlf);
            F.ax[a].wr = (const float*)(base + o.wrf);
            F.ax[a].rw = (const float*)(base + o.rwf);
            F.ax[a].tsub = (const float*)(base + o.subf);
            F.ax[a].tinv = (const float*)(base + o.invf);
            F.ax[a].tcp = (const float*)(base + o.cpf);
            G.ax[a].wl = (const double*)(base + o.wld);
            G.ax[a].wr = (const double*)(base + o.wrd);
            G.ax[a].rw = (const double*)(base + o.rwd);
            G.ax[a].tsub = (const double*)(base + o.subd);
            G.ax[a].tinv = (const double*)(base + o.invd);
            G.ax[a].tcp = (const double*)(base + o.cpd);
            F.ax[a].ireg = G.ax[a].ireg = o.ireg;
            F.ax[a].rlo = G.ax[a].rlo = o.rlo;
            F.ax[a].rhi = G.ax[a].rhi = o.rhi;
            for (int t = 0; t < 5; ++t) {
                F.ax[a].rwi[t] = (float)o.rwi[t];
                G.ax[a].rwi[t] = o.rwi[t];
            }
        }
    }
    return MGARD_OK;
}

mgard_status get_plan(int ndim, const int64_t* shape, int max_levels, const Plan** out,
                      bool device) {
    int64_t n4[4];
    int D;
    MGB_TRY(squeeze_shape(ndim, shape, n4, &D));
    int L = level_count(n4, D, max_levels);
    int dev = -1;   // host-only plans use key -1
    if (device && cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_error("no CUDA device");
        return MGARD_ECUDA;
    }
    auto key = std::make_tuple(dev, L, n4[0], n4[1], n4[2], n4[3]);
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = it->second.get();
        return MGARD_OK;
    }
    auto p = std::make_unique<Plan>();
    MGB_TRY(build_plan(n4, D, L, *p, device));
    *out = p.get();
    g_plans[key] = std::move(p);
    return MGARD_OK;
}

void release_plans() {
    std::lock_guard<std::mutex> lock(g_mutex);
    g_plans.clear();
}

void width_denominators(const Plan& p, double s, double* den) {
    const int L = p.L;
    if (std::isinf(s)) {
        double denom = 1.0;   // 1 + sum_l c_l, in level order
        for (int l = 1; l <= L; ++l) denom += p.linf_c[l];
        for (int l = 0; l <= L; ++l) den[l] = denom;
    } else {
        for (int l = 0; l <= L; ++l) {
            const double m = p.D ? p.mu[l] : 1.0;
            const double n = p.D ? (double)p.count[l] : 1.0;
            den[l] = std::sqrt((double)(L + 1) * std::pow(4.0, s * l) * m * n);
        }
    }
}

void bin_widths(const Plan& p, double tol_abs, double s, double* w) {
    std::vector<double> den(p.L + 1);
    width_denominators(p, s, den.data());
    for (int l = 0; l <= p.L; ++l) w[l] = 2.0 * tol_abs / den[l] * WIDTH_MARGIN;
}

}  // namespace mgb
