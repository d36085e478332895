// Ratio-targeted compression: the sizer (one decomposition, exact sizes at
// any tolerance), the predictor's features, and mgard_compress_to_ratio.
//
// The paper states compression as "given tau, produce a buffer"; asking for
// a compression ratio instead means searching tau.  The sizer makes every
// probe cheap and exact: the decomposition does not depend on tau, so only
// widths, quantization, codebook and the count pass run per probe, and the
// count pass yields the exact buffer size (no payload is packed).  The
// network proposes tau from statistics of the decomposition; a bracketed
// bisection on log10(tau) corrects it when the size misses the target.  The
// bound belongs to the chosen tau exactly as in mgard_compress.
#include <cmath>
#include <cstring>
#include <memory>

#include "predictor.cuh"
#include "quantize.cuh"
#include "rows3.cuh"

namespace mgb {

namespace {

constexpr int NLEV = 12;
constexpr int PER_LEVEL = 3 + FEAT_BINS - 1;
static_assert(NLEV * PER_LEVEL + 4 == MGARD_NFEAT, "feature layout");

__global__ void k_feat_amax(const double* __restrict__ maxparts, double* amax) {
    double m = 0.0;
    for (int i = threadIdx.x; i < RED_PARTS; i += 32) m = fmax(m, maxparts[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *amax = m;
}

struct FeatArgs {
    int L, D;
    double logN, logR;
    long long off[NLEV + 1];     // partial records of slot k: off[k] .. off[k+1]
    double count[NLEV];          // coefficients of the level in slot k
};

// One warp per level slot (finest first), then the global inputs.
__global__ void k_feat_final(FeatArgs a, const FeatPart* __restrict__ part, float* __restrict__ f) {
    const int slot = blockIdx.x, lane = threadIdx.x;
    if (slot == NLEV) {
        if (lane == 0) {
            f[NLEV * PER_LEVEL + 0] = (float)a.D;
            f[NLEV * PER_LEVEL + 1] = (float)a.L;
            f[NLEV * PER_LEVEL + 2] = (float)a.logN;
            f[NLEV * PER_LEVEL + 3] = (float)a.logR;
        }
        return;
    }
    float* o = f + slot * PER_LEVEL;
    if (slot > a.L) {
        for (int k = lane; k < PER_LEVEL; k += 32) o[k] = 0.f;
        return;
    }
    double s = 0.0, s2 = 0.0;
    for (long long b = a.off[slot] + lane; b < a.off[slot + 1]; b += 32) {
        s += part[b].sum;
        s2 += part[b].sum2;
    }
    unsigned long long h = 0;   // lane k < FEAT_BINS: records with exactly k thresholds above |c|
    for (long long b = a.off[slot]; b < a.off[slot + 1]; ++b)
        if (lane < FEAT_BINS) h += part[b].hist[lane];
    for (int d = 16; d > 0; d >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, d);
        s2 += __shfl_xor_sync(0xffffffffu, s2, d);
    }
    // fraction below threshold j = records with k > j
    unsigned long long above = 0;
    for (int k = FEAT_BINS - 1; k >= 1; --k) {
        const unsigned long long hk = __shfl_sync(0xffffffffu, h, k);
        above += hk;
        if (lane == k - 1) o[3 + lane] = (float)((double)above / a.count[slot]);
    }
    if (lane == 0) {
        const double n = a.count[slot];
        const double m = s / n;
        o[0] = (float)log10(n);
        o[1] = (float)m;
        o[2] = (float)sqrt(fmax(s2 / n - m * m, 0.0));
    }
}

}  // namespace

}  // namespace mgb

// The sizer: a plan, the workspace holding one decomposition, and the
// scratch of the feature pass.
struct mgard_sizer_s {
    const mgb::Plan* p = nullptr;
    mgard_dtype dtype = MGARD_F32;
    const void* field = nullptr;
    int ndim = 0;
    int64_t shape[4] = {1, 1, 1, 1};
    double s = 0.0;
    std::unique_ptr<mgb::CompressWork<float>> wf;
    std::unique_ptr<mgb::CompressWork<double>> wd;
    mgb::DevBuf meta, amax, fparts;
    mgb::CompressMeta hmeta;
};

namespace mgb {

namespace {

mgard_status sizer_encode(mgard_sizer* z, double tol, mgard_tolmode mode, char* dd, uint64_t cap,
                          cudaStream_t st) {
    const mgard_header h0 = header_template(*z->p, z->dtype, z->ndim, z->shape, tol, z->s, mode);
    CompressMeta* meta = z->meta.as<CompressMeta>();
    if (z->dtype == MGARD_F32)
        return compress_encode<float>(*z->p, (const float*)z->field, h0, tol, z->s, mode, dd, cap,
                                      *z->wf, meta, st);
    return compress_encode<double>(*z->p, (const double*)z->field, h0, tol, z->s, mode, dd, cap,
                                   *z->wd, meta, st);
}

mgard_status sizer_read_meta(mgard_sizer* z, cudaStream_t st) {
    MGB_CUDA(cudaMemcpyAsync(&z->hmeta, z->meta.p, sizeof(CompressMeta), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    return MGARD_OK;
}

mgard_status meta_error(unsigned st) {
    if (st & ST_NONFINITE) {
        set_error("input holds NaN or Inf");
        return MGARD_ENONFINITE;
    }
    if (st & ST_RANGE) {
        set_error("tolerance too small: a quantized value exceeds the 32-bit range");
        return MGARD_ERANGE;
    }
    if (st & ST_NOCODE) {
        set_error("a symbol has no Huffman code");
        return MGARD_EINVAL;
    }
    return MGARD_OK;
}

}  // namespace

}  // namespace mgb

using namespace mgb;

extern "C" {

mgard_status mgard_sizer_create(const void* field, int ndim, const int64_t* shape,
                                mgard_dtype dtype, double s, mgard_sizer** out, void* stream) {
    if (!field || !out || std::isnan(s) || s < 0.0) return MGARD_EINVAL;
    if (dtype != MGARD_F32 && dtype != MGARD_F64) return MGARD_EDTYPE;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, field) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        set_error("the sizer takes a device field");
        return MGARD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::unique_ptr<mgard_sizer> z(new mgard_sizer());
    MGB_TRY(get_plan(ndim, shape, -1, &z->p));
    z->dtype = dtype;
    z->field = field;
    z->ndim = ndim;
    for (int i = 0; i < ndim && i < 4; ++i) z->shape[i] = shape[i];
    z->s = s;
    MGB_TRY(z->meta.alloc(sizeof(CompressMeta), st));
    MGB_TRY(z->amax.alloc(sizeof(double), st));
    int64_t nparts = 0;
    for (int l = 0; l <= z->p->L; ++l) nparts += feature_blocks(*z->p, l);
    MGB_TRY(z->fparts.alloc(nparts * sizeof(FeatPart), st));
    // the decomposition for both tolerance modes (energies when s is finite)
    if (dtype == MGARD_F32) {
        z->wf.reset(new CompressWork<float>());
        MGB_TRY(z->wf->alloc(*z->p, st));
        MGB_TRY(compress_decompose<float>(*z->p, (const float*)field, s, MGARD_REL, *z->wf,
                                          z->meta.as<CompressMeta>(), st));
    } else {
        z->wd.reset(new CompressWork<double>());
        MGB_TRY(z->wd->alloc(*z->p, st));
        MGB_TRY(compress_decompose<double>(*z->p, (const double*)field, s, MGARD_REL, *z->wd,
                                           z->meta.as<CompressMeta>(), st));
    }
    MGB_TRY(sizer_read_meta(z.get(), st));
    MGB_TRY(meta_error(z->hmeta.status));
    *out = z.release();
    return MGARD_OK;
}

mgard_status mgard_sizer_size(mgard_sizer* z, double tol, mgard_tolmode mode, size_t* bytes,
                              void* stream) {
    if (!z || !bytes || !(tol > 0.0) || !std::isfinite(tol)) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    MGB_TRY(sizer_encode(z, tol, mode, nullptr, 0, st));
    MGB_TRY(sizer_read_meta(z, st));
    MGB_TRY(meta_error(z->hmeta.status));
    *bytes = z->hmeta.total;
    return MGARD_OK;
}

mgard_status mgard_sizer_features(mgard_sizer* z, double target_ratio, float* features,
                                  void* stream) {
    if (!z || !features || !(target_ratio > 0.0)) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const Plan& p = *z->p;
    const int L = p.L;
    const double* maxparts = z->dtype == MGARD_F32 ? z->wf->parts.as<double>() : z->wd->parts.as<double>();
    MGB_LAUNCH("k_feat_amax", st, k_feat_amax<<<1, 32, 0, st>>>(maxparts, z->amax.as<double>()));
    FeatArgs a;
    std::memset(&a, 0, sizeof(a));
    a.L = L;
    a.D = p.D;
    a.logN = std::log10((double)p.total());
    a.logR = std::log10(target_ratio);
    FeatPart* parts = z->fparts.as<FeatPart>();
    int64_t off = 0;
    for (int slot = 0; slot < NLEV; ++slot) {
        a.off[slot] = off;
        if (slot > L) continue;
        const int l = L - slot;
        a.count[slot] = (double)p.count[l];
        const int64_t nb = feature_blocks(p, l);
        // row-kernel shapes keep the coefficients in symbol order in `top`
        if (z->dtype == MGARD_F32) {
            const float* lvl = rows3_ok(p) ? z->wf->top.as<float>() + p.offset[l]
                                           : (l == L ? (L ? z->wf->top.as<float>() : (const float*)z->field) : z->wf->py.lv[l]);
            MGB_TRY(level_features<float>(p, l, lvl, z->amax.as<double>(), parts + off, st));
        } else {
            const double* lvl = rows3_ok(p) ? z->wd->top.as<double>() + p.offset[l]
                                            : (l == L ? (L ? z->wd->top.as<double>() : (const double*)z->field) : z->wd->py.lv[l]);
            MGB_TRY(level_features<double>(p, l, lvl, z->amax.as<double>(), parts + off, st));
        }
        off += nb;
    }
    a.off[NLEV] = off;
    MGB_LAUNCH("k_feat_final", st, k_feat_final<<<NLEV + 1, 32, 0, st>>>(a, parts, features));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status mgard_sizer_compress(mgard_sizer* z, double tol, mgard_tolmode mode, void* out,
                                  size_t* out_bytes, void* stream) {
    if (!z || !out || !out_bytes || !(tol > 0.0) || !std::isfinite(tol)) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t N = (uint64_t)z->p->total();
    const Sections fx = layout(z->p->L, (N + CHUNK - 1) / CHUNK, 0, 0);
    if (*out_bytes < fx.outliers || ((uintptr_t)out & 15) != 0) {
        set_error("output buffer too small or not 16-byte aligned");
        return MGARD_EINVAL;
    }
    char* dd = (char*)out;
    MGB_CUDA(cudaMemsetAsync(dd, 0, fx.outliers, st));
    MGB_TRY(sizer_encode(z, tol, mode, dd, *out_bytes, st));
    CompressMeta* meta = z->meta.as<CompressMeta>();
    if (z->dtype == MGARD_F32) MGB_TRY(compress_pack<float>(*z->p, dd, *z->wf, meta, st));
    else MGB_TRY(compress_pack<double>(*z->p, dd, *z->wd, meta, st));
    MGB_TRY(sizer_read_meta(z, st));
    MGB_TRY(meta_error(z->hmeta.status));
    *out_bytes = z->hmeta.total;
    if (z->hmeta.status & ST_CAPACITY) {
        set_error("output buffer too small");
        return MGARD_ECAPACITY;
    }
    return MGARD_OK;
}

void mgard_sizer_free(mgard_sizer* z) {
    if (!z) return;
    cudaDeviceSynchronize();   // workspaces free asynchronously on their streams
    delete z;
}

mgard_status mgard_compress_to_ratio(const void* field, int ndim, const int64_t* shape,
                                     mgard_dtype dtype, double target_ratio, double s,
                                     const float* params, double rel_err, double* tol_used,
                                     void* out, size_t* out_bytes, int* passes, void* stream) {
    if (!(target_ratio > 0.0) || !(rel_err > 0.0) || !out || !out_bytes) return MGARD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    mgard_sizer* zr = nullptr;
    MGB_TRY(mgard_sizer_create(field, ndim, shape, dtype, s, &zr, stream));
    std::unique_ptr<mgard_sizer, void (*)(mgard_sizer*)> z(zr, mgard_sizer_free);
    const double fbytes = (double)z->p->total() * (dtype == MGARD_F64 ? 8.0 : 4.0);
    int npass = 0;
    double best_tol = 0.0, best_err = 1e300;
    // probe: exact ratio at tol, remembering the closest one
    auto probe = [&](double tol, double* ratio) -> mgard_status {
        size_t b = 0;
        MGB_TRY(mgard_sizer_size(z.get(), tol, MGARD_REL, &b, stream));
        ++npass;
        *ratio = fbytes / (double)b;
        const double e = std::fabs(*ratio / target_ratio - 1.0);
        if (e < best_err) {
            best_err = e;
            best_tol = tol;
        }
        return MGARD_OK;
    };
    const double TMIN = 1e-9, TMAX = 1.0;
    double lo = 1e-7, hi = 1.0, r;
    bool done = false;
    if (params) {
        // three forward passes: at log10(target) and 0.05 either side, for
        // the proposal and the network's local slope of log tol over log ratio
        DevBuf feat, y;
        MGB_TRY(feat.alloc(3 * MGARD_NFEAT * sizeof(float), st));
        MGB_TRY(y.alloc(3 * sizeof(float), st));
        float* f = feat.as<float>();
        MGB_TRY(mgard_sizer_features(z.get(), target_ratio, f, stream));
        MGB_CUDA(cudaMemcpyAsync(f + MGARD_NFEAT, f, MGARD_NFEAT * sizeof(float), cudaMemcpyDeviceToDevice, st));
        MGB_CUDA(cudaMemcpyAsync(f + 2 * MGARD_NFEAT, f, MGARD_NFEAT * sizeof(float), cudaMemcpyDeviceToDevice, st));
        const float side_in[2] = {(float)(std::log10(target_ratio) + 0.05),
                                  (float)(std::log10(target_ratio) - 0.05)};
        MGB_CUDA(cudaMemcpyAsync(f + 2 * MGARD_NFEAT - 1, &side_in[0], sizeof(float), cudaMemcpyHostToDevice, st));
        MGB_CUDA(cudaMemcpyAsync(f + 3 * MGARD_NFEAT - 1, &side_in[1], sizeof(float), cudaMemcpyHostToDevice, st));
        MGB_TRY(mlp_forward(params, f, 3, y.as<float>(), st));
        float hy[3] = {0.f, 0.f, 0.f};
        MGB_CUDA(cudaMemcpyAsync(hy, y.p, sizeof(hy), cudaMemcpyDeviceToHost, st));
        MGB_CUDA(cudaStreamSynchronize(st));
        double t0 = std::pow(10.0, std::isfinite(hy[0]) ? (double)hy[0] : -3.0);
        t0 = std::fmin(std::fmax(t0, TMIN), TMAX);
        const double dinv = ((double)hy[1] - (double)hy[2]) / 0.1;   // d log tol / d log ratio
        double slope0 = std::isfinite(dinv) && dinv > 0.2 ? 1.0 / dinv : 0.5;
        slope0 = std::fmin(std::fmax(slope0, 0.02), 5.0);
        // Safeguarded secant on (log10 tol, log ratio), started at the
        // network's proposal: probes below the target raise the lower end of
        // the bracket, probes above lower the upper end; a step that leaves
        // the bracket, or a second step on the same side, is replaced by the
        // bracket's midpoint.  The first step uses the network's slope, later
        // ones the last secant.
        const double Y = std::log10(target_ratio);
        double x = std::log10(t0), lx = std::log10(TMIN), hx = std::log10(TMAX);
        bool have_lo = false, have_hi = false;
        double px = 0.0, py = 0.0, slope = slope0;
        bool have_prev = false;
        int same_side = 0, last_side = 0;
        for (int it = 0; it < 40; ++it) {
            MGB_TRY(probe(std::pow(10.0, x), &r));
            if (best_err <= rel_err) {
                done = true;
                break;
            }
            const double yv = std::log10(r);
            const int side = yv < Y ? -1 : 1;
            if (side < 0) {
                lx = x;
                have_lo = true;
            } else {
                hx = x;
                have_hi = true;
            }
            same_side = side == last_side ? same_side + 1 : 0;
            last_side = side;
            if (have_prev && std::fabs(x - px) > 1e-12) {
                const double sl = (yv - py) / (x - px);
                if (sl > 1e-3) slope = sl;
            }
            px = x;
            py = yv;
            have_prev = true;
            if (hx - lx < 1e-9) break;
            double nx = x + (Y - yv) / slope;
            const double step = 2.0;   // at most two decades per step
            nx = std::fmin(std::fmax(nx, x - step), x + step);
            const bool bracketed = have_lo && have_hi;
            if (nx <= lx || nx >= hx || (bracketed && same_side >= 1)) nx = 0.5 * (lx + hx);
            if (!bracketed && (nx <= lx || nx >= hx)) nx = side < 0 ? std::fmin(x + step, hx) : std::fmax(x - step, lx);
            x = nx;
        }
        done = true;   // the secant keeps the closest probe either way
    } else {
        double rl, rh;
        MGB_TRY(probe(lo, &rl));
        MGB_TRY(probe(hi, &rh));
        done = best_err <= rel_err;
    }
    for (int it = 0; !done && it < 60 && hi / lo > 1.0 + 1e-9; ++it) {
        const double mid = std::sqrt(lo * hi);
        MGB_TRY(probe(mid, &r));
        if (best_err <= rel_err) break;
        if (r < target_ratio) lo = mid;
        else hi = mid;
    }
    MGB_TRY(mgard_sizer_compress(z.get(), best_tol, MGARD_REL, out, out_bytes, stream));
    if (tol_used) *tol_used = best_tol;
    if (passes) *passes = npass;
    return MGARD_OK;
}

}  // extern "C"
