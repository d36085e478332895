// Multilevel decomposition / recomposition on the device (declarations).
#pragma once

#include <vector>

#include "plan.cuh"

namespace mgb {

// The library's stream-ordered memory pool on the current device (created
// on first use, never trimmed, so repeated calls reuse their workspace).
cudaMemPool_t workspace_pool();

// Stream-ordered device allocation that frees itself.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, st);
    }
    mgard_status alloc(size_t bytes, cudaStream_t s) {
        st = s;
        if (bytes == 0) bytes = 16;
        cudaMemPool_t pool = workspace_pool();
        count_device_alloc();
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error(std::string("device allocation: ") + cudaGetErrorString(e));
            return MGARD_ENOMEM;
        }
        return MGARD_OK;
    }
    template <typename T> T* as() const { return (T*)p; }
};

// Compact per-level arrays of the pyramid: level l < L has its own
// row-major array of the level-l grid; level L is the caller's array.
template <typename T>
struct Pyramid {
    std::vector<T*> lv;       // [l] compact array of level l (l < L)
    DevBuf store;
    DevBuf temp0, temp1;      // restriction ping-pong buffers
    // device status word for kernels' bounded waits (ST_TIMEOUT); null: the
    // library's per-device fallback word
    unsigned* status = nullptr;
    // with defer_tail, decompose_pyramid leaves the one-block tail (and the
    // copy of level 0 into the symbol-order array) to the caller, which runs
    // it (a batched tail launch) and then decompose_finish; tail_pending
    // tells whether it did
    bool defer_tail = false;
    bool tail_pending = false;
    // recompose_pyramid with defer_tail stops after level 0 in the same way
    // (tail_pending); called again with tail_done it skips the tail
    bool tail_done = false;
    mgard_status alloc(const Plan& p, cudaStream_t st);
};

// Coarse grids with fewer nodes than this run their restriction and
// tridiagonal solves in double precision.  None do: on B300 FP64 runs at
// about 2 lanes per clock per SM, and float32 corrections keep every level
// within the float32 tolerance of the FP64 decomposition.
constexpr int64_t FP64_SOLVE_NODES = 0;

// Opt a kernel in to `bytes` of dynamic shared memory where its current
// limit (48 KB minus its static shared memory by default) is lower.
mgard_status allow_dynamic_smem(const void* kern, size_t bytes);
// The per-device status word that kernels with bounded waits use when the
// caller has none of its own (device address; set-up on first use).
unsigned* fallback_status();

// A grid of persistent blocks of `kern`: as many as stay resident on the
// device at once (occupancy at this block size and dynamic shared memory),
// at most `work`.
mgard_status resident_grid(const void* kern, int threads, size_t smem, int64_t work, int* grid);

// Levels of at most TAIL_NODES nodes (TAIL_LEVELS of them at most) run in a
// single one-block launch each way (tail.cu) on the symbol-order path.
constexpr int64_t TAIL_NODES = 5000;
constexpr int TAIL_LEVELS = 8;
// The number Lt of such levels above level 0 (levels 1..Lt); 0 if none.
int tail_levels(const Plan& p);
// Levels Lt..1 of a decomposition: level_Lt holds level Lt's nodal values
// (py.lv[Lt], or the input when Lt = L); writes the coefficients of levels
// 1..Lt into zs (symbol order) or, with zs null, over the new nodes of each
// level's own array (py.lv[l], `top` for l = L), and the nodal values of
// levels Lt-1..0 into the pyramid.  Scratch: py.temp0 and py.temp1.
template <typename T>
mgard_status tail_decompose(const Plan& p, int Lt, Pyramid<T>& py, const T* level_Lt, T* zs,
                            T* top, cudaStream_t st);
// The same for many fields in one launch: tail_job fills one field's
// arguments (host memory of tail_args_bytes<T>() bytes; *smem receives the
// shared memory they need); tail_decompose_batch runs n of them (device
// array `jobs`) on a persistent grid whose blocks take jobs from *counter
// (device; reset here, stream-ordered), with smem the largest need.
template <typename T>
size_t tail_args_bytes();
template <typename T>
mgard_status tail_job(const Plan& p, int Lt, Pyramid<T>& py, const T* level_Lt, T* zs, T* top,
                      void* args, size_t* smem);
template <typename T>
mgard_status tail_decompose_batch(const void* jobs, int n, size_t smem, unsigned* counter,
                                  cudaStream_t st);
template <typename T>
mgard_status tail_recompose_batch(const void* jobs, int n, size_t smem, unsigned* counter,
                                  cudaStream_t st);
// The inverse for levels 1..Lt: from py.lv[0] and the coefficients (zs, or
// the level arrays), writes level Lt's nodal values to level_Lt (and
// levels 1..Lt-1 into the pyramid).
template <typename T>
mgard_status tail_recompose(const Plan& p, int Lt, Pyramid<T>& py, const T* zs, const T* top,
                            T* level_Lt, cudaStream_t st);

// Decompose `in` (level-L nodal values) into `top` (coefficients on the
// level-L new nodes; coarse positions untouched) and the pyramid levels.
// `in` may equal `top`.  If `E` is non-null, E[l] receives u_l^T M_l u_l of
// every level's nodal values (FP64 accumulation; host array of L+1).
// With `Epart` (device, energy_parts_total(p) doubles) the same energies
// are left as partial sums on the device instead (no host round trip):
// level l's partials start at energy_parts_offset(p, l).  With `zs` (device,
// N values; row-kernel shapes only) every level's coefficients, and the
// level-0 values first, go to zs in symbol order (level 0, then the nodes
// new on levels 1..L, row-major per level) instead of `top` and the
// pyramid; `top` is then unused.
template <typename T>
mgard_status decompose_pyramid(const Plan& p, const T* in, T* top, Pyramid<T>& py,
                               cudaStream_t st, double* E, double* Epart = nullptr,
                               T* zs = nullptr);

// What decompose_pyramid left when it deferred the tail, after the tail
// has run: level 0 into the symbol-order array zs.
template <typename T>
mgard_status decompose_finish(const Plan& p, Pyramid<T>& py, T* zs, cudaStream_t st);

// Recompose: `top` holds level-L coefficients (coarse positions ignored),
// py.lv[l] the coefficients of level l >= 1 (coarse positions ignored) and
// py.lv[0] the level-0 values.  Writes nodal values to `out` (may equal
// `top`).  Overwrites the pyramid.
// With `zs` the coefficients (and level-0 values) are read from an array
// in symbol order, as decompose_pyramid writes them; `top` is then unused.
template <typename T>
mgard_status recompose_pyramid(const Plan& p, const T* top, T* out, Pyramid<T>& py,
                               cudaStream_t st, const T* zs = nullptr);

// coarse += sign * M_{l-1}^{-1} P^T M_l z for level l (the correction of a
// decomposition step, sign = +1, or of a recomposition step, sign = -1);
// t0, t1 are the pyramid's restriction buffers.
template <typename T>
mgard_status correct_coarse(const Plan& p, int l, const T* z, T* coarse, void* t0, void* t1,
                            T sign, cudaStream_t st);

// In-place layout <-> pyramid (levels below L only).
template <typename T>
mgard_status scatter_levels(const Plan& p, const Pyramid<T>& py, T* data, cudaStream_t st);
template <typename T>
mgard_status gather_levels(const Plan& p, const T* data, Pyramid<T>& py, cudaStream_t st);

// Reductions (FP64 results, deterministic order; synchronize the stream).
template <typename T>
mgard_status max_abs(const T* a, const T* b, int64_t n, double* out, unsigned* status,
                     cudaStream_t st);
template <typename T>
mgard_status mass_norm2(const Plan& p, int l, const T* u, double* out, cudaStream_t st);

// Launch-only forms for pipelines without host round trips: partial
// results stay in device memory.  max_abs_partials writes RED_PARTS values
// (their maximum is max|a|); mass_norm2_partials writes mass_norm_parts(p, l)
// values (their sum is u^T M_l u).
constexpr int RED_PARTS = 592;
template <typename T>
mgard_status max_abs_partials(const T* a, int64_t n, double* part, unsigned* status,
                              cudaStream_t st);
int64_t mass_norm_parts(const Plan& p, int l);
int64_t energy_parts_total(const Plan& p);
int64_t energy_parts_offset(const Plan& p, int l);
template <typename T>
mgard_status mass_norm2_partials(const Plan& p, int l, const T* u, double* part, cudaStream_t st);

// y = b - a in double (device), for error norms.
template <typename T>
mgard_status difference(const T* a, const T* b, double* y, int64_t n, cudaStream_t st);

}  // namespace mgb
