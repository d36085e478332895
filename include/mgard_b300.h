/*
 * mgard_b300.h -- C ABI of a B300 (sm_103a) implementation of MGARD's
 * multilevel decomposition, level-wise quantization and Huffman coding.
 *
 * The operations follow the MGARD paper (Gong et al., "MGARD: A multigrid
 * framework for high-performance, error-controlled data compression and
 * refactoring"): "Software design" (decomposition of u into multilevel
 * coefficients u_mc, linear quantization to multiples of a bin width chosen
 * by error estimators from tau and s, lossless encoding into a
 * self-describing buffer; decompression is the inverse procedure), "APIs"
 * (high-level compress/decompress with buffer-location detection; low-level
 * per-step functions with device asynchrony) and Listing 1 (the argument
 * list of compress/decompress).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Arrays are row-major (last axis contiguous), 1 <= ndim <= 4, every
 *    extent >= 1.  Axes of extent 1 are ignored.  Level L is the input grid;
 *    along an axis the next coarser level keeps the even positions plus the
 *    last one; L = min over axes of the number of such coarsenings before an
 *    axis has two nodes (capped by max_levels when max_levels >= 0).
 *  - dtype selects float (MGARD_F32) or double (MGARD_F64) data.  F32 data is
 *    decomposed in float with float accumulation on every level, the
 *    restriction and tridiagonal solves of the coarse grids included; F64
 *    data in double.  Error norms and verification are always double.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    stream-ordered.  Functions documented as taking device pointers require
 *    pointers to device (or managed) memory of the current device.
 *  - Every function returns a status; nothing is thrown and no function
 *    aborts the process.  A failing CUDA call is reported as MGARD_ECUDA
 *    (MGARD_ENOMEM for allocations) with its text in mgard_last_error().
 *  - The library keeps per-shape tables (the "plan") in device memory for
 *    the life of the process; mgard_release_plans() drops them.  Workspace is
 *    taken from the stream-ordered allocator (cudaMallocAsync) on `stream`.
 */
#ifndef MGARD_B300_H
#define MGARD_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MGARD_OK = 0,
    MGARD_EINVAL = 1,     /* bad argument (tolerance <= 0 or NaN, s < 0, null pointer, ...) */
    MGARD_ESHAPE = 2,     /* ndim outside 1..4 or an extent < 1 */
    MGARD_EDTYPE = 3,     /* unknown dtype */
    MGARD_ENONFINITE = 4, /* input holds NaN or Inf */
    MGARD_ENOMEM = 5,     /* device or host allocation failed */
    MGARD_ECUDA = 6,      /* a CUDA runtime call failed */
    MGARD_ECORRUPT = 7,   /* compressed buffer fails validation */
    MGARD_EBOUND = 8,     /* verification found the error above the tolerance */
    MGARD_ETIMEOUT = 9,   /* a bounded device wait gave up */
    MGARD_ECAPACITY = 10, /* preallocated output too small; required size returned */
    MGARD_ERANGE = 11     /* tolerance so small that a quantized value exceeds 32 bits */
} mgard_status;

typedef enum { MGARD_F32 = 0, MGARD_F64 = 1 } mgard_dtype;
typedef enum { MGARD_ABS = 0, MGARD_REL = 1 } mgard_tolmode;

/* Size of the quantization dictionary and the escape symbol.  Symbol
 * q + MGARD_DICT/2 codes |q| < MGARD_DICT/2; symbol 0 marks an outlier whose
 * value q is carried separately as a 32-bit integer. */
#define MGARD_DICT 4096
#define MGARD_ESC 0
/* Huffman stream: chunks of MGARD_CHUNK symbols, each starting on a 32-bit
 * word, bits MSB-first within a word; codes are at most MGARD_LMAX bits. */
#define MGARD_CHUNK 1024
#define MGARD_SUB 256
#define MGARD_LMAX 32

const char* mgard_strerror(mgard_status status);
/* Text of the most recent failure in the calling thread ("" if none). */
const char* mgard_last_error(void);
/* Number of CUDA allocation calls (device memory, the stream-ordered
 * workspace pool, pinned host memory) the library has made in this process
 * so far.  For diagnostics and tests: a caller can check that a sequence of
 * calls allocated nothing. */
uint64_t mgard_device_allocations(void);
/* Library version as 0xMMmmpp. */
uint32_t mgard_version(void);

/* Number of levels L for a shape (after squeezing extent-1 axes). */
mgard_status mgard_levels(int ndim, const int64_t* shape, int max_levels, int* nlevels);

/* ---- Low-level API: decomposition ("Software design", first paragraph) ---
 * In-place multilevel decomposition of `data` (device pointer, `dtype`).
 * On return (stream-ordered) every node holds the coefficient of the level
 * on which it first appears: c = u_l - (multilinear interpolation of the
 * level-(l-1) values), where u_l are the nodal values of the L2 projection
 * of the piecewise-multilinear u onto level l; level-0 nodes hold the
 * values of the projection onto level 0.  Workspace: about 1/7 of the
 * array for the coarser levels plus two restriction buffers of at most
 * half of it.  May return before the device work completes. */
mgard_status mgard_decompose(void* data, int ndim, const int64_t* shape, mgard_dtype dtype,
                             int max_levels, void* stream);
/* Inverse of mgard_decompose, in place (device pointer). */
mgard_status mgard_recompose(void* data, int ndim, const int64_t* shape, mgard_dtype dtype,
                             int max_levels, void* stream);

/* ---- Low-level API: error estimators ("Software design", second paragraph)
 * Bin widths w_0..w_L (host array of L+1 doubles) for an absolute
 * tolerance.  s = INFINITY selects the L-infinity bound
 *   w = 2 tau / (1 + sum_{l=1..L} c_l),
 * c_l an upper bound of the largest row sum of level l's error operator
 * I_new - P C_l (C_l = M_{l-1}^{-1} P^T M_l, P interpolation, I_new the
 * identity on the new nodes): with, per axis, the row sums T of
 * B_d = P_d C_d, their parts Tc over coarse columns and the diagonals b, a
 * row sums to prod T - prod Tc + [row new](|1 - prod b| - prod |b|), and
 * c_l takes per-axis extremes over each class of rows (which axes are
 * coarse); finer levels only interpolate, so |e| <= (w/2)(1 + sum c_l);
 * finite s >= 0 the s-norm bound
 *   w_l = 2 tau / sqrt((L+1) 4^{s l} mu_l n_l),
 *   mu_l = prod_d max_i (h_{i-1}+h_i)/2, n_l = nodes new on level l;
 * every width is multiplied by (1 - 2^-8) so float32 quantization rounding
 * stays inside the bound.  Host-only (builds the plan on first use). */
mgard_status mgard_bin_widths(int ndim, const int64_t* shape, int max_levels, double tol_abs,
                              double s, double* widths, int* nlevels);

/* Norm of a field (device pointer): s = INFINITY gives max|u|; finite s
 * gives ||u||_s with ||u||_s^2 = sum_l 4^{s l} ||(Q_l - Q_{l-1}) u||_{L2}^2
 * (s = 0: the L2 norm of the piecewise-multilinear interpolant).  FP64
 * accumulation; the projections are computed in the data's precision.
 * Synchronizes the stream; result in *out (host). */
mgard_status mgard_norm(const void* data, int ndim, const int64_t* shape, mgard_dtype dtype,
                        int max_levels, double s, double* out, void* stream);
/* The same norm of the difference b - a (device pointers), evaluated with
 * the difference and its projections in FP64 (verification of the error
 * bound).  MGARD_ENONFINITE if either array holds NaN or Inf. */
mgard_status mgard_error_norm(const void* a, const void* b, int ndim, const int64_t* shape,
                              mgard_dtype dtype, int max_levels, double s, double* out,
                              void* stream);

/* ---- Low-level API: quantization ("Software design", second paragraph) --
 * Quantize an in-place decomposed array (device pointer) with bin widths
 * `widths` (host, L+1 entries).  Symbols are written in level order (level
 * 0 nodes, then the nodes new on levels 1..L, each in row-major order of
 * that level's grid): n = product of the extents symbols in total.  F32 data
 * decides q = rint(float(c) * float(1/w)) in float; F64 data
 * q = rint(c / w) in double.  |q| < MGARD_DICT/2 -> symbol q + MGARD_DICT/2,
 * else MGARD_ESC and escapes[position] = q, where for F32 data with
 * |q| >= MGARD_DICT the escape is recomputed as rint(c / w) in double (the
 * kernels reach the same integer through two-float arithmetic where it
 * provably agrees).
 * hist (device, MGARD_DICT uint64) is overwritten with symbol counts.
 * symbols, escapes: device arrays of n entries.  Synchronizes the stream;
 * MGARD_ERANGE if some |rint(c/w)| > 2^31-1, MGARD_ENONFINITE for NaN/Inf. */
mgard_status mgard_quantize(const void* coeffs, int ndim, const int64_t* shape, mgard_dtype dtype,
                            int max_levels, const double* widths, uint16_t* symbols,
                            int32_t* escapes, uint64_t* hist, void* stream);
/* Inverse: writes the in-place coefficient array (device pointer) from
 * symbols and escapes (device, n entries each): c = q * w (float32 product
 * for F32 symbols and escapes with |q| < MGARD_DICT; otherwise the double
 * product rounded to the dtype). */
mgard_status mgard_dequantize(const uint16_t* symbols, const int32_t* escapes, int ndim,
                              const int64_t* shape, mgard_dtype dtype, int max_levels,
                              const double* widths, void* coeffs, void* stream);

/* ---- Low-level API: Huffman coding ("Software design", third paragraph) --
 * Code lengths (device uint8[MGARD_DICT]) and canonical codes (device
 * uint32[MGARD_DICT]) from a histogram (device uint64[MGARD_DICT]).  Leaves
 * (symbols with nonzero count) sorted by (count, symbol) are merged with two
 * FIFO queues, leaf queue first on equal weight; lengths over MGARD_LMAX
 * repeat the construction on max(1, count >> k) for the smallest k >= 1 that
 * fits; a single used symbol gets length 1.  Canonical codes are consecutive
 * in (length, symbol) order. */
mgard_status mgard_huffman_codebook(const uint64_t* hist, uint8_t* lengths, uint32_t* codes,
                                    void* stream);
/* Encode n symbols (device) with code lengths `lengths` (device).  Outputs
 * (device): words (capacity `words_cap` uint32), word_off / esc_off
 * (ceil(n / MGARD_CHUNK) uint64 each: exclusive prefix of per-chunk word
 * counts and escape counts), sub_off (6 uint16 per chunk: the bit offsets
 * inside the chunk where its sub-chunks of MGARD_SUB symbols 1..3 start, then
 * the chunk's escapes before each of them; a sub-chunk past the end of the
 * data starts at the chunk's end), outliers (escapes gathered in symbol order
 * from `escapes`, which is indexed by symbol position; capacity
 * `outliers_cap`).  A chunk whose symbols are all MGARD_DICT/2 (q = 0) is
 * stored with no words and zero sub-chunk offsets.
 * *nwords and *noutliers (host) receive the totals; synchronizes the
 * stream.  MGARD_ECAPACITY (totals still returned, nothing packed) if a
 * capacity is short; MGARD_EINVAL if a symbol has no code or `symbols` is
 * not 16-byte aligned (it is read with 16-byte vector loads). */
mgard_status mgard_huffman_encode(const uint16_t* symbols, uint64_t n, const uint8_t* lengths,
                                  const int32_t* escapes, uint32_t* words, uint64_t words_cap,
                                  uint64_t* word_off, uint64_t* esc_off, uint16_t* sub_off,
                                  int32_t* outliers, uint64_t outliers_cap, uint64_t* nwords,
                                  uint64_t* noutliers, void* stream);
/* Allocation-free variant of mgard_huffman_encode, for callers that cannot
 * allocate device memory (code running under an external memory manager, or
 * where cudaMalloc is not allowed).  The paper has no counterpart.  Same
 * arguments, results and errors as mgard_huffman_encode; it calls no
 * allocator.  Its scratch is a fixed device array of 90,704 bytes inside the
 * library, held by every device that loads the library until the process
 * exits.  Limits: n <= 2048 * 4096 * 1024 symbols (MGARD_EINVAL beyond).
 * Like mgard_huffman_encode it synchronizes the stream to return the totals.
 * The first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  All
 * calls share the array and it keeps the previous call's contents (the call
 * clears what must start at zero), so calls that overlap on the GPU -- on
 * different streams or threads -- race and must not be issued. */
mgard_status mgard_huffman_encode_noalloc(const uint16_t* symbols, uint64_t n,
                                          const uint8_t* lengths, const int32_t* escapes,
                                          uint32_t* words, uint64_t words_cap, uint64_t* word_off,
                                          uint64_t* esc_off, uint16_t* sub_off, int32_t* outliers,
                                          uint64_t outliers_cap, uint64_t* nwords,
                                          uint64_t* noutliers, void* stream);
/* Decode n symbols (device output) from a stream produced by
 * mgard_huffman_encode (every sub-chunk is decoded independently from its
 * recorded start); escapes[position] receives each outlier value.
 * Reads never leave the stream: a chunk that runs past its end or holds an
 * invalid code gives MGARD_ECORRUPT (synchronizes the stream).  `symbols`
 * must be 16-byte aligned (MGARD_EINVAL otherwise). */
mgard_status mgard_huffman_decode(const uint32_t* words, uint64_t nwords, const uint64_t* word_off,
                                  const uint64_t* esc_off, const uint16_t* sub_off,
                                  const uint8_t* lengths, uint64_t n, const int32_t* outliers,
                                  uint64_t noutliers, uint16_t* symbols, int32_t* escapes,
                                  void* stream);

/* ---- High-level API (Listing 1: compress / decompress) -----------------
 * Upper bound on the compressed size in bytes for a shape. */
size_t mgard_compress_bound(int ndim, const int64_t* shape, mgard_dtype dtype);

/* Compress `field` (host or device pointer; the location is detected).
 * tol > 0; s = INFINITY for L-infinity, else s >= 0 for the s-norm; mode
 * MGARD_REL scales tol by max|u| (L-infinity) or ||u||_s.
 * out_preallocated = 0: *out receives a new buffer (device memory if field
 * is on the device, host memory otherwise) to be released with mgard_free;
 * out_preallocated = 1: *out is the caller's buffer (host or device) of
 * *out_bytes capacity.  In both cases *out_bytes receives the size.
 * Synchronizes the stream before returning. */
mgard_status mgard_compress(const void* field, int ndim, const int64_t* shape, mgard_dtype dtype,
                            double tol, double s, mgard_tolmode mode, void** out,
                            size_t* out_bytes, int out_preallocated, void* stream);
/* Decompress a buffer made by mgard_compress or mgard_compress_regions
 * (host or device pointer).
 * out_preallocated = 0: *field receives a new buffer (device memory if the
 * compressed buffer is on the device) to be released with mgard_free;
 * = 1: *field is the caller's buffer (host or device), large enough for the
 * shape.  Header and section bounds are validated (MGARD_ECORRUPT).
 * Synchronizes the stream before returning. */
mgard_status mgard_decompress(const void* in, size_t in_bytes, void** field,
                              int out_preallocated, void* stream);
/* ---- Batched compression ---------------------------------------------------
 * Many fields or timesteps of possibly different shapes in one call; the
 * paper has no batched call, this serves workloads of many small fields,
 * where launch latency on the coarse levels would dominate.
 *   fields[i]   device pointer to field i (ndims[i], shapes[i], all `dtype`)
 *   outs[i]     device buffer of caps[i] bytes, 16-byte aligned; a buffer of
 *               mgard_compress_bound bytes always suffices
 *   out_bytes[i] (host) receives the compressed size of field i (the size
 *               needed when field i failed with MGARD_ECAPACITY)
 *   statuses[i] (host, may be NULL) receives the status of field i
 * tol, s, mode as for mgard_compress (one setting for the whole batch).
 * The fields run on internal streams forked from `stream` (and joined back
 * into it), so small fields overlap.  With MGARD_BATCH_GRAPH the whole batch
 * is captured into one CUDA graph the first time and replayed by later calls
 * with identical arguments (same pointers, shapes and settings); the
 * library keeps the graph and its workspaces until mgard_release_plans.
 * Every output is byte-identical to mgard_compress of the same field.
 * Synchronizes `stream` once, at the end.  Returns MGARD_OK when every
 * field succeeded, else the status of the first failing field. */
#define MGARD_BATCH_GRAPH 1
#define MGARD_BATCH_AUTOTUNE 2   /* run mgard_autotune on every new shape of the batch first */
#define MGARD_BATCH_REPEAT 4     /* capture and replay a graph once an identical call repeats */
/* Run the batch in phases with persistent multi-field launches: every
 * field's decomposition down to its small levels; one launch for all those
 * one-block tails (levels of at most a few thousand nodes); every field's
 * widths and quantization; one launch for all codebooks and decoding
 * tables; every field's encoding.  Each persistent launch is a grid of up
 * to one block per SM whose blocks take one field at a time from a device
 * counter.  Same bytes as without the flag. */
#define MGARD_BATCH_PERSISTENT 8
mgard_status mgard_compress_batch(int n, const void* const* fields, const int* ndims,
                                  const int64_t* const* shapes, mgard_dtype dtype, double tol,
                                  double s, mgard_tolmode mode, void* const* outs,
                                  const size_t* caps, size_t* out_bytes, mgard_status* statuses,
                                  int flags, void* stream);

/* Batched decompression of buffers made by mgard_compress /
 * mgard_compress_batch: ins[i] (device, in_bytes[i] bytes) into fields[i]
 * (device, field_caps[i] bytes, at least the field's size).  The headers
 * come to the host in one round trip; the buffers then decompress on
 * internal streams (MGARD_BATCH_GRAPH: from a captured graph, replayed for
 * identical arguments and headers; MGARD_BATCH_PERSISTENT, for buffers of
 * one dtype: every buffer decoded to level 0, one persistent launch for all
 * their small levels, then every buffer's larger levels; same results).
 * statuses[i] (host, may be NULL):
 * MGARD_ECORRUPT for a buffer that fails validation, MGARD_ECAPACITY for a
 * field buffer that is too small; the other buffers still decompress.
 * Synchronizes `stream`.  Returns MGARD_OK or the first failing status. */
mgard_status mgard_decompress_batch(int n, const void* const* ins, const size_t* in_bytes,
                                    void* const* fields, const size_t* field_caps,
                                    mgard_status* statuses, int flags, void* stream);

/* Autotuner: times every launch shape of the row kernels (elements per
 * lane per batch 2/4/8, grids sized for 4/8/16 blocks per SM) on each level
 * of `shape` and keeps the fastest for all later calls on that shape in
 * this process (kept in the shape's plan; mgard_release_plans forgets it).
 * Results are bit-identical for every launch shape.  `report` (may be
 * NULL) receives one line per level and kernel.  Synchronizes `stream`.
 * Shapes that run on the generic 4D kernels have nothing to tune. */
mgard_status mgard_autotune(int ndim, const int64_t* shape, mgard_dtype dtype, char* report,
                            size_t report_cap, void* stream);

/* ---- Ratio-targeted compression and the learned tolerance predictor -----
 * No counterpart in the paper.  A "sizer" decomposes a field once and then
 * gives the exact compressed size at any tolerance (quantization, codebook
 * and count pass; no packing), the predictor's features, and the final
 * compression, all from that one decomposition.  The field (device) must
 * stay unchanged while the sizer lives. */
typedef struct mgard_sizer_s mgard_sizer;
mgard_status mgard_sizer_create(const void* field, int ndim, const int64_t* shape,
                                mgard_dtype dtype, double s, mgard_sizer** out, void* stream);
/* Exact size in bytes of mgard_compress(field, tol, s, mode); synchronizes. */
mgard_status mgard_sizer_size(mgard_sizer* z, double tol, mgard_tolmode mode, size_t* bytes,
                              void* stream);
/* Predictor inputs (device, MGARD_NFEAT floats): per level, finest first
 * (at most 12 levels, missing ones zero): log10 of the coefficient count,
 * mean and standard deviation of r = log10(max(|c|, 1e-12 a) / a) with
 * a = max|u|, and the fractions of |c| below 10^(-j/2) a for j = 0..14;
 * then the number of active axes, L, log10 N and log10(target_ratio). */
#define MGARD_NFEAT 220
mgard_status mgard_sizer_features(mgard_sizer* z, double target_ratio, float* features,
                                  void* stream);
/* mgard_compress at `tol` from the sizer's decomposition into `out` (device,
 * 16-byte aligned, *out_bytes capacity in, size out). */
mgard_status mgard_sizer_compress(mgard_sizer* z, double tol, mgard_tolmode mode, void* out,
                                  size_t* out_bytes, void* stream);
void mgard_sizer_free(mgard_sizer* z);

/* Network: MGARD_NFEAT inputs standardized as (x - mean) / max(sd, 0.05)
 * -> 2 x MGARD_MLP_HIDDEN relu
 * units -> 1 output (log10 of the relative tolerance).  Parameters (device
 * floats): W1 [H, NFEAT] row-major, b1, W2 [H, H], b2, w3, b3 (the first
 * MGARD_MLP_NTRAIN, trained), then the inputs' mean and standard deviation. */
#define MGARD_MLP_HIDDEN 64
#define MGARD_MLP_NTRAIN (MGARD_MLP_HIDDEN * MGARD_NFEAT + \
                          MGARD_MLP_HIDDEN * MGARD_MLP_HIDDEN + 3 * MGARD_MLP_HIDDEN + 1)
#define MGARD_MLP_NPARAM (MGARD_MLP_NTRAIN + 2 * MGARD_NFEAT)
/* He-uniform weights from a counter-based generator (splitmix64), zero
 * biases, identity standardization. */
mgard_status mgard_mlp_init(float* params, uint64_t seed, void* stream);
/* Set the standardization to the mean / standard deviation of x [B, NFEAT]. */
mgard_status mgard_mlp_set_norm(float* params, const float* x, int B, void* stream);
/* y [B] = network(x [B, NFEAT]); all device pointers. */
mgard_status mgard_mlp_forward(const float* params, const float* x, int B, float* y,
                               void* stream);
/* Mean squared error over the batch and its gradient (MGARD_MLP_NTRAIN
 * floats) by backpropagation; loss may be NULL. */
mgard_status mgard_mlp_loss_grad(const float* params, const float* x, const float* t, int B,
                                 float* grad, float* loss, void* stream);
/* Adam (bias-corrected) on the first n parameters; t counts from 1. */
mgard_status mgard_adam_step(float* params, const float* grad, float* m, float* v, int n,
                             float lr, float beta1, float beta2, float eps, int t, void* stream);
/* `steps` full-batch steps of loss_grad + Adam(lr, 0.9, 0.999, 1e-8),
 * Adam's step counter continuing from t0; losses[k] (device, may be NULL)
 * receives the loss before step k. */
mgard_status mgard_mlp_train(float* params, float* m, float* v, const float* x, const float* t,
                             int B, int steps, int t0, float lr, float* losses, void* stream);

/* Compress `field` (device) with the relative tolerance whose compressed
 * size is within rel_err of field_bytes / target_ratio.  With params
 * (device, MGARD_MLP_NPARAM) the network proposes the tolerance and a
 * bracketed bisection on log10(tol) corrects it if needed; with params =
 * NULL the bisection starts from [1e-7, 1].  Every probe is an exact
 * size from one shared decomposition; *passes counts them.  The error
 * bound of the chosen tolerance holds as for mgard_compress: the target
 * only selects tol.  *tol_used receives it; out (device, 16-byte aligned)
 * gets the buffer (*out_bytes: capacity in, size out).  When no tolerance
 * in [1e-9, 1] reaches the target within rel_err, the closest probe is used
 * and MGARD_OK is still returned (check the size). */
mgard_status mgard_compress_to_ratio(const void* field, int ndim, const int64_t* shape,
                                     mgard_dtype dtype, double target_ratio, double s,
                                     const float* params, double rel_err, double* tol_used,
                                     void* out, size_t* out_bytes, int* passes, void* stream);

/* Read the header of a compressed buffer (host or device pointer). */
mgard_status mgard_info(const void* in, size_t in_bytes, int* ndim, int64_t shape[4],
                        mgard_dtype* dtype, double* tol_abs, int* nlevels);
/* ---- Refactoring: progressive retrieval ----------------------------------
 * Paper: "Software design" (the refactoring pipeline: the multilevel
 * coefficients are encoded into precision segments, an error estimate is
 * kept per segment, and retrieval picks segments greedily until the
 * requested error is met) and "APIs" (MDRefactor, MDRequest, MDReconstruct).
 *
 * A refactored buffer is an mgard_mdr_header followed, for every level l
 * (l = 0 the coarsest), by the level's sign plane and its `planes` magnitude
 * planes (plane 0 the most significant), each level[l].words uint32 words,
 * starting at byte level[l].offset (16-byte aligned).  The coefficients of a
 * level are in level order (level 0's nodes, then the nodes new on each
 * level, row-major in the level grid); coefficient 32 w + i sits in bit i of
 * word w.  Plane b holds bit planes-1-b of q = floor(|c| 2^(planes -
 * exponent)); the sign plane holds c < 0.  Reading P planes of a level
 * reconstructs every coefficient within 2^(exponent - P) (0 when q's first P
 * bits are 0, else the middle of the truncation interval).  The L-infinity
 * error of the recomposed field is then at most sum_l weight_l
 * 2^(exponent_l - P_l) in exact arithmetic (weight_0 = 1, weight_l = c_l of
 * the compressor's L-infinity bound; all-zero levels count 0); the float
 * arithmetic of decomposition and recomposition adds its own rounding.
 * Grids of up to three active axes (MGARD_ESHAPE otherwise). */
#define MGARD_MDR_MAX_LEVELS 64
typedef struct {
    uint64_t count;      /* coefficients of the level */
    uint64_t offset;     /* byte offset of the level's sign plane in the buffer */
    uint32_t words;      /* words per plane: ceil(count / 32) */
    int32_t exponent;    /* every |c| < 2^exponent (0 for an all-zero level) */
    uint32_t nonzero;    /* 0 if every coefficient of the level is 0 */
    uint32_t reserved;
    double weight;       /* weight of the level's errors in the estimate */
} mgard_mdr_level;

typedef struct {
    char magic[8];       /* "MGARDMDR" */
    uint32_t version;    /* 1 */
    uint32_t dtype;      /* mgard_dtype of the field */
    uint32_t ndim;
    uint32_t nlevels;    /* L + 1 */
    uint32_t planes;     /* magnitude planes per level, 1..32 */
    uint32_t reserved;
    int64_t shape[4];
    double max_abs;      /* max |u| of the refactored field */
    uint64_t total_bytes;
    mgard_mdr_level level[MGARD_MDR_MAX_LEVELS + 1];
} mgard_mdr_header;

/* Bytes of a refactored buffer of this shape at most. */
size_t mgard_refactor_bound(int ndim, const int64_t* shape, int planes);
/* MDRefactor: decompose `field` (device) and write the header and every
 * level's sign and magnitude planes to `out` (device, 16-byte aligned;
 * *out_bytes: capacity in, size out; MGARD_ECAPACITY with the size if
 * short).  planes in 1..32.  MGARD_ENONFINITE for NaN/Inf input.
 * Synchronizes the stream. */
mgard_status mgard_refactor(const void* field, int ndim, const int64_t* shape, mgard_dtype dtype,
                            int planes, void* out, size_t* out_bytes, void* stream);
/* MDRequest (host only): the planes to read per level (planes_per_level,
 * host array of header->nlevels) for an absolute L-infinity tolerance,
 * chosen greedily: while the estimate exceeds tol, add the next plane of
 * the level whose plane lowers the estimate most per byte (the first plane
 * of a level also costs its sign plane; ties to the lower level).  *bytes
 * receives the size of the selected planes, *estimate the estimate.  If
 * every plane is selected and the estimate still exceeds tol, all planes
 * are returned with MGARD_EBOUND. */
mgard_status mgard_request(const mgard_mdr_header* header, double tol, int32_t* planes_per_level,
                           uint64_t* bytes, double* estimate);
/* MDReconstruct: decode planes_per_level[l] planes of every level from
 * `refactored` (device; only the header and the selected planes are read)
 * and recompose into `field` (device, the header's shape and dtype).
 * Synchronizes the stream. */
mgard_status mgard_reconstruct(const void* refactored, const int32_t* planes_per_level,
                               void* field, void* stream);

/* ---- Linear quantities of interest ("Software design": guarantees on
 * quantities derived from the data; "Application impact", plasma physics) -
 * A linear QoI is Q(v) = sum_p g_p v_p with FP64 weights g: device memory,
 * one weight per grid node, row-major in the field's shape.  Its
 * representer is the P1 function r with M_L r = g (M_L the finest grid's
 * mass matrix, unit spacing), so Q(e) = <r, e>_{L2}; splitting both over the
 * level spaces (Q_l - Q_{l-1}) V_L gives |Q(e)| <= ||Q||_{-s} ||e||_s with
 * ||Q||_{-s} = ||r||_{-s}, the s-norm with -s in place of s.  For
 * s = INFINITY the dual norm is ||g||_1 (|Q(e)| <= ||g||_1 max|e|).
 * MGARD_ENONFINITE when g holds NaN or Inf. */

/* r = M_L^{-1} g (device, N doubles; r may equal g): one FP64 tridiagonal
 * solve per line along every active axis.  Stream-ordered after a check of
 * the weights (which synchronizes). */
mgard_status mgard_qoi_representer(const double* g, int ndim, const int64_t* shape, double* r,
                                   void* stream);
/* *norm = ||Q||_{-s} (host) on the hierarchy of max_levels levels (-1: all,
 * as mgard_compress uses); s >= 0 or INFINITY, else MGARD_EINVAL.  The
 * representer's level energies come from the FP64 decomposition.
 * Synchronizes the stream. */
mgard_status mgard_qoi_norm(const double* g, int ndim, const int64_t* shape, int max_levels,
                            double s, double* norm, void* stream);
/* *value = Q(field) = sum_p g_p field_p accumulated in FP64 in a fixed
 * order (field: device, dtype).  Synchronizes the stream. */
mgard_status mgard_qoi_value(const void* field, const double* g, int ndim, const int64_t* shape,
                             mgard_dtype dtype, double* value, void* stream);
/* Compress so that |Q(decompress(out)) - Q(field)| <= tol_qoi: mgard_compress
 * with the absolute s-norm tolerance tol_qoi / ||Q||_{-s} (written to
 * *tol_used when non-null).  field, out, out_bytes, out_preallocated and the
 * ownership of the output are those of mgard_compress; g is device memory.
 * MGARD_EINVAL for tol_qoi <= 0, s < 0 or weights that are all zero. */
mgard_status mgard_compress_qoi(const void* field, int ndim, const int64_t* shape,
                                mgard_dtype dtype, const double* g, double tol_qoi, double s,
                                void** out, size_t* out_bytes, int out_preallocated,
                                double* tol_used, void* stream);

/* ---- Region-adaptive error bounds ("Application impact", Earth and
 * cosmological science: tighter errors kept in chosen regions) ----------
 * A box is an inclusive index range per axis of the field's shape as passed
 * (entries beyond ndim ignored) with its own absolute tolerance tol, at
 * most the background tolerance.  The compressed field then satisfies
 * |u~(p) - u(p)| <= the smallest tol of the boxes holding p, and <= the
 * background tolerance everywhere (L-infinity).
 *
 * Rule (rigorous, from the recomposition's error propagation): a node
 * first appearing on level l gets the bin width w 2^-k, w the uniform
 * L-infinity width of the background tolerance and k the largest k_r of the
 * boxes whose dilation on level l contains it (0 if none).  Dilation along
 * an axis: H_0 on level 0 and (rho + 1) H_l + H_{l-1} above, H_l the largest
 * spacing of level-l nodes.  rho is the smallest radius (0..48) at which the
 * far-field rows of the correction operators M_{l-1}^{-1} P^T M_l, weighted
 * by the background width, cost at most 1/8 of the tightest box's
 * tolerance; k_r the smallest k with 2^-k tol <= tol_r - that far-field
 * error.  Scaling a coefficient by 2^k is exact, so the compressor scales
 * and quantizes with w, and the decompressor scales back. */
#define MGARD_MAX_REGIONS 8
typedef struct {
    int64_t lo[4];
    int64_t hi[4];
    double tol;
} mgard_region;

/* Host only: the radius rho and every box's exponent k_r (nregions
 * entries) for these boxes and background tolerance tol.  MGARD_EINVAL for
 * more than 8 boxes, boxes outside the field, box tolerances outside
 * (0, tol] or too small to reach (k above 60); MGARD_ESHAPE for a grid
 * without levels. */
mgard_status mgard_region_plan(int ndim, const int64_t* shape, double tol,
                               const mgard_region* regions, int nregions, int* rho, int32_t* k);
/* The exponent k of every node (device, N bytes, row-major).  Synchronizes. */
mgard_status mgard_region_exponents(int ndim, const int64_t* shape, double tol,
                                    const mgard_region* regions, int nregions, uint8_t* k,
                                    void* stream);
/* Compress with region-adaptive bounds: background tolerance tol
 * (absolute, L-infinity) and the boxes.  The output (format in
 * include/mgard_format.h: a region header, then an ordinary buffer) is
 * self-describing; mgard_decompress and mgard_info read it.  field, out,
 * out_bytes, out_preallocated and ownership as mgard_compress. */
mgard_status mgard_compress_regions(const void* field, int ndim, const int64_t* shape,
                                    mgard_dtype dtype, double tol, const mgard_region* regions,
                                    int nregions, void** out, size_t* out_bytes,
                                    int out_preallocated, void* stream);

/* ---- Out-of-core compression ("Software architecture": the out-of-core
 * module that chunks arrays to fit device memory) ------------------------
 * A host field (pinned memory gives full overlap of the PCIe copies with
 * the kernels; pageable memory works too) is cut along its first axis into
 * nblocks blocks of as equal sizes as possible (1 <= nblocks <= shape[0]);
 * every block is compressed independently with the L-infinity bound (ABS,
 * or REL against max|u| of the whole field from a first streaming pass), so
 * the whole field keeps it.  Two internal streams alternate over the blocks:
 * one block's kernels run while the next block's host-to-device copy and
 * the previous block's device-to-host copy proceed.  Device memory: about
 * two blocks' input, output and workspace, independent of the field size.
 * Format: include/mgard_format.h (mgard_ooc_header, block offsets, then one
 * ordinary buffer per block).  mgard_decompress (host buffer, host field)
 * and mgard_info read it; decompression is pipelined the same way. */

/* Bytes an out-of-core buffer of this shape can need at most. */
size_t mgard_compress_ooc_bound(int ndim, const int64_t* shape, mgard_dtype dtype,
                                int64_t nblocks);
/* field and *out are host memory.  out_preallocated = 0: *out receives a
 * malloc'd buffer (release with mgard_free); = 1: *out_bytes is the
 * capacity (MGARD_ECAPACITY with the size needed when short).  MGARD_EINVAL
 * for device pointers or bad block counts.  Synchronizes the stream. */
mgard_status mgard_compress_ooc(const void* field, int ndim, const int64_t* shape,
                                mgard_dtype dtype, double tol, mgard_tolmode mode,
                                int64_t nblocks, void** out, size_t* out_bytes,
                                int out_preallocated, void* stream);

/* ---- Tracing -------------------------------------------------------------
 * When enabled, every kernel launch of the library is bracketed by a pair
 * of CUDA events recorded on its launch stream (adds about a microsecond
 * per launch; off by default). */
void mgard_timing_enable(int on);
/* Waits for the recorded events and writes one line per kernel,
 * "name launches total_ms", into buf (capacity cap, NUL-terminated) and
 * clears the records.  Returns the size the full report needs; with
 * buf = NULL only the size is returned and the records are kept. */
size_t mgard_timing_report(char* buf, size_t cap);

/* Release a buffer allocated by this library (host or device). */
void mgard_free(void* p);
/* Drop cached per-shape tables. */
void mgard_release_plans(void);

#ifdef __cplusplus
}
#endif
#endif /* MGARD_B300_H */
