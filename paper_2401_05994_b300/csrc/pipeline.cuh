// Compression pipeline that runs entirely in stream order on the device
// (declarations).  Every value that depends on the data -- the norm behind a
// relative tolerance, the bin widths, the payload size and the section
// offsets that follow from it -- is computed and consumed on the device, so
// a whole compression is one stream of launches with no host round trip and
// can be captured in a CUDA graph (batched compression uses that).
#pragma once

#include <string>

#include "../../include/mgard_format.h"
#include "multilevel.cuh"
#include "huffman.cuh"
#include "quantize.cuh"

namespace mgb {

// Byte offsets of the sections after the header (include/mgard_format.h).
struct Sections {
    size_t widths, lengths, word_off, esc_off, sub_off, outliers, words, total;
};
Sections layout(int L, uint64_t nchunks, uint64_t nout, uint64_t nwords);

// Results of one compression, written by the device.
struct CompressMeta {
    unsigned long long total;       // bytes of the compressed buffer
    unsigned long long off_words;   // byte offset of the payload
    unsigned long long nwords, noutliers;
    double tol_abs;
    unsigned status;                // ST_* bits; ST_CAPACITY if the buffer is too small
    unsigned pad;
};

// Device workspace of one compression, sized for one plan.  Allocated from
// the library's pool before any capture and reused by every run.
template <typename T>
struct CompressWork {
    Pyramid<T> py;
    DevBuf top, sym, esc, hist, lengths, codes, dt, offs, totals, parts, scan, wdev;
    mgard_status alloc(const Plan& p, cudaStream_t st);
};

// The header fields known on the host before the run.
mgard_header header_template(const Plan& p, mgard_dtype dtype, int ndim, const int64_t* shape,
                             double tol, double s, mgard_tolmode mode);

// Compress `din` (device, the plan's shape) into `dd` (device, 16-byte
// aligned, `cap` bytes, cap >= layout(L, nchunks, 0, 0).outliers).  Only
// launches and device-to-device copies on `st`: the caller reads `*meta`
// after the stream has reached this point.  When the data does not fit in
// `cap` bytes, meta->status has ST_CAPACITY, meta->total the size needed and
// the payload is not written.
// With `rs`, region-adaptive widths (quantize.cuh): the coefficients are
// scaled by 2^k of their node between decomposition and quantization.
// A second stream beside the caller's and the events that fork work onto
// it and join it back.  With one, compression runs the small levels'
// one-block tail beside the larger levels' quantization instead of before
// it; graph capture records the fork and the join as edges.  Null:
// everything on the caller's stream.
struct AuxLane {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, mid = nullptr, join = nullptr;
};

template <typename T>
mgard_status compress_core(const Plan& p, const T* din, const mgard_header& h0, double tol,
                           double s, mgard_tolmode mode, char* dd, uint64_t cap,
                           CompressWork<T>& w, CompressMeta* meta, cudaStream_t st,
                           const RegionScale* rs = nullptr, const AuxLane* aux = nullptr);

// Map device status bits (ST_*) to an mgard_status with its message.
mgard_status status_to_error(unsigned st);

// Host validation of a header read from a buffer of in_bytes bytes
// (magic, version, sizes and section offsets); MGARD_ECORRUPT on failure.
mgard_status check_header(const mgard_header& h, size_t in_bytes);
bool widths_valid(const double* w, int L);

// Device workspace of one decompression.
template <typename T>
struct DecompressWork {
    Pyramid<T> py;
    DevBuf codes, dt, sym, esc, zs;   // zs (row-kernel shapes) or sym + esc
    DevBuf grab;                      // the decoder's work counter
    mgard_status alloc(const Plan& p, cudaStream_t st);
};

// Decompress the device image `din` (header h and widths w validated on
// the host) into `dout` (device).  Launches only; a corrupt stream ORs
// ST_CORRUPT into *status (device) and leaves `dout` meaningless but every
// access in bounds.
// With `rs`, the dequantized coefficients are scaled back by 2^-k.
template <typename T>
mgard_status decompress_core(const Plan& p, const mgard_header& h, const double* w,
                             const char* din, T* dout, DecompressWork<T>& work, unsigned* status,
                             cudaStream_t st, const RegionScale* rs = nullptr);

// Time every launch shape of the row kernels on each level of the plan's
// shape and keep the fastest in the plan (tune.cu); `report` receives one
// line per level and kernel.
mgard_status autotune_plan(const Plan& p, mgard_dtype dtype, cudaStream_t st, std::string* report);

// The three phases of compress_core, for callers that encode one
// decomposition at several tolerances (ratio targeting):
//  decompose  norm partials (max|u|, level energies) and the decomposition
//             into the workspace; resets *meta;
//  encode     widths, quantization, codebook and the count pass: *meta gets
//             the exact compressed size; with dd != null the header is
//             written and ST_CAPACITY reflects `cap`;
//  pack       the remaining sections and the payload into dd.
template <typename T>
mgard_status compress_decompose(const Plan& p, const T* din, double s, mgard_tolmode mode,
                                CompressWork<T>& w, CompressMeta* meta, cudaStream_t st);
template <typename T>
mgard_status compress_encode(const Plan& p, const T* din, const mgard_header& h0, double tol,
                             double s, mgard_tolmode mode, char* dd, uint64_t cap,
                             CompressWork<T>& w, CompressMeta* meta, cudaStream_t st);
template <typename T>
mgard_status compress_pack(const Plan& p, char* dd, CompressWork<T>& w, CompressMeta* meta,
                           cudaStream_t st);
// compress_encode in three parts, for batches that build the codebooks of
// all fields in one launch (huffman_codebook_tables_batch on the jobs of
// codebook_job): front = widths and quantization, back = count pass and
// header.  front, the codebook and tables, then back equal compress_encode.
// With quantize false, front stops after the widths.
template <typename T>
mgard_status compress_encode_front(const Plan& p, const T* din, double tol, double s,
                                   mgard_tolmode mode, CompressWork<T>& w, CompressMeta* meta,
                                   cudaStream_t st, bool quantize = true);
template <typename T>
CodebookJob codebook_job(const Plan& p, CompressWork<T>& w);
template <typename T>
mgard_status compress_encode_back(const Plan& p, const mgard_header& h0, char* dd, uint64_t cap,
                                  CompressWork<T>& w, CompressMeta* meta, cudaStream_t st);

// Out-of-core buffers (ooc.cu), read by mgard_decompress and mgard_info on
// host memory.
bool is_ooc_buffer(const void* in, size_t in_bytes);
mgard_status ooc_info(const void* in, size_t in_bytes, mgard_ooc_header* h);
mgard_status decompress_ooc(const void* in, size_t in_bytes, void** field, int prealloc,
                            cudaStream_t st);

// Drop the cached batches of mgard_compress_batch / mgard_decompress_batch
// (graphs and workspaces).
void release_batches();
void release_decompress_batches();

}  // namespace mgb
