// Level-wise quantization (declarations).
#pragma once

#include "plan.cuh"

namespace mgb {

// Quantize the level-l coefficients of `c` (compact level array when
// inplace = false, the whole in-place array otherwise) with the bin width
// *w (device memory, so widths computed on the device need no round trip);
// accumulates into `hist` (DICT counters) and ORs ST_* bits into status.
template <typename T>
mgard_status quantize_level(const Plan& p, int l, const T* c, bool inplace, const double* w,
                            uint16_t* sym, int32_t* esc, unsigned long long* hist,
                            unsigned* status, cudaStream_t st);

// Inverse; writes 0 on the positions of coarser nodes in a compact level
// array and leaves them untouched in the in-place layout.
template <typename T>
mgard_status dequantize_level(const Plan& p, int l, const uint16_t* sym, const int32_t* esc,
                              bool inplace, double w, T* c, cudaStream_t st);

// Quantization of all levels' coefficients held in symbol order (zs, N
// values; w: device widths of levels 0..L).  Same symbols, escape values and
// histogram as quantize_level over the levels, but the escapes are stored
// compacted per Huffman sub-chunk: the r-th escape of sub-chunk s at
// esc[s * (MGARD_CHUNK / MGARD_NSUB) + r] (huffman_pack's `compact` layout).
LevelOffsets level_offsets(const Plan& p);
template <typename T>
mgard_status quantize_stream(const Plan& p, const T* zs, const double* w, uint16_t* sym,
                             int32_t* esc, unsigned long long* hist, unsigned* status,
                             cudaStream_t st);

// Statistics of the level-l coefficients (the features of the tolerance
// predictor): feature_blocks(p, l) FeatPart records, reduced in a fixed
// order by the caller.  amax: device max|u|.  `c`: for shapes on the row
// kernels the level's run of coefficients in symbol order, otherwise its
// compact level array.
int64_t feature_blocks(const Plan& p, int l);
template <typename T>
mgard_status level_features(const Plan& p, int l, const T* c, const double* amax, FeatPart* part,
                            cudaStream_t st);

}  // namespace mgb
