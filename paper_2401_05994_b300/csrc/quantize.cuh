// Level-wise quantization (declarations).
#pragma once

#include <vector>

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
// With i_begin / i_end (i_begin a multiple of the sub-chunk size, 256), only
// symbols [i_begin, i_end) are quantized (the histogram accumulates); with
// spare_sm the grid leaves one SM's worth of blocks free for a kernel
// running beside it.
template <typename T>
mgard_status quantize_stream(const Plan& p, const T* zs, const double* w, uint16_t* sym,
                             int32_t* esc, unsigned long long* hist, unsigned* status,
                             cudaStream_t st, int64_t i_begin = 0, int64_t i_end = -1,
                             bool spare_sm = false);

// Statistics of the level-l coefficients (the features of the tolerance
// predictor): feature_blocks(p, l) FeatPart records, reduced in a fixed
// order by the caller.  amax: device max|u|.  `c`: for shapes on the row
// kernels the level's run of coefficients in symbol order, otherwise its
// compact level array.
int64_t feature_blocks(const Plan& p, int l);
template <typename T>
mgard_status level_features(const Plan& p, int l, const T* c, const double* amax, FeatPart* part,
                            cudaStream_t st);

// Region-adaptive widths: on level l a node at input-grid position g (4D
// view) takes the width w_l 2^-k with k the largest k[r] of the boxes
// lo[r] <= g <= hi[r] (boxes already dilated for that level), 0 if none.
// The compressor scales such a coefficient by 2^k before quantizing with
// w_l (the same integer, exactly) and the decompressor by 2^-k after
// dequantizing.
constexpr int REGION_MAX = 8;
struct RegionLevel {
    int n;
    int k[REGION_MAX];
    int64_t lo[REGION_MAX][4], hi[REGION_MAX][4];
};
struct RegionScale {
    std::vector<RegionLevel> lv;   // [l], l = 0..L
};
// Multiply every level's coefficients by 2^(sign k): zs (symbol order, all
// levels) when non-null, else the compact level arrays levels[l] (l = 0..L).
template <typename T>
mgard_status region_scale(const Plan& p, const RegionScale& rs, T* zs, T* const* levels, int sign,
                          cudaStream_t st);
// The exponent k of every node of the input grid (row-major, N bytes).
mgard_status region_exponents(const Plan& p, const RegionScale& rs, uint8_t* k, cudaStream_t st);

}  // namespace mgb
