// Huffman codebook, encoder and decoder (declarations).
#pragma once

#include <cstddef>

#include "common.cuh"

namespace mgb {

constexpr int LUT_BITS = 14;
// A chunk made only of this symbol (q = 0) is stored with no payload words.
constexpr unsigned FILL_SYMBOL = MGARD_DICT / 2;
constexpr unsigned FILL_PAIR = FILL_SYMBOL | (FILL_SYMBOL << 16);
constexpr int SUB = 256;                 // symbols per independently decodable sub-chunk
constexpr int NSUB = MGARD_CHUNK / SUB;  // sub-chunks per chunk
constexpr int SUBREC = 2 * (NSUB - 1);   // uint16 offsets recorded per chunk

struct DecodeTables {
    // 14-bit prefix -> (length << 12) | symbol for codes of at most 14 bits;
    // (15 << 12) | L when every code under the prefix is longer and all have
    // the same length L; 0 otherwise (longer codes of several lengths, or no
    // code has the prefix)
    uint16_t lut[1 << LUT_BITS];
    unsigned long long lim[LMAX + 2];   // lim[l]: first code of length l+1, left-justified in 32 bits
    uint32_t first_code[LMAX + 2];
    uint32_t first_index[LMAX + 2];
    uint16_t sorted[DICT];              // used symbols in (length, symbol) order
    uint32_t maxlen;
    uint32_t valid;                     // 0 if the lengths violate the Kraft inequality
};
// the decoder copies lut and sorted in 16-byte units
static_assert(offsetof(DecodeTables, sorted) % 16 == 0, "sorted must stay 16-byte aligned");

// One-time per-device setup of the kernels (launch attributes); called by
// huffman_codebook and, before any stream capture, by batched compression.
mgard_status huffman_prepare();
// Code lengths from a histogram (single CTA).  `wide` selects 64-bit merge
// weights (needed when the histogram totals 2^32 symbols or more).
mgard_status huffman_codebook(const unsigned long long* hist, uint8_t* lengths, uint32_t* codes,
                              cudaStream_t st, bool wide = true);
// Canonical codes and decode tables from code lengths (single CTA); with
// dt null only the codes.
mgard_status huffman_tables(const uint8_t* lengths, uint32_t* codes, DecodeTables* dt,
                            cudaStream_t st);
// Codebooks and tables of n fields in one launch: a persistent grid (up to
// one block per SM) whose blocks take jobs from *counter (device; reset
// here, stream-ordered).  Results equal huffman_codebook + huffman_tables
// of every job.
struct CodebookJob {
    const unsigned long long* hist;
    uint8_t* lengths;
    uint32_t* codes;
    DecodeTables* dt;
    int wide;
};
mgard_status huffman_codebook_tables_batch(const CodebookJob* jobs, int n, unsigned* counter,
                                           cudaStream_t st);
// Pass 1 of encoding: per-chunk word and escape counts and their exclusive
// prefixes; totals (device, 2 x uint64) receive total words / escapes.
// `scratch` (device, count_scratch_bytes(n)) may be null: then it is
// allocated from the workspace pool.
mgard_status huffman_count(const uint16_t* sym, uint64_t n, const uint8_t* lengths,
                           uint64_t* word_off, uint64_t* esc_off, unsigned long long* totals,
                           unsigned* status, cudaStream_t st,
                           unsigned long long* scratch = nullptr);
size_t count_scratch_bytes(uint64_t n);

// Device-side conditions of the pack pass (both optional): it writes nothing
// when *status is non-zero, and the payload starts *words_byte_off bytes
// after `words` (an offset known only on the device).
struct PackGuard {
    const unsigned* status = nullptr;
    const unsigned long long* words_byte_off = nullptr;
};
// Pass 2: pack codes, record sub-chunk offsets and gather escapes.  The
// escape values are indexed by symbol position, or with `compact` stored per
// sub-chunk in order (escapes[s * 256 + r] for the r-th escape of sub-chunk s).
mgard_status huffman_pack(const uint16_t* sym, uint64_t n, const uint8_t* lengths,
                          const uint32_t* codes, const uint64_t* word_off, const uint64_t* esc_off,
                          const int32_t* escapes, uint32_t* words, uint16_t* sub_off,
                          int32_t* outliers, cudaStream_t st, PackGuard guard = PackGuard(),
                          bool compact = false);
// Widths for decoding straight to dequantized values: level l's symbols
// [lo.off[l], lo.off[l+1]) dequantize with w[l] (wf[l] = float(w[l])).
struct DeqArgs {
    LevelOffsets lo;
    double w[MAX_LEVELS + 1];
    float wf[MAX_LEVELS + 1];
    WidthSplit ws[MAX_LEVELS + 1];   // split_width(w[l])
};
// Decoding with bounds checks (ST_CORRUPT on failure).
mgard_status huffman_decode(const uint32_t* words, uint64_t nwords, const uint64_t* word_off,
                            const uint16_t* sub_off, const DecodeTables* dt, uint64_t n,
                            const int32_t* outliers, uint64_t noutliers, const uint64_t* esc_off,
                            uint16_t* sym, int32_t* escapes, unsigned* status, cudaStream_t st);

// Decoding straight to dequantized coefficients in symbol order (vals, n
// values), as the dequantization of the decoded symbols would give them.
// grab (device, 8 bytes; reset here): warps take runs of sub-chunks from
// it, so the launch ends when the work does rather than when its slowest
// block does; null: a fixed assignment in grid order.
template <typename T>
mgard_status huffman_decode_values(const uint32_t* words, uint64_t nwords, const uint64_t* word_off,
                                   const uint16_t* sub_off, const DecodeTables* dt, uint64_t n,
                                   const int32_t* outliers, uint64_t noutliers,
                                   const uint64_t* esc_off, const DeqArgs& dq, T* vals,
                                   unsigned* status, cudaStream_t st,
                                   unsigned long long* grab = nullptr);

}  // namespace mgb
