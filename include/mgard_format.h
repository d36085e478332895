/*
 * mgard_format.h -- layout of the self-describing compressed buffer.
 *
 * The paper ("APIs", high-level features) asks for output that carries
 * everything a decompressor needs: version, error bounds, data topology and
 * encoder.  This build stores, little-endian:
 *
 *   mgard_header                      (fixed size, below)
 *   widths    [nlevels + 1] double    bin width of each level
 *   lengths   [dict] uint8            Huffman code length per symbol
 *   word_off  [nchunks] uint64        exclusive prefix of words per chunk
 *   esc_off   [nchunks] uint64        exclusive prefix of escapes per chunk
 *   sub_off   [nchunks][6] uint16     per chunk: bit offsets (inside the chunk) of
 *                                     its sub-chunks 1..3 (256 symbols each), then the
 *                                     escapes of the chunk before each of them
 *   outliers  [noutliers] int32       escaped quantized values, symbol order
 *   words     [nwords] uint32         Huffman payload; a chunk of no words holds
 *                                     only the symbol of q = 0 (MGARD_DICT/2)
 *
 * Every section starts at the byte offset recorded in the header, a
 * multiple of 16.  Decompression rejects a buffer whose magic, version,
 * sizes or offsets are inconsistent (MGARD_ECORRUPT).
 */
#ifndef MGARD_FORMAT_H
#define MGARD_FORMAT_H

#include <stdint.h>

#define MGARD_MAGIC "MGARDB3"
#define MGARD_FORMAT_VERSION 2u

typedef struct {
    char magic[8];        /* "MGARDB3\0" */
    uint32_t version;     /* MGARD_FORMAT_VERSION */
    uint32_t dtype;       /* mgard_dtype */
    uint32_t ndim;        /* as passed to compress */
    uint32_t nlevels;     /* L */
    int64_t shape[4];     /* as passed to compress; unused entries 1 */
    double s;             /* smoothness; +infinity for L-infinity */
    double tol;           /* requested tolerance */
    double tol_abs;       /* absolute tolerance the widths were derived from */
    uint32_t mode;        /* mgard_tolmode */
    uint32_t dict;        /* dictionary size (MGARD_DICT) */
    uint32_t chunk;       /* symbols per chunk (MGARD_CHUNK) */
    uint32_t reserved;
    uint64_t nsymbols;    /* product of the extents */
    uint64_t nchunks;
    uint64_t nwords;
    uint64_t noutliers;
    uint64_t off_widths;
    uint64_t off_lengths;
    uint64_t off_word_off;
    uint64_t off_esc_off;
    uint64_t off_sub_off;
    uint64_t off_outliers;
    uint64_t off_words;
    uint64_t total_bytes;
} mgard_header;

/*
 * Region-adaptive buffers (mgard_compress_regions) wrap an ordinary buffer:
 *
 *   mgard_region_header               (fixed size, below)
 *   inner     [inner_bytes]           an mgard_compress buffer (L-infinity,
 *                                     absolute tolerance = the background
 *                                     tolerance) at byte MGARD_REGION_INNER
 *
 * whose coefficients were scaled by 2^k of their node before quantization
 * (k from the boxes, rho and k below, dilated per level as
 * include/mgard_b300.h describes); decompression scales them back.
 */
#define MGARD_REGION_MAGIC "MGARDRG"
#define MGARD_REGION_VERSION 1u
#define MGARD_REGION_SLOTS 8

typedef struct {
    char magic[8];        /* "MGARDRG\0" */
    uint32_t version;     /* MGARD_REGION_VERSION */
    uint32_t nregions;    /* 0 .. MGARD_REGION_SLOTS */
    int32_t rho;          /* radius of the near field, level-l nodes */
    int32_t k[MGARD_REGION_SLOTS];   /* width exponent of every box */
    uint32_t reserved;
    double tol;           /* background tolerance (absolute) */
    struct {
        int64_t lo[4], hi[4];   /* inclusive index box, axes as passed */
        double tol;
    } box[MGARD_REGION_SLOTS];
    uint64_t inner_bytes;
} mgard_region_header;

#define MGARD_REGION_INNER ((sizeof(mgard_region_header) + 15) & ~(size_t)15)

/*
 * Out-of-core buffers (mgard_compress_ooc) hold independent blocks of the
 * field along its first axis:
 *
 *   mgard_ooc_header                  (fixed size, below)
 *   offsets   [nblocks + 1] uint64    byte offset of every block's buffer
 *                                     (16-byte aligned; the last entry is
 *                                     total_bytes)
 *   blocks                            one mgard_compress buffer per block
 *                                     (L-infinity, absolute tolerance tol_abs)
 *
 * Block b covers first-axis indices [b q + min(b, r), (b + 1) q + min(b + 1, r))
 * with q = shape[0] / nblocks and r = shape[0] % nblocks.
 */
#define MGARD_OOC_MAGIC "MGARDOC"
#define MGARD_OOC_VERSION 1u

typedef struct {
    char magic[8];        /* "MGARDOC\0" */
    uint32_t version;     /* MGARD_OOC_VERSION */
    uint32_t dtype;
    uint32_t ndim;
    uint32_t nblocks;
    int64_t shape[4];
    double tol;           /* requested tolerance */
    double tol_abs;       /* absolute L-infinity tolerance of every block */
    uint32_t mode;        /* mgard_tolmode of tol */
    uint32_t reserved;
    uint64_t total_bytes;
} mgard_ooc_header;

#endif /* MGARD_FORMAT_H */
