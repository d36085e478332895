// Huffman coding of quantization symbols.
//
// Paper, "Software design": the quantized coefficients are losslessly
// encoded into the self-describing buffer.  This build's coder:
//  * code lengths: leaves (used symbols) sorted by (count, symbol), merged
//    with two FIFO queues (leaf queue first on equal weight); depth = length;
//    lengths over LMAX repeat on max(1, count >> k); one used symbol -> 1 bit;
//  * canonical codes, consecutive in (length, symbol) order;
//  * chunks of CHUNK symbols, each starting on a 32-bit word, MSB-first.
// The codebook is built by one CTA: a sort of the leaves (warp bitonic
// networks on runs of 32, then merge passes), the queue merge in doubling
// rounds (see round_merge) and depths by pointer jumping.
// Encoding is a count pass, an exclusive scan over chunks and a pack pass
// with one warp per chunk (a shared-memory buffer of one round's words).
// Decoding runs one thread per 256-symbol sub-chunk with a 14-bit prefix
// table in shared memory and a canonical first-code search for longer codes.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>

#include <type_traits>

#include "huffman.cuh"
#include "multilevel.cuh"

namespace mgb {

namespace {

constexpr int CB_THREADS = 1024;
constexpr unsigned long long KEY_NONE = ~0ull;

// Ascending sort of DICT 64-bit keys by the whole block (a multiple of 32
// threads): every warp sorts runs of 32 keys in registers with a shuffle
// bitonic network, then log2(DICT/32) merge passes double the run length,
// each key placed by one binary search in the partner run (ties: the left
// run first, so equal keys keep their order).  `tmp` holds DICT keys; the
// result ends in `keys`.  Ends with a barrier.
__device__ void block_sort(unsigned long long* keys, unsigned long long* tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int run = warp; run < DICT / 32; run += nw) {
        unsigned long long k = keys[run * 32 + lane];
#pragma unroll
        for (int len = 2; len <= 32; len <<= 1)
#pragma unroll
            for (int j = len >> 1; j > 0; j >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, k, j);
                const bool up = (lane & len) == 0, lower = (lane & j) == 0;
                k = (lower == up) ? (o < k ? o : k) : (o > k ? o : k);
            }
        keys[run * 32 + lane] = k;
    }
    __syncthreads();
    unsigned long long* src = keys;
    unsigned long long* dst = tmp;
    for (int w = 32; w < DICT; w <<= 1) {
        for (int i = threadIdx.x; i < DICT; i += blockDim.x) {
            const int base = i & ~(2 * w - 1), pos = i - base;
            const bool right = pos >= w;
            const int own = right ? pos - w : pos;
            const unsigned long long* other = src + base + (right ? 0 : w);
            const unsigned long long k = src[i];
            int lo = 0, hi = w;   // partner keys before k: < k (left run), <= k (right run)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const unsigned long long v = other[mid];
                if (right ? v <= k : v < k) lo = mid + 1;
                else hi = mid;
            }
            dst[base + own + lo] = k;
        }
        __syncthreads();
        unsigned long long* t = src;
        src = dst;
        dst = t;
    }
    if (src != keys) {
        for (int i = threadIdx.x; i < DICT; i += blockDim.x) keys[i] = src[i];
        __syncthreads();
    }
}

struct CodebookSmem {
    unsigned long long keys[DICT];        // sorted leaves: (weight << 12) | symbol
    unsigned long long iw[DICT];          // internal node weights in creation order
    unsigned long long pw[2 * DICT];      // one round's picks: weight ...
    short pid[2 * DICT];                  // ... and node id (leaf j or n + internal k)
    short parent[2 * DICT];
    short anc[2 * DICT];
    unsigned short dep[2 * DICT];
    unsigned long long pend_w;            // a pick still waiting for its partner
    int pend_id;
    int li, ii, m, K;                     // leaves / internals consumed, picks made, internals made
    unsigned long long bound;
    int n;
    int maxlen;
};

// First index in [lo, hi) whose weight exceeds w (leaf weights when `leaf`).
template <typename W>
__device__ __forceinline__ int upper_w(const CodebookSmem& S, const W* I, bool leaf, int lo,
                                       int hi, W w) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const W v = leaf ? (W)(S.keys[mid] >> 12) : I[mid];
        if (v <= w) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// First index in [lo, hi) of the internal queue whose weight is not below w.
template <typename W>
__device__ __forceinline__ int lower_int(const W* I, int lo, int hi, W w) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (I[mid] < w) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Two-queue Huffman merge, computed in rounds by the whole block.
//
// The picks of the serial algorithm (smaller head first, the leaf on equal
// weight) form one sorted sequence P, the stable merge of the sorted leaves
// with the internal nodes, where internal k = P[2k] + P[2k+1].  If P[m] is
// the smallest head, every internal made from picks m, m+1, ... weighs at
// least 2 P[m]; so every node already present with weight <= 2 P[m] is
// picked before any of them (leaf first and FIFO on ties), in the order of
// the merge of the two present runs.  A round takes that whole run at once
// (ranks by binary search), then pairs consecutive picks into new internal
// nodes.  The bound at least doubles each round, so there are at most
// (bits of the total weight) + 1 rounds, and the tree is the serial one.
template <typename W>
__device__ void round_merge(CodebookSmem& S, int n) {
    const W INF = (W)~0ull;
    W* I = reinterpret_cast<W*>(S.iw);
    W* pw = reinterpret_cast<W*>(S.pw);
    const int tid = threadIdx.x;
    const int total = 2 * n - 2;
    if (tid == 0) {
        S.li = S.ii = S.m = S.K = 0;
    }
    __syncthreads();
    for (int round = 0; round < 2 * 64 + 4; ++round) {
        if (tid == 0 && S.m < total) {
            int li = S.li, ii = S.ii, m = S.m, K = S.K;
            const W hl = li < n ? (W)(S.keys[li] >> 12) : INF;
            const W hi = ii < K ? I[ii] : INF;
            const W head = hl <= hi ? hl : hi;
            S.bound = head > INF / 2 ? (unsigned long long)INF : (unsigned long long)(2 * head);
            if (m & 1) {   // complete the pair left open by the previous round
                int id;
                if (hl <= hi) id = li++;
                else id = n + ii++;
                I[K] = (W)S.pend_w + head;
                S.parent[S.pend_id] = (short)(n + K);
                S.parent[id] = (short)(n + K);
                ++K;
                ++m;
            }
            S.li = li;
            S.ii = ii;
            S.m = m;
            S.K = K;
        }
        __syncthreads();
        const int li = S.li, ii = S.ii, m = S.m, K = S.K;
        if (m >= total) break;
        const W B = (W)S.bound;
        const int lend = upper_w<W>(S, I, true, li, n, B);
        const int iend = upper_w<W>(S, I, false, ii, K, B);
        const int r = (lend - li) + (iend - ii);
        for (int j = li + tid; j < lend; j += blockDim.x) {
            const W w = (W)(S.keys[j] >> 12);
            const int rank = (j - li) + (lower_int<W>(I, ii, iend, w) - ii);
            pw[rank] = w;
            S.pid[rank] = (short)j;
        }
        for (int i = ii + tid; i < iend; i += blockDim.x) {
            const W w = I[i];
            const int rank = (i - ii) + (upper_w<W>(S, I, true, li, lend, w) - li);
            pw[rank] = w;
            S.pid[rank] = (short)(n + i);
        }
        __syncthreads();
        for (int p = tid; p < r / 2; p += blockDim.x) {
            const int a = S.pid[2 * p], b = S.pid[2 * p + 1];
            I[K + p] = pw[2 * p] + pw[2 * p + 1];
            S.parent[a] = (short)(n + K + p);
            S.parent[b] = (short)(n + K + p);
        }
        if (tid == 0) {
            if (r & 1) {
                S.pend_w = (unsigned long long)pw[r - 1];
                S.pend_id = S.pid[r - 1];
            }
            S.li = lend;
            S.ii = iend;
            S.m = m + r;
            S.K = K + r / 2;
        }
        __syncthreads();
    }
}

// Code lengths of one histogram by one block of CB_THREADS threads (S in
// shared memory).  Every return is taken by the whole block.
__device__ void codebook_body(const unsigned long long* __restrict__ hist,
                              uint8_t* __restrict__ lengths, int wide, CodebookSmem& S) {
    const int tid = threadIdx.x;
    for (int s = tid; s < DICT; s += blockDim.x) lengths[s] = 0;
    for (int shift = 0; shift < 64; ++shift) {
        for (int s = tid; s < DICT; s += blockDim.x) {
            unsigned long long f = hist[s];
            if (f) {
                f >>= shift;
                if (f == 0) f = 1;
                S.keys[s] = (f << 12) | (unsigned long long)s;
            } else {
                S.keys[s] = KEY_NONE;
            }
        }
        if (tid == 0) {
            S.maxlen = 0;
            S.n = 0;
        }
        __syncthreads();
        block_sort(S.keys, S.pw);   // pw is free until the merge rounds; ends with a barrier
        // number of used symbols: the last used key sits before the first KEY_NONE
        for (int i = tid; i < DICT; i += blockDim.x)
            if (S.keys[i] != KEY_NONE && (i + 1 == DICT || S.keys[i + 1] == KEY_NONE)) S.n = i + 1;
        __syncthreads();
        const int n = S.n;
        if (n == 0) return;
        if (n == 1) {
            if (tid == 0) lengths[S.keys[0] & 0xFFF] = 1;
            return;
        }
        if (wide) round_merge<unsigned long long>(S, n);
        else round_merge<uint32_t>(S, n);
        // depths by pointer jumping: dep[i] = distance to anc[i]
        const int root = 2 * n - 2;
        for (int i = tid; i <= root; i += blockDim.x) {
            S.anc[i] = i == root ? (short)root : S.parent[i];
            S.dep[i] = i == root ? 0 : 1;
        }
        __syncthreads();
        for (int round = 0; round < 13; ++round) {
            short na[8];
            unsigned short nd[8];
            int c = 0;
            for (int i = tid; i <= root; i += blockDim.x, ++c) {
                const int a = S.anc[i];
                nd[c] = S.dep[i] + S.dep[a];
                na[c] = S.anc[a];
            }
            __syncthreads();
            c = 0;
            bool done = true;
            for (int i = tid; i <= root; i += blockDim.x, ++c) {
                S.dep[i] = nd[c];
                S.anc[i] = na[c];
                done = done && na[c] == root;
            }
            if (__syncthreads_and(done)) break;
        }
        int mx = 0;
        for (int i = tid; i < n; i += blockDim.x) mx = max(mx, (int)S.dep[i]);
        atomicMax(&S.maxlen, mx);
        __syncthreads();
        if (S.maxlen <= LMAX) {
            for (int i = tid; i < n; i += blockDim.x) lengths[S.keys[i] & 0xFFF] = (uint8_t)S.dep[i];
            return;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CB_THREADS) k_codebook(const unsigned long long* __restrict__ hist,
                                                         uint8_t* __restrict__ lengths, int wide) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    codebook_body(hist, lengths, wide, *reinterpret_cast<CodebookSmem*>(smem_raw));
}

// Canonical codes and decoding tables from the code lengths, one block
// (dt null: the codes alone).
// A symbol's place in (length, symbol) order is fi[len] plus the number of
// lower symbols of the same length: counts per 32-symbol chunk (one warp
// match each), an exclusive scan over the chunks per length (one warp per
// length), and the rank inside the chunk give it without a sort.
__device__ void tables_body(const uint8_t* __restrict__ lengths, uint32_t* __restrict__ codes,
                            DecodeTables* __restrict__ dt) {
    constexpr int NCH = DICT / 32;                 // chunks of 32 symbols
    constexpr int PER = DICT / CB_THREADS;         // symbols per thread
    static_assert(NCH == 4 * 32 && PER * CB_THREADS == DICT && LMAX <= CB_THREADS / 32,
                  "chunk scan layout");
    __shared__ unsigned cc[NCH][LMAX + 2];         // chunk counts, then exclusive prefixes
    __shared__ uint16_t ssym[DICT];                // used symbols in (length, symbol) order
    __shared__ unsigned cnt[LMAX + 2];
    __shared__ unsigned long long fc[LMAX + 2];
    __shared__ unsigned fi[LMAX + 2];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < NCH * (LMAX + 2); k += blockDim.x) (&cc[0][0])[k] = 0;
    for (int k = tid; k < DICT; k += blockDim.x) ssym[k] = 0;
    if (tid < LMAX + 2) cnt[tid] = 0;
    if (tid == 0) bad = 0;
    __syncthreads();
    unsigned mylen[PER], myrank[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int s = it * CB_THREADS + tid;   // a warp holds one chunk
        const unsigned len = lengths[s];
        if (len > LMAX) bad = 1;
        const bool ok = len && len <= LMAX;
        const unsigned grp = __match_any_sync(0xffffffffu, ok ? (int)len : -1);
        mylen[it] = ok ? len : 0u;
        myrank[it] = __popc(grp & ((1u << lane) - 1u));
        if (ok && lane == __ffs(grp) - 1) cc[s >> 5][len] = __popc(grp);
    }
    __syncthreads();
    if (warp < LMAX) {   // warp w scans length w + 1 over the chunks (4 per lane)
        const int l = warp + 1;
        unsigned v[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = cc[lane * 4 + j][l];
            sum += v[j];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        unsigned run = incl - sum;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cc[lane * 4 + j][l] = run;
            run += v[j];
        }
        if (lane == 31) cnt[l] = incl;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long code = 0, kraft = 0;
        unsigned idx = 0, maxlen = 0;
        for (int l = 1; l <= LMAX; ++l) kraft += (unsigned long long)cnt[l] << (LMAX - l);
        for (int l = 1; l <= LMAX; ++l) {
            fc[l] = code;
            fi[l] = idx;
            code = (code + cnt[l]) << 1;
            idx += cnt[l];
            if (cnt[l]) maxlen = l;
        }
        const bool valid = !bad && kraft <= (1ull << LMAX);
        for (int l = 0; dt && l < LMAX + 2; ++l) {
            const bool in = l >= 1 && l <= LMAX;
            dt->first_code[l] = in ? (uint32_t)fc[l] : 0;
            dt->first_index[l] = in ? fi[l] : 0;
            dt->lim[l] = in ? ((fc[l] + cnt[l]) << (LMAX - l)) : 0;
        }
        if (dt) {
            dt->maxlen = maxlen;
            dt->valid = valid ? 1 : 0;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int s = it * CB_THREADS + tid;
        const unsigned len = mylen[it];
        if (!len) {
            codes[s] = 0;
            continue;
        }
        const unsigned rank = cc[s >> 5][len] + myrank[it];
        const unsigned p = fi[len] + rank;
        ssym[p] = (uint16_t)s;
        if (dt) dt->sorted[p] = (uint16_t)s;
        codes[s] = (uint32_t)(fc[len] + rank);
    }
    if (!dt) return;   // codes only (the encoder needs no decoding tables)
    __syncthreads();
    // prefix table: the code under each 14-bit prefix, found from the
    // canonical limits (every entry costs the same, whatever the lengths).
    // lim[l], the first code of length l + 1 left-justified, never
    // decreases with l, so a prefix's length is one plus the number of
    // limits it reaches; for l <= 14 the limits are multiples of 2^18 and
    // compare exactly with the prefix in 14-bit units.
    unsigned lim14[LUT_BITS + 1];
#pragma unroll
    for (int l = 1; l <= LUT_BITS; ++l)
        lim14[l] = (unsigned)(((fc[l] + cnt[l]) << (LMAX - l)) >> (32 - LUT_BITS));
    for (int k = tid; k < (1 << LUT_BITS); k += blockDim.x) {
        const unsigned long long top = (unsigned long long)k << (32 - LUT_BITS);
        unsigned l = 1;
#pragma unroll
        for (int j = 1; j <= LUT_BITS; ++j) l += (unsigned)k >= lim14[j];
        uint16_t ent = 0;
        if (l <= LUT_BITS) {
            const unsigned long long idx = fi[l] + ((top >> (32 - l)) - fc[l]);
            if ((top >> (32 - l)) >= fc[l] && idx < DICT)
                ent = (uint16_t)((l << 12) | (unsigned)ssym[idx]);
        } else {
            // longer codes: when every code under the prefix has the same
            // length L (the first and last value under it reach the same
            // number of limits), the entry is 15 << 12 | L and the decoder
            // skips the search over the limits
            const unsigned long long last = top + ((1ull << (32 - LUT_BITS)) - 1);
            unsigned la = 1, lb = 1;
            for (int j = 1; j <= LMAX; ++j) {
                const unsigned long long lj = (fc[j] + cnt[j]) << (LMAX - j);
                la += top >= lj;
                lb += last >= lj;
            }
            if (la == lb && la > LUT_BITS && la <= LMAX && cnt[la])
                ent = (uint16_t)((15u << 12) | la);
        }
        dt->lut[k] = ent;
    }
}

__global__ void __launch_bounds__(CB_THREADS) k_tables(const uint8_t* __restrict__ lengths,
                                                       uint32_t* __restrict__ codes,
                                                       DecodeTables* __restrict__ dt) {
    tables_body(lengths, codes, dt);
}

// Codebooks and tables of many histograms: a persistent grid whose blocks
// take jobs from a device counter (one atomicAdd per job, no waits between
// blocks) until the list is exhausted.  Each job is one field's codebook
// followed by its canonical codes and decoding tables, exactly as the
// single-field kernels compute them.
__global__ void __launch_bounds__(CB_THREADS) k_codebook_tables_batch(const CodebookJob* __restrict__ jobs,
                                                                      int n, unsigned* next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CodebookSmem& S = *reinterpret_cast<CodebookSmem*>(smem_raw);
    __shared__ int job;
    for (;;) {
        if (threadIdx.x == 0) job = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int j = job;
        __syncthreads();   // every thread holds j before the next job is taken
        if (j >= n) return;
        const CodebookJob J = jobs[j];
        codebook_body(J.hist, J.lengths, J.wide, S);
        __syncthreads();   // the lengths are in global memory, visible to the block
        tables_body(J.lengths, J.codes, J.dt);
        __syncthreads();
    }
}

// -- encoding ------------------------------------------------------------------
constexpr int ENC_WARPS = 8;

__global__ void __launch_bounds__(ENC_WARPS * 32) k_chunk_count(
    const uint16_t* __restrict__ sym, uint64_t n, const uint8_t* __restrict__ lengths,
    uint64_t* __restrict__ wcnt, uint64_t* __restrict__ ecnt, uint64_t nchunks, unsigned* status) {
    __shared__ uint8_t len_s[DICT];
    for (int s = threadIdx.x; s < DICT; s += blockDim.x) len_s[s] = lengths[s];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool nocode = false;
    for (uint64_t c = blockIdx.x * (uint64_t)ENC_WARPS + warp; c < nchunks;
         c += (uint64_t)gridDim.x * ENC_WARPS) {
        const uint64_t base = c * CHUNK + lane * 32;
        unsigned bits = 0, esc = 0;
        bool fill = true;
        if (base + 32 <= n) {
            const uint4* v = reinterpret_cast<const uint4*>(sym + base);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 w = v[q];
                const unsigned ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const unsigned s0 = ww[h] & 0xFFFF, s1 = ww[h] >> 16;
                    const unsigned l0 = len_s[s0], l1 = len_s[s1];
                    nocode |= (l0 == 0) | (l1 == 0);
                    bits += l0 + l1;
                    esc += (s0 == MGARD_ESC) + (s1 == MGARD_ESC);
                    fill = fill && ww[h] == FILL_PAIR;
                }
            }
        } else {
            for (uint64_t k = base; k < n && k < base + 32; ++k) {
                const unsigned s = sym[k], l = len_s[s];
                nocode |= l == 0;
                bits += l;
                esc += s == MGARD_ESC;
                fill = fill && s == FILL_SYMBOL;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bits += __shfl_xor_sync(0xffffffffu, bits, o);
            esc += __shfl_xor_sync(0xffffffffu, esc, o);
        }
        fill = __all_sync(0xffffffffu, fill);
        if (lane == 0) {
            wcnt[c] = fill ? 0 : (bits + 31) / 32;   // a chunk of the zero symbol only: no words
            ecnt[c] = esc;
        }
    }
    if (nocode) atomicOr(status, ST_NOCODE);
}

// Exclusive scan of two arrays in place, in three phases: per-tile sums,
// a scan of the tile sums (one CTA), and per-tile scans with the carry.
constexpr int SCAN_T = 1024;            // threads per tile block
constexpr int SCAN_TILE = SCAN_T * 4;   // elements per tile

__device__ inline void block_scan2(unsigned long long& a, unsigned long long& b,
                                   unsigned long long* sa, unsigned long long* sb) {
    // inclusive scan of (a, b) across the block; returns inclusive values
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long va = __shfl_up_sync(0xffffffffu, a, o);
        const unsigned long long vb = __shfl_up_sync(0xffffffffu, b, o);
        if (lane >= o) {
            a += va;
            b += vb;
        }
    }
    if (lane == 31) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x / 32;
        unsigned long long xa = lane < nw ? sa[lane] : 0, xb = lane < nw ? sb[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long va = __shfl_up_sync(0xffffffffu, xa, o);
            const unsigned long long vb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) {
                xa += va;
                xb += vb;
            }
        }
        if (lane < nw) {
            sa[lane] = xa;
            sb[lane] = xb;
        }
    }
    __syncthreads();
    if (warp > 0) {
        a += sa[warp - 1];
        b += sb[warp - 1];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(const uint64_t* __restrict__ a,
                                                      const uint64_t* __restrict__ b, uint64_t n,
                                                      unsigned long long* tsum) {
    __shared__ unsigned long long sa[32], sb[32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    unsigned long long xa = 0, xb = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) {
            xa += a[base + k];
            xb += b[base + k];
        }
    block_scan2(xa, xb, sa, sb);
    if (threadIdx.x == blockDim.x - 1) {
        tsum[2 * blockIdx.x] = xa;
        tsum[2 * blockIdx.x + 1] = xb;
    }
}

// Scan of the tile sums (exclusive, in place); totals[0..1] = grand totals.
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(unsigned long long* tsum, uint64_t ntiles,
                                                       unsigned long long* totals) {
    __shared__ unsigned long long sa[32], sb[32];
    unsigned long long carry_a = 0, carry_b = 0;
    for (uint64_t t0 = 0; t0 < ntiles; t0 += SCAN_T) {
        const uint64_t t = t0 + threadIdx.x;
        const unsigned long long xa = t < ntiles ? tsum[2 * t] : 0, xb = t < ntiles ? tsum[2 * t + 1] : 0;
        unsigned long long ia = xa, ib = xb;
        block_scan2(ia, ib, sa, sb);
        if (t < ntiles) {
            tsum[2 * t] = carry_a + ia - xa;
            tsum[2 * t + 1] = carry_b + ib - xb;
        }
        __shared__ unsigned long long last[2];
        if (threadIdx.x == blockDim.x - 1) {
            last[0] = ia;
            last[1] = ib;
        }
        __syncthreads();
        carry_a += last[0];
        carry_b += last[1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        totals[0] = carry_a;
        totals[1] = carry_b;
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(uint64_t* a, uint64_t* b, uint64_t n,
                                                       const unsigned long long* tsum) {
    __shared__ unsigned long long sa[32], sb[32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
    unsigned long long va[4], vb[4], xa = 0, xb = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        va[k] = base + k < n ? a[base + k] : 0;
        vb[k] = base + k < n ? b[base + k] : 0;
        xa += va[k];
        xb += vb[k];
    }
    unsigned long long ia = xa, ib = xb;
    block_scan2(ia, ib, sa, sb);
    unsigned long long ra = tsum[2 * blockIdx.x] + ia - xa, rb = tsum[2 * blockIdx.x + 1] + ib - xb;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) {
            a[base + k] = ra;
            b[base + k] = rb;
            ra += va[k];
            rb += vb[k];
        }
}

constexpr int PACK_WARPS = 8;
constexpr int PACK_WB = SUB + 4;   // one round's words (256 codes of <= 32 bits) and the carried word

// One warp per chunk, in four rounds of 256 symbols: lane j packs symbols
// [8j, 8j+8) of the round (one 16-byte load).  Lane bit offsets come from a
// warp scan; bits accumulate MSB-first in a 64-bit register and the words a
// lane shares with its neighbours (its first and last) are merged with OR in
// a shared-memory buffer of the round's words.  After each round its
// complete words go out (coalesced) and the partial last word is carried
// into the next round's buffer.  A chunk of the zero symbol only (found
// from the symbols loaded up front) gets no words.  COMPACT: escape values
// arrive compacted per sub-chunk (escapes[s * SUB + r], as the streaming
// quantizer writes them) and each round copies its run to the outlier
// section with coalesced accesses; otherwise escapes[] is indexed by symbol
// position and gathered.
template <bool COMPACT>
__global__ void __launch_bounds__(PACK_WARPS * 32) k_pack(
    const uint16_t* __restrict__ sym, uint64_t n, const uint8_t* __restrict__ lengths,
    const uint32_t* __restrict__ codes, const uint64_t* __restrict__ word_off,
    const uint64_t* __restrict__ esc_off, const int32_t* __restrict__ escapes,
    uint32_t* __restrict__ words, uint16_t* __restrict__ sub_off, int32_t* __restrict__ outliers,
    uint64_t nchunks, PackGuard guard) {
    __shared__ uint8_t len_s[DICT];
    __shared__ uint32_t code_s[DICT];
    __shared__ uint32_t buf[PACK_WARPS][PACK_WB];
    if (guard.status && *guard.status) return;   // an earlier step failed: write nothing
    if (guard.words_byte_off)
        words = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(words) + *guard.words_byte_off);
    for (int s = threadIdx.x; s < DICT; s += blockDim.x) {
        len_s[s] = lengths[s];
        code_s[s] = codes[s];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* wb = buf[warp];
    for (uint64_t c = blockIdx.x * (uint64_t)PACK_WARPS + warp; c < nchunks;
         c += (uint64_t)gridDim.x * PACK_WARPS) {
        const uint64_t cbase = c * CHUNK;
        const int ccnt = (int)min((uint64_t)CHUNK, n - cbase);
        const uint64_t wo = word_off[c];
        const uint64_t eo = esc_off[c];
        // all of the lane's symbols of the chunk are loaded up front (one
        // memory latency per chunk instead of one per round)
        uint4 raw[NSUB];
        bool fill = true;   // every symbol of the lane is the zero symbol
#pragma unroll
        for (int rd = 0; rd < NSUB; ++rd) {
            const int first = rd * SUB + lane * 8;
            if (first + 8 <= ccnt) {
                raw[rd] = *reinterpret_cast<const uint4*>(sym + cbase + first);
                fill = fill && raw[rd].x == FILL_PAIR && raw[rd].y == FILL_PAIR &&
                       raw[rd].z == FILL_PAIR && raw[rd].w == FILL_PAIR;
            } else {
                unsigned t[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    t[k] = first + k < ccnt ? sym[cbase + first + k] : 0;
                    if (first + k < ccnt) fill = fill && t[k] == FILL_SYMBOL;
                }
                raw[rd] = make_uint4(t[0] | (t[1] << 16), t[2] | (t[3] << 16), t[4] | (t[5] << 16),
                                     t[6] | (t[7] << 16));
            }
        }
        if (__all_sync(0xffffffffu, fill)) {   // stored without words; offsets 0
            if (lane < SUBREC) sub_off[c * SUBREC + lane] = 0;
            continue;
        }
        unsigned bit0 = 0, esc0 = 0;   // chunk-relative offsets of the current round
        uint32_t carry = 0;            // the partial word the round starts in
        int64_t pend_at = -1;          // escape values are stored one escape late
        int32_t pend_v = 0;
        // a full chunk (every lane has 8 symbols in every round) runs
        // without the per-symbol count tests
        auto rounds = [&](auto full_tag) {
            constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
            for (int rd = 0; rd < NSUB; ++rd) {
                for (int k = lane; k < PACK_WB; k += 32) wb[k] = k == 0 ? carry : 0u;
                __syncwarp();
                if (rd > 0 && lane == 0) {   // where sub-chunk rd starts inside the chunk
                    sub_off[c * SUBREC + rd - 1] = (uint16_t)bit0;
                    sub_off[c * SUBREC + (NSUB - 1) + rd - 1] = (uint16_t)esc0;
                }
                const int first = rd * SUB + lane * 8;
                const int cnt = FULL ? 8 : max(0, min(8, ccnt - first));
                unsigned sv[8];
                {
                    const uint4 v = raw[rd];
                    sv[0] = v.x & 0xFFFF; sv[1] = v.x >> 16; sv[2] = v.y & 0xFFFF; sv[3] = v.y >> 16;
                    sv[4] = v.z & 0xFFFF; sv[5] = v.z >> 16; sv[6] = v.w & 0xFFFF; sv[7] = v.w >> 16;
                }
                unsigned bits = 0, esc = 0, ln[8];   // code lengths, looked up once
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    ln[k] = k < cnt ? len_s[sv[k]] : 0u;
                    bits += ln[k];
                    if (k < cnt) esc += sv[k] == MGARD_ESC;
                }
                unsigned ib = bits, ie = esc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned vb = __shfl_up_sync(0xffffffffu, ib, o);
                    const unsigned ve = __shfl_up_sync(0xffffffffu, ie, o);
                    if (lane >= o) {
                        ib += vb;
                        ie += ve;
                    }
                }
                const unsigned base = bit0 >> 5;   // the round's first word in the chunk
                const unsigned bpos = bit0 + ib - bits;
                unsigned epos = esc0 + ie - esc;
                const unsigned rtot = __shfl_sync(0xffffffffu, ie, 31);   // escapes of the round
                if (COMPACT)
                    for (unsigned k = lane; k < rtot; k += 32)
                        outliers[eo + esc0 + k] = escapes[cbase + rd * SUB + k];
                bit0 += __shfl_sync(0xffffffffu, ib, 31);
                esc0 += rtot;
                unsigned w = (bpos >> 5) - base;
                int nb = (int)(bpos & 31);
                unsigned long long acc = 0;
                bool firstw = true;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (k < cnt) {
                        const unsigned s = sv[k], len = ln[k];
                        acc = (acc << len) | code_s[s];
                        nb += (int)len;
                        if (nb >= 32) {
                            const uint32_t word = (uint32_t)(acc >> (nb - 32));
                            if (firstw) atomicOr(&wb[w], word);
                            else wb[w] = word;
                            firstw = false;
                            ++w;
                            nb -= 32;
                            acc &= (nb ? ((1ull << nb) - 1) : 0ull);
                        }
                        if (!COMPACT && s == MGARD_ESC) {
                            if (pend_at >= 0) outliers[pend_at] = pend_v;
                            pend_at = (int64_t)(eo + epos++);
                            pend_v = escapes[cbase + first + k];
                        }
                    }
                if (nb > 0) atomicOr(&wb[w], (uint32_t)(acc << (32 - nb)));
                __syncwarp();
                // the round's complete words; the word holding its end carries over
                const unsigned nfull = (bit0 >> 5) - base;
                for (unsigned k = lane; k < nfull; k += 32) words[wo + base + k] = wb[k];
                carry = wb[nfull];
                __syncwarp();
            }
        };
        if (ccnt == CHUNK) rounds(std::true_type{});
        else rounds(std::false_type{});
        if ((bit0 & 31) && lane == 0) words[wo + (bit0 >> 5)] = carry;
        if (!COMPACT && pend_at >= 0) outliers[pend_at] = pend_v;
        __syncwarp();
    }
}

// -- decoding ------------------------------------------------------------------
constexpr int DEC_THREADS = 640;
constexpr int DEC_BLOCKS_PER_SM = 2;   // 33 KB of tables per block; registers capped to fit 2

// Two blocks of 640 threads (40 warps per SM, as five blocks of 256 would
// give) hold two copies of the decode tables instead of five, so more of
// the SM's shared L1 stays cache for the threads' payload words.

// Decoding: one thread per sub-chunk of SUB symbols, in a grid that stays
// resident (each block copies the prefix table once).  The bit window is a
// left-justified 64-bit register refilled one word at a time; a symbol costs
// one shared-memory lookup unless its code is longer than LUT_BITS (then the
// prefix entry gives its length when all codes under the prefix share one,
// else the canonical limits are searched).  Word and escape indices are
// relative to the chunk and the sub-chunk (32-bit arithmetic), and whole
// groups of eight symbols inside one level run without tests for the
// sub-chunk's end or a level boundary.  Word
// loads never leave the chunk, escape reads never leave the chunk's escape
// range, and a sub-chunk whose code stream does not end where its recorded
// offsets say (or that meets a prefix with no code) marks the stream corrupt.
__device__ inline void store8(float* p, const float* v) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ inline void store8(double* p, const double* v) {
#pragma unroll
    for (int k = 0; k < 4; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
}
__device__ inline void store8(uint16_t*, const uint16_t*) {}

// OutT = uint16_t: symbols to `sym`, escape values to `escapes` (indexed by
// symbol position).  OutT = float or double: the dequantized coefficient of
// every symbol to `vals` (symbol order), with the widths of DeqArgs.
template <typename OutT>
__global__ void __launch_bounds__(DEC_THREADS, 2) k_decode(
    const uint32_t* __restrict__ words, uint64_t nwords, const uint64_t* __restrict__ word_off,
    const uint16_t* __restrict__ sub_off, const DecodeTables* __restrict__ gdt, uint64_t n,
    const int32_t* __restrict__ outliers, uint64_t noutliers, const uint64_t* __restrict__ esc_off,
    uint16_t* __restrict__ sym, int32_t* __restrict__ escapes, OutT* __restrict__ vals,
    DeqArgs dq, unsigned* status, uint64_t nchunks, unsigned long long* grab) {
    constexpr bool SYM = sizeof(OutT) == 2;
    __shared__ __align__(16) uint16_t lut[1 << LUT_BITS];
    __shared__ unsigned long long lim[LMAX + 2];
    __shared__ uint32_t fcode[LMAX + 2], findex[LMAX + 2];
    __shared__ __align__(16) uint16_t ssorted[DICT];   // symbols of codes longer than LUT_BITS
    {
        const uint4* src = reinterpret_cast<const uint4*>(gdt->lut);
        uint4* dst = reinterpret_cast<uint4*>(lut);
        for (int k = threadIdx.x; k < (int)(sizeof(lut) / 16); k += blockDim.x) dst[k] = src[k];
        const uint4* ssrc = reinterpret_cast<const uint4*>(gdt->sorted);
        uint4* sdst = reinterpret_cast<uint4*>(ssorted);
        for (int k = threadIdx.x; k < (int)(sizeof(ssorted) / 16); k += blockDim.x) sdst[k] = ssrc[k];
        for (int k = threadIdx.x; k < LMAX + 2; k += blockDim.x) {   // blocks may be one warp
            lim[k] = gdt->lim[k];
            fcode[k] = gdt->first_code[k];
            findex[k] = gdt->first_index[k];
        }
    }
    __syncthreads();
    const unsigned maxlen = gdt->maxlen;
    if (!gdt->valid) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(status, ST_CORRUPT);
        return;
    }
    const uint16_t* sorted = ssorted;
    bool ok = true;
    const uint64_t nsub = nchunks * NSUB;
    // sub-chunks in runs of 32, one per warp: taken from a device counter
    // when one is given (a warp that finishes early takes the next run, so
    // no block waits on a slow one), else in grid order
    const int wl = threadIdx.x & 31;
    const uint64_t wstep = (uint64_t)gridDim.x * blockDim.x;
    uint64_t wbase = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u);
    auto next_run = [&](uint64_t b) -> uint64_t {
        if (!grab) return b;
        unsigned long long r = 0;
        if (wl == 0) r = atomicAdd(grab, 32ull);
        return __shfl_sync(0xffffffffu, r, 0);
    };
    for (wbase = next_run(wbase); wbase < nsub; wbase = next_run(wbase + wstep)) {
        const uint64_t gid = wbase + wl;
        if (gid >= nsub) continue;
        const uint64_t c = gid / NSUB;
        const int sc = (int)(gid % NSUB);
        const uint64_t first = c * CHUNK + (uint64_t)sc * SUB;
        if (first >= n) continue;
        const int cnt = (int)min((uint64_t)SUB, n - first);
        // bit and escape ranges of this sub-chunk, validated against its chunk
        const uint64_t cw0 = word_off[c];
        const uint64_t cw1 = c + 1 < nchunks ? word_off[c + 1] : nwords;
        const uint64_t ce0 = esc_off[c];
        const uint64_t ce1 = c + 1 < nchunks ? esc_off[c + 1] : noutliers;
        if (cw0 > cw1 || cw1 > nwords || ce0 > ce1 || ce1 > noutliers) {
            ok = false;
            continue;
        }
        if (cw1 == cw0) {   // a chunk without words holds only the zero symbol
            if (ce1 != ce0) {
                ok = false;
                continue;
            }
            if (SYM)
                for (int k = 0; k < cnt; ++k) sym[first + k] = (uint16_t)FILL_SYMBOL;
            else
                for (int k = 0; k < cnt; ++k) vals[first + k] = OutT(0);
            continue;
        }
        const uint16_t* so = sub_off + c * SUBREC;
        const uint64_t bstart = cw0 * 32 + (sc ? so[sc - 1] : 0);
        const uint64_t endbit = sc + 1 < NSUB ? cw0 * 32 + so[sc] : cw1 * 32;
        uint64_t e = ce0 + (sc ? so[NSUB - 1 + sc - 1] : 0);
        const uint64_t e_end = sc + 1 < NSUB ? ce0 + so[NSUB - 1 + sc] : ce1;
        if (bstart > endbit || endbit > cw1 * 32 || e > e_end || e_end > ce1) {
            ok = false;
            continue;
        }
        // window: `nb` valid bits, left-justified in `win`; the next two
        // words wait in f[] (loaded two refills ahead of their use; a longer
        // queue covered more latency but cost more moves than it saved)
        // word indices relative to the chunk (a chunk holds at most
        // CHUNK * LMAX / 32 words), so the refill does 32-bit arithmetic
        const uint32_t* __restrict__ cwp = words + cw0;
        const uint32_t nwc = (uint32_t)min(cw1 - cw0, (uint64_t)0x7fffffff);
        uint32_t wi = (uint32_t)min((bstart >> 5) - cw0, (uint64_t)0x7fffffff);
        const uint32_t w0 = wi < nwc ? cwp[wi] : 0u;
        ++wi;
        uint32_t f[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) f[q] = wi + q < nwc ? cwp[wi + q] : 0u;
        const unsigned skip = (unsigned)(bstart & 31);
        const uint64_t wi_start = wi;   // words entered into the window so far: wi - wi_start + 1
        uint64_t win = ((uint64_t)w0 << 32) << skip;
        int nb = 32 - (int)skip;
        // escapes relative to the sub-chunk's first (at most SUB of them)
        const int32_t* __restrict__ ep = outliers + e;
        const uint32_t ne = (uint32_t)min(e_end - e, (uint64_t)0x7fffffff);
        uint32_t ei = 0;
        int32_t next_out = ei < ne ? ep[ei] : 0;   // the next escape value, loaded ahead
        uint32_t pk[4] = {0, 0, 0, 0};
        OutT vk[8];
        // level of the current symbol (dequantizing output)
        // (level, its widths and the sub-chunk index where the next level
        // starts) stay in registers; the boundary test is one compare
        int lvl = 0, next_lvl = 1 << 30;
        float cwf = 0.f;
        double cw = 0.0;
        WidthSplit cws{0.f, 0.f};
        auto enter_level = [&](long long i) {
            while (lvl < dq.lo.L && i >= dq.lo.off[lvl + 1]) ++lvl;
            const long long rel = dq.lo.off[lvl + 1] - (long long)first;
            next_lvl = (int)(rel < (long long)SUB + 1 ? rel : (long long)SUB + 1);
            cwf = dq.wf[lvl];
            cw = dq.w[lvl];
            cws = dq.ws[lvl];
        };
        if (!SYM) enter_level((long long)first);
        // groups of eight symbols, unrolled so that the per-group buffers
        // (pk, vk) stay in registers.  A malformed stream only raises `bad`
        // (every access stays bounded); the sub-chunk is then rejected.
        bool bad = false;
        // one symbol; FAST: the group is whole and stays in one level, so
        // neither the sub-chunk's end nor a level boundary is tested
        auto decode_one = [&](auto fast_tag, int k0, int slot) {
            constexpr bool FAST = decltype(fast_tag)::value;
            const int k = k0 + slot;
            if (!FAST && k >= cnt) return;
            if (nb <= 32) {
                win |= (uint64_t)f[0] << (32 - nb);
                nb += 32;
                f[0] = f[1];
                // past the chunk's last word the load repeats it: those bits
                // never reach a code (the used-bit check below holds)
                f[1] = cwp[min(wi + 2, nwc - 1)];
                ++wi;
            }
            const unsigned ent = lut[(unsigned)(win >> (64 - LUT_BITS))];
            unsigned len, s;
            if ((ent >> 12) - 1u < (unsigned)LUT_BITS) {   // a code of at most LUT_BITS
                len = ent >> 12;
                s = ent & 0xFFF;
            } else {
                const uint32_t top = (uint32_t)(win >> 32);
                unsigned l = ent & 0xFFF;   // the prefix's one length, or 0: search
                if (!l) {
                    l = LUT_BITS + 1;
                    while (l <= maxlen && (unsigned long long)top >= lim[l]) ++l;
                    if (l > maxlen) {   // no code has this prefix
                        bad = true;
                        l = LUT_BITS + 1;
                    }
                }
                len = l;
                s = sorted[min(findex[l] + ((top >> (32 - l)) - fcode[l]), (unsigned)DICT - 1)];
            }
            win <<= len;
            nb -= (int)len;
            int32_t qesc = 0;
            if (s == MGARD_ESC) {
                bad = bad || ei >= ne;   // more escapes than the sub-chunk holds
                qesc = next_out;
                if (SYM) escapes[first + k] = next_out;
                ++ei;
                next_out = ei < ne ? ep[ei] : 0;
            }
            if (SYM) {
                if (slot & 1) pk[slot >> 1] |= s << 16;
                else pk[slot >> 1] = s;
            } else {
                if (!FAST && k >= next_lvl) enter_level((long long)(first + k));
                OutT v;
                if (s == MGARD_ESC) v = dequant_escape<OutT>(qesc, (OutT)cwf, cws, cw);
                else if (sizeof(OutT) == 4) v = (OutT)__fmul_rn((float)((int)s - RADIUS), cwf);
                else v = (OutT)((double)((int)s - RADIUS) * cw);
                vk[slot] = v;
            }
        };
        for (int k0 = 0; k0 < cnt; k0 += 8) {
            const bool whole = k0 + 8 <= cnt;
            if (whole && (SYM || k0 + 8 <= next_lvl)) {
#pragma unroll
                for (int slot = 0; slot < 8; ++slot) decode_one(std::true_type{}, k0, slot);
            } else {
#pragma unroll
                for (int slot = 0; slot < 8; ++slot) decode_one(std::false_type{}, k0, slot);
            }
            if (!whole) continue;
            if (SYM) *reinterpret_cast<uint4*>(sym + first + k0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            else store8(vals + first + k0, vk);
        }
        if (bad) {
            ok = false;
            continue;
        }
        // bits taken from the window: the words that entered it minus the
        // skipped and the unread bits
        const uint64_t used = 32 * (wi - wi_start + 1) - skip - (uint64_t)nb;
        const int rem = cnt & 7;   // symbols decoded after the last full group
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (r >= rem) continue;
            if (SYM) {
                const uint32_t w = pk[r >> 1];
                sym[first + (cnt - rem) + r] = (uint16_t)((r & 1) ? (w >> 16) : (w & 0xFFFF));
            } else {
                vals[first + (cnt - rem) + r] = vk[r];
            }
        }
        // the codes must end inside the sub-chunk's bit range (exactly at its
        // end unless padding follows) and use exactly its escapes
        const uint64_t span = endbit - bstart;
        if (used > span || (sc + 1 < NSUB && used != span) || ei != ne) ok = false;
    }
    if (!ok) atomicOr(status, ST_CORRUPT);
}

}  // namespace

mgard_status huffman_prepare() {
    static std::mutex mu;
    static std::map<int, bool> done;   // per device
    int dev = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev]) {
        MGB_CUDA(cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(CodebookSmem)));
        MGB_CUDA(cudaFuncSetAttribute(k_codebook_tables_batch,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(CodebookSmem)));
        // The decoder's threads read their payload words one at a time and
        // rely on L1 keeping each thread's line between reads.  Left to
        // itself the driver configures shared memory for a third block that
        // the register cap never admits; asking for the two resident blocks'
        // tables (plus the per-block reservation) leaves the rest to L1.
        int smem_sm = 0;
        MGB_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        auto carve = [&](const void* f) -> mgard_status {
            cudaFuncAttributes fa{};
            MGB_CUDA(cudaFuncGetAttributes(&fa, f));
            const long need = (long)DEC_BLOCKS_PER_SM * ((long)fa.sharedSizeBytes + 1024) + 4096;
            const int pct = (int)std::min(100L, (need * 100 + smem_sm - 1) / smem_sm);
            MGB_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
            return MGARD_OK;
        };
        MGB_TRY(carve((const void*)k_decode<float>));
        MGB_TRY(carve((const void*)k_decode<double>));
        MGB_TRY(carve((const void*)k_decode<uint16_t>));
        done[dev] = true;
    }
    return MGARD_OK;
}

mgard_status huffman_codebook(const unsigned long long* hist, uint8_t* lengths, uint32_t* codes,
                              cudaStream_t st, bool wide) {
    const size_t smem = sizeof(CodebookSmem);
    MGB_TRY(huffman_prepare());
    MGB_LAUNCH("k_codebook", st, k_codebook<<<1, CB_THREADS, smem, st>>>(hist, lengths, wide ? 1 : 0));
    MGB_CUDA(cudaGetLastError());
    (void)codes;
    return MGARD_OK;
}

mgard_status huffman_tables(const uint8_t* lengths, uint32_t* codes, DecodeTables* dt,
                            cudaStream_t st) {
    MGB_LAUNCH("k_tables", st, k_tables<<<1, CB_THREADS, 0, st>>>(lengths, codes, dt));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status huffman_codebook_tables_batch(const CodebookJob* jobs, int n, unsigned* counter,
                                           cudaStream_t st) {
    if (n <= 0) return MGARD_OK;
    MGB_TRY(huffman_prepare());
    int dev = 0, sms = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    MGB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MGB_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    MGB_LAUNCH("k_codebook_tables_batch", st,
               k_codebook_tables_batch<<<std::min(n, sms), CB_THREADS, sizeof(CodebookSmem), st>>>(
                   jobs, n, counter));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

size_t count_scratch_bytes(uint64_t n) {
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    return 16 * ((nchunks + SCAN_TILE - 1) / SCAN_TILE + 1);
}

mgard_status huffman_count(const uint16_t* sym, uint64_t n, const uint8_t* lengths,
                           uint64_t* word_off, uint64_t* esc_off, unsigned long long* totals,
                           unsigned* status, cudaStream_t st, unsigned long long* scratch) {
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    if (nchunks) {
        MGB_LAUNCH("k_chunk_count", st, k_chunk_count<<<grid_for((int64_t)nchunks, ENC_WARPS, 148LL * 16), ENC_WARPS * 32, 0, st>>>(
            sym, n, lengths, word_off, esc_off, nchunks, status));
        MGB_CUDA(cudaGetLastError());
    }
    const uint64_t ntiles = (nchunks + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf tbuf;
    unsigned long long* tsum = scratch;
    if (!tsum) {
        MGB_TRY(tbuf.alloc(count_scratch_bytes(n), st));
        tsum = tbuf.as<unsigned long long>();
    }
    if (ntiles) {
        MGB_LAUNCH("k_scan_sums", st, k_scan_sums<<<(unsigned)ntiles, SCAN_T, 0, st>>>(word_off, esc_off, nchunks, tsum));
    }
    MGB_LAUNCH("k_scan_tiles", st, k_scan_tiles<<<1, SCAN_T, 0, st>>>(tsum, ntiles, totals));
    if (ntiles) {
        MGB_LAUNCH("k_scan_apply", st, k_scan_apply<<<(unsigned)ntiles, SCAN_T, 0, st>>>(word_off, esc_off, nchunks, tsum));
    }
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status huffman_pack(const uint16_t* sym, uint64_t n, const uint8_t* lengths,
                          const uint32_t* codes, const uint64_t* word_off, const uint64_t* esc_off,
                          const int32_t* escapes, uint32_t* words, uint16_t* sub_off,
                          int32_t* outliers, cudaStream_t st, PackGuard guard, bool compact) {
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    if (!nchunks) return MGARD_OK;
    int grid = 0;
    MGB_TRY(resident_grid(compact ? (const void*)k_pack<true> : (const void*)k_pack<false>, PACK_WARPS * 32, 0,
                          (int64_t)((nchunks + PACK_WARPS - 1) / PACK_WARPS), &grid));
    if (compact)
        MGB_LAUNCH("k_pack", st, k_pack<true><<<grid, PACK_WARPS * 32, 0, st>>>(
            sym, n, lengths, codes, word_off, esc_off, escapes, words, sub_off, outliers, nchunks, guard));
    else
        MGB_LAUNCH("k_pack", st, k_pack<false><<<grid, PACK_WARPS * 32, 0, st>>>(
            sym, n, lengths, codes, word_off, esc_off, escapes, words, sub_off, outliers, nchunks, guard));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

mgard_status huffman_decode(const uint32_t* words, uint64_t nwords, const uint64_t* word_off,
                            const uint16_t* sub_off, const DecodeTables* dt, uint64_t n,
                            const int32_t* outliers, uint64_t noutliers, const uint64_t* esc_off,
                            uint16_t* sym, int32_t* escapes, unsigned* status, cudaStream_t st) {
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    if (!nchunks) return MGARD_OK;
    const int grid = grid_for((int64_t)(nchunks * NSUB), DEC_THREADS, 148LL * DEC_BLOCKS_PER_SM);
    MGB_TRY(huffman_prepare());
    DeqArgs dq;
    std::memset(&dq, 0, sizeof(dq));
    MGB_LAUNCH("k_decode", st, k_decode<uint16_t><<<grid, DEC_THREADS, 0, st>>>(words, nwords, word_off, sub_off, dt, n, outliers, noutliers,
                                          esc_off, sym, escapes, nullptr, dq, status, nchunks, nullptr));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}

template <typename T>
mgard_status huffman_decode_values(const uint32_t* words, uint64_t nwords, const uint64_t* word_off,
                                   const uint16_t* sub_off, const DecodeTables* dt, uint64_t n,
                                   const int32_t* outliers, uint64_t noutliers,
                                   const uint64_t* esc_off, const DeqArgs& dq, T* vals,
                                   unsigned* status, cudaStream_t st, unsigned long long* grab) {
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    if (!nchunks) return MGARD_OK;
    const int grid = grid_for((int64_t)(nchunks * NSUB), DEC_THREADS, 148LL * DEC_BLOCKS_PER_SM);
    MGB_TRY(huffman_prepare());
    if (grab) MGB_CUDA(cudaMemsetAsync(grab, 0, sizeof(*grab), st));
    MGB_LAUNCH("k_decode", st, k_decode<T><<<grid, DEC_THREADS, 0, st>>>(words, nwords, word_off, sub_off, dt, n, outliers, noutliers,
                                          esc_off, nullptr, nullptr, vals, dq, status, nchunks, grab));
    MGB_CUDA(cudaGetLastError());
    return MGARD_OK;
}
template mgard_status huffman_decode_values<float>(const uint32_t*, uint64_t, const uint64_t*,
                                                   const uint16_t*, const DecodeTables*, uint64_t,
                                                   const int32_t*, uint64_t, const uint64_t*,
                                                   const DeqArgs&, float*, unsigned*, cudaStream_t,
                                                   unsigned long long*);
template mgard_status huffman_decode_values<double>(const uint32_t*, uint64_t, const uint64_t*,
                                                    const uint16_t*, const DecodeTables*, uint64_t,
                                                    const int32_t*, uint64_t, const uint64_t*,
                                                    const DeqArgs&, double*, unsigned*, cudaStream_t,
                                                    unsigned long long*);


// ---------------------------------------------------------------------------
// Allocation-free encoding.  The paper has no counterpart: this serves callers
// that cannot allocate device memory at all (code running under an external
// memory manager or inside a region where cudaMalloc is forbidden).  All
// scratch lives in one file-scope device array of fixed size; every call on a
// device shares it.
namespace {

constexpr uint64_t NOALLOC_MAX_TILES = 2048;   // up to 2048 * 4096 chunks = 8.6e9 symbols
struct NoAllocScratch {
    uint32_t codes[DICT];
    DecodeTables dt;
    unsigned long long tsum[2 * NOALLOC_MAX_TILES + 2];
    unsigned long long totals[2];
    unsigned status;
};

}  // namespace

// Fixed scratch of sizeof(NoAllocScratch) (90,704 bytes) held by every device
// that loads the library until the process exits.  In host code the name is
// only a stand-in for the device address; cudaGetSymbolAddress gives the
// real one.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];
static_assert(sizeof(NoAllocScratch) == 90704,
              "the documented size of the allocation-free scratch (90,704 bytes) is stale");

namespace {

std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_addr;

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
mgard_status noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    MGB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it == g_noalloc_addr.end()) {
        void* ptr = nullptr;
        MGB_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        it = g_noalloc_addr.emplace(dev, ptr).first;
    }
    *out = (NoAllocScratch*)it->second;
    return MGARD_OK;
}

}  // namespace

}  // namespace mgb

extern "C" mgard_status mgard_huffman_encode_noalloc(
    const uint16_t* symbols, uint64_t n, const uint8_t* lengths, const int32_t* escapes,
    uint32_t* words, uint64_t words_cap, uint64_t* word_off, uint64_t* esc_off, uint16_t* sub_off,
    int32_t* outliers, uint64_t outliers_cap, uint64_t* nwords, uint64_t* noutliers, void* stream) {
    using namespace mgb;
    if ((!symbols && n) || !lengths || !nwords || !noutliers ||
        (n && (!word_off || !esc_off || !sub_off)))
        return MGARD_EINVAL;
    if (((uintptr_t)symbols & 15) != 0) {
        set_error("symbols must be 16-byte aligned");
        return MGARD_EINVAL;
    }
    const uint64_t nchunks = (n + CHUNK - 1) / CHUNK;
    const uint64_t ntiles = (nchunks + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles > NOALLOC_MAX_TILES) {
        set_error("mgard_huffman_encode_noalloc: more than 2048 * 4096 * 1024 symbols; use "
                  "mgard_huffman_encode");
        return MGARD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    NoAllocScratch* sc = nullptr;
    MGB_TRY(noalloc_scratch(&sc));
    // the scratch keeps the previous call's contents: clear what must start at zero
    MGB_CUDA(cudaMemsetAsync(&sc->status, 0, sizeof(unsigned), st));
    MGB_CUDA(cudaMemsetAsync(sc->totals, 0, sizeof(sc->totals), st));
    if (nchunks) {
        MGB_LAUNCH("k_chunk_count", st,
                   k_chunk_count<<<grid_for((int64_t)nchunks, ENC_WARPS, 148LL * 16), ENC_WARPS * 32, 0, st>>>(
                       symbols, n, lengths, word_off, esc_off, nchunks, &sc->status));
        MGB_LAUNCH("k_scan_sums", st, k_scan_sums<<<(unsigned)ntiles, SCAN_T, 0, st>>>(word_off, esc_off, nchunks, sc->tsum));
    }
    MGB_LAUNCH("k_scan_tiles", st, k_scan_tiles<<<1, SCAN_T, 0, st>>>(sc->tsum, ntiles, sc->totals));
    if (nchunks)
        MGB_LAUNCH("k_scan_apply", st, k_scan_apply<<<(unsigned)ntiles, SCAN_T, 0, st>>>(word_off, esc_off, nchunks, sc->tsum));
    MGB_CUDA(cudaGetLastError());
    unsigned long long tot[2];
    unsigned status = 0;
    MGB_CUDA(cudaMemcpyAsync(tot, sc->totals, sizeof(tot), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaMemcpyAsync(&status, &sc->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGB_CUDA(cudaStreamSynchronize(st));
    *nwords = tot[0];
    *noutliers = tot[1];
    if (status & ST_NOCODE) {
        set_error("a symbol has no Huffman code");
        return MGARD_EINVAL;
    }
    if (tot[0] > words_cap || tot[1] > outliers_cap) {
        set_error("encode capacity too small");
        return MGARD_ECAPACITY;
    }
    MGB_LAUNCH("k_tables", st, k_tables<<<1, CB_THREADS, 0, st>>>(lengths, sc->codes, &sc->dt));
    if (nchunks) {
        int pgrid = 0;
        MGB_TRY(resident_grid((const void*)k_pack<false>, PACK_WARPS * 32, 0,
                              ((int64_t)nchunks + PACK_WARPS - 1) / PACK_WARPS, &pgrid));
        MGB_LAUNCH("k_pack", st,
                   k_pack<false><<<pgrid, PACK_WARPS * 32, 0, st>>>(
                       symbols, n, lengths, sc->codes, word_off, esc_off, escapes, words, sub_off,
                       outliers, nchunks, PackGuard()));
    }
    MGB_CUDA(cudaGetLastError());
    MGB_CUDA(cudaStreamSynchronize(st));
    return MGARD_OK;
}

namespace mgb {
}  // namespace mgb
