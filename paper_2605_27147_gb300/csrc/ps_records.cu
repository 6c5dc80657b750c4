// Records: rows of W 32-bit words ordered lexicographically (the paper's
// blob types, Sec. 5 "Input data types": randomBlob30, zeroBlob30, and the
// rows ptr points to).
//
// The merge tree of Algorithm 1 depends only on where the runs are, and the
// runs only on which neighbours descend.  So:
//   1. k_rec_scan compares every row with its predecessor (the first word
//      that differs decides) and writes the exact descent mask, and finds L,
//      the length of the prefix all rows share (the smallest first
//      difference over all neighbours);
//   2. k_rec_key extracts the window key, word L of every row: the first
//      word in which rows differ at all, and an order-preserving image of
//      the row (a smaller row never has a larger window);
//   3. the 32-bit pipeline sorts the window keys with the permutation, its
//      run detection reading the descent mask, so runs, powers, merge tree
//      and merge cost are those of the records;
//   4. rows whose windows are equal may still differ later: every group of
//      equal windows comes out of the merges in input order (every merge is
//      stable), and the fix-up sorts each group by the rest of the row, ties
//      by input index: k_rec_fix sorts blocks of up to REC_SMEM entries in
//      shared memory (bitonic; a small group whole by one CTA, the blocks of
//      larger groups spread over all CTAs), and the cooperative
//      k_rec_fix_big merges those blocks pass by pass, every pass spread over
//      the whole grid (a grid barrier between passes).  With one word left
//      to compare (64-bit keys: the low word) entries are packed as (word <<
//      32 | index) and compared directly, without reading rows;
//      With two-word rows whose first words tie in groups larger than
//      REC_SMEM (64-bit keys of a small range: the window is the high word,
//      one word is left), the merge passes are replaced: the library's own
//      batched 32-bit sort (a second, internal context) orders every such
//      group's last words, stably, in one call (k_rec_nested_*; the call is
//      a CUDA graph whose conditional node runs it only when such a group
//      exists);
//   5. the rows move once, through the permutation (ps_gather_rows' kernel),
//      instead of at every merge.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr int REC_BLOCK = 256;
constexpr uint32_t REC_SMEM = 2048;   // group entries sorted in shared memory
constexpr uint32_t REC_TILE_WORDS = 64;   // rows up to this width are scanned through shared memory

// Row a sorts strictly before row b, comparing words w0 .. W-1; equal rows by index.
__device__ __forceinline__ bool rec_less(const uint32_t* rec, uint32_t W, uint32_t w0, uint32_t a, uint32_t b)
{
    const uint32_t* ra = rec + (size_t)a * W;
    const uint32_t* rb = rec + (size_t)b * W;
    for (uint32_t w = w0; w < W; ++w) {
        const uint32_t x = __ldg(ra + w), y = __ldg(rb + w);
        if (x != y) return x < y;
    }
    return a < b;
}

// Outputs [o0, o0 + 16) of one merge pass of width w over a group of g
// entries: the pair [x, x + w) + [x + w, x + 2w) holding o0 is merged from
// src to dst, the first run winning ties.
__device__ void merge_chunk16(const uint32_t* rec, uint32_t W, uint32_t w0, const uint32_t* src, uint32_t* dst,
                              uint32_t g, uint32_t w, uint32_t o0)
{
    const uint32_t x = o0 - o0 % (2 * w);
    const uint32_t na = min(w, g - x), nb = g - x > w ? min(w, g - x - w) : 0u;
    const uint32_t* A = src + x;
    const uint32_t* B = src + x + na;
    const uint32_t d = o0 - x;
    uint32_t lo = d > nb ? d - nb : 0u, hi = min(d, na);
    while (lo < hi) {                                  // A wins ties: take A while !(B < A)
        const uint32_t mid = (lo + hi) >> 1;
        if (!rec_less(rec, W, w0, B[d - 1 - mid], A[mid])) lo = mid + 1; else hi = mid;
    }
    uint32_t ia = lo, ib = d - lo;
    const uint32_t end = min(o0 + 16u, x + na + nb);
    for (uint32_t o = o0; o < end; ++o) {
        const bool take_a = ia < na && (ib >= nb || !rec_less(rec, W, w0, B[ib], A[ia]));
        dst[o] = take_a ? A[ia++] : B[ib++];
    }
}

// Merge passes a group of g > REC_SMEM entries needs (blocks of REC_SMEM).
__device__ __forceinline__ uint32_t merge_passes(uint32_t g)
{
    uint32_t p = 0;
    for (unsigned long long w = REC_SMEM; w < g; w <<= 1) ++p;
    return p;
}

}  // namespace

// Descent mask (bit i: row i-1 > row i; bit 0 clear) and the shared prefix,
// for rows of at most REC_TILE_WORDS words: a CTA stages a tile of 256 rows
// and the row before it (contiguous words, coalesced loads), then every
// thread compares its row with the one before in shared memory.
__global__ void __launch_bounds__(REC_BLOCK) k_rec_scan_tiled(const uint32_t* rec, uint32_t W, unsigned long long n,
                                                              uint32_t* mask, uint32_t* keys, Ctr* C)
{
    extern __shared__ uint32_t rows[];   // (REC_BLOCK + 1) * W words
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    uint32_t lcp = W;
    for (unsigned long long t0 = (unsigned long long)blockIdx.x * REC_BLOCK; t0 < n;
         t0 += (unsigned long long)gridDim.x * REC_BLOCK) {
        // rows t0 - 1 .. t0 + 255 (those that exist) at slots 0 .. 256
        const unsigned long long r0 = t0 ? t0 - 1 : 0ull;
        const unsigned long long r1 = min(t0 + REC_BLOCK, n);
        const uint32_t slot0 = t0 ? 0u : 1u;
        const uint32_t nw = (uint32_t)(r1 - r0) * W;
        const uint32_t* g = rec + (size_t)r0 * W;
        uint32_t* d = rows + slot0 * W;
        for (uint32_t x = tid; x < nw; x += REC_BLOCK) d[x] = __ldg(g + x);
        __syncthreads();
        const unsigned long long i = t0 + tid;
        // word 0 is the window whenever any two neighbours differ there (the
        // usual case): written now, k_rec_key then has nothing to do
        if (i < n) keys[i] = rows[(size_t)(tid + 1) * W];
        bool desc = false;
        if (i > 0 && i < n) {
            const uint32_t* ra = rows + (size_t)tid * W;   // row i - 1 at slot tid
            const uint32_t* rb = ra + W;                    // row i at slot tid + 1
            uint32_t f = W;
            for (uint32_t k = 0; k < W; ++k) {
                if (ra[k] != rb[k]) {
                    f = k;
                    desc = ra[k] > rb[k];
                    break;
                }
            }
            lcp = min(lcp, f);
        }
        const uint32_t word = __ballot_sync(0xffffffffu, desc);
        if (lane == 0 && i < n) mask[i >> 5] = word;
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lcp = min(lcp, __shfl_xor_sync(0xffffffffu, lcp, o));
    if (lane == 0 && lcp < W) atomicMin(&C->rec_lcp, lcp);
}

// The same for wider rows, straight from global memory (a warp per 32 rows).
__global__ void __launch_bounds__(REC_BLOCK) k_rec_scan(const uint32_t* rec, uint32_t W, unsigned long long n,
                                                        uint32_t* mask, Ctr* C)
{
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long warps = ((unsigned long long)gridDim.x * REC_BLOCK) >> 5;
    uint32_t lcp = W;
    for (unsigned long long w = (((unsigned long long)blockIdx.x * REC_BLOCK) >> 5) + (threadIdx.x >> 5);
         w * 32 < n; w += warps) {
        const unsigned long long i = w * 32 + lane;
        bool desc = false;
        if (i > 0 && i < n) {
            const uint32_t* ra = rec + (size_t)(i - 1) * W;
            const uint32_t* rb = rec + (size_t)i * W;
            uint32_t f = W;
            for (uint32_t k = 0; k < W; ++k) {
                const uint32_t x = __ldg(ra + k), y = __ldg(rb + k);
                if (x != y) {
                    f = k;
                    desc = x > y;
                    break;
                }
            }
            lcp = min(lcp, f);
        }
        const uint32_t word = __ballot_sync(0xffffffffu, desc);
        if (lane == 0) mask[w] = word;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lcp = min(lcp, __shfl_xor_sync(0xffffffffu, lcp, o));
    if (lane == 0 && lcp < W) atomicMin(&C->rec_lcp, lcp);
}

// The window key of every row: word L (0 when every row is equal).  When
// skip0 is set the tiled scan has already written word 0, which is the
// window when L = 0.
__global__ void __launch_bounds__(REC_BLOCK) k_rec_key(const uint32_t* rec, uint32_t W, unsigned long long n,
                                                       uint32_t* keys, const Ctr* C, int skip0)
{
    const uint32_t L = *(volatile const uint32_t*)&C->rec_lcp;
    if (skip0 && L == 0) return;
    const unsigned long long stride = (unsigned long long)gridDim.x * REC_BLOCK;
    for (unsigned long long i = (unsigned long long)blockIdx.x * REC_BLOCK + threadIdx.x; i < n; i += stride)
        keys[i] = L < W ? __ldg(rec + (size_t)i * W + L) : 0u;
}

// Groups of equal windows (two or more rows) in the sorted window keys: a
// thread per group start lists it (start, end) -- only when the rows can
// still differ after word L.
__global__ void __launch_bounds__(REC_BLOCK) k_rec_groups(const uint32_t* keys, uint32_t W, unsigned long long n,
                                                          uint32_t* groups, uint32_t cap, uint32_t* big,
                                                          uint32_t big_cap, Ctr* C)
{
    const uint32_t L = *(volatile const uint32_t*)&C->rec_lcp;
    if (L >= W - 1 || *(volatile uint32_t*)&C->error) return;   // NONE: all rows equal
    const unsigned long long stride = (unsigned long long)gridDim.x * REC_BLOCK;
    for (unsigned long long i = (unsigned long long)blockIdx.x * REC_BLOCK + threadIdx.x; i + 1 < n; i += stride) {
        const uint32_t k = keys[i];
        if (keys[i + 1] != k || (i > 0 && keys[i - 1] == k)) continue;
        // the keys are sorted: the group ends at the first key above k,
        // found by galloping then bisection (O(log size) loads)
        unsigned long long lo = i + 1, step = 1;   // keys[lo] == k
        while (lo + step < n && keys[lo + step] == k) {
            lo += step;
            step <<= 1;
        }
        unsigned long long hi = min(lo + step, n);  // keys[hi] != k or hi == n
        while (hi - lo > 1) {
            const unsigned long long mid = (lo + hi) >> 1;
            if (keys[mid] == k) lo = mid; else hi = mid;
        }
        const unsigned long long e = hi;
        const uint32_t at = atomicAdd(&C->rec_groups, 1u);
        if (at < cap) {
            groups[2 * at] = (uint32_t)i;
            groups[2 * at + 1] = (uint32_t)e;
        } else {
            set_error(C, DERR_INTERNAL, 80);
        }
        if (e - i > REC_SMEM) {   // its merge passes run in k_rec_fix_big
            const uint32_t b = atomicAdd(&C->rec_nbig, 1u);
            atomicMax(&C->rec_gmax, (uint32_t)(e - i));
            if (b < big_cap) {
                big[2 * b] = (uint32_t)i;
                big[2 * b + 1] = (uint32_t)e;
            } else {
                set_error(C, DERR_INTERNAL, 81);
            }
        }
    }
}

// One block of up to REC_SMEM entries of a group, sorted by (row from word
// w0, index) in shared memory (bitonic).  With one word left to compare
// (w0 = W - 1) every entry becomes one 64-bit word (that word << 32 |
// index) and the network compares words; otherwise entries compare their
// rows.  The sorted entries go back to perm, or (packed words of a group
// that still needs merge passes) to comp.
__device__ void fix_block(const uint32_t* rec, uint32_t W, uint32_t w0, uint32_t* perm,
                          unsigned long long* comp, uint32_t base, uint32_t m, uint32_t* s,
                          unsigned long long* s64)
{
    const uint32_t tid = threadIdx.x;
    const bool packed = w0 + 1 == W;
    uint32_t P = 2;
    while (P < m) P <<= 1;
    for (uint32_t x = tid; x < P; x += REC_BLOCK) {
        const uint32_t p = x < m ? perm[base + x] : NONE;
        if (packed) s64[x] = x < m ? ((unsigned long long)__ldg(rec + (size_t)p * W + w0) << 32) | p : ~0ull;
        else s[x] = p;
    }
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t x = tid; x < P; x += REC_BLOCK) {
                const uint32_t y = x ^ j;
                if (y <= x) continue;
                const bool up = (x & k) == 0;
                if (packed) {
                    const unsigned long long u = s64[x], v = s64[y];
                    if (up ? v < u : u < v) {
                        s64[x] = v;
                        s64[y] = u;
                    }
                } else {
                    const uint32_t u = s[x], v = s[y];
                    // NONE (padding) sorts last
                    const bool v_first = u == NONE ? v != NONE : (v != NONE && rec_less(rec, W, w0, v, u));
                    if (up ? v_first : !v_first && u != v) {
                        s[x] = v;
                        s[y] = u;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t x = tid; x < m; x += REC_BLOCK) {
        if (!packed) perm[base + x] = s[x];
        else if (comp) comp[base + x] = s64[x];
        else perm[base + x] = (uint32_t)s64[x];
    }
    __syncthreads();
}

// Sort every group by (row from word L + 1, index): a group of up to
// REC_SMEM entries whole, by one CTA; the blocks of larger groups spread
// over all CTAs (their merge passes follow in k_rec_fix_big).
__global__ void __launch_bounds__(REC_BLOCK) k_rec_fix(const uint32_t* rec, uint32_t W, uint32_t* perm,
                                                       unsigned long long* comp, const uint32_t* groups,
                                                       uint32_t cap, const uint32_t* big, uint32_t big_cap, Ctr* C,
                                                       uint32_t nested)
{
    __shared__ uint32_t s[REC_SMEM];
    __shared__ unsigned long long s64[REC_SMEM];
    const uint32_t L = *(volatile const uint32_t*)&C->rec_lcp;
    if (L >= W - 1 || *(volatile uint32_t*)&C->error) return;   // NONE: all rows equal
    const uint32_t w0 = L + 1;
    const uint32_t ng = min(*(volatile const uint32_t*)&C->rec_groups, cap);
    for (uint32_t gi = blockIdx.x; gi < ng; gi += gridDim.x) {
        const uint32_t a = groups[2 * gi], g = groups[2 * gi + 1] - a;
        if (g <= REC_SMEM) fix_block(rec, W, w0, perm, nullptr, a, g, s, s64);
    }
    // big groups: blocks for the merge passes, unless the nested sort
    // orders them (one word left to compare)
    const uint32_t nbig = (nested && w0 + 1 == W) ? 0u : min(*(volatile const uint32_t*)&C->rec_nbig, big_cap);
    for (uint32_t b = 0; b < nbig; ++b) {
        const uint32_t a = big[2 * b], g = big[2 * b + 1] - a;
        const uint32_t nblk = (g + REC_SMEM - 1) / REC_SMEM;
        for (uint32_t k = blockIdx.x; k < nblk; k += gridDim.x)
            fix_block(rec, W, w0, perm, comp, a + k * REC_SMEM, min(REC_SMEM, g - k * REC_SMEM), s, s64);
    }
}

// Outputs [o0, o0 + 16) of one merge pass over packed words (distinct, so
// no tie rule is needed).
__device__ void merge_chunk16_packed(const unsigned long long* src, unsigned long long* dst, uint32_t g, uint32_t w,
                                     uint32_t o0)
{
    const uint32_t x = o0 - o0 % (2 * w);
    const uint32_t na = min(w, g - x), nb = g - x > w ? min(w, g - x - w) : 0u;
    const unsigned long long* A = src + x;
    const unsigned long long* B = src + x + na;
    const uint32_t d = o0 - x;
    uint32_t lo = d > nb ? d - nb : 0u, hi = min(d, na);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] < B[d - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    uint32_t ia = lo, ib = d - lo;
    const uint32_t end = min(o0 + 16u, x + na + nb);
    for (uint32_t o = o0; o < end; ++o) {
        const bool take_a = ia < na && (ib >= nb || A[ia] < B[ib]);
        dst[o] = take_a ? A[ia++] : B[ib++];
    }
}

// The merge passes of every group larger than REC_SMEM (its blocks already
// sorted by k_rec_fix): pass p merges pairs of width REC_SMEM << p, for
// every group that still has pairs; chunks of 16 outputs of all such groups
// are spread over the grid, and a grid barrier separates the passes.  Rows
// compared through perm <-> tmp, or packed words through comp <-> comp2;
// at the end every group's entries are back in perm.
__global__ void __launch_bounds__(REC_BLOCK) k_rec_fix_big(const uint32_t* rec, uint32_t W, uint32_t* perm,
                                                           uint32_t* tmp, unsigned long long* comp,
                                                           unsigned long long* comp2, const uint32_t* big,
                                                           uint32_t big_cap, Ctr* C)
{
    const uint32_t L = *(volatile const uint32_t*)&C->rec_lcp;
    if (L >= W - 1 || *(volatile uint32_t*)&C->error) return;
    const uint32_t gmax = *(volatile const uint32_t*)&C->rec_gmax;
    if (gmax <= REC_SMEM) return;                     // the same answer in every CTA
    const uint32_t w0 = L + 1;
    const bool packed = w0 + 1 == W;
    const uint32_t nbig = min(*(volatile const uint32_t*)&C->rec_nbig, big_cap);
    const uint32_t gt = blockIdx.x * REC_BLOCK + threadIdx.x, gs = gridDim.x * REC_BLOCK;
    const uint32_t passes = merge_passes(gmax);
    for (uint32_t p = 0; p < passes; ++p) {
        const uint32_t w = REC_SMEM << p;
        for (uint32_t b = 0; b < nbig; ++b) {
            const uint32_t a = big[2 * b], g = big[2 * b + 1] - a;
            if (g <= w) continue;
            const uint32_t chunks = (g + 15u) >> 4;
            for (uint32_t c = gt; c < chunks; c += gs) {
                if (packed) {
                    const unsigned long long* from = (p & 1u) ? comp2 : comp;
                    unsigned long long* to = (p & 1u) ? comp : comp2;
                    merge_chunk16_packed(from + a, to + a, g, w, c * 16u);
                } else {
                    const uint32_t* from = (p & 1u) ? tmp : perm;
                    uint32_t* to = (p & 1u) ? perm : tmp;
                    merge_chunk16(rec, W, w0, from + a, to + a, g, w, c * 16u);
                }
            }
        }
        if (!grid_barrier(C)) return;
    }
    for (uint32_t b = 0; b < nbig; ++b) {
        const uint32_t a = big[2 * b], g = big[2 * b + 1] - a;
        const bool odd = (merge_passes(g) & 1u) != 0;   // the last pass wrote the second buffer
        if (packed) {
            const unsigned long long* fin = odd ? comp2 : comp;
            for (uint32_t x = gt; x < g; x += gs) perm[a + x] = (uint32_t)fin[a + x];
        } else if (odd) {
            for (uint32_t x = gt; x < g; x += gs) perm[a + x] = tmp[a + x];
        }
    }
}

// The nested sort of the big groups (one word left, w0 = W - 1): the number
// of groups it orders (0 when there is nothing to fix up).
__device__ __forceinline__ uint32_t nested_groups(uint32_t W, uint32_t big_cap, Ctr* C)
{
    const uint32_t L = *(volatile const uint32_t*)&C->rec_lcp;
    if (L >= W || L + 2 != W || *(volatile uint32_t*)&C->error) return 0u;
    return min(*(volatile const uint32_t*)&C->rec_nbig, big_cap);
}

// One CTA: the nested sort's instance offsets -- the big groups in list
// order, then empty instances up to big_cap.
__global__ void __launch_bounds__(1024) k_rec_nested_offsets(uint32_t W, const uint32_t* big, uint32_t big_cap,
                                                              unsigned long long* off, Ctr* C)
{
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    const uint32_t nbig = nested_groups(W, big_cap, C);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < big_cap; b0 += 1024) {
        const uint32_t b = b0 + threadIdx.x;
        const unsigned long long v = b < nbig ? (unsigned long long)(big[2 * b + 1] - big[2 * b]) : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        unsigned long long before = carry, tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < warp) before += ws[w];
            tot += ws[w];
        }
        if (b < big_cap) off[b] = before + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[big_cap] = carry;
}

// The big group holding entry j of the nested sort (its offsets
// non-decreasing): the last b < nbig with off[b] <= j.
__device__ __forceinline__ uint32_t nested_group_of(const unsigned long long* off, uint32_t nbig, unsigned long long j)
{
    uint32_t lo = 0, hi = nbig;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
    }
    return lo;
}

// The nested sort's keys: the last word of every big group's rows in the
// group's current (input) order; and the entries themselves, kept.
__global__ void __launch_bounds__(REC_BLOCK) k_rec_nested_gather(const uint32_t* rec, uint32_t W, const uint32_t* perm,
                                                                 const uint32_t* big, uint32_t big_cap,
                                                                 const unsigned long long* off, uint32_t* keys2,
                                                                 uint32_t* save, Ctr* C)
{
    const uint32_t nbig = nested_groups(W, big_cap, C);
    if (!nbig) return;
    const unsigned long long total = off[nbig];
    for (unsigned long long j = (unsigned long long)blockIdx.x * REC_BLOCK + threadIdx.x; j < total;
         j += (unsigned long long)gridDim.x * REC_BLOCK) {
        const uint32_t b = nested_group_of(off, nbig, j);
        const uint32_t p = perm[big[2 * b] + (uint32_t)(j - off[b])];
        keys2[j] = __ldg(rec + (size_t)p * W + (W - 1));
        save[j] = p;
    }
}

// Every big group's entries in the nested sort's order (its permutation is
// local to the group).  An error of the nested sort (its own counters, C2)
// becomes this sort's error and leaves perm as the window sort left it.
__global__ void __launch_bounds__(REC_BLOCK) k_rec_nested_apply(uint32_t W, uint32_t* perm, const uint32_t* big,
                                                                uint32_t big_cap, const unsigned long long* off,
                                                                const uint32_t* perm2, const uint32_t* save, Ctr* C,
                                                                const Ctr* C2)
{
    const uint32_t nbig = nested_groups(W, big_cap, C);
    if (!nbig) return;
    const uint32_t e2 = *(volatile const uint32_t*)&C2->error;
    if (e2) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_error(C, e2, 83);
        return;
    }
    const unsigned long long total = off[nbig];
    for (unsigned long long j = (unsigned long long)blockIdx.x * REC_BLOCK + threadIdx.x; j < total;
         j += (unsigned long long)gridDim.x * REC_BLOCK) {
        const uint32_t b = nested_group_of(off, nbig, j);
        const uint32_t g = big[2 * b + 1] - big[2 * b];
        const uint32_t local = perm2[j];
        if (local >= g) {
            set_error(C, DERR_INTERNAL, 82);
            continue;
        }
        perm[big[2 * b] + (uint32_t)(j - off[b])] = save[off[b] + local];
    }
}

// The nested sort runs (a graph's conditional node) only when there is a
// big group to order.
__global__ void k_rec_nested_cond(cudaGraphConditionalHandle h, uint32_t W, uint32_t big_cap, Ctr* C)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, nested_groups(W, big_cap, C) ? 1u : 0u);
}

const void* records_nested_cond_kernel()
{
    return reinterpret_cast<const void*>(k_rec_nested_cond);
}

cudaError_t launch_records_nested_prep(const uint32_t* rec, uint32_t W, const uint32_t* perm, const uint32_t* big,
                                       uint32_t big_cap, unsigned long long* off, uint32_t* keys2, uint32_t* save,
                                       Ctr* C, int grid, cudaStream_t s)
{
    k_rec_nested_offsets<<<1, 1024, 0, s>>>(W, big, big_cap, off, C);
    k_rec_nested_gather<<<grid, REC_BLOCK, 0, s>>>(rec, W, perm, big, big_cap, off, keys2, save, C);
    return cudaGetLastError();
}

cudaError_t launch_records_nested_apply(uint32_t W, uint32_t* perm, const uint32_t* big, uint32_t big_cap,
                                        const unsigned long long* off, const uint32_t* perm2, const uint32_t* save,
                                        Ctr* C, const Ctr* C2, int grid, cudaStream_t s)
{
    k_rec_nested_apply<<<grid, REC_BLOCK, 0, s>>>(W, perm, big, big_cap, off, perm2, save, C, C2);
    return cudaGetLastError();
}

cudaError_t launch_records_prepare(const uint32_t* rec, uint32_t W, unsigned long long n, uint32_t* mask,
                                   uint32_t* keys, Ctr* C, int grid, cudaStream_t s)
{
    if (W <= REC_TILE_WORDS) {
        const size_t smem = (size_t)(REC_BLOCK + 1) * W * sizeof(uint32_t);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_rec_scan_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rec_scan_tiled<<<grid, REC_BLOCK, smem, s>>>(rec, W, n, mask, keys, C);
        k_rec_key<<<grid, REC_BLOCK, 0, s>>>(rec, W, n, keys, C, 1);
    } else {
        k_rec_scan<<<grid, REC_BLOCK, 0, s>>>(rec, W, n, mask, C);
        k_rec_key<<<grid, REC_BLOCK, 0, s>>>(rec, W, n, keys, C, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_records_fix(const uint32_t* rec, uint32_t W, unsigned long long n, const uint32_t* keys,
                               uint32_t* perm, uint32_t* tmp, unsigned long long* comp, unsigned long long* comp2,
                               uint32_t* groups, uint32_t cap, uint32_t* big, uint32_t big_cap, Ctr* C, int grid,
                               int coop_grid, bool nested, cudaStream_t s)
{
    k_rec_groups<<<grid, REC_BLOCK, 0, s>>>(keys, W, n, groups, cap, big, big_cap, C);
    k_rec_fix<<<grid, REC_BLOCK, 0, s>>>(rec, W, perm, comp, groups, cap, big, big_cap, C, nested ? 1u : 0u);
    if (nested) return cudaGetLastError();       // the big groups go to the nested sort
    void* args[] = {(void*)&rec, (void*)&W,   (void*)&perm,    (void*)&tmp, (void*)&comp,
                    (void*)&comp2, (void*)&big, (void*)&big_cap, (void*)&C};
    return cudaLaunchCooperativeKernel((const void*)k_rec_fix_big, dim3(coop_grid), dim3(REC_BLOCK), args, 0, s);
}

int records_fix_big_grid(int num_sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rec_fix_big, REC_BLOCK, 0);
    const int g = num_sms * (per_sm > 0 ? per_sm : 1);
    return g < 1024 ? g : 1024;   // the grid barrier counts at most 1024 CTAs
}

}  // namespace ps
