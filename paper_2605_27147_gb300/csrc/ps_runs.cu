// Run detection with the minimum-run-length rule (ExtractRun, Sec. 2;
// minrun rule, Sec. 5 "Algorithm variants") for a batch of instances.
//
// Sequentially, the run starts are the orbit of 0 under
//     f(s) = max(d(s), min(s + minrun, n)),
// d(s) = the first descent position e > s (a[e-1] > a[e]) or n.  A natural
// run of at least minrun elements keeps its end d(s); a shorter one is forced
// to min(s + minrun, n) elements (the insertion sort of the forced run is done
// later, on chip, by the tile kernel -- it does not move any run boundary).
//
// Parallel form.  The instance is cut into chunks of RUN_CHUNK elements.  The
// first run start at or after a chunk's begin B can only be
//     B + delta (0 <= delta < minrun)        -- a forced step landed there, or
//     D0 = the first descent at or after B   -- a natural step ended there,
// so a chunk has at most minrun + 1 <= 64 entry states.  Each chunk walks the
// chain from every entry state (one lane per state) over its descent bitmask,
// which gives a map  entry state -> (exit state of the next chunk, runs
// started in this chunk).  The descent bitmask reaches RUN_HALO positions past
// the chunk, so a forced step from inside the chunk (length <= 63) is always
// decided locally; a natural run that runs past the halo ends at the next
// chunk's D0, which is one of that chunk's entry states.  An instance's first
// chunk is entered at state 0 whatever came before: its map is constant, and
// it restarts the run count.
//
// Decreasing runs (the variant Sec. 5 "Algorithm variants" names, taken when
// Job::desc_runs is set): a run whose first pair descends strictly ends at the
// first non-descent instead (or at n), and is reversed later by the tile
// kernel.  A run that spans the chunk start B is then either ascending (no
// descent at B) or strictly decreasing (a descent at B), so the natural state
// becomes X0 = the first position after B whose descent bit differs from B's;
// when B's own bit decides (a run ends at B) the state is B + 0.  The entry
// states stay at most minrun + 1.
//
// The maps are composed by a reduce-then-scan.  k_runs: every CTA owns a
// contiguous range of chunks, computes their maps and folds them into one
// 64-entry map for the range; the last CTA to finish walks the ranges' maps
// in order and records the entry state and run count at every range start.
// k_runs_emit: every CTA walks its range's chunk maps from that entry,
// giving each chunk's entry state and the number of runs before it, and
// writes the chunk's run starts -- in closed form when every step in the
// chunk is forced (the usual case for unsorted data), otherwise by walking
// the one chain it actually takes over the chunk's descent bitmask.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_sums, T& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    T before = warp ? warp_sums[warp - 1] : T(0);
    total = warp_sums[nwarps - 1];
    __syncthreads();
    return before + x - v;
}

// Sec. 5: l = n; while l >= 64: l = ceil(l / 2).
__device__ __forceinline__ uint32_t minrun_of(uint32_t n)
{
    uint32_t l = n;
    while (l >= 64) l = (l + 1) >> 1;
    return l;
}

}  // namespace

// One CTA: per-instance sizes, minrun, chunk bases and run-slot bases
// (exclusive scans), counters reset.  Instances with n < 64 are one run
// (minrun = n) and need no chunk: their run list is written here.
__global__ void __launch_bounds__(1024) k_setup(Job J)
{
    __shared__ unsigned long long ws64[32];
    __shared__ uint32_t ws32[32];
    __shared__ unsigned long long carry_slots;
    __shared__ uint32_t carry_chunks, carry_gmap;
    Ctr* C = J.ctr;
    __shared__ uint32_t s_bad;
    if (threadIdx.x == 0) {
        carry_slots = 0;
        carry_chunks = 0;
        carry_gmap = 0;
        s_bad = 0;
        C->error = 0;
        C->err_where = 0;
        C->runs_done = 0;
        C->n_tiles = 0;
        C->n_gnodes = 0;
        C->rounds = 0;
        C->bar_count = 0;
        C->max_power = 0;
        C->leaf_moves = 0;
        C->M_total = 0;
        C->runs_total = 0;
        C->n_total = 0;
        C->hbm_elems = 0;
        C->merge_t0 = 0;
    }
    if (threadIdx.x < 32) {
        C->bar_group[threadIdx.x] = 0;
        C->runs_grp_done[threadIdx.x] = 0;
    }
    for (int r = threadIdx.x; r < NPOW + 2; r += blockDim.x) {
        if (r < NPOW) {
            C->round_ns[r][0] = C->round_ns[r][2] = ~0ull;   // minima
            C->round_ns[r][1] = C->round_ns[r][3] = 0;       // maxima
            C->chunk_next[r] = 0;
        }
        if (r < NPOW + 1) {
            C->bucket_count[r] = 0;
            C->bucket_nchunk[r] = 0;
            C->bucket_cursor[r] = 0;
        }
        C->bucket_start[r] = 0;
        C->bucket_chunk[r] = 0;
    }
    __syncthreads();
    for (uint32_t base = 0; base < J.count; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < J.count;
        unsigned long long off = 0, n64 = 0;
        if (valid) {
            if (J.offsets) {
                off = J.offsets[i];
                const unsigned long long end = J.offsets[i + 1];
                // the table must start at 0, never decrease and respect the limits
                if ((i == 0 && off != 0) || end < off || end - off > J.max_n || end > J.max_total) {
                    atomicOr(&s_bad, 1u);
                    n64 = 0;
                } else {
                    n64 = end - off;
                }
            } else {
                n64 = J.single_n;
            }
        }
        const uint32_t n = (uint32_t)n64;
        const uint32_t nchunks = (valid && n >= 64) ? (n + RUN_CHUNK - 1) / RUN_CHUNK : 0u;
        const unsigned long long cap = valid ? (unsigned long long)(n / 32) + 2ull : 0ull;
        // merge-map entries: an HBM merge (more than T elements) has an index
        // below 4n / T (merge_index)
        const uint32_t gspan = (valid && n > J.tile_cap) ? (uint32_t)((4ull * n + J.tile_cap - 1) / J.tile_cap) : 0u;
        uint32_t tot_c, tot_g;
        unsigned long long tot_s;
        const uint32_t cb = block_exclusive_scan<uint32_t>(nchunks, ws32, tot_c);
        const unsigned long long sb = block_exclusive_scan<unsigned long long>(cap, ws64, tot_s);
        const uint32_t gb = block_exclusive_scan<uint32_t>(gspan, ws32, tot_g);
        if (valid) {
            Inst I;
            I.off = off;
            I.run_base = carry_slots + sb;
            I.M = 0;
            I.n = n;
            I.minrun = minrun_of(n);
            I.recip = n ? 0xffffffffffffffffull / n : 0ull;
            I.chunk_base = carry_chunks + cb;
            I.nchunks = nchunks;
            I.max_power = 0;
            I.g_base = carry_gmap + gb;
            I.g_span = gspan;
            I.runs = n == 0 ? 0u : (n < 64 ? 1u : 0u);
            J.inst[i] = I;
            if (n < 64 && I.run_base + 1 < J.slot_cap) {   // one run [0, n) (or none)
                J.run_start[I.run_base] = 0;
                if (n) J.run_start[I.run_base + 1] = n;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_chunks += tot_c;
            carry_slots += tot_s;
            carry_gmap += tot_g;
        }
        __syncthreads();
    }
    if (J.vm) {
        // virtual-memory storage: every virtual page starts as its own array page;
        // the free-page ring (filled by the rounds kernel) starts with the pool pages
        const uint32_t na = J.single_n ? (uint32_t)((J.single_n + (1ull << J.vm_plog2) - 1) >> J.vm_plog2) : 0u;
        for (uint32_t u = threadIdx.x; u < J.vm_na_cap; u += blockDim.x) {
            J.pt[u] = u;
            J.page_cnt[u] = 0;
            J.consumed[u] = 0;
        }
        if (threadIdx.x == 0) {
            C->vm_free_top = 0;
            C->vm_ring_head = 0;
            C->vm_ring_tail = J.vm_pool;
            C->vm_round_base = 0;
            C->vm_touched = 0;
            C->vm_wave = 0;
            C->vm_in_use_peak = 0;
            C->vm_waves = 0;
            C->vm_copy_moves = 0;
            C->vm_spliced = 0;
            if (na > J.vm_na_cap) set_error(C, DERR_INTERNAL, 3);
        }
    }
    if (threadIdx.x == 0) {
        C->total_chunks = carry_chunks;
        C->total_slots = carry_slots;
        if (s_bad) set_error(C, DERR_INVAL, 2);
        else if (carry_chunks > J.chunk_cap || carry_slots > J.slot_cap || carry_gmap > J.gmap_cap)
            set_error(C, DERR_INTERNAL, 1);
    }
}

namespace {

// A chunk's descent bitmask is followed, in the same shared array, by two
// summaries of its words for the searches below: bit w of the first is set
// when word w has a set bit, bit w of the second when word w has a clear bit.
// A search then skips a long run of empty (or full) words in one step instead
// of a dependent load per word.
constexpr int SUM_WORDS = (RUN_WORDS + 31) / 32;
constexpr int BITS_NZ = RUN_WORDS;                  // words with a descent
constexpr int BITS_NF = RUN_WORDS + SUM_WORDS;      // words with a non-descent
constexpr int BITS_SLOTS = RUN_WORDS + 2 * SUM_WORDS;
static_assert(RUN_WORDS <= RUN_BLOCK - 32, "k_runs' last warp has no bitmask words to check");

// Warp 0, once the bitmask is complete: its summaries.
__device__ __forceinline__ void bits_summary(uint32_t* bits)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < SUM_WORDS; ++j) {
        const int w = j * 32 + lane;
        const uint32_t b = w < RUN_WORDS ? bits[w] : 0u;
        const uint32_t nz = __ballot_sync(FULL, w < RUN_WORDS && b != 0u);
        const uint32_t nf = __ballot_sync(FULL, w < RUN_WORDS && b != FULL);
        if (lane == 0) {
            bits[BITS_NZ + j] = nz;
            bits[BITS_NF + j] = nf;
        }
    }
}

// First word index >= w0 whose bit is set in the summary sum, or wmax.
__device__ __forceinline__ int next_word(const uint32_t* sum, int w0, int wmax)
{
    if (w0 >= wmax) return wmax;
    int j = w0 >> 5;
    uint32_t m = sum[j] & (FULL << (w0 & 31));
    while (m == 0) {
        if (++j >= SUM_WORDS) return wmax;
        m = sum[j];
    }
    const int w = (j << 5) + __ffs(m) - 1;
    return w < wmax ? w : wmax;
}

// First set bit at index >= k0 in bits[0, kmax), kmax a multiple of 32 and at
// most KMAX; kmax when there is none.
__device__ __forceinline__ int next_desc(const uint32_t* bits, int k0, int kmax)
{
    if (k0 >= kmax) return kmax;
    const int w = k0 >> 5, wmax = kmax >> 5;
    const uint32_t word = bits[w] & (FULL << (k0 & 31));
    if (word) return (w << 5) + __ffs(word) - 1;
    const int w2 = next_word(bits + BITS_NZ, w + 1, wmax);
    return w2 < wmax ? (w2 << 5) + __ffs(bits[w2]) - 1 : kmax;
}

// First clear bit at index >= k0 in bits[0, kmax), kmax a multiple of 32 and
// at most KMAX; kmax when there is none.
__device__ __forceinline__ int next_clear(const uint32_t* bits, int k0, int kmax)
{
    if (k0 >= kmax) return kmax;
    const int w = k0 >> 5, wmax = kmax >> 5;
    const uint32_t word = ~bits[w] & (FULL << (k0 & 31));
    if (word) return (w << 5) + __ffs(word) - 1;
    const int w2 = next_word(bits + BITS_NF, w + 1, wmax);
    return w2 < wmax ? (w2 << 5) + __ffs(~bits[w2]) - 1 : kmax;
}

__device__ __forceinline__ bool desc_bit(const uint32_t* bits, int k)
{
    return ((bits[k >> 5] >> (k & 31)) & 1u) != 0;
}

constexpr int KMAX = RUN_WORDS * 32;
constexpr int WIN = 32;                      // maps staged in shared memory per batch

// The chunk g of instance qi as seen by both kernels.
struct ChunkView {
    uint32_t qi, c, n, m, B, E, span, rem;
    const uint32_t* a;
};

// qi: the instance of the previous chunk of the same range (NONE at the
// range start); chunks of a range are consecutive, so it only moves forward.
__device__ __forceinline__ ChunkView chunk_view(const Job& J, uint32_t g, uint32_t& qi)
{
    ChunkView v;
    if (qi == NONE) {
        qi = find_inst(J.count, g, [&](uint32_t i) { return (unsigned long long)J.inst[i].chunk_base; });
    } else {
        while (qi + 1 < J.count && J.inst[qi + 1].chunk_base <= g) ++qi;
    }
    v.qi = qi;
    const Inst& I = J.inst[v.qi];
    v.c = g - I.chunk_base;
    v.n = I.n;
    v.m = I.minrun;
    v.B = v.c * RUN_CHUNK;
    v.E = min(v.B + (uint32_t)RUN_CHUNK, v.n);
    v.span = v.E - v.B;
    v.rem = v.n - v.B;
    v.a = J.keysA + I.off;
    return v;
}

// The chunk's key window [W0, W1), W0 = max(B, 1) - 1 (the key before the
// chunk, when there is one), W1 = min(B + KMAX, n), staged in shared memory
// by asynchronous copies (cp.async: no registers held while they fly): the
// 16-byte-aligned interior 16 bytes at a time, the at most three keys at each
// end 4 bytes at a time.  Key x sits at slot x - W0 + shift, where shift
// keeps the slot congruent to the global address modulo 16 bytes.
constexpr int WIN_SLOTS = KMAX + 8;

struct KeyWindow {
    uint32_t W0, len, shift;
};

__device__ __forceinline__ KeyWindow window_of(const ChunkView& v)
{
    KeyWindow w;
    w.W0 = v.B > 0 ? v.B - 1 : 0u;
    const uint32_t W1 = (uint32_t)min((unsigned long long)v.B + KMAX, (unsigned long long)v.n);
    w.len = W1 - w.W0;
    w.shift = (uint32_t)(((uintptr_t)(v.a + w.W0) >> 2) & 3u);
    return w;
}


// Start staging the window (one commit group per call).
__device__ __forceinline__ void stage_keys(const ChunkView& v, const KeyWindow& w, uint32_t* keys)
{
    const int tid = threadIdx.x;
    const uint32_t* g = v.a + w.W0;
    const uint32_t head = min((4u - w.shift) & 3u, w.len);
    const uint32_t nvec = (w.len - head) >> 2;
    for (uint32_t i = tid; i < nvec; i += RUN_BLOCK)
        cp_async16(&keys[w.shift + head + 4 * i], g + head + 4 * i);
    const uint32_t tail0 = head + 4 * nvec;
    for (uint32_t x = tid; x < head; x += RUN_BLOCK) cp_async4(&keys[w.shift + x], g + x);
    for (uint32_t x = tail0 + tid; x < w.len; x += RUN_BLOCK) cp_async4(&keys[w.shift + x], g + x);
    cp_async_commit();
}

// Descent bitmask of the chunk from its staged window: bit k <-> position
// B + k (the end n counts as one).
__device__ __forceinline__ void bits_from_keys(const ChunkView& v, const KeyWindow& w, const uint32_t* keys,
                                               uint32_t* bits)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll 4
    for (int j = 0; j < RUN_LOADS; ++j) {
        const unsigned long long P = (unsigned long long)v.B + (unsigned)(j * RUN_BLOCK + tid);
        bool d = P == v.n;
        if (P < v.n && P > 0) {
            const uint32_t x = (uint32_t)P - w.W0 + w.shift;
            d = keys[x - 1] > keys[x];
        }
        const uint32_t word = __ballot_sync(FULL, d);
        if (lane == 0) bits[j * (RUN_BLOCK / 32) + warp] = word;
    }
}

// Bit p of the result: bits p .. p + 30 of x are all set.
__device__ __forceinline__ unsigned long long ones31(unsigned long long x)
{
    unsigned long long r = x & (x >> 1);   // runs of 2
    r &= r >> 2;                           // 4
    r &= r >> 4;                           // 8
    r &= r >> 8;                           // 16
    return r & (r >> 15);                  // 31
}

// The same bitmask from a precomputed descent mask (bit i <-> position i of
// the instance; records compare whole rows, which the keys cannot): chunks
// start at multiples of 32, so the chunk's words are whole mask words; the
// end n counts as a descent, positions past it as none.
__device__ __forceinline__ void bits_from_mask(const ChunkView& v, const uint32_t* mask, uint32_t* bits)
{
    for (int w = threadIdx.x; w < RUN_WORDS; w += RUN_BLOCK) {
        const unsigned long long P0 = (unsigned long long)v.B + 32u * (unsigned)w;
        uint32_t word = 0;
        if (P0 < v.n) word = mask[(P0 >> 5)];
        // clear positions >= n, then set position n
        if (P0 + 32 > v.n) {
            const uint32_t k = P0 < v.n ? (uint32_t)(v.n - P0) : 0u;   // positions of the word below n
            word &= k ? (0xffffffffu >> (32u - k)) : 0u;
            if (P0 <= v.n && v.n < P0 + 32) word |= 1u << (uint32_t)(v.n - P0);
        }
        if (P0 == 0) word &= ~1u;   // position 0 has no predecessor
        bits[w] = word;
    }
}

// Can any step from inside the chunk be natural?  Only if a run start s in
// the chunk is followed by minrun - 1 >= 31 positions without a descent (or,
// with decreasing runs, 31 positions with one).  Each thread looks for 31
// clear (or set) bits starting in its word (a 64-bit window over it and the
// next word); finding none proves every chain forced all the way, with a
// closed form.  Finding one only selects the exact chain walk.
__device__ __forceinline__ bool chunk_may_natural(const ChunkView& v, const uint32_t* bits, bool desc)
{
    const int tid = threadIdx.x;
    bool may = false;
    for (int w = tid; w < RUN_WORDS && w * 32 <= (int)v.span; w += RUN_BLOCK) {
        const unsigned long long hi = w + 1 < RUN_WORDS ? bits[w + 1] : 0u;
        const unsigned long long x = (unsigned long long)bits[w] | (hi << 32);
        unsigned long long r = ones31(~x);     // bit p set <=> bits p .. p + 30 clear
        if (desc) r |= ones31(x);              // ... or all set
        // run starts p = e + 1 with 1 <= p <= span (e = 0: the chunk's first position)
        uint32_t starts = (uint32_t)r;
        if (w == 0) starts &= ~1u;
        const uint32_t lo = (uint32_t)w * 32u;
        if (v.span - lo + 1u < 32u) starts &= (1u << (v.span - lo + 1u)) - 1u;
        may = may || starts != 0;
    }
    return __syncthreads_or(may) != 0;
}

// Natural end (chunk offset) of the run that starts at offset k < span, or
// KMAX when it lies past the halo.  An ascending run ends at the first descent
// (the end n carries a descent bit).  With decreasing runs, a run whose first
// pair descends ends at the first non-descent; n's bit is set, so the search
// is capped at n instead.
__device__ __forceinline__ int natural_end(const ChunkView& v, const uint32_t* bits, int k, bool desc)
{
    if (desc && (uint32_t)k + 1u < v.rem && desc_bit(bits, k + 1)) {
        const int e = next_clear(bits, k + 2, KMAX);
        return (uint32_t)e > v.rem ? (int)v.rem : e;
    }
    return next_desc(bits, k + 1, KMAX);
}

// Offset of entry state m: D0, the first descent at or after the chunk start;
// with decreasing runs X0, the first offset > 0 whose descent bit differs from
// offset 0's (capped at n).  KMAX (or beyond span) when outside the chunk.
__device__ __forceinline__ int natural_state_offset(const ChunkView& v, const uint32_t* bits, bool desc)
{
    if (!desc) return next_desc(bits, 0, KMAX);
    const int x = desc_bit(bits, 0) ? next_clear(bits, 1, KMAX) : next_desc(bits, 1, KMAX);
    return (uint32_t)x > v.rem ? (int)v.rem : x;
}

// Exit state of a chain that stopped at chunk offset k (or ran past the halo).
__device__ __forceinline__ uint32_t exit_state(const ChunkView& v, int k, bool symbolic)
{
    // the last chunk's chains all end at n; elsewhere the exit is an entry state
    // of the next chunk (a position past the next chunk's first minrun positions
    // can only be its D0 -- X0 with decreasing runs -- even when it is n)
    if (v.E == v.n) return STATE_END;
    if (symbolic) return v.m;
    const uint32_t x = (uint32_t)k - v.span;
    return x < v.m ? x : v.m;
}

// Start offset of the chain entered in state s (s < m: offset s; s = m: D0,
// or X0 with decreasing runs), or -1 when no run starts in the chunk from there.
__device__ __forceinline__ int entry_offset(const ChunkView& v, const uint32_t* bits, uint32_t s, bool desc)
{
    if (s < v.m) return (int)s;
    const int d0 = natural_state_offset(v, bits, desc);
    return (d0 >= KMAX || (uint32_t)d0 >= v.span) ? -1 : d0;
}

// Map entry of state s: (runs started in the chunk << 8) | exit state.
__device__ uint32_t chain_map(const ChunkView& v, const uint32_t* bits, uint32_t s, bool walk, bool desc)
{
    const int k0 = entry_offset(v, bits, s, desc);
    if (k0 < 0) return v.E == v.n ? STATE_END : v.m;
    if (!walk) {
        // forced steps only: starts k0, k0 + m, k0 + 2m, ... below span
        const uint32_t cnt = (uint32_t)k0 < v.span ? (v.span - (uint32_t)k0 + v.m - 1) / v.m : 0u;
        const uint32_t ex = v.E == v.n ? STATE_END : (uint32_t)k0 + cnt * v.m - v.span;   // < m
        return (cnt << 8) | ex;
    }
    uint32_t cnt = 0;
    int k = k0;
    bool symbolic = false;
    while ((uint32_t)k < v.span) {
        ++cnt;
        const int d = natural_end(v, bits, k, desc);
        if (d >= KMAX) { symbolic = true; break; }   // f = d = next chunk's D0 (X0)
        k = max(d, (int)min((uint32_t)k + v.m, v.rem));
    }
    return (cnt << 8) | exit_state(v, k, symbolic);
}

// One step of the scan: (runs so far << 8 | state) through map entry word f,
// where f already includes a restart when the chunk begins an instance.
__device__ __forceinline__ unsigned long long apply_map(unsigned long long at, const uint32_t* map, bool restart)
{
    const uint32_t st = (uint32_t)(at & 0xffu);
    const uint32_t f = map[st < (uint32_t)MAP_STATES ? st : 0u];
    const unsigned long long before = restart ? 0ull : (at >> 8);
    return ((before + ((f & RANGE_COUNT_MASK) >> 8)) << 8) | (f & 0xffu);
}

}  // namespace

// Pass 1: chunk maps, range maps, and (by the last CTA) the range entries.
__global__ void __launch_bounds__(RUN_BLOCK) k_runs(Job J)
{
    __shared__ __align__(16) uint32_t keys[2][WIN_SLOTS];   // double-buffered key windows
    __shared__ uint32_t bits[BITS_SLOTS];
    __shared__ uint32_t mapv[MAP_STATES];
    __shared__ uint32_t agg[MAP_STATES];     // (runs << 8 | state) after the range so far, per entry state
    __shared__ uint32_t s_last, s_reset;

    const int tid = threadIdx.x;
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    const uint32_t T = C->total_chunks, G = gridDim.x;
    const uint32_t K = (T + G - 1) / G;
    const uint32_t g0 = min(blockIdx.x * K, T), g1 = min(g0 + K, T);
    if (tid < MAP_STATES) agg[tid] = (uint32_t)tid;
    if (tid == 0) s_reset = 0;
    __syncthreads();

    uint32_t qi = NONE;
    ChunkView vn = {};
    KeyWindow wn = {};
    if (g0 < g1) {
        vn = chunk_view(J, g0, qi);
        wn = window_of(vn);
        if (!J.desc_mask) stage_keys(vn, wn, keys[0]);
    }
    for (uint32_t g = g0; g < g1; ++g) {
        const ChunkView v = vn;
        const KeyWindow w = wn;
        const int buf = (int)((g - g0) & 1u);
        // the next chunk's keys fly while this one is scanned
        if (g + 1 < g1) {
            vn = chunk_view(J, g + 1, qi);
            wn = window_of(vn);
            if (!J.desc_mask) {
                stage_keys(vn, wn, keys[buf ^ 1]);
                cp_async_wait<1>();
            }
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (J.desc_mask) bits_from_mask(v, J.desc_mask, bits);
        else bits_from_keys(v, w, keys[buf], bits);
        __syncthreads();
        const bool desc = J.desc_runs != 0;
        // the summaries by the last warp, which has no words to check in
        // chunk_may_natural (so they cost that barrier no time); published
        // by its barrier
        if (tid >= RUN_BLOCK - 32) bits_summary(bits);
        const bool walk = chunk_may_natural(v, bits, desc);
        if (tid <= (int)v.m) mapv[tid] = chain_map(v, bits, (uint32_t)tid, walk, desc);
        __syncthreads();
        // an instance's first chunk is entered at state 0 whatever came before:
        // its map is constant; states above m never occur and copy state m
        const bool first = v.c == 0;
        uint32_t f = 0;
        if (tid < MAP_STATES) f = first ? mapv[0] : mapv[min((uint32_t)tid, v.m)];
        if (tid == 0) {
            const int d0 = natural_state_offset(v, bits, desc);
            J.chunk_info[g] = (walk ? 0u : CHUNK_FORCED) | (first ? CHUNK_FIRST : 0u) | (uint32_t)min(d0, 0xffff);
            if (first) s_reset = RANGE_RESET;
        }
        __syncthreads();
        if (tid < MAP_STATES) {
            mapv[tid] = f;
            J.chunk_map[(size_t)g * MAP_STATES + tid] = f;
        }
        __syncthreads();
        if (tid < MAP_STATES) {
            // fold the chunk into the range map (a restart discards the runs before it)
            const uint32_t a = agg[tid], st = a & 0xffu;
            if (first || st < (uint32_t)MAP_STATES) {
                const uint32_t fm = mapv[first ? 0u : st];
                agg[tid] = (((first ? 0u : a >> 8) + (fm >> 8)) << 8) | (fm & 0xffu);
            }
        }
        __syncthreads();
    }
    if (tid < MAP_STATES) J.range_agg[(size_t)blockIdx.x * MAP_STATES + tid] = agg[tid] | s_reset;

    // The range entries in two levels.  The last CTA of every group of 32
    // ranges folds the group's range maps into one map (a lane per two entry
    // states); the last of those walks the group maps in order and writes
    // each group's entry (runs before it << 8 | state).  Every range's own
    // entry follows in k_runs_emit from its group's entry and the maps of
    // the ranges before it in the group.
    constexpr uint32_t GROUP = 32;
    static_assert(RUN_RANGES_MAX <= GROUP * 32, "at most 32 groups");
    static_assert(GROUP * MAP_STATES <= 2 * WIN_SLOTS, "a group's maps fit the key windows");
    uint32_t (*win)[MAP_STATES] = reinterpret_cast<uint32_t (*)[MAP_STATES]>(&keys[0][0]);
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t grp = blockIdx.x / GROUP, ngroups = (G + GROUP - 1) / GROUP;
    const uint32_t gsize = min(GROUP, G - grp * GROUP);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&C->runs_grp_done[grp], 1u) == gsize - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (uint32_t i = tid; i < gsize * MAP_STATES; i += RUN_BLOCK)
        win[i / MAP_STATES][i % MAP_STATES] = __ldcg(J.range_agg + (size_t)grp * GROUP * MAP_STATES + i);
    __syncthreads();
    if (warp == 0) {
        bool reset = false;
        for (int h = 0; h < 2; ++h) {
            const uint32_t s0 = (uint32_t)lane + 32u * h;
            unsigned long long a = s0;
            for (uint32_t q = 0; q < gsize; ++q) {
                const bool rq = (win[q][0] & RANGE_RESET) != 0;
                a = apply_map(a, win[q], rq);
                reset = reset || rq;
            }
            J.run_grp_agg[(size_t)grp * MAP_STATES + s0] =
                (uint32_t)(a & 0xffu) | (uint32_t)((a >> 8) << 8) | (reset ? RANGE_RESET : 0u);
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&C->runs_done, 1u) == ngroups - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (uint32_t i = tid; i < ngroups * MAP_STATES; i += RUN_BLOCK)
        win[i / MAP_STATES][i % MAP_STATES] = __ldcg(J.run_grp_agg + i);
    __syncthreads();
    if (tid == 0) {
        unsigned long long at = 0;               // range 0 begins chunk 0: state 0, no runs before
        for (uint32_t q = 0; q < ngroups; ++q) {
            J.range_entry[q] = at;
            at = apply_map(at, win[q], (win[q][0] & RANGE_RESET) != 0);
        }
    }
}

// Pass 2: every CTA walks its range's chunk maps from the range entry and
// writes the run starts of each chunk: a warp per chunk in closed form when
// every step in it is forced; otherwise the whole CTA rebuilds the chunk's
// descent bitmask (from the keys, as pass 1 did, or from the record mask)
// and one thread walks the one chain the chunk takes.  Rebuilding reads the
// chunk's keys a second time instead of keeping every bitmask between the
// passes (RUN_WORDS words per chunk, an eighth of the keys' size).
__global__ void __launch_bounds__(RUN_BLOCK) k_runs_emit(Job J)
{
    constexpr int NW = RUN_BLOCK / 32;
    __shared__ __align__(16) uint32_t keys[WIN_SLOTS];   // one chunk's key window
    __shared__ uint32_t bits[BITS_SLOTS];
    __shared__ uint32_t win[WIN][MAP_STATES];
    __shared__ unsigned long long entry[WIN];    // runs before the chunk << 8 | its entry state

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    const uint32_t T = C->total_chunks, G = gridDim.x;
    const uint32_t K = (T + G - 1) / G;
    const uint32_t g0 = min(blockIdx.x * K, T), g1 = min(g0 + K, T);
    // this range's entry: its group's, through the maps of the ranges before
    // it in the group (staged in the chunk-map window)
    __shared__ unsigned long long s_at;
    {
        constexpr uint32_t GROUP = 32;
        static_assert(WIN >= (int)GROUP, "a group's range maps fit the window");
        const uint32_t q0 = blockIdx.x / GROUP * GROUP, nq = blockIdx.x - q0;
        for (uint32_t i = tid; i < nq * MAP_STATES; i += RUN_BLOCK)
            win[i / MAP_STATES][i % MAP_STATES] = __ldcg(J.range_agg + (size_t)q0 * MAP_STATES + i);
        __syncthreads();
        if (tid == 0) {
            unsigned long long a = __ldcg(J.range_entry + blockIdx.x / GROUP);
            for (uint32_t q = 0; q < nq; ++q) a = apply_map(a, win[q], (win[q][0] & RANGE_RESET) != 0);
            s_at = a;
        }
        __syncthreads();
    }
    unsigned long long at = s_at;
    const bool desc = J.desc_runs != 0;

    // the run starts of chunk g, from its map entry: count checks, and the
    // instance's end after its last chunk
    auto finish_chunk = [&](const ChunkView& v, uint32_t me, unsigned long long prefix, uint32_t cnt) {
        const Inst& I = J.inst[v.qi];
        const unsigned long long cap = (unsigned long long)(v.n / 32) + 2;
        if (v.c + 1 == I.nchunks) {
            const unsigned long long R = prefix + cnt;
            if ((me & 0xffu) != STATE_END || R + 1 > cap) {
                set_error(C, DERR_INTERNAL, 12);
            } else {
                J.run_start[I.run_base + R] = v.n;
                J.inst[v.qi].runs = (uint32_t)R;
            }
        }
    };

    uint32_t qb = NONE;                          // the block's instance cursor (walked chunks)
    for (uint32_t b0 = g0; b0 < g1; b0 += WIN) {
        const uint32_t nb = min((uint32_t)WIN, g1 - b0);
        for (uint32_t i = tid; i < nb * MAP_STATES; i += RUN_BLOCK)
            win[i / MAP_STATES][i % MAP_STATES] = J.chunk_map[(size_t)b0 * MAP_STATES + i];
        __syncthreads();
        if (tid == 0) {
            for (uint32_t i = 0; i < nb; ++i) {
                const bool first = (J.chunk_info[b0 + i] & CHUNK_FIRST) != 0;
                if (first) at = 0;               // an instance starts: state 0, no runs before
                entry[i] = at;
                at = apply_map(at, win[i], first);
            }
        }
        __syncthreads();
        // forced-only chunks: one warp per chunk, in closed form
        uint32_t qi = NONE;
        for (uint32_t i = warp; i < nb; i += NW) {
            const uint32_t g = b0 + i;
            const uint32_t info = J.chunk_info[g];
            if (!(info & CHUNK_FORCED)) continue;
            const ChunkView v = chunk_view(J, g, qi);
            const Inst& I = J.inst[v.qi];
            const uint32_t st = (uint32_t)(entry[i] & 0xffu);
            const unsigned long long prefix = entry[i] >> 8;
            const uint32_t me = win[i][st < (uint32_t)MAP_STATES ? st : 0u];
            const uint32_t cnt = (me & RANGE_COUNT_MASK) >> 8;
            uint32_t* rs = J.run_start + I.run_base + prefix;
            const unsigned long long cap = (unsigned long long)(v.n / 32) + 2;
            if (st > v.m || prefix + cnt + 1 > cap || cnt > (uint32_t)RUN_REC) {
                if (lane == 0) set_error(C, DERR_INTERNAL, 13);
                continue;
            }
            // starts k0, k0 + m, ... (k0: the entry offset or D0 / X0)
            const uint32_t d0 = info & 0xffffu;
            const uint32_t k0 = st < v.m ? st : d0;
            for (uint32_t x = lane; x < cnt; x += 32) rs[x] = v.B + k0 + x * v.m;
            if (lane == 0) finish_chunk(v, me, prefix, cnt);
        }
        // chunks with a natural step: the whole block, one chunk at a time
        for (uint32_t i = 0; i < nb; ++i) {
            const uint32_t g = b0 + i;
            if (J.chunk_info[g] & CHUNK_FORCED) continue;   // the same for every thread
            const ChunkView v = chunk_view(J, g, qb);
            if (J.desc_mask) {
                bits_from_mask(v, J.desc_mask, bits);
            } else {
                const KeyWindow w = window_of(v);
                stage_keys(v, w, keys);
                cp_async_wait<0>();
                __syncthreads();
                bits_from_keys(v, w, keys, bits);
            }
            __syncthreads();
            if (tid < 32) bits_summary(bits);    // thread 0, which walks, wrote it
            if (tid == 0) {
                const Inst& I = J.inst[v.qi];
                const uint32_t st = (uint32_t)(entry[i] & 0xffu);
                const unsigned long long prefix = entry[i] >> 8;
                const uint32_t me = win[i][st < (uint32_t)MAP_STATES ? st : 0u];
                const uint32_t cnt = (me & RANGE_COUNT_MASK) >> 8;
                uint32_t* rs = J.run_start + I.run_base + prefix;
                const unsigned long long cap = (unsigned long long)(v.n / 32) + 2;
                if (st > v.m || prefix + cnt + 1 > cap || cnt > (uint32_t)RUN_REC) {
                    set_error(C, DERR_INTERNAL, 13);
                } else {
                    uint32_t c2 = 0;
                    int k = entry_offset(v, bits, st, desc);
                    if (k >= 0) {
                        while ((uint32_t)k < v.span && c2 < cnt) {
                            rs[c2++] = v.B + (uint32_t)k;
                            const int d = natural_end(v, bits, k, desc);
                            if (d >= KMAX) break;
                            k = max(d, (int)min((uint32_t)k + v.m, v.rem));
                        }
                    }
                    if (c2 != cnt) set_error(C, DERR_INTERNAL, 14);
                    finish_chunk(v, me, prefix, cnt);
                }
            }
            __syncthreads();                     // the window and bitmask are free again
        }
        __syncthreads();
    }
}

cudaError_t launch_setup(const Job& J, cudaStream_t s)
{
    k_setup<<<1, 1024, 0, s>>>(J);
    return cudaGetLastError();
}

cudaError_t launch_runs(const Job& J, int grid, cudaStream_t s)
{
    k_runs<<<grid, RUN_BLOCK, 0, s>>>(J);
    k_runs_emit<<<grid, RUN_BLOCK, 0, s>>>(J);
    return cudaGetLastError();
}

}  // namespace ps
