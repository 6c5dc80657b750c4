// HBM merges: the merges of Algorithm 1 whose inputs exceed the tile size,
// executed as stable out-of-place merges (Algorithm 2, StandardMerge: ties
// take the left run) between the caller's arrays and the scratch arrays
// (Pingpong storage, Sec. 3).
//
// Every merge is cut into chunks of E outputs (E = the kernel shape's consumer
// threads x MERGE_K).  Chunks are numbered
// round by round (rounds go from the largest power to the smallest), so a
// merge's children always carry smaller chunk numbers than the merge itself.
// One persistent launch processes every chunk as a dataflow,
// without grid-wide barriers: a merge starts as soon as both of its children
// are complete, while other merges of the previous round may still run.
//
//   dep[e]  chunks of merge e's HBM children not yet written (set by the
//           planning kernels; children that are tiles are finished before the
//           launch).  Whoever writes a chunk decrements its parent's counter
//           once the chunk has reached global memory.
//
// A CTA has three roles.
//   Search warp: NSEARCH lanes, each holding one chunk.  A lane claims the
//     next chunk number (one global ticket, so chunks are claimed in order),
//     waits until the chunk's merge has dep = 0, and finds the merge-path
//     splits of the chunk's first and last output (how many of the merge's
//     first d outputs come from the left child: the largest i with
//     A[i-1] <= B[d-i], ties to the left).  All lanes run one loop in which
//     each advances its own chunk by one step per iteration (one probe of each
//     of its two binary searches), so the probes of different chunks overlap.
//     A prepared chunk goes into the lane's slot of a shared-memory ring.
//   Producer warp: takes the prepared chunk with the smallest number, waits
//     for a free shared-memory stage (an "empty" mbarrier), starts the 1-D
//     bulk copies (cp.async.bulk, TMA) of the chunk's two input slices (keys
//     and permutation) and loads the elements outside the slices'
//     16-byte-aligned interiors (at most three at each end) with ordinary
//     loads; the stage's "full" mbarrier completes when both have landed.
//   Consumer warps (BLOCK / 32 of them): merge a full stage into the output
//     staging arrays (each thread MERGE_K consecutive outputs: merge-path
//     split inside shared memory, then a branch-free serial merge), release
//     it, and write the chunk back: the aligned interior by a bulk store, the
//     ends by ordinary stores.  One chunk later, or as soon as the CTA has
//     nothing to merge, the store is known to be complete and the parent's
//     counter drops.
//
// Progress: chunks are claimed in increasing order and wait only for smaller
// chunk numbers, so the smallest unfinished chunk always has its inputs
// complete; every written chunk is announced (at the latest when its CTA goes
// idle).  A CTA claims chunks only while it runs and leaves only when it
// holds none, so every chunk a running CTA waits for is held by a running CTA:
// progress needs no co-residency, and the kernel is an ordinary launch.  CTAs
// that cannot start yet (the SMs busy with another stream's kernels, as in
// the server) start later or find no chunk left; nothing waits for them.
// Every wait is bounded and records DERR_TIMEOUT instead of hanging.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL_MASK = 0xffffffffu;
constexpr int EDGE_SLOTS = 8;        // unaligned elements of one slice (<= 7)
constexpr int MERGE_K = 9;           // outputs per consumer thread (odd: conflict-free strides)
#ifndef PS_MERGE_NSEARCH
#define PS_MERGE_NSEARCH 16
#endif
constexpr int NSEARCH = PS_MERGE_NSEARCH;         // chunks a CTA prepares ahead (<= 32)
static_assert(NSEARCH >= 1 && NSEARCH <= 32, "one search warp");

// The kernel's shape: NST shared-memory stages, BLOCK consumer threads (each
// MERGE_K outputs of a chunk of E = BLOCK x MERGE_K), one producer warp and
// one search warp.
template <int NST, int BLOCK>
struct Shape {
    static constexpr int E = BLOCK * MERGE_K;
    static constexpr int SLOT = E + 16;           // a staged array: up to 3 + 3 + 3 shift slots
    static constexpr int NCONS = BLOCK / 32;      // consumer warps
    static constexpr int PRODUCER_WARP = NCONS;
    static constexpr int SEARCH_WARP = NCONS + 1;
    static constexpr int MTHREADS = BLOCK + 64;
};

constexpr uint32_t RS_EMPTY = 0, RS_FULL = 1, RS_END = 2;   // ring slot states

// A chunk whose inputs are complete and whose splits are known.
struct Prep {
    GSorted g;             // its merge
    uint32_t c;            // chunk number
    uint32_t a0, a1;       // left-child elements before its first / after its last output
    uint32_t round;
    unsigned long long t_ready;   // globaltimer when its inputs were found complete
};

// A contiguous slice of one array: its 16-byte-aligned interior moves by
// bulk copy, the rest (head / tail, at most 3 elements each, or the whole
// slice when it has no aligned 16-byte block) by ordinary accesses.
struct Slice {
    uint32_t head;    // elements before the aligned interior (or the whole slice)
    uint32_t nint;    // elements of the aligned interior (multiple of 4)
    uint32_t len;
};

__device__ __forceinline__ Slice slice_of(const uint32_t* g, uint32_t len)
{
    Slice s;
    s.len = len;
    const uint32_t mis = (uint32_t)(((uintptr_t)g >> 2) & 3u);     // elements past a 16-byte boundary
    const uint32_t head = (4u - mis) & 3u;
    if (len > head) {
        s.head = head;
        s.nint = (len - head) & ~3u;
    } else {
        s.head = len;
        s.nint = 0;
    }
    if (s.nint == 0) s.head = len;
    return s;
}

// index inside the slice of unaligned element number j (j < EDGE_SLOTS), or NONE
__device__ __forceinline__ uint32_t edge_index(const Slice& s, uint32_t j)
{
    if (j < s.head) return j;
    const uint32_t i = s.head + s.nint + (j - s.head);
    return i < s.len ? i : NONE;
}

// shared-memory slot of a slice start: congruent to its global address mod 16
__device__ __forceinline__ uint32_t shift_of(const uint32_t* g)
{
    return (uint32_t)(((uintptr_t)g >> 2) & 3u);
}

struct Stage {
    const uint32_t* gk[2];   // slice starts in global memory: [0] left, [1] right (keys)
    const uint32_t* gp[2];   // same for the permutation (nullptr: keys only)
    uint32_t sk[2], sp[2];   // slice starts inside the staged arrays
    Slice slk[2], slp[2];
    uint32_t na, nb;
    uint32_t* ok;            // output chunk start (keys, permutation)
    uint32_t* op;
    uint32_t sok, sop;       // output start inside the output staging arrays
    Slice osk, osp;          // the output chunk (keys, permutation) as slices
    uint32_t cnt;
    uint32_t parent;         // the merge's parent (GSorted index; NONE for a root)
    uint32_t round;
    uint32_t last;           // nonzero: no chunk; the CTA's work is over
    unsigned long long t_ready;
};

// Per-round timeline kept in shared memory by consumer thread 0 and merged
// into the counters whenever the round of its chunks changes (a CTA receives
// its chunks in increasing order).
struct Timeline {
    unsigned long long ready_min, ready_max, done_min, done_max;
    uint32_t round;
};

template <int NST, int BLOCK>
struct __align__(16) MergeSmem {
    static constexpr int SLOT = Shape<NST, BLOCK>::SLOT;
    uint32_t in_k[NST][SLOT];
    uint32_t in_p[NST][SLOT];
    uint32_t out_k[SLOT];
    uint32_t out_p[SLOT];
    uint64_t full[NST];      // producer -> consumers: the stage holds a chunk
    uint64_t empty[NST];     // consumers -> producer: the stage may be refilled
    Stage st[NST];
    Prep ring[NSEARCH];      // search lane l -> producer
    uint32_t ring_state[NSEARCH];
    uint32_t round_chunk[NPOW + 1];   // first chunk of every round; [NPOW] = all chunks
    uint32_t err;
    uint32_t pend;           // consumer thread 0: parent of the written, unannounced chunk
    Timeline tl;
};

// 228 KiB of shared memory per SM, 1 KiB of it reserved per CTA
// CTAs per SM the stages leave room for (228 KiB of shared memory per SM,
// 1 KiB of it reserved per CTA), at most 4
template <int NST, int BLOCK>
constexpr int merge_min_ctas()
{
    return 233472 / (int)(sizeof(MergeSmem<NST, BLOCK>) + 1024) < 4
               ? 233472 / (int)(sizeof(MergeSmem<NST, BLOCK>) + 1024)
               : 4;
}

__device__ __forceinline__ uint32_t ld_vol(const uint32_t* p)
{
    return *(const volatile uint32_t*)p;
}

__device__ __forceinline__ void st_vol(uint32_t* p, uint32_t v)
{
    *(volatile uint32_t*)p = v;
}

// Producer lane 0: the stage's addresses for a prepared chunk (chunks of E outputs).
template <int E>
__device__ void describe(const Job& J, const Prep& p, Stage& S)
{
    const GSorted& g = p.g;
    const uint32_t total = g.la + g.lb;
    const uint32_t d0 = (p.c - g.chunk_base) * E;
    const uint32_t d1 = min(d0 + (uint32_t)E, total);
    const uint32_t a0 = p.a0, a1 = p.a1;
    const uint32_t b0 = d0 - a0, b1 = d1 - a1;
    const bool src_b = ((g.depth + 1) & 1u) != 0, dst_b = (g.depth & 1u) != 0;
    const uint32_t* ks = (src_b ? J.keysB : J.keysA) + g.goff;
    const uint32_t* ps = J.want_perm ? (src_b ? J.permB : J.permA) + g.goff : nullptr;
    S.na = a1 - a0;
    S.nb = b1 - b0;
    S.cnt = d1 - d0;
    S.gk[0] = ks + a0;
    S.gk[1] = ks + g.la + b0;
    S.gp[0] = ps ? ps + a0 : nullptr;
    S.gp[1] = ps ? ps + g.la + b0 : nullptr;
    S.sk[0] = shift_of(S.gk[0]);
    S.sk[1] = ((S.sk[0] + S.na + 3u) & ~3u) + shift_of(S.gk[1]);
    S.slk[0] = slice_of(S.gk[0], S.na);
    S.slk[1] = slice_of(S.gk[1], S.nb);
    S.sp[0] = S.sp[1] = 0;
    if (ps) {
        S.sp[0] = shift_of(S.gp[0]);
        S.sp[1] = ((S.sp[0] + S.na + 3u) & ~3u) + shift_of(S.gp[1]);
        S.slp[0] = slice_of(S.gp[0], S.na);
        S.slp[1] = slice_of(S.gp[1], S.nb);
    }
    S.ok = (dst_b ? J.keysB : J.keysA) + g.goff + d0;
    S.op = J.want_perm ? (dst_b ? J.permB : J.permA) + g.goff + d0 : nullptr;
    S.sok = shift_of(S.ok);
    S.sop = S.op ? shift_of(S.op) : 0u;
    S.osk = slice_of(S.ok, S.cnt);
    S.osp = S.op ? slice_of(S.op, S.cnt) : Slice{0u, 0u, 0u};
    S.parent = g.parent;
    S.round = p.round;
    S.t_ready = p.t_ready;
}

__device__ __forceinline__ bool aligned16(const void* p)
{
    return (((uintptr_t)p) & 15u) == 0;
}

// Producer lane 0: announce the stage's bytes and start its bulk copies.
template <int NST, int BLOCK>
__device__ void issue_loads(MergeSmem<NST, BLOCK>& sm, int s, Ctr* C)
{
    const Stage& S = sm.st[s];
    uint32_t bytes = 0;
    const void* src[4];
    void* dst[4];
    uint32_t sz[4];
    int k = 0;
    for (int side = 0; side < 2; ++side) {
        const Slice& a = S.slk[side];
        if (a.nint) {
            src[k] = S.gk[side] + a.head;
            dst[k] = &sm.in_k[s][S.sk[side] + a.head];
            sz[k] = a.nint * 4u;
            ++k;
        }
        if (S.gp[side]) {
            const Slice& b = S.slp[side];
            if (b.nint) {
                src[k] = S.gp[side] + b.head;
                dst[k] = &sm.in_p[s][S.sp[side] + b.head];
                sz[k] = b.nint * 4u;
                ++k;
            }
        }
    }
    bool ok = true;
    for (int i = 0; i < k; ++i) {
        ok = ok && aligned16(src[i]) && aligned16(dst[i]) && (sz[i] & 15u) == 0;
        bytes += sz[i];
    }
    if (!ok) {                       // never expected: report, copy nothing
        set_error(C, DERR_INTERNAL, 41);
        k = 0;
        bytes = 0;
    }
    fence_proxy_async_smem();        // earlier generic accesses of this stage come first
    mbar_arrive_expect_tx(&sm.full[s], bytes);
    for (int i = 0; i < k; ++i) tma_load_1d(dst[i], src[i], sz[i], &sm.full[s]);
}

// Producer lane l: the unaligned element l % 8 of slice l / 8 (0: left
// keys, 1: right keys, 2: left perm, 3: right perm) goes into the stage.
// Loads bypass L1: the data were written by other SMs during this launch.
template <int NST, int BLOCK>
__device__ __forceinline__ void copy_edge(MergeSmem<NST, BLOCK>& sm, int s, int lane)
{
    const Stage& S = sm.st[s];
    const int which = lane >> 3, j = lane & 7;
    const int side = which & 1;
    const bool is_perm = which >= 2;
    if (is_perm && !S.gp[side]) return;
    const Slice& sl = is_perm ? S.slp[side] : S.slk[side];
    const uint32_t i = edge_index(sl, (uint32_t)j);
    if (i == NONE) return;
    if (is_perm) sm.in_p[s][S.sp[side] + i] = __ldcg(S.gp[side] + i);
    else sm.in_k[s][S.sk[side] + i] = __ldcg(S.gk[side] + i);
}

__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, Ctr* C, uint32_t where)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > SPIN_LIMIT_CYCLES) {
            set_error(C, DERR_TIMEOUT, where);
            return false;
        }
    }
    return true;
}

template <int BLOCK>
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(BLOCK) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// every committed bulk store but the most recent group has completed
__device__ __forceinline__ void bulk_wait_all_but_one()
{
    asm volatile("cp.async.bulk.wait_group 1;" ::: "memory");
}

// The chunk written before has reached global memory (its bulk store
// completed, its edge stores precede a warp barrier this thread passed):
// make it visible and count it off the parent's dependencies.
__device__ __forceinline__ void announce(const Job& J, uint32_t parent)
{
    fence_proxy_async_global();
    __threadfence();
    atomicSub(&J.dep[parent], 1u);
}

__device__ void timeline_reset(Timeline& t)
{
    t.round = NONE;
    t.ready_min = t.done_min = ~0ull;
    t.ready_max = t.done_max = 0;
}

__device__ void timeline_flush(Timeline& t, Ctr* C)
{
    if (t.round == NONE) return;
    atomicMin(&C->round_ns[t.round][0], t.ready_min);
    atomicMax(&C->round_ns[t.round][1], t.ready_max);
    atomicMin(&C->round_ns[t.round][2], t.done_min);
    atomicMax(&C->round_ns[t.round][3], t.done_max);
    timeline_reset(t);
}

__device__ void timeline_note(Timeline& t, Ctr* C, uint32_t r, unsigned long long t_ready, unsigned long long t_done)
{
    if (r != t.round) {
        timeline_flush(t, C);
        t.round = r;
    }
    t.ready_min = min(t.ready_min, t_ready);
    t.ready_max = max(t.ready_max, t_ready);
    t.done_min = min(t.done_min, t_done);
    t.done_max = max(t.done_max, t_done);
}

// ---------------------------------------------------------------- roles

template <int NST, int BLOCK>
__device__ __noinline__ void search_warp(const Job& J, MergeSmem<NST, BLOCK>& sm, Ctr* C)
{
    // Each iteration a lane issues the one global access its state needs and
    // takes the result at the end of the iteration, so the accesses of all
    // lanes overlap.
    enum : uint32_t { S_CLAIM, S_NODE, S_INFO, S_WAIT, S_SEARCH, S_PUB, S_DONE };
    const int lane = threadIdx.x & 31;
    const uint32_t total_chunks = sm.round_chunk[NPOW];
    // Lanes in use: about one round's share of chunks per CTA (at least 2, at
    // most NSEARCH), so that when a round has few chunks the first claims
    // still spread it over every CTA instead of filling the first ones.
    uint32_t rounds = 0;
    for (int r = 0; r < NPOW; ++r) rounds += sm.round_chunk[r + 1] > sm.round_chunk[r] ? 1u : 0u;
    const uint32_t share = rounds ? (total_chunks + rounds * gridDim.x - 1) / (rounds * gridDim.x) : 0u;
    const uint32_t cap = J.merge_lanes ? min(J.merge_lanes, (uint32_t)NSEARCH) : (uint32_t)NSEARCH;
    const int lanes = (int)min(cap, max(min(2u, cap), share));
    uint32_t state = lane < lanes ? S_CLAIM : S_DONE;
    if (lane >= lanes && lane < NSEARCH) st_vol(&sm.ring_state[lane], RS_END);
    uint32_t c = 0, e = 0, d0 = 0, d1 = 0, round = 0;
    GSorted g = {};
    uint32_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
    long long t_wait = 0;
    unsigned long long t_ready = 0;
    uint32_t gap = 1, next_poll = 0;     // a waiting lane polls every gap iterations (1, then 2)
    for (uint32_t iter = 0;; ++iter) {
        // ---- issue
        const uint32_t want = __ballot_sync(FULL_MASK, state == S_CLAIM);
        const int leader = want ? __ffs(want) - 1 : 0;
        uint32_t base = 0;
        if (want && lane == leader) base = atomicAdd(&C->chunk_next[0], (uint32_t)__popc(want));
        uint32_t e_new = 0;
        if (state == S_NODE) e_new = __ldcg(J.chunk_node + c);
        GSorted g_new = {};
        if (state == S_INFO) g_new = J.gsorted[e];
        const bool poll = state == S_WAIT && iter >= next_poll;
        uint32_t depv = 1;
        if (poll) depv = ld_acquire_u32(&J.dep[e]);
        const bool s0 = state == S_SEARCH && lo0 < hi0, s1 = state == S_SEARCH && lo1 < hi1;
        const uint32_t m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
        uint32_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
        const uint32_t* A = (((g.depth + 1) & 1u) ? J.keysB : J.keysA) + g.goff;
        if (s0) {
            x0 = __ldcg(A + m0);
            y0 = __ldcg(A + g.la + (d0 - 1u - m0));
        }
        if (s1) {
            x1 = __ldcg(A + m1);
            y1 = __ldcg(A + g.la + (d1 - 1u - m1));
        }
        const bool pub_free = state == S_PUB && ld_vol(&sm.ring_state[lane]) == RS_EMPTY;
        // ---- take the results
        if (want) base = __shfl_sync(FULL_MASK, base, leader);
        if (state == S_CLAIM) {
            c = base + (uint32_t)__popc(want & ((1u << lane) - 1u));
            if (c < total_chunks) {
                state = S_NODE;
            } else {
                state = S_DONE;
                st_vol(&sm.ring_state[lane], RS_END);
            }
        } else if (state == S_NODE) {
            e = e_new;
            state = S_INFO;
        } else if (state == S_INFO) {
            g = g_new;
            d0 = (c - g.chunk_base) * Shape<NST, BLOCK>::E;
            d1 = min(d0 + (uint32_t)Shape<NST, BLOCK>::E, g.la + g.lb);
            uint32_t lo = 0, hi = NPOW;              // last round starting at or before c
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sm.round_chunk[mid] <= c) lo = mid; else hi = mid;
            }
            round = lo;
            state = S_WAIT;
            t_wait = clock64();
            gap = 1;
            next_poll = iter + 1;
        } else if (poll) {
            if (depv == 0u) {
                lo0 = d0 > g.lb ? d0 - g.lb : 0u;
                hi0 = min(d0, g.la);
                lo1 = d1 > g.lb ? d1 - g.lb : 0u;
                hi1 = min(d1, g.la);
                t_ready = globaltimer_ns();
                state = S_SEARCH;
            } else if (clock64() - t_wait > SPIN_LIMIT_CYCLES) {
                set_error(C, DERR_TIMEOUT, 45);
                state = S_DONE;
                st_vol(&sm.ring_state[lane], RS_END);
            } else {
                next_poll = iter + gap;
                gap = 2u;
            }
        } else if (state == S_SEARCH) {
            if (s0) {
                if (x0 <= y0) lo0 = m0 + 1u; else hi0 = m0;
            }
            if (s1) {
                if (x1 <= y1) lo1 = m1 + 1u; else hi1 = m1;
            }
            if (lo0 >= hi0 && lo1 >= hi1) {      // splits: lo0, lo1
                Prep& p = sm.ring[lane];
                p.g = g;
                p.c = c;
                p.a0 = lo0;
                p.a1 = lo1;
                p.round = round;
                p.t_ready = t_ready;
                __threadfence_block();
                st_vol(&sm.ring_state[lane], RS_FULL);
                state = S_PUB;
            }
        } else if (pub_free) {
            state = S_CLAIM;
        }
        if (__all_sync(FULL_MASK, state == S_DONE)) break;
        // lane 0 decides for the warp, which must leave the loop together
        uint32_t stop = 0;
        if (lane == 0 && (iter & 63u) == 63u) stop = *(volatile uint32_t*)&C->error;
        if (__shfl_sync(FULL_MASK, stop, 0)) {
            if (lane < NSEARCH) st_vol(&sm.ring_state[lane], RS_END);
            break;
        }
        const bool moving = state == S_CLAIM || state == S_NODE || state == S_INFO || state == S_SEARCH;
        if (!__any_sync(FULL_MASK, moving)) __nanosleep(64);
    }
}

template <int NST, int BLOCK>
__device__ __noinline__ void producer_warp(const Job& J, MergeSmem<NST, BLOCK>& sm, Ctr* C)
{
    const int lane = threadIdx.x & 31;
    uint32_t k = 0;                      // stages filled so far (stage k % NST)
    long long t_idle = clock64();
    for (;;) {
        // the prepared chunk with the smallest number
        const uint32_t rs = lane < NSEARCH ? ld_vol(&sm.ring_state[lane]) : RS_END;
        __threadfence_block();
        const uint32_t key = rs == RS_FULL ? sm.ring[lane].c : 0xffffffffu;
        const uint32_t m = __reduce_min_sync(FULL_MASK, key);
        if (m == 0xffffffffu) {
            if (__all_sync(FULL_MASK, rs == RS_END)) break;
            // lane 0 decides for the warp, which must leave the loop together
            uint32_t stop = 0;
            if (lane == 0) {
                if (*(volatile uint32_t*)&C->error) {
                    stop = 1;
                } else if (clock64() - t_idle > SPIN_LIMIT_CYCLES) {
                    set_error(C, DERR_TIMEOUT, 46);
                    stop = 1;
                }
            }
            if (__shfl_sync(FULL_MASK, stop, 0)) break;
            __nanosleep(32);
            continue;
        }
        t_idle = clock64();
        const int src = __ffs(__ballot_sync(FULL_MASK, key == m)) - 1;
        const int s = (int)(k % NST);
        if (k >= (uint32_t)NST && !mbar_wait_bounded(&sm.empty[s], ((k / NST) - 1u) & 1u, C, 44)) return;
        ++k;
        if (lane == 0) {
            const Prep p = sm.ring[src];
            __threadfence_block();
            st_vol(&sm.ring_state[src], RS_EMPTY);
            sm.st[s].last = 0;
            describe<Shape<NST, BLOCK>::E>(J, p, sm.st[s]);
            fence_proxy_async_global();   // the inputs were written by other CTAs' bulk stores
            issue_loads<NST, BLOCK>(sm, s, C);
        }
        __syncwarp();
        copy_edge<NST, BLOCK>(sm, s, lane);
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.full[s]);
    }
    // close the consumers' loop with a stage that carries no chunk
    const int s = (int)(k % NST);
    if (k >= (uint32_t)NST && !mbar_wait_bounded(&sm.empty[s], ((k / NST) - 1u) & 1u, C, 47)) return;
    if (lane == 0) {
        sm.st[s].last = 1;
        sm.st[s].cnt = 0;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&sm.full[s], 0);
        mbar_arrive(&sm.full[s]);
    }
    __syncwarp();
}

template <int NST, int BLOCK>
__device__ __noinline__ void consumer_warps(const Job& J, MergeSmem<NST, BLOCK>& sm, Ctr* C)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool perm = J.want_perm != 0;
    uint32_t u = 0;                      // stages taken so far (stage u % NST)
    if (tid == 0) {
        sm.pend = NONE;
        timeline_reset(sm.tl);
    }
    for (;;) {
        const int s = (int)(u % NST);
        const uint32_t parity = (u / NST) & 1u;
        if (!mbar_test_wait(&sm.full[s], parity)) {
            // nothing to merge yet: announce the last chunk before waiting
            if (tid == 0 && sm.pend != NONE) {
                bulk_wait_all();
                announce(J, sm.pend);
                sm.pend = NONE;
            }
            if (!mbar_wait_bounded(&sm.full[s], parity, C, 42)) break;
        }
        ++u;
        const Stage& S = sm.st[s];
        if (S.last) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[s]);
            break;
        }
        const uint32_t na = S.na, nb = S.nb, cnt = S.cnt;
        const uint32_t sok = S.sok, sop = S.sop;
        const uint32_t* Ak = &sm.in_k[s][S.sk[0]];
        const uint32_t* Bk = &sm.in_k[s][S.sk[1]];
        const uint32_t* Ap = &sm.in_p[s][S.sp[0]];
        const uint32_t* Bp = &sm.in_p[s][S.sp[1]];
        // the split of this thread's outputs reads only the stage, so it runs
        // while the previous chunk's store may still be reading the output
        // staging arrays
        const uint32_t x0 = tid * MERGE_K;
        uint32_t ia = 0, ib = 0, va = 0, vb = 0;
        if (x0 < cnt) {
            uint32_t lo = x0 > nb ? x0 - nb : 0u, hi = min(x0, na);
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (Ak[mid] <= Bk[x0 - 1 - mid]) lo = mid + 1; else hi = mid;
            }
            ia = lo;
            ib = x0 - lo;
            va = ia < na ? Ak[ia] : 0xffffffffu;
            vb = ib < nb ? Bk[ib] : 0xffffffffu;
        }
        if (tid == 0) bulk_wait_read_all();         // the previous output has left the staging arrays
        consumers_sync<BLOCK>();
        if (x0 < cnt) {
            uint32_t* outk = &sm.out_k[sok + x0];
            uint32_t* outp = &sm.out_p[sop + x0];
            const uint32_t nout = min(cnt - x0, (uint32_t)MERGE_K);
            // branch-free serial merge straight into the staging arrays; an
            // exhausted side is read at slot 0 (a valid address whose value is
            // never used)
#pragma unroll
            for (int j = 0; j < MERGE_K; ++j) {
                const bool take_a = ia < na && (ib >= nb || va <= vb);
                if ((uint32_t)j < nout) {
                    outk[j] = take_a ? va : vb;
                    if (perm) outp[j] = take_a ? Ap[ia < na ? ia : 0u] : Bp[ib < nb ? ib : 0u];
                }
                ia += take_a;
                ib += !take_a;
                const uint32_t nxt = take_a ? Ak[ia < na ? ia : 0u] : Bk[ib < nb ? ib : 0u];
                va = take_a ? nxt : va;
                vb = take_a ? vb : nxt;
            }
        }
        __syncwarp();
        uint32_t parent = NONE, round = 0;
        unsigned long long t_ready = 0;
        uint32_t* gok = nullptr;
        uint32_t* gop = nullptr;
        Slice ok_sl = {0u, 0u, 0u}, op_sl = {0u, 0u, 0u};
        if (warp == 0) {                            // read before warp 0 releases the stage
            parent = S.parent;
            round = S.round;
            t_ready = S.t_ready;
            gok = S.ok;
            gop = S.op;
            ok_sl = S.osk;
            op_sl = S.osp;
        }
        if (lane == 0) mbar_arrive(&sm.empty[s]);   // this warp is done with the stage
        fence_proxy_async_smem();
        consumers_sync<BLOCK>();
        if (warp != 0) continue;
        // warp 0 sends the chunk out: the ends by ordinary stores (lanes 0-7
        // keys, 16-23 permutation), ordered before thread 0's announcement by
        // __syncwarp; the aligned interior by bulk store
        if ((lane & 15) < EDGE_SLOTS) {
            const bool is_perm = lane >= 16;
            if (!is_perm || perm) {
                const uint32_t i = edge_index(is_perm ? op_sl : ok_sl, (uint32_t)(lane & 15));
                if (i != NONE) {
                    if (is_perm) gop[i] = sm.out_p[sop + i];
                    else gok[i] = sm.out_k[sok + i];
                }
            }
        }
        __syncwarp();
        if (tid == 0) {
            bool good = true;
            if (ok_sl.nint) {
                void* g = gok + ok_sl.head;
                const void* l = &sm.out_k[sok + ok_sl.head];
                good = good && aligned16(g) && aligned16(l);
                if (good) tma_store_1d(g, l, ok_sl.nint * 4u);
            }
            if (perm && op_sl.nint) {
                void* g = gop + op_sl.head;
                const void* l = &sm.out_p[sop + op_sl.head];
                const bool g2 = aligned16(g) && aligned16(l);
                if (g2) tma_store_1d(g, l, op_sl.nint * 4u);
                good = good && g2;
            }
            if (!good) set_error(C, DERR_INTERNAL, 43);
            bulk_commit();
            // the previous chunk's store is complete once at most this one is pending
            if (sm.pend != NONE) {
                bulk_wait_all_but_one();
                announce(J, sm.pend);
            }
            sm.pend = parent;
            timeline_note(sm.tl, C, round, t_ready, globaltimer_ns());
        }
    }
    if (tid == 0) {
        bulk_wait_all();
        if (sm.pend != NONE) announce(J, sm.pend);
        timeline_flush(sm.tl, C);
    }
}

}  // namespace

template <int NST, int BLOCK>
__global__ void __launch_bounds__(Shape<NST, BLOCK>::MTHREADS, merge_min_ctas<NST, BLOCK>()) k_merge_rounds(Job J)
{
    extern __shared__ __align__(16) unsigned char merge_raw[];
    MergeSmem<NST, BLOCK>& sm = *reinterpret_cast<MergeSmem<NST, BLOCK>*>(merge_raw);
    Ctr* C = J.ctr;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&sm.full[s], 2);        // expect_tx arrival + edge arrival
            mbar_init(&sm.empty[s], Shape<NST, BLOCK>::NCONS);   // one arrival per consumer warp
        }
        fence_mbar_init();
        sm.err = *(volatile uint32_t*)&C->error;
        if (blockIdx.x == 0) C->merge_t0 = globaltimer_ns();
    }
    if (tid < NSEARCH) sm.ring_state[tid] = RS_EMPTY;
    for (int r = tid; r <= NPOW; r += blockDim.x) sm.round_chunk[r] = C->bucket_chunk[r];
    __syncthreads();
    if (sm.err) return;
    if (warp == Shape<NST, BLOCK>::SEARCH_WARP) search_warp<NST, BLOCK>(J, sm, C);
    else if (warp == Shape<NST, BLOCK>::PRODUCER_WARP) producer_warp<NST, BLOCK>(J, sm, C);
    else consumer_warps<NST, BLOCK>(J, sm, C);
}

// The shape used: two shared-memory stages of 512 consumer threads (two CTAs
// per SM).  Measured on GB300 against 256-448 consumer threads and 2-4 stages,
// it was the fastest from 10^5 elements to 2^28 and for batches.
using MergeShape = Shape<2, 512>;

int merge_rounds_max_grid(int num_sms)
{
    int per_sm = 0;
    const int bytes = (int)sizeof(MergeSmem<2, 512>);
    cudaFuncSetAttribute(k_merge_rounds<2, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_rounds<2, 512>, MergeShape::MTHREADS, bytes);
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

uint32_t merge_chunk()
{
    return (uint32_t)MergeShape::E;
}

cudaError_t launch_merge_rounds(const Job& J, int grid, cudaStream_t s)
{
    k_merge_rounds<2, 512><<<grid, MergeShape::MTHREADS, sizeof(MergeSmem<2, 512>), s>>>(J);
    return cudaGetLastError();
}

}  // namespace ps
