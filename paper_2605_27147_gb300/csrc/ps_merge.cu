// HBM merge rounds: the merges of Algorithm 1 whose inputs exceed the tile
// size, executed as stable out-of-place merges (Algorithm 2, StandardMerge:
// ties take the left run) between the caller's arrays and the scratch arrays
// (Pingpong storage, Sec. 3).
//
// Rounds go from the largest power to the smallest; all merges of one round
// are disjoint and their children are finished.  Every merge is cut into
// chunks of MERGE_E outputs.
//
// Phase A: for every chunk, how many of its merge's first d outputs come
// from the left child (merge-path split: the largest i with A[i-1] <= B[d-i],
// ties to the left).  The chunk -> merge table is built once per call by the
// planning kernels.
//
// Phase B is warp specialised.  A producer warp walks the CTA's chunks: it
// waits until a shared-memory stage is free (an "empty" mbarrier), describes
// the chunk, starts the 1-D bulk copies (cp.async.bulk, TMA) of the chunk's
// two input slices (keys and permutation) into the stage, and loads the
// elements outside the slices' 16-byte-aligned interiors (at most three at
// each end) with ordinary loads; the stage's "full" mbarrier completes when
// both have landed.  Eight consumer warps wait on "full", merge (each thread
// MERGE_K consecutive outputs: merge-path split inside shared memory, then a
// serial merge), release the stage, and send the chunk's output out through a
// bulk store (plus ordinary stores for its unaligned ends).  With two stages
// the producer runs one chunk ahead of the consumers.
//
// One persistent cooperative launch runs every round; a grid barrier (bounded
// spin, error flag on timeout) separates the phases.  Cooperative launch
// guarantees that all CTAs are resident, so the barrier cannot starve.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr int SLOT = MERGE_E + 16;   // a staged array: up to 3 + 3 + 3 shift slots
constexpr int EDGE_SLOTS = 8;        // unaligned elements of one slice (<= 7)

// Grid barrier in two levels: CTAs arrive at a counter of their group of 32,
// the last of a group arrives at the global counter, the last group bumps the
// generation.  Arrivals on 20-odd different words proceed in parallel instead
// of 600 atomics serialising on one.
__device__ bool grid_barrier(Ctr* C)
{
    __syncthreads();
    __shared__ uint32_t s_ok;
    if (threadIdx.x == 0) {
        uint32_t ok = 1;
        const uint32_t gen = ld_acquire_u32(&C->bar_gen);
        __threadfence();
        const uint32_t grp = blockIdx.x >> 5;
        const uint32_t ngroups = (gridDim.x + 31) >> 5;
        const uint32_t gsize = min(32u, gridDim.x - (grp << 5));
        bool last = false;
        if (atomicAdd(&C->bar_group[grp], 1u) == gsize - 1) {
            atomicExch(&C->bar_group[grp], 0u);
            last = atomicAdd(&C->bar_count, 1u) == ngroups - 1;
        }
        if (last) {
            atomicExch(&C->bar_count, 0u);
            __threadfence();
            st_release_u32(&C->bar_gen, gen + 1);
        } else {
            // poll with relaxed loads, back off, acquire once the generation moved
            const long long t0 = clock64();
            uint32_t nap = 64;
            while (ld_relaxed_u32(&C->bar_gen) == gen) {
                __nanosleep(nap);
                nap = nap < 1024 ? nap * 2 : 1024;
                if (clock64() - t0 > SPIN_LIMIT_CYCLES) {
                    set_error(C, DERR_TIMEOUT, 40);
                    ok = 0;
                    break;
                }
            }
            fence_acquire_gpu();
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Number of left-run elements among the first d outputs of the stable merge.
__device__ __forceinline__ uint32_t merge_path(const uint32_t* A, uint32_t la, const uint32_t* B, uint32_t lb,
                                               uint32_t d)
{
    uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

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
    uint32_t cnt;
    uint32_t last;           // nonzero: no chunk; the round is over for this CTA
};

constexpr int NCONS = MERGE_BLOCK / 32;          // consumer warps
constexpr int MTHREADS = MERGE_BLOCK + 32;        // + the producer warp
constexpr int NST = 2;                            // shared-memory stages

struct __align__(16) MergeSmem {
    uint32_t in_k[NST][SLOT];
    uint32_t in_p[NST][SLOT];
    uint32_t out_k[SLOT];
    uint32_t out_p[SLOT];
    uint64_t full[NST];      // producer -> consumers: the stage holds a chunk
    uint64_t empty[NST];     // consumers -> producer: the stage may be refilled
    Stage st[NST];
};

// Describe chunk q (round-local index; global chunk id c0 + q) of the current round.
__device__ void describe(const Job& J, uint32_t q, uint32_t c0, uint32_t nch, Stage& S)
{
    const uint32_t e = J.chunk_node[c0 + q];
    const GSorted g = J.gsorted[e];
    const uint32_t total = g.la + g.lb;
    const uint32_t d0 = (c0 + q - g.chunk_base) * MERGE_E;
    const uint32_t d1 = min(d0 + (uint32_t)MERGE_E, total);
    const uint32_t a0 = J.splits[q];
    const uint32_t a1 = (d1 == total || q + 1 >= nch) ? g.la : J.splits[q + 1];
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
}

__device__ __forceinline__ bool aligned16(const void* p)
{
    return (((uintptr_t)p) & 15u) == 0;
}

// Producer lane 0: announce the stage's bytes and start its bulk copies.
__device__ void issue_loads(MergeSmem& sm, int s, Ctr* C)
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
__device__ __forceinline__ void copy_edge(MergeSmem& sm, int s, int lane)
{
    const Stage& S = sm.st[s];
    const int which = lane >> 3, j = lane & 7;
    const int side = which & 1;
    const bool is_perm = which >= 2;
    if (is_perm && !S.gp[side]) return;
    const Slice& sl = is_perm ? S.slp[side] : S.slk[side];
    const uint32_t i = edge_index(sl, (uint32_t)j);
    if (i == NONE) return;
    if (is_perm) sm.in_p[s][S.sp[side] + i] = S.gp[side][i];
    else sm.in_k[s][S.sk[side] + i] = S.gk[side][i];
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

__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(MERGE_BLOCK) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

}  // namespace

__global__ void __launch_bounds__(MTHREADS, 4) k_merge_rounds(Job J)
{
    extern __shared__ __align__(16) unsigned char merge_raw[];
    MergeSmem& sm = *reinterpret_cast<MergeSmem*>(merge_raw);
    Ctr* C = J.ctr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool producer = warp == NCONS;
    const bool perm = J.want_perm != 0;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&sm.full[s], 2);        // expect_tx arrival + edge arrival
            mbar_init(&sm.empty[s], NCONS);   // one arrival per consumer warp
        }
        fence_mbar_init();
    }
    __syncthreads();
    // stage use counters: the producer fills stages round robin, the consumers
    // take them in the same order, so both sides keep identical counts
    uint32_t fills[NST] = {0u, 0u}, uses[NST] = {0u, 0u};
    uint32_t slot = 0;

    for (int r = 0; r < NPOW; ++r) {
        if (*(volatile uint32_t*)&C->error) return;
        const uint32_t e0 = C->bucket_start[r], e1 = C->bucket_start[r + 1];
        if (e0 == e1) continue;
        const uint32_t c0 = C->bucket_chunk[r], c1 = C->bucket_chunk[r + 1];
        const uint32_t nch = c1 - c0;
        const bool stamp = blockIdx.x == 0 && tid == 0;
        if (stamp) C->round_ns[r][0] = globaltimer_ns();

        // phase A: the merge-path split of every chunk start, chunks interleaved
        // over all CTAs so every CTA searches and none idles
        for (uint32_t q = tid * gridDim.x + blockIdx.x; q < nch; q += gridDim.x * blockDim.x) {
            const GSorted g = J.gsorted[J.chunk_node[c0 + q]];
            const uint32_t d = (c0 + q - g.chunk_base) * MERGE_E;
            const uint32_t* A = (((g.depth + 1) & 1u) ? J.keysB : J.keysA) + g.goff;
            J.splits[q] = merge_path(A, g.la, A + g.la, g.lb, d);
        }
        if (stamp) C->round_ns[r][4] = globaltimer_ns();
        if (!grid_barrier(C)) return;
        if (stamp) C->round_ns[r][1] = globaltimer_ns();

        // phase B: chunks handed out dynamically (one atomic per chunk), the
        // last stage of the round carries no chunk
        if (producer) {
            if (lane == 0) fence_proxy_async_global();   // earlier generic writes before async reads
            __syncwarp();
            for (;;) {
                uint32_t q = 0;
                if (lane == 0) q = atomicAdd(&C->chunk_next[r], 1u);
                q = __shfl_sync(0xffffffffu, q, 0);
                const int s = (int)slot;
                if (fills[s] > 0 && !mbar_wait_bounded(&sm.empty[s], (fills[s] - 1) & 1u, C, 44)) return;
                ++fills[s];
                slot = (slot + 1) % NST;
                if (q >= nch) {                       // close the round for the consumers
                    if (lane == 0) {
                        sm.st[s].last = 1;
                        sm.st[s].cnt = 0;
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(&sm.full[s], 0);
                        mbar_arrive(&sm.full[s]);
                    }
                    __syncwarp();
                    break;
                }
                if (lane == 0) {
                    sm.st[s].last = 0;
                    describe(J, q, c0, nch, sm.st[s]);
                    issue_loads(sm, s, C);
                }
                __syncwarp();
                copy_edge(sm, s, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.full[s]);
            }
        } else {
            for (;;) {
                const int s = (int)slot;
                if (!mbar_wait_bounded(&sm.full[s], uses[s] & 1u, C, 42)) return;
                ++uses[s];
                slot = (slot + 1) % NST;
                const Stage& S = sm.st[s];
                if (S.last) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.empty[s]);
                    break;
                }
                const uint32_t na = S.na, nb = S.nb, cnt = S.cnt;
                uint32_t* const gok = S.ok;
                uint32_t* const gop = S.op;
                const uint32_t sok = S.sok, sop = S.sop;
                const uint32_t* Ak = &sm.in_k[s][S.sk[0]];
                const uint32_t* Bk = &sm.in_k[s][S.sk[1]];
                const uint32_t* Ap = &sm.in_p[s][S.sp[0]];
                const uint32_t* Bp = &sm.in_p[s][S.sp[1]];
                uint32_t ok[MERGE_K], op[MERGE_K];
                const uint32_t x0 = tid * MERGE_K;
                if (x0 < cnt) {
                    uint32_t lo = x0 > nb ? x0 - nb : 0u, hi = min(x0, na);
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (Ak[mid] <= Bk[x0 - 1 - mid]) lo = mid + 1; else hi = mid;
                    }
                    uint32_t ia = lo, ib = x0 - lo;
                    uint32_t va = ia < na ? Ak[ia] : 0xffffffffu, vb = ib < nb ? Bk[ib] : 0xffffffffu;
                    // branch-free serial merge; an exhausted side is read at slot 0
                    // (a valid address whose value is never used)
#pragma unroll
                    for (int j = 0; j < MERGE_K; ++j) {
                        const bool take_a = ia < na && (ib >= nb || va <= vb);
                        ok[j] = take_a ? va : vb;
                        if (perm) op[j] = take_a ? Ap[ia < na ? ia : 0u] : Bp[ib < nb ? ib : 0u];
                        ia += take_a;
                        ib += !take_a;
                        const uint32_t nxt = take_a ? Ak[ia < na ? ia : 0u] : Bk[ib < nb ? ib : 0u];
                        va = take_a ? nxt : va;
                        vb = take_a ? vb : nxt;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[s]);   // this warp is done with the stage
                if (tid == 0) bulk_wait_read_all();         // the previous output has left shared memory
                consumers_sync();
                if (x0 < cnt) {
#pragma unroll
                    for (int j = 0; j < MERGE_K; ++j) {
                        if (x0 + j < cnt) {
                            sm.out_k[sok + x0 + j] = ok[j];
                            if (perm) sm.out_p[sop + x0 + j] = op[j];
                        }
                    }
                }
                fence_proxy_async_smem();
                consumers_sync();
                // output: aligned interior by bulk store, the ends by ordinary stores
                const Slice ok_sl = slice_of(gok, cnt);
                const Slice op_sl = perm ? slice_of(gop, cnt) : Slice{0u, 0u, 0u};
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
                }
                if (warp == 1 && (lane & 15) < EDGE_SLOTS) {   // lanes 0-7: keys, 16-23: permutation
                    const bool is_perm = lane >= 16;
                    if (!is_perm || perm) {
                        const uint32_t i = edge_index(is_perm ? op_sl : ok_sl, (uint32_t)(lane & 15));
                        if (i != NONE) {
                            if (is_perm) gop[i] = sm.out_p[sop + i];
                            else gok[i] = sm.out_k[sok + i];
                        }
                    }
                }
            }
            if (tid == 0) {
                bulk_wait_all();                    // this round's output is in global memory
                fence_proxy_async_global();
                if (stamp) C->round_ns[r][2] = globaltimer_ns();
            }
        }
        if (producer) {
            for (int s = 0; s < NST; ++s) uses[s] = fills[s];
        } else {
            for (int s = 0; s < NST; ++s) fills[s] = uses[s];
        }
        if (!grid_barrier(C)) return;
        if (stamp) C->round_ns[r][3] = globaltimer_ns();
    }
}

int merge_rounds_grid_for(int num_sms, int ctas_per_sm)
{
    const int mx = merge_rounds_max_grid(num_sms) / num_sms;
    const int k = (ctas_per_sm > 0 && ctas_per_sm < mx) ? ctas_per_sm : mx;
    return num_sms * k;
}

int merge_rounds_max_grid(int num_sms)
{
    int per_sm = 0;
    cudaFuncSetAttribute(k_merge_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MergeSmem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_rounds, MTHREADS, sizeof(MergeSmem));
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_merge_rounds(const Job& J, int grid, cudaStream_t s)
{
    void* args[] = {(void*)&J};
    return cudaLaunchCooperativeKernel((const void*)k_merge_rounds, dim3(grid), dim3(MTHREADS), args,
                                       sizeof(MergeSmem), s);
}

}  // namespace ps
