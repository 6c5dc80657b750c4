// Virtual-memory storage (Sec. 4): the HBM merges without an n-element
// scratch buffer.
//
// The instance's index range is cut into virtual pages of P = 2^plog2
// elements.  A page table maps every virtual page to a physical page: one of
// the caller's array pages (physical id < vm_na_cap) or a page of a small
// pool (the rest).  The tiles are merged in place, so at first every virtual
// page is its own array page.  A merge round writes the output of every page
// its merges touch into a fresh physical page taken from a free-page stack
// (elements of a touched page that no merge of the round covers are carried
// over unchanged); an input page goes back to the stack once all of its
// elements have been consumed (the paper's PopFront freeing an emptied page).
// Inside a round the output pages form a dataflow in page order: each takes
// the next free page from a FIFO ring and pushes the input pages it was the
// last to consume: a merge consumes exactly as many input elements as it
// writes, so the freed pages keep pace with the taken ones, and the pool needs
// about one page per page group in flight plus a few partly consumed pages --
// not n elements.  Every merge-path split a page needs (at page boundaries
// inside a merge) is searched at the start of the round, all pages in
// parallel, while every input page still holds its data; the pages then only
// stream.  Finally Copy (Sec. 4) moves every virtual page to its own
// array page: a page still holding data that is needed later is first moved
// to a free page, exactly as the paper describes.
#include <algorithm>

#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr int VM_BLOCK = 256;
constexpr int VM_WARPS = VM_BLOCK / 32;
// outputs per thread of a merge sub-chunk: odd, so that the threads of a
// warp search and merge at positions spread over the shared-memory banks
// (with 16 the split positions of a warp fell on a few banks), and at least
// 16, so that a group's sub-chunk holds a page
constexpr int VM_K = 17;
constexpr int VM_GROUP_PAD = 16;          // staging words per group beyond its sub-chunk (slice phases)
constexpr int VM_SLOTS = VM_BLOCK * VM_K + VM_GROUP_PAD * VM_WARPS;   // staging words per CTA

// A CTA works on several output pages at once: groups of W warps, W = P / 512
// clamped to 1..8, each group merging sub-chunks of 544 W = VM_K x its
// threads outputs (at least one page) in its own slice of shared memory, with
// its own named barrier.
struct VmGroup {
    uint32_t g;        // group index inside the CTA
    uint32_t groups;   // groups per CTA
    uint32_t nthr;     // threads per group
    uint32_t tid;      // thread index inside the group
    uint32_t cap;      // outputs per sub-chunk
};

__device__ __forceinline__ VmGroup vm_group(uint32_t plog2)
{
    VmGroup G;
    const uint32_t w = plog2 >= 9 ? min(1u << (plog2 - 9), (uint32_t)VM_WARPS) : 1u;
    G.groups = VM_WARPS / w;
    G.nthr = 32u * w;
    G.g = threadIdx.x / G.nthr;
    G.tid = threadIdx.x % G.nthr;
    G.cap = G.nthr * VM_K;
    return G;
}

__device__ __forceinline__ void group_sync(const VmGroup& G)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1u + G.g), "r"(G.nthr) : "memory");
}

__device__ __forceinline__ uint32_t* phys_k(const Job& J, uint32_t p)
{
    const size_t P = (size_t)1 << J.vm_plog2;
    return p < J.vm_na_cap ? J.keysA + (size_t)p * P : J.pool_keys + (size_t)(p - J.vm_na_cap) * P;
}

__device__ __forceinline__ uint32_t* phys_p(const Job& J, uint32_t p)
{
    const size_t P = (size_t)1 << J.vm_plog2;
    return p < J.vm_na_cap ? J.permA + (size_t)p * P : J.pool_perm + (size_t)(p - J.vm_na_cap) * P;
}

// key at virtual index v (through the page table)
__device__ __forceinline__ uint32_t vkey(const Job& J, uint32_t v)
{
    return phys_k(J, J.pt[v >> J.vm_plog2])[v & ((1u << J.vm_plog2) - 1)];
}

__device__ __forceinline__ uint32_t page_size(const Job& J, uint32_t u, uint32_t n)
{
    const uint32_t P = 1u << J.vm_plog2;
    return (u + 1 == J.vm_na) ? n - u * P : P;
}

// Left-child elements among the first d outputs of merge g (merge path over
// the page-table-translated keys), by a team of eight lanes (lane & ~7 ..
// lane | 7, converged): an 8-ary search, seven probes per step.  The
// predicate L[m] <= R[d-1-m] is true below the split and false from it on,
// so the trues among increasing probes form a prefix.
__device__ uint32_t vm_split_team(const Job& J, const GSorted& g, uint32_t d, uint32_t lane)
{
    const uint32_t tl = lane & 7u, shift = lane & 24u;
    const uint32_t tmask = 0xffu << shift;
    const uint32_t lo = (uint32_t)g.goff, mid = lo + g.la;
    uint32_t l = d > g.lb ? d - g.lb : 0u;
    uint32_t h = min(d, g.la);
    while (l < h) {
        const uint32_t span = h - l;
        // probes: l + 1 .. l + span when span <= 7, else seven evenly spaced
        const uint32_t k = span <= 7u ? span : 7u;
        const uint32_t m = span <= 7u ? l + tl : l + (uint32_t)(((unsigned long long)(tl + 1) * span) >> 3);
        bool t = false;
        if (tl < k) t = vkey(J, lo + m) <= vkey(J, mid + d - 1 - m);
        const uint32_t bits = (__ballot_sync(tmask, t) >> shift) & 0x7fu;
        const uint32_t trues = __popc(bits);   // a prefix of the probes
        if (span <= 7u) {
            l += trues;
            break;
        }
        const uint32_t m_lo = trues ? l + (uint32_t)(((unsigned long long)trues * span) >> 3) : 0u;
        const uint32_t m_hi = trues < 7u ? l + (uint32_t)(((unsigned long long)(trues + 1) * span) >> 3) : h;
        if (trues) l = m_lo + 1;
        h = m_hi;
    }
    return l;
}

// Push a free physical page onto the ring.
__device__ __forceinline__ void ring_push(const Job& J, uint32_t page)
{
    const uint32_t at = atomicAdd(&J.ctr->vm_ring_tail, 1u);
    if (at < J.vm_ring_cap) st_release_u32(&J.free_stack[at], page);
    else set_error(J.ctr, DERR_INTERNAL, 66);
}

// Consumed-element counting, split in two so that the atomic's latency
// overlaps the merge: consume_start counts thread q's share (q < 4) of the
// consumed virtual ranges [v0, v0 + c0) and [v1, v1 + c1) -- each at most a
// page long, so two pages each -- and consume_finish pushes the page onto the
// free ring if this count completed it.  The caller's last array page may be
// partial: like the paper's partial input page it is never declared free.
struct Consumed {
    uint32_t u, take, before;
};

__device__ __forceinline__ Consumed consume_start(const Job& J, uint32_t q, uint32_t v0, uint32_t c0, uint32_t v1,
                                                  uint32_t c1)
{
    Consumed r = {NONE, 0u, 0u};
    if (q >= 4) return r;
    const uint32_t L = J.vm_plog2;
    const uint32_t v = q < 2 ? v0 : v1, c = q < 2 ? c0 : c1;
    if (!c) return r;
    const uint32_t first = min(c, (((v >> L) + 1) << L) - v);   // elements in v's page
    if ((q & 1u) == 0) {
        r.u = v >> L;
        r.take = first;
    } else if (c > first) {
        r.u = (v >> L) + 1;
        r.take = c - first;
    } else {
        return r;
    }
    r.before = atomicAdd(&J.consumed[r.u], r.take);
    return r;
}

__device__ __forceinline__ void consume_finish(const Job& J, const Consumed& r, uint32_t n)
{
    if (r.u == NONE || r.before + r.take != page_size(J, r.u, n)) return;
    const uint32_t old = J.pt[r.u];
    const bool partial_tail = old + 1 == J.vm_na && (n & ((1u << J.vm_plog2) - 1)) != 0;
    if (!partial_tail) ring_push(J, old);
}

// Sum of v over the CTA (every thread gets it); ws: one word per warp.
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    return t;
}

// Number of threads below this one (in thread order) whose flag is set, and
// the CTA's total; ws: one word per warp.
__device__ __forceinline__ uint32_t block_rank(bool flag, uint32_t* ws, uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t m = __ballot_sync(0xffffffffu, flag);
    __syncthreads();
    if (lane == 0) ws[warp] = __popc(m);
    __syncthreads();
    uint32_t before = __popc(m & ((1u << lane) - 1u)), t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < warp) before += ws[w];
        t += ws[w];
    }
    total = t;
    return before;
}

struct __align__(16) VmSmem {
    uint32_t k[VM_SLOTS];
    uint32_t p[VM_SLOTS];
    uint16_t src[VM_SLOTS];                     // the merge's choice per output: slot in k / p
    // the page's record, the split block of its start, the split at its end
    uint32_t rec[VM_WARPS][VM_REC_WORDS + 6];
    uint32_t claim[VM_WARPS][2];                // (virtual page, output page) of the group's current page
};

// One output page by one group: its merge segments and copy gaps, from the
// record the round's step 2 wrote, into the fresh physical page `out`.
__device__ void vm_page(const Job& J, VmSmem& sm, const VmGroup& G, uint32_t u, uint32_t out, uint32_t n,
                        bool perm)
{
    const uint32_t tid = G.tid, gi = G.g;
    uint32_t* sk = sm.k + gi * (G.cap + VM_GROUP_PAD);   // 16-byte aligned: cap is a multiple of 4
    uint32_t* sp = sm.p + gi * (G.cap + VM_GROUP_PAD);
    uint32_t* rec = sm.rec[gi];
    const uint32_t L = J.vm_plog2;
    const uint32_t ps0 = u << L;
    uint32_t* dk = phys_k(J, out);
    uint32_t* dp = perm ? phys_p(J, out) : nullptr;
    // the record, the split block of the page's start and the split at its
    // end, in one round trip
    for (uint32_t i = tid; i < VM_REC_WORDS + 6; i += G.nthr) {
        uint32_t x;
        if (i < VM_REC_WORDS) x = J.vm_rec[(size_t)u * VM_REC_WORDS + i];
        else if (i < VM_REC_WORDS + 5) x = J.vm_split_at[(size_t)u * VM_SPLIT_WORDS + (i - VM_REC_WORDS)];
        else x = u + 1 < J.vm_na ? J.vm_split_at[(size_t)(u + 1) * VM_SPLIT_WORDS] : 0u;
        rec[i] = x;
    }
    group_sync(G);
    const uint32_t nseg = min(rec[0], 3u);
    for (uint32_t sg = 0; sg < nseg; ++sg) {
        const uint32_t* R = rec + 1 + VM_SEG_WORDS * sg;
        const uint32_t s0 = R[0], s1 = R[1], lo = R[2];
        if (lo == NONE) {                        // carried over unchanged (a gap)
            const uint32_t ph = R[5];
#pragma unroll 8
            for (uint32_t v = s0 + tid; v < s1; v += G.nthr) {
                const uint32_t off = v & ((1u << L) - 1u);
                dk[v - ps0] = phys_k(J, ph)[off];
                if (dp) dp[v - ps0] = phys_p(J, ph)[off];
            }
            group_sync(G);
            consume_finish(J, consume_start(J, tid, s0, s1 - s0, 0u, 0u), n);
            continue;
        }
        const uint32_t mid = R[3], hi = R[4], la = mid - lo;
        // the splits: 0 / la at the merge's ends; at a page end inside the
        // merge the round's search left them in vm_split_at (with the pages
        // of the slices starting there)
        const bool inside = s0 != lo;
        const uint32_t a0 = inside ? rec[VM_REC_WORDS] : 0u;
        const uint32_t a1 = s1 == hi ? la : rec[VM_REC_WORDS + 5];
        const uint32_t* sph = inside ? rec + VM_REC_WORDS + 1 : R + 5;
        const uint32_t b0 = (s0 - lo) - a0, b1 = (s1 - lo) - a1;
        const uint32_t na = a1 - a0, nb = b1 - b0, cnt = na + nb;
        if (cnt > G.cap) {   // a segment never exceeds a page, and a page fits a group
            if (tid == 0) set_error(J.ctr, DERR_INTERNAL, 65);
            return;
        }
        // page splicing: when the whole output page is one whole input page
        // (a page-aligned slice of a single run), the output page takes over
        // that physical page through the page table and no element moves; the
        // input page is consumed by this page alone, so it is not freed, and
        // the fresh page goes back to the ring
        if (cnt == (1u << L) && s0 == ps0 && ((na == cnt && ((lo + a0) & (cnt - 1u)) == 0) ||
                                              (nb == cnt && ((mid + b0) & (cnt - 1u)) == 0))) {
            if (tid == 0) {
                J.pt_new[u] = na == cnt ? sph[0] : sph[2];
                ring_push(J, out);
                atomicAdd(&J.ctr->vm_spliced, 1u);
            }
            return;
        }
        // the slices' keys (and permutation): each slice is at most a page, so
        // it spans at most two physical pages, named in the record.  A slice
        // is staged at the 16-byte phase of its first element (the left one
        // from slot sa, the right one from sb), so the 16-byte blocks of a
        // page land on 16-byte blocks of the staging arrays and move by
        // 16-byte asynchronous copies; the up to three elements before and
        // after the blocks of each page move one by one (everything in flight
        // at once; one by one throughout when a page's base is not 16-byte
        // aligned, as a caller's array may not be)
        const uint32_t va = lo + a0, vb = mid + b0;
        const uint32_t sa = va & 3u, sb = ((sa + na + 3u) & ~3u) + (vb & 3u);
        for (uint32_t side = 0; side < 2; ++side) {
            const uint32_t v0 = side ? vb : va, len = side ? nb : na, d0 = side ? sb : sa;
            for (uint32_t part = 0, done = 0; part < 2 && done < len; ++part) {
                const uint32_t off = (v0 + done) & ((1u << L) - 1u);
                const uint32_t run = min(len - done, (1u << L) - off);
                const uint32_t ph = sph[2u * side + part];
                const uint32_t* gk = phys_k(J, ph) + off;
                const uint32_t* gp = perm ? phys_p(J, ph) + off : nullptr;
                const uint32_t d = d0 + done;           // staging slot of the run's first element
                const uint32_t phase = (d & 3u) << 2;   // its byte offset in a 16-byte block
                const bool al = (reinterpret_cast<uintptr_t>(gk) & 15u) == phase &&
                                (!perm || (reinterpret_cast<uintptr_t>(gp) & 15u) == phase);
                const uint32_t head = al ? min(run, (4u - (d & 3u)) & 3u) : run;
                const uint32_t body = al ? ((run - head) & ~3u) : 0u;
                for (uint32_t q = tid; q < body / 4u; q += G.nthr) {
                    cp_async16(&sk[d + head + 4u * q], gk + head + 4u * q);
                    if (perm) cp_async16(&sp[d + head + 4u * q], gp + head + 4u * q);
                }
                for (uint32_t j = tid; j < run - body; j += G.nthr) {
                    const uint32_t x = j < head ? j : j + body;
                    cp_async4(&sk[d + x], gk + x);
                    if (perm) cp_async4(&sp[d + x], gp + x);
                }
                done += run;
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
        group_sync(G);
        // every input element is read: the consumed counts go out now and are
        // looked at after the merge (a freed page is not read again in this merge round)
        const Consumed cons = consume_start(J, tid, lo + a0, na, mid + b0, nb);
        // each thread merges VM_K consecutive outputs, recording for each the
        // staging slot it comes from; then the group writes the page out in
        // order, consecutive threads on consecutive words
        uint16_t* ssrc = sm.src + gi * (G.cap + VM_GROUP_PAD);
        const uint32_t* A = sk + sa;
        const uint32_t* B = sk + sb;
        const uint32_t t0 = tid * VM_K;
        if (t0 < cnt) {
            uint32_t l = t0 > nb ? t0 - nb : 0u, h = min(t0, na);
            while (l < h) {
                const uint32_t m = (l + h) >> 1;
                if (A[m] <= B[t0 - 1 - m]) l = m + 1; else h = m;
            }
            uint32_t ia = l, ib = t0 - l;
#pragma unroll 4
            for (int j = 0; j < VM_K; ++j) {
                if (t0 + j < cnt) {
                    const bool ta = ia < na && (ib >= nb || A[ia] <= B[ib]);
                    ssrc[t0 + j] = (uint16_t)(ta ? sa + ia : sb + ib);
                    ia += ta;
                    ib += !ta;
                }
            }
        }
        group_sync(G);
        uint32_t* ok = dk + (s0 - ps0);
        uint32_t* op = dp ? dp + (s0 - ps0) : nullptr;
#pragma unroll 4
        for (uint32_t i = tid; i < cnt; i += G.nthr) {
            const uint32_t from = ssrc[i];
            ok[i] = sk[from];
            if (op) op[i] = sp[from];
        }
        consume_finish(J, cons, n);
        group_sync(G);
    }
}

}  // namespace

// The HBM merge rounds with virtual-memory storage.  Per round:
//   1. every merge marks the pages it touches (a team of warps per merge);
//   2. one thread per touched page writes the page's record (its merge
//      segments and gaps, in order) and, for a page start inside a merge, the
//      merge-path split there -- all before any page of the round is recycled;
//   3. CTA 0 lists the touched pages in page order;
//   4. the pages, as a dataflow: every page group takes tickets from one
//      counter (the next one while it merges the current page); ticket t
//      names the touched page t - base and the ring slot t its output page is
//      popped from.  Pages therefore take free pages in
//      page order, and a group holding a page never waits: it reads its
//      inputs, merges into the fresh page and pushes every input page it
//      consumed last.  When every group waits for a free page, all pages
//      before the first waiting ticket are done: every segment left of it has
//      returned all its input pages, and the merge in progress has taken at
//      most five pages more than it returned (two partly consumed pages per
//      run and the page it shares with its left neighbour), so a pool of 16
//      pages always has one to give (a bounded wait records PS_ETIMEOUT
//      should that ever fail);
//   5. the written pages become current.
// Grid barriers separate the steps; there are none between pages.
__global__ void __launch_bounds__(VM_BLOCK, 4) k_vm_rounds(Job J)
{
    __shared__ VmSmem sm;
    __shared__ uint32_t warp_sums[VM_BLOCK / 32];
    Ctr* C = J.ctr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool perm = J.want_perm != 0;
    const uint32_t n = J.inst[0].n;
    const uint32_t L = J.vm_plog2, NA = J.vm_na;
    const uint32_t nwarps_grid = gridDim.x * (VM_BLOCK / 32);
    const uint32_t gwarp = blockIdx.x * (VM_BLOCK / 32) + warp;
    const uint32_t gtid = blockIdx.x * VM_BLOCK + tid, gstride = gridDim.x * VM_BLOCK;

    // the ring: the pool's pages, then empty slots
    for (uint32_t i = gtid; i < J.vm_ring_cap; i += gstride)
        J.free_stack[i] = i < J.vm_pool ? J.vm_na_cap + i : NONE;
    if (!grid_barrier(C)) return;

    // pages per CTA block of step 3
    const uint32_t BK = (NA + gridDim.x - 1) / gridDim.x;
    if (blockIdx.x == 0 && tid == 0) C->merge_t0 = globaltimer_ns();
    for (int r = 0; r < NPOW; ++r) {
        if (*(volatile uint32_t*)&C->error) return;
        const uint32_t e0 = C->bucket_start[r], e1 = C->bucket_start[r + 1];
        if (e0 == e1) continue;
        if (blockIdx.x == 0 && tid == 0) C->round_ns[r][0] = globaltimer_ns();
        // 1. the pages each merge of the round touches: a team of W warps per
        //    merge, W = the grid's warps / the round's merges (at least 1), so
        //    that a round of few large merges still spreads over the grid
        const uint32_t W = e1 - e0 >= nwarps_grid ? 1u : nwarps_grid / (e1 - e0);
        const uint32_t teams = nwarps_grid / W, team = gwarp / W, tw = gwarp % W;
        for (uint32_t e = e0 + team; team < teams && e < e1; e += teams) {
            const GSorted g = J.gsorted[e];
            const uint32_t lo = (uint32_t)g.goff, hi = lo + g.la + g.lb;
            const uint32_t first = lo >> L, last = (hi - 1) >> L;
            for (uint32_t u = first + tw * 32u + lane; u <= last; u += W * 32u) {
                if (u == first || u == last) {
                    const uint32_t slot = atomicAdd(&J.page_cnt[u], 1u);
                    if (slot < 2) J.page_nodes[2 * u + slot] = e;
                    else set_error(C, DERR_INTERNAL, 61);
                } else {
                    J.page_cnt[u] = 1;
                    J.page_nodes[2 * u] = e;
                }
            }
        }
        if (!grid_barrier(C)) return;
        // the touched pages of this CTA's block of pages (listed in step 3)
        {
            const uint32_t b0 = min(blockIdx.x * BK, NA), b1 = min(b0 + BK, NA);
            uint32_t c = 0;
            for (uint32_t u = b0 + tid; u < b1; u += VM_BLOCK) c += J.page_cnt[u] > 0 ? 1u : 0u;
            c = block_sum(c, warp_sums);
            if (tid == 0) J.vm_cta_count[blockIdx.x] = c;
        }
        // 2. per touched page (a thread each): its record -- up to two merges,
        //    ordered, with the gaps between them filled by copies; and per page
        //    start inside a merge (eight lanes each) the merge-path split there,
        //    searched while every input page still holds its data
        for (uint32_t u = gtid; u < NA; u += gstride) {
            const uint32_t c = min(J.page_cnt[u], 2u);
            if (c == 0) continue;
            const uint32_t ps0 = u << L, pe = min(ps0 + (1u << L), n);
            GSorted g[2];
            g[0] = J.gsorted[J.page_nodes[2 * u]];
            if (c == 2) {
                g[1] = J.gsorted[J.page_nodes[2 * u + 1]];
                if (g[0].goff > g[1].goff) {
                    const GSorted t = g[0];
                    g[0] = g[1];
                    g[1] = t;
                }
            }
            uint32_t w[VM_REC_WORDS];
            for (uint32_t i = 0; i < VM_REC_WORDS; ++i) w[i] = 0;
            uint32_t ns = 0, cur = ps0;
            const uint32_t own = J.pt[u];
            for (uint32_t i = 0; i < c; ++i) {
                const uint32_t lo = (uint32_t)g[i].goff, mid = lo + g[i].la, hi = mid + g[i].lb;
                const uint32_t s0 = max(lo, ps0), s1 = min(hi, pe);
                if (s0 >= s1) continue;
                uint32_t* W = w + 1 + VM_SEG_WORDS * ns;
                if (s0 > cur) {
                    W[0] = cur; W[1] = s0; W[2] = NONE; W[5] = own;
                    ++ns;
                    W += VM_SEG_WORDS;
                }
                W[0] = s0; W[1] = s1; W[2] = lo; W[3] = mid; W[4] = hi;
                if (s0 == lo) {
                    // the slices start at the runs' starts: their pages are known now
                    // (a page start inside the merge gets them from the split search)
                    W[5] = J.pt[lo >> L];
                    W[6] = (lo >> L) + 1 < NA ? J.pt[(lo >> L) + 1] : 0u;
                    W[7] = (mid >> L) < NA ? J.pt[mid >> L] : 0u;
                    W[8] = (mid >> L) + 1 < NA ? J.pt[(mid >> L) + 1] : 0u;
                }
                ++ns;
                cur = s1;
            }
            if (cur < pe) {
                uint32_t* W = w + 1 + VM_SEG_WORDS * ns;
                W[0] = cur; W[1] = pe; W[2] = NONE; W[5] = own;
                ++ns;
            }
            w[0] = ns;
            uint4* dst = reinterpret_cast<uint4*>(J.vm_rec + (size_t)u * VM_REC_WORDS);
#pragma unroll
            for (int q = 0; q < (int)VM_REC_WORDS / 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
        for (uint32_t u = gtid >> 3; u < NA; u += gstride >> 3) {
            const uint32_t c = min(J.page_cnt[u], 2u), ps0 = u << L;
            for (uint32_t i = 0; i < c; ++i) {
                const GSorted g = J.gsorted[J.page_nodes[2 * u + i]];
                const uint32_t lo = (uint32_t)g.goff;
                if (lo < ps0 && ps0 < lo + g.la + g.lb) {
                    const uint32_t a = vm_split_team(J, g, ps0 - lo, lane);
                    // the split, and the pages of the two slices that start here
                    const uint32_t tl = lane & 7u;
                    uint32_t x = a;
                    if (tl >= 1 && tl <= 4) {
                        const uint32_t v = tl <= 2 ? lo + a : lo + g.la + (ps0 - lo - a);
                        const uint32_t vp = (v >> L) + ((tl - 1) & 1u);
                        x = vp < NA ? J.pt[vp] : 0u;
                    }
                    if (tl <= 4) J.vm_split_at[(size_t)u * VM_SPLIT_WORDS + tl] = x;
                }
            }
        }
        // 3. the touched pages, in page order: every CTA lists the pages of
        //    its own contiguous block of BK pages, after the touched pages of
        //    the blocks before it (counted at the start of step 2)
        if (!grid_barrier(C)) return;
        {
            __shared__ uint32_t s_before;
            uint32_t before = 0;                      // touched pages in the blocks before this one
            for (uint32_t j = tid; j < blockIdx.x; j += VM_BLOCK) before += __ldcg(J.vm_cta_count + j);
            before = block_sum(before, warp_sums);
            if (tid == 0) s_before = before;
            __syncthreads();
            uint32_t carry = s_before;
            const uint32_t b0 = min(blockIdx.x * BK, NA), b1 = min(b0 + BK, NA);
            for (uint32_t u0 = b0; u0 < b1; u0 += VM_BLOCK) {
                const uint32_t u = u0 + tid;
                const bool t = u < b1 && J.page_cnt[u] > 0;
                uint32_t tot;
                const uint32_t at = carry + block_rank(t, warp_sums, tot);
                if (t) J.touched[at] = u;
                carry += tot;
            }
            if (blockIdx.x == gridDim.x - 1 && tid == 0) {
                C->vm_touched = carry;                // the last block's end: every touched page
                C->vm_round_base = C->vm_ring_head;
                C->vm_waves += 1;
            }
        }
        if (!grid_barrier(C)) return;
        if (blockIdx.x == 0 && tid == 0) C->round_ns[r][1] = globaltimer_ns();
        // 4. the pages, as a dataflow over tickets
        {
            const uint32_t ntouched = C->vm_touched, base = C->vm_round_base;
            const VmGroup G = vm_group(L);
            // the group's next ticket is drawn while its current page is merged
            uint32_t t_next = G.tid == 0 ? atomicAdd(&C->vm_ring_head, 1u) : 0u;
            for (;;) {
                if (G.tid == 0) {
                    uint32_t u = NONE, out = NONE;
                    const uint32_t t = t_next;
                    if (t - base < ntouched && !*(volatile uint32_t*)&C->error) {
                        u = J.touched[t - base];
                        if (t >= J.vm_ring_cap) {
                            set_error(C, DERR_INTERNAL, 67);
                        } else {
                            // pop slot t: wait (bounded) until a free page is pushed there
                            const long long c0 = clock64();
                            uint32_t nap = 32;
                            for (;;) {
                                const uint32_t v = ld_acquire_u32(&J.free_stack[t]);
                                if (v != NONE) {
                                    out = v;
                                    break;
                                }
                                if (*(volatile uint32_t*)&C->error) break;
                                if (clock64() - c0 > SPIN_LIMIT_CYCLES) {
                                    set_error(C, DERR_TIMEOUT, 68);
                                    break;
                                }
                                __nanosleep(nap);
                                nap = nap < 512 ? nap * 2 : 512;
                            }
                            if (out != NONE) {
                                J.pt_new[u] = out;
                                // pages beyond the array's n / P in use after this pop
                                const uint32_t tail = ld_relaxed_u32(&C->vm_ring_tail);
                                const uint32_t free_after = tail > t + 1 ? tail - (t + 1) : 0u;
                                if (J.vm_pool > free_after) atomicMax(&C->vm_in_use_peak, J.vm_pool - free_after);
                            }
                        }
                    }
                    sm.claim[G.g][0] = u;
                    sm.claim[G.g][1] = out;
                    if (out != NONE) t_next = atomicAdd(&C->vm_ring_head, 1u);
                }
                group_sync(G);
                const uint32_t u = sm.claim[G.g][0], out = sm.claim[G.g][1];
                group_sync(G);
                if (u == NONE || out == NONE) break;
                vm_page(J, sm, G, u, out, n, perm);
            }
        }
        if (!grid_barrier(C)) return;
        if (blockIdx.x == 0 && tid == 0) C->round_ns[r][2] = globaltimer_ns();
        // 5. the written pages become current; reset the per-round tables; the
        //    over-drawn tickets are returned
        const uint32_t ntouched = C->vm_touched;
        for (uint32_t j = gtid; j < ntouched; j += gstride) {
            const uint32_t u = J.touched[j];
            J.pt[u] = J.pt_new[u];
            J.page_cnt[u] = 0;
            J.consumed[u] = 0;
        }
        if (gtid == 0) C->vm_ring_head = C->vm_round_base + ntouched;
        if (!grid_barrier(C)) return;
        if (blockIdx.x == 0 && tid == 0) C->round_ns[r][3] = globaltimer_ns();
    }
}

// One page copied by the whole CTA: 16-byte vectors when the caller's arrays
// are 16-byte aligned (pool pages always are, and a page is a multiple of 16
// bytes), else word by word; the partial last page's tail word by word.
// Every thread issues its loads of both arrays (keys, then permutation) for
// up to VM_COPY_U vectors each before it stores, so a page of up to
// VM_BLOCK * VM_COPY_U * 4 elements takes one memory round trip.  Sources
// are read at L2 (other CTAs wrote them in earlier steps).
constexpr uint32_t VM_COPY_U = 4;

__device__ __noinline__ void vm_copy_keys_perm(const Job& J, uint32_t* dkw, uint32_t* dpw, const uint32_t* skw,
                                               const uint32_t* spw, uint32_t cnt, bool perm)
{
    const bool vec = ((reinterpret_cast<uintptr_t>(J.keysA) | reinterpret_cast<uintptr_t>(J.permA)) & 15u) == 0;
    const uint32_t nv = vec ? cnt >> 2 : 0u;
    const uint4* sk = reinterpret_cast<const uint4*>(skw);
    uint4* dk = reinterpret_cast<uint4*>(dkw);
    const uint4* sp = perm ? reinterpret_cast<const uint4*>(spw) : nullptr;
    uint4* dp = perm ? reinterpret_cast<uint4*>(dpw) : nullptr;
    for (uint32_t i0 = threadIdx.x; i0 < nv; i0 += VM_BLOCK * VM_COPY_U) {
        uint4 a[VM_COPY_U], b[VM_COPY_U];
#pragma unroll
        for (uint32_t u = 0; u < VM_COPY_U; ++u) {
            const uint32_t i = i0 + u * VM_BLOCK;
            if (i < nv) {
                a[u] = __ldcg(sk + i);
                if (perm) b[u] = __ldcg(sp + i);
            }
        }
#pragma unroll
        for (uint32_t u = 0; u < VM_COPY_U; ++u) {
            const uint32_t i = i0 + u * VM_BLOCK;
            if (i < nv) {
                dk[i] = a[u];
                if (perm) dp[i] = b[u];
            }
        }
    }
    for (int pass = 0; pass < (perm ? 2 : 1); ++pass) {
        const uint32_t* s = pass ? spw : skw;
        uint32_t* d = pass ? dpw : dkw;
        for (uint32_t i = (nv << 2) + threadIdx.x; i < cnt; i += VM_BLOCK) d[i] = __ldcg(s + i);
    }
}

__device__ __forceinline__ void vm_copy_page(const Job& J, uint32_t dst, uint32_t src, uint32_t cnt, bool perm)
{
    vm_copy_keys_perm(J, phys_k(J, dst), perm ? phys_p(J, dst) : nullptr, phys_k(J, src), perm ? phys_p(J, src) : nullptr,
                      cnt, perm);
}

// Copy (Sec. 4): every virtual page u moves from its physical page pt[u] to
// the caller's array page u.  The paper walks the virtual pages in order: a
// target array page that still holds data needed later is first moved out
// to a free page, then the page's own data is copied in.  The moves form
// chains: array page u receives virtual page u's data from pt[u]; when
// pt[u] = v is itself a target, v can receive its own data only after that,
// and so on, until pt[.] is a pool page.  A chain starts at a target that
// holds nothing, and a cycle of targets has no start.  So Copy walks every
// chain from its start, one page move per target (the paper's walk in the
// order that needs no evictions), with the chains in parallel:
//   1. holder[p], the virtual page physical page p holds;
//   2. the rank of every target along its chain, by pointer jumping over
//      the predecessor links (holder) -- a target on a cycle never reaches a
//      start; its cycle's smallest target becomes its start, whose data is
//      saved to a free pool page first, and the ranks are taken again;
//   3. long chains are cut into segments of S moves at the ranks divisible
//      by S: the data of every segment start but a chain's first is saved
//      to a temporary page, so the segment before it reads the saved copy
//      while the segment itself overwrites the page.  The temporaries are
//      the free pool pages and page-sized slots of the page-record and split
//      tables (rewritten by every round, unused during Copy) and of the
//      free-page ring past the two lists Copy keeps in it.  S is the
//      smallest power of two (and at least the moves per CTA) for which the
//      temporaries cover every save;
//   4. a CTA per segment walks it, page by page.
// Two targets that hold each other's data (a cycle of two, as a reversal of
// the page order makes) trade it directly, one CTA per pair, and need no
// temporary.
// When no S of at most COPY_SEG_MAX moves fits the free pages, the batched
// order below runs instead: batches of up to pool - 1 consecutive targets (a
// multiple of the CTAs when there are more) in two parallel steps, a CTA per
// page: (1) every target of the batch that holds another page's data moves
// it out to a free page; (2) every target receives its own data.  After
// step 1 no target of the batch holds needed data, so the copies of step 2
// never overwrite a source; each copy frees its source, so the number of
// free pages is the same after every batch, and counting pages shows that
// with at most pool - 1 targets per batch the free pages cover every move
// out.  A free page is one that holds nothing, is not a target of this or an
// earlier batch, and is not the caller's partial last page (never freed, as
// in the paper).  The free pages of the next batch are gathered during step
// 2 -- this batch's unused ones and the sources step 2 frees, without the
// next batch's targets -- into the other of two stacks, so a batch needs two
// grid barriers.
constexpr uint32_t COPY_SEG_MAX = 1024;   // longest segment the chain walk accepts
constexpr uint32_t COPY_KMAX = 17;        // segment lengths 2^0 .. 2^16 counted

// scratch of the chain walk in the page-record table (free during Copy):
// arrays of vm_na_cap words -- the ranking's ancestor, distance and minimum,
// double-buffered (the minimum arrays then hold every target's move: its
// source and the next target of its segment), the flags and the saves'
// temporaries, then the counters
enum : uint32_t { CW_ANC0, CW_DIST0, CW_MIN0, CW_ANC1, CW_DIST1, CW_MIN1, CW_FLAGS, CW_TEMP, CW_COUNTERS };
constexpr uint32_t CF_DONE = 1u, CF_CYCLE = 2u, CF_SAVED = 4u, CF_SWAP = 8u;
// counters after the arrays: [0, COPY_KMAX) saves needed per segment length,
// then cycles, moves to make, and a flag "a cycle exists"
enum : uint32_t { CC_CYCLES = COPY_KMAX, CC_MOVES, CC_ANY_CYCLE, CC_WORDS };
static_assert(CW_COUNTERS + 1 <= VM_REC_WORDS, "the chain walk's scratch fits the page records");

__device__ bool copy_in_batches(const Job& J, Ctr* C, uint32_t n, bool perm)
{
    __shared__ uint32_t s_f;
    const int tid = threadIdx.x;
    const uint32_t NA = J.vm_na, NP = J.vm_na_cap + J.vm_pool;
    const uint32_t gtid = blockIdx.x * VM_BLOCK + tid, gstride = gridDim.x * VM_BLOCK;
    const bool tail_partial = (n & ((1u << J.vm_plog2) - 1)) != 0;
    // targets per batch: pool - 1, rounded down to a multiple of the grid
    // when that leaves at least one per CTA (every CTA then copies as many
    // pages as the others in each step)
    const uint32_t BMAX = J.vm_pool - 1 >= gridDim.x ? (J.vm_pool - 1) / gridDim.x * gridDim.x : J.vm_pool - 1;
    uint32_t* stack[2] = {J.free_stack, J.free_stack + NP};
    // a page that may serve as a free page for batches ending before qend
    auto usable = [&](uint32_t p, uint32_t qend) {
        if (p >= J.vm_na_cap) return true;                    // a pool page
        return p < NA && p >= qend && !(tail_partial && p + 1 == NA);
    };
    // the first batch's free pages
    {
        const uint32_t q1 = min(BMAX, NA);
        for (uint32_t p = gtid; p < NP; p += gstride)
            if (usable(p, q1) && J.holder[p] == NONE) stack[0][atomicAdd(&C->vm_copy_top[0], 1u)] = p;
    }
    if (!grid_barrier(C)) return false;
    for (uint32_t q0 = 0, k = 0; q0 < NA; ++k) {
        const uint32_t cur = k & 1u, nxt = cur ^ 1u;
        const uint32_t q1 = q0 + min(BMAX, NA - q0);
        const uint32_t q2 = q1 + min(BMAX, NA - q1);
        // step 1: move needed data out of the batch's targets (a CTA per target)
        if (gtid == 0) {
            C->vm_copy_top[nxt] = 0;          // the next batch's stack fills in step 2
            C->vm_copy_taken[nxt] = 0;
        }
        for (uint32_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
            const uint32_t r = __ldcg(J.holder + q);
            if (r == NONE || r == q) continue;
            if (tid == 0) {
                const uint32_t at = atomicAdd(&C->vm_copy_taken[cur], 1u);
                s_f = at < __ldcg(&C->vm_copy_top[cur]) ? __ldcg(stack[cur] + at) : NONE;
                if (s_f == NONE) set_error(C, DERR_INTERNAL, 65);
            }
            __syncthreads();
            const uint32_t f = s_f;
            if (f != NONE) vm_copy_page(J, f, q, page_size(J, r, n), perm);
            __syncthreads();
            if (tid == 0 && f != NONE) {
                J.pt[r] = f;
                J.holder[f] = r;
                J.holder[q] = NONE;
                atomicAdd(&C->vm_copy_moves, 1u);
            }
        }
        if (!grid_barrier(C)) return false;
        if (*(volatile uint32_t*)&C->error) return false;
        // step 2: every target receives its own data (a CTA per target); the
        // freed sources and the unused free pages that the next batch may use
        // go onto the other stack
        for (uint32_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
            const uint32_t src = __ldcg(J.pt + q);
            if (src == q) continue;
            vm_copy_page(J, q, src, page_size(J, q, n), perm);
            __syncthreads();
            if (tid == 0) {
                J.holder[src] = NONE;
                J.pt[q] = q;
                J.holder[q] = q;
                atomicAdd(&C->vm_copy_moves, 1u);
                if (usable(src, q2)) stack[nxt][atomicAdd(&C->vm_copy_top[nxt], 1u)] = src;
            }
        }
        {
            const uint32_t top = __ldcg(&C->vm_copy_top[cur]);
            const uint32_t taken = min(__ldcg(&C->vm_copy_taken[cur]), top);
            for (uint32_t i = taken + gtid; i < top; i += gstride) {
                const uint32_t p = __ldcg(stack[cur] + i);
                if (usable(p, q2)) stack[nxt][atomicAdd(&C->vm_copy_top[nxt], 1u)] = p;
            }
        }
        if (!grid_barrier(C)) return false;
        q0 = q1;
    }
    return true;
}

// Pointer jumping over the predecessor links: after the rounds, a target on
// a chain has anc = NONE and dist = its rank (moves before it on its chain);
// a target on a cycle keeps anc != NONE, and min is the smallest target on
// its cycle (the jumps have covered it).  Returns the buffer the result is in.
__device__ int copy_rank(const Job& J, Ctr* C, uint32_t* W, uint32_t NAC, uint32_t NA, int rounds, bool& ok)
{
    const uint32_t gtid = blockIdx.x * VM_BLOCK + threadIdx.x, gstride = gridDim.x * VM_BLOCK;
    int cur = 0;
    for (int r = 0; r < rounds; ++r) {
        const uint32_t* anc = W + (cur ? CW_ANC1 : CW_ANC0) * NAC;
        const uint32_t* dist = W + (cur ? CW_DIST1 : CW_DIST0) * NAC;
        const uint32_t* mn = W + (cur ? CW_MIN1 : CW_MIN0) * NAC;
        uint32_t* anc2 = W + (cur ? CW_ANC0 : CW_ANC1) * NAC;
        uint32_t* dist2 = W + (cur ? CW_DIST0 : CW_DIST1) * NAC;
        uint32_t* mn2 = W + (cur ? CW_MIN0 : CW_MIN1) * NAC;
        for (uint32_t u = gtid; u < NA; u += gstride) {
            const uint32_t a = __ldcg(anc + u);
            uint32_t d = __ldcg(dist + u), m = __ldcg(mn + u), a2 = NONE;
            if (a != NONE && a < NA) {
                a2 = __ldcg(anc + a);
                d += __ldcg(dist + a);
                m = min(m, __ldcg(mn + a));
            }
            anc2[u] = a2;
            dist2[u] = d;
            mn2[u] = m;
        }
        cur ^= 1;
        if (!grid_barrier(C)) {
            ok = false;
            return cur;
        }
    }
    ok = true;
    return cur;
}

// Two array pages that hold each other's data (a cycle of two) trade it by
// one CTA, every thread loading both of its words before storing either:
// page u receives cu elements from v, page v receives cv from u.
__device__ __noinline__ void vm_swap_pages(const Job& J, uint32_t u, uint32_t v, uint32_t cu, uint32_t cv, bool perm)
{
    const bool vec = ((reinterpret_cast<uintptr_t>(J.keysA) | reinterpret_cast<uintptr_t>(J.permA)) & 15u) == 0;
    for (int pass = 0; pass < (perm ? 2 : 1); ++pass) {
        uint32_t* a = pass ? phys_p(J, u) : phys_k(J, u);
        uint32_t* b = pass ? phys_p(J, v) : phys_k(J, v);
        const uint32_t na = vec ? cu >> 2 : 0u, nb = vec ? cv >> 2 : 0u, nv = max(na, nb);
        uint4* a4 = reinterpret_cast<uint4*>(a);
        uint4* b4 = reinterpret_cast<uint4*>(b);
        for (uint32_t i = threadIdx.x; i < nv; i += VM_BLOCK) {
            uint4 x = make_uint4(0u, 0u, 0u, 0u), y = x;
            if (i < na) x = __ldcg(b4 + i);
            if (i < nb) y = __ldcg(a4 + i);
            if (i < na) a4[i] = x;
            if (i < nb) b4[i] = y;
        }
        for (uint32_t i = threadIdx.x; i < max(cu, cv); i += VM_BLOCK) {
            const bool ia = i >= (na << 2) && i < cu, ib = i >= (nb << 2) && i < cv;
            const uint32_t x = ia ? __ldcg(b + i) : 0u, y = ib ? __ldcg(a + i) : 0u;
            if (ia) a[i] = x;
            if (ib) b[i] = y;
        }
    }
}

// Temporary pages of the chain walk beyond the pool: page-sized slots (keys,
// then permutation) in the page-record table past the walk's own scratch,
// then in the split table.  Slot ids follow the physical page ids.
struct CopySlots {
    uint32_t* a;      // first region and its slots
    uint32_t na;
    uint32_t* b;      // second region and its slots
    uint32_t nb;
    uint32_t* c;      // third region (the free-page ring past Copy's two lists) and its slots
    uint32_t nc;
};

__device__ __forceinline__ CopySlots copy_slots(const Job& J)
{
    const size_t P = (size_t)1 << J.vm_plog2, NAC = J.vm_na_cap, NP = NAC + J.vm_pool;
    const size_t a0 = ((CW_COUNTERS * NAC + CC_WORDS) + 3) & ~(size_t)3;     // 16-byte aligned
    const size_t c0 = (2 * NP + 3) & ~(size_t)3;
    const size_t a_words = (size_t)VM_REC_WORDS * NAC, b_words = (NAC + 1) * VM_SPLIT_WORDS;
    CopySlots c;
    c.a = J.vm_rec + a0;
    c.na = a_words > a0 ? (uint32_t)((a_words - a0) / (2 * P)) : 0u;
    c.b = J.vm_split_at;
    c.nb = (uint32_t)(b_words / (2 * P));
    c.c = J.free_stack + c0;
    c.nc = J.vm_ring_cap > c0 ? (uint32_t)((J.vm_ring_cap - c0) / (2 * P)) : 0u;
    return c;
}

__device__ __noinline__ uint32_t* temp_k(const Job& J, uint32_t NP, uint32_t id)
{
    if (id < NP) return phys_k(J, id);
    const CopySlots cs = copy_slots(J);
    const size_t P = (size_t)1 << J.vm_plog2;
    const uint32_t i = id - NP;
    if (i < cs.na) return cs.a + 2 * P * i;
    if (i < cs.na + cs.nb) return cs.b + 2 * P * (i - cs.na);
    return cs.c + 2 * P * (i - cs.na - cs.nb);
}

__device__ __forceinline__ uint32_t* temp_p(const Job& J, uint32_t NP, uint32_t id)
{
    if (id < NP) return phys_p(J, id);
    return temp_k(J, NP, id) + ((size_t)1 << J.vm_plog2);
}

__global__ void __launch_bounds__(VM_BLOCK, 4) k_vm_copy(Job J)
{
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    __shared__ uint32_t s_cnt[CC_WORDS];
    const int tid = threadIdx.x;
    const bool perm = J.want_perm != 0;
    const uint32_t n = J.inst[0].n;
    const uint32_t NA = J.vm_na, NAC = J.vm_na_cap, NP = J.vm_na_cap + J.vm_pool;
    const uint32_t gtid = blockIdx.x * VM_BLOCK + tid, gstride = gridDim.x * VM_BLOCK;
    uint32_t* W = J.vm_rec;                         // the chain walk's scratch
    uint32_t* cnt = W + CW_COUNTERS * NAC;         // its counters
    uint32_t* free_pool = J.free_stack;            // free pool pages
    uint32_t* seg = J.free_stack + NP;             // segment starts
    // 1. holder[p]: the virtual page whose data physical page p holds
    for (uint32_t p = gtid; p < NP; p += gstride) J.holder[p] = NONE;
    if (gtid < CC_WORDS) cnt[gtid] = 0;
    if (gtid == 0) {
        C->vm_copy_top[0] = C->vm_copy_top[1] = 0;
        C->vm_copy_taken[0] = C->vm_copy_taken[1] = 0;
    }
    if (!grid_barrier(C)) return;
    for (uint32_t u = gtid; u < NA; u += gstride) J.holder[J.pt[u]] = u;
    if (!grid_barrier(C)) return;
    if (J.vm_batched_copy) {                       // the batched order, asked for
        copy_in_batches(J, C, n, perm);
        return;
    }
    // the free pool pages; every target's predecessor link (the target whose
    // data it holds) and rank 1, or none and rank 0 at a chain's start
    for (uint32_t p = NAC + gtid; p < NP; p += gstride)
        if (J.holder[p] == NONE) free_pool[atomicAdd(&C->vm_copy_top[0], 1u)] = p;
    {
        const CopySlots cs = copy_slots(J);
        for (uint32_t i = gtid; i < cs.na + cs.nb + cs.nc; i += gstride)
            free_pool[atomicAdd(&C->vm_copy_top[0], 1u)] = NP + i;
    }
    for (uint32_t u = gtid; u < NA; u += gstride) {
        const uint32_t pu = J.pt[u];
        const uint32_t h = J.holder[u];
        // a cycle of two trades its pages directly and stays out of the ranks
        const bool swap = pu != u && pu < NA && h == pu;
        const bool done = pu == u || swap;
        W[CW_FLAGS * NAC + u] = (done ? CF_DONE : 0u) | (swap ? CF_SWAP : 0u);
        W[CW_ANC0 * NAC + u] = (done || h == NONE) ? NONE : h;
        W[CW_DIST0 * NAC + u] = (done || h == NONE) ? 0u : 1u;
        W[CW_MIN0 * NAC + u] = u;
    }
    if (!grid_barrier(C)) return;
    // 2. ranks by pointer jumping (2^rounds > NA covers every chain and cycle)
    const int rounds = 33 - __clz(max(NA, 1u));
    bool ok = true;
    int fin = copy_rank(J, C, W, NAC, NA, rounds, ok);
    if (!ok) return;
    // targets on cycles: the smallest of each is its start; rank again with
    // the starts' links cut (the chains' ranks stay)
    for (uint32_t u = gtid; u < NA; u += gstride) {
        const uint32_t f = W[CW_FLAGS * NAC + u];
        if (f & CF_DONE) continue;
        if (W[(fin ? CW_ANC1 : CW_ANC0) * NAC + u] != NONE) {
            W[CW_FLAGS * NAC + u] = f | CF_CYCLE;
            if (W[(fin ? CW_MIN1 : CW_MIN0) * NAC + u] == u) atomicAdd(&cnt[CC_CYCLES], 1u);
            cnt[CC_ANY_CYCLE] = 1u;
        }
    }
    if (!grid_barrier(C)) return;
    if (__ldcg(&cnt[CC_CYCLES]) > __ldcg(&C->vm_copy_top[0])) {
        // more cycles than temporaries: batches (before ranking again)
        if (gtid == 0) C->vm_copy_top[0] = 0;
        if (!grid_barrier(C)) return;
        copy_in_batches(J, C, n, perm);
        return;
    }
    if (__ldcg(&cnt[CC_ANY_CYCLE])) {
        for (uint32_t u = gtid; u < NA; u += gstride) {
            const uint32_t f = W[CW_FLAGS * NAC + u];
            uint32_t a = NONE, d = 0;
            if (f & CF_CYCLE) {
                const bool start = W[(fin ? CW_MIN1 : CW_MIN0) * NAC + u] == u;
                a = start ? NONE : J.holder[u];
                d = start ? 0u : 1u;
            } else if (!(f & CF_DONE)) {
                d = W[(fin ? CW_DIST1 : CW_DIST0) * NAC + u];
            }
            W[CW_ANC0 * NAC + u] = a;
            W[CW_DIST0 * NAC + u] = d;
            W[CW_MIN0 * NAC + u] = u;
        }
        if (!grid_barrier(C)) return;
        fin = copy_rank(J, C, W, NAC, NA, rounds, ok);
        if (!ok) return;
    }
    const uint32_t* rank = W + (fin ? CW_DIST1 : CW_DIST0) * NAC;
    // 3. saves needed for every segment length 2^k: the targets of rank > 0
    //    divisible by 2^k, plus one per cycle; and the moves to make
    for (int i = tid; i < CC_WORDS; i += VM_BLOCK) s_cnt[i] = 0;
    __syncthreads();
    for (uint32_t u = gtid; u < NA; u += gstride) {
        if (W[CW_FLAGS * NAC + u] & CF_DONE) continue;
        const uint32_t rk = __ldcg(rank + u);
        atomicAdd(&s_cnt[CC_MOVES], 1u);
        if (rk == 0) continue;
        for (uint32_t k = 0; k < COPY_KMAX; ++k)
            if ((rk & ((1u << k) - 1u)) == 0) atomicAdd(&s_cnt[k], 1u);
    }
    __syncthreads();
    for (int i = tid; i < (int)CC_CYCLES; i += VM_BLOCK)
        if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
    if (tid == 0 && s_cnt[CC_MOVES]) atomicAdd(&cnt[CC_MOVES], s_cnt[CC_MOVES]);
    if (!grid_barrier(C)) return;
    // every thread takes the same S
    const uint32_t nfree = __ldcg(&C->vm_copy_top[0]), ncyc = __ldcg(&cnt[CC_CYCLES]);
    const uint32_t moves = __ldcg(&cnt[CC_MOVES]);
    uint32_t k = 0;
    while (k + 1 < COPY_KMAX && (1u << k) * 2u * gridDim.x < moves) ++k;   // at least the moves per CTA / 2
    while (k < COPY_KMAX && __ldcg(&cnt[k]) + ncyc > nfree) ++k;
    if (k >= COPY_KMAX || (1u << k) > COPY_SEG_MAX) {
        // the chains do not split into short enough segments: batches
        if (gtid == 0) C->vm_copy_top[0] = 0;
        if (!grid_barrier(C)) return;
        copy_in_batches(J, C, n, perm);
        return;
    }
    const uint32_t S = 1u << k;
    // the segment starts, and a free pool page for the data of every one
    // that holds data (a cycle's start, or rank > 0 divisible by S)
    for (uint32_t u = gtid; u < NA; u += gstride) {
        const uint32_t f = W[CW_FLAGS * NAC + u];
        if ((f & CF_SWAP) && u < J.pt[u]) seg[atomicAdd(&C->vm_copy_top[1], 1u)] = u;   // a pair, once
        if (f & CF_DONE) continue;
        const uint32_t rk = __ldcg(rank + u);
        if ((rk & (S - 1u)) != 0) continue;
        if (rk > 0 || (f & CF_CYCLE)) {
            const uint32_t at = atomicAdd(&C->vm_copy_taken[0], 1u);
            if (at >= nfree) {
                set_error(C, DERR_INTERNAL, 69);
                continue;
            }
            W[CW_TEMP * NAC + u] = __ldcg(free_pool + at);
            W[CW_FLAGS * NAC + u] = f | CF_SAVED;
        }
        seg[atomicAdd(&C->vm_copy_top[1], 1u)] = u;
    }
    if (!grid_barrier(C)) return;
    if (*(volatile uint32_t*)&C->error) return;
    const uint32_t nseg = __ldcg(&C->vm_copy_top[1]);
    // the saves (a CTA per page): the data a segment start holds is its
    // predecessor's
    uint32_t made = 0;
    for (uint32_t i = blockIdx.x; i < nseg; i += gridDim.x) {
        const uint32_t u = __ldcg(seg + i);
        if (!(__ldcg(W + CW_FLAGS * NAC + u) & CF_SAVED)) continue;
        const uint32_t t = __ldcg(W + CW_TEMP * NAC + u);
        vm_copy_keys_perm(J, temp_k(J, NP, t), temp_p(J, NP, t), phys_k(J, u), phys_p(J, u),
                          page_size(J, J.holder[u], n), perm);
        ++made;
    }
    // every target's move, so that a walk reads one step ahead: the page it
    // receives its data from (the saved copy when pt[u] starts a segment),
    // and the next target of its segment (NONE: the segment ends here)
    uint32_t* msrc = W + CW_MIN0 * NAC;
    uint32_t* mnext = W + CW_MIN1 * NAC;
    for (uint32_t u = gtid; u < NA; u += gstride) {
        const uint32_t p = J.pt[u];
        const bool target = p < NA;
        const bool saved = target && (W[CW_FLAGS * NAC + p] & CF_SAVED);
        msrc[u] = saved ? W[CW_TEMP * NAC + p] : p;
        mnext[u] = (!target || saved) ? NONE : p;
    }
    if (!grid_barrier(C)) return;
    // 4. the walks (a CTA per segment): u receives its data from pt[u] -- or
    //    from the saved copy when pt[u] starts the next segment, which ends
    //    this one; a pool page ends the chain
    for (uint32_t i = blockIdx.x; i < nseg; i += gridDim.x) {
        uint32_t u = __ldcg(seg + i);
        if (__ldcg(W + CW_FLAGS * NAC + u) & CF_SWAP) {
            const uint32_t v = __ldcg(J.pt + u);
            vm_swap_pages(J, u, v, page_size(J, u, n), page_size(J, v, n), perm);
            made += 2;
            continue;
        }
        uint32_t src = __ldcg(msrc + u), nxt = __ldcg(mnext + u);
        for (uint32_t step = 0;; ++step) {
            if (step > S) {                         // never expected: a segment has at most S moves
                if (tid == 0) set_error(C, DERR_INTERNAL, 70);
                break;
            }
            // the next step's move flies with this step's copy
            const uint32_t src2 = nxt < NA ? __ldcg(msrc + nxt) : 0u;
            const uint32_t nxt2 = nxt < NA ? __ldcg(mnext + nxt) : NONE;
            vm_copy_keys_perm(J, phys_k(J, u), phys_p(J, u), temp_k(J, NP, src), temp_p(J, NP, src),
                              page_size(J, u, n), perm);
            ++made;
            __syncthreads();                       // u's loads of its source are complete before it is written
            if (nxt >= NA) break;
            u = nxt;
            src = src2;
            nxt = nxt2;
        }
    }
    if (tid == 0 && made) atomicAdd(&C->vm_copy_moves, made);
    if (!grid_barrier(C)) return;
    for (uint32_t u = gtid; u < NA; u += gstride) J.pt[u] = u;
}

int vm_rounds_max_grid(int num_sms)
{
    // both cooperative kernels run on this grid: the smaller residency
    int per_sm = 0, copy_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vm_rounds, VM_BLOCK, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&copy_per_sm, k_vm_copy, VM_BLOCK, 0);
    if (copy_per_sm < per_sm) per_sm = copy_per_sm;
    if (per_sm > 6) per_sm = 6;
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

uint32_t vm_groups_per_cta(uint32_t plog2)
{
    const uint32_t w = plog2 >= 9 ? std::min(1u << (plog2 - 9), (uint32_t)VM_WARPS) : 1u;
    return VM_WARPS / w;
}

cudaError_t launch_vm(const Job& J, int grid, cudaStream_t s)
{
    void* args[] = {(void*)&J};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_vm_rounds, dim3(grid), dim3(VM_BLOCK), args, 0, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void*)k_vm_copy, dim3(grid), dim3(VM_BLOCK), args, 0, s);
}

}  // namespace ps
