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
// Rounds run in waves of at most vm_wave_max output pages, in page order, each
// wave taking its pages from the stack: a merge consumes exactly as many
// input elements as it writes, so the pages freed by one wave cover the next
// one, and the pool needs only about one wave of pages plus a few partly
// consumed pages -- not n elements.  Every merge-path split a page needs (at
// page boundaries inside a merge) is searched at the start of the round, all
// pages in parallel, while every input page still holds its data; the waves
// then only stream.  Finally Copy (Sec. 4) moves every virtual page to its own
// array page: a page still holding data that is needed later is first moved
// to a free page, exactly as the paper describes.
#include <algorithm>

#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr int VM_BLOCK = 256;
constexpr int VM_WARPS = VM_BLOCK / 32;
constexpr int VM_K = 16;                  // outputs per thread of a merge sub-chunk
constexpr int VM_SLOTS = VM_BLOCK * VM_K + 8 * VM_WARPS;   // staging words per CTA

// A CTA works on several output pages at once: groups of W warps, W = P / 512
// clamped to 1..8, each group merging sub-chunks of 512 W = 16 x its threads
// outputs (at least one page) in its own slice of shared memory, with its own
// named barrier.
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

__device__ bool vm_barrier(Ctr* C)
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
            const long long t0 = clock64();
            uint32_t nap = 64;
            while (ld_relaxed_u32(&C->bar_gen) == gen) {
                __nanosleep(nap);
                nap = nap < 1024 ? nap * 2 : 1024;
                if (clock64() - t0 > SPIN_LIMIT_CYCLES) {
                    set_error(C, DERR_TIMEOUT, 60);
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

// Left-child elements among the first d outputs of merge g (merge path over
// the page-table-translated keys).
__device__ uint32_t vm_split(const Job& J, const GSorted& g, uint32_t d)
{
    const uint32_t lo = (uint32_t)g.goff, mid = lo + g.la;
    uint32_t l = d > g.lb ? d - g.lb : 0u;
    uint32_t h = min(d, g.la);
    while (l < h) {
        const uint32_t m = (l + h) >> 1;
        if (vkey(J, lo + m) <= vkey(J, mid + d - 1 - m)) l = m + 1; else h = m;
    }
    return l;
}

// Count `cnt` consumed elements of virtual range [v0, v0 + cnt); a page whose
// every element is consumed goes back to the free stack.
__device__ void consume(const Job& J, uint32_t v0, uint32_t cnt, uint32_t n)
{
    const uint32_t L = J.vm_plog2;
    while (cnt) {
        const uint32_t u = v0 >> L;
        const uint32_t take = min(cnt, ((u + 1) << L) - v0);
        const uint32_t before = atomicAdd(&J.consumed[u], take);
        if (before + take == page_size(J, u, n)) {
            // the caller's last array page may be partial: like the paper's partial
            // input page it is never declared free (it could not hold a full page)
            const uint32_t old = J.pt[u];
            const bool partial_tail = old + 1 == J.vm_na && (n & ((1u << J.vm_plog2) - 1)) != 0;
            if (!partial_tail) {
                const uint32_t at = atomicAdd(&J.ctr->vm_free_top, 1u);
                J.free_stack[at] = old;
            }
        }
        v0 += take;
        cnt -= take;
    }
}

struct VmSmem {
    uint32_t k[VM_SLOTS];
    uint32_t p[VM_SLOTS];
    uint32_t seg_lo[VM_WARPS][6], seg_hi[VM_WARPS][6], seg_node[VM_WARPS][6];
    uint32_t nseg[VM_WARPS];
    uint32_t a[VM_WARPS][2];
};

// One output page of the current wave, by one group: its merge segments and
// copy gaps.
__device__ void vm_page(const Job& J, VmSmem& sm, const VmGroup& G, uint32_t u, uint32_t n, bool perm)
{
    const uint32_t tid = G.tid, gi = G.g;
    uint32_t* sk = sm.k + gi * (G.cap + 8);
    uint32_t* sp = sm.p + gi * (G.cap + 8);
    const uint32_t L = J.vm_plog2;
    const uint32_t ps0 = u << L, pe = min(ps0 + (1u << L), n);
    uint32_t* dk = phys_k(J, J.pt_new[u]);
    uint32_t* dp = perm ? phys_p(J, J.pt_new[u]) : nullptr;
    if (tid == 0) {
        // up to two merges touch the page; order them, fill the gaps with copies
        uint32_t e[2] = {NONE, NONE};
        const uint32_t c = min(J.page_cnt[u], 2u);
        for (uint32_t i = 0; i < c; ++i) e[i] = J.page_nodes[2 * u + i];
        if (c == 2 && J.gsorted[e[0]].goff > J.gsorted[e[1]].goff) {
            const uint32_t t = e[0];
            e[0] = e[1];
            e[1] = t;
        }
        uint32_t cur = ps0, ns = 0;
        for (uint32_t i = 0; i < c; ++i) {
            const GSorted g = J.gsorted[e[i]];
            const uint32_t lo = (uint32_t)g.goff, hi = lo + g.la + g.lb;
            const uint32_t s0 = max(lo, ps0), s1 = min(hi, pe);
            if (s0 >= s1) continue;
            if (s0 > cur) { sm.seg_lo[gi][ns] = cur; sm.seg_hi[gi][ns] = s0; sm.seg_node[gi][ns] = NONE; ++ns; }
            sm.seg_lo[gi][ns] = s0; sm.seg_hi[gi][ns] = s1; sm.seg_node[gi][ns] = e[i]; ++ns;
            cur = s1;
        }
        if (cur < pe) { sm.seg_lo[gi][ns] = cur; sm.seg_hi[gi][ns] = pe; sm.seg_node[gi][ns] = NONE; ++ns; }
        sm.nseg[gi] = ns;
    }
    group_sync(G);
    const uint32_t nseg = sm.nseg[gi];
    for (uint32_t sg = 0; sg < nseg; ++sg) {
        const uint32_t s0 = sm.seg_lo[gi][sg], s1 = sm.seg_hi[gi][sg], e = sm.seg_node[gi][sg];
        if (e == NONE) {                         // carried over unchanged (a gap)
#pragma unroll 8
            for (uint32_t v = s0 + tid; v < s1; v += G.nthr) {
                const uint32_t ph = J.pt[v >> L], off = v & ((1u << L) - 1u);
                dk[v - ps0] = phys_k(J, ph)[off];
                if (dp) dp[v - ps0] = phys_p(J, ph)[off];
            }
            group_sync(G);
            if (tid == 0) consume(J, s0, s1 - s0, n);
            continue;
        }
        const GSorted g = J.gsorted[e];
        const uint32_t lo = (uint32_t)g.goff, mid = lo + g.la;
        for (uint32_t x0 = s0; x0 < s1; x0 += G.cap) {
            const uint32_t x1 = min(x0 + G.cap, s1);
            const uint32_t d0 = x0 - lo, d1 = x1 - lo;
            if (tid < 2) {
                // the splits at the merge's ends are 0 and la; at a page start
                // inside the merge the round's search left it in vm_split_at
                // (a sub-chunk always holds a whole page, so no other boundary
                // occurs)
                const uint32_t x = tid == 0 ? x0 : x1, d = x - lo;
                uint32_t a;
                if (d == 0) a = 0;
                else if (d == g.la + g.lb) a = g.la;
                else if ((x & ((1u << L) - 1u)) == 0) a = J.vm_split_at[x >> L];
                else { a = 0; set_error(J.ctr, DERR_INTERNAL, 65); }   // a sub-chunk holds a whole page
                sm.a[gi][tid] = a;
            }
            group_sync(G);
            const uint32_t a0 = sm.a[gi][0], a1 = sm.a[gi][1], b0 = d0 - a0, b1 = d1 - a1;
            const uint32_t na = a1 - a0, nb = b1 - b0, cnt = na + nb;
            // the slices' keys (and permutation) through the page table; eight
            // iterations per thread in flight at once
#pragma unroll 8
            for (uint32_t i = tid; i < cnt; i += G.nthr) {
                const uint32_t v = i < na ? lo + a0 + i : mid + b0 + (i - na);
                const uint32_t ph = J.pt[v >> L], off = v & ((1u << L) - 1u);
                sk[i] = phys_k(J, ph)[off];
                if (perm) sp[i] = phys_p(J, ph)[off];
            }
            group_sync(G);
            // each thread merges VM_K consecutive outputs straight into the
            // fresh output page (a pool page nobody else reads this wave)
            const uint32_t t0 = tid * VM_K;
            if (t0 < cnt) {
                uint32_t l = t0 > nb ? t0 - nb : 0u, h = min(t0, na);
                while (l < h) {
                    const uint32_t m = (l + h) >> 1;
                    if (sk[m] <= sk[na + t0 - 1 - m]) l = m + 1; else h = m;
                }
                uint32_t ia = l, ib = na + (t0 - l);
                uint32_t* ok = dk + (x0 - ps0) + t0;
                uint32_t* op = dp ? dp + (x0 - ps0) + t0 : nullptr;
#pragma unroll 4
                for (int j = 0; j < VM_K; ++j) {
                    if (t0 + j < cnt) {
                        const bool ta = ia < na && (ib >= cnt || sk[ia] <= sk[ib]);
                        const uint32_t src = ta ? ia : ib;
                        ok[j] = sk[src];
                        if (op) op[j] = sp[src];
                        ia += ta;
                        ib += !ta;
                    }
                }
            }
            group_sync(G);
            if (tid == 0) {
                consume(J, lo + a0, na, n);
                consume(J, mid + b0, nb, n);
            }
        }
    }
}

}  // namespace

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

    for (int r = 0; r < NPOW; ++r) {
        if (*(volatile uint32_t*)&C->error) return;
        const uint32_t e0 = C->bucket_start[r], e1 = C->bucket_start[r + 1];
        if (e0 == e1) continue;
        // 1. the pages each merge of the round touches (a warp per merge)
        for (uint32_t e = e0 + gwarp; e < e1; e += nwarps_grid) {
            const GSorted g = J.gsorted[e];
            const uint32_t lo = (uint32_t)g.goff, hi = lo + g.la + g.lb;
            const uint32_t first = lo >> L, last = (hi - 1) >> L;
            for (uint32_t u = first + lane; u <= last; u += 32) {
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
        if (!vm_barrier(C)) return;
        // 1b. the merge-path split at every page start that lies inside a merge,
        //     one thread per page, before any input page can be recycled
        for (uint32_t u = blockIdx.x * VM_BLOCK + tid; u < NA; u += gridDim.x * VM_BLOCK) {
            const uint32_t c = min(J.page_cnt[u], 2u), ps0 = u << L;
            for (uint32_t i = 0; i < c; ++i) {
                const GSorted g = J.gsorted[J.page_nodes[2 * u + i]];
                const uint32_t lo = (uint32_t)g.goff;
                if (lo < ps0 && ps0 < lo + g.la + g.lb) J.vm_split_at[u] = vm_split(J, g, ps0 - lo);
            }
        }
        if (!vm_barrier(C)) return;
        // 2. the touched pages, in page order (CTA 0; each thread takes
        //    TOUCH_PER consecutive pages per pass)
        if (blockIdx.x == 0) {
            constexpr uint32_t TOUCH_PER = 8;
            uint32_t carry = 0;
            for (uint32_t base = 0; base < NA; base += VM_BLOCK * TOUCH_PER) {
                const uint32_t u0 = base + tid * TOUCH_PER;
                uint32_t flags = 0;
#pragma unroll
                for (uint32_t i = 0; i < TOUCH_PER; ++i)
                    if (u0 + i < NA && J.page_cnt[u0 + i] > 0) flags |= 1u << i;
                const uint32_t c = __popc(flags);
                uint32_t x = c;                       // inclusive warp scan of the counts
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) warp_sums[warp] = x;
                __syncthreads();
                uint32_t before = carry + x - c, tot = 0;
                for (int w = 0; w < VM_BLOCK / 32; ++w) {
                    if (w < warp) before += warp_sums[w];
                    tot += warp_sums[w];
                }
                for (uint32_t i = 0; i < TOUCH_PER; ++i)
                    if (flags & (1u << i)) J.touched[before++] = u0 + i;
                carry += tot;
                __syncthreads();
            }
            if (tid == 0) C->vm_touched = carry;
        }
        if (!vm_barrier(C)) return;
        // 3. waves of output pages
        const uint32_t ntouched = C->vm_touched;
        for (uint32_t pos = 0; pos < ntouched;) {
            if (blockIdx.x == 0) {
                // the wave's output pages come off the top of the free stack
                __shared__ uint32_t s_top, s_k;
                if (tid == 0) {
                    const uint32_t top = C->vm_free_top;
                    const uint32_t k = min(min(J.vm_wave_max, top), ntouched - pos);
                    if (k == 0) set_error(C, DERR_INTERNAL, 62);      // no free page: cannot progress
                    C->vm_free_top = top - k;
                    C->vm_wave = k;
                    C->vm_waves += 1;
                    const uint32_t extra = J.vm_pool > top - k ? J.vm_pool - (top - k) : 0u;   // pages beyond n/P
                    if (extra > C->vm_in_use_peak) C->vm_in_use_peak = extra;
                    s_top = top;
                    s_k = k;
                }
                __syncthreads();
                for (uint32_t j = tid; j < s_k; j += VM_BLOCK) J.pt_new[J.touched[pos + j]] = J.free_stack[s_top - 1 - j];
            }
            if (!vm_barrier(C)) return;
            if (*(volatile uint32_t*)&C->error) return;
            const uint32_t k = C->vm_wave;
            const VmGroup G = vm_group(L);
            for (uint32_t j = blockIdx.x * G.groups + G.g; j < k; j += gridDim.x * G.groups)
                vm_page(J, sm, G, J.touched[pos + j], n, perm);
            if (!vm_barrier(C)) return;
            pos += k;
        }
        // 4. the written pages become current; reset the per-round tables
        for (uint32_t j = blockIdx.x * VM_BLOCK + tid; j < ntouched; j += gridDim.x * VM_BLOCK) {
            const uint32_t u = J.touched[j];
            J.pt[u] = J.pt_new[u];
            J.page_cnt[u] = 0;
            J.consumed[u] = 0;
        }
        if (!vm_barrier(C)) return;
    }
}

// Copy (Sec. 4), in batches of target pages.  The paper walks the virtual
// pages in order: a target array page that still holds data needed later is
// first moved out to a free page, then the page's own data is copied in.
// Here a batch of up to `pool` consecutive targets does the same in two
// parallel steps: (1) every target of the batch that holds another page's
// data moves it out to a free page; (2) every target receives its own data.
// After step 1 no target of the batch holds needed data, so the copies of
// step 2 never overwrite a source; each copy frees its source, so the number
// of free pages is the same after every batch.  Counting pages shows that
// with at most pool - 1 targets per batch the free pages cover every move out.
__device__ void vm_copy_page(const Job& J, uint32_t dst, uint32_t src, uint32_t cnt, bool perm)
{
    uint32_t* dk = phys_k(J, dst);
    const uint32_t* sk = phys_k(J, src);
    for (uint32_t i = threadIdx.x; i < cnt; i += VM_BLOCK) dk[i] = sk[i];
    if (perm) {
        uint32_t* dp = phys_p(J, dst);
        const uint32_t* sp = phys_p(J, src);
        for (uint32_t i = threadIdx.x; i < cnt; i += VM_BLOCK) dp[i] = sp[i];
    }
}

__global__ void __launch_bounds__(VM_BLOCK) k_vm_copy(Job J)
{
    __shared__ uint32_t s_src;
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    const int tid = threadIdx.x;
    const bool perm = J.want_perm != 0;
    const uint32_t n = J.inst[0].n;
    const uint32_t NA = J.vm_na, NP = J.vm_na_cap + J.vm_pool;
    const uint32_t gtid = blockIdx.x * VM_BLOCK + tid, gstride = gridDim.x * VM_BLOCK;
    const bool tail_partial = (n & ((1u << J.vm_plog2) - 1)) != 0;
    // holder[p]: the virtual page whose data physical page p holds (NONE: none)
    for (uint32_t p = gtid; p < NP; p += gstride) J.holder[p] = NONE;
    if (!vm_barrier(C)) return;
    for (uint32_t u = gtid; u < NA; u += gstride) J.holder[J.pt[u]] = u;
    if (!vm_barrier(C)) return;
    for (uint32_t q0 = 0; q0 < NA;) {
        // at most pool - 1 targets: then the free pages always cover the moves out
        // (one page of slack for the partial last array page, which is never free)
        const uint32_t B = min(J.vm_pool - 1, NA - q0);
        const uint32_t q1 = q0 + B;
        // free pages: hold nothing, are not a target of this or an earlier batch,
        // and are not the partial last array page
        if (gtid == 0) {
            C->vm_free_top = 0;
            C->vm_wave = 0;
        }
        if (!vm_barrier(C)) return;
        for (uint32_t p = gtid; p < NP; p += gstride) {
            if (p >= J.vm_na_cap && p - J.vm_na_cap >= J.vm_pool) continue;
            const bool is_array = p < J.vm_na_cap;
            if (is_array && (p >= NA || p < q1)) continue;
            if (is_array && tail_partial && p + 1 == NA) continue;
            if (J.holder[p] == NONE) J.free_stack[atomicAdd(&C->vm_free_top, 1u)] = p;
        }
        if (!vm_barrier(C)) return;
        // step 1: move needed data out of the batch's targets
        for (uint32_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
            const uint32_t r = J.holder[q];
            if (r == NONE || r == q) continue;
            if (tid == 0) {
                const uint32_t at = atomicAdd(&C->vm_wave, 1u);
                s_src = at < C->vm_free_top ? J.free_stack[at] : NONE;
                if (s_src == NONE) set_error(C, DERR_INTERNAL, 65);
            }
            __syncthreads();
            const uint32_t f = s_src;
            if (f != NONE) {
                vm_copy_page(J, f, q, page_size(J, r, n), perm);
                __syncthreads();
                if (tid == 0) {
                    J.pt[r] = f;
                    J.holder[f] = r;
                    J.holder[q] = NONE;
                    atomicAdd(&C->vm_copy_moves, 1u);
                }
            }
            __syncthreads();
        }
        if (!vm_barrier(C)) return;
        if (*(volatile uint32_t*)&C->error) return;
        // step 2: every target receives its own data
        for (uint32_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
            const uint32_t src = J.pt[q];
            if (src != q) {
                vm_copy_page(J, q, src, page_size(J, q, n), perm);
                __syncthreads();
                if (tid == 0) {
                    J.holder[src] = NONE;
                    J.pt[q] = q;
                    J.holder[q] = q;
                    atomicAdd(&C->vm_copy_moves, 1u);
                }
            }
            __syncthreads();
        }
        if (!vm_barrier(C)) return;
        q0 = q1;
    }
}

int vm_rounds_max_grid(int num_sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vm_rounds, VM_BLOCK, 0);
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
