// Powers, the merge tree and the merge schedule.
//
// Power (Sec. 2 Theorem).  For adjacent runs a = [i, j), b = [j, k) the power
// is the smallest p such that a multiple of 2^-p lies in (l, r] with
// l = (i+j)/(2n), r = (j+k)/(2n), the two runs' midpoints scaled to [0, 1).
// A multiple of 2^-p lies in (l, r] exactly when floor(r 2^p) > floor(l 2^p),
// i.e. when the first p binary digits of l and r differ.  With the 32-digit
// fixed-point midpoints  kappa(run) = floor((start + end) 2^31 / n)  (exact
// integer division), floor(x 2^p) = kappa >> (32 - p) for every p <= 32, so
//     Power = 1 + (number of leading binary digits kappa_left and kappa_right
//                  share) = clz(kappa_left ^ kappa_right) + 1,
// exact for n < 2^32 because Power <= ceil(log2 n) <= 32.  kappa is computed
// from the run starts where it is needed; comparisons kappa >= X are made as
// (start + end) 2^31 >= X n, without a division.
//
// The merge tree.  Algorithm 1 merges the stack top while its power is >= the
// new power, so the merge made at boundary t joins all runs between the
// nearest boundary on the left with a smaller power and the nearest one on
// the right with a smaller power (the Cartesian tree of the powers; two equal
// powers always have a smaller one between them).  In midpoint terms: if the
// point found for boundary t is c / 2^p (c odd), that merge covers exactly the
// runs whose midpoints lie in [(c-1)/2^p, (c+1)/2^p).  node_range finds the
// first and last such run by galloping over the runs' midpoints; the total
// work is linear in the number of runs for balanced trees.
//
// Sizes.  The midpoints of a merge's first and last run are less than 2n/2^p
// apart, and the merge's size is at most twice that distance, so a merge of
// Power p has fewer than 4n/2^p elements.  A merge of more than T elements
// (an HBM merge) therefore has 2^p < 4n/T: an instance has fewer than 4n/T
// HBM merges, and (p, c) indexes them densely (merge_index).
//
// The schedule.  A node (merge) whose range has at most T elements, and whose
// parent's range has more, is a tile: its whole subtree is merged in shared
// memory by one CTA.  Every tile is a child of an HBM merge (or the whole
// instance), so k_nodes lists the tiles with the HBM merges: the left part
// [a, t) and the right part [t, b) of an HBM merge at boundary t are its two
// children.  HBM merges are done in rounds of equal power (children have
// larger powers than their parent, and merges of equal power are disjoint).
// Each writes buffer depth & 1 (0 = the caller's array, 1 = scratch) and
// reads buffer (depth + 1) & 1, the Pingpong discipline of Sec. 3 arranged so
// that the root lands in the caller's array without a final copy.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

constexpr int NODE_HALO = 768;                          // k_nodes: staged run starts on each side
constexpr int NODE_WIN = PLAN_BLOCK + 2 * NODE_HALO + 2;
// k_nodes buffers the HBM merges and tiles it finds in shared memory and
// appends them to the global lists in bulk: a pass adds at most PLAN_BLOCK
// merges and 2 PLAN_BLOCK tiles, so the buffers are flushed whenever another
// pass could overflow them (for unsorted data about once per block)
constexpr int NODE_BUF_G = PLAN_BLOCK + 64;
constexpr int NODE_BUF_T = 2 * PLAN_BLOCK + 128;

__device__ __forceinline__ uint32_t inst_of_slot(const Job& J, unsigned long long slot)
{
    return find_inst(J.count, slot, [&](uint32_t i) { return J.inst[i].run_base; });
}

// The fixed-point midpoint of the run [s, e) of an instance of n elements:
// floor(x / n) for x = (s + e) 2^31 < 2^64, without a division.  With
// recip = floor((2^64 - 1) / n) > (2^64 - 1) / n - 1, the high half of
// x * recip is at most x / n and more than x / n - 2, so the quotient is it
// or one of the next two integers, found by comparing the remainder with n.
__device__ __forceinline__ uint32_t kappa_of(uint32_t s, uint32_t e, uint32_t n, unsigned long long recip)
{
    const unsigned long long x = ((unsigned long long)s + e) << 31;
    unsigned long long q = __umul64hi(x, recip);
    unsigned long long r = x - q * n;
    if (r >= n) { ++q; r -= n; }
    if (r >= n) ++q;
    return (uint32_t)q;
}

// kappa_of(s, e, n) >= X for an integer X <= 2^32, without the division.
__device__ __forceinline__ bool kappa_ge(uint32_t s, uint32_t e, uint32_t n, unsigned long long X)
{
    return (((unsigned long long)s + e) << 31) >= X * n;
}

struct NodeRange {
    uint32_t a, b;   // the merge joins runs [a, t) and [t, b)
    uint32_t p, c;   // its Power and dyadic point c / 2^p (c odd)
};

// Power of boundary t (1 <= t < R) and its point.  rs(x) = start of run x
// (x <= R, rs(R) = n).
template <typename RS>
__device__ __forceinline__ void power_of(RS rs, uint32_t n, unsigned long long recip, uint32_t t, uint32_t& p,
                                         uint32_t& c)
{
    const uint32_t X = kappa_of(rs(t - 1), rs(t), n, recip), Y = kappa_of(rs(t), rs(t + 1), n, recip);
    p = __clz(X ^ Y) + 1;                 // 1..32
    c = Y >> (32 - p);                    // odd
}

// The merge Algorithm 1 makes at boundary t: the runs whose midpoints lie in
// [(c-1)/2^p, (c+1)/2^p), found by galloping out from t.
template <typename RS>
__device__ NodeRange node_range(RS rs, uint32_t R, uint32_t n, unsigned long long recip, uint32_t t)
{
    NodeRange r;
    power_of(rs, n, recip, t, r.p, r.c);
    const unsigned long long XL = (unsigned long long)(r.c - 1) << (32 - r.p);
    const unsigned long long XR = (unsigned long long)(r.c + 1) << (32 - r.p);
    auto ge = [&](long long x, unsigned long long X) { return kappa_ge(rs(x), rs(x + 1), n, X); };
    // first run with midpoint >= XL (run t-1 qualifies): gallop left
    long long j = (long long)t - 1, bad = -1, step = 1;
    for (;;) {
        const long long q = j - step;
        if (q < 0) { bad = -1; break; }
        if (!ge(q, XL)) { bad = q; break; }
        j = q;
        step <<= 1;
    }
    long long lo = bad + 1, hi = j;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (ge(mid, XL)) hi = mid; else lo = mid + 1;
    }
    r.a = (uint32_t)lo;
    // first run after t with midpoint >= XR (run t does not qualify), or R
    j = t;
    long long good = R;
    step = 1;
    for (;;) {
        const long long q = j + step;
        if (q > (long long)R - 1) { good = R; break; }
        if (ge(q, XR)) { good = q; break; }
        j = q;
        step <<= 1;
    }
    lo = j + 1;
    hi = good;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (ge(mid, XR)) hi = mid; else lo = mid + 1;
    }
    r.b = (uint32_t)lo;
    return r;
}

}  // namespace

// Power of every boundary, the merge cost, and the schedule's lists: every
// HBM merge (more than T elements) with its parent's merge-map index, and
// every tile (a child of an HBM merge that has at most T elements or is a
// single run, or the whole instance when it has at most T elements or is a
// single run).
__global__ void __launch_bounds__(PLAN_BLOCK) k_nodes(Job J)
{
    // run starts of the block's slots and NODE_HALO slots on each side,
    // staged in shared memory: the probes of every node no wider than the
    // halo stay on chip, and only wide nodes (small powers, few of them) go
    // to L2
    __shared__ uint32_t rw[NODE_WIN];
    __shared__ uint32_t s_err;
    // buffered HBM merges (inst, t, a, b, power, midx, pidx) and tiles (inst,
    // r0, r1, buffered index of the parent merge or NONE), their counts and
    // the global places of a flush
    __shared__ uint32_t sg[NODE_BUF_G][7];
    __shared__ uint32_t st[NODE_BUF_T][4];
    __shared__ uint32_t s_ng, s_nt, s_bg, s_bt;
    if (threadIdx.x == 0) {
        s_err = *(volatile uint32_t*)&J.ctr->error;
        s_ng = 0;
        s_nt = 0;
    }
    __syncthreads();
    if (s_err) return;                                       // the whole block leaves together
    // the buffered items to the global lists: one atomic per list
    auto flush_items = [&]() {
        if (threadIdx.x == 0) {
            s_bg = s_ng ? atomicAdd(&J.ctr->n_gnodes, s_ng) : 0u;
            s_bt = s_nt ? atomicAdd(&J.ctr->n_tiles, s_nt) : 0u;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < s_ng; i += PLAN_BLOCK) {
            const uint32_t g = s_bg + i;
            const uint32_t* b = sg[i];
            if (g < J.gnode_cap) {
                J.gnodes[g] = GNode{b[0], b[1], b[2], b[3], b[4], 0u, b[5], b[6]};
                J.gmap[J.inst[b[0]].g_base + b[5]] = g;
            } else {
                set_error(J.ctr, DERR_INTERNAL, 22);
            }
        }
        for (uint32_t j = threadIdx.x; j < s_nt; j += PLAN_BLOCK) {
            const uint32_t at = s_bt + j;
            const uint32_t* b = st[j];
            if (at < J.tile_cap_items) J.tiles[at] = TileItem{b[0], b[1], b[2], b[3] == NONE ? NONE : s_bg + b[3], 0u, 0u};
            else set_error(J.ctr, DERR_INTERNAL, 20);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_ng = 0;
            s_nt = 0;
        }
        __syncthreads();
    };
    const unsigned long long total = J.ctr->total_slots;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const uint32_t T = J.tile_cap;
    // lane 0: the instance whose merge cost and largest power this warp accumulates
    uint32_t acc_q = NONE, acc_p = 0;
    unsigned long long acc_m = 0;
    auto flush = [&]() {
        if (acc_q != NONE) {
            if (acc_m) atomicAdd(&J.inst[acc_q].M, acc_m);
            if (acc_p) atomicMax(&J.inst[acc_q].max_power, acc_p);
        }
        acc_q = NONE;
        acc_m = 0;
        acc_p = 0;
    };
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long w0 = (long long)base - NODE_HALO;   // global slot of rw[0]
        __syncthreads();                                     // the previous pass's probes are done
        for (int i = threadIdx.x; i < NODE_WIN; i += PLAN_BLOCK) {
            const long long g = w0 + i;
            if (g >= 0 && g < (long long)total) rw[i] = J.run_start[g];
        }
        __syncthreads();
        const unsigned long long slot = base + threadIdx.x;
        unsigned long long cost = 0;
        uint32_t q = NONE, p = 0;
        bool want_g = false, want_l = false, want_r = false, want_root = false;
        GNode gn = {};
        if (slot < total) {
            q = inst_of_slot(J, slot);
            const Inst& I = J.inst[q];
            const unsigned long long t64 = slot - I.run_base;
            const uint32_t R = I.runs, n = I.n;
            const uint32_t* rs_g = J.run_start + I.run_base;
            const long long off = (long long)I.run_base - w0;
            // start of run x of this instance (0 <= x <= R: a staged slot when
            // it falls in the window, else a load)
            auto rs = [&](long long x) -> uint32_t {
                const long long w = off + x;
                return (w >= 0 && w < NODE_WIN) ? rw[w] : rs_g[x];
            };
            if (t64 >= 1 && t64 + 1 <= R) {
                const uint32_t t = (uint32_t)t64;
                const NodeRange nr = node_range(rs, R, n, I.recip, t);
                p = nr.p;
                J.power[slot] = (uint8_t)p;
                const uint32_t lo = rs(nr.a), mid = rs(t), hi = rs(nr.b);
                cost = (unsigned long long)(hi - lo);
                if (hi - lo > T) {
                    // an HBM merge; its parent is the one of the two boundaries
                    // around it with the larger power (both have smaller powers)
                    want_g = true;
                    // a child is a tile when it has at most T elements or is a
                    // single run (a leaf, whatever its length); otherwise it is
                    // an HBM merge, listed by its own boundary
                    want_l = mid - lo <= T || t - nr.a == 1;
                    want_r = hi - mid <= T || nr.b - t == 1;
                    uint32_t pa = 0, pb = 0, ca = 0, cb = 0;
                    if (nr.a >= 1) power_of(rs, n, I.recip, nr.a, pa, ca);
                    if (nr.b + 1 <= R) power_of(rs, n, I.recip, nr.b, pb, cb);
                    uint32_t pidx = NONE;
                    if (pa || pb) pidx = pa > pb ? merge_index(pa, ca) : merge_index(pb, cb);
                    const uint32_t midx = merge_index(p, nr.c);
                    if (midx >= I.g_span || (pidx != NONE && pidx >= I.g_span)) {
                        set_error(J.ctr, DERR_INTERNAL, 23);   // a merge larger than its power allows
                        want_g = want_l = want_r = false;
                    }
                    gn = GNode{q, t, nr.a, nr.b, p, 0u, midx, pidx};
                }
            } else if (t64 == 0 && R >= 1 && (R == 1 || n <= T)) {
                want_root = true;                      // the whole instance is one tile
            }
        }
        // this pass's items into the block's buffers (they have room: see
        // the flush below)
        uint32_t lg = NONE;
        if (want_g) {
            lg = atomicAdd(&s_ng, 1u);
            uint32_t* b = sg[lg];
            b[0] = q; b[1] = gn.t; b[2] = gn.a; b[3] = gn.b; b[4] = gn.power; b[5] = gn.midx; b[6] = gn.pidx;
        }
        if (want_l) {
            uint32_t* b = st[atomicAdd(&s_nt, 1u)];
            b[0] = q; b[1] = gn.a; b[2] = gn.t; b[3] = lg;
        }
        if (want_r) {
            uint32_t* b = st[atomicAdd(&s_nt, 1u)];
            b[0] = q; b[1] = gn.t; b[2] = gn.b; b[3] = lg;
        }
        if (want_root) {
            uint32_t* b = st[atomicAdd(&s_nt, 1u)];
            b[0] = q; b[1] = 0u; b[2] = J.inst[q].runs; b[3] = NONE;
        }
        __syncthreads();
        if (s_ng > (uint32_t)(NODE_BUF_G - PLAN_BLOCK) || s_nt > (uint32_t)(NODE_BUF_T - 2 * PLAN_BLOCK)) flush_items();
        // merge cost and largest power, per instance: summed over the warp
        // when the whole warp works on one instance, and over the warp's
        // passes while the instance stays the same (one atomic per warp and
        // instance: every warp updating the same instance at every pass
        // queued on one cache line)
        const uint32_t q0 = __shfl_sync(FULL, q, 0);
        if (__all_sync(FULL, q == q0) && q0 != NONE) {
            unsigned long long sum = cost;
            uint32_t pm = p;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sum += __shfl_xor_sync(FULL, sum, o);
                pm = max(pm, __shfl_xor_sync(FULL, pm, o));
            }
            if ((threadIdx.x & 31) == 0) {
                if (acc_q != q0) {
                    flush();
                    acc_q = q0;
                }
                acc_m += sum;
                acc_p = max(acc_p, pm);
            }
        } else if (q != NONE) {
            if (cost) atomicAdd(&J.inst[q].M, cost);
            if (p) atomicMax(&J.inst[q].max_power, p);
        }
    }
    if ((threadIdx.x & 31) == 0) flush();
    __syncthreads();
    if (s_ng || s_nt) flush_items();
}

// Depth (number of ancestors) of every HBM merge, by walking the parent
// links through the merge map (an HBM merge's parent is an HBM merge);
// merges are counted per round (round r holds power 32 - r, so larger powers
// go first).
__global__ void __launch_bounds__(PLAN_BLOCK) k_depth(Job J)
{
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const uint32_t ng = min(J.ctr->n_gnodes, J.gnode_cap);
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const GNode gn = J.gnodes[g];
        const Inst& I = J.inst[gn.inst];
        const uint32_t* gm = J.gmap + I.g_base;
        uint32_t d = 0, up = gn.pidx;
        while (up != NONE) {
            const uint32_t h = gm[up];
            if (h >= ng || d > NPOW) {
                set_error(J.ctr, DERR_INTERNAL, 25);
                break;
            }
            ++d;
            up = J.gnodes[h].pidx;
        }
        J.gnodes[g].depth = d;
        const uint32_t* rs = J.run_start + I.run_base;
        const uint32_t size = rs[gn.b] - rs[gn.a];
        atomicAdd(&J.ctr->bucket_count[32 - gn.power], 1u);
        atomicAdd(&J.ctr->bucket_nchunk[32 - gn.power], (size + J.merge_e - 1) / J.merge_e);
    }
}

// One small CTA: where each round starts among the HBM merges and among the
// chunks (prefix sums of the per-round counts), and the table limits.
__global__ void __launch_bounds__(32) k_bucket_scan(Job J)
{
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    if (threadIdx.x != 0) return;
    uint32_t acc = 0, chunks = 0, rounds = 0;
    for (int r = 0; r < NPOW; ++r) {
        C->bucket_start[r] = acc;
        C->bucket_chunk[r] = chunks;
        acc += C->bucket_count[r];
        chunks += C->bucket_nchunk[r];
        rounds += C->bucket_count[r] ? 1u : 0u;
    }
    C->bucket_start[NPOW] = acc;
    C->bucket_chunk[NPOW] = chunks;
    C->rounds = rounds;
    if (!J.vm && chunks > J.chunk_node_cap) set_error(C, DERR_INTERNAL, 31);
}

// Every HBM merge takes the next place of its round with one 64-bit atomic
// that advances the round's merge count and chunk count together, so within
// a round the chunk bases grow with the merge order (the chunk -> merge
// table below relies on it); its merge-map entry becomes its GSorted index.
// Every tile takes the depth below its parent merge.
__global__ void __launch_bounds__(PLAN_BLOCK) k_bucket(Job J)
{
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    const uint32_t ng = min(C->n_gnodes, J.gnode_cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x; base < ng; base += stride) {
        const uint32_t e = base + threadIdx.x;
        unsigned long long size = 0;
        if (e < ng) {
            const GNode gn = J.gnodes[e];
            const Inst& I = J.inst[gn.inst];
            const uint32_t* rs = J.run_start + I.run_base;
            const uint32_t lo = rs[gn.a], mid = rs[gn.t], hi = rs[gn.b];
            const uint32_t r = 32 - gn.power;
            const uint32_t nch = (hi - lo + J.merge_e - 1) / J.merge_e;
            const unsigned long long old = atomicAdd(&C->bucket_cursor[r], (1ull << 40) | nch);
            const uint32_t at = C->bucket_start[r] + (uint32_t)(old >> 40);
            GSorted o;
            o.goff = I.off + lo;
            o.la = mid - lo;
            o.lb = hi - mid;
            o.chunk_base = C->bucket_chunk[r] + (uint32_t)(old & ((1ull << 40) - 1));
            o.depth = gn.depth;
            o.parent = NONE;                  // linked by k_chunk_nodes
            o.pad = 0;
            if (at < C->bucket_start[r + 1]) {
                J.gsorted[at] = o;
                J.dep[at] = 0;
                J.gmap[I.g_base + gn.midx] = at;
            } else {
                set_error(C, DERR_INTERNAL, 32);
            }
            size = hi - lo;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) size += __shfl_xor_sync(FULL, size, o);
        if ((threadIdx.x & 31) == 0 && size) atomicAdd(&C->hbm_elems, size);
    }
    const uint32_t nt = min(C->n_tiles, J.tile_cap_items);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nt; e += stride) {
        const uint32_t par = J.tiles[e].parent;
        J.tiles[e].depth = par == NONE ? 0u : (par < ng ? J.gnodes[par].depth + 1u : 0u);
    }
}

// Chunk -> merge table for every round (chunk ids are global across rounds):
// each thread covers 32 consecutive chunks with one binary search and a walk.
// Then every HBM merge is linked to its parent merge and adds its chunk
// count to the parent's dependencies.  (VM storage runs its rounds with grid
// barriers and needs neither.)
__global__ void __launch_bounds__(PLAN_BLOCK) k_chunk_nodes(Job J)
{
    if (J.vm || *(volatile uint32_t*)&J.ctr->error) return;
    const Ctr* C = J.ctr;
    const uint32_t ng = min(C->n_gnodes, J.gnode_cap);
    const uint32_t total = C->bucket_chunk[NPOW];
    if (ng == 0 || total > J.chunk_node_cap) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        const GNode gn = J.gnodes[i];
        if (gn.pidx == NONE) continue;           // the instance's root
        const uint32_t* gm = J.gmap + J.inst[gn.inst].g_base;
        const uint32_t me = gm[gn.midx], par = gm[gn.pidx];
        if (me >= ng || par >= ng) {
            set_error(J.ctr, DERR_INTERNAL, 33);
            continue;
        }
        J.gsorted[me].parent = par;
        const GSorted g = J.gsorted[me];
        atomicAdd(&J.dep[par], (g.la + g.lb + J.merge_e - 1) / J.merge_e);
    }
    const uint32_t groups = (total + 31) / 32;
    for (uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < groups; gi += gridDim.x * blockDim.x) {
        const uint32_t c0 = gi * 32, c1 = min(c0 + 32, total);
        uint32_t lo = 0, hi = ng;     // last node with chunk_base <= c0
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (J.gsorted[mid].chunk_base <= c0) lo = mid; else hi = mid;
        }
        uint32_t e = lo;
        uint32_t next = e + 1 < ng ? J.gsorted[e + 1].chunk_base : 0xffffffffu;
        for (uint32_t c = c0; c < c1; ++c) {
            while (c >= next) {
                ++e;
                next = e + 1 < ng ? J.gsorted[e + 1].chunk_base : 0xffffffffu;
            }
            J.chunk_node[c] = e;
        }
    }
}

// Introspection: the element range [lo, hi) of the merge at every boundary of
// instance q (the same node_range as k_nodes), two words per boundary.
__global__ void __launch_bounds__(PLAN_BLOCK) k_node_ranges(Job J, uint32_t q, uint32_t* out)
{
    const Inst& I = J.inst[q];
    const uint32_t R = I.runs, n = I.n;
    const uint32_t* rs_g = J.run_start + I.run_base;
    auto rs = [&](long long x) -> uint32_t { return rs_g[x]; };
    for (uint32_t t = 1 + blockIdx.x * blockDim.x + threadIdx.x; t < R; t += gridDim.x * blockDim.x) {
        const NodeRange nr = node_range(rs, R, n, I.recip, t);
        out[2 * (t - 1)] = rs_g[nr.a];
        out[2 * (t - 1) + 1] = rs_g[nr.b];
    }
}

// One CTA: call totals (elements, runs, merge cost, largest power).
__global__ void __launch_bounds__(1024) k_finish(Job J)
{
    __shared__ unsigned long long sn, sr, sm;
    __shared__ uint32_t sp;
    if (threadIdx.x == 0) { sn = 0; sr = 0; sm = 0; sp = 0; }
    __syncthreads();
    unsigned long long n = 0, r = 0, m = 0;
    uint32_t p = 0;
    for (uint32_t i = threadIdx.x; i < J.count; i += blockDim.x) {
        const Inst& I = J.inst[i];
        n += I.n;
        r += I.runs;
        m += I.M;
        p = max(p, I.max_power);
    }
    atomicAdd(&sn, n);
    atomicAdd(&sr, r);
    atomicAdd(&sm, m);
    atomicMax(&sp, p);
    __syncthreads();
    if (threadIdx.x == 0) {
        J.ctr->n_total = sn;
        J.ctr->runs_total = sr;
        J.ctr->M_total = sm;
        J.ctr->max_power = sp;
    }
}

cudaError_t launch_finish(const Job& J, cudaStream_t s)
{
    k_finish<<<1, 1024, 0, s>>>(J);
    return cudaGetLastError();
}

int nodes_max_grid(int num_sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nodes, PLAN_BLOCK, 0);
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_plan(const Job& J, int grid, int nodes_grid, cudaStream_t s)
{
    // k_nodes: every CTA resident at once (its passes are equal shares), and
    // an odd number of them: the grid stride is then an odd multiple of
    // PLAN_BLOCK slots, so the boundaries at multiples of 2^k (the wide
    // merges of a balanced tree, whose searches leave the staged window) fall
    // to every CTA in turn instead of to the same CTAs in every pass
    const int ng = nodes_grid > 1 && (nodes_grid & 1) == 0 ? nodes_grid - 1 : nodes_grid;
    k_nodes<<<ng, PLAN_BLOCK, 0, s>>>(J);
    k_depth<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_bucket_scan<<<1, 32, 0, s>>>(J);
    k_bucket<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_chunk_nodes<<<grid, PLAN_BLOCK, 0, s>>>(J);
    return cudaGetLastError();
}

cudaError_t launch_node_ranges(const Job& J, uint32_t q, uint32_t nbound, uint32_t* out, cudaStream_t s)
{
    const int grid = (int)((nbound + PLAN_BLOCK - 1) / PLAN_BLOCK);
    if (grid > 0) k_node_ranges<<<grid < 4096 ? grid : 4096, PLAN_BLOCK, 0, s>>>(J, q, out);
    return cudaGetLastError();
}

}  // namespace ps
