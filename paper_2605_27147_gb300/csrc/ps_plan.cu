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
// exact for n < 2^32 because Power <= ceil(log2 n) <= 32.
//
// The merge tree.  Algorithm 1 merges the stack top while its power is >= the
// new power, so the merge made at boundary t joins all runs between the
// nearest boundary on the left with a smaller power and the nearest one on
// the right with a smaller power (the Cartesian tree of the powers; two equal
// powers always have a smaller one between them).  In midpoint terms: if the
// point found for boundary t is c / 2^p (c odd), that merge covers exactly the
// runs whose midpoints lie in [(c-1)/2^p, (c+1)/2^p).  k_nodes finds the first
// and last such run by galloping over the sorted kappa values; the total work
// is linear in the number of runs for balanced trees.
//
// The schedule.  A node (merge) whose range has at most T elements, and whose
// parent's range has more, is a tile: its whole subtree is merged in shared
// memory by one CTA.  Nodes above T are HBM nodes, merged in rounds of equal
// power (children have larger powers than their parent, and nodes of equal
// power are disjoint).  Each HBM node writes buffer depth & 1 (0 = the
// caller's array, 1 = scratch) and reads buffer (depth + 1) & 1, the
// Pingpong discipline of Sec. 3 arranged so that the root lands in the
// caller's array without a final copy.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

constexpr int NODE_HALO = 768;                          // k_nodes: staged slots on each side
constexpr int NODE_WIN = PLAN_BLOCK + 2 * NODE_HALO;

__device__ __forceinline__ uint32_t inst_of_slot(const Job& J, unsigned long long slot)
{
    return find_inst(J.count, slot, [&](uint32_t i) { return J.inst[i].run_base; });
}

// Warp-aggregated append to a list: returns the slot for this lane (or NONE).
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, bool want)
{
    const uint32_t mask = __ballot_sync(FULL, want);
    if (!mask) return NONE;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
    base = __shfl_sync(FULL, base, leader);
    return want ? base + __popc(mask & ((1u << lane) - 1u)) : NONE;
}

__device__ __forceinline__ uint32_t node_size(const uint32_t* rs, const uint32_t* na, const uint32_t* nb, uint32_t t)
{
    return rs[nb[t]] - rs[na[t]];
}

// Parent of boundary t: the nearer-in-tree of its two smaller neighbours,
// i.e. the one with the larger power (NONE for the root).
__device__ __forceinline__ uint32_t parent_of(const uint8_t* pw, const uint32_t* na, const uint32_t* nb,
                                              uint32_t t, uint32_t R)
{
    const uint32_t a = na[t], b = nb[t];
    const bool va = a >= 1, vb = b <= R - 1;
    if (va && vb) return pw[a] > pw[b] ? a : b;
    if (va) return a;
    if (vb) return b;
    return NONE;
}

// Parent boundary of leaf s: whichever of boundaries s and s+1 exists with the
// larger power (NONE when the instance is a single run).
__device__ __forceinline__ uint32_t leaf_parent(const uint8_t* pw, uint32_t s, uint32_t R)
{
    const bool vl = s >= 1, vr = s + 1 <= R - 1;
    if (vl && vr) return pw[s] > pw[s + 1] ? s : s + 1;
    if (vl) return s;
    if (vr) return s + 1;
    return NONE;
}

// Number of ancestors of boundary t: its left records (chain of nearest
// smaller boundaries to the left) plus its right records.
__device__ uint32_t depth_of(const uint32_t* na, const uint32_t* nb, uint32_t t, uint32_t R)
{
    uint32_t d = 0, u = t;
    while (na[u] >= 1) { u = na[u]; ++d; }
    u = t;
    while (nb[u] <= R - 1) { u = nb[u]; ++d; }
    return d;
}

}  // namespace

// kappa of every run: the run midpoint in 32-digit fixed point.
__global__ void __launch_bounds__(PLAN_BLOCK) k_kappa(Job J)
{
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const unsigned long long total = J.ctr->total_slots;
    for (unsigned long long slot = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; slot < total;
         slot += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t q = inst_of_slot(J, slot);
        const Inst& I = J.inst[q];
        const unsigned long long s = slot - I.run_base;
        if (s >= I.runs) continue;
        const uint32_t* rs = J.run_start + I.run_base;
        const unsigned long long twice_mid = (unsigned long long)rs[s] + rs[s + 1];
        J.kappa[slot] = (uint32_t)((twice_mid << 31) / I.n);
    }
}

// Power and node range [na, nb) (run indices) of every boundary; merge cost.
__global__ void __launch_bounds__(PLAN_BLOCK) k_nodes(Job J)
{
    // kappa of the block's slots and NODE_HALO slots on each side, staged in
    // shared memory: the probes of every node no wider than the halo stay on
    // chip, and only wide nodes (small powers, few of them) go to L2
    __shared__ uint32_t kw[NODE_WIN];
    __shared__ uint32_t s_err;
    if (threadIdx.x == 0) s_err = *(volatile uint32_t*)&J.ctr->error;
    __syncthreads();
    if (s_err) return;                                       // the whole block leaves together
    const unsigned long long total = J.ctr->total_slots;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long w0 = (long long)base - NODE_HALO;   // global slot of kw[0]
        __syncthreads();                                     // the previous pass's probes are done
        for (int i = threadIdx.x; i < NODE_WIN; i += PLAN_BLOCK) {
            const long long g = w0 + i;
            if (g >= 0 && g < (long long)total) kw[i] = J.kappa[g];
        }
        __syncthreads();
        const unsigned long long slot = base + threadIdx.x;
        unsigned long long cost = 0;
        uint32_t q = NONE, p = 0;
        if (slot < total) {
            q = inst_of_slot(J, slot);
            const Inst& I = J.inst[q];
            const unsigned long long t64 = slot - I.run_base;
            const uint32_t R = I.runs;
            if (t64 >= 1 && t64 + 1 <= R) {
                const uint32_t t = (uint32_t)t64;
                const uint32_t* kap_g = J.kappa + I.run_base;
                const long long off = (long long)I.run_base - w0;
                // kappa of run x of this instance (0 <= x < R: a staged slot
                // when it falls in the window, else a load)
                auto kap = [&](long long x) -> uint32_t {
                    const long long w = off + x;
                    return (w >= 0 && w < NODE_WIN) ? kw[w] : kap_g[x];
                };
                const uint32_t* rs = J.run_start + I.run_base;
                const uint32_t X = kap(t - 1), Y = kap(t);
                p = __clz(X ^ Y) + 1;                      // 1..32
                const uint32_t c = Y >> (32 - p);          // odd: the dyadic point is c / 2^p
                const unsigned long long XL = (unsigned long long)(c - 1) << (32 - p);
                const unsigned long long XR = (unsigned long long)(c + 1) << (32 - p);
                // first run with kappa >= XL (run t-1 qualifies): gallop left
                long long j = (long long)t - 1, bad = -1, step = 1;
                for (;;) {
                    const long long qq = j - step;
                    if (qq < 0) { bad = -1; break; }
                    if (kap(qq) < XL) { bad = qq; break; }
                    j = qq;
                    step <<= 1;
                }
                long long lo = bad + 1, hi = j;
                while (lo < hi) {
                    const long long mid = (lo + hi) >> 1;
                    if (kap(mid) >= XL) hi = mid; else lo = mid + 1;
                }
                const uint32_t a = (uint32_t)lo;
                // first run with kappa >= XR after t (run t does not qualify), or R
                j = t;
                long long good = R;
                step = 1;
                for (;;) {
                    const long long qq = j + step;
                    if (qq > (long long)R - 1) { good = R; break; }
                    if (kap(qq) >= XR) { good = qq; break; }
                    j = qq;
                    step <<= 1;
                }
                lo = j + 1;
                hi = good;
                while (lo < hi) {
                    const long long mid = (lo + hi) >> 1;
                    if (kap(mid) >= XR) hi = mid; else lo = mid + 1;
                }
                const uint32_t b = (uint32_t)lo;
                J.power[slot] = (uint8_t)p;
                J.na[slot] = a;
                J.nb[slot] = b;
                cost = (unsigned long long)(rs[b] - rs[a]);
            }
        }
        // merge cost and largest power, per instance (warp-aggregated when
        // the whole warp works on one instance)
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
                if (sum) atomicAdd(&J.inst[q0].M, sum);
                if (pm) atomicMax(&J.inst[q0].max_power, pm);
            }
        } else if (q != NONE) {
            if (cost) atomicAdd(&J.inst[q].M, cost);
            if (p) atomicMax(&J.inst[q].max_power, p);
        }
    }
}

// Tiles (subtrees of at most T elements whose parent is larger, and runs whose
// parent is larger) and HBM nodes (merges of more than T elements).
__global__ void __launch_bounds__(PLAN_BLOCK) k_classify(Job J)
{
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const unsigned long long total = J.ctr->total_slots;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const uint32_t T = J.tile_cap;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const unsigned long long slot = base + threadIdx.x;
        bool want_node_tile = false, want_leaf_tile = false, want_g = false;
        uint32_t q = 0, s = 0, r0 = 0, r1 = 0;
        if (slot < total) {
            q = inst_of_slot(J, slot);
            const Inst& I = J.inst[q];
            const unsigned long long s64 = slot - I.run_base;
            const uint32_t R = I.runs;
            if (s64 < R) {
                s = (uint32_t)s64;
                const uint32_t* rs = J.run_start + I.run_base;
                const uint8_t* pw = J.power + I.run_base;
                const uint32_t* na = J.na + I.run_base;
                const uint32_t* nb = J.nb + I.run_base;
                if (s >= 1) {                         // boundary s
                    const uint32_t size = node_size(rs, na, nb, s);
                    if (size > T) {
                        want_g = true;
                    } else {
                        const uint32_t par = parent_of(pw, na, nb, s, R);
                        if (par == NONE || node_size(rs, na, nb, par) > T) {
                            want_node_tile = true;
                            r0 = na[s];
                            r1 = nb[s];
                        }
                    }
                }
                const uint32_t lp = leaf_parent(pw, s, R);   // leaf s
                if (lp == NONE || node_size(rs, na, nb, lp) > T) want_leaf_tile = true;
            }
        }
        uint32_t at = warp_append(&J.ctr->n_tiles, want_node_tile);
        if (want_node_tile) {
            if (at < J.entry_cap) J.tiles[at] = TileItem{q, r0, r1, s, 0u, 0u};
            else set_error(J.ctr, DERR_INTERNAL, 20);
        }
        at = warp_append(&J.ctr->n_tiles, want_leaf_tile);
        if (want_leaf_tile) {
            if (at < J.entry_cap) J.tiles[at] = TileItem{q, s, s + 1, NONE, 0u, 0u};
            else set_error(J.ctr, DERR_INTERNAL, 21);
        }
        at = warp_append(&J.ctr->n_gnodes, want_g);
        if (want_g) {
            if (at < J.entry_cap) J.gnodes[at] = GNode{q, s, 0u, J.power[slot]};
            else set_error(J.ctr, DERR_INTERNAL, 22);
        }
    }
}

// Depth (number of ancestors) of every tile root and HBM node; HBM nodes are
// counted per round (round r holds power 32 - r, so larger powers go first).
__global__ void __launch_bounds__(PLAN_BLOCK) k_depth(Job J)
{
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const uint32_t nt = min(J.ctr->n_tiles, J.entry_cap);
    const uint32_t ng = min(J.ctr->n_gnodes, J.entry_cap);
    const uint32_t total = nt + ng;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        if (e < nt) {
            TileItem it = J.tiles[e];
            const Inst& I = J.inst[it.inst];
            const uint32_t R = I.runs;
            const uint32_t* na = J.na + I.run_base;
            const uint32_t* nb = J.nb + I.run_base;
            uint32_t d;
            if (it.t != NONE) {
                d = depth_of(na, nb, it.t, R);
            } else {
                const uint32_t lp = leaf_parent(J.power + I.run_base, it.r0, R);
                d = lp == NONE ? 0u : depth_of(na, nb, lp, R) + 1u;
            }
            J.tiles[e].depth = d;
        } else {
            const uint32_t g = e - nt;
            GNode gn = J.gnodes[g];
            const Inst& I = J.inst[gn.inst];
            const uint32_t* na = J.na + I.run_base;
            const uint32_t* nb = J.nb + I.run_base;
            J.gnodes[g].depth = depth_of(na, nb, gn.t, I.runs);
            const uint32_t size = node_size(J.run_start + I.run_base, na, nb, gn.t);
            atomicAdd(&J.ctr->bucket_count[32 - gn.power], 1u);
            atomicAdd(&J.ctr->bucket_nchunk[32 - gn.power], (size + J.merge_e - 1) / J.merge_e);
        }
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
    if (chunks > J.chunk_node_cap) set_error(C, DERR_INTERNAL, 31);
}

// Every HBM merge takes the next place of its round with one 64-bit atomic
// that advances the round's merge count and chunk count together, so within
// a round the chunk bases grow with the merge order (the chunk -> merge
// table below relies on it).
__global__ void __launch_bounds__(PLAN_BLOCK) k_bucket(Job J)
{
    Ctr* C = J.ctr;
    if (*(volatile uint32_t*)&C->error) return;
    const uint32_t ng = min(C->n_gnodes, J.entry_cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x; base < ng; base += stride) {
        const uint32_t e = base + threadIdx.x;
        unsigned long long size = 0;
        if (e < ng) {
            const GNode gn = J.gnodes[e];
            const Inst& I = J.inst[gn.inst];
            const uint32_t* rs = J.run_start + I.run_base;
            const uint32_t lo = rs[J.na[I.run_base + gn.t]];
            const uint32_t mid = rs[gn.t];
            const uint32_t hi = rs[J.nb[I.run_base + gn.t]];
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
                J.gidx[I.run_base + gn.t] = at;
            } else {
                set_error(C, DERR_INTERNAL, 32);
            }
            size = hi - lo;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) size += __shfl_xor_sync(FULL, size, o);
        if ((threadIdx.x & 31) == 0 && size) atomicAdd(&C->hbm_elems, size);
    }
}

// Chunk -> merge table for every round (chunk ids are global across rounds):
// each thread covers 32 consecutive chunks with one binary search and a walk.
// Then every HBM merge is linked to its parent merge (which is larger, hence
// an HBM merge too) and adds its chunk count to the parent's dependencies.
__global__ void __launch_bounds__(PLAN_BLOCK) k_chunk_nodes(Job J)
{
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const Ctr* C = J.ctr;
    const uint32_t ng = min(C->n_gnodes, J.entry_cap);
    const uint32_t total = C->bucket_chunk[NPOW];
    if (ng == 0 || total > J.chunk_node_cap) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        const GNode gn = J.gnodes[i];
        const Inst& I = J.inst[gn.inst];
        const uint32_t me = J.gidx[I.run_base + gn.t];
        const uint32_t p = parent_of(J.power + I.run_base, J.na + I.run_base, J.nb + I.run_base, gn.t, I.runs);
        if (p == NONE) continue;                 // the instance's root
        const uint32_t par = J.gidx[I.run_base + p];
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

cudaError_t launch_plan(const Job& J, int grid, cudaStream_t s)
{
    k_kappa<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_nodes<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_classify<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_depth<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_bucket_scan<<<1, 32, 0, s>>>(J);
    k_bucket<<<grid, PLAN_BLOCK, 0, s>>>(J);
    k_chunk_nodes<<<grid, PLAN_BLOCK, 0, s>>>(J);
    return cudaGetLastError();
}

}  // namespace ps
