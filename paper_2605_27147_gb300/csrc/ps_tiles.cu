// On-chip merging of small subtrees of the merge tree ("tiles").
//
// A tile is a node of Algorithm 1's merge tree whose range holds at most T
// elements while its parent's range holds more, or a single run whose parent
// is larger than T.  One CTA loads the tile's keys into shared memory, sorts
// every forced run (the minrun insertion sort of Sec. 5; any stable sort of
// the run gives the same result) and then performs the tile's merges bottom
// up, one power level at a time: at level p every boundary of power p joins
// the two segments around it (the segments being delimited by the boundaries
// of smaller power), exactly the merges Algorithm 1 performs inside this
// subtree, in an order that respects the tree.  Each merge is the stable merge
// of Algorithm 2 (ties take the left segment); every element carries its
// input position inside the tile (16 bits), from which the permutation is
// written at the end.
//
// The finished tile goes to buffer depth & 1 (0 = caller's arrays, 1 = the
// scratch arrays) with its stable permutation, ready for the HBM rounds.
// A single run longer than T (always a natural run) is streamed: keys copied
// when its buffer is the scratch one, perm written.
//
// With decreasing runs on (Job::desc_runs), a natural run -- longer than
// minrun, or a single streamed run -- whose first pair descends is strictly
// decreasing and is reversed here, keys and positions together (its elements
// are distinct, so the reversal is the stable order).  Runs of at most 64
// elements need nothing extra: the forced-run sort orders them anyway.
//
// Whatever order its merges run in, a subtree's result is the stable sort of
// its range: the elements ordered by (key, input position).  A tile made of
// many short runs (the usual case for unsorted data: forced runs of minrun
// elements) therefore takes a faster road to the same result: each element
// becomes one 64-bit word (key << 32 | position), every thread sorts 16
// consecutive words in registers with a sorting network, and the sorted
// blocks are merged pairwise in shared memory (merge path, 16 outputs per
// thread, comparing keys with ties to the left block) up to the whole
// tile.  The words are distinct, so no tie rule is
// needed and the order is exactly the stable one.  Tiles of few runs follow
// the tree level by level as described above.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int TILE_MAX = 1 << TILE_MAX_LOG2;
constexpr int TILE_RUNS = TILE_MAX / 32 + 2;   // runs of a tile (minrun >= 32 when n >= 64)
constexpr int TILE_K = 17;                     // outputs per thread per level (odd: conflict-free strides)
static_assert(TILE_K * TILE_BLOCK >= TILE_MAX, "a level must cover a whole tile");

struct TileSmem {
    uint32_t key[2][TILE_MAX];
    uint16_t idx[2][TILE_MAX];   // input position inside the tile (the permutation)
};

constexpr int NET_PER = 16;                          // words per thread in the network road
constexpr int NET_SLOTS = TILE_MAX + TILE_MAX / NET_PER;   // one spare slot per 16: fewer bank conflicts
constexpr uint32_t NET_MIN_RUNS = 8;                 // tiles with this many runs take the network road
static_assert(NET_PER * TILE_BLOCK >= TILE_MAX, "one block of 16 words per thread covers a tile");

struct NetSmem {
    unsigned long long w[2][NET_SLOTS];
};

__device__ __forceinline__ uint32_t net_slot(uint32_t x)
{
    return x + (x >> 4);
}

// Batcher's odd-even merge sorting network over N words held in registers
// (ascending): 63 comparators for N = 16, where the bitonic network takes 80.
// Merges sorted runs of p words pairwise, for p = 1, 2, 4, ...; comparator
// (a, a + k) acts only within one run of 2p words.
template <int N>
__device__ __forceinline__ void sort_registers(unsigned long long (&v)[N])
{
#pragma unroll
    for (int p = 1; p < N; p <<= 1) {
#pragma unroll
        for (int k = p; k >= 1; k >>= 1) {
#pragma unroll
            for (int j = k % p; j + k < N; j += 2 * k) {
#pragma unroll
                for (int i = 0; i < k && i + j + k < N; ++i) {
                    const int a = i + j, b = a + k;
                    if (a / (2 * p) == b / (2 * p)) {
                        const unsigned long long x = v[a], y = v[b];
                        const bool swap = y < x;
                        v[a] = swap ? y : x;
                        v[b] = swap ? x : y;
                    }
                }
            }
        }
    }
}

// Key of the word at slot s of a word array: its high half.
__device__ __forceinline__ uint32_t net_key(const unsigned long long* w, uint32_t s)
{
    return reinterpret_cast<const uint32_t*>(w)[2 * s + 1];
}

// The network road for one tile of `size` elements: sorted (key, position)
// words end in sm.w[result]; returns result.  The tile is padded to N, a
// multiple of 16 words (padding sorts last); the merge levels pair blocks of
// w words up to the largest power of two below N, the last pair of a level
// possibly partial or without a partner, so a tile costs its own size, not
// the next power of two.
__device__ int tile_network(NetSmem& sm, const uint32_t* ksrc, uint32_t size)
{
    const int tid = threadIdx.x;
    const uint32_t N = (size + NET_PER - 1) & ~(uint32_t)(NET_PER - 1);
    for (uint32_t x = tid; x < N; x += TILE_BLOCK)
        sm.w[0][net_slot(x)] = x < size ? ((unsigned long long)__ldg(ksrc + x) << 32) | x : ~0ull;
    __syncthreads();
    const uint32_t x0 = (uint32_t)tid * NET_PER;
    if (x0 < N) {
        unsigned long long v[NET_PER];
#pragma unroll
        for (int j = 0; j < NET_PER; ++j) v[j] = sm.w[0][net_slot(x0) + j];
        sort_registers<NET_PER>(v);
#pragma unroll
        for (int j = 0; j < NET_PER; ++j) sm.w[0][net_slot(x0) + j] = v[j];
    }
    __syncthreads();
    int cur = 0;
    for (uint32_t w = NET_PER; w < N; w <<= 1) {
        const unsigned long long* src = sm.w[cur];
        unsigned long long* dst = sm.w[cur ^ 1];
        if (x0 < N) {
            const uint32_t blk = x0 & ~(2 * w - 1), d = x0 - blk;
            const uint32_t A = blk, B = blk + w;
            const uint32_t la = min(w, N - A), lb = B < N ? min(w, N - B) : 0u;
            // keys only: the blocks are stably sorted and A's positions come
            // before B's, so ties to A keep the (key, position) order (a block
            // holding padding is followed only by padding); a block without a
            // partner (lb = 0) is copied
            uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (net_key(src, net_slot(A + mid)) <= net_key(src, net_slot(B + d - 1 - mid))) lo = mid + 1;
                else hi = mid;
            }
            uint32_t ia = lo, ib = d - lo;
            unsigned long long va = ia < la ? src[net_slot(A + ia)] : 0ull;
            unsigned long long vb = ib < lb ? src[net_slot(B + ib)] : 0ull;
            unsigned long long* out = dst + net_slot(x0);
            // branch-free serial merge; an exhausted side is read at the
            // first slot of A (a valid address whose value is never used)
#pragma unroll
            for (int j = 0; j < NET_PER; ++j) {
                const bool take_a = ia < la && (ib >= lb || (uint32_t)(va >> 32) <= (uint32_t)(vb >> 32));
                out[j] = take_a ? va : vb;
                ia += take_a;
                ib += !take_a;
                const unsigned long long nxt = src[net_slot(take_a ? A + (ia < la ? ia : 0u) : (ib < lb ? B + ib : A))];
                va = take_a ? nxt : va;
                vb = take_a ? vb : nxt;
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    return cur;
}

}  // namespace

__global__ void __launch_bounds__(TILE_BLOCK) k_tiles(Job J)
{
    extern __shared__ __align__(16) unsigned char tile_raw[];
    TileSmem& sm = *reinterpret_cast<TileSmem*>(tile_raw);
    NetSmem& net = *reinterpret_cast<NetSmem*>(tile_raw);
    __shared__ uint32_t rs_s[TILE_RUNS + 1];
    __shared__ uint8_t pw_s[TILE_RUNS + 1];
    __shared__ uint32_t seg_lo[TILE_RUNS + 2];
    __shared__ uint32_t seg_mid[TILE_RUNS + 2];
    __shared__ uint32_t warp_cnt[TILE_BLOCK / 32];
    __shared__ uint32_t s_mask, s_nseg;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const uint32_t ntiles = min(J.ctr->n_tiles, J.tile_cap_items);

    for (uint32_t e = blockIdx.x; e < ntiles; e += gridDim.x) {
        const TileItem it = J.tiles[e];
        const Inst I = J.inst[it.inst];
        const uint32_t* rs = J.run_start + I.run_base;
        const uint32_t lo = rs[it.r0], hi = rs[it.r1];
        const uint32_t size = hi - lo;
        // Pingpong: buffer of the subtree root's depth parity; VM storage: in place
        const bool to_scratch = !J.vm && (it.depth & 1u) != 0;
        uint32_t* kdst = (to_scratch ? J.keysB : J.keysA) + I.off + lo;
        uint32_t* pdst = J.want_perm ? (to_scratch ? J.permB : J.permA) + I.off + lo : nullptr;
        const uint32_t* ksrc = J.keysA + I.off + lo;

        if (size > (uint32_t)TILE_MAX) {
            // only a single natural run can exceed the tile size: sorted, or
            // strictly decreasing (reversed pairwise: x and size-1-x by one
            // thread, so in place is safe)
            // every thread reads the first pair before any thread writes
            const bool down = __syncthreads_or(J.desc_runs && ksrc[0] > ksrc[1]) != 0;
            if (down) {
                for (uint32_t x = tid; x < size - 1 - x; x += TILE_BLOCK) {
                    const uint32_t y = size - 1 - x;
                    const uint32_t a = ksrc[x], b = ksrc[y];
                    kdst[x] = b;
                    kdst[y] = a;
                    if (pdst) {
                        pdst[x] = lo + y;
                        pdst[y] = lo + x;
                    }
                }
                if ((size & 1u) && tid == 0) {
                    const uint32_t x = size >> 1;
                    kdst[x] = ksrc[x];
                    if (pdst) pdst[x] = lo + x;
                }
            } else {
                for (uint32_t x = tid; x < size; x += TILE_BLOCK) {
                    if (to_scratch) kdst[x] = ksrc[x];
                    if (pdst) pdst[x] = lo + x;
                }
            }
            if (to_scratch && tid == 0) atomicAdd(&J.ctr->leaf_moves, (unsigned long long)size);
            __syncthreads();
            continue;
        }

        const uint32_t nr = it.r1 - it.r0;   // runs in the tile (<= TILE_RUNS - 1)
        if (nr + 1 > (uint32_t)TILE_RUNS) {  // cannot happen for minrun >= 32
            if (tid == 0) set_error(J.ctr, DERR_INTERNAL, 50);
            continue;
        }
        if (nr >= NET_MIN_RUNS) {
            const int res = tile_network(net, ksrc, size);
            for (uint32_t x = tid; x < size; x += TILE_BLOCK) {
                const unsigned long long w = net.w[res][net_slot(x)];
                kdst[x] = (uint32_t)(w >> 32);
                if (pdst) pdst[x] = lo + (uint32_t)(w & 0xffffffffu);
            }
            __syncthreads();
            continue;
        }
        int cur = 0;
        if (tid == 0) s_mask = 0;
        __syncthreads();
        for (uint32_t k = tid; k <= nr; k += TILE_BLOCK) {
            rs_s[k] = rs[it.r0 + k] - lo;
            if (k >= 1 && k < nr) {
                const uint8_t p = J.power[I.run_base + it.r0 + k];
                pw_s[k] = p;
                atomicOr(&s_mask, 1u << (p - 1));
            }
        }
        for (uint32_t x = tid; x < size; x += TILE_BLOCK) {
            sm.key[0][x] = ksrc[x];
            sm.idx[0][x] = (uint16_t)x;
        }
        __syncthreads();

        // forced runs (length <= 63 whenever unsorted): one warp each, bitonic
        // network on (key, input position) pairs -- the pairs are distinct, so
        // the result is the stable order an insertion sort gives
        for (uint32_t r = warp; r < nr; r += TILE_BLOCK / 32) {
            const uint32_t rlo = rs_s[r], len = rs_s[r + 1] - rlo;
            if (len > 64) {
                // a natural run; reversed when strictly decreasing
                // every lane reads the first pair before any lane writes
                const bool down = J.desc_runs && sm.key[0][rlo] > sm.key[0][rlo + 1];
                if (__any_sync(FULL, down)) {
                    for (uint32_t x = lane; x < len - 1 - x; x += 32) {
                        const uint32_t y = rlo + len - 1 - x;
                        const uint32_t a = sm.key[0][rlo + x], b = sm.key[0][y];
                        const uint16_t ia = sm.idx[0][rlo + x], ib = sm.idx[0][y];
                        sm.key[0][rlo + x] = b;
                        sm.key[0][y] = a;
                        sm.idx[0][rlo + x] = ib;
                        sm.idx[0][y] = ia;
                    }
                    __syncwarp();
                }
                continue;
            }
            if (len < 2) continue;
            const bool ok0 = lane < (int)len, ok1 = lane + 32 < (int)len;
            uint32_t k0 = ok0 ? sm.key[0][rlo + lane] : FULL;
            uint32_t k1 = ok1 ? sm.key[0][rlo + lane + 32] : FULL;
            const uint32_t nk0 = __shfl_down_sync(FULL, k0, 1), f1 = __shfl_sync(FULL, k1, 0);
            const uint32_t nk1 = __shfl_down_sync(FULL, k1, 1);
            const bool d0 = lane + 1 < (int)len && k0 > (lane == 31 ? f1 : nk0);
            const bool d1 = lane + 33 < (int)len && k1 > nk1;
            if (!__any_sync(FULL, d0 || d1)) continue;
            // padding sorts last: key FULL and a position beyond any tile
            uint32_t i0 = ok0 ? rlo + lane : 0x10000u + lane;
            uint32_t i1 = ok1 ? rlo + lane + 32 : 0x10020u + lane;
            const uint32_t kmax = len > 32 ? 64u : 32u;
            for (uint32_t k = 2; k <= kmax; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    if (j == 32) {   // partners in the same lane: slot 0 (i) with slot 1 (i + 32)
                        const bool swap = (k1 < k0) || (k1 == k0 && i1 < i0);   // ascending (i & 64 == 0)
                        if (swap) {
                            const uint32_t tk = k0, ti = i0;
                            k0 = k1; i0 = i1; k1 = tk; i1 = ti;
                        }
                        continue;
                    }
                    const uint32_t pk0 = __shfl_xor_sync(FULL, k0, j), pi0 = __shfl_xor_sync(FULL, i0, j);
                    {
                        const uint32_t idx = (uint32_t)lane;
                        const bool asc = (idx & k) == 0;
                        const bool lower = (idx & j) == 0;
                        const bool pless = (pk0 < k0) || (pk0 == k0 && pi0 < i0);
                        // the lower element keeps the min when ascending, the max otherwise
                        if (pless == (lower == asc)) { k0 = pk0; i0 = pi0; }
                    }
                    if (kmax == 64) {
                        const uint32_t pk1 = __shfl_xor_sync(FULL, k1, j), pi1 = __shfl_xor_sync(FULL, i1, j);
                        const uint32_t idx = (uint32_t)lane + 32;
                        const bool asc = (idx & k) == 0;
                        const bool lower = (idx & j) == 0;
                        const bool pless = (pk1 < k1) || (pk1 == k1 && pi1 < i1);
                        if (pless == (lower == asc)) { k1 = pk1; i1 = pi1; }
                    }
                }
            }
            if (ok0) { sm.key[0][rlo + lane] = k0; sm.idx[0][rlo + lane] = (uint16_t)i0; }
            if (ok1) { sm.key[0][rlo + lane + 32] = k1; sm.idx[0][rlo + lane + 32] = (uint16_t)i1; }
            __syncwarp();
        }
        __syncthreads();

        // merge levels, largest power first
        uint32_t mask = s_mask;
        while (mask) {
            const uint32_t p = 32 - __clz(mask);
            mask &= ~(1u << (p - 1));
            // segments: delimited by boundaries of power < p; a boundary of power
            // p inside a segment is its merge point
            const bool is_b = tid >= 1 && (uint32_t)tid < nr;
            const bool lt = is_b && pw_s[tid] < p;
            const bool eq = is_b && pw_s[tid] == p;
            const uint32_t bl = __ballot_sync(FULL, lt);
            if (lane == 0) warp_cnt[warp] = __popc(bl);
            __syncthreads();
            uint32_t before = __popc(bl & ((1u << lane) - 1u));
            uint32_t total = 0;
            for (int w = 0; w < TILE_BLOCK / 32; ++w) {
                if (w < warp) before += warp_cnt[w];
                total += warp_cnt[w];
            }
            if (tid == 0) {
                seg_lo[0] = 0;
                seg_lo[total + 1] = size;
                s_nseg = total + 1;
            }
            if (lt) seg_lo[before + 1] = rs_s[tid];
            __syncthreads();
            const uint32_t nseg = s_nseg;
            for (uint32_t k = tid; k < nseg; k += TILE_BLOCK) seg_mid[k] = seg_lo[k + 1];
            __syncthreads();
            if (eq) seg_mid[before] = rs_s[tid];
            __syncthreads();

            const uint32_t* ck = sm.key[cur];
            const uint16_t* ci = sm.idx[cur];
            uint32_t* nk = sm.key[cur ^ 1];
            uint16_t* ni = sm.idx[cur ^ 1];
            const uint32_t x0 = tid * TILE_K;
            if (x0 < size) {
                const uint32_t x1 = min(x0 + TILE_K, size);
                uint32_t sg = 0, hiS = nseg;       // last segment with seg_lo <= x0
                while (hiS - sg > 1) {
                    const uint32_t mid = (sg + hiS) >> 1;
                    if (seg_lo[mid] <= x0) sg = mid; else hiS = mid;
                }
                uint32_t x = x0;
                while (x < x1) {
                    const uint32_t slo = seg_lo[sg], smid = seg_mid[sg], shi = seg_lo[sg + 1];
                    const uint32_t end = min(x1, shi);
                    if (smid == shi) {
                        for (; x < end; ++x) {
                            nk[x] = ck[x];
                            ni[x] = ci[x];
                        }
                    } else {
                        // stable merge: keys only, the left segment wins ties
                        const uint32_t la = smid - slo, lb = shi - smid, d = x - slo;
                        uint32_t ilo = d > lb ? d - lb : 0u, ihi = min(d, la);
                        while (ilo < ihi) {
                            const uint32_t m = (ilo + ihi) >> 1;
                            if (ck[slo + m] <= ck[smid + d - 1 - m]) ilo = m + 1; else ihi = m;
                        }
                        uint32_t ia = ilo, ib = d - ilo;
                        uint32_t va = ia < la ? ck[slo + ia] : 0u;
                        uint32_t vb = ib < lb ? ck[smid + ib] : 0u;
                        // branch-free serial merge; an exhausted side is read at the
                        // segment start (a valid slot whose value is never used)
                        for (; x < end; ++x) {
                            const bool take_a = ia < la && (ib >= lb || va <= vb);
                            const uint32_t src = take_a ? slo + ia : smid + ib;
                            nk[x] = take_a ? va : vb;
                            ni[x] = ci[src];
                            ia += take_a;
                            ib += !take_a;
                            const uint32_t nxt = ck[take_a ? (ia < la ? slo + ia : slo) : (ib < lb ? smid + ib : slo)];
                            va = take_a ? nxt : va;
                            vb = take_a ? vb : nxt;
                        }
                    }
                    ++sg;
                }
            }
            __syncthreads();
            cur ^= 1;
        }

        for (uint32_t x = tid; x < size; x += TILE_BLOCK) {
            kdst[x] = sm.key[cur][x];
            if (pdst) pdst[x] = lo + sm.idx[cur][x];
        }
        if (to_scratch && nr == 1 && tid == 0) atomicAdd(&J.ctr->leaf_moves, (unsigned long long)size);
        __syncthreads();
    }
}

constexpr size_t TILE_SMEM = sizeof(TileSmem) > sizeof(NetSmem) ? sizeof(TileSmem) : sizeof(NetSmem);

int tiles_max_grid(int num_sms)
{
    int per_sm = 0;
    cudaFuncSetAttribute(k_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiles, TILE_BLOCK, TILE_SMEM);
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_tiles(const Job& J, int grid, cudaStream_t s)
{
    k_tiles<<<grid, TILE_BLOCK, TILE_SMEM, s>>>(J);
    return cudaGetLastError();
}

}  // namespace ps
