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
// subtree, in an order that respects the tree.  Elements carry their input
// index in the low half of a 64-bit word, so the merges compare (key, index)
// pairs; the left segment's indices are all smaller than the right one's, so
// this is the stable merge of Algorithm 2 (ties take the left run).
//
// The finished tile goes to buffer depth & 1 (0 = caller's arrays, 1 = the
// scratch arrays) with its stable permutation, ready for the HBM rounds.
// A single run longer than T (always a natural, sorted run) is streamed:
// keys copied when its buffer is the scratch one, perm written.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int TILE_MAX = 1 << TILE_MAX_LOG2;
constexpr int TILE_RUNS = TILE_MAX / 32 + 2;   // runs of a tile (minrun >= 32 when n >= 64)
constexpr int TILE_K = TILE_MAX / TILE_BLOCK;  // outputs per thread per level
constexpr unsigned long long PACK_MAX = ~0ull;

}  // namespace

__global__ void __launch_bounds__(TILE_BLOCK) k_tiles(Job J)
{
    extern __shared__ unsigned long long tile_sm[];   // 2 x TILE_MAX packed (key, index)
    __shared__ uint32_t rs_s[TILE_RUNS + 1];
    __shared__ uint8_t pw_s[TILE_RUNS + 1];
    __shared__ uint32_t seg_lo[TILE_RUNS + 2];
    __shared__ uint32_t seg_mid[TILE_RUNS + 2];
    __shared__ uint32_t warp_cnt[TILE_BLOCK / 32];
    __shared__ uint32_t s_mask, s_nseg;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (*(volatile uint32_t*)&J.ctr->error) return;
    const uint32_t ntiles = min(J.ctr->n_tiles, J.entry_cap);

    for (uint32_t e = blockIdx.x; e < ntiles; e += gridDim.x) {
        const TileItem it = J.tiles[e];
        const Inst I = J.inst[it.inst];
        const uint32_t* rs = J.run_start + I.run_base;
        const uint32_t lo = rs[it.r0], hi = rs[it.r1];
        const uint32_t size = hi - lo;
        const bool to_scratch = (it.depth & 1u) != 0;
        uint32_t* kdst = (to_scratch ? J.keysB : J.keysA) + I.off + lo;
        uint32_t* pdst = J.want_perm ? (to_scratch ? J.permB : J.permA) + I.off + lo : nullptr;
        const uint32_t* ksrc = J.keysA + I.off + lo;

        if (size > (uint32_t)TILE_MAX) {
            // only a single natural run (hence sorted) can exceed the tile size
            for (uint32_t x = tid; x < size; x += TILE_BLOCK) {
                if (to_scratch) kdst[x] = ksrc[x];
                if (pdst) pdst[x] = lo + x;
            }
            if (to_scratch && tid == 0) atomicAdd(&J.ctr->leaf_moves, (unsigned long long)size);
            __syncthreads();
            continue;
        }

        unsigned long long* cur = tile_sm;
        unsigned long long* nxt = tile_sm + TILE_MAX;
        const uint32_t nr = it.r1 - it.r0;   // runs in the tile (<= TILE_RUNS - 1)
        if (nr + 1 > (uint32_t)TILE_RUNS) {  // cannot happen for minrun >= 32
            if (tid == 0) set_error(J.ctr, DERR_INTERNAL, 50);
            continue;
        }
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
        for (uint32_t x = tid; x < size; x += TILE_BLOCK)
            cur[x] = ((unsigned long long)ksrc[x] << 32) | x;
        __syncthreads();

        // forced runs (length <= 63 whenever unsorted): sort by rank, one warp each
        for (uint32_t r = warp; r < nr; r += TILE_BLOCK / 32) {
            const uint32_t rlo = rs_s[r], len = rs_s[r + 1] - rlo;
            if (len > 64 || len < 2) continue;
            const unsigned long long v0 = lane < (int)len ? cur[rlo + lane] : PACK_MAX;
            const unsigned long long v1 = lane + 32 < (int)len ? cur[rlo + lane + 32] : PACK_MAX;
            // any descent inside the run?
            const unsigned long long nx0 = __shfl_down_sync(FULL, v0, 1);
            const unsigned long long first1 = __shfl_sync(FULL, v1, 0);
            const unsigned long long nx1 = __shfl_down_sync(FULL, v1, 1);
            const unsigned long long succ0 = lane == 31 ? first1 : nx0;
            const bool d0 = (lane + 1 < (int)len) && (v0 >> 32) > (succ0 >> 32);
            const bool d1 = (lane + 33 < (int)len) && (v1 >> 32) > (nx1 >> 32);
            if (!__any_sync(FULL, d0 || d1)) continue;
            uint32_t rk0 = 0, rk1 = 0;
            for (uint32_t j = 0; j < len; ++j) {
                const unsigned long long y = __shfl_sync(FULL, j < 32 ? v0 : v1, j & 31);
                rk0 += y < v0;
                rk1 += y < v1;
            }
            __syncwarp();
            if (lane < (int)len) cur[rlo + rk0] = v0;
            if (lane + 32 < (int)len) cur[rlo + rk1] = v1;
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
                        for (; x < end; ++x) nxt[x] = cur[x];
                    } else {
                        const uint32_t la = smid - slo, lb = shi - smid, d = x - slo;
                        uint32_t ilo = d > lb ? d - lb : 0u, ihi = min(d, la);
                        while (ilo < ihi) {
                            const uint32_t m = (ilo + ihi) >> 1;
                            if (cur[slo + m] < cur[smid + d - 1 - m]) ilo = m + 1; else ihi = m;
                        }
                        uint32_t ia = ilo, ib = d - ilo;
                        unsigned long long va = ia < la ? cur[slo + ia] : PACK_MAX;
                        unsigned long long vb = ib < lb ? cur[smid + ib] : PACK_MAX;
                        for (; x < end; ++x) {
                            if (va < vb) {
                                nxt[x] = va;
                                ++ia;
                                va = ia < la ? cur[slo + ia] : PACK_MAX;
                            } else {
                                nxt[x] = vb;
                                ++ib;
                                vb = ib < lb ? cur[smid + ib] : PACK_MAX;
                            }
                        }
                    }
                    ++sg;
                }
            }
            __syncthreads();
            unsigned long long* t = cur;
            cur = nxt;
            nxt = t;
        }

        for (uint32_t x = tid; x < size; x += TILE_BLOCK) {
            const unsigned long long v = cur[x];
            kdst[x] = (uint32_t)(v >> 32);
            if (pdst) pdst[x] = lo + (uint32_t)v;
        }
        if (to_scratch && nr == 1 && tid == 0) atomicAdd(&J.ctr->leaf_moves, (unsigned long long)size);
        __syncthreads();
    }
}

int tiles_max_grid(int num_sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiles, TILE_BLOCK,
                                                  2 * TILE_MAX * sizeof(unsigned long long));
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_tiles(const Job& J, int grid, cudaStream_t s)
{
    const size_t smem = 2 * TILE_MAX * sizeof(unsigned long long);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_tiles<<<grid, TILE_BLOCK, smem, s>>>(J);
    return cudaGetLastError();
}

}  // namespace ps
