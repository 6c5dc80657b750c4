// HBM merge rounds: the merges of Algorithm 1 whose inputs exceed the tile
// size, executed as stable out-of-place merges (Algorithm 2, StandardMerge:
// ties take the left run) between the caller's arrays and the scratch arrays
// (Pingpong storage, Sec. 3).
//
// Rounds go from the largest power to the smallest; all merges of one round
// are disjoint and their children are finished.  Every merge is cut into
// chunks of MERGE_E outputs.  Phase A finds, for every chunk start, how many
// of the first d outputs come from the left child (merge-path split: the
// largest i with A[i-1] <= B[d-i], ties to the left).  Phase B gives each
// chunk to a CTA, which stages the chunk's two input slices in shared memory,
// merges them (each thread K outputs, again split by merge path) and writes
// keys and permutation entries back with coalesced stores.
//
// One persistent cooperative launch runs every round; a grid barrier (bounded
// spin, error flag on timeout) separates the phases.  Cooperative launch
// guarantees that all CTAs are resident, so the barrier cannot starve.
#include "ps_internal.cuh"

namespace ps {

namespace {

__device__ bool grid_barrier(Ctr* C)
{
    __syncthreads();
    __shared__ uint32_t s_ok;
    if (threadIdx.x == 0) {
        uint32_t ok = 1;
        const uint32_t gen = ld_acquire_u32(&C->bar_gen);
        __threadfence();
        const uint32_t arrived = atomicAdd(&C->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&C->bar_count, 0u);
            __threadfence();
            st_release_u32(&C->bar_gen, gen + 1);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_u32(&C->bar_gen) == gen) {
                __nanosleep(32);
                if (clock64() - t0 > SPIN_LIMIT_CYCLES) {
                    set_error(C, DERR_TIMEOUT, 40);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ uint32_t node_of_chunk(const GSorted* gs, uint32_t e0, uint32_t e1, uint32_t cid)
{
    uint32_t lo = e0, hi = e1;   // last e in [e0, e1) with chunk_base <= cid
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (gs[mid].chunk_base <= cid) lo = mid; else hi = mid;
    }
    return lo;
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

}  // namespace

__global__ void __launch_bounds__(MERGE_BLOCK) k_merge_rounds(Job J)
{
    __shared__ uint32_t sk[MERGE_E];
    __shared__ uint32_t sp[MERGE_E];
    __shared__ GSorted s_node;
    __shared__ uint32_t s_e;
    Ctr* C = J.ctr;
    const int tid = threadIdx.x;
    const bool perm = J.want_perm != 0;

    for (int r = 0; r < NPOW; ++r) {
        if (*(volatile uint32_t*)&C->error) return;
        const uint32_t e0 = C->bucket_start[r], e1 = C->bucket_start[r + 1];
        if (e0 == e1) continue;
        const uint32_t c0 = C->bucket_chunk[r], c1 = C->bucket_chunk[r + 1];
        const uint32_t nch = c1 - c0;

        // phase A: merge-path split of every chunk start
        for (uint32_t q = blockIdx.x * blockDim.x + tid; q < nch; q += gridDim.x * blockDim.x) {
            const uint32_t cid = c0 + q;
            const GSorted g = J.gsorted[node_of_chunk(J.gsorted, e0, e1, cid)];
            const uint32_t d = (cid - g.chunk_base) * MERGE_E;
            const uint32_t* src = ((g.depth + 1) & 1u) ? J.keysB : J.keysA;
            const uint32_t* A = src + g.goff;
            J.splits[q] = merge_path(A, g.la, A + g.la, g.lb, d);
        }
        if (!grid_barrier(C)) return;

        // phase B: one chunk per CTA iteration
        for (uint32_t q = blockIdx.x; q < nch; q += gridDim.x) {
            const uint32_t cid = c0 + q;
            if (tid == 0) {
                s_e = node_of_chunk(J.gsorted, e0, e1, cid);
                s_node = J.gsorted[s_e];
            }
            __syncthreads();
            const GSorted g = s_node;
            const uint32_t total = g.la + g.lb;
            const uint32_t d0 = (cid - g.chunk_base) * MERGE_E;
            const uint32_t d1 = min(d0 + (uint32_t)MERGE_E, total);
            const uint32_t a0 = J.splits[q];
            const uint32_t a1 = d1 == total ? g.la : J.splits[q + 1];
            const uint32_t b0 = d0 - a0, b1 = d1 - a1;
            const uint32_t na = a1 - a0, nb = b1 - b0, cnt = na + nb;
            const bool src_b = ((g.depth + 1) & 1u) != 0;
            const uint32_t* ksrc = (src_b ? J.keysB : J.keysA) + g.goff;
            const uint32_t* psrc = perm ? (src_b ? J.permB : J.permA) + g.goff : nullptr;
            uint32_t* kdst = ((g.depth & 1u) ? J.keysB : J.keysA) + g.goff + d0;
            uint32_t* pdst = perm ? ((g.depth & 1u) ? J.permB : J.permA) + g.goff + d0 : nullptr;

            // stage: left slice then right slice
#pragma unroll
            for (int j = 0; j < MERGE_K; ++j) {
                const uint32_t i = tid + j * MERGE_BLOCK;
                if (i < cnt) {
                    const uint32_t gi = i < na ? a0 + i : g.la + b0 + (i - na);
                    sk[i] = ksrc[gi];
                    if (perm) sp[i] = psrc[gi];
                }
            }
            __syncthreads();

            // each thread: MERGE_K consecutive outputs
            uint32_t ok[MERGE_K], op[MERGE_K];
            const uint32_t x0 = tid * MERGE_K;
            if (x0 < cnt) {
                uint32_t lo = x0 > nb ? x0 - nb : 0u, hi = min(x0, na);
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (sk[mid] <= sk[na + x0 - 1 - mid]) lo = mid + 1; else hi = mid;
                }
                uint32_t ia = lo, ib = na + (x0 - lo);
                const uint32_t bend = cnt;
#pragma unroll
                for (int j = 0; j < MERGE_K; ++j) {
                    if (x0 + j < cnt) {
                        const bool take_a = ia < na && (ib >= bend || sk[ia] <= sk[ib]);
                        const uint32_t src = take_a ? ia : ib;
                        ok[j] = sk[src];
                        op[j] = perm ? sp[src] : 0u;
                        if (take_a) ++ia; else ++ib;
                    }
                }
            }
            __syncthreads();
            if (x0 < cnt) {
#pragma unroll
                for (int j = 0; j < MERGE_K; ++j) {
                    if (x0 + j < cnt) {
                        sk[x0 + j] = ok[j];
                        if (perm) sp[x0 + j] = op[j];
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < MERGE_K; ++j) {
                const uint32_t i = tid + j * MERGE_BLOCK;
                if (i < cnt) {
                    kdst[i] = sk[i];
                    if (perm) pdst[i] = sp[i];
                }
            }
            __syncthreads();
        }
        if (!grid_barrier(C)) return;
    }
}

int merge_rounds_max_grid(int num_sms)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_rounds, MERGE_BLOCK, 0);
    return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_merge_rounds(const Job& J, int grid, cudaStream_t s)
{
    void* args[] = {(void*)&J};
    return cudaLaunchCooperativeKernel((const void*)k_merge_rounds, dim3(grid), dim3(MERGE_BLOCK), args, 0, s);
}

}  // namespace ps
