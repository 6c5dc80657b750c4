// Internal declarations shared by the CUDA translation units of the library.
//
// Pipeline of one call (single instance = batch of one):
//   k_setup        per-instance sizes, minrun (Sec. 5), chunk / slot bases
//   k_runs         run detection with minrun extension (ExtractRun, Sec. 2/5):
//                  chunk maps of the chain scan, folded per range, scanned
//   k_runs_emit    run starts of every chunk from its entry state
//   k_nodes        Power per boundary (Sec. 2 Theorem), the element range of
//                  the merge Algorithm 1 performs there, and the split of the
//                  merge tree into HBM merges and on-chip tiles
//   k_depth        depth of the HBM merges (Pingpong buffer parity, Sec. 3)
//   k_bucket_scan  round starts (prefix sums of per-round merge / chunk counts)
//   k_bucket       HBM merges placed by round, chunk numbers; tile depths
//   k_chunk_nodes  chunk -> merge table; parent links and dependency counts
//   k_tiles        runs sorted and merged inside shared memory
//   k_merge_rounds persistent kernel: every HBM merge, scheduled
//                  as a dataflow over the merge tree
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/powersort.h"

namespace ps {

constexpr int RUN_CHUNK = 4096;   // elements per run-detection chunk
constexpr int RUN_HALO = 256;     // descent bits examined past a chunk's end (>= 64)
constexpr int RUN_WORDS = (RUN_CHUNK + RUN_HALO) / 32;
constexpr int RUN_BLOCK = 256;
constexpr int RUN_LOADS = RUN_WORDS * 32 / RUN_BLOCK;   // keys loaded per thread per chunk
static_assert(RUN_WORDS * 32 % RUN_BLOCK == 0, "the bitmask window is a whole number of block loads");
constexpr int MAP_STATES = 64;    // entry states of a chunk: minrun (<= 63) + 1
constexpr int RUN_REC = RUN_CHUNK / 32 + 2;  // run starts one chain can put in a chunk
constexpr uint32_t STATE_END = 255;
constexpr uint32_t CHUNK_FORCED = 1u << 31;   // chunk_info: every step in the chunk is forced
constexpr uint32_t CHUNK_FIRST = 1u << 30;    // chunk_info: the instance's first chunk
constexpr uint32_t RANGE_RESET = 1u << 31;    // range map word: the range restarts an instance
constexpr uint32_t RANGE_COUNT_MASK = 0x7fffffffu;
constexpr int RUN_GRID_PER_SM = 4;            // run-detection CTAs (chunk ranges) per SM
constexpr int RUN_RANGES_MAX = 1024;


constexpr int TILE_BLOCK = 256;
constexpr int TILE_MAX_LOG2 = 12;  // tile capacity bound of the shared-memory layout

constexpr int PLAN_BLOCK = 256;
constexpr int NPOW = 33;           // powers are 1..32 for n < 2^32
constexpr uint32_t NONE = 0xffffffffu;
// VM page record: segment count, then up to 3 segments of (s0, s1, lo, mid,
// hi, four physical pages: the left slice's first page and the next, the
// right slice's first page and the next); a gap has lo = NONE and its page first
constexpr uint32_t VM_REC_WORDS = 32;
constexpr uint32_t VM_SEG_WORDS = 9;
// per page start inside a merge: the split, then the four physical pages of
// the slices that start there
constexpr uint32_t VM_SPLIT_WORDS = 8;

// device error codes (mirrors ps_status)
constexpr uint32_t DERR_INVAL = 1;
constexpr uint32_t DERR_TIMEOUT = 4;
constexpr uint32_t DERR_INTERNAL = 5;

struct Inst {
    unsigned long long off;       // first element in the concatenated arrays
    unsigned long long run_base;  // first slot in the run / boundary arrays
    unsigned long long M;         // merge cost (Sec. 2 Definition)
    uint32_t n;
    uint32_t minrun;
    uint32_t chunk_base;
    uint32_t nchunks;
    uint32_t runs;                // R, written by run detection
    uint32_t max_power;
    uint32_t g_base;              // first entry of the instance's merge map (Job::gmap)
    uint32_t g_span;              // its entries: ceil(4 n / T) when n > T, else 0
    unsigned long long recip;     // floor((2^64 - 1) / n): divisions by n as a multiply (0 when n = 0)
};

// Index of the merge with Power p and dyadic point c / 2^p (c odd) in its
// instance's merge map: merges of one power have distinct points, so
// (p, c) names a merge uniquely; an HBM merge (more than T elements) has
// 2^p < 4n / T, so its index 2^(p-1) - 1 + (c - 1) / 2 < 4n / T.
__host__ __device__ __forceinline__ uint32_t merge_index(uint32_t p, uint32_t c)
{
    return (1u << (p - 1)) - 1u + (c >> 1);
}

// A subtree merged on chip: runs [r0, r1) of an instance; parent = the GNode
// index of the HBM merge it is a child of (NONE: the whole instance).  depth
// = depth of the subtree root.
struct TileItem {
    uint32_t inst, r0, r1, parent, depth, pad;
};

// A merge done through HBM: boundary t of an instance joining runs [a, t)
// and [t, b); midx / pidx = merge-map indices of itself and of its parent
// merge (NONE for the instance's root).
struct GNode {
    uint32_t inst, t, a, b, power, depth, midx, pidx;
};

// HBM merge in round order: output [goff, goff + la + lb), left child
// [goff, goff + la), right child [goff + la, ...), children in buffer
// (depth + 1) & 1, output in buffer depth & 1 (0 = caller's arrays).
struct GSorted {
    unsigned long long goff;
    uint32_t la, lb;
    uint32_t chunk_base;   // number of its first chunk (chunks are numbered round by round)
    uint32_t depth;
    uint32_t parent;       // GSorted index of the parent merge (NONE for an instance's root)
    uint32_t pad;
};

struct Ctr {
    uint32_t error;
    uint32_t err_where;
    uint32_t runs_done;                // run-detection CTAs finished (the last one scans)
    uint32_t total_chunks;
    unsigned long long total_slots;
    uint32_t n_tiles;
    uint32_t n_gnodes;
    uint32_t bucket_count[NPOW + 1];   // HBM merges of round r
    uint32_t bucket_nchunk[NPOW + 1];  // their chunks (merge_e outputs each)
    unsigned long long bucket_cursor[NPOW + 1];   // (merges << 40) | chunks placed so far
    uint32_t bucket_start[NPOW + 2];   // GSorted index where round r starts
    uint32_t bucket_chunk[NPOW + 2];   // chunks of round r: [0, bucket_chunk[r])
    uint32_t rounds;                   // non-empty rounds
    uint32_t bar_count;
    uint32_t bar_gen;
    uint32_t bar_group[32];            // arrivals per group of 32 CTAs (grids of <= 1024 CTAs)
    uint32_t runs_grp_done[32];        // run detection: finished CTAs per group of 32 ranges
    uint32_t chunk_next[NPOW];         // per round: next chunk to hand out (dynamic scheduling)
    // virtual-memory storage
    uint32_t vm_free_top;              // entries on the free-page stack
    uint32_t vm_touched;               // pages written by the current round
    uint32_t vm_wave;                  // final Copy: free pages handed out in the batch
    uint32_t vm_in_use_peak;           // most physical pages holding data at once
    uint32_t vm_waves;                 // VM rounds run by the call
    uint32_t vm_copy_moves;            // page copies made by the final Copy
    uint32_t vm_spliced;               // output pages that took over a whole input page
    uint32_t vm_copy_top[2];           // final Copy: entries on the two free-page stacks
    uint32_t vm_copy_taken[2];         // final Copy: entries of each stack handed out
    uint32_t keys_mapped;              // typed keys: the forward map ran (the inverse must too)
    uint32_t rec_lcp;                  // records: words every row shares (NONE: all rows equal)
    uint32_t rec_groups;               // records: groups of equal window keys listed for the fix-up
    uint32_t rec_nbig;                 // records: groups too large for one CTA's shared memory
    uint32_t rec_gmax;                 // records: the largest group
    uint32_t vm_ring_head;             // tickets handed out: the ring slot each output page pops
    uint32_t vm_ring_tail;             // free pages pushed onto the ring so far
    uint32_t vm_round_base;            // ring_head at the start of the current round
    uint32_t max_power;
    unsigned long long leaf_moves;
    unsigned long long M_total;
    unsigned long long runs_total;
    unsigned long long n_total;
    unsigned long long hbm_elems;      // sum of the sizes of the HBM merges
    // HBM merge timeline (globaltimer, ns): per round the first and last time a
    // chunk's inputs were found complete, the first and last time a chunk's
    // output was sent; merge_t0 = the merge kernel's start
    unsigned long long round_ns[NPOW][4];
    unsigned long long merge_t0;
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct Job {
    uint32_t* keysA;            // caller's keys (buffer 0)
    uint32_t* permA;            // caller's perm or nullptr
    uint32_t* keysB;            // scratch keys (buffer 1)
    uint32_t* permB;            // scratch perm or nullptr
    const unsigned long long* offsets;  // count + 1 entries, or nullptr
    unsigned long long single_n;        // instance size when offsets == nullptr
    uint32_t count;
    uint32_t want_perm;
    uint32_t desc_runs;         // nonzero: strictly decreasing runs are taken and reversed
    uint32_t vm_batched_copy;   // nonzero: VM storage's Copy in batches (PS_FLAG_VM_BATCHED_COPY)
    uint32_t key_type;          // ps_key_type: keys are mapped to order-preserving u32 and back
    const uint32_t* desc_mask;  // records: descent bit per position (run detection reads it, not keys)
    uint32_t tile_cap;          // T: largest merge-tree node merged on chip
    uint32_t merge_e;           // outputs per HBM merge chunk (set from the merge kernel's shape)
    uint32_t merge_lanes;       // search lanes per CTA of the merge kernel (at most its ring size)
    unsigned long long max_n;   // limits the offsets table is checked against
    unsigned long long max_total;
    Inst* inst;
    // run detection's tables (chunk_map, chunk_info) live only until the run
    // starts are written; the merge planning's (tiles, gnodes, gmap) only
    // until the tiles are merged; VM storage's page pool only after that:
    // the three share one region of the context
    uint32_t* chunk_map;        // MAP_STATES per chunk: (runs << 8) | exit state, per entry state
    uint32_t* chunk_info;       // per chunk: CHUNK_FORCED | CHUNK_FIRST | first descent offset
    uint32_t* range_agg;        // MAP_STATES per run-detection CTA: its range's map
    unsigned long long* range_entry;   // per group of 32 run-detection CTAs: (runs before << 8) | entry state
    uint32_t* run_grp_agg;      // MAP_STATES per group of 32 ranges: the group's map
    uint32_t* run_start;        // per run slot: the run's first element (R + 1 per instance)
    uint8_t* power;             // per boundary slot: its Power
    TileItem* tiles;
    GNode* gnodes;
    uint32_t* gmap;             // merge map: per (power, point) index, the merge's GNode index,
                                // then (from k_bucket on) its GSorted index
    GSorted* gsorted;
    uint32_t* dep;              // per GSorted entry: chunks of its HBM children not yet written
    uint32_t* chunk_node;       // per chunk (ids global across rounds): its GSorted index
    Ctr* ctr;
    unsigned long long slot_cap;
    uint32_t chunk_cap;
    uint32_t gnode_cap;         // capacity of gnodes / gsorted / dep
    uint32_t tile_cap_items;    // capacity of tiles
    uint32_t gmap_cap;          // entries of the merge map (all instances)
    uint32_t chunk_node_cap;
    // virtual-memory storage (Sec. 4): pages of P = 2^vm_plog2 elements
    uint32_t vm;                // nonzero: VM storage instead of Pingpong
    uint32_t vm_plog2;
    uint32_t vm_na;             // virtual pages of the instance: ceil(n / P) (set per call)
    uint32_t vm_na_cap;         // capacity of the page tables
    uint32_t vm_pool;           // pool pages (physical pages vm_na_cap .. vm_na_cap + pool)
    uint32_t vm_wave_max;       // output pages in flight at once (one per page group)
    uint32_t vm_ring_cap;       // slots of the free-page ring (never wraps within a call)
    uint32_t* pool_keys;        // pool pages, P keys each
    uint32_t* pool_perm;
    uint32_t* pt;               // virtual page -> physical page
    uint32_t* pt_new;           // the page written for it by the current round
    uint32_t* page_cnt;         // merges of the current round touching the page
    uint32_t* page_nodes;       // 2 per page: those merges (GSorted index)
    uint32_t* consumed;         // elements of the page consumed by the current round
    uint32_t* touched;          // the round's written pages, in order
    uint32_t* free_stack;       // free physical pages: a FIFO ring in the rounds, a stack in Copy
    uint32_t* vm_rec;           // per touched page: its merge segments and gaps (VM_REC_WORDS)
    uint32_t* holder;           // physical page -> virtual page it holds (final Copy)
    uint32_t* vm_split_at;      // per page start inside a merge of the round: its merge-path split
                                // and the slices' pages (VM_SPLIT_WORDS)
    uint32_t* vm_cta_count;     // per CTA of the rounds kernel: touched pages of its block of pages
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void set_error(Ctr* c, uint32_t code, uint32_t where)
{
    if (atomicCAS(&c->error, 0u, code) == 0u) c->err_where = where;
}

// ---- TMA (1-D bulk copies) and mbarrier helpers (sm_90+ PTX) -------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of transaction traffic
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// non-blocking probe of a phase completion
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// global -> shared bulk copy; completes `bytes` on the mbarrier.  Both
// addresses 16-byte aligned, bytes a multiple of 16 (checked by callers).
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// shared -> global bulk copy in the current bulk group (same alignment rules)
__device__ __forceinline__ void tma_store_1d(void* dst_gmem, const void* src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// the shared-memory sources of every committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read_all()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Asynchronous global -> shared copies (cp.async): no registers held while
// they fly; commit groups, then wait for all but the newest N.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Upper bound of spin waits in cycles (about two seconds at 2 GHz); a wait
// that exceeds it records DERR_TIMEOUT and gives up.
constexpr long long SPIN_LIMIT_CYCLES = 4000000000ll;

// Grid-wide barrier of a cooperative launch (all CTAs resident, at most
// 1024): arrivals are counted per group of 32 CTAs, the last group's last
// arrival bumps a generation that the others wait for -- at most
// SPIN_LIMIT_CYCLES, after which DERR_TIMEOUT is recorded and false returned.
__device__ __forceinline__ bool grid_barrier(Ctr* C)
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

// Index of the instance whose [base, base + size) range holds x, for a
// non-decreasing array of bases (binary search; the last of equal bases).
template <typename F>
__device__ __forceinline__ uint32_t find_inst(uint32_t count, unsigned long long x, F base_of)
{
    uint32_t lo = 0, hi = count;  // answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (base_of(mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_setup(const Job& J, cudaStream_t s);
cudaError_t launch_runs(const Job& J, int grid, cudaStream_t s);
uint32_t merge_chunk();
cudaError_t launch_plan(const Job& J, int grid, int nodes_grid, cudaStream_t s);
int nodes_max_grid(int num_sms);
cudaError_t launch_node_ranges(const Job& J, uint32_t q, uint32_t nbound, uint32_t* out, cudaStream_t s);
cudaError_t launch_tiles(const Job& J, int grid, cudaStream_t s);
cudaError_t launch_merge_rounds(const Job& J, int grid, cudaStream_t s);
cudaError_t launch_finish(const Job& J, cudaStream_t s);
cudaError_t launch_vm(const Job& J, int grid, cudaStream_t s);
int vm_rounds_max_grid(int num_sms);
cudaError_t launch_key_map(const Job& J, bool forward, int grid, cudaStream_t s);
cudaError_t launch_records_prepare(const uint32_t* rec, uint32_t W, unsigned long long n, uint32_t* mask,
                                   uint32_t* keys, Ctr* C, int grid, cudaStream_t s);
cudaError_t launch_records_fix(const uint32_t* rec, uint32_t W, unsigned long long n, const uint32_t* keys,
                               uint32_t* perm, uint32_t* tmp, unsigned long long* comp, unsigned long long* comp2,
                               uint32_t* groups, uint32_t cap, uint32_t* big, uint32_t big_cap, Ctr* C, int grid,
                               int coop_grid, bool nested, cudaStream_t s);
int records_fix_big_grid(int num_sms);
// k_rec_nested_cond(cudaGraphConditionalHandle, uint32_t W, uint32_t big_cap, Ctr*): sets
// a graph's condition to "a big group needs the nested sort"
const void* records_nested_cond_kernel();
cudaError_t launch_records_nested_prep(const uint32_t* rec, uint32_t W, const uint32_t* perm, const uint32_t* big,
                                       uint32_t big_cap, unsigned long long* off, uint32_t* keys2, uint32_t* save,
                                       Ctr* C, int grid, cudaStream_t s);
cudaError_t launch_records_nested_apply(uint32_t W, uint32_t* perm, const uint32_t* big, uint32_t big_cap,
                                        const unsigned long long* off, const uint32_t* perm2, const uint32_t* save,
                                        Ctr* C, const Ctr* C2, int grid, cudaStream_t s);
cudaError_t launch_key64(bool in, const void* rows, void* keys, unsigned long long n, uint32_t type, int grid,
                         cudaStream_t s);
cudaError_t launch_wait_probe(Ctr* C, cudaStream_t s);
cudaError_t launch_gather_rows(const uint32_t* perm, const unsigned long long* offsets, uint32_t count,
                               unsigned long long n, unsigned long long max_total, const void* src, void* dst,
                               uint32_t row_bytes, Ctr* ctr, int grid, cudaStream_t s);
uint32_t vm_groups_per_cta(uint32_t plog2);
int merge_rounds_max_grid(int num_sms);
int tiles_max_grid(int num_sms);

}  // namespace ps
