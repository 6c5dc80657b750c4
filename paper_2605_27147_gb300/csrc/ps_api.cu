// C ABI of the library (include/powersort.h): argument checks, the context
// with every device buffer allocated up front, and the launch sequence.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ps_internal.cuh"

struct ps_ctx {
    ps_config cfg;
    int device;
    cudaStream_t stream;
    int num_sms;
    int grid_runs, grid_plan, grid_nodes, grid_tiles, grid_vm;
    int grid_merge;
    unsigned long long max_total;
    uint32_t max_count;
    ps::Job base;               // device buffers; per-call fields filled by each run
    ps::Ctr* h_ctr;             // pinned host copy of the counters
    ps::Inst* h_inst;           // pinned host copy of one instance record
    uint32_t last_count;
    int last_valid;
    size_t scratch_bytes;
    std::vector<void*> allocs;
    std::vector<unsigned char*> guards;   // canary words after every allocation
    bool timing;
    bool capturing;             // inside ps_graph_create_batched: no events, no syncs
    cudaEvent_t ev[7];          // phase boundaries of the last call (PS_FLAG_TIMING)
    uint32_t* io_keys;          // device arrays of ps_run_host (PS_FLAG_HOST_IO)
    uint32_t* io_perm;
    uint32_t* rec_keys;         // ps_sort_records (PS_FLAG_RECORDS): window keys,
    uint32_t* rec_mask;         //   descent mask,
    uint32_t* rec_tmp;          //   merge scratch of the tie fix-up,
    uint32_t* rec_groups;       //   groups of equal windows (start, end)
    uint32_t rec_group_cap;
    uint32_t* rec_rows;         //   ps_sort_keys64: the sorted (high, low) rows
    uint32_t* rec_big;          //   the groups larger than one CTA's shared memory
    uint32_t rec_big_cap;
    int grid_rec_big;           //   cooperative grid of their merge passes
    unsigned long long* rec_off; //  two-word rows: the big groups as instances of
    ps_ctx* rec_inner;          //   a batched 32-bit sort in this inner context,
    cudaStream_t rec_cap_stream; //  captured on this stream into the body of a
    cudaGraph_t rec_graph;      //   graph's conditional node (run only when a
    cudaGraphExec_t rec_exec;   //   big group exists)
};

namespace {

constexpr unsigned long long LIMIT_N = 0xffffffffull;  // instance sizes and totals < 2^32
constexpr uint32_t LAUNCHES_PER_CALL = 11;  // setup, 2 run detection, 5 planning, tiles, merges, finish
constexpr uint32_t NPHASES = 6;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr size_t GUARD_BYTES = 64;
constexpr unsigned char GUARD_BYTE = 0xa5;

// Device allocation owned by the context, followed by GUARD_BYTES of canary
// (ps_check_guards reads them back).
template <typename T>
ps_status dev_alloc(ps_ctx* c, T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) return PS_OK;
    void* q = nullptr;
    const size_t bytes = (count * sizeof(T) + 15) & ~(size_t)15;
    if (cudaMalloc(&q, bytes + GUARD_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return PS_ENOMEM;
    }
    c->allocs.push_back(q);
    unsigned char* g = static_cast<unsigned char*>(q) + bytes;
    if (cudaMemset(g, GUARD_BYTE, GUARD_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return PS_ECUDA;
    }
    c->guards.push_back(g);
    c->scratch_bytes += count * sizeof(T);
    *p = static_cast<T*>(q);
    return PS_OK;
}

void free_all(ps_ctx* c)
{
    if (c->rec_exec) cudaGraphExecDestroy(c->rec_exec);
    if (c->rec_graph) cudaGraphDestroy(c->rec_graph);
    c->rec_exec = nullptr;
    c->rec_graph = nullptr;
    if (c->rec_inner) ::ps_destroy(c->rec_inner);
    c->rec_inner = nullptr;
    if (c->rec_cap_stream) cudaStreamDestroy(c->rec_cap_stream);
    c->rec_cap_stream = nullptr;
    if (c->timing)
        for (cudaEvent_t& e : c->ev)
            if (e) cudaEventDestroy(e);
    c->timing = false;
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->guards.clear();
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->h_inst) cudaFreeHost(c->h_inst);
    c->h_ctr = nullptr;
    c->h_inst = nullptr;
}

ps_status from_device_error(uint32_t e)
{
    if (e == ps::DERR_INVAL) return PS_EINVAL;
    if (e == ps::DERR_TIMEOUT) return PS_ETIMEOUT;
    if (e != 0) return PS_EINTERNAL;
    return PS_OK;
}

ps_status enqueue(ps_ctx* c, const ps::Job& J)
{
    cudaStream_t s = c->stream;
    auto mark = [&](int i) {
        return !c->timing || c->capturing || cudaEventRecord(c->ev[i], s) == cudaSuccess;
    };
    if (!mark(0)) return PS_ECUDA;
    if (ps::launch_setup(J, s) != cudaSuccess) return PS_ECUDA;
    // typed keys: to order-preserving unsigned words before run detection
    if (J.key_type != PS_KEY_U32 && ps::launch_key_map(J, true, c->grid_runs, s) != cudaSuccess) return PS_ECUDA;
    if (!mark(1)) return PS_ECUDA;
    if (ps::launch_runs(J, c->grid_runs, s) != cudaSuccess || !mark(2)) return PS_ECUDA;
    if (ps::launch_plan(J, c->grid_plan, c->grid_nodes, s) != cudaSuccess || !mark(3)) return PS_ECUDA;
    if (ps::launch_tiles(J, c->grid_tiles, s) != cudaSuccess || !mark(4)) return PS_ECUDA;
    if (J.vm) {
        if (ps::launch_vm(J, c->grid_vm, s) != cudaSuccess || !mark(5)) return PS_ECUDA;
    } else {
        if (ps::launch_merge_rounds(J, c->grid_merge, s) != cudaSuccess || !mark(5)) return PS_ECUDA;
    }
    if (ps::launch_finish(J, s) != cudaSuccess) return PS_ECUDA;
    if (J.key_type != PS_KEY_U32 && ps::launch_key_map(J, false, c->grid_runs, s) != cudaSuccess) return PS_ECUDA;
    if (!mark(6)) return PS_ECUDA;
    if (cudaMemcpyAsync(c->h_ctr, J.ctr, sizeof(ps::Ctr), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PS_ECUDA;
    return PS_OK;
}

ps_status sync_and_check(ps_ctx* c)
{
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return PS_ECUDA;
    }
    return from_device_error(c->h_ctr->error);
}

void fill_stats(const ps_ctx* c, ps_stats* st, uint32_t count)
{
    std::memset(st, 0, sizeof(*st));
    const ps::Ctr* h = c->h_ctr;
    st->n = h->n_total;
    st->runs = h->runs_total;
    st->merge_cost = h->M_total;
    st->tiles = h->n_tiles;
    st->global_nodes = h->n_gnodes;
    st->leaf_moves = h->leaf_moves;
    st->scratch_bytes = c->scratch_bytes;
    st->peak_pages = c->base.vm ? h->vm_in_use_peak : 0;
    st->max_power = h->max_power;
    st->rounds = h->rounds;
    st->instances = count;
    st->hbm_merge_elems = h->hbm_elems;
    // VM: rounds + the final Copy; typed keys: the two maps
    st->launches = LAUNCHES_PER_CALL + (c->base.vm ? 1u : 0u) + (c->base.key_type != PS_KEY_U32 ? 2u : 0u);
    st->pages_spliced = c->base.vm ? h->vm_spliced : 0u;
    st->page_size = c->base.vm ? 1u << c->base.vm_plog2 : 0u;
    st->pool_pages = c->base.vm ? c->base.vm_pool : 0u;
    st->copy_pages = c->base.vm ? h->vm_copy_moves : 0u;
}

ps_status run_common(ps_ctx* c, uint32_t* d_keys, uint32_t* d_perm, const uint64_t* d_offsets,
                     unsigned long long single_n, uint32_t count, ps_stats* stats)
{
    DeviceGuard g(c->device);
    ps::Job J = c->base;
    J.keysA = d_keys;
    J.permA = d_perm;
    J.want_perm = d_perm ? 1u : 0u;
    if (!d_perm) {
        J.permB = nullptr;
        J.permA = nullptr;
    }
    if (J.vm) J.vm_na = (uint32_t)((single_n + (1ull << J.vm_plog2) - 1) >> J.vm_plog2);
    J.offsets = reinterpret_cast<const unsigned long long*>(d_offsets);
    J.single_n = single_n;
    J.count = count;
    c->last_valid = 0;
    ps_status st = enqueue(c, J);
    if (st != PS_OK) {
        cudaGetLastError();
        return st;
    }
    c->last_valid = 1;
    c->last_count = count;
    if (stats) {
        st = sync_and_check(c);
        if (st != PS_OK) return st;
        fill_stats(c, stats, count);
        // minrun of the first instance
        if (cudaMemcpy(c->h_inst, J.inst, sizeof(ps::Inst), cudaMemcpyDeviceToHost) != cudaSuccess) return PS_ECUDA;
        stats->minrun = c->h_inst->minrun;
    }
    return PS_OK;
}

ps_status read_inst(ps_ctx* c, uint32_t q, ps::Inst* out)
{
    if (!c->last_valid || q >= c->last_count) return PS_EINVAL;
    ps_status st = sync_and_check(c);
    if (st != PS_OK) return st;
    if (cudaMemcpy(c->h_inst, c->base.inst + q, sizeof(ps::Inst), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PS_ECUDA;
    *out = *c->h_inst;
    return PS_OK;
}

}  // namespace

extern "C" {

PS_API const char* ps_status_str(ps_status s)
{
    switch (s) {
    case PS_OK: return "PS_OK";
    case PS_EINVAL: return "PS_EINVAL: invalid argument";
    case PS_ENOMEM: return "PS_ENOMEM: device allocation failed";
    case PS_ECUDA: return "PS_ECUDA: CUDA call failed";
    case PS_ETIMEOUT: return "PS_ETIMEOUT: device-side wait exceeded its limit";
    case PS_EINTERNAL: return "PS_EINTERNAL: device-side consistency check failed";
    case PS_ECANCELED: return "PS_ECANCELED: request cancelled before it ran";
    }
    return "unknown ps_status";
}

namespace {

// The nested sort of two-word rows' big tie groups as a graph: a kernel sets
// the condition from the device-side count of big groups, and the
// conditional node's body is the inner context's batched sort of the fixed
// buffers (captured once).  On failure the graph is left out.
void build_nested_graph(ps_ctx* c)
{
    ps_ctx* in = c->rec_inner;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNode_t kn = nullptr, cn = nullptr;
    uint32_t W = 2, cap = c->rec_big_cap;
    ps::Ctr* C = c->base.ctr;
    void* args[] = {&h, &W, &cap, &C};
    if (ok) {
        cudaGraphNodeParams kp = {};
        kp.type = cudaGraphNodeTypeKernel;
        kp.kernel.func = const_cast<void*>(ps::records_nested_cond_kernel());
        kp.kernel.gridDim = dim3(1);
        kp.kernel.blockDim = dim3(32);
        kp.kernel.kernelParams = args;
        ok = cudaGraphAddNode(&kn, g, nullptr, nullptr, 0, &kp) == cudaSuccess;
    }
    cudaGraph_t body = nullptr;
    if (ok) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&cn, g, &kn, nullptr, 1, &cp) == cudaSuccess;
        if (ok) body = cp.conditional.phGraph_out[0];
    }
    if (ok) {
        ok = cudaStreamBeginCaptureToGraph(c->rec_cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            in->capturing = true;
            const ps_status st = run_common(in, c->rec_tmp, c->rec_tmp + c->cfg.max_n,
                                            reinterpret_cast<const uint64_t*>(c->rec_off), 0, c->rec_big_cap, nullptr);
            in->capturing = false;
            cudaGraph_t captured = nullptr;
            const cudaError_t e = cudaStreamEndCapture(c->rec_cap_stream, &captured);
            ok = st == PS_OK && e == cudaSuccess;
            in->last_valid = 0;
        }
    }
    cudaGraphExec_t ex = nullptr;
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        return;
    }
    c->rec_graph = g;
    c->rec_exec = ex;
}

}  // namespace

PS_API ps_status ps_create(const ps_config* cfg, int device, void* cuda_stream, ps_ctx** out)
{
    if (!out) return PS_EINVAL;
    *out = nullptr;
    if (!cfg) return PS_EINVAL;
    if (cfg->mode != PS_MODE_PINGPONG && cfg->mode != PS_MODE_VM) return PS_EINVAL;
    if (cfg->key_type > PS_KEY_F32) return PS_EINVAL;
    if (cfg->mode == PS_MODE_VM && cfg->max_count > 1) return PS_EINVAL;   // VM storage: one instance per call
    if (cfg->max_n == 0 || cfg->max_n > LIMIT_N) return PS_EINVAL;
    const unsigned long long max_total = cfg->max_total ? cfg->max_total : cfg->max_n;
    if (max_total < cfg->max_n || max_total > LIMIT_N) return PS_EINVAL;
    const uint32_t tile_log2 = cfg->tile_log2 ? cfg->tile_log2 : (uint32_t)ps::TILE_MAX_LOG2;
    if (tile_log2 < 10 || tile_log2 > (uint32_t)ps::TILE_MAX_LOG2) return PS_EINVAL;
    if (device < 0) return PS_EINVAL;
    if (cfg->merge_lanes > 16 || cfg->merge_ctas > 2) return PS_EINVAL;

    ps_ctx* c = new (std::nothrow) ps_ctx();
    if (!c) return PS_ENOMEM;
    c->cfg = *cfg;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->max_total = max_total;
    c->max_count = cfg->max_count ? cfg->max_count : 1u;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
        cudaGetLastError();
        delete c;
        return PS_ECUDA;
    }
    DeviceGuard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return PS_ECUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    c->grid_runs = std::min(c->num_sms * ps::RUN_GRID_PER_SM, ps::RUN_RANGES_MAX);
    c->grid_plan = c->num_sms * 8;
    c->grid_nodes = ps::nodes_max_grid(c->num_sms);
    c->grid_tiles = ps::tiles_max_grid(c->num_sms);
    c->grid_merge = ps::merge_rounds_max_grid(c->num_sms);
    if (cfg->merge_ctas && c->grid_merge > c->num_sms * (int)cfg->merge_ctas)
        c->grid_merge = c->num_sms * (int)cfg->merge_ctas;
    c->grid_vm = ps::vm_rounds_max_grid(c->num_sms);
    if (c->grid_vm > 1024) c->grid_vm = 1024;

    ps::Job& J = c->base;
    std::memset(&J, 0, sizeof(J));
    J.tile_cap = 1u << tile_log2;
    J.merge_e = ps::merge_chunk();
    J.merge_lanes = cfg->merge_lanes;
    J.max_n = cfg->max_n;
    J.max_total = max_total;
    const unsigned long long slot_cap = max_total / 32 + 2ull * c->max_count + 2;
    const unsigned long long chunk_cap = max_total / ps::RUN_CHUNK + c->max_count + 1;
    const unsigned long long T = J.tile_cap;
    // the merge map: ceil(4 n / T) entries per instance of more than T
    // elements (an HBM merge of Power p has 2^p < 4n / T)
    const unsigned long long gmap_cap = (4ull * max_total + T - 1) / T + c->max_count + 1;
    // HBM merges: at most one per merge-map entry; for one instance, at most
    // min(2^(p-1), n / (T + 1)) of every power p with 2^p < 4n / T (merges of
    // one power have distinct odd points c < 2^p, are disjoint, and each has
    // more than T elements)
    unsigned long long gnode_cap = gmap_cap;
    unsigned pmax = 0;                 // the largest power an HBM merge can have
    while (pmax < 34 && ((1ull << (pmax + 1)) * T < 4ull * cfg->max_n)) ++pmax;
    if (c->max_count == 1) {
        unsigned long long g = 0;
        for (unsigned p = 1; p <= pmax; ++p) g += std::min(1ull << (p - 1), (unsigned long long)cfg->max_n / (T + 1));
        gnode_cap = std::min(gnode_cap, g + 1);
    }
    // tiles: the two children of every HBM merge, or the whole instance
    const unsigned long long tile_items_cap = 2 * gnode_cap + c->max_count + 1;
    // chunks summed over all rounds: the HBM merges of one power are disjoint,
    // so every power holds at most max_total outputs, plus one partial chunk
    // per merge
    const unsigned long long chunk_node_cap =
        (unsigned long long)pmax * (max_total / ps::merge_chunk()) + gnode_cap + 2;
    if (chunk_cap > 0xffffffffull || gmap_cap > 0xffffffffull || tile_items_cap > 0xffffffffull ||
        chunk_node_cap > 0xffffffffull) {
        delete c;
        return PS_EINVAL;
    }
    J.slot_cap = slot_cap;
    J.chunk_cap = (uint32_t)chunk_cap;
    J.gnode_cap = (uint32_t)gnode_cap;
    J.tile_cap_items = (uint32_t)tile_items_cap;
    J.gmap_cap = (uint32_t)gmap_cap;
    J.chunk_node_cap = (uint32_t)chunk_node_cap;

    ps_status st = PS_OK;
    const bool vm = cfg->mode == PS_MODE_VM;
    if (vm) {
        // page size: sqrt(n / log2 n) rounded to a power of two (Sec. 4), at most
        // the tile size (so a page meets at most two HBM merges), at least 2^8
        uint32_t plog2 = cfg->page_log2;
        if (!plog2) {
            const double nn = (double)cfg->max_n > 4.0 ? (double)cfg->max_n : 4.0;
            plog2 = (uint32_t)std::lround(std::log2(std::sqrt(nn / std::log2(nn))));
        }
        if (plog2 < 8) plog2 = 8;
        if (plog2 > tile_log2) plog2 = tile_log2;
        J.vm = 1;
        J.vm_plog2 = plog2;
        J.vm_na_cap = (uint32_t)((cfg->max_n + (1ull << plog2) - 1) >> plog2);
        // pages in flight: one output page per page group of every CTA; the
        // pool holds them plus slack for partly consumed pages.  A quarter
        // more than the groups keeps the groups from waiting for freed pages
        // (measured on GB300: 2^28 keys, pages of 4096, the page dataflow
        // took 22.8 ms with 64 pages of slack and 21.4 ms with 292; 2^24,
        // pages of 1024, the merge phase 2.20 and 2.05 ms with 64 and 668)
        J.vm_wave_max = (uint32_t)c->grid_vm * ps::vm_groups_per_cta(plog2);
        J.vm_pool = cfg->pool_pages ? cfg->pool_pages : J.vm_wave_max + J.vm_wave_max / 4 + 64;
        if (J.vm_pool < 16) J.vm_pool = 16;
        // the free-page ring: the pool's pages plus at most one push per page per round
        J.vm_ring_cap = J.vm_pool + (uint32_t)ps::NPOW * J.vm_na_cap;
        // the final Copy keeps two free-page stacks of up to every physical page
        if (J.vm_ring_cap < 2 * (J.vm_na_cap + J.vm_pool)) J.vm_ring_cap = 2 * (J.vm_na_cap + J.vm_pool);
        if (st == PS_OK) st = dev_alloc(c, &J.pt, J.vm_na_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.pt_new, J.vm_na_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.page_cnt, J.vm_na_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.page_nodes, 2ull * J.vm_na_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.consumed, J.vm_na_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.touched, J.vm_na_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.free_stack, (size_t)J.vm_ring_cap);
        if (st == PS_OK) st = dev_alloc(c, &J.vm_rec, (size_t)J.vm_na_cap * ps::VM_REC_WORDS);
        if (st == PS_OK) st = dev_alloc(c, &J.holder, (size_t)J.vm_na_cap + J.vm_pool);
        if (st == PS_OK) st = dev_alloc(c, &J.vm_split_at, ((size_t)J.vm_na_cap + 1) * ps::VM_SPLIT_WORDS);
        if (st == PS_OK) st = dev_alloc(c, &J.vm_cta_count, (size_t)c->grid_vm);
    } else {
        if (st == PS_OK) st = dev_alloc(c, &J.keysB, max_total);
        if (st == PS_OK && cfg->want_perm) st = dev_alloc(c, &J.permB, max_total);
        if (st == PS_OK) st = dev_alloc(c, &J.chunk_node, chunk_node_cap);
    }
    // One region for three sets of tables whose lifetimes do not overlap (all
    // on the context's stream): run detection's chunk maps (until the run
    // starts are written), the merge planning's tiles, HBM merges and merge
    // map (until the tiles are merged), and VM storage's page pool (the merge
    // rounds and Copy).
    {
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        const size_t b_map = al(chunk_cap * ps::MAP_STATES * 4), b_info = al(chunk_cap * 4);
        const size_t b_tiles = al(tile_items_cap * sizeof(ps::TileItem)), b_gn = al(gnode_cap * sizeof(ps::GNode));
        const size_t b_gmap = al(gmap_cap * 4);
        const size_t b_pool = vm ? al((size_t)J.vm_pool << J.vm_plog2 << 2) : 0;
        const size_t bytes = std::max(std::max(b_map + b_info, b_tiles + b_gn + b_gmap),
                                      b_pool * (cfg->want_perm ? 2u : 1u));
        unsigned char* U = nullptr;
        if (st == PS_OK) st = dev_alloc(c, &U, bytes);
        if (U) {
            J.chunk_map = reinterpret_cast<uint32_t*>(U);
            J.chunk_info = reinterpret_cast<uint32_t*>(U + b_map);
            J.tiles = reinterpret_cast<ps::TileItem*>(U);
            J.gnodes = reinterpret_cast<ps::GNode*>(U + b_tiles);
            J.gmap = reinterpret_cast<uint32_t*>(U + b_tiles + b_gn);
            if (vm) {
                J.pool_keys = reinterpret_cast<uint32_t*>(U);
                J.pool_perm = cfg->want_perm ? reinterpret_cast<uint32_t*>(U + b_pool) : nullptr;
            }
        }
    }
    if (st == PS_OK) st = dev_alloc(c, &J.inst, c->max_count);
    if (st == PS_OK) st = dev_alloc(c, &J.range_agg, (size_t)c->grid_runs * ps::MAP_STATES);
    if (st == PS_OK) st = dev_alloc(c, &J.range_entry, (size_t)c->grid_runs);
    if (st == PS_OK) st = dev_alloc(c, &J.run_grp_agg, (size_t)32 * ps::MAP_STATES);
    if (st == PS_OK) st = dev_alloc(c, &J.run_start, slot_cap);
    if (st == PS_OK) st = dev_alloc(c, &J.power, slot_cap);
    if (st == PS_OK) st = dev_alloc(c, &J.gsorted, gnode_cap);
    if (st == PS_OK) st = dev_alloc(c, &J.dep, gnode_cap);
    if (st == PS_OK) st = dev_alloc(c, &J.ctr, 1);
    if (st == PS_OK && (cfg->flags & PS_FLAG_RECORDS)) {
        c->rec_group_cap = (uint32_t)(cfg->max_n / 2 + 1);
        st = dev_alloc(c, &c->rec_keys, cfg->max_n);
        if (st == PS_OK) st = dev_alloc(c, &c->rec_mask, cfg->max_n / 32 + 2);
        if (st == PS_OK) st = dev_alloc(c, &c->rec_tmp, 2ull * cfg->max_n);   // u32 scratch, or packed u64 words
        if (st == PS_OK) st = dev_alloc(c, &c->rec_groups, 2ull * c->rec_group_cap);
        c->rec_big_cap = (uint32_t)(cfg->max_n / 2048 + 2);
        if (st == PS_OK) st = dev_alloc(c, &c->rec_big, 2ull * c->rec_big_cap);
        if (st == PS_OK) st = dev_alloc(c, &c->rec_rows, 2ull * cfg->max_n);
        c->grid_rec_big = ps::records_fix_big_grid(c->num_sms);
        if (st == PS_OK && cfg->mode == PS_MODE_PINGPONG) {
            // two-word rows (64-bit keys): the big tie groups' last words are
            // sorted as one batch of 32-bit instances
            st = dev_alloc(c, &c->rec_off, (size_t)c->rec_big_cap + 1);
            ps_config ic{};
            ic.mode = PS_MODE_PINGPONG;
            ic.want_perm = 1;
            ic.max_n = cfg->max_n;
            ic.max_total = cfg->max_n;
            ic.max_count = c->rec_big_cap;
            ic.merge_lanes = cfg->merge_lanes;
            ic.merge_ctas = cfg->merge_ctas;
            // the inner context enqueues on a private stream, so that its sort
            // can be captured (the caller's stream may be the legacy one)
            if (st == PS_OK && cudaStreamCreateWithFlags(&c->rec_cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                st = PS_ECUDA;
            if (st == PS_OK) st = ps_create(&ic, device, c->rec_cap_stream, &c->rec_inner);
            if (st == PS_OK) c->scratch_bytes += c->rec_inner->scratch_bytes;
            if (st == PS_OK) build_nested_graph(c);   // without it the sort is enqueued directly
        }
    }
    if (st == PS_OK && (cfg->flags & PS_FLAG_HOST_IO)) {
        st = dev_alloc(c, &c->io_keys, max_total);
        if (st == PS_OK && cfg->want_perm) st = dev_alloc(c, &c->io_perm, max_total);
    }
    J.desc_runs = (cfg->flags & PS_FLAG_DESCENDING_RUNS) ? 1u : 0u;
    J.vm_batched_copy = (cfg->flags & PS_FLAG_VM_BATCHED_COPY) ? 1u : 0u;
    J.key_type = cfg->key_type;
    if (st == PS_OK && (cfg->flags & PS_FLAG_TIMING)) {
        c->timing = true;
        for (cudaEvent_t& e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) st = PS_ECUDA;
    }
    if (st == PS_OK && cudaMallocHost(&c->h_ctr, sizeof(ps::Ctr)) != cudaSuccess) st = PS_ENOMEM;
    if (st == PS_OK && cudaMallocHost(&c->h_inst, sizeof(ps::Inst)) != cudaSuccess) st = PS_ENOMEM;
    if (st == PS_OK && cudaMemset(J.ctr, 0, sizeof(ps::Ctr)) != cudaSuccess)
        st = PS_ECUDA;
    if (st == PS_OK && cudaDeviceSynchronize() != cudaSuccess) st = PS_ECUDA;
    // every table the kernels write must exist (permB only with want_perm)
    if (st == PS_OK && ((!vm && (!J.keysB || !J.chunk_node)) || !J.inst || !J.chunk_map || !J.chunk_info ||
                        !J.range_agg || !J.range_entry || !J.run_grp_agg || !J.run_start || !J.power || !J.tiles || !J.gnodes ||
                        !J.gmap || !J.gsorted || !J.dep || !J.ctr || (!vm && cfg->want_perm && !J.permB) ||
                        (vm && (!J.pool_keys || !J.pt || !J.vm_split_at || !J.vm_rec || !J.free_stack || !J.vm_cta_count))))
        st = PS_EINTERNAL;
    if (st != PS_OK) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return st;
    }
    std::memset(c->h_ctr, 0, sizeof(ps::Ctr));
    *out = c;
    return PS_OK;
}

PS_API ps_status ps_run(ps_ctx* ctx, uint32_t* d_keys, uint32_t* d_perm, uint64_t n, ps_stats* stats)
{
    if (!ctx) return PS_EINVAL;
    if (n > ctx->cfg.max_n) return PS_EINVAL;
    if (n > 0 && !d_keys) return PS_EINVAL;
    if (d_perm && !ctx->cfg.want_perm) return PS_EINVAL;
    return run_common(ctx, d_keys, d_perm, nullptr, n, 1, stats);
}

PS_API ps_status ps_run_batched(ps_ctx* ctx, uint32_t* d_keys, uint32_t* d_perm, const uint64_t* d_offsets,
                                uint32_t count, ps_stats* stats)
{
    if (!ctx || !d_offsets) return PS_EINVAL;
    if (ctx->base.vm) return PS_EINVAL;          // VM storage sorts one instance per call
    if (count == 0 || count > ctx->max_count) return PS_EINVAL;
    if (!d_keys) return PS_EINVAL;
    if (d_perm && !ctx->cfg.want_perm) return PS_EINVAL;
    // the offsets table lives on the device and is checked there (k_setup)
    return run_common(ctx, d_keys, d_perm, d_offsets, 0, count, stats);
}

PS_API ps_status ps_run_host(ps_ctx* ctx, uint32_t* h_keys, uint32_t* h_perm, uint64_t n, ps_stats* stats)
{
    if (!ctx) return PS_EINVAL;
    if (!ctx->io_keys) return PS_EINVAL;
    if (n > ctx->cfg.max_n) return PS_EINVAL;
    if (n > 0 && !h_keys) return PS_EINVAL;
    if (h_perm && !ctx->cfg.want_perm) return PS_EINVAL;
    if (n == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return PS_OK;
    }
    DeviceGuard g(ctx->device);
    const size_t bytes = n * sizeof(uint32_t);
    if (cudaMemcpyAsync(ctx->io_keys, h_keys, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    ps_stats local;
    ps_status st = run_common(ctx, ctx->io_keys, h_perm ? ctx->io_perm : nullptr, nullptr, n, 1, nullptr);
    if (st != PS_OK) return st;
    if (cudaMemcpyAsync(h_keys, ctx->io_keys, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    if (h_perm && cudaMemcpyAsync(h_perm, ctx->io_perm, bytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    st = sync_and_check(ctx);
    if (st != PS_OK) return st;
    fill_stats(ctx, &local, 1);
    if (stats) *stats = local;
    return PS_OK;
}

PS_API ps_status ps_get_phase_times(ps_ctx* ctx, float* h_ms, uint32_t cap, uint32_t* count)
{
    if (!ctx || (!h_ms && cap)) return PS_EINVAL;
    if (!ctx->timing || !ctx->last_valid) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    if (cudaEventSynchronize(ctx->ev[NPHASES]) != cudaSuccess) return PS_ECUDA;
    if (count) *count = NPHASES;
    for (uint32_t i = 0; i < NPHASES && i < cap; ++i)
        if (cudaEventElapsedTime(&h_ms[i], ctx->ev[i], ctx->ev[i + 1]) != cudaSuccess) return PS_ECUDA;
    return PS_OK;
}

PS_API ps_status ps_get_round_times(ps_ctx* ctx, float* h_us, uint32_t cap, uint32_t* count)
{
    if (!ctx || (!h_us && cap)) return PS_EINVAL;
    if (!ctx->last_valid) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    ps_status st = sync_and_check(ctx);
    if (st != PS_OK) return st;
    const ps::Ctr* h = ctx->h_ctr;
    uint32_t k = 0;
    const unsigned long long t0 = h->merge_t0;
    for (int r = 0; r < ps::NPOW; ++r) {
        const unsigned long long* t = h->round_ns[r];
        if (h->bucket_start[r] == h->bucket_start[r + 1] || t[0] == ~0ull || t[2] == ~0ull) continue;
        for (int i = 0; i < 4; ++i, ++k)
            if (k < cap) h_us[k] = t[i] > t0 ? (float)(t[i] - t0) * 1e-3f : 0.0f;
    }
    if (count) *count = k;
    return PS_OK;
}

}  // extern "C"

struct ps_graph {
    ps_ctx* ctx;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    uint32_t count;
};

extern "C" {

PS_API ps_status ps_graph_create_batched(ps_ctx* ctx, uint32_t* d_keys, uint32_t* d_perm,
                                         const uint64_t* d_offsets, uint32_t count, ps_graph** out)
{
    if (!out) return PS_EINVAL;
    *out = nullptr;
    if (!ctx || !d_keys || !d_offsets || count == 0 || count > ctx->max_count) return PS_EINVAL;
    if (ctx->base.vm) return PS_EINVAL;          // VM storage sorts one instance per call
    if (d_perm && !ctx->cfg.want_perm) return PS_EINVAL;
    if (!ctx->stream) return PS_EINVAL;           // the legacy default stream cannot be captured
    DeviceGuard g(ctx->device);
    ps_graph* pg = new (std::nothrow) ps_graph();
    if (!pg) return PS_ENOMEM;
    pg->ctx = ctx;
    pg->count = count;
    if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        delete pg;
        return PS_ECUDA;
    }
    ctx->capturing = true;
    const ps_status st = run_common(ctx, d_keys, d_perm, d_offsets, 0, count, nullptr);
    ctx->capturing = false;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &pg->graph);
    if (st != PS_OK || e != cudaSuccess) {
        cudaGetLastError();
        if (e == cudaSuccess && pg->graph) cudaGraphDestroy(pg->graph);
        delete pg;
        ctx->last_valid = 0;
        return st != PS_OK ? st : PS_ECUDA;
    }
    if (cudaGraphInstantiate(&pg->exec, pg->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(pg->graph);
        delete pg;
        ctx->last_valid = 0;
        return PS_ECUDA;
    }
    ctx->last_valid = 0;                          // nothing ran yet
    *out = pg;
    return PS_OK;
}

PS_API ps_status ps_graph_launch(ps_graph* g)
{
    if (!g) return PS_EINVAL;
    DeviceGuard dg(g->ctx->device);
    if (cudaGraphLaunch(g->exec, g->ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return PS_ECUDA;
    }
    g->ctx->last_valid = 1;
    g->ctx->last_count = g->count;
    return PS_OK;
}

PS_API void ps_graph_destroy(ps_graph* g)
{
    if (!g) return;
    DeviceGuard dg(g->ctx->device);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
}

namespace {

// The record sort, enqueued (n >= 1, arguments checked by the caller).
ps_status records_async(ps_ctx* ctx, const uint32_t* d_rec, uint32_t words, uint64_t n, uint32_t* d_perm,
                        uint32_t* d_rec_out)
{
    cudaStream_t s = ctx->stream;
    ps::Ctr* C = ctx->base.ctr;
    const int grid = ctx->num_sms * 8;
    // the shared prefix starts at "every word", the group list empty
    if (cudaMemsetAsync(&C->rec_lcp, 0xff, sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(&C->rec_groups, 0, 3 * sizeof(uint32_t), s) != cudaSuccess)   // groups, nbig, gmax
        return PS_ECUDA;
    if (ps::launch_records_prepare(d_rec, words, n, ctx->rec_mask, ctx->rec_keys, C, grid, s) != cudaSuccess)
        return PS_ECUDA;
    // the 32-bit pipeline on the window keys, runs from the descent mask
    ctx->base.desc_mask = ctx->rec_mask;
    ps_status st = run_common(ctx, ctx->rec_keys, d_perm, nullptr, n, 1, nullptr);
    ctx->base.desc_mask = nullptr;
    if (st != PS_OK) return st;
    // packed fix-up words: rec_tmp and rec_rows (free until the row gather)
    const bool nested = words == 2 && ctx->rec_inner;
    if (ps::launch_records_fix(d_rec, words, n, ctx->rec_keys, d_perm, ctx->rec_tmp,
                               reinterpret_cast<unsigned long long*>(ctx->rec_tmp),
                               reinterpret_cast<unsigned long long*>(ctx->rec_rows), ctx->rec_groups,
                               ctx->rec_group_cap, ctx->rec_big, ctx->rec_big_cap, C, grid, ctx->grid_rec_big,
                               nested, s) != cudaSuccess)
        return PS_ECUDA;
    if (nested) {
        // the big groups' last words (rec_tmp[0, n)) sorted with their local
        // permutation (rec_tmp[n, 2n)); their entries kept in rec_rows
        uint32_t* keys2 = ctx->rec_tmp;
        uint32_t* perm2 = ctx->rec_tmp + ctx->cfg.max_n;
        if (ps::launch_records_nested_prep(d_rec, words, d_perm, ctx->rec_big, ctx->rec_big_cap, ctx->rec_off, keys2,
                                           ctx->rec_rows, C, grid, s) != cudaSuccess)
            return PS_ECUDA;
        if (ctx->rec_exec) {
            if (cudaGraphLaunch(ctx->rec_exec, s) != cudaSuccess) return PS_ECUDA;
        } else {
            // no graph: the inner sort on the caller's stream, whatever the count
            ctx->rec_inner->stream = s;
            st = ps_run_batched(ctx->rec_inner, keys2, perm2, reinterpret_cast<const uint64_t*>(ctx->rec_off),
                                ctx->rec_big_cap, nullptr);
            if (st != PS_OK) return st;
        }
        if (ps::launch_records_nested_apply(words, d_perm, ctx->rec_big, ctx->rec_big_cap, ctx->rec_off, perm2,
                                            ctx->rec_rows, C, ctx->rec_inner->base.ctr, grid, s) != cudaSuccess)
            return PS_ECUDA;
    }
    if (d_rec_out && ps::launch_gather_rows(d_perm, nullptr, 0, n, ctx->max_total, d_rec, d_rec_out, words * 4u, C,
                                            grid, s) != cudaSuccess)
        return PS_ECUDA;
    return PS_OK;
}

// After an enqueued record sort: surface its errors, and the statistics.
ps_status records_finish(ps_ctx* ctx, ps_stats* stats, uint32_t extra_launches, bool nested)
{
    if (cudaMemcpyAsync(&ctx->h_ctr->error, &ctx->base.ctr->error, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    if (!stats) return PS_OK;
    ps_status st = sync_and_check(ctx);
    if (st != PS_OK) return st;
    fill_stats(ctx, stats, 1);
    if (cudaMemcpy(ctx->h_inst, ctx->base.inst, sizeof(ps::Inst), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PS_ECUDA;
    stats->minrun = ctx->h_inst->minrun;
    // scan, window keys, groups, fix-up, and the big groups' merge passes
    // -- or, for two-word rows, their nested sort (offsets, gather, the
    // condition, apply, and the batched sort when a big group exists)
    uint32_t nested_launches = 0;
    if (nested) {
        uint32_t nbig = 0;
        if (cudaMemcpy(&nbig, &ctx->base.ctr->rec_nbig, sizeof(nbig), cudaMemcpyDeviceToHost) != cudaSuccess)
            return PS_ECUDA;
        nested_launches = (ctx->rec_exec ? 4u : 3u) + (nbig || !ctx->rec_exec ? LAUNCHES_PER_CALL : 0u);
    }
    stats->launches += 4u + (nested ? nested_launches : 1u) + extra_launches;
    return PS_OK;
}

bool records_ready(const ps_ctx* ctx)
{
    return ctx && ctx->rec_keys && ctx->cfg.want_perm && !ctx->base.desc_runs && ctx->base.key_type == PS_KEY_U32;
}

}  // namespace

PS_API ps_status ps_sort_records(ps_ctx* ctx, const uint32_t* d_rec, uint32_t words, uint64_t n,
                                 uint32_t* d_perm, uint32_t* d_rec_out, ps_stats* stats)
{
    if (!records_ready(ctx)) return PS_EINVAL;
    if (words == 0 || words > PS_RECORD_MAX_WORDS || n > ctx->cfg.max_n) return PS_EINVAL;
    if (n > 0 && (!d_rec || !d_perm)) return PS_EINVAL;
    if (n == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return PS_OK;
    }
    DeviceGuard g(ctx->device);
    ps_status st = records_async(ctx, d_rec, words, n, d_perm, d_rec_out);
    if (st != PS_OK) return st;
    return records_finish(ctx, stats, d_rec_out ? 1u : 0u, words == 2 && ctx->rec_inner);
}

PS_API ps_status ps_sort_keys64(ps_ctx* ctx, uint64_t* d_keys, uint64_t n, uint32_t* d_perm, uint32_t key_type,
                                ps_stats* stats)
{
    if (!records_ready(ctx) || key_type > PS_KEY_F32 || n > ctx->cfg.max_n) return PS_EINVAL;
    if (n > 0 && (!d_keys || !d_perm)) return PS_EINVAL;
    if (n == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return PS_OK;
    }
    DeviceGuard g(ctx->device);
    const int grid = ctx->num_sms * 8;
    // keys -> order-preserving (high, low) rows in place; sort the rows into
    // rec_rows; back to keys in order
    if (ps::launch_key64(true, nullptr, d_keys, n, key_type, grid, ctx->stream) != cudaSuccess) return PS_ECUDA;
    ps_status st = records_async(ctx, reinterpret_cast<const uint32_t*>(d_keys), 2, n, d_perm, ctx->rec_rows);
    if (st != PS_OK) return st;
    if (ps::launch_key64(false, ctx->rec_rows, d_keys, n, key_type, grid, ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    return records_finish(ctx, stats, 3u, ctx->rec_inner != nullptr);   // the row gather and the two maps
}

PS_API ps_status ps_gather_rows(ps_ctx* ctx, const uint32_t* d_perm, const uint64_t* d_offsets, uint32_t count,
                                uint64_t n, const void* d_src, void* d_dst, uint32_t row_bytes)
{
    if (!ctx || row_bytes == 0) return PS_EINVAL;
    if (d_offsets ? count == 0 : n > ctx->max_total) return PS_EINVAL;
    if (!d_offsets && n == 0) return PS_OK;
    if (!d_perm || !d_src || !d_dst) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    const int grid = ctx->num_sms * 8;
    if (ps::launch_gather_rows(d_perm, reinterpret_cast<const unsigned long long*>(d_offsets), count, n,
                               ctx->max_total, d_src, d_dst, row_bytes, ctx->base.ctr, grid, ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    // a bad row surfaces at the next synchronising call, as a sort's would
    if (cudaMemcpyAsync(&ctx->h_ctr->error, &ctx->base.ctr->error, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess)
        return PS_ECUDA;
    return PS_OK;
}

PS_API ps_status ps_check_guards(ps_ctx* ctx)
{
    if (!ctx) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return PS_ECUDA;
    }
    unsigned char h[GUARD_BYTES];
    for (unsigned char* d : ctx->guards) {
        if (cudaMemcpy(h, d, GUARD_BYTES, cudaMemcpyDeviceToHost) != cudaSuccess) return PS_ECUDA;
        for (size_t i = 0; i < GUARD_BYTES; ++i)
            if (h[i] != GUARD_BYTE) return PS_EINTERNAL;
    }
    // the context a record sort keeps for its nested sort
    return ctx->rec_inner ? ps_check_guards(ctx->rec_inner) : PS_OK;
}

PS_API ps_status ps_selftest_wait_timeout(ps_ctx* ctx)
{
    if (!ctx) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    ps::Ctr* C = ctx->base.ctr;
    cudaStream_t s = ctx->stream;
    // a clean status and barrier, the probe, then the barrier counters reset
    // (a CTA that never arrived leaves its group's count behind)
    if (cudaMemsetAsync(&C->error, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) return PS_ECUDA;   // error, err_where
    if (ps::launch_wait_probe(C, s) != cudaSuccess) return PS_ECUDA;
    if (cudaMemcpyAsync(&ctx->h_ctr->error, &C->error, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PS_ECUDA;
    if (cudaMemsetAsync(&C->bar_count, 0, sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(C->bar_group, 0, sizeof(C->bar_group), s) != cudaSuccess)
        return PS_ECUDA;
    return sync_and_check(ctx);
}

PS_API ps_status ps_sync(ps_ctx* ctx)
{
    if (!ctx) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    return sync_and_check(ctx);
}

PS_API ps_status ps_get_runs(ps_ctx* ctx, uint32_t q, uint32_t* h_out, uint64_t cap, uint64_t* count)
{
    if (!ctx || (!h_out && cap)) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    ps::Inst I;
    ps_status st = read_inst(ctx, q, &I);
    if (st != PS_OK) return st;
    const uint64_t avail = I.n ? (uint64_t)I.runs + 1 : 1;
    if (count) *count = avail;
    const uint64_t k = avail < cap ? avail : cap;
    if (k && cudaMemcpy(h_out, ctx->base.run_start + I.run_base, k * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
                 cudaSuccess)
        return PS_ECUDA;
    return PS_OK;
}

PS_API ps_status ps_get_powers(ps_ctx* ctx, uint32_t q, uint8_t* h_out, uint64_t cap, uint64_t* count)
{
    if (!ctx || (!h_out && cap)) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    ps::Inst I;
    ps_status st = read_inst(ctx, q, &I);
    if (st != PS_OK) return st;
    const uint64_t avail = I.runs >= 2 ? (uint64_t)I.runs - 1 : 0;
    if (count) *count = avail;
    const uint64_t k = avail < cap ? avail : cap;
    if (k && cudaMemcpy(h_out, ctx->base.power + I.run_base + 1, k, cudaMemcpyDeviceToHost) != cudaSuccess)
        return PS_ECUDA;
    return PS_OK;
}

PS_API ps_status ps_get_nodes(ps_ctx* ctx, uint32_t q, uint32_t* h_out, uint64_t cap, uint64_t* count)
{
    if (!ctx || (!h_out && cap)) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    ps::Inst I;
    ps_status st = read_inst(ctx, q, &I);
    if (st != PS_OK) return st;
    const uint64_t nbound = I.runs >= 2 ? (uint64_t)I.runs - 1 : 0;
    if (count) *count = 2 * nbound;
    if (!nbound || !cap) return PS_OK;
    // the ranges are not kept after the call (the sort needs them only for
    // its HBM merges): the planning's node_range recomputes them for every
    // boundary from the run starts, into a buffer of this call
    uint32_t* d = nullptr;
    if (cudaMalloc(&d, 2 * nbound * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return PS_ENOMEM;
    }
    ps_status rc = PS_OK;
    if (ps::launch_node_ranges(ctx->base, q, (uint32_t)nbound, d, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        rc = PS_ECUDA;
    const uint64_t k = 2 * nbound < cap ? 2 * nbound : cap;
    if (rc == PS_OK && cudaMemcpy(h_out, d, k * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess) rc = PS_ECUDA;
    cudaFree(d);
    if (rc != PS_OK) cudaGetLastError();
    return rc;
}

PS_API ps_status ps_get_instance_stats(ps_ctx* ctx, uint32_t q, ps_stats* stats)
{
    if (!ctx || !stats) return PS_EINVAL;
    DeviceGuard g(ctx->device);
    ps::Inst I;
    ps_status st = read_inst(ctx, q, &I);
    if (st != PS_OK) return st;
    std::memset(stats, 0, sizeof(*stats));
    stats->n = I.n;
    stats->runs = I.runs;
    stats->merge_cost = I.M;
    stats->max_power = I.max_power;
    stats->minrun = I.minrun;
    stats->instances = 1;
    stats->scratch_bytes = ctx->scratch_bytes;
    return PS_OK;
}

PS_API ps_status ps_get_scratch_bytes(const ps_ctx* ctx, uint64_t* bytes)
{
    if (!ctx || !bytes) return PS_EINVAL;
    *bytes = ctx->scratch_bytes;
    return PS_OK;
}

PS_API void ps_destroy(ps_ctx* ctx)
{
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        free_all(ctx);
    }
    delete ctx;
}

}  // extern "C"
