// Serving: a request loop that sorts independent host arrays on the GPU with
// continuous batching under a device-memory budget.
//
// The server owns `lanes` lanes; a lane is a batched Powersort context with
// its own CUDA stream, device input/output arrays and offsets table, sized so
// that all lanes together stay within the budget.  With VM storage a lane's
// context is a paged one (a page pool and tables instead of an n-element
// scratch buffer) and the lane sorts its batch's requests one after another.  A dispatcher thread keeps
// every idle lane busy: it takes queued requests in arrival order while they
// fit the lane (elements and count), enqueues their host->device copies, one
// ps_run_batched over the batch and the device->host copies of the sorted
// keys and permutations, and records an event.  Lanes run concurrently, so a
// request arriving while other batches are on the GPU is admitted as soon as
// a lane frees up, and its work overlaps theirs: one batch's host->device
// copies and another's device->host copies run on the copy engines while a
// third batch computes.  The batches' kernels themselves run one batch after
// the other, in dispatch order (each batch's sort waits for the previous
// batch's sort): a batch's kernels fill the GPU, and a small batch whose
// dependent kernels interleaved with a large batch's would wait behind one
// of its long kernels at almost every step.  A ticket completes when its
// lane's event has fired; its latency is measured from submission.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ps_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState : int { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3 };

struct Req {
    const uint32_t* in;
    uint32_t* kout;
    uint32_t* pout;
    uint64_t n;
    Clock::time_point t_submit;
    double latency_s;
    int state;
    ps_status status;
};

struct Lane {
    ps_ctx* ctx = nullptr;
    ps_ctx* ctx_small = nullptr;    // VM storage: batches of small requests (Pingpong)
    cudaStream_t stream = nullptr;
    uint32_t* dkeys = nullptr;
    uint32_t* dperm = nullptr;
    uint64_t* doff = nullptr;
    uint64_t* hoff = nullptr;       // pinned
    cudaEvent_t done = nullptr;
    cudaEvent_t computed = nullptr; // the batch's sort has finished (its copies out may still run)
    std::vector<uint64_t> batch;    // tickets in flight
    std::vector<Req> jobs;          // their arrays, copied under the lock
    uint64_t small_max = 0, small_total = 0;   // VM storage: the small context's limits
    bool busy = false;
    bool signalled = false;         // the stream reached the batch's end (host callback, under the lock)
    struct ps_server* owner = nullptr;
    // tracing (PS_SERVER_TRACE): timing events of the batch in flight -- its
    // first copy in, copies in done, sort start, sort end, copies out done --
    // and the host times it was enqueued
    cudaEvent_t tev[5] = {};
    double t_enq0 = 0.0, t_enq1 = 0.0;
};

// One traced batch: host times in seconds and device times in milliseconds,
// both since the server started.
struct TraceRow {
    uint32_t lane, requests;
    uint64_t elements;
    double t_enq0, t_enq1, t_seen;
    float gpu[5];
};

// Only for choosing a lane size when the caller gives none: lane arrays
// (keys + permutation) plus a Pingpong context's scratch and tables, per
// element.  What the lanes are charged is measured (lane_bytes below).
constexpr double BYTES_PER_ELEM_ESTIMATE = 18.0;
constexpr double BYTES_PER_ELEM_ESTIMATE_VM = 9.0;   // arrays + a page pool and tables
// VM storage: a request of at most SMALL_MAX elements joins a batch of small
// requests (at most SMALL_TOTAL elements) sorted by the lane's small Pingpong
// context; a larger one is a batch by itself, sorted with paged storage.
constexpr uint64_t SMALL_MAX = 1ull << 20, SMALL_TOTAL = 1ull << 22;

}  // namespace

struct ps_server {
    ps_server_config cfg;
    uint64_t lane_total = 0;
    uint32_t lane_count = 0;
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::vector<Req> reqs;
    std::thread th;
    bool stop = false;
    uint64_t bytes = 0;
    uint64_t completed = 0, elements = 0, batches = 0, failed = 0;
    uint32_t max_in_flight_lanes = 0;
    cudaEvent_t last_computed = nullptr;   // the sort of the batch dispatched last (dispatcher only)
    // tracing: on when PS_SERVER_TRACE names a file, written at destroy
    std::string trace_path;
    cudaEvent_t trace_t0 = nullptr;
    Clock::time_point t_start;
    std::vector<TraceRow> trace;
};

namespace {

// Host function enqueued after a batch's last copy: wakes the dispatcher
// instead of having it poll the lanes' events.  It calls no CUDA function.
void CUDART_CB on_batch_end(void* arg)
{
    Lane* L = static_cast<Lane*>(arg);
    ps_server* S = L->owner;
    std::lock_guard<std::mutex> lk(S->mu);
    L->signalled = true;
    S->cv_work.notify_one();
}

void lane_free(Lane& L)
{
    if (L.ctx) ps_destroy(L.ctx);
    if (L.ctx_small) ps_destroy(L.ctx_small);
    if (L.dkeys) cudaFree(L.dkeys);
    if (L.dperm) cudaFree(L.dperm);
    if (L.doff) cudaFree(L.doff);
    if (L.hoff) cudaFreeHost(L.hoff);
    if (L.done) cudaEventDestroy(L.done);
    if (L.computed) cudaEventDestroy(L.computed);
    for (cudaEvent_t& e : L.tev)
        if (e) cudaEventDestroy(e);
    if (L.stream) cudaStreamDestroy(L.stream);
    L = Lane{};
}

// Enqueue one batch on a lane (no lock held; the tickets are RUNNING).
ps_status launch_batch(ps_server* S, Lane& L)
{
    const size_t k = L.jobs.size();
    const bool tr = S->trace_t0 != nullptr;
    if (tr) {
        L.t_enq0 = std::chrono::duration<double>(Clock::now() - S->t_start).count();
        if (cudaEventRecord(L.tev[0], L.stream) != cudaSuccess) return PS_ECUDA;
    }
    uint64_t acc = 0;
    L.hoff[0] = 0;
    for (size_t i = 0; i < k; ++i) {
        acc += L.jobs[i].n;
        L.hoff[i + 1] = acc;
    }
    if (cudaMemcpyAsync(L.doff, L.hoff, (k + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, L.stream) != cudaSuccess)
        return PS_ECUDA;
    for (size_t i = 0; i < k; ++i) {
        const Req& r = L.jobs[i];
        if (r.n && cudaMemcpyAsync(L.dkeys + L.hoff[i], r.in, r.n * 4, cudaMemcpyHostToDevice, L.stream) != cudaSuccess)
            return PS_ECUDA;
    }
    if (tr && cudaEventRecord(L.tev[1], L.stream) != cudaSuccess) return PS_ECUDA;
    // the sort starts after the previous batch's sort (copies in are not held back)
    if (S->last_computed && cudaStreamWaitEvent(L.stream, S->last_computed, 0) != cudaSuccess) return PS_ECUDA;
    if (tr && cudaEventRecord(L.tev[2], L.stream) != cudaSuccess) return PS_ECUDA;
    if (S->cfg.storage == PS_MODE_VM && (k != 1 || L.jobs[0].n <= L.small_max)) {
        // a batch of small requests: the small Pingpong context
        const ps_status st =
            ps_run_batched(L.ctx_small, L.dkeys, S->cfg.want_perm ? L.dperm : nullptr, L.doff, (uint32_t)k, nullptr);
        if (st != PS_OK) return st;
    } else if (S->cfg.storage == PS_MODE_VM) {
        // a large request by itself, with paged storage
        const ps_status st = ps_run(L.ctx, L.dkeys, S->cfg.want_perm ? L.dperm : nullptr, L.jobs[0].n, nullptr);
        if (st != PS_OK) return st;
    } else {
        const ps_status st =
            ps_run_batched(L.ctx, L.dkeys, S->cfg.want_perm ? L.dperm : nullptr, L.doff, (uint32_t)k, nullptr);
        if (st != PS_OK) return st;
    }
    if (cudaEventRecord(L.computed, L.stream) != cudaSuccess) return PS_ECUDA;
    if (tr && cudaEventRecord(L.tev[3], L.stream) != cudaSuccess) return PS_ECUDA;
    S->last_computed = L.computed;
    for (size_t i = 0; i < k; ++i) {
        const Req& r = L.jobs[i];
        if (!r.n) continue;
        if (cudaMemcpyAsync(r.kout, L.dkeys + L.hoff[i], r.n * 4, cudaMemcpyDeviceToHost, L.stream) != cudaSuccess)
            return PS_ECUDA;
        if (r.pout && S->cfg.want_perm &&
            cudaMemcpyAsync(r.pout, L.dperm + L.hoff[i], r.n * 4, cudaMemcpyDeviceToHost, L.stream) != cudaSuccess)
            return PS_ECUDA;
    }
    if (cudaEventRecord(L.done, L.stream) != cudaSuccess) return PS_ECUDA;
    if (tr && cudaEventRecord(L.tev[4], L.stream) != cudaSuccess) return PS_ECUDA;
    if (cudaLaunchHostFunc(L.stream, on_batch_end, &L) != cudaSuccess) return PS_ECUDA;
    if (tr) L.t_enq1 = std::chrono::duration<double>(Clock::now() - S->t_start).count();
    return PS_OK;
}

// A completed batch's trace row (dispatcher, lock held; the events are done).
void trace_batch(ps_server* S, Lane& L, uint32_t lane)
{
    TraceRow row;
    row.lane = lane;
    row.requests = (uint32_t)L.jobs.size();
    row.elements = 0;
    for (const Req& r : L.jobs) row.elements += r.n;
    row.t_enq0 = L.t_enq0;
    row.t_enq1 = L.t_enq1;
    row.t_seen = std::chrono::duration<double>(Clock::now() - S->t_start).count();
    for (int i = 0; i < 5; ++i)
        if (cudaEventElapsedTime(&row.gpu[i], S->trace_t0, L.tev[i]) != cudaSuccess) row.gpu[i] = -1.0f;
    cudaGetLastError();
    S->trace.push_back(row);
}

void trace_write(const ps_server* S)
{
    FILE* f = std::fopen(S->trace_path.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "lane,requests,elements,host_enqueue_begin_s,host_enqueue_end_s,host_seen_s,"
                    "gpu_first_copy_in_ms,gpu_copies_in_done_ms,gpu_sort_start_ms,gpu_sort_end_ms,gpu_copies_out_done_ms\n");
    for (const TraceRow& r : S->trace)
        std::fprintf(f, "%u,%u,%llu,%.6f,%.6f,%.6f,%.4f,%.4f,%.4f,%.4f,%.4f\n", r.lane, r.requests,
                     (unsigned long long)r.elements, r.t_enq0, r.t_enq1, r.t_seen, r.gpu[0], r.gpu[1], r.gpu[2],
                     r.gpu[3], r.gpu[4]);
    std::fclose(f);
}

void dispatcher(ps_server* S)
{
    cudaSetDevice((int)S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        // completions
        for (Lane& L : S->lanes) {
            if (!L.busy || !L.signalled) continue;
            L.signalled = false;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) continue;
            ps_status st = q == cudaSuccess ? PS_OK : PS_ECUDA;
            if (st == PS_OK) {
                lk.unlock();
                st = ps_sync(L.ctx);            // device-side status of the batch
                lk.lock();
            } else {
                cudaGetLastError();
            }
            if (st == PS_OK && S->trace_t0) trace_batch(S, L, (uint32_t)(&L - &S->lanes[0]));
            const auto now = Clock::now();
            for (uint64_t t : L.batch) {
                Req& r = S->reqs[t];
                r.latency_s = std::chrono::duration<double>(now - r.t_submit).count();
                r.state = st == PS_OK ? DONE : FAILED;
                r.status = st;
                if (st == PS_OK) {
                    ++S->completed;
                    S->elements += r.n;
                } else {
                    ++S->failed;
                }
            }
            L.batch.clear();
            L.jobs.clear();
            L.busy = false;
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // admissions: fill idle lanes from the queue head (arrival order)
        for (Lane& L : S->lanes) {
            if (L.busy || S->queue.empty()) continue;
            uint64_t total = 0;
            const bool vm = S->cfg.storage == PS_MODE_VM;
            while (!S->queue.empty() && L.batch.size() < S->lane_count) {
                const uint64_t t = S->queue.front();
                const uint64_t n = S->reqs[t].n;
                if (total + n > S->lane_total && !L.batch.empty()) break;
                // VM storage: small requests batch together (within the small
                // context's total); a large one goes alone
                if (vm && !L.batch.empty() &&
                    (n > L.small_max || S->reqs[L.batch[0]].n > L.small_max || total + n > L.small_total))
                    break;
                S->queue.pop_front();
                S->reqs[t].state = RUNNING;
                L.batch.push_back(t);
                L.jobs.push_back(S->reqs[t]);
                total += n;
            }
            if (L.batch.empty()) continue;
            L.busy = true;
            ++S->batches;
            lk.unlock();
            const ps_status st = launch_batch(S, L);
            lk.lock();
            if (st != PS_OK) {             // nothing in flight: fail the batch now
                cudaStreamSynchronize(L.stream);
                cudaGetLastError();
                for (uint64_t t : L.batch) {
                    S->reqs[t].state = FAILED;
                    S->reqs[t].status = st;
                    ++S->failed;
                }
                L.batch.clear();
                L.jobs.clear();
                L.busy = false;
                S->cv_done.notify_all();
            }
            progress = true;
        }
        uint32_t busy = 0;
        for (const Lane& L : S->lanes) busy += L.busy ? 1u : 0u;
        if (busy > S->max_in_flight_lanes) S->max_in_flight_lanes = busy;
        if (S->stop && S->queue.empty() && busy == 0) break;
        if (!progress) {
            // nothing changed: sleep until a submission or a batch's end wakes
            // the dispatcher (the timeout only bounds a missed wake-up)
            S->cv_work.wait_for(lk, std::chrono::milliseconds(busy ? 5 : 50));
        }
    }
}

}  // namespace

extern "C" {

PS_API ps_status ps_server_create(const ps_server_config* cfg, ps_server** out)
{
    if (!out) return PS_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->max_n == 0 || cfg->max_n > 0xffffffffull || cfg->budget_bytes == 0) return PS_EINVAL;
    if (cfg->storage != PS_MODE_PINGPONG && cfg->storage != PS_MODE_VM) return PS_EINVAL;
    ps_server* S = new (std::nothrow) ps_server();
    if (!S) return PS_ENOMEM;
    S->cfg = *cfg;
    if (!S->cfg.lanes) S->cfg.lanes = 4;
    S->lane_count = S->cfg.lane_max_count ? S->cfg.lane_max_count : 1024;
    uint64_t lane_total = S->cfg.lane_max_total;
    if (!lane_total) {
        const double per_elem = S->cfg.storage == PS_MODE_VM ? BYTES_PER_ELEM_ESTIMATE_VM : BYTES_PER_ELEM_ESTIMATE;
        lane_total = (uint64_t)((double)S->cfg.budget_bytes / S->cfg.lanes / per_elem);
        if (lane_total > (1ull << 28)) lane_total = 1ull << 28;
    }
    if (lane_total < S->cfg.max_n) lane_total = S->cfg.max_n;
    S->lane_total = lane_total;
    // the lane arrays alone must fit before anything is allocated
    const double arrays = (double)lane_total * 4.0 * (S->cfg.want_perm ? 2.0 : 1.0) * S->cfg.lanes;
    if (arrays > (double)S->cfg.budget_bytes) {
        delete S;
        return PS_ENOMEM;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice((int)S->cfg.device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return PS_ECUDA;
    }
    ps_status st = PS_OK;
    S->lanes.resize(S->cfg.lanes);
    for (Lane& L : S->lanes) {
        L.owner = S;
        bool ev_ok = true;
        if (std::getenv("PS_SERVER_TRACE"))
            for (cudaEvent_t& e : L.tev) ev_ok = ev_ok && cudaEventCreate(&e) == cudaSuccess;
        if (!ev_ok || cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.computed, cudaEventDisableTiming) != cudaSuccess) {
            st = PS_ECUDA;
            break;
        }
        if (cudaMalloc(&L.dkeys, lane_total * 4) != cudaSuccess ||
            (S->cfg.want_perm && cudaMalloc(&L.dperm, lane_total * 4) != cudaSuccess) ||
            cudaMalloc(&L.doff, (S->lane_count + 1) * sizeof(uint64_t)) != cudaSuccess ||
            cudaMallocHost(&L.hoff, (S->lane_count + 1) * sizeof(uint64_t)) != cudaSuccess) {
            st = PS_ENOMEM;
            break;
        }
        ps_config c;
        std::memset(&c, 0, sizeof(c));
        c.mode = S->cfg.storage;
        c.want_perm = S->cfg.want_perm;
        c.key_type = S->cfg.key_type;
        c.flags = S->cfg.flags & PS_FLAG_DESCENDING_RUNS;
        c.max_n = S->cfg.max_n;
        c.max_total = S->cfg.storage == PS_MODE_VM ? S->cfg.max_n : lane_total;   // VM: one request per call
        c.max_count = S->cfg.storage == PS_MODE_VM ? 1u : S->lane_count;
        st = ps_create(&c, (int)S->cfg.device, L.stream, &L.ctx);
        if (st != PS_OK) break;
        uint64_t scratch = 0;
        st = ps_get_scratch_bytes(L.ctx, &scratch);
        if (st != PS_OK) break;
        if (S->cfg.storage == PS_MODE_VM) {
            L.small_max = std::min<uint64_t>(SMALL_MAX, S->cfg.max_n);
            L.small_total = std::min<uint64_t>(SMALL_TOTAL, lane_total);
            ps_config cs = c;
            cs.mode = PS_MODE_PINGPONG;
            cs.max_n = L.small_max;
            cs.max_total = L.small_total;
            cs.max_count = S->lane_count;
            st = ps_create(&cs, (int)S->cfg.device, L.stream, &L.ctx_small);
            if (st != PS_OK) break;
            uint64_t small = 0;
            st = ps_get_scratch_bytes(L.ctx_small, &small);
            if (st != PS_OK) break;
            scratch += small;
        }
        // what this lane holds: its arrays, its offsets table and its context
        S->bytes += lane_total * 4 * (S->cfg.want_perm ? 2 : 1) + (S->lane_count + 1) * sizeof(uint64_t) + scratch;
        if (S->bytes > S->cfg.budget_bytes) {   // stop as soon as the lanes overrun the budget
            st = PS_ENOMEM;
            break;
        }
    }
    if (st == PS_OK && S->bytes > S->cfg.budget_bytes) st = PS_ENOMEM;
    if (st != PS_OK) {
        cudaGetLastError();
        for (Lane& L : S->lanes) lane_free(L);
        if (prev >= 0) cudaSetDevice(prev);
        delete S;
        return st;
    }
    S->reqs.reserve(1 << 16);
    S->t_start = Clock::now();
    if (const char* tp = std::getenv("PS_SERVER_TRACE")) {
        if (*tp && cudaEventCreate(&S->trace_t0) == cudaSuccess &&
            cudaEventRecord(S->trace_t0, S->lanes[0].stream) == cudaSuccess) {
            S->trace_path = tp;
            S->trace.reserve(1 << 16);
        } else {
            cudaGetLastError();
            if (S->trace_t0) cudaEventDestroy(S->trace_t0);
            S->trace_t0 = nullptr;
        }
    }
    S->th = std::thread(dispatcher, S);
    if (prev >= 0) cudaSetDevice(prev);
    *out = S;
    return PS_OK;
}

PS_API ps_status ps_server_submit(ps_server* S, const uint32_t* h_in, uint32_t* h_keys_out, uint32_t* h_perm_out,
                                  uint64_t n, uint64_t* ticket)
{
    if (!S || !ticket || (n && (!h_in || !h_keys_out))) return PS_EINVAL;
    if (n > S->cfg.max_n) return PS_EINVAL;
    if (h_perm_out && !S->cfg.want_perm) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return PS_EINVAL;
    Req r;
    r.in = h_in;
    r.kout = h_keys_out;
    r.pout = h_perm_out;
    r.n = n;
    r.t_submit = Clock::now();
    r.latency_s = 0.0;
    r.state = QUEUED;
    r.status = PS_OK;
    *ticket = S->reqs.size();
    S->reqs.push_back(r);
    S->queue.push_back(*ticket);
    S->cv_work.notify_one();
    return PS_OK;
}

PS_API ps_status ps_server_cancel(ps_server* S, uint64_t ticket)
{
    if (!S) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (ticket >= S->reqs.size() || S->reqs[ticket].state != QUEUED) return PS_EINVAL;
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        if (*it == ticket) {
            S->queue.erase(it);
            break;
        }
    }
    Req& r = S->reqs[ticket];
    r.state = FAILED;
    r.status = PS_ECANCELED;
    r.latency_s = std::chrono::duration<double>(Clock::now() - r.t_submit).count();
    ++S->failed;
    S->cv_done.notify_all();
    return PS_OK;
}

PS_API ps_status ps_server_poll(ps_server* S, uint64_t ticket, int* done, double* latency_s)
{
    if (!S || !done) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (ticket >= S->reqs.size()) return PS_EINVAL;
    const Req& r = S->reqs[ticket];
    *done = r.state == DONE || r.state == FAILED;
    if (latency_s) *latency_s = r.latency_s;
    return r.state == FAILED ? r.status : PS_OK;
}

PS_API ps_status ps_server_wait(ps_server* S, uint64_t ticket, double timeout_s, double* latency_s)
{
    if (!S) return PS_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket >= S->reqs.size()) return PS_EINVAL;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (S->reqs[ticket].state != DONE && S->reqs[ticket].state != FAILED) {
        if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
            S->reqs[ticket].state != DONE && S->reqs[ticket].state != FAILED)
            return PS_ETIMEOUT;
    }
    if (latency_s) *latency_s = S->reqs[ticket].latency_s;
    return S->reqs[ticket].state == FAILED ? S->reqs[ticket].status : PS_OK;
}

PS_API ps_status ps_server_get_stats(ps_server* S, ps_server_stats* st)
{
    if (!S || !st) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->reqs.size();
    st->completed = S->completed;
    st->failed = S->failed;
    st->elements = S->elements;
    st->batches = S->batches;
    st->queued = S->queue.size();
    st->device_bytes = S->bytes;
    st->lane_max_total = S->lane_total;
    st->lanes = (uint32_t)S->lanes.size();
    st->max_busy_lanes = S->max_in_flight_lanes;
    return PS_OK;
}

PS_API void ps_server_destroy(ps_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice((int)S->cfg.device);
    for (Lane& L : S->lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    if (S->trace_t0) {
        trace_write(S);
        cudaEventDestroy(S->trace_t0);
    }
    for (Lane& L : S->lanes) lane_free(L);
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
