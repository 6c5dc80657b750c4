// Run detection with the minimum-run-length rule (ExtractRun, Sec. 2;
// minrun rule, Sec. 5 "Algorithm variants") for a batch of instances.
//
// Sequentially, the run starts are the orbit of 0 under
//     f(s) = max(d(s), min(s + minrun, n)),
// d(s) = the first descent position e > s (a[e-1] > a[e]) or n.  A natural
// run of at least minrun elements keeps its end d(s); a shorter one is forced
// to min(s + minrun, n) elements (the insertion sort of the forced run is done
// later, on chip, by the tile kernel -- it does not move any run boundary).
//
// Parallel form.  The instance is cut into chunks of RUN_CHUNK elements.  The
// first run start at or after a chunk's begin B can only be
//     B + delta (0 <= delta < minrun)        -- a forced step landed there, or
//     D0 = the first descent at or after B   -- a natural step ended there,
// so a chunk has at most minrun + 1 <= 64 entry states.  Each chunk walks the
// chain from every entry state (one lane per state) over its descent bitmask,
// which gives a map  entry state -> (exit state of the next chunk, runs
// started in this chunk).  A decoupled look-back composes the maps of the
// predecessors (chunks are claimed in order through an atomic ticket, so a
// predecessor is always resident or finished) to find the real entry state
// and the number of runs before the chunk; the chunk then writes its run
// starts.  The descent bitmask reaches RUN_HALO positions past the chunk, so a
// forced step from inside the chunk (length <= 63) is always decided locally;
// a natural run that runs past the halo ends at the next chunk's D0, which is
// one of that chunk's entry states.
#include "ps_internal.cuh"

namespace ps {

namespace {

constexpr uint32_t FULL = 0xffffffffu;

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_sums, T& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    T before = warp ? warp_sums[warp - 1] : T(0);
    total = warp_sums[nwarps - 1];
    __syncthreads();
    return before + x - v;
}

// Sec. 5: l = n; while l >= 64: l = ceil(l / 2).
__device__ __forceinline__ uint32_t minrun_of(uint32_t n)
{
    uint32_t l = n;
    while (l >= 64) l = (l + 1) >> 1;
    return l;
}

}  // namespace

// One CTA: per-instance sizes, minrun, chunk bases and run-slot bases
// (exclusive scans), counters reset.  Instances with n < 64 are one run
// (minrun = n) and need no chunk: their run list is written here.
__global__ void __launch_bounds__(1024) k_setup(Job J)
{
    __shared__ unsigned long long ws64[32];
    __shared__ uint32_t ws32[32];
    __shared__ unsigned long long carry_slots;
    __shared__ uint32_t carry_chunks;
    Ctr* C = J.ctr;
    __shared__ uint32_t s_bad;
    if (threadIdx.x == 0) {
        carry_slots = 0;
        carry_chunks = 0;
        s_bad = 0;
        C->error = 0;
        C->err_where = 0;
        C->epoch = (C->epoch + 1) & 0x3fffffffu;          // never 0: fresh words read "not ready"
        if (C->epoch == 0) C->epoch = 1;
        C->chunk_ticket = 0;
        C->n_tiles = 0;
        C->n_gnodes = 0;
        C->rounds = 0;
        C->bar_count = 0;
        C->max_power = 0;
        C->leaf_moves = 0;
        C->M_total = 0;
        C->runs_total = 0;
        C->n_total = 0;
        C->hbm_elems = 0;
        C->merge_t0 = 0;
    }
    if (threadIdx.x < 32) C->bar_group[threadIdx.x] = 0;
    for (int r = threadIdx.x; r < NPOW + 2; r += blockDim.x) {
        if (r < NPOW) {
            C->round_ns[r][0] = C->round_ns[r][2] = ~0ull;   // minima
            C->round_ns[r][1] = C->round_ns[r][3] = 0;       // maxima
            C->chunk_next[r] = 0;
        }
        if (r < NPOW + 1) {
            C->bucket_count[r] = 0;
            C->bucket_nchunk[r] = 0;
            C->bucket_cursor[r] = 0;
        }
        C->bucket_start[r] = 0;
        C->bucket_chunk[r] = 0;
    }
    __syncthreads();
    for (uint32_t base = 0; base < J.count; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < J.count;
        unsigned long long off = 0, n64 = 0;
        if (valid) {
            if (J.offsets) {
                off = J.offsets[i];
                const unsigned long long end = J.offsets[i + 1];
                // the table must start at 0, never decrease and respect the limits
                if ((i == 0 && off != 0) || end < off || end - off > J.max_n || end > J.max_total) {
                    atomicOr(&s_bad, 1u);
                    n64 = 0;
                } else {
                    n64 = end - off;
                }
            } else {
                n64 = J.single_n;
            }
        }
        const uint32_t n = (uint32_t)n64;
        const uint32_t nchunks = (valid && n >= 64) ? (n + RUN_CHUNK - 1) / RUN_CHUNK : 0u;
        const unsigned long long cap = valid ? (unsigned long long)(n / 32) + 2ull : 0ull;
        uint32_t tot_c;
        unsigned long long tot_s;
        const uint32_t cb = block_exclusive_scan<uint32_t>(nchunks, ws32, tot_c);
        const unsigned long long sb = block_exclusive_scan<unsigned long long>(cap, ws64, tot_s);
        if (valid) {
            Inst I;
            I.off = off;
            I.run_base = carry_slots + sb;
            I.M = 0;
            I.n = n;
            I.minrun = minrun_of(n);
            I.chunk_base = carry_chunks + cb;
            I.nchunks = nchunks;
            I.max_power = 0;
            I.runs = n == 0 ? 0u : (n < 64 ? 1u : 0u);
            J.inst[i] = I;
            if (n < 64 && I.run_base + 1 < J.slot_cap) {   // one run [0, n) (or none)
                J.run_start[I.run_base] = 0;
                if (n) J.run_start[I.run_base + 1] = n;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_chunks += tot_c;
            carry_slots += tot_s;
        }
        __syncthreads();
    }
    if (J.vm) {
        // virtual-memory storage: every virtual page starts as its own array page,
        // the free stack holds the pool pages
        const uint32_t na = J.single_n ? (uint32_t)((J.single_n + (1ull << J.vm_plog2) - 1) >> J.vm_plog2) : 0u;
        for (uint32_t u = threadIdx.x; u < J.vm_na_cap; u += blockDim.x) {
            J.pt[u] = u;
            J.page_cnt[u] = 0;
            J.consumed[u] = 0;
        }
        for (uint32_t i = threadIdx.x; i < J.vm_pool; i += blockDim.x) J.free_stack[i] = J.vm_na_cap + i;
        if (threadIdx.x == 0) {
            C->vm_free_top = J.vm_pool;
            C->vm_touched = 0;
            C->vm_wave = 0;
            C->vm_in_use_peak = 0;
            C->vm_waves = 0;
            C->vm_copy_moves = 0;
            if (na > J.vm_na_cap) set_error(C, DERR_INTERNAL, 3);
        }
    }
    if (threadIdx.x == 0) {
        C->total_chunks = carry_chunks;
        C->total_slots = carry_slots;
        if (s_bad) set_error(C, DERR_INVAL, 2);
        else if (carry_chunks > J.chunk_cap || carry_slots > J.slot_cap) set_error(C, DERR_INTERNAL, 1);
    }
}

namespace {

// First set bit at index >= k0 in bits[0, kmax), kmax a multiple of 32;
// kmax when there is none.
__device__ __forceinline__ int next_desc(const uint32_t* bits, int k0, int kmax)
{
    if (k0 >= kmax) return kmax;
    int w = k0 >> 5;
    uint32_t word = bits[w] & (FULL << (k0 & 31));
    const int wmax = kmax >> 5;
    while (word == 0) {
        if (++w >= wmax) return kmax;
        word = bits[w];
    }
    return (w << 5) + __ffs(word) - 1;
}

}  // namespace

__global__ void __launch_bounds__(RUN_BLOCK) k_runs(Job J)
{
    __shared__ uint32_t bits[RUN_WORDS];
    __shared__ uint16_t rec[MAP_STATES][RUN_REC];
    __shared__ uint32_t mapv[MAP_STATES];
    __shared__ uint32_t s_g, s_entry, s_prefix, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctr* C = J.ctr;
    const uint32_t epoch = C->epoch;
    const uint32_t ST_AGG = epoch * 4u + 1u, ST_INC = epoch * 4u + 2u;
    const int KMAX = RUN_WORDS * 32;
    if (*(volatile uint32_t*)&C->error) return;

    for (;;) {
        if (tid == 0) s_g = atomicAdd(&C->chunk_ticket, 1u);
        __syncthreads();
        const uint32_t g = s_g;
        if (g >= C->total_chunks) return;
        const uint32_t qi = find_inst(J.count, g, [&](uint32_t i) { return (unsigned long long)J.inst[i].chunk_base; });
        const Inst I = J.inst[qi];
        const uint32_t c = g - I.chunk_base;
        const uint32_t n = I.n, m = I.minrun;
        const uint32_t B = c * RUN_CHUNK;
        const uint32_t E = min(B + (uint32_t)RUN_CHUNK, n);
        const uint32_t span = E - B;
        const uint32_t rem = n - B;
        const uint32_t* a = J.keysA + I.off;

        // 1. descent bitmask: bit k <-> position B + k (the end n counts as one).
        //    Every load of a thread is issued before the first comparison, so a
        //    CTA keeps its whole window (RUN_LOADS keys per thread) in flight.
        uint32_t cur[RUN_LOADS], prv[RUN_LOADS];
#pragma unroll
        for (int j = 0; j < RUN_LOADS; ++j) {
            const unsigned long long P = (unsigned long long)B + (unsigned)(j * RUN_BLOCK + tid);
            cur[j] = P < n ? __ldg(a + P) : 0u;
            prv[j] = (P > 0 && P < n) ? __ldg(a + P - 1) : 0u;
        }
#pragma unroll
        for (int j = 0; j < RUN_LOADS; ++j) {
            const unsigned long long P = (unsigned long long)B + (unsigned)(j * RUN_BLOCK + tid);
            const bool d = P == n || (P < n && P > 0 && prv[j] > cur[j]);
            const uint32_t word = __ballot_sync(FULL, d);
            if (lane == 0) bits[j * (RUN_BLOCK / 32) + warp] = word;
        }
        __syncthreads();

        // 2a. can any step from inside this chunk be natural?  Only if two
        //     consecutive descents (or position 0 and the first descent) lie at
        //     least minrun apart; otherwise every chain is forced all the way
        //     and has a closed form (the usual case for unsorted data).
        bool may_natural = false;
        for (int w = tid; w < RUN_WORDS && w * 32 < (int)span; w += RUN_BLOCK) {
            uint32_t word = bits[w];
            if (w == 0) word |= 1u;                    // position 0 starts a gap too
            while (word) {
                const int e = w * 32 + __ffs(word) - 1;
                word &= word - 1;
                if ((uint32_t)e >= span) break;
                if (next_desc(bits, e + 1, KMAX) - e >= (int)m) { may_natural = true; break; }
            }
            if (may_natural) break;
        }
        const bool walk_all = __syncthreads_or(may_natural) != 0;

        // 2b. the chain from every entry state (lane = state; state m = D0)
        if (tid <= (int)m) {
            uint32_t cnt = 0, exitv = 0;
            int k = 0;
            bool walk = true;
            if (tid < (int)m) {
                k = tid;
            } else {
                const int d0 = next_desc(bits, 0, KMAX);
                if (d0 >= KMAX || (uint32_t)d0 >= span) {   // no run starts here
                    walk = false;
                    exitv = E == n ? STATE_END : m;
                } else {
                    k = d0;
                }
            }
            if (walk && !walk_all) {
                // forced steps only: starts k, k + m, k + 2m, ... below span
                cnt = (uint32_t)k < span ? (span - (uint32_t)k + m - 1) / m : 0u;
                if (E == n) exitv = STATE_END;
                else exitv = (uint32_t)k + cnt * m - span;   // < m
                rec[tid][0] = (uint16_t)k;                    // the progression's start
            } else if (walk) {
                bool symbolic = false;
                while ((uint32_t)k < span) {
                    rec[tid][cnt++] = (uint16_t)k;
                    const int d = next_desc(bits, k + 1, KMAX);
                    if (d >= KMAX) { symbolic = true; break; }   // f = d = next chunk's D0
                    const int forced = (int)min((uint32_t)(k + (int)m), rem);
                    k = max(d, forced);
                }
                // the last chunk's chains all end at n; elsewhere the exit is an
                // entry state of the next chunk (a position past the next chunk's
                // first minrun positions can only be its D0, even when it is n)
                if (E == n) exitv = STATE_END;
                else if (symbolic) exitv = m;
                else {
                    const uint32_t x = (uint32_t)k - span;
                    exitv = x < m ? x : m;
                }
            }
            mapv[tid] = (cnt << 8) | exitv;
        }
        __syncthreads();

        // 3. decoupled look-back over the chunks of this instance (warp 0)
        if (warp == 0) {
            uint32_t entry = 0;
            uint32_t prefix = 0;
            bool abort = false;
            if (c > 0) {
                uint32_t* gmap = J.chunk_map + (size_t)g * MAP_STATES;
                gmap[lane] = mapv[lane];
                gmap[lane + 32] = mapv[lane + 32];
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release_u32(&J.chunk_status[g], ST_AGG);
                // h maps entry states of chunk k + 1 to (state of chunk g, runs in between)
                uint32_t hs0 = lane, hs1 = lane + 32, hc0 = 0, hc1 = 0;
                uint32_t k = g - 1;
                for (;;) {
                    // every lane acquires the flag itself (bounded wait); the
                    // branch taken is lane 0's view, so the warp stays uniform
                    uint32_t sv = ld_acquire_u32(&J.chunk_status[k]);
                    if (sv != ST_AGG && sv != ST_INC) {
                        const long long t0 = clock64();
                        do {
                            __nanosleep(64);
                            sv = ld_acquire_u32(&J.chunk_status[k]);
                            if (clock64() - t0 > SPIN_LIMIT_CYCLES) break;
                        } while (sv != ST_AGG && sv != ST_INC);
                    }
                    if (!__all_sync(FULL, sv == ST_AGG || sv == ST_INC)) {
                        if (lane == 0) set_error(C, DERR_TIMEOUT, 10);
                        abort = true;
                        break;
                    }
                    sv = __shfl_sync(FULL, sv, 0);
                    if (sv == ST_INC) {
                        unsigned long long inc = 0;
                        if (lane == 0) inc = J.chunk_incl[k];   // lane 0 acquired ST_INC
                        inc = __shfl_sync(FULL, inc, 0);
                        const uint32_t y = (uint32_t)(inc & 0xffu);
                        const uint32_t cy = (uint32_t)(inc >> 8);
                        const uint32_t s0 = __shfl_sync(FULL, hs0, y & 31), s1 = __shfl_sync(FULL, hs1, y & 31);
                        const uint32_t c0 = __shfl_sync(FULL, hc0, y & 31), c1 = __shfl_sync(FULL, hc1, y & 31);
                        entry = y < 32 ? s0 : s1;
                        prefix = cy + (y < 32 ? c0 : c1);
                        if (y > m) { if (lane == 0) set_error(C, DERR_INTERNAL, 11); abort = true; }
                        break;
                    }
                    const uint32_t* kmap = J.chunk_map + (size_t)k * MAP_STATES;
                    const uint32_t m0 = kmap[lane], m1 = kmap[lane + 32];
                    const uint32_t y0 = m0 & 0xffu, y1 = m1 & 0xffu;
                    const uint32_t a0 = __shfl_sync(FULL, hs0, y0 & 31), a1 = __shfl_sync(FULL, hs1, y0 & 31);
                    const uint32_t b0 = __shfl_sync(FULL, hc0, y0 & 31), b1 = __shfl_sync(FULL, hc1, y0 & 31);
                    const uint32_t e0 = __shfl_sync(FULL, hs0, y1 & 31), e1 = __shfl_sync(FULL, hs1, y1 & 31);
                    const uint32_t f0 = __shfl_sync(FULL, hc0, y1 & 31), f1 = __shfl_sync(FULL, hc1, y1 & 31);
                    hs0 = y0 < 32 ? a0 : a1;
                    hc0 = (m0 >> 8) + (y0 < 32 ? b0 : b1);
                    hs1 = y1 < 32 ? e0 : e1;
                    hc1 = (m1 >> 8) + (y1 < 32 ? f0 : f1);
                    --k;
                }
            }
            if (!abort) {
                const uint32_t me = mapv[entry];
                if (lane == 0) {
                    J.chunk_incl[g] = ((unsigned long long)(prefix + (me >> 8)) << 8) | (me & 0xffu);
                    __threadfence();
                    st_release_u32(&J.chunk_status[g], ST_INC);
                }
            }
            if (lane == 0) {
                s_entry = entry;
                s_prefix = prefix;
                s_abort = abort ? 1u : 0u;
            }
        }
        __syncthreads();

        // 4. write this chunk's run starts
        if (!s_abort) {
            const uint32_t entry = s_entry, prefix = s_prefix;
            const uint32_t me = mapv[entry];
            const uint32_t cnt = me >> 8;
            uint32_t* rs = J.run_start + I.run_base + prefix;
            const unsigned long long cap = (unsigned long long)(n / 32) + 2;
            if ((unsigned long long)prefix + cnt + 1 > cap || cnt > (uint32_t)RUN_REC) {
                if (tid == 0) set_error(C, DERR_INTERNAL, 13);
            } else if (!walk_all) {
                const uint32_t k0 = B + rec[entry][0];
                for (uint32_t i = tid; i < cnt; i += RUN_BLOCK) rs[i] = k0 + i * m;
            } else {
                for (uint32_t i = tid; i < cnt; i += RUN_BLOCK) rs[i] = B + rec[entry][i];
            }
            if (c + 1 == I.nchunks && tid == 0) {
                const uint32_t R = prefix + cnt;
                if ((me & 0xffu) != STATE_END || (unsigned long long)R + 1 > (unsigned long long)(n / 32) + 2)
                    set_error(C, DERR_INTERNAL, 12);
                else {
                    J.run_start[I.run_base + R] = n;
                    J.inst[qi].runs = R;
                }
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_setup(const Job& J, cudaStream_t s)
{
    k_setup<<<1, 1024, 0, s>>>(J);
    return cudaGetLastError();
}

cudaError_t launch_runs(const Job& J, int grid, cudaStream_t s)
{
    // the setup kernel bumps the epoch in device memory, so status words left
    // by earlier calls (or earlier replays of a captured graph) read as "not ready"
    k_runs<<<grid, RUN_BLOCK, 0, s>>>(J);
    return cudaGetLastError();
}

}  // namespace ps
