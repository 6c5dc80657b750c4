// ps_run_noalloc: the sort for small arrays without any device allocation.
//
// Some callers cannot call cudaMalloc: code that owns a fixed, pre-sized
// budget of device memory (a foreign allocation would overrun it or fragment
// it), and latency-sensitive loops where cudaMalloc / cudaFree would
// synchronise the device.  For them this entry point takes only the caller's
// input and output arrays and uses, as scratch, one file-scope static device
// array of NA_BYTES bytes (about 2 MiB), which the CUDA driver places with the
// module: every GPU that loads the library holds it until the process exits.
//
// The kernel is a single-CTA variant of the on-chip tile kernel: run
// detection with the minrun rule, boundary powers, the forced-run sort, then
// the merges of the merge tree one power level at a time -- here ping-ponging
// between the caller's arrays and the static scratch array instead of
// between two shared-memory buffers, which lifts the size limit to
// NA_MAX_N elements.  The result is the same stable sort (keys and
// permutation) that ps_run produces.
//
// The scratch array is shared by every call and keeps the last call's
// contents; the kernel writes every scratch word before it reads it, so
// nothing has to start at zero.  Calls whose work overlaps on the GPU (two
// streams, two threads) race on the scratch array and must be serialised by
// the caller.
#include <mutex>

#include "ps_internal.cuh"

namespace {

constexpr uint32_t NA_MAX_N = PS_NOALLOC_MAX_N;
constexpr uint32_t NA_MAX_RUNS = NA_MAX_N / 32 + 2;       // run starts + end (minrun >= 32 for n >= 64)
constexpr size_t NA_OFF_BKEYS = 0;
constexpr size_t NA_OFF_BPERM = NA_OFF_BKEYS + (size_t)NA_MAX_N * 4;
constexpr size_t NA_OFF_RUNS = NA_OFF_BPERM + (size_t)NA_MAX_N * 4;
constexpr size_t NA_OFF_POW = NA_OFF_RUNS + (size_t)NA_MAX_RUNS * 4;
constexpr size_t NA_BYTES = NA_OFF_POW + (((size_t)NA_MAX_RUNS + 255) & ~(size_t)255);

constexpr int NA_BLOCK = 1024;
constexpr uint32_t NA_BITWORDS = NA_MAX_N / 32 + 2;
constexpr size_t NA_SMEM_BITS = (size_t)NA_BITWORDS * 4;
constexpr size_t NA_SMEM_SEGS = (size_t)2 * (NA_MAX_RUNS + 1) * 4;
constexpr size_t NA_SMEM = NA_SMEM_BITS > NA_SMEM_SEGS ? NA_SMEM_BITS : NA_SMEM_SEGS;
constexpr uint32_t FULL = 0xffffffffu;
constexpr int NA_MAX_DEVICES = 64;

}  // namespace

// The scratch: pingpong keys, pingpong permutation, run starts, powers.
static __device__ __align__(256) unsigned char g_ps_noalloc_scratch[NA_BYTES];

namespace {

__device__ __forceinline__ uint32_t na_minrun(uint32_t n)
{
    uint32_t l = n;
    while (l >= 64) l = (l + 1) >> 1;
    return l;
}

// First set bit at index >= k0 (bits of positions 0 .. n, n itself set).
__device__ __forceinline__ uint32_t na_next_desc(const uint32_t* bits, uint32_t k0, uint32_t n)
{
    if (k0 >= n) return n;
    uint32_t w = k0 >> 5;
    uint32_t word = bits[w] & (FULL << (k0 & 31));
    while (word == 0) word = bits[++w];
    const uint32_t k = (w << 5) + __ffs(word) - 1;
    return k < n ? k : n;
}

__device__ __forceinline__ uint32_t na_kappa(const uint32_t* rs, uint32_t s, uint32_t n)
{
    return (uint32_t)((((unsigned long long)rs[s] + rs[s + 1]) << 31) / n);
}

__global__ void __launch_bounds__(NA_BLOCK) k_small_noalloc(uint32_t* keys, uint32_t* perm, uint32_t n,
                                                            unsigned char* scratch)
{
    extern __shared__ uint32_t na_sm[];
    __shared__ uint32_t s_R, s_mask, s_total;
    __shared__ uint32_t warp_sums[NA_BLOCK / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* bkeys = reinterpret_cast<uint32_t*>(scratch + NA_OFF_BKEYS);
    uint32_t* bperm = reinterpret_cast<uint32_t*>(scratch + NA_OFF_BPERM);
    uint32_t* runs = reinterpret_cast<uint32_t*>(scratch + NA_OFF_RUNS);
    uint8_t* pw = reinterpret_cast<uint8_t*>(scratch + NA_OFF_POW);

    if (n <= 1) {
        if (n == 1 && perm && tid == 0) perm[0] = 0;
        return;
    }
    const uint32_t m = na_minrun(n);

    // 1. descent bitmask (the end n counts as a descent)
    uint32_t* bits = na_sm;
    const uint32_t nwords = n / 32 + 2;
    for (uint32_t w = warp; w < nwords; w += NA_BLOCK / 32) {
        const uint32_t P = w * 32 + lane;
        const bool d = P == n || (P > 0 && P < n && keys[P - 1] > keys[P]);
        const uint32_t word = __ballot_sync(FULL, d);
        if (lane == 0) bits[w] = word;
    }
    if (tid == 0) s_mask = 0;
    __syncthreads();

    // 2. run starts: the orbit of 0 under f(s) = max(d(s), min(s + minrun, n))
    if (tid == 0) {
        uint32_t s = 0, R = 0;
        while (s < n) {
            runs[R++] = s;
            const uint32_t d = na_next_desc(bits, s + 1, n);
            const uint32_t forced = s + m < n ? s + m : n;
            s = d > forced ? d : forced;
        }
        runs[R] = n;
        s_R = R;
    }
    __syncthreads();
    const uint32_t R = s_R;

    // 3. powers (fixed-point midpoints) and the identity permutation
    for (uint32_t t = 1 + tid; t < R; t += NA_BLOCK) {
        const uint32_t p = __clz(na_kappa(runs, t - 1, n) ^ na_kappa(runs, t, n)) + 1;
        pw[t] = (uint8_t)p;
        atomicOr(&s_mask, 1u << (p - 1));
    }
    if (perm)
        for (uint32_t i = tid; i < n; i += NA_BLOCK) perm[i] = i;
    __syncthreads();

    // 4. forced runs (at most 63 elements whenever unsorted): stable rank sort
    for (uint32_t r = warp; r < R; r += NA_BLOCK / 32) {
        const uint32_t lo = runs[r], len = runs[r + 1] - lo;
        if (len < 2 || len > 64) continue;
        const bool ok0 = lane < (int)len, ok1 = lane + 32 < (int)len;
        const uint32_t k0 = ok0 ? keys[lo + lane] : FULL, k1 = ok1 ? keys[lo + lane + 32] : FULL;
        const uint32_t p0 = (ok0 && perm) ? perm[lo + lane] : 0u, p1 = (ok1 && perm) ? perm[lo + lane + 32] : 0u;
        const uint32_t nk0 = __shfl_down_sync(FULL, k0, 1), f1 = __shfl_sync(FULL, k1, 0);
        const uint32_t nk1 = __shfl_down_sync(FULL, k1, 1);
        const bool d0 = lane + 1 < (int)len && k0 > (lane == 31 ? f1 : nk0);
        const bool d1 = lane + 33 < (int)len && k1 > nk1;
        if (!__any_sync(FULL, d0 || d1)) continue;
        uint32_t rk0 = 0, rk1 = 0;
        for (uint32_t j = 0; j < len; ++j) {
            const uint32_t y = __shfl_sync(FULL, j < 32 ? k0 : k1, j & 31);
            rk0 += (y < k0) || (y == k0 && j < (uint32_t)lane);
            rk1 += (y < k1) || (y == k1 && j < (uint32_t)lane + 32);
        }
        __syncwarp();
        if (ok0) { keys[lo + rk0] = k0; if (perm) perm[lo + rk0] = p0; }
        if (ok1) { keys[lo + rk1] = k1; if (perm) perm[lo + rk1] = p1; }
        __syncwarp();
    }
    __syncthreads();

    // 5. merge levels, largest power first, between the caller's arrays and
    //    the scratch arrays; boundaries of smaller power delimit segments
    uint32_t* seg_lo = na_sm;
    uint32_t* seg_mid = na_sm + NA_MAX_RUNS + 1;
    uint32_t* ck = keys;
    uint32_t* cp = perm;
    uint32_t* ok = bkeys;
    uint32_t* op = perm ? bperm : nullptr;
    uint32_t mask = s_mask;
    const uint32_t nb = R - 1;                                    // boundaries 1 .. R-1
    const uint32_t per = (nb + NA_BLOCK - 1) / NA_BLOCK;
    const uint32_t t0 = 1 + tid * per, t1 = min(t0 + per, R);
    while (mask) {
        const uint32_t p = 32 - __clz(mask);
        mask &= ~(1u << (p - 1));
        uint32_t local = 0;
        for (uint32_t t = t0; t < t1; ++t) local += pw[t] < p;
        uint32_t x = local;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
            if (lane == 31) s_total = w;
        }
        __syncthreads();
        uint32_t before = (warp ? warp_sums[warp - 1] : 0u) + x - local;
        const uint32_t total = s_total;
        const uint32_t nseg = total + 1;
        if (tid == 0) {
            seg_lo[0] = 0;
            seg_lo[nseg] = n;
        }
        {
            uint32_t c = before;
            for (uint32_t t = t0; t < t1; ++t)
                if (pw[t] < p) seg_lo[++c] = runs[t];
        }
        __syncthreads();
        for (uint32_t k = tid; k < nseg; k += NA_BLOCK) seg_mid[k] = seg_lo[k + 1];
        __syncthreads();
        {
            uint32_t c = before;
            for (uint32_t t = t0; t < t1; ++t) {
                if (pw[t] < p) ++c;
                else if (pw[t] == p) seg_mid[c] = runs[t];
            }
        }
        __syncthreads();

        const uint32_t kper = (n + NA_BLOCK - 1) / NA_BLOCK;
        const uint32_t x0 = tid * kper;
        if (x0 < n) {
            const uint32_t x1 = min(x0 + kper, n);
            uint32_t sg = 0, hiS = nseg;
            while (hiS - sg > 1) {
                const uint32_t mid = (sg + hiS) >> 1;
                if (seg_lo[mid] <= x0) sg = mid; else hiS = mid;
            }
            uint32_t xx = x0;
            while (xx < x1) {
                const uint32_t slo = seg_lo[sg], smid = seg_mid[sg], shi = seg_lo[sg + 1];
                const uint32_t end = min(x1, shi);
                if (smid == shi) {
                    for (; xx < end; ++xx) {
                        ok[xx] = ck[xx];
                        if (op) op[xx] = cp[xx];
                    }
                } else {
                    const uint32_t la = smid - slo, lb = shi - smid, d = xx - slo;
                    uint32_t ilo = d > lb ? d - lb : 0u, ihi = min(d, la);
                    while (ilo < ihi) {
                        const uint32_t mm = (ilo + ihi) >> 1;
                        if (ck[slo + mm] <= ck[smid + d - 1 - mm]) ilo = mm + 1; else ihi = mm;
                    }
                    uint32_t ia = ilo, ib = d - ilo;
                    for (; xx < end; ++xx) {
                        const bool ta = ia < la && (ib >= lb || ck[slo + ia] <= ck[smid + ib]);
                        const uint32_t src = ta ? slo + ia : smid + ib;
                        ok[xx] = ck[src];
                        if (op) op[xx] = cp[src];
                        if (ta) ++ia; else ++ib;
                    }
                }
                ++sg;
            }
        }
        __syncthreads();
        uint32_t* t = ck; ck = ok; ok = t;
        t = cp; cp = op; op = t;
    }
    // 6. the result must end in the caller's arrays
    if (ck != keys) {
        for (uint32_t i = tid; i < n; i += NA_BLOCK) {
            keys[i] = ck[i];
            if (perm) perm[i] = cp[i];
        }
    }
}

std::mutex g_na_mu;
void* g_na_ptr[NA_MAX_DEVICES];
bool g_na_ready[NA_MAX_DEVICES];

}  // namespace

extern "C" PS_API ps_status ps_run_noalloc(uint32_t* d_keys, uint32_t* d_perm, uint64_t n, int device,
                                           void* cuda_stream)
{
    if (n > NA_MAX_N) return PS_EINVAL;                   // the scratch array holds NA_MAX_N elements
    if (n > 0 && !d_keys) return PS_EINVAL;
    if (device < 0 || device >= NA_MAX_DEVICES) return PS_EINVAL;
    if (n == 0) return PS_OK;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        return PS_ECUDA;
    }
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PS_ECUDA;
    }
    ps_status st = PS_OK;
    {
        // set-up, once per device, with that device current: the device
        // address of the scratch array (the host-side name is only a stand-in)
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_ready[device]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_ps_noalloc_scratch) != cudaSuccess || !p) {
                st = PS_ECUDA;
            } else if (cudaFuncSetAttribute(k_small_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)NA_SMEM) != cudaSuccess) {
                st = PS_ECUDA;
            } else {
                g_na_ptr[device] = p;
                g_na_ready[device] = true;
            }
        }
    }
    if (st == PS_OK) {
        k_small_noalloc<<<1, NA_BLOCK, NA_SMEM, static_cast<cudaStream_t>(cuda_stream)>>>(
            d_keys, d_perm, (uint32_t)n, static_cast<unsigned char*>(g_na_ptr[device]));
        if (cudaGetLastError() != cudaSuccess) st = PS_ECUDA;
    } else {
        cudaGetLastError();
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
