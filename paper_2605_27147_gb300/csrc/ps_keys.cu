// The key-value generalisation: keys of other 32-bit types, and payloads of
// any width that follow the keys through the stable permutation.
//
// Typed keys.  A signed or floating-point key order is an order on the bit
// patterns that one bijection of 32-bit words turns into the unsigned order:
//   int32:  flip the sign bit (two's complement -> offset binary);
//   float:  a negative value (sign set) flips every bit, so a larger
//           magnitude maps lower; a positive value flips the sign bit only,
//           so it maps above every negative one.  The result orders as IEEE
//           754 totalOrder: -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN.
// The forward map runs over the caller's keys before run detection, the
// inverse after the last merge (or Copy), so every kernel in between sorts
// plain unsigned words and the keys come back as the caller's bit patterns.
// Both maps are elementwise and in place: 8 bytes per element of traffic.
//
// Payloads.  The sort's permutation gives every row's source: row r of the
// output is row perm[r] of the input.  One instance of rows that are whole
// words goes by tiles: a CTA reads 256 permutation entries,
// then copies the tile's words (16, 8 or 4 bytes, as alignment allows) in
// output order, consecutive threads on consecutive words (coalesced
// stores, every load independent).  Otherwise
// a thread copies a row of up to 16 bytes, a warp a wider one, with the
// widest word (16, 4 or 1 bytes) that the alignment and the width allow.
#include "ps_internal.cuh"

namespace ps {

namespace {

__device__ __forceinline__ uint32_t key_to_order(uint32_t x, uint32_t type)
{
    if (type == PS_KEY_I32) return x ^ 0x80000000u;
    return x ^ ((uint32_t)((int32_t)x >> 31) | 0x80000000u);
}

__device__ __forceinline__ uint32_t key_from_order(uint32_t y, uint32_t type)
{
    if (type == PS_KEY_I32) return y ^ 0x80000000u;
    return y ^ (((y >> 31) - 1u) | 0x80000000u);
}

// Rows of one call: n, or the offsets table's end (0 when it exceeds the limit).
__device__ __forceinline__ unsigned long long rows_of(const unsigned long long* off, uint32_t count,
                                                      unsigned long long n, unsigned long long max_total)
{
    if (!off) return n;
    const unsigned long long t = off[count];
    return t <= max_total ? t : 0ull;
}

}  // namespace

__global__ void __launch_bounds__(256) k_key_map(Job J, int forward)
{
    Ctr* C = J.ctr;
    if (forward) {
        // a bad offsets table (found by k_setup) leaves the keys untouched
        if (*(volatile uint32_t*)&C->error) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) C->keys_mapped = 1;
    } else if (!*(volatile uint32_t*)&C->keys_mapped) {
        return;
    }
    const unsigned long long total = rows_of(J.offsets, J.count, J.single_n, J.max_total);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const uint32_t x = J.keysA[i];
        J.keysA[i] = forward ? key_to_order(x, J.key_type) : key_from_order(x, J.key_type);
    }
}

template <typename W>
__device__ __forceinline__ void copy_row(const unsigned char* src, unsigned char* dst, uint32_t words, uint32_t lane,
                                         uint32_t step)
{
    const W* s = reinterpret_cast<const W*>(src);
    W* d = reinterpret_cast<W*>(dst);
    for (uint32_t i = lane; i < words; i += step) d[i] = s[i];
}

__global__ void __launch_bounds__(256) k_gather_rows(const uint32_t* perm, const unsigned long long* off,
                                                     uint32_t count, unsigned long long n,
                                                     unsigned long long max_total, const unsigned char* src,
                                                     unsigned char* dst, uint32_t row_bytes, Ctr* C)
{
    const unsigned long long rows = rows_of(off, count, n, max_total);
    if (off && off[count] > max_total) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_error(C, DERR_INVAL, 70);
        return;
    }
    const uint32_t wide = (((uintptr_t)src | (uintptr_t)dst | row_bytes) & 15u) == 0 ? 16u
                        : (((uintptr_t)src | (uintptr_t)dst | row_bytes) & 3u) == 0 ? 4u : 1u;
    const bool by_warp = row_bytes > 16u;
    const uint32_t lane = by_warp ? (threadIdx.x & 31u) : 0u, step = by_warp ? 32u : 1u;
    const unsigned long long unit = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long first = by_warp ? unit >> 5 : unit;
    const unsigned long long stride = ((unsigned long long)gridDim.x * blockDim.x) >> (by_warp ? 5 : 0);
    for (unsigned long long r = first; r < rows; r += stride) {
        unsigned long long base = 0, size = rows;
        if (off) {
            // the instance holding row r
            const uint32_t q = find_inst(count, r, [&](uint32_t i) { return off[i]; });
            base = off[q];
            size = off[q + 1] >= base ? off[q + 1] - base : 0ull;
            if (base > rows) base = rows;
            if (size > rows - base) size = rows - base;   // every source row stays inside the arrays
            if (r < base || r - base >= size) {            // a decreasing table
                if (lane == 0) set_error(C, DERR_INVAL, 72);
                continue;
            }
        }
        const uint32_t p = perm[r];
        if ((unsigned long long)p >= size) {
            if (lane == 0) set_error(C, DERR_INVAL, 71);
            continue;
        }
        const unsigned char* s = src + (base + p) * row_bytes;
        unsigned char* d = dst + r * row_bytes;
        if (wide == 16u) copy_row<uint4>(s, d, row_bytes >> 4, lane, step);
        else if (wide == 4u) copy_row<uint32_t>(s, d, row_bytes >> 2, lane, step);
        else copy_row<unsigned char>(s, d, row_bytes, lane, step);
    }
}

template <typename Wd>
__global__ void __launch_bounds__(256) k_gather_tiled(const uint32_t* perm, unsigned long long n, const Wd* src,
                                                      Wd* dst, uint32_t wpr, Ctr* C)
{
    __shared__ uint32_t sp[256];
    const uint32_t tid = threadIdx.x;
    const uint32_t drow = 256u / wpr, dword = 256u % wpr;
    for (unsigned long long t0 = (unsigned long long)blockIdx.x * 256; t0 < n;
         t0 += (unsigned long long)gridDim.x * 256) {
        const uint32_t rows = (uint32_t)min(256ull, n - t0);
        if (tid < rows) {
            uint32_t p = perm[t0 + tid];
            if (p >= n) {
                set_error(C, DERR_INVAL, 71);
                p = NONE;
            }
            sp[tid] = p;
        }
        __syncthreads();
        const uint32_t total = rows * wpr;
        uint32_t row = tid / wpr, word = tid % wpr;
#pragma unroll 8
        for (uint32_t q = tid; q < total; q += 256) {
            const uint32_t p = sp[row];
            if (p != NONE) dst[(t0 + row) * wpr + word] = src[(unsigned long long)p * wpr + word];
            row += drow;
            word += dword;
            if (word >= wpr) {
                word -= wpr;
                ++row;
            }
        }
        __syncthreads();
    }
}

// 64-bit keys as two-word records: the same order-preserving maps at 64
// bits, and the halves swapped so that the high word comes first in memory.
__device__ __forceinline__ unsigned long long key64_to_order(unsigned long long x, uint32_t type)
{
    if (type == PS_KEY_I32) return x ^ 0x8000000000000000ull;
    if (type == PS_KEY_F32) return x ^ ((unsigned long long)((long long)x >> 63) | 0x8000000000000000ull);
    return x;
}

__device__ __forceinline__ unsigned long long key64_from_order(unsigned long long y, uint32_t type)
{
    if (type == PS_KEY_I32) return y ^ 0x8000000000000000ull;
    if (type == PS_KEY_F32) return y ^ (((y >> 63) - 1ull) | 0x8000000000000000ull);
    return y;
}

__global__ void __launch_bounds__(256) k_key64_in(unsigned long long* keys, unsigned long long n, uint32_t type)
{
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long y = key64_to_order(keys[i], type);
        keys[i] = (y << 32) | (y >> 32);   // words (high, low)
    }
}

__global__ void __launch_bounds__(256) k_key64_out(const unsigned long long* rows, unsigned long long* keys,
                                                   unsigned long long n, uint32_t type)
{
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long r = rows[i];
        keys[i] = key64_from_order((r << 32) | (r >> 32), type);
    }
}

cudaError_t launch_key64(bool in, const void* rows, void* keys, unsigned long long n, uint32_t type, int grid,
                         cudaStream_t s)
{
    if (in) k_key64_in<<<grid, 256, 0, s>>>(static_cast<unsigned long long*>(keys), n, type);
    else k_key64_out<<<grid, 256, 0, s>>>(static_cast<const unsigned long long*>(rows),
                                           static_cast<unsigned long long*>(keys), n, type);
    return cudaGetLastError();
}

cudaError_t launch_key_map(const Job& J, bool forward, int grid, cudaStream_t s)
{
    k_key_map<<<grid, 256, 0, s>>>(J, forward ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const uint32_t* perm, const unsigned long long* offsets, uint32_t count,
                               unsigned long long n, unsigned long long max_total, const void* src, void* dst,
                               uint32_t row_bytes, Ctr* ctr, int grid, cudaStream_t s)
{
    const uintptr_t al = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | row_bytes;
    if (!offsets && (al & 15u) == 0) {
        k_gather_tiled<uint4><<<grid, 256, 0, s>>>(perm, n, static_cast<const uint4*>(src), static_cast<uint4*>(dst),
                                                   row_bytes >> 4, ctr);
    } else if (!offsets && (al & 7u) == 0) {
        k_gather_tiled<uint2><<<grid, 256, 0, s>>>(perm, n, static_cast<const uint2*>(src), static_cast<uint2*>(dst),
                                                   row_bytes >> 3, ctr);
    } else if (!offsets && (al & 3u) == 0) {
        k_gather_tiled<uint32_t><<<grid, 256, 0, s>>>(perm, n, static_cast<const uint32_t*>(src),
                                                      static_cast<uint32_t*>(dst), row_bytes >> 2, ctr);
    } else {
        k_gather_rows<<<grid, 256, 0, s>>>(perm, offsets, count, n, max_total, static_cast<const unsigned char*>(src),
                                           static_cast<unsigned char*>(dst), row_bytes, ctr);
    }
    return cudaGetLastError();
}

}  // namespace ps
