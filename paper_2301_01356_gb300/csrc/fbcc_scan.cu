// Exclusive prefix sum used by the outputs: popcount ranks of the BCC key
// bitmap, in one pass with decoupled look-back.
#include "fbcc_internal.cuh"

namespace fbcc {

// out[i] = number of set bits in words[0..i) for i in [0, len].
__global__ void __launch_bounds__(kThreads) k_scan_popc(const uint32_t *words, int32_t *out, int64_t len,
                                                        long long *ticket, uint64_t *status, int *err)
{
    const int64_t ntiles = (len + 1 + kTile - 1) / kTile;
    while (true) {
        int64_t t = scan_ticket(ticket);
        if (t >= ntiles) return;
        static_assert(kItems == 8, "two 16-byte loads and stores per thread");
        long long v[kItems];
        const int64_t i0 = t * kTile + (int64_t)threadIdx.x * kItems;
        // whole groups of eight move as 16-byte vectors (the workspace's pieces are
        // 256-byte aligned and i0 is a multiple of 8)
        const bool whole = i0 + kItems <= len;
        if (whole) {
            const uint4 a = *reinterpret_cast<const uint4 *>(words + i0);
            const uint4 b = *reinterpret_cast<const uint4 *>(words + i0 + 4);
            v[0] = __popc(a.x); v[1] = __popc(a.y); v[2] = __popc(a.z); v[3] = __popc(a.w);
            v[4] = __popc(b.x); v[5] = __popc(b.y); v[6] = __popc(b.z); v[7] = __popc(b.w);
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j) v[j] = (i0 + j < len) ? __popc(words[i0 + j]) : 0;
        }
        scan_tile_exclusive(v, t, status, err);
        if (whole) {
            *reinterpret_cast<int4 *>(out + i0) = make_int4((int32_t)v[0], (int32_t)v[1], (int32_t)v[2], (int32_t)v[3]);
            *reinterpret_cast<int4 *>(out + i0 + 4) =
                make_int4((int32_t)v[4], (int32_t)v[5], (int32_t)v[6], (int32_t)v[7]);
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j)
                if (i0 + j <= len) out[i0 + j] = (int32_t)v[j];
        }
    }
}

// In place: a[i] = a[0] + ... + a[i-1] for i in [0, len], a[len] = the total (a holds
// len + 1 entries; the last is ignored on input).
__global__ void __launch_bounds__(kThreads) k_scan_i32(int32_t *a, int64_t len, long long *ticket, uint64_t *status,
                                                       int *err)
{
    const int64_t ntiles = (len + 1 + kTile - 1) / kTile;
    while (true) {
        int64_t t = scan_ticket(ticket);
        if (t >= ntiles) return;
        long long v[kItems];
        const int64_t i0 = t * kTile + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int j = 0; j < kItems; ++j) v[j] = i0 + j < len ? a[i0 + j] : 0;
        scan_tile_exclusive(v, t, status, err);   // (synchronises the CTA before any write below)
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            if (i0 + j <= len) a[i0 + j] = (int32_t)v[j];
    }
}

static cudaError_t reset_scan(const Dev &d, int64_t len, const Launch &L)
{
    const int64_t ntiles = (len + 1 + kTile - 1) / kTile;
    cudaError_t e = cudaMemsetAsync(d.counters, 0, sizeof(long long), L.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.scan_status, 0, ntiles * sizeof(uint64_t), L.s);
    return e;
}

cudaError_t launch_scan_popc(const Dev &d, const uint32_t *words, int32_t *out, int64_t len, const Launch &L)
{
    cudaError_t e = reset_scan(d, len, L);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (len + 1 + kTile - 1) / kTile;
    k_scan_popc<<<grid_for(L, ntiles), kThreads, 0, L.s>>>(words, out, len, d.counters, d.scan_status, d.err);
    L.mark("k_scan_popc");
    return cudaGetLastError();
}

cudaError_t launch_scan_i32(const Dev &d, int32_t *a, int64_t len, const Launch &L)
{
    cudaError_t e = reset_scan(d, len, L);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (len + 1 + kTile - 1) / kTile;
    k_scan_i32<<<grid_for(L, ntiles), kThreads, 0, L.s>>>(a, len, d.counters, d.scan_status, d.err);
    L.mark("k_scan_i32");
    return cudaGetLastError();
}

}  // namespace fbcc
