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
        long long v[kItems];
        const int64_t i0 = t * kTile + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int j = 0; j < kItems; ++j) v[j] = (i0 + j < len) ? __popc(words[i0 + j]) : 0;
        scan_tile_exclusive(v, t, status, err);
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            if (i0 + j <= len) out[i0 + j] = (int32_t)v[j];
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

}  // namespace fbcc
