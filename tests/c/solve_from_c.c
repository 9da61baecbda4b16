/*
 * A C99 consumer of libfbcc, with no Python between the caller and the library:
 * it reads a graph (int64 n and nnz, then n + 1 int32 offsets and nnz int32 ids),
 * solves it with fbcc_solve on device buffers of its own (cudaMalloc), solves it
 * a second time on the same workspace, and writes both results (int64 n_bcc,
 * n_ap, n_bridge, n_cc and device_status, then edge_bcc, bcc_head[0..n_bcc),
 * is_ap and is_bridge) to the output file. The tests compare them with the
 * oracle.
 *
 *   solve_from_c graph.bin out.bin
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "fbcc.h"

static int cuda_ok(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
        return 0;
    }
    return 1;
}

static int fbcc_ok(fbcc_status s, const char *what)
{
    if (s != FBCC_OK) {
        fprintf(stderr, "%s: %s\n", what, fbcc_status_string(s));
        return 0;
    }
    return 1;
}

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s graph.bin out.bin\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 2;
    int64_t hdr[2];
    if (fread(hdr, sizeof(int64_t), 2, in) != 2) return 2;
    const int64_t n = hdr[0], nnz = hdr[1];
    int32_t *off = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *adj = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *eb = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    int32_t *bh = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *ap = malloc((size_t)(n > 0 ? n : 1));
    uint8_t *br = malloc((size_t)(nnz > 0 ? nnz : 1));
    if (!off || !adj || !eb || !bh || !ap || !br) return 2;
    if (fread(off, sizeof(int32_t), (size_t)(n + 1), in) != (size_t)(n + 1)) return 2;
    if (fread(adj, sizeof(int32_t), (size_t)nnz, in) != (size_t)nnz) return 2;
    fclose(in);

    void *d_off = NULL, *d_adj = NULL, *d_eb = NULL, *d_bh = NULL, *d_ap = NULL, *d_br = NULL;
    const size_t zb = (size_t)(nnz > 0 ? nnz : 1), nb = (size_t)(n > 0 ? n : 1);
    if (!cuda_ok(cudaMalloc(&d_off, sizeof(int32_t) * (size_t)(n + 1)), "cudaMalloc") ||
        !cuda_ok(cudaMalloc(&d_adj, sizeof(int32_t) * zb), "cudaMalloc") ||
        !cuda_ok(cudaMalloc(&d_eb, sizeof(int32_t) * zb), "cudaMalloc") ||
        !cuda_ok(cudaMalloc(&d_bh, sizeof(int32_t) * nb), "cudaMalloc") ||
        !cuda_ok(cudaMalloc(&d_ap, nb), "cudaMalloc") || !cuda_ok(cudaMalloc(&d_br, zb), "cudaMalloc"))
        return 1;
    if (!cuda_ok(cudaMemcpy(d_off, off, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice), "H2D") ||
        !cuda_ok(cudaMemcpy(d_adj, adj, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice), "H2D"))
        return 1;

    fbcc_workspace *ws = NULL;
    if (!fbcc_ok(fbcc_workspace_create(n, nnz, &ws), "fbcc_workspace_create")) return 1;
    FILE *out = fopen(argv[2], "wb");
    if (!out) return 2;
    for (int rep = 0; rep < 2; ++rep) {
        fbcc_stats st;
        if (!fbcc_ok(fbcc_solve(d_off, 0, (const int32_t *)d_adj, n, nnz / 2, (int32_t *)d_eb, (int32_t *)d_bh,
                                (uint8_t *)d_ap, (uint8_t *)d_br, &st, ws, NULL),
                     "fbcc_solve"))
            return 1;
        if (!cuda_ok(cudaDeviceSynchronize(), "cudaDeviceSynchronize")) return 1;
        if (!cuda_ok(cudaMemcpy(eb, d_eb, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost), "D2H") ||
            !cuda_ok(cudaMemcpy(bh, d_bh, sizeof(int32_t) * (size_t)st.n_bcc, cudaMemcpyDeviceToHost), "D2H") ||
            !cuda_ok(cudaMemcpy(ap, d_ap, (size_t)n, cudaMemcpyDeviceToHost), "D2H") ||
            !cuda_ok(cudaMemcpy(br, d_br, (size_t)nnz, cudaMemcpyDeviceToHost), "D2H"))
            return 1;
        const int64_t head[5] = {st.n_bcc, st.n_ap, st.n_bridge, st.n_cc, st.device_status};
        fwrite(head, sizeof(int64_t), 5, out);
        fwrite(eb, sizeof(int32_t), (size_t)nnz, out);
        fwrite(bh, sizeof(int32_t), (size_t)st.n_bcc, out);
        fwrite(ap, 1, (size_t)n, out);
        fwrite(br, 1, (size_t)nnz, out);
    }
    fclose(out);
    fbcc_workspace_destroy(ws);
    cudaFree(d_off);
    cudaFree(d_adj);
    cudaFree(d_eb);
    cudaFree(d_bh);
    cudaFree(d_ap);
    cudaFree(d_br);
    free(off);
    free(adj);
    free(eb);
    free(bh);
    free(ap);
    free(br);
    return 0;
}
