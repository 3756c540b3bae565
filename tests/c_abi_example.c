/*
 * c_abi_example.c -- the C ABI (include/wxpy.h) from a plain C99 program, for
 * the tests: w = RN(RN(alpha*x) + y) through wxpy() and the same update with
 * its squared 2-norm through wxpy_norm2(), on device memory from cudaMalloc.
 * Inputs are exact binary64 values from a formula the test repeats:
 *   x[i] = (i % 97) / 64 - 0.7,  y[i] = (i % 31) / 128 - 0.1,  alpha = 0.75.
 * Prints the bits of every w[i] (hex, one per line), then the norm's bits.
 */
#include <cuda_runtime.h>
#include <inttypes.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "wxpy.h"

static int check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
        return 1;
    }
    return 0;
}

int main(int argc, char **argv) {
    const int64_t n = argc > 1 ? (int64_t)atoll(argv[1]) : 4099;
    const double alpha = 0.75;
    double *hx = malloc((size_t)n * 8), *hy = malloc((size_t)n * 8), *hw = malloc((size_t)n * 8);
    if (!hx || !hy || !hw) return 3;
    for (int64_t i = 0; i < n; ++i) {
        hx[i] = (double)(i % 97) / 64.0 - 0.7;
        hy[i] = (double)(i % 31) / 128.0 - 0.1;
    }
    double *dx, *dy, *dw, *dr;
    void *ws;
    const int64_t ws_bytes = wxpy_reduce_workspace_bytes(n);
    if (check_cuda(cudaMalloc((void **)&dx, (size_t)n * 8), "malloc") ||
        check_cuda(cudaMalloc((void **)&dy, (size_t)n * 8), "malloc") ||
        check_cuda(cudaMalloc((void **)&dw, (size_t)n * 8), "malloc") ||
        check_cuda(cudaMalloc((void **)&dr, 8), "malloc") ||
        check_cuda(cudaMalloc(&ws, (size_t)ws_bytes), "malloc") ||
        check_cuda(cudaMemcpy(dx, hx, (size_t)n * 8, cudaMemcpyHostToDevice), "copy") ||
        check_cuda(cudaMemcpy(dy, hy, (size_t)n * 8, cudaMemcpyHostToDevice), "copy"))
        return 2;
    int st = wxpy(n, alpha, dx, dy, dw, NULL);
    if (st != WXPY_OK) {
        fprintf(stderr, "wxpy: %s\n", wxpy_strerror(st));
        return 2;
    }
    if (check_cuda(cudaMemcpy(hw, dw, (size_t)n * 8, cudaMemcpyDeviceToHost), "copy")) return 2;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t b;
        memcpy(&b, &hw[i], 8);
        printf("%016" PRIx64 "\n", b);
    }
    st = wxpy_norm2(n, alpha, dx, dy, dw, dr, ws, ws_bytes, NULL);
    if (st != WXPY_OK) {
        fprintf(stderr, "wxpy_norm2: %s\n", wxpy_strerror(st));
        return 2;
    }
    double r;
    if (check_cuda(cudaMemcpy(&r, dr, 8, cudaMemcpyDeviceToHost), "copy")) return 2;
    uint64_t rb;
    memcpy(&rb, &r, 8);
    printf("norm2 %016" PRIx64 "\n", rb);
    cudaFree(dx);
    cudaFree(dy);
    cudaFree(dw);
    cudaFree(dr);
    cudaFree(ws);
    free(hx);
    free(hy);
    free(hw);
    return 0;
}
