// oz_gemm.cuh -- binary64-accurate residual product on the bf16 tensor cores (oz_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "arith.cuh"

namespace expm {

// workspace of one residual product: slices of A and its row scales (depend on n and
// complex_a only, written by oz_split_a), then slices of X and column scales
size_t oz_resid_bytes(int n, int kc, int nsys, int complex_a);
bool oz_resid_supported(int n, int kc, int nsys);
// slices of A (n x n, row stride lda in elements, real or interleaved complex) into ws
cudaError_t oz_split_a(int n, const double *A, int64_t lda, int complex_a, void *ws, cudaStream_t st);
// slices of X_s, s < nsys (n x kc complex, system stride nk) into ws
cudaError_t oz_split_x(int n, int kc, int nsys, int complex_a, const cx<double> *X, int64_t nk, void *ws,
                       cudaStream_t st);
// R_s -= t A X_s (R_s: n x kc complex, system stride nk) from the slices in ws.  When
// `timeout` is non-null the stream is synchronised and *timeout set to 1 if a bounded
// wait in the kernel gave up.
cudaError_t oz_product(int n, int kc, int nsys, int complex_a, double t, int64_t nk, cx<double> *R, void *ws,
                       cudaStream_t st, int *timeout);

// The light update for a binary32 correction D (|D| << |X|): four slices of D into ws,
// then R_s -= t A D_s with four slices of A and the 10 products of order <= 3 -- about
// 2^-30 of max|A_i.| max|D_.j| K, enough once D is ~1e-6 of X.
cudaError_t oz_split_d(int n, int kc, int nsys, int complex_a, const cx<float> *D, int64_t nk, void *ws,
                       cudaStream_t st);
cudaError_t oz_product_light(int n, int kc, int nsys, int complex_a, double t, int64_t nk, cx<double> *R, void *ws,
                             cudaStream_t st, int *timeout);
// the product's time-out flag (1 if a bounded wait gave up); synchronises st
cudaError_t oz_read_timeout(int n, int kc, int nsys, int complex_a, void *ws, cudaStream_t st, int *timeout);

}  // namespace expm
