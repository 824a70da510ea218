// tc_gemm.cuh -- tensor-core (tcgen05) update C -= A B^T, operands TF32 (kind::tf32) or
// bf16 (kind::f16), fp32 accumulation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace expm {

// A: M x K, B: N x K (both K-major: fp32 read as TF32, or bf16), C: M x N fp32 row-major.
// Operand leading dimensions must be multiples of 16 bytes (4 floats / 8 bf16), C's of 4
// floats, and A, B, C 16-byte aligned (TMA rules).
// With batch strides (elements; batch entry z of A at A + z sA, likewise B and C) they
// must be multiples of 16 bytes as well.
bool tc_gemm_supported(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const void *C, int ldc,
                       bool bf16 = false, int64_t sA = 0, int64_t sB = 0, int64_t sC = 0);
// err_flag (device int) is set to 1 if a bounded wait inside the kernel gave up.
cudaError_t tc_gemm_tf32_sub(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                             int *err_flag, cudaStream_t st);
cudaError_t tc_gemm_bf16_sub(int M, int N, int K, const uint16_t *A, int lda, const uint16_t *B, int ldb, float *C,
                             int ldc, int *err_flag, cudaStream_t st);
// `batch` products in one launch (grid z = batch entry); operands bf16 or fp32 (TF32)
cudaError_t tc_gemm_batched(bool bf16, int M, int N, int K, const void *A, int lda, int64_t sA, const void *B, int ldb,
                            int64_t sB, float *C, int ldc, int64_t sC, int batch, int *err_flag, cudaStream_t st);

}  // namespace expm
