// tc_gemm.cuh -- tensor-core (tcgen05, kind::tf32) update C -= A B^T.
#pragma once
#include <cuda_runtime.h>

namespace expm {

// A: M x K, B: N x K (both K-major, fp32 read as TF32), C: M x N fp32 row-major.
// Leading dimensions must be multiples of 4 floats and A, B, C 16-byte aligned (TMA rules).
bool tc_gemm_supported(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const void *C, int ldc);
// err_flag (device int) is set to 1 if a bounded wait inside the kernel gave up.
cudaError_t tc_gemm_tf32_sub(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                             int *err_flag, cudaStream_t st);

}  // namespace expm
