// laplace2d.cu -- expm_apply_laplacian2d: Y = e^c R_n(tA - cI) V for the separable 2D
// operator A = I_y (x) T_x + T_y (x) I_x of the finite-difference Laplacian (the paper's
// second workload, Sec. 5), T_x = tridiag(ax, bx, ax) (dx points), T_y = tridiag(ay, by, ay)
// (dy points), unknown iy * dx + ix.
//
// T_y = S diag(mu) S with S the orthonormal DST-I (S = S^T = S^{-1}), mu_j = by + 2 ay
// cos((j+1) pi/(dy+1)).  So A = (S (x) I) [ (+)_j (T_x + mu_j I) ] (S (x) I), and by
// Remark 3.1
//     W = (S (x) I) V,   Z = e^c R_n(tB - cI) W,   Y = (S (x) I) Z,
// with B = (+)_j (T_x + mu_j I) one real symmetric tridiagonal matrix of dx * dy rows whose
// off-diagonal is zero between the blocks -- the pole-batched tridiagonal path as it is.
// The transform along y is a dense product with S (dy x dy times dy x (dx r)): in binary64
// for EXPM_FP64; for the mixed precisions the binary64-accurate slice product on the bf16
// tensor cores of oz_gemm.cu (S as the "matrix", V viewed as dy x (dx r / 2) complex
// columns of one system, R = 0 - (-1) S V), whose error is a few 2^-48 of the row and
// column scales -- far below those paths' tolerances.
#include <cmath>

#include "../../include/expm.h"
#include "oz_gemm.cuh"
#include "plan.cuh"

namespace expm {
namespace {

// S[j][i] = sqrt(2/(dy+1)) sin((j+1)(i+1) pi/(dy+1))
__global__ void dst_matrix(int dy, double *S) {
    const int j = blockIdx.x;
    const double sc = sqrt(2.0 / (dy + 1));
    for (int i = threadIdx.x; i < dy; i += blockDim.x) {
        // (j+1)(i+1) reduced modulo 2(dy+1) keeps the sine argument small and exact
        const long long q = ((long long)(j + 1) * (i + 1)) % (2LL * (dy + 1));
        S[(int64_t)j * dy + i] = sc * sinpi((double)q / (dy + 1));
    }
}

// d' and e' of the block-diagonal B: block j is T_x + mu_j I; e' = 0 across blocks
__global__ void blocks_tridiag(int dx, int dy, double ax, double bx, double ay, double by, double *d, double *e) {
    const int64_t N = (int64_t)dx * dy;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / dx), ix = (int)(q % dx);
        d[q] = bx + by + 2.0 * ay * cospi((double)(j + 1) / (dy + 1));
        if (q + 1 < N) e[q] = (ix + 1 < dx) ? ax : 0.0;
    }
}

// C (M x Nc) = S (M x M) B (M x Nc), binary64, all row-major.  64 x 64 output tiles,
// 16 x 16 threads with 4 x 4 outputs each, K in steps of 16 through shared memory.
__global__ void __launch_bounds__(256) dgemm_s(int M, int64_t Nc, const double *__restrict__ S,
                                               const double *__restrict__ B, double *__restrict__ C) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * 64;
    const int64_t col0 = (int64_t)blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < M; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e & 15, rr = e >> 4;  // As[kk][rr] = S[row0 + rr][k0 + kk]
            const int r = row0 + rr, k = k0 + kk;
            As[kk][rr] = (r < M && k < M) ? S[(int64_t)r * M + k] : 0.0;
            const int cc = e & 63, kb = e >> 6;  // Bs[kb][cc] = B[k0 + kb][col0 + cc]
            const int64_t c = col0 + cc;
            Bs[kb][cc] = (k0 + kb < M && c < Nc) ? B[(int64_t)(k0 + kb) * Nc + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty * 4 + u];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = row0 + ty * 4 + u;
        if (r >= M) continue;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int64_t c = col0 + tx * 4 + w;
            if (c < Nc) C[(int64_t)r * Nc + c] = acc[u][w];
        }
    }
}

cudaError_t apply_s(int dy, int64_t ncols, const double *S, const double *B, double *C, cudaStream_t st,
                    Profiler &prof) {
    return prof.timed("dst_y", st, [&] {
        const dim3 grid((unsigned)((ncols + 63) / 64), (unsigned)((dy + 63) / 64));
        dgemm_s<<<grid, 256, 0, st>>>(dy, ncols, S, B, C);
        return cudaGetLastError();
    });
}

}  // namespace
}  // namespace expm

using namespace expm;

extern "C" expm_status expm_apply_laplacian2d(expm_plan p, int dx, int dy, double ax, double bx, double ay, double by,
                                              const void *V, int r, int v_is_complex, void *Y, const expm_opts *opts_in,
                                              expm_info *info) {
    if (!p) return set_error(EXPM_EINVAL, "apply_laplacian2d: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (dx < 1 || dy < 1 || (int64_t)dx * dy > (1LL << 28) || r < 1 || r > 512)
        return set_error(EXPM_EINVAL, "apply_laplacian2d: need dx, dy >= 1, dx * dy <= 2^28, 1 <= r <= 512");
    if (!std::isfinite(ax) || !std::isfinite(bx) || !std::isfinite(ay) || !std::isfinite(by))
        return set_error(EXPM_EINVAL, "apply_laplacian2d: non-finite coefficients");
    if (!V || !Y || !is_device_ptr(V) || !is_device_ptr(Y))
        return set_error(EXPM_EINVAL, "apply_laplacian2d: V and Y must be device memory");
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)opts.stream;
    const int64_t N = (int64_t)dx * dy;
    const int64_t ncols = (int64_t)dx * r * (v_is_complex ? 2 : 1);  // real columns of V viewed as dy x ncols
    // the tensor-core transform: mixed precisions, an even number of real columns (pairs
    // viewed as complex), within the slice product's limits
    const int64_t kc = ncols / 2;
    const bool tc = opts.prec != EXPM_FP64 && ncols % 2 == 0 && kc <= (1 << 29) && oz_resid_supported(dy, (int)kc, 1);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t oS = 0, oD = oS + al((size_t)dy * dy * 8), oE = oD + al((size_t)N * 8), oW = oE + al((size_t)N * 8),
                 oZ = oW + al((size_t)dy * ncols * 8), oT = oZ + al((size_t)dy * ncols * 8),
                 total = oT + (tc ? al(oz_resid_bytes(dy, (int)kc, 1, 0)) : 0);
    expm_status s = plan_reserve(p, &p->stage, &p->stage_bytes, total);
    if (s != EXPM_OK) return s;
    unsigned char *b = (unsigned char *)p->stage;
    double *S = (double *)(b + oS), *d = (double *)(b + oD), *e = (double *)(b + oE), *W = (double *)(b + oW),
           *Z = (double *)(b + oZ);
    void *ws = b + oT;
    dst_matrix<<<dy, 256, 0, st>>>(dy, S);
    blocks_tridiag<<<(unsigned)std::min<int64_t>((N + 255) / 256, 152 * 8), 256, 0, st>>>(dx, dy, ax, bx, ay, by, d, e);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && tc) err = oz_split_a(dy, S, dy, 0, ws, st);  // slices of S, used by both transforms
    // C = (S x I) B
    auto transform = [&](const double *B, double *C) -> cudaError_t {
        if (!tc) return apply_s(dy, ncols, S, B, C, st, p->prof);
        return p->prof.timed("dst_y<tc>", st, [&] {
            const int64_t nk = (int64_t)dy * kc;
            cudaError_t x = cudaMemsetAsync(C, 0, (size_t)dy * ncols * 8, st);
            if (x == cudaSuccess) x = oz_split_x(dy, (int)kc, 1, 0, (const cx<double> *)B, nk, ws, st);
            if (x == cudaSuccess) x = oz_product(dy, (int)kc, 1, 0, -1.0, nk, (cx<double> *)C, ws, st, nullptr);
            return x;
        });
    };
    if (err == cudaSuccess) err = transform((const double *)V, W);  // W = (S x I) V
    if (err != cudaSuccess) return cuda_error(err, "apply_laplacian2d: transform");
    s = expm_apply_tridiag(p, N, d, e, 0, W, r, v_is_complex, Z, &opts, info);
    if (s != EXPM_OK && s != EXPM_ENOCONV) return s;
    err = transform(Z, (double *)Y);  // Y = (S x I) Z
    if (err != cudaSuccess) return cuda_error(err, "apply_laplacian2d: transform back");
    if (tc) {  // a bounded wait of the tensor-core product that gave up (one synchronisation)
        int to = 0;
        err = oz_read_timeout(dy, (int)kc, 1, 0, ws, st, &to);
        if (err != cudaSuccess) return cuda_error(err, "apply_laplacian2d: transform status");
        if (to) return set_error(EXPM_ETIMEOUT, "apply_laplacian2d: tensor-core transform wait gave up");
    }
    return s;
}
