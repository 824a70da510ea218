// dense_small.cu -- one-launch evaluation of small dense problems (n <= 64, at most 4
// right-hand-side columns, at most 16 solved systems).
//
// Y = sum_s W_s X_s with (tA - cI + theta_s I) X_s = V (eq. expAx; for real A and V one
// member of each conjugate pair with W_s = 2 e^c a_s and Y = Re(...), Remark 5.1).  For
// such sizes the blocked path of dense.cu is bound by its launches (a few hundred
// microseconds for n = 64 whatever the arithmetic), so here everything happens in one
// launch of a thread-block cluster with one CTA per solved system:
//   * the CTA forms M_s = tA - cI + theta_s I and inverts or factors it without pivoting
//     (the Hermitian part of (-i sign(Im theta)) M_s is |Im theta| I, positive definite,
//     so every pivot exists), recording max|M_s| and max|U_s| for the growth check;
//   * binary64 mode: LU in shared memory, then forward and back substitution one warp per
//     right-hand-side column (lanes over rows, the solved entry broadcast by a shuffle);
//   * mixed mode: M_s^{-1} in binary32 by Gauss-Jordan elimination held in registers, so
//     that each refinement sweep is two matrix-vector products with no sequential
//     substitution: D = M~^{-1} R in binary32, X += D, R = V - M_s X in binary64 from A kept
//     in shared memory, with the dense path's stopping test
//     ||R||_F <= tol (||tA||_F + |theta - c|) ||X||_F and at most max_refine corrections;
//   * the CTAs meet at a cluster barrier and CTA 0 adds the weighted solutions of all
//     systems from their shared memory (distributed shared memory), in system order, so
//     the sum is deterministic, writes Y and the worst growth / residual / sweep count.
#include <cooperative_groups.h>

#include <atomic>
#include <cmath>
#include <cstdint>

#include "arith.cuh"
#include "dense.cuh"
#include "plan.cuh"

namespace cg = cooperative_groups;

namespace expm {

namespace {

constexpr int DS_N = 64;       // largest order
constexpr int DS_K = 4;        // largest number of complex right-hand-side columns
constexpr int DS_THREADS = 256;
constexpr int DS_LD = DS_N + 1;  // padded row stride of the shared matrix

using DsArgs = SmallReq;

template <class W> EXPM_D cx<W> cmulW(cx<W> a, cx<W> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class W> EXPM_D cx<W> cfmsW(cx<W> s, cx<W> a, cx<W> b) {  // s - a b
    return {s.re - a.re * b.re + a.im * b.im, s.im - a.re * b.im - a.im * b.re};
}
// 1/w = conj(w) / |w|^2.  The reciprocal of |w|^2 in binary64: a binary32 seed refined by two Newton-Raphson steps r <- r (2 - q r) (the reciprocal
// iteration of Markstein, IBM J. Res. Dev. 34(1), 1990; each step doubles the correct
// bits, 24 -> 48 -> ~96), four FMAs instead of a binary64 division.
EXPM_D double recip_w(double q) {
    double r = (double)__frcp_rn((float)q);
    r = r * fma(-q, r, 2.0);
    r = r * fma(-q, r, 2.0);
    return r;
}
template <class W> EXPM_D cx<W> cinvW(cx<W> w) {
    const W n2 = w.re * w.re + w.im * w.im;
    const W r = recip_w(n2);
    return {w.re * r, -w.im * r};
}
template <class W> EXPM_D W cabs2(cx<W> a) { return a.re * a.re + a.im * a.im; }

// Packed (re, im) pairs of the mixed kernel's registers (pk2 / ffma2 of arith.cuh)
EXPM_D cx<float> upk2c(uint64_t v) {
    cx<float> r;
    upk2(v, r.re, r.im);
    return r;
}

// A_ij of the input (real symmetric or complex Hermitian)
EXPM_D cx<double> load_a(const DsArgs &a, int i, int j) {
    if (a.complex_a) {
        const double *p = a.A + 2 * ((int64_t)i * a.lda + j);
        return {p[0], p[1]};
    }
    return {a.A[(int64_t)i * a.lda + j], 0.0};
}
EXPM_D cx<double> load_v(const DsArgs &a, int i, int c) {
    if (a.v_cplx) {
        const double *p = a.V + 2 * ((int64_t)i * a.ldv + c);
        return {p[0], p[1]};
    }
    return {a.V[(int64_t)i * a.ldv + c], 0.0};
}

// (max of a, sum of b) over the block, both in every thread, one pair of barriers; the sum
// in a fixed order
EXPM_D void block_max_sum(double &a, double &b, double *red) {
    for (int off = 16; off > 0; off >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = a;
        red[DS_THREADS / 32 + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int w = 0; w < DS_THREADS / 32; ++w) {
        a = fmax(a, red[w]);
        b += red[DS_THREADS / 32 + w];
    }
}

// Forward (unit lower L) and back (U) substitution of one column in binary64, one warp:
// lane l owns rows l and l + 32; the row just solved is broadcast from its owner.  Dinv
// holds the reciprocals of U's diagonal.  The loops are split where one half of the rows
// is finished, so that no FP64 warp instruction is issued for it.
EXPM_D void warp_solve(const cx<double> *M, const cx<double> *Dinv, int n, cx<double> &y0, cx<double> &y1) {
    const int lane = threadIdx.x & 31;
    const int r0 = lane, r1 = lane + 32;
    const int nlo = n < 31 ? n : 31;
    for (int j = 0; j < nlo; ++j) {  // rows above 31 and below still change
        const cx<double> yj = {__shfl_sync(0xffffffffu, y0.re, j), __shfl_sync(0xffffffffu, y0.im, j)};
        if (r0 > j) y0 = cfmsW(y0, M[r0 * DS_LD + j], yj);
        if (r1 < n) y1 = cfmsW(y1, M[r1 * DS_LD + j], yj);
    }
    for (int j = nlo; j < n; ++j) {  // only rows 32 and above change
        const double sre = j < 32 ? y0.re : y1.re, sim = j < 32 ? y0.im : y1.im;
        const cx<double> yj = {__shfl_sync(0xffffffffu, sre, j & 31), __shfl_sync(0xffffffffu, sim, j & 31)};
        if (r1 > j && r1 < n) y1 = cfmsW(y1, M[r1 * DS_LD + j], yj);
    }
    for (int j = n - 1; j > 32; --j) {  // x_j in the upper half; both halves change
        cx<double> xj = {__shfl_sync(0xffffffffu, y1.re, j - 32), __shfl_sync(0xffffffffu, y1.im, j - 32)};
        xj = cmulW(xj, Dinv[j]);
        if (lane == j - 32) y1 = xj;
        y0 = cfmsW(y0, M[r0 * DS_LD + j], xj);
        if (r1 < j) y1 = cfmsW(y1, M[r1 * DS_LD + j], xj);
    }
    for (int j = (n - 1 < 32 ? n - 1 : 32); j >= 0; --j) {  // only rows below 32 change
        const double sre = j < 32 ? y0.re : y1.re, sim = j < 32 ? y0.im : y1.im;
        cx<double> xj = {__shfl_sync(0xffffffffu, sre, j & 31), __shfl_sync(0xffffffffu, sim, j & 31)};
        xj = cmulW(xj, Dinv[j]);
        if (j < 32) {
            if (lane == j) y0 = xj;
        } else if (lane == 0) {
            y1 = xj;
        }
        if (r0 < j) y0 = cfmsW(y0, M[r0 * DS_LD + j], xj);
    }
}

// The weighted solutions W_s X_s of all systems, added by CTA 0 in system order through
// distributed shared memory, and the worst growth / residual / sweep count.
EXPM_D void cluster_sum(const DsArgs &a, const DenseSystems &sys, cx<double> *Xs, double *stat) {
    cg::cluster_group cluster = cg::this_cluster();
    const int s = (int)cluster.block_rank(), tid = threadIdx.x;
    const cx<double> wgt = {sys.w_re[s], sys.w_im[s]};
    __syncthreads();
    for (int e = tid; e < a.n * a.kc; e += DS_THREADS) {
        cx<double> &x = Xs[(e / a.kc) * DS_K + e % a.kc];
        x = cmulW(wgt, x);
    }
    cluster.sync();
    if (s == 0) {
        for (int e = tid; e < a.n * a.kc; e += DS_THREADS) {
            const int i = e / a.kc, c = e % a.kc;
            cx<double> acc = {0.0, 0.0};
            for (int r = 0; r < a.nsys; ++r) {
                const cx<double> *xr = cluster.map_shared_rank(Xs, r);
                acc.re += xr[i * DS_K + c].re;
                acc.im += xr[i * DS_K + c].im;
            }
            if (a.y_real) {
                a.Y[(int64_t)i * a.ldy + c] = acc.re;
            } else {
                double *p = a.Y + 2 * ((int64_t)i * a.ldy + c);
                p[0] = acc.re;
                p[1] = acc.im;
            }
        }
        if (tid == 0) {
            double g = 0.0, r = 0.0, sw = 0.0;
            for (int q = 0; q < a.nsys; ++q) {
                const double *st = cluster.map_shared_rank(stat, q);
                g = fmax(g, st[0]);
                r = fmax(r, st[1]);
                sw = fmax(sw, st[2]);
            }
            a.out[0] = g;
            a.out[1] = r;
            a.out[2] = sw;
        }
    }
    cluster.sync();  // the other CTAs' shared memory stays valid until CTA 0 has read it
}

// ---------------------------------------------------------------------------------------
// binary64: unpivoted LU in shared memory, one warp per column for the solves.
EXPM_D void ds_f64_body(const DsArgs &a, const DenseSystems &sys) {
    extern __shared__ __align__(16) unsigned char ds_smem[];
    cx<double> *M = reinterpret_cast<cx<double> *>(ds_smem);                                // DS_N x DS_LD
    cx<double> *Xs = reinterpret_cast<cx<double> *>(ds_smem + sizeof(cx<double>) * DS_N * DS_LD);  // DS_N x DS_K
    __shared__ double red[2 * (DS_THREADS / 32)];
    __shared__ double stat[3];
    __shared__ cx<double> Dinv[DS_N];
    __shared__ cx<double> pinv;  // reciprocal of the next pivot
    const int s = (int)cg::this_cluster().block_rank();
    const int n = a.n, tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const cx<double> dsh = {sys.th_re[s] - sys.cshift, sys.th_im[s]};  // theta - c on the diagonal

    // M_s = tA - cI + theta_s I and max |M_s|^2; thread (ty, tx) takes rows ty + 8r and
    // columns tx + 32c (all sixteen loads in flight at once)
    double mmax = 0.0, unused = 0.0;
#pragma unroll
    for (int r = 0; r < DS_N / 8; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = ty + 8 * r, j = tx + 32 * c;
            if (i < n && j < n) {
                cx<double> m = load_a(a, i, j);
                m = {a.t * m.re, a.t * m.im};
                if (i == j) m = {m.re + dsh.re, m.im + dsh.im};
                M[i * DS_LD + j] = m;
                mmax = fmax(mmax, cabs2(m));
            }
        }
    block_max_sum(mmax, unused, red);
    mmax = sqrt(mmax);
    if (tid == 0) pinv = cinvW(M[0]);
    // unpivoted LU in place: L strictly below the diagonal (unit diagonal), U on and above.
    // The FP64 unit is the bound, so every lane takes trailing entries (no idle columns at
    // the short end); the next pivot's reciprocal is formed as soon as that pivot is final.
    for (int j = 0; j < n - 1; ++j) {
        __syncthreads();
        if (j + 1 + tid < n) {  // n <= 64 < DS_THREADS: one row of the column per thread
            M[(j + 1 + tid) * DS_LD + j] = cmulW(M[(j + 1 + tid) * DS_LD + j], pinv);
        }
        __syncthreads();
        const int w = n - j - 1;
        for (int e = tid; e < w * w; e += DS_THREADS) {
            const int i = j + 1 + e / w, k = j + 1 + e % w;
            const cx<double> v = cfmsW(M[i * DS_LD + k], M[i * DS_LD + j], M[j * DS_LD + k]);
            M[i * DS_LD + k] = v;
            if (e == 0) pinv = cinvW(v);  // (j+1, j+1): the next pivot
        }
    }
    __syncthreads();
    if (tid < n) Dinv[tid] = cinvW(M[tid * DS_LD + tid]);
    double umax = 0.0;
    for (int i = ty; i < n; i += DS_THREADS / 32)
        for (int j = i + tx; j < n; j += 32) umax = fmax(umax, cabs2(M[i * DS_LD + j]));
    block_max_sum(umax, unused, red);
    umax = sqrt(umax);

    const int warp = tid >> 5, lane = tid & 31;
    if (warp < a.kc) {
        const cx<double> v0 = lane < n ? load_v(a, lane, warp) : cx<double>{0, 0};
        const cx<double> v1 = lane + 32 < n ? load_v(a, lane + 32, warp) : cx<double>{0, 0};
        cx<double> y0 = v0, y1 = v1;
        warp_solve(M, Dinv, n, y0, y1);
        if (lane < n) Xs[lane * DS_K + warp] = y0;
        if (lane + 32 < n) Xs[(lane + 32) * DS_K + warp] = y1;
    }
    if (tid == 0) {
        stat[0] = mmax > 0.0 ? umax / mmax : 0.0;
        stat[1] = 0.0;
        stat[2] = 0.0;
    }
    cluster_sum(a, sys, Xs, stat);
}

// ---------------------------------------------------------------------------------------
// mixed: the inverse of M_s in binary32 by Gauss-Jordan elimination held in registers,
// refined against a binary64 residual.
//
// Thread (ty, tx) keeps entries (ty + 8r, tx + 32c), r < 8, c < 2, of a 64 x 64 array
// that holds M_s in its leading n x n block and the identity elsewhere, so elimination
// over the first n pivots leaves M_s^{-1} there.  Step j: the warp holding row j and the
// lane holding column j of every warp publish them to shared memory (double-buffered,
// one barrier per step); every thread then forms the reciprocal of the pivot and updates
// its sixteen entries:  pivot row  M_jk <- M_jk / M_jj,  M_jj <- 1 / M_jj;  other rows
// M_ik <- M_ik - M_ij M_jk / M_jj,  M_ij <- -M_ij / M_jj.  Row j as published at step j
// is row j of U in the LU factorization (the same updates with the same multipliers), so
// max |U| for the growth check is taken from it.  A sweep is then two matrix-vector
// products: D = M~^{-1} R (binary32) and R = V - M_s X (binary64, from A in shared memory).
constexpr int DS_Q = DS_THREADS / DS_N;  // column chunks of the matrix-vector products (4)

// KC = number of right-hand-side columns (a template argument, so that no binary64 warp
// instruction is issued for absent columns).
template <int KC>
EXPM_D void ds_mixed_body(const DsArgs &a, const DenseSystems &sys) {
    extern __shared__ __align__(16) unsigned char ds_smem[];
    cx<float> *MT = reinterpret_cast<cx<float> *>(ds_smem);  // DS_N x DS_LD: (M~^{-1})^T
    unsigned char *p = ds_smem + sizeof(cx<float>) * DS_N * DS_LD;
    void *As = p;  // DS_N x DS_LD: A (double or complex double), zero outside n x n
    p += sizeof(cx<double>) * DS_N * DS_LD;
    cx<double> *Xs = reinterpret_cast<cx<double> *>(p);  // DS_N x DS_K
    p += sizeof(cx<double>) * DS_N * DS_K;
    cx<double> *Ps = reinterpret_cast<cx<double> *>(p);  // DS_Q x DS_N x DS_K partial sums
    cx<float> *Pf = reinterpret_cast<cx<float> *>(p);    // (the binary32 ones alias them)
    p += sizeof(cx<double>) * DS_Q * DS_N * DS_K;
    cx<float> *Rf = reinterpret_cast<cx<float> *>(p);  // DS_N x DS_K: residual in binary32
    __shared__ uint64_t rowbuf[2][DS_N], colbuf[2][DS_N];  // packed (re, im) pairs
    __shared__ double red[2 * (DS_THREADS / 32)];
    __shared__ double tot[3];  // ||R||^2, ||X||^2, stop
    __shared__ double stat[3];
    const int s = (int)cg::this_cluster().block_rank();
    const int n = a.n, tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const cx<double> dsh = {sys.th_re[s] - sys.cshift, sys.th_im[s]};  // theta - c on the diagonal
    double *Ar = reinterpret_cast<double *>(As);
    cx<double> *Ac = reinterpret_cast<cx<double> *>(As);

    // A into shared memory (binary64) and M_s into registers (binary32), with max |M_s|^2
    // and ||tA||_F^2 (binary32: this mode takes tA within binary32 range); all sixteen
    // loads of a thread in flight at once
    const float tw = (float)a.t;
    const cx<float> dw = {(float)dsh.re, (float)dsh.im};
    cx<float> m[DS_N / 8][2];
    float mmax_f = 0.0f, a2_f = 0.0f;
#pragma unroll
    for (int r = 0; r < DS_N / 8; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = ty + 8 * r, j = tx + 32 * c;
            const bool in = i < n && j < n;
            const cx<double> ad = in ? load_a(a, i, j) : cx<double>{0.0, 0.0};
            if (a.complex_a)
                Ac[i * DS_LD + j] = ad;
            else
                Ar[i * DS_LD + j] = ad.re;
            const cx<float> af = {(float)ad.re, (float)ad.im};
            cx<float> v = {tw * af.re, tw * af.im};
            a2_f += cabs2(v);
            if (i == j) v = in ? cx<float>{v.re + dw.re, v.im + dw.im} : cx<float>{1.0f, 0.0f};
            m[r][c] = v;
            if (in) mmax_f = fmaxf(mmax_f, cabs2(v));
        }
    double mmax = (double)mmax_f, a2 = (double)a2_f;
    block_max_sum(mmax, a2, red);
    mmax = sqrt(mmax);
    const double anorm = sqrt(a2);  // ||tA||_F

    // Gauss-Jordan over the first n pivots on packed (re, im) pairs: the update of an entry,
    // M_ik - l uh with l = M_ij and uh = M_jk / M_jj, is two fma.rn.f32x2:
    //   (re, im) += (l.re, l.re) * (-uh.re, -uh.im);  (re, im) += (l.im, l.im) * (uh.im, -uh.re).
    // Column j takes the identity's column in place: the lane holding it publishes and then
    // zeroes its entries, and uh_j = 1 / M_jj, so the same update leaves -l / M_jj there; the
    // pivot row is then overwritten with uh by the warp holding it.
    uint64_t mp[DS_N / 8][2];
#pragma unroll
    for (int r = 0; r < DS_N / 8; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) mp[r][c] = pk2(m[r][c].re, m[r][c].im);
    float umax_f = 0.0f;
    for (int j = 0; j < n; ++j) {
        const int b = j & 1, rj = j >> 3, cj = j >> 5;
        if (ty == (j & 7)) {
#pragma unroll
            for (int r = 0; r < DS_N / 8; ++r)
                if (r == rj) {
                    rowbuf[b][tx] = mp[r][0];
                    rowbuf[b][tx + 32] = mp[r][1];
                }
        }
        if (tx == (j & 31)) {
#pragma unroll
            for (int r = 0; r < DS_N / 8; ++r) {
                colbuf[b][ty + 8 * r] = cj ? mp[r][1] : mp[r][0];
                if (cj)
                    mp[r][1] = 0;
                else
                    mp[r][0] = 0;
            }
        }
        __syncthreads();
        const cx<float> piv = upk2c(rowbuf[b][j]);
        const float q = __frcp_rn(piv.re * piv.re + piv.im * piv.im);
        const cx<float> inv = {piv.re * q, -piv.im * q};
        uint64_t ua[2], ub[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const cx<float> u = upk2c(rowbuf[b][tx + 32 * c]);
            if (tx + 32 * c >= j) umax_f = fmaxf(umax_f, cabs2(u));
            const cx<float> uh = (tx + 32 * c == j) ? inv : cmulW(u, inv);
            ua[c] = pk2(-uh.re, -uh.im);
            ub[c] = pk2(uh.im, -uh.re);
        }
#pragma unroll
        for (int r = 0; r < DS_N / 8; ++r) {
            const cx<float> l = upk2c(colbuf[b][ty + 8 * r]);
            const uint64_t lr = pk2(l.re, l.re), li = pk2(l.im, l.im);
#pragma unroll
            for (int c = 0; c < 2; ++c) mp[r][c] = ffma2(li, ub[c], ffma2(lr, ua[c], mp[r][c]));
        }
        if (ty == (j & 7)) {
#pragma unroll
            for (int r = 0; r < DS_N / 8; ++r)
                if (r == rj) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const cx<float> na = upk2c(ua[c]);
                        mp[r][c] = pk2(-na.re, -na.im);
                    }
                }
        }
    }
    // (M~^{-1})^T into shared memory for the column-chunked products
#pragma unroll
    for (int r = 0; r < DS_N / 8; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) MT[(tx + 32 * c) * DS_LD + ty + 8 * r] = upk2c(mp[r][c]);
    double umax = (double)umax_f, unused = 0.0;
    block_max_sum(umax, unused, red);
    umax = sqrt(umax);

    // X = 0, R = V; sweep: D = M~^{-1} R, X += D, R = V - (tA - cI + theta I) X.
    // Thread (row i, chunk q) sums columns 16q .. 16q+15 of its row; thread (i, column c)
    // adds the DS_Q chunks in order and owns X_ic, V_ic and R_ic.
    const int ri = tid & (DS_N - 1), rq = tid / DS_N;
    const bool owner = rq < KC;  // thread (ri, c = rq)
    const cx<double> vi = owner && ri < n ? load_v(a, ri, rq) : cx<double>{0.0, 0.0};
    if (owner) {
        Xs[ri * DS_K + rq] = {0.0, 0.0};
        Rf[ri * DS_K + rq] = {(float)vi.re, (float)vi.im};
    }
    const double tol2 = a.tol * a.tol, dshn = sqrt(cabs2(dsh));
    const double den2 = (anorm + dshn) * (anorm + dshn);
    double rn2 = 0.0, xn2 = 0.0;
    int it = 0;
    for (;; ++it) {
        __syncthreads();
        {  // D partial sums (binary32)
            cx<float> acc[KC];
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[c] = {0.0f, 0.0f};
#pragma unroll 4
            for (int jj = 0; jj < DS_N / DS_Q; ++jj) {
                const int j = rq * (DS_N / DS_Q) + jj;
                const cx<float> g = MT[j * DS_LD + ri];
#pragma unroll
                for (int c = 0; c < KC; ++c) {
                    const cx<float> rv = Rf[j * DS_K + c];
                    acc[c] = {fmaf(g.re, rv.re, fmaf(-g.im, rv.im, acc[c].re)),
                              fmaf(g.re, rv.im, fmaf(g.im, rv.re, acc[c].im))};
                }
            }
#pragma unroll
            for (int c = 0; c < KC; ++c) Pf[(rq * DS_N + ri) * DS_K + c] = acc[c];
        }
        __syncthreads();
        if (owner) {
            cx<float> d = {0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < DS_Q; ++q) {
                const cx<float> t = Pf[(q * DS_N + ri) * DS_K + rq];
                d = {d.re + t.re, d.im + t.im};
            }
            cx<double> &x = Xs[ri * DS_K + rq];
            x = {x.re + (double)d.re, x.im + (double)d.im};
        }
        __syncthreads();
        {  // A X partial sums (binary64)
            cx<double> acc[KC];
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[c] = {0.0, 0.0};
            if (a.complex_a) {
#pragma unroll 4
                for (int jj = 0; jj < DS_N / DS_Q; ++jj) {
                    const int j = rq * (DS_N / DS_Q) + jj;
                    const cx<double> g = Ac[ri * DS_LD + j];
#pragma unroll
                    for (int c = 0; c < KC; ++c) {
                        const cx<double> xv = Xs[j * DS_K + c];
                        acc[c] = {fma(g.re, xv.re, fma(-g.im, xv.im, acc[c].re)),
                                  fma(g.re, xv.im, fma(g.im, xv.re, acc[c].im))};
                    }
                }
            } else {  // real A: two binary64 FMAs per entry and column
#pragma unroll 4
                for (int jj = 0; jj < DS_N / DS_Q; ++jj) {
                    const int j = rq * (DS_N / DS_Q) + jj;
                    const double g = Ar[ri * DS_LD + j];
#pragma unroll
                    for (int c = 0; c < KC; ++c) {
                        const cx<double> xv = Xs[j * DS_K + c];
                        acc[c] = {fma(g, xv.re, acc[c].re), fma(g, xv.im, acc[c].im)};
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < KC; ++c) Ps[(rq * DS_N + ri) * DS_K + c] = acc[c];
        }
        __syncthreads();
        rn2 = 0.0;
        xn2 = 0.0;
        if (owner) {
            cx<double> ax = {0.0, 0.0};
#pragma unroll
            for (int q = 0; q < DS_Q; ++q) {
                const cx<double> t = Ps[(q * DS_N + ri) * DS_K + rq];
                ax = {ax.re + t.re, ax.im + t.im};
            }
            const cx<double> xi = Xs[ri * DS_K + rq];
            const cx<double> r = {vi.re - (a.t * ax.re + dsh.re * xi.re - dsh.im * xi.im),
                                  vi.im - (a.t * ax.im + dsh.re * xi.im + dsh.im * xi.re)};
            Rf[ri * DS_K + rq] = {(float)r.re, (float)r.im};
            rn2 = cabs2(r);
            xn2 = cabs2(xi);
        }
        // ||R||_F <= tol (||tA||_F + |theta - c|) ||X||_F, squared: the owner warps reduce,
        // warp 0 adds their sums in order and decides for the block
        if (tid < DS_N * KC) {
            for (int off = 16; off > 0; off >>= 1) {
                rn2 += __shfl_xor_sync(0xffffffffu, rn2, off);
                xn2 += __shfl_xor_sync(0xffffffffu, xn2, off);
            }
            if (tx == 0) {
                red[ty] = rn2;
                red[DS_THREADS / 32 + ty] = xn2;
            }
        }
        __syncthreads();
        if (ty == 0) {
            rn2 = tx < DS_N * KC / 32 ? red[tx] : 0.0;
            xn2 = tx < DS_N * KC / 32 ? red[DS_THREADS / 32 + tx] : 0.0;
            for (int off = 4; off > 0; off >>= 1) {  // lanes 0 .. 7 (2 KC <= 8 owner warps), fixed order
                rn2 += __shfl_xor_sync(0xffffffffu, rn2, off);
                xn2 += __shfl_xor_sync(0xffffffffu, xn2, off);
            }
            if (tx == 0) {
                tot[0] = rn2;
                tot[1] = xn2;
                tot[2] = (rn2 <= tol2 * den2 * xn2 || it >= a.max_refine) ? 1.0 : 0.0;
            }
        }
        __syncthreads();
        if (tot[2] != 0.0) break;
    }
    rn2 = tot[0];
    xn2 = tot[1];
    if (tid == 0) {
        const double den = sqrt(den2 * xn2);
        stat[0] = mmax > 0.0 ? umax / mmax : 0.0;
        stat[1] = den > 0.0 ? sqrt(rn2) / den : 0.0;
        stat[2] = (double)it;
    }
    cluster_sum(a, sys, Xs, stat);
}

__global__ void __launch_bounds__(DS_THREADS) dense_small_f64_kernel(DsArgs a, DenseSystems sys) {
    ds_f64_body(a, sys);
}
template <int KC>
__global__ void __launch_bounds__(DS_THREADS, 1) dense_small_mixed_kernel(DsArgs a, DenseSystems sys) {
    ds_mixed_body<KC>(a, sys);
}

// ---------------------------------------------------------------------------------------
// Device-fed queue: a persistent kernel of `nclusters` clusters of nsys CTAs.  Thread 0 of
// each cluster's CTA 0 claims the next ticket (atomic counter), waits until the host has
// published that ticket's request in mapped host memory (sequence word = ticket + 1),
// broadcasts it to the cluster's CTAs through distributed shared memory, and after the
// evaluation -- the same body as the one-launch kernels -- publishes ticket + 1 as the
// slot's completion word (system-scope release after a system fence, so Y and the slot's
// statistics are visible first).  Every wait is bounded: a cluster that waits longer than
// idle_ns for a request sets the device halt flag and the ETIMEOUT exit status, and every
// cluster leaves at its next claim once halt or the host's stop flag is set (a request
// already being evaluated is finished first).  After a restart the claim counter starts at
// the host's oldest unfinished ticket; tickets already completed are skipped.
EXPM_D unsigned long long ld_acquire_sys(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
EXPM_D unsigned ld_relaxed_sys(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
EXPM_D void st_release_sys(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
EXPM_D long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int MODE>
__global__ void __launch_bounds__(DS_THREADS, 1) dense_small_queue_kernel(SmallQueueArgs q) {
    __shared__ DsArgs s_a;
    __shared__ DenseSystems s_sys;
    __shared__ unsigned long long s_ticket;
    __shared__ int s_go;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank(), tid = threadIdx.x;
    bool timed_out = false;
    for (;;) {
        if (rank == 0 && tid == 0) {
            int go = 0;
            unsigned long long t = 0;
            if (!ld_relaxed_sys(q.halt) && !ld_relaxed_sys(q.stop)) {
                t = atomicAdd(q.claim, 1ull);
                const long long t0 = global_ns();
                for (;;) {
                    if (ld_acquire_sys(q.seq + t % q.cap) == t + 1) {
                        if (ld_acquire_sys(q.done + t % q.cap) == t + 1) {  // completed before a restart
                            t = atomicAdd(q.claim, 1ull);
                            continue;
                        }
                        go = 1;
                        break;
                    }
                    if (ld_relaxed_sys(q.halt) || ld_relaxed_sys(q.stop)) break;
                    if (global_ns() - t0 > q.idle_ns) {
                        atomicExch(q.halt, 1u);
                        timed_out = true;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            for (int r = 0; r < q.nsys; ++r) {
                *cluster.map_shared_rank(&s_go, r) = go;
                *cluster.map_shared_rank(&s_ticket, r) = t;
            }
        }
        cluster.sync();
        if (!s_go) break;
        const int slot = (int)(s_ticket % (unsigned long long)q.cap);
        // every CTA acquires the published sequence word itself (system scope, on its own
        // SM), so that its loads of the slot and of the request's A and V see what the host
        // ordered before publishing, not lines cached by an earlier request
        if (tid == 0) (void)ld_acquire_sys(q.seq + slot);
        __syncthreads();
        {  // the request into shared memory (one 8-byte word per thread and pass)
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&q.slots[slot].sys);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_sys);
            for (int w = tid; w < (int)(sizeof(DenseSystems) / 8); w += DS_THREADS) dst[w] = __ldcv(src + w);
            const unsigned long long *sa = reinterpret_cast<const unsigned long long *>(&q.slots[slot].a);
            unsigned long long *da = reinterpret_cast<unsigned long long *>(&s_a);
            if (tid < (int)(sizeof(DsArgs) / 8)) da[tid] = __ldcv(sa + tid);
        }
        __syncthreads();
        if (tid == 0) s_a.out = q.stat + 3 * slot;
        __syncthreads();
        if constexpr (MODE == 0) {
            ds_f64_body(s_a, s_sys);
        } else {
            ds_mixed_body<MODE>(s_a, s_sys);
        }
        if (rank == 0 && tid == 0) {  // Y and the statistics first, then the completion word
            __threadfence_system();
            st_release_sys(q.done + slot, s_ticket + 1);
        }
    }
    if (rank == 0 && tid == 0 && timed_out) atomicExch(q.exit_status, (unsigned)EXPM_ETIMEOUT);
}

constexpr size_t DS_SMEM_F64 = sizeof(cx<double>) * DS_N * DS_LD + sizeof(cx<double>) * DS_N * DS_K;
constexpr size_t DS_SMEM_MIXED = sizeof(cx<float>) * DS_N * DS_LD + sizeof(cx<double>) * DS_N * DS_LD +
                                 sizeof(cx<double>) * DS_N * DS_K + sizeof(cx<double>) * DS_Q * DS_N * DS_K +
                                 sizeof(cx<float>) * DS_N * DS_K;

// Kernel attributes (dynamic shared memory, cluster size) are per device: set once for
// each kernel variant and device, so that a launch inside stream capture makes no other
// API call.
constexpr int DS_VARIANTS = 5, DS_MAXDEV = 64;
std::atomic<unsigned char> ds_attr_set[DS_VARIANTS][DS_MAXDEV];

template <class K>
cudaError_t launch_small(K kernel, int variant, size_t smem, const DsArgs &a, const DenseSystems &sys, int nsys,
                         cudaStream_t st, Profiler &prof, const char *name) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)nsys);
    cfg.blockDim = dim3(DS_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nsys;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= DS_MAXDEV || !ds_attr_set[variant][dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < DS_MAXDEV) ds_attr_set[variant][dev].store(1, std::memory_order_release);
    }
    return prof.timed(name, st, [&] { return cudaLaunchKernelEx(&cfg, kernel, a, sys); });
}

}  // namespace

namespace {
constexpr size_t ds_smem_of(int mode) { return mode == 0 ? DS_SMEM_F64 : DS_SMEM_MIXED; }

template <int MODE>
cudaLaunchConfig_t queue_config(int nsys, int nclusters, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(nsys * nclusters));
    cfg.blockDim = dim3(DS_THREADS);
    cfg.dynamicSmemBytes = ds_smem_of(MODE);
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nsys;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <int MODE>
cudaError_t queue_attrs() {
    auto k = dense_small_queue_kernel<MODE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ds_smem_of(MODE));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int MODE>
cudaError_t queue_launch(const SmallQueueArgs &q, int nclusters, cudaStream_t st) {
    cudaError_t e = queue_attrs<MODE>();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = queue_config<MODE>(q.nsys, nclusters, st, attr);
    return cudaLaunchKernelEx(&cfg, dense_small_queue_kernel<MODE>, q);
}

template <int MODE>
int queue_clusters(int nsys) {
    if (queue_attrs<MODE>() != cudaSuccess) return 0;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = queue_config<MODE>(nsys, 1, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, dense_small_queue_kernel<MODE>, &cfg) != cudaSuccess) return 0;
    return n;
}
}  // namespace

cudaError_t dense_small_queue_launch(const SmallQueueArgs &q, int mode, int nclusters, cudaStream_t st) {
    if (q.nsys < 1 || q.nsys > 16 || nclusters < 1 || q.cap < 1) return cudaErrorInvalidValue;
    switch (mode) {
        case 0: return queue_launch<0>(q, nclusters, st);
        case 1: return queue_launch<1>(q, nclusters, st);
        case 2: return queue_launch<2>(q, nclusters, st);
        case 3: return queue_launch<3>(q, nclusters, st);
        case 4: return queue_launch<4>(q, nclusters, st);
    }
    return cudaErrorInvalidValue;
}

int dense_small_queue_max_clusters(int mode, int nsys) {
    switch (mode) {
        case 0: return queue_clusters<0>(nsys);
        case 1: return queue_clusters<1>(nsys);
        case 2: return queue_clusters<2>(nsys);
        case 3: return queue_clusters<3>(nsys);
        case 4: return queue_clusters<4>(nsys);
    }
    return 0;
}

bool dense_small_fits(const DenseGeom &g) {
    return g.ninst == 1 && g.n <= DS_N && g.kc <= DS_K && g.nsys >= 1 && g.nsys <= 16;
}

size_t dense_small_workspace_bytes() { return 256; }

cudaError_t dense_small_launch(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, double *out,
                               cudaStream_t st, Profiler &prof) {
    DsArgs a{};
    a.n = g.n;
    a.kc = g.kc;
    a.nsys = g.nsys;
    a.complex_a = g.complex_a;
    a.v_cplx = io.v_cplx;
    a.y_real = io.y_real;
    a.mixed = g.mixed;
    a.max_refine = g.max_refine;
    a.t = g.t;
    a.tol = g.tol;
    a.A = io.A;
    a.lda = io.lda;
    a.V = io.V;
    a.ldv = io.ldv;
    a.Y = io.Y;
    a.ldy = io.ldy;
    a.out = out;
    if (!g.mixed)
        return launch_small(dense_small_f64_kernel, 0, DS_SMEM_F64, a, sys, g.nsys, st, prof, "dense_small<f64>");
    if (g.kc == 1)
        return launch_small(dense_small_mixed_kernel<1>, 1, DS_SMEM_MIXED, a, sys, g.nsys, st, prof, "dense_small<f32>");
    if (g.kc == 2)
        return launch_small(dense_small_mixed_kernel<2>, 2, DS_SMEM_MIXED, a, sys, g.nsys, st, prof, "dense_small<f32>");
    if (g.kc == 3)
        return launch_small(dense_small_mixed_kernel<3>, 3, DS_SMEM_MIXED, a, sys, g.nsys, st, prof, "dense_small<f32>");
    return launch_small(dense_small_mixed_kernel<4>, 4, DS_SMEM_MIXED, a, sys, g.nsys, st, prof, "dense_small<f32>");
}

cudaError_t dense_small_run(const DenseGeom &g, const DenseIO &io, const DenseSystems &sys, void *work,
                            cudaStream_t st, Profiler &prof, DenseResult *res) {
    cudaError_t err = dense_small_launch(g, io, sys, (double *)work, st, prof);
    if (err != cudaSuccess) return err;
    double h[3];
    err = cudaMemcpyAsync(h, work, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return err;
    res->tc_timeout = 0;
    res->growth_max = h[0];
    res->resid_rel_max = h[1];
    res->iters = (int)h[2];
    res->inst_iters.assign(1, res->iters);
    res->inst_resid.assign(1, h[1]);
    res->inst_growth.assign(1, h[0]);
    return cudaSuccess;
}

}  // namespace expm
