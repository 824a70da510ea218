// tridiag_noalloc.cu -- the tridiagonal path with a fixed, library-owned scratch area.
//
// expm_apply_tridiag normally sizes its scratch on first use and grows it with
// cudaMalloc.  Some callers cannot allow that: a serving process whose device
// memory is reserved up front by another framework's caching allocator, or a
// latency-critical loop that must never hit cudaMalloc/cudaFree (they can
// synchronise the device and take unbounded time).  For them this file provides
// expm_apply_tridiag_noalloc, which runs the same kernels with their scratch in a
// file-scope __device__ array of EXPM_NOALLOC_SCRATCH_BYTES bytes.  The array is
// part of the module: every GPU that loads the library holds it until the process
// exits.
#include <cmath>
#include <mutex>

#include "../../include/expm.h"
#include "plan.cuh"
#include "tridiag.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[EXPM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `dev` (which must be current).  In host
// code the symbol itself is only a host-side stand-in, so the address is queried
// once per device and cached.
cudaError_t scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

using namespace expm;

extern "C" expm_status expm_apply_tridiag_noalloc(expm_plan p, int64_t N, const double *d, const void *e,
                                                  int e_is_complex, const void *V, int r, int v_is_complex, void *Y,
                                                  const expm_opts *opts_in, expm_info *info) {
    if (!p) return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: NULL plan");
    expm_opts opts;
    if (opts_in) opts = *opts_in; else expm_opts_default(&opts);
    if (N < 1) return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: N must be >= 1");
    if (r < 1 || r > 64) return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: r must be in 1..64");
    if (!d || !V || !Y || (N > 1 && !e)) return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: NULL data pointer");
    if (opts.prec != EXPM_FP64 && opts.prec != EXPM_MIXED_F32X2)
        return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: precision must be EXPM_FP64 or EXPM_MIXED_F32X2");
    if (opts.flags != 0) return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: opts.flags must be 0");
    if (!std::isfinite(opts.t) || !std::isfinite(opts.shift_c))
        return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: t and shift_c must be finite");
    if (info) *info = expm_info{0, 0.0, 0.0, EXPM_OK};

    DeviceGuard guard(p->device);
    // host buffers would need device staging memory: this entry point takes device pointers only
    if (!is_device_ptr(d) || (N > 1 && !is_device_ptr(e)) || !is_device_ptr(V) || !is_device_ptr(Y))
        return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: d, e, V and Y must be device memory");

    const bool ff = opts.prec == EXPM_MIXED_F32X2;
    const bool herm = e_is_complex != 0;  // complex T: solved as D^H T D (real) on D^H V
    const int Rc = herm ? 2 * r : r * (v_is_complex ? 2 : 1);
    const int S = p->degree / 2;
    TriPoles ps{};
    const double ec = std::exp(opts.shift_c);
    for (int s = 0; s < S; ++s) {
        ps.th_re[s] = -p->lam[4 * s];
        ps.th_im[s] = -p->lam[4 * s + 1];
        ps.w_re[s] = 2.0 * ec * p->w[4 * s];
        ps.w_im[s] = 2.0 * ec * p->w[4 * s + 1];
    }
    TriGeom g = tri_geometry(N, S, Rc, ff, p->sm_count);
    g.t = opts.t;
    g.cshift = opts.shift_c;
    const size_t base_need = tri_workspace_bytes(g, ff);
    const size_t herm_off = (base_need + 255) & ~(size_t)255;
    const size_t need = herm ? herm_off + herm_scratch_bytes(N, r) : base_need;
    if (need > (size_t)EXPM_NOALLOC_SCRATCH_BYTES)
        return set_error(EXPM_EINVAL, "apply_tridiag_noalloc: problem needs " + std::to_string(need) +
                                          " bytes of scratch, more than the fixed " +
                                          std::to_string((size_t)EXPM_NOALLOC_SCRATCH_BYTES) +
                                          " (EXPM_NOALLOC_SCRATCH_BYTES); use expm_apply_tridiag");
    void *scratch = nullptr;
    cudaError_t err = scratch_address(p->device, &scratch);
    if (err != cudaSuccess) return cuda_error(err, "apply_tridiag_noalloc: cudaGetSymbolAddress");
    Profiler off;  // no event timing: this path creates no CUDA objects
    const cudaStream_t st = (cudaStream_t)opts.stream;
    const double *dE = (const double *)e, *dV = (const double *)V;
    HermWork hw{};
    if (herm) {
        hw = herm_carve((unsigned char *)scratch + herm_off, N, r);
        err = herm_prepare(N, dE, dV, r, v_is_complex, hw, p->sm_count, st);
        if (err != cudaSuccess) return cuda_error(err, "apply_tridiag_noalloc: Hermitian phases");
        dE = hw.eabs;
        dV = hw.Vp;
    }
    err = tri_run(g, ff, d, dE, dV, (double *)Y, ps, scratch, st, off);
    if (err == cudaSuccess && herm) err = herm_finish(N, r, hw, (double *)Y, p->sm_count, st);
    if (err != cudaSuccess) return cuda_error(err, "apply_tridiag_noalloc: kernel launch");
    return EXPM_OK;
}
