// plan.cuh -- the opaque plan object behind expm_plan and shared host helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/expm.h"

namespace expm {
// Per-kernel CUDA-event timing (see expm_profile_enable).
struct Profiler {
    struct Pending {
        int kernel;
        cudaEvent_t a, b;
    };
    bool on = false;
    std::vector<const char *> names;
    std::vector<long long> launches;
    std::vector<double> total_ms;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int kernel_index(const char *name);
    cudaEvent_t take();
    // record an event pair around `launch` (a callable returning cudaError_t)
    template <class F> cudaError_t timed(const char *name, cudaStream_t st, F &&launch) {
        if (!on) return launch();
        Pending p{kernel_index(name), take(), take()};
        cudaEventRecord(p.a, st);
        cudaError_t e = launch();
        cudaEventRecord(p.b, st);
        pending.push_back(p);
        return e;
    }
    void flush();   // synchronise pending events and accumulate
    void reset();
    void release();
};
}  // namespace expm

struct expm_plan_s {
    uint64_t id = 0;          // unique per plan over the process (never reused, unlike the address)
    int degree = 0;
    int device = 0;
    int sm_count = 0;
    std::vector<double> lam;  // poles lambda_k, interleaved re/im (2*degree)
    std::vector<double> w;    // weights w_k = a_k, interleaved re/im (2*degree)
    void *work = nullptr;     // device workspace for the kernels
    size_t work_bytes = 0;
    void *stage = nullptr;    // device staging area for host buffers
    size_t stage_bytes = 0;
    cudaStream_t copy = nullptr;            // second stream: host-to-device copies that overlap kernels
    cudaEvent_t ev_fork = nullptr, ev_copied = nullptr;
    expm::Profiler prof;
};

namespace expm {

expm_status set_error(expm_status s, const std::string &msg);
expm_status cuda_error(cudaError_t e, const char *where);
bool is_device_ptr(const void *p);
expm_status plan_reserve(expm_plan p, void **buf, size_t *have, size_t need);
bool plan_copy_stream(expm_plan p);

// Makes a device current for the lifetime of the object and restores the previous one.
class DeviceGuard {
  public:
    explicit DeviceGuard(int dev);
    ~DeviceGuard();

  private:
    int prev_ = 0;
};

}  // namespace expm
