// C-ABI of the selection library: contexts, workspace, argument checks and launches.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"
#include "select.cuh"
#include "api_internal.h"

using namespace gbs;

namespace {
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// One CTA at a grid barrier that counts two arrivals: the barrier can never complete, so
// its bounded wait gives up after limit_ns and records GBS_ETIMEOUT (the failure path of
// every persistent launch, taken without a fault).
__global__ void wait_probe_kernel(Ctrl* c, unsigned long long limit_ns) {
  if (!grid_sync(c, 2u, limit_ns)) return;
  if (threadIdx.x == 0) atomicCAS(&c->status, 0, (int)GBS_EINTERNAL);   // the barrier passed: impossible
}
}  // namespace

// ---------------------------------------------------------------------------------
// Workspace.
// ---------------------------------------------------------------------------------
gbs_status gbs_internal_ensure(gbs_ctx* c, size_t z_bytes) {
  size_t fixed = 0;
  const size_t o_ctrl = fixed; fixed += align_up(sizeof(Ctrl), 256);
  const size_t o_part = fixed; fixed += align_up(sizeof(PassPartial) * 2 * kMaxGrid, 256);
  const size_t o_spart = fixed; fixed += align_up(sizeof(StatsPartial) * kMaxGrid, 256);
  const size_t o_ghist = fixed; fixed += align_up(sizeof(unsigned long long) * kMaxRounds * kBins, 256);
  const size_t o_rs = fixed; fixed += align_up(sizeof(gbs_run_stats), 256);
  const size_t o_aux = fixed; fixed += align_up(c->aux_bytes, 256);
  const size_t o_z = fixed;
  const size_t need = o_z + align_up(z_bytes, 256);
  if (c->ws && c->ws_bytes >= need) return GBS_OK;
  // grow (synchronous): keep at least what was reserved before
  size_t want = std::max(need, c->ws_bytes);
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ENOMEM;
  }
  if (cudaMemset(p, 0, o_z) != cudaSuccess) {
    cudaFree(p);
    return GBS_ECUDA;
  }
  c->ws = p;
  c->ws_bytes = want;
  char* b = static_cast<char*>(p);
  c->ctrl = reinterpret_cast<Ctrl*>(b + o_ctrl);
  c->part = reinterpret_cast<PassPartial*>(b + o_part);
  c->spart = reinterpret_cast<StatsPartial*>(b + o_spart);
  c->ghist = reinterpret_cast<unsigned long long*>(b + o_ghist);
  c->rs = reinterpret_cast<gbs_run_stats*>(b + o_rs);
  c->aux = b + o_aux;
  c->z = b + o_z;
  c->z_bytes = want - o_z;
  return GBS_OK;
}

template <typename T>
static gbs_status select_checked(gbs_ctx* c, const T* x, int64_t n, int64_t k, T* out, void* stream) {
  if (!c || !x || !out) return GBS_EINVAL;
  if (n < 1 || k < 1 || k > n) return GBS_EINVAL;
  if (reinterpret_cast<uintptr_t>(x) % sizeof(T) != 0) return GBS_EINVAL;
  return run_select(c, x, n, k, out, kModeSelect, 0.0, 0.0, nullptr, nullptr,
                    static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------------
// C-ABI.
// ---------------------------------------------------------------------------------
extern "C" {

gbs_status gbs_create(gbs_ctx** out, int device) {
  if (!out) return GBS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  if (device < 0 || device >= ndev) return GBS_EINVAL;
  gbs_ctx* c = new (std::nothrow) gbs_ctx();
  if (!c) return GBS_ENOMEM;
  c->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete c;
    return GBS_ECUDA;
  }
  if (!prop.cooperativeLaunch) {
    delete c;
    return GBS_ECUDA;
  }
  c->num_sms = prop.multiProcessorCount;
  std::memset(&c->cfg, 0, sizeof(c->cfg));
  *out = c;
  return GBS_OK;
}

void gbs_destroy(gbs_ctx* c) {
  if (!c) return;
  {
    DeviceGuard g(c->device);
    gbs_internal_release(c);
    if (c->ws) {
      cudaDeviceSynchronize();
      cudaFree(c->ws);
    }
  }
  delete c;
}

gbs_status gbs_reserve(gbs_ctx* c, int64_t n, int32_t elem_bytes) {
  if (!c || n < 1 || (elem_bytes != 4 && elem_bytes != 8)) return GBS_EINVAL;
  return reserve_select(c, n, elem_bytes);
}

gbs_status gbs_set_config(gbs_ctx* c, const gbs_config* cfg) {
  if (!c || !cfg) return GBS_EINVAL;
  if (cfg->cap < 0 || cfg->maxit < 0 || cfg->blocks_per_sm < 0) return GBS_EINVAL;
  if (cfg->lms_start < 0 || cfg->lms_start > 1) return GBS_EINVAL;
  if (cfg->knn_start < 0 || cfg->knn_start > 1) return GBS_EINVAL;
  c->cfg = *cfg;
  return GBS_OK;
}

gbs_status gbs_get_config(gbs_ctx* c, gbs_config* cfg) {
  if (!c || !cfg) return GBS_EINVAL;
  *cfg = c->cfg;
  return GBS_OK;
}

gbs_status gbs_select_kth_f32(gbs_ctx* c, const float* x, int64_t n, int64_t k, float* out, void* stream) {
  return select_checked<float>(c, x, n, k, out, stream);
}
gbs_status gbs_select_kth_f64(gbs_ctx* c, const double* x, int64_t n, int64_t k, double* out, void* stream) {
  return select_checked<double>(c, x, n, k, out, stream);
}
gbs_status gbs_median_f32(gbs_ctx* c, const float* x, int64_t n, float* out, void* stream) {
  return select_checked<float>(c, x, n, (n + 1) / 2, out, stream);
}
gbs_status gbs_median_f64(gbs_ctx* c, const double* x, int64_t n, double* out, void* stream) {
  return select_checked<double>(c, x, n, (n + 1) / 2, out, stream);
}

gbs_status gbs_array_stats_f32(gbs_ctx* c, const float* x, int64_t n, gbs_array_stats* out, void* stream) {
  if (!c || !x || !out || n < 1) return GBS_EINVAL;
  return run_select(c, x, n, 1, nullptr, kModeStats, 0, 0, out, nullptr, (cudaStream_t)stream);
}
gbs_status gbs_array_stats_f64(gbs_ctx* c, const double* x, int64_t n, gbs_array_stats* out, void* stream) {
  if (!c || !x || !out || n < 1) return GBS_EINVAL;
  return run_select(c, x, n, 1, nullptr, kModeStats, 0, 0, out, nullptr, (cudaStream_t)stream);
}

gbs_status gbs_cost_pass_f32(gbs_ctx* c, const float* x, int64_t n, int64_t k, double a, double t,
                             gbs_cost_eval* out, void* stream) {
  if (!c || !x || !out || n < 1 || k < 1 || k > n) return GBS_EINVAL;
  if (!((float)a < (float)t) || !std::isfinite((float)a) || !std::isfinite((float)t)) return GBS_EINVAL;
  return run_select(c, x, n, k, nullptr, kModeEval, a, t, nullptr, out, (cudaStream_t)stream);
}
gbs_status gbs_cost_pass_f64(gbs_ctx* c, const double* x, int64_t n, int64_t k, double a, double t,
                             gbs_cost_eval* out, void* stream) {
  if (!c || !x || !out || n < 1 || k < 1 || k > n) return GBS_EINVAL;
  if (!(a < t) || !std::isfinite(a) || !std::isfinite(t)) return GBS_EINVAL;
  return run_select(c, x, n, k, nullptr, kModeEval, a, t, nullptr, out, (cudaStream_t)stream);
}

gbs_status gbs_last_stats(gbs_ctx* c, gbs_run_stats* out) {
  if (!c || !out) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  std::memset(out, 0, sizeof(*out));
  if (!c->ws) return GBS_OK;
  if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  Ctrl ctrl;
  if (cudaMemcpy(out, c->rs, sizeof(*out), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&ctrl, c->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  if (ctrl.status != 0) out->status = ctrl.status;
  return GBS_OK;
}

gbs_status gbs_check_wait_timeout(gbs_ctx* c, int64_t limit_ns, int32_t* device_status, void* stream) {
  if (!c || !device_status || limit_ns < 1000 || limit_ns > 1000000000) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  gbs_status st = gbs_internal_ensure(c, 0);
  if (st != GBS_OK) return st;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  Ctrl ctrl;
  if (cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), strm) != cudaSuccess) return GBS_ECUDA;
  wait_probe_kernel<<<1, 32, 0, strm>>>(c->ctrl, (unsigned long long)limit_ns);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(strm) != cudaSuccess ||
      cudaMemcpy(&ctrl, c->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  *device_status = ctrl.status;
  return GBS_OK;
}

const char* gbs_status_string(gbs_status s) {
  switch (s) {
    case GBS_OK: return "ok";
    case GBS_EINVAL: return "invalid argument";
    case GBS_ENAN: return "input contains NaN";
    case GBS_ENOMEM: return "out of device memory";
    case GBS_ECUDA: return "CUDA runtime error";
    case GBS_ETIMEOUT: return "device-side wait timed out";
    case GBS_EINTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

}  // extern "C"
