// Allocation-free float32 selection: the same persistent kernel as
// gbs_select_kth_f32, with its scratch memory in a fixed device array of this file
// instead of a context's cudaMalloc'd workspace.
//
// Some callers cannot let a library allocate device memory: hosts whose device memory is
// owned by an arena or pool of their own (a framework's caching allocator, an embedded
// runtime with a fixed budget), and latency-critical loops where cudaMalloc / cudaFree
// would synchronise the device.  This entry point serves them.  Its scratch is the
// static array below (about 4.1 MiB), which every GPU that loads the library holds
// until the process exits.
#include <cstddef>
#include <mutex>

#include "api_internal.h"
#include "common.cuh"
#include "select.cuh"

using namespace gbs;

namespace {

constexpr long long kNoAllocMaxN = 1ll << 20;   // largest n this entry point accepts
constexpr int kNoAllocMaxGrid = 512;            // CTAs of its persistent launch, at most
// Compaction area: whole chunks of the largest input plus the scalar head and tail,
// chunk_count(n/4 + 1) * kChunkVecs * 4 + 8 floats.
constexpr long long kNoAllocZ = ((kNoAllocMaxN / 4 + 1 + kChunkVecs - 1) / kChunkVecs) * kChunkVecs * 4 + 8;

constexpr size_t up256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffPart = kOffCtrl + up256(sizeof(Ctrl));
constexpr size_t kOffSpart = kOffPart + up256(sizeof(PassPartial) * 2 * kNoAllocMaxGrid);
constexpr size_t kOffHist = kOffSpart + up256(sizeof(StatsPartial) * kNoAllocMaxGrid);
constexpr size_t kOffRs = kOffHist + up256(sizeof(unsigned long long) * kMaxRounds * kBins);
constexpr size_t kOffZ = kOffRs + up256(sizeof(gbs_run_stats));
constexpr size_t kScratchBytes = kOffZ + up256(sizeof(float) * kNoAllocZ);

// The scratch.  In host code this name is only a stand-in: the device address comes from
// cudaGetSymbolAddress below, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch on this device
  int grid = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Resolves the array's device address and the launch shape for the current device.
gbs_status setup_current_device(int dev, DeviceSetup* out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return GBS_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      return GBS_ECUDA;
    }
    // one CTA per SM: inputs here are at most 4 MiB, where the per-pass barrier and
    // reductions cost more with more CTAs
    int grid = sms;
    if (grid > kNoAllocMaxGrid) grid = kNoAllocMaxGrid;
    s.base = static_cast<unsigned char*>(p);
    s.grid = grid;
    s.ready = true;
  }
  *out = s;
  return GBS_OK;
}

}  // namespace

extern "C" gbs_status gbs_select_kth_f32_noalloc(const float* x, int64_t n, int64_t k, float* out,
                                                 void* stream) {
  if (!x || !out || n < 1 || k < 1 || k > n) return GBS_EINVAL;
  if (n > kNoAllocMaxN) return GBS_EINVAL;
  if (reinterpret_cast<uintptr_t>(x) % sizeof(float) != 0) return GBS_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  DeviceSetup s;
  gbs_status st = setup_current_device(dev, &s);
  if (st != GBS_OK) return st;
  const long long zel = select_z_elems_f32(n, s.grid);
  if (zel > kNoAllocZ) return GBS_EINVAL;   // cannot happen for n <= kNoAllocMaxN

  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  SelArgs<float> A;
  A.x = x; A.n = n; A.k = k; A.out = out; A.mode = kModeSelect;
  A.maxit = 64;
  A.cap = n / 4 > 4096 ? n / 4 : 4096;   // the float32 default of the context path
  A.a_eval = 0.0; A.t_eval = 0.0;
  A.sigma_stats = select_stats_sigma_f32(n, s.grid);
  A.ctrl = reinterpret_cast<Ctrl*>(s.base + kOffCtrl);
  A.part = reinterpret_cast<PassPartial*>(s.base + kOffPart);
  A.spart = reinterpret_cast<StatsPartial*>(s.base + kOffSpart);
  A.ghist = reinterpret_cast<unsigned long long*>(s.base + kOffHist);
  A.rs = reinterpret_cast<gbs_run_stats*>(s.base + kOffRs);
  A.z = reinterpret_cast<float*>(s.base + kOffZ);
  A.z_elems = zel;
  A.z2 = nullptr;   // no second-level buffer: every round of the finish reads the regions
  A.z2_cap = 0;
  A.stats_out = nullptr;
  A.eval_out = nullptr;
  A.proposal = nullptr;
  // The array keeps the previous call's contents: the barrier and status words must
  // start at zero.  The radix histograms are cleared by the kernel itself, and the run
  // record is rewritten by CTA 0 on every normal exit and never read back here.
  if (cudaMemsetAsync(A.ctrl, 0, sizeof(Ctrl), strm) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  if (select_launch_f32(A, s.grid, strm) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  return GBS_OK;
}
