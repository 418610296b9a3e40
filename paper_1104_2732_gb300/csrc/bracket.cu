// Learned bracket proposal for the cutting plane: a sketch of x (1024 strided samples,
// sorted, summarised as 32 quantiles plus extremes, mean and spread) feeds a small MLP
// (36 -> 64 -> 64 -> 2, GELU) whose outputs (c, omega) propose the bracket
// mu + sd * (c -+ exp(omega)) for the median.  The selection kernel checks the proposal
// by counts in its first pass and falls back to the data's extremes for any side that
// fails, so the result never depends on the network; only the number of passes does.
//
// The network is trained on the GPU by the kernels below: a Philox4x32-10 generator of
// training arrays, the sketch features, the exact median from the selection kernel, a
// forward + backward kernel and an Adam step.  The paper has no learned component; the
// starting bracket it replaces is Algorithm 1's step 0 (Sec. 3).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "api_internal.h"
#include "bracket.cuh"
#include "common.cuh"

namespace gbs {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by
// 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

namespace {

// uniform in (0, 1] from the top 24 bits
__device__ __forceinline__ float u01(uint32_t u) { return ((u >> 8) + 1u) * (1.0f / 16777216.0f); }
// one standard normal from two words (Box-Muller, cosine branch)
__device__ __forceinline__ float normal2(uint32_t a, uint32_t b) {
  return sqrtf(-2.0f * logf(u01(a))) * cospif(2.0f * u01(b));
}

__global__ void philox_kernel(const unsigned int* ctr, const unsigned int* key, unsigned int* out, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint4 r = philox4x32_10(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                                make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

// Training array: element i uses counters (i, j, 0, 0), j = 0, 1, ..., under key `seed`.
//   family 0: normal           1: Student-t with integer nu = p0 (1..5)
//   family 2: lognormal(0, p0) 3: N(0,1) contaminated with probability p0 by N(p1, p2)
// then loc + scale * value.
__global__ void gen_train_kernel(float* __restrict__ x, long long n, int family, float p0, float p1, float p2,
                                 float loc, float scale, unsigned long long seed) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint4 r0 = philox4x32_10(make_uint4((uint32_t)i, 0u, (uint32_t)(i >> 32), 0u), key);
    float v = normal2(r0.x, r0.y);
    if (family == 1) {
      const int nu = (int)p0;
      float chi = 0.f;
      for (int j = 0; j < nu; j += 2) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 1u + j, (uint32_t)(i >> 32), 0u), key);
        const float a = normal2(r.x, r.y);
        chi += a * a;
        if (j + 1 < nu) {
          const float b = normal2(r.z, r.w);
          chi += b * b;
        }
      }
      v = v * sqrtf((float)nu / chi);
    } else if (family == 2) {
      v = expf(p0 * v);
    } else if (family == 3) {
      if (u01(r0.z) <= p0) v = p1 + p2 * normal2(r0.w, r0.x ^ 0x5bd1e995u);
    }
    x[i] = fmaf(scale, v, loc);
  }
}

__device__ __forceinline__ float gelu_grad(float u) {
  return 0.5f * (1.0f + erff(u * 0.70710678118654752f)) + u * 0.39894228040143268f * expf(-0.5f * u * u);
}

// Sketch of x in one CTA of 1024 threads: features (36 floats) into f, mean and spread
// into *mu, *sd.  Returns false (in every thread) if a sample is not finite or n < 1024.
// The sample is sorted on its totalOrder keys (integer compares; the float64 pipe of this
// GPU is narrow): a bitonic network whose stages of distance < 32 run in registers by
// warp shuffles and whose 15 longer stages go through a double-buffered shared array.
// One warp then forms the float64 mean, spread and quantile features.
template <typename T>
__device__ bool sketch(const T* __restrict__ x, long long n, double* sv, float* f, double* mu, double* sd) {
  using K = decltype(ukey(T()));
  __shared__ K kb[2][kSample];
  const int tid = threadIdx.x;
  if (n < kSample) return false;
  const long long stride = n / kSample;
  const T v = x[tid * stride];
  if (__syncthreads_or(!isfinite(v))) return false;
  K key = ukey(v);
  int buf = 0;
  for (int k = 2; k <= kSample; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      K other;
      if (j >= 32) {
        kb[buf][tid] = key;
        __syncthreads();
        other = kb[buf][tid ^ j];
        buf ^= 1;
      } else {
        other = __shfl_xor_sync(0xffffffffu, key, j);
      }
      const bool keep_min = ((tid & j) == 0) == ((tid & k) == 0);
      key = keep_min ? (other < key ? other : key) : (other > key ? other : key);
    }
  }
  sv[tid] = (double)ukey_value(key, T());
  __syncthreads();
  if (tid < 32) sketch_features_warp(sv, f, mu, sd);
  __syncthreads();
  return true;
}

// MLP forward of one feature vector f (shared memory) by the first 64 threads.
__device__ void mlp_forward_cta(const float* __restrict__ W, const float* f, float* h1, float* h2, float* o) {
  const int tid = threadIdx.x;
  if (tid < kHid) {
    float u = W[kOffB1 + tid];
    for (int i = 0; i < kIn; ++i) u = fmaf(W[kOffW1 + tid * kIn + i], f[i], u);
    h1[tid] = gelu(u);
  }
  __syncthreads();
  if (tid < kHid) {
    float u = W[kOffB2 + tid];
    for (int i = 0; i < kHid; ++i) u = fmaf(W[kOffW2 + tid * kHid + i], h1[i], u);
    h2[tid] = gelu(u);
  }
  __syncthreads();
  if (tid < kOut) {
    float u = W[kOffB3 + tid];
    for (int i = 0; i < kHid; ++i) u = fmaf(W[kOffW3 + tid * kHid + i], h2[i], u);
    o[tid] = u;
  }
  __syncthreads();
}

// Proposed bracket {a, b, valid} for the median of x.
// The same network evaluated by a CTA of 1024 threads: warp w computes outputs w and
// w + 32 of each hidden layer (and output w of the last, for w < 2), its lanes splitting
// the dot product.  Each warp loads its weight rows into registers (coalesced) before the
// sketch, so that their latency hides behind the sort.
struct WarpRows {
  float w1[2][2], w2[2][2], w3[2], b1[2], b2[2], b3;
  __device__ void load(const float* __restrict__ W) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int j = warp + 32 * r;
      w1[r][0] = W[kOffW1 + j * kIn + lane];
      w1[r][1] = lane + 32 < kIn ? W[kOffW1 + j * kIn + 32 + lane] : 0.f;
      w2[r][0] = W[kOffW2 + j * kHid + lane];
      w2[r][1] = W[kOffW2 + j * kHid + 32 + lane];
      b1[r] = W[kOffB1 + j];
      b2[r] = W[kOffB2 + j];
    }
    const int o = warp < kOut ? warp : 0;
    w3[0] = W[kOffW3 + o * kHid + lane];
    w3[1] = W[kOffW3 + o * kHid + 32 + lane];
    b3 = W[kOffB3 + o];
  }
};


__device__ void mlp_forward_warps(const WarpRows& R, const float* f, float* h1, float* h2, float* o) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float u = warp_dot(R.w1[r][0], R.w1[r][1], f, kIn);
    if (lane == 0) h1[warp + 32 * r] = gelu(u + R.b1[r]);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float u = warp_dot(R.w2[r][0], R.w2[r][1], h1, kHid);
    if (lane == 0) h2[warp + 32 * r] = gelu(u + R.b2[r]);
  }
  __syncthreads();
  if (warp < kOut) {
    const float u = warp_dot(R.w3[0], R.w3[1], h2, kHid);
    if (lane == 0) o[warp] = u + R.b3;
  }
  __syncthreads();
}

// Proposal for the median of x: prop = {a, b, valid} (one CTA of 1024 threads).
template <typename T>
__global__ void __launch_bounds__(1024) propose_kernel(const T* __restrict__ x, long long n,
                                                       const float* __restrict__ W, double* __restrict__ prop) {
  __shared__ double sv[kSample];
  __shared__ float f[kIn], h1[kHid], h2[kHid], o[kOut];
  __shared__ double mu, sd;
  WarpRows R;
  R.load(W);
  const bool ok = sketch<T>(x, n, sv, f, &mu, &sd);
  if (!ok) {
    if (threadIdx.x == 0) { prop[0] = 0.0; prop[1] = 0.0; prop[2] = 0.0; }
    return;
  }
  mlp_forward_warps(R, f, h1, h2, o);
  if (threadIdx.x == 0) {
    double a, b;
    const bool valid = proposal_from_outputs(o, mu, sd, &a, &b);
    prop[0] = a;
    prop[1] = b;
    prop[2] = valid ? 1.0 : 0.0;
  }
}

// Features of x into feat[0..35] and {mu, sd} into musd (one CTA).
template <typename T>
__global__ void __launch_bounds__(1024) features_kernel(const T* __restrict__ x, long long n,
                                                        float* __restrict__ feat, double* __restrict__ musd) {
  __shared__ double sv[kSample];
  __shared__ float f[kIn];
  __shared__ double mu, sd;
  const bool ok = sketch<T>(x, n, sv, f, &mu, &sd);
  if (threadIdx.x < kIn) feat[threadIdx.x] = ok ? f[threadIdx.x] : NAN;
  if (threadIdx.x == 0) {
    musd[0] = ok ? mu : NAN;
    musd[1] = ok ? sd : NAN;
  }
}

// Outputs for B feature rows (one CTA of 64 threads per row).
__global__ void __launch_bounds__(64) forward_kernel(const float* __restrict__ W, const float* __restrict__ F,
                                                     int B, float* __restrict__ out) {
  __shared__ float f[kIn], h1[kHid], h2[kHid], o[kOut];
  const int r = blockIdx.x;
  if (r >= B) return;
  if (threadIdx.x < kIn) f[threadIdx.x] = F[(long long)r * kIn + threadIdx.x];
  __syncthreads();
  mlp_forward_cta(W, f, h1, h2, o);
  if (threadIdx.x < kOut) out[r * kOut + threadIdx.x] = o[threadIdx.x];
}

// Gradient of the mean batch loss (see bracket.cuh) with respect to the parameters.
// One warp per sample; every CTA sums its samples' gradients in shared memory and adds
// them to `grad` (pre-zeroed); loss sums go to *loss (float64, pre-zeroed).
constexpr int kGradWarps = 8;
__global__ void __launch_bounds__(kGradWarps * 32) grad_kernel(const float* __restrict__ W,
                                                                const float* __restrict__ F,
                                                                const float* __restrict__ Z,
                                                                const int* __restrict__ idx, int B, float inv_b,
                                                                float tau, float* __restrict__ grad,
                                                                double* __restrict__ loss) {
  __shared__ float g[kNParams];
  __shared__ float fs[kGradWarps][kIn];
  __shared__ float h1s[kGradWarps][kHid], gu2s[kGradWarps][kHid];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) g[i] = 0.f;
  __syncthreads();
  double lsum = 0.0;
  for (int r = blockIdx.x * kGradWarps + w; r < B; r += gridDim.x * kGradWarps) {
    const long long row = idx ? idx[r] : r;
    for (int i = lane; i < kIn; i += 32) fs[w][i] = F[row * kIn + i];
    const float z = Z[row];
    __syncwarp();
    float u1[2], u2[2], h2v[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      float u = W[kOffB1 + j];
      for (int i = 0; i < kIn; ++i) u = fmaf(W[kOffW1 + j * kIn + i], fs[w][i], u);
      u1[q] = u;
      h1s[w][j] = gelu(u);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      float u = W[kOffB2 + j];
      for (int i = 0; i < kHid; ++i) u = fmaf(W[kOffW2 + j * kHid + i], h1s[w][i], u);
      u2[q] = u;
      h2v[q] = gelu(u);
    }
    __syncwarp();
    float o0 = 0.f, o1 = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      o0 = fmaf(W[kOffW3 + j], h2v[q], o0);
      o1 = fmaf(W[kOffW3 + kHid + j], h2v[q], o1);
    }
    for (int off = 16; off > 0; off >>= 1) {
      o0 += __shfl_xor_sync(0xffffffffu, o0, off);
      o1 += __shfl_xor_sync(0xffffffffu, o1, off);
    }
    o0 += W[kOffB3];
    o1 += W[kOffB3 + 1];
    // loss (z - c)^2 + rho_tau(|z - c| - exp(omega)) and its derivatives
    const float d = z - o0;
    const float wd = expf(o1);
    const float u = fabsf(d) - wd;
    const float drho = u < 0.f ? tau - 1.f : tau;
    if (lane == 0) lsum += (double)d * d + (double)u * drho;
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    const float gc = (-2.f * d - drho * sgn) * inv_b;
    const float gw = (-drho * wd) * inv_b;
    if (lane == 0) {
      atomicAdd(&g[kOffB3], gc);
      atomicAdd(&g[kOffB3 + 1], gw);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;
      atomicAdd(&g[kOffW3 + j], gc * h2v[q]);
      atomicAdd(&g[kOffW3 + kHid + j], gw * h2v[q]);
      const float gh2 = gc * W[kOffW3 + j] + gw * W[kOffW3 + kHid + j];
      const float gu2 = gh2 * gelu_grad(u2[q]);
      gu2s[w][j] = gu2;
      atomicAdd(&g[kOffB2 + j], gu2);
      for (int i = 0; i < kHid; ++i) atomicAdd(&g[kOffW2 + j * kHid + i], gu2 * h1s[w][i]);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = lane + 32 * q;   // hidden unit of layer 1
      float gh1 = 0.f;
      for (int i = 0; i < kHid; ++i) gh1 = fmaf(gu2s[w][i], W[kOffW2 + i * kHid + j], gh1);
      const float gu1 = gh1 * gelu_grad(u1[q]);
      atomicAdd(&g[kOffB1 + j], gu1);
      for (int i = 0; i < kIn; ++i) atomicAdd(&g[kOffW1 + j * kIn + i], gu1 * fs[w][i]);
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x)
    if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
  if (lane == 0 && lsum != 0.0) atomicAdd(loss, lsum * inv_b);
}

__global__ void adam_kernel(float* __restrict__ W, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  W[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

gbs_status ensure_model(gbs_ctx* c) {
  if (c->model) return GBS_OK;
  void* p = nullptr;
  const size_t bytes = sizeof(float) * kNParams * 4;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ENOMEM;
  }
  if (cudaMemset(p, 0, bytes) != cudaSuccess) {
    cudaFree(p);
    return GBS_ECUDA;
  }
  c->model = static_cast<float*>(p);   // weights | Adam m | Adam v | gradient
  c->model_loaded = 0;
  c->adam_t = 0;
  return GBS_OK;
}
float* adam_m(gbs_ctx* c) { return c->model + kNParams; }
float* adam_v(gbs_ctx* c) { return c->model + 2 * kNParams; }
float* gradbuf(gbs_ctx* c) { return c->model + 3 * kNParams; }

}  // namespace

// Launches the proposal kernel into prop (3 doubles) when a model is loaded.
gbs_status launch_propose_f32(gbs_ctx* c, const float* x, long long n, double* prop, cudaStream_t s) {
  if (!c->model || !c->model_loaded || n < kSample) return GBS_EINVAL;
  propose_kernel<float><<<1, kSample, 0, s>>>(x, n, c->model, prop);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}
gbs_status launch_propose_f64(gbs_ctx* c, const double* x, long long n, double* prop, cudaStream_t s) {
  if (!c->model || !c->model_loaded || n < kSample) return GBS_EINVAL;
  propose_kernel<double><<<1, kSample, 0, s>>>(x, n, c->model, prop);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

}  // namespace gbs

void gbs_internal_release_model(gbs_ctx* c) {
  if (c->model) {
    cudaDeviceSynchronize();
    cudaFree(c->model);
    c->model = nullptr;
  }
}

using namespace gbs;

extern "C" {

gbs_status gbs_philox4x32_10(gbs_ctx* c, const uint32_t* counters, const uint32_t* keys, uint32_t* out, int32_t m,
                             void* stream) {
  if (!c || !counters || !keys || !out || m < 1) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  philox_kernel<<<(m + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(counters, keys, out, m);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status gbs_generate_training_array_f32(gbs_ctx* c, float* x, int64_t n, int32_t family, float p0, float p1,
                                           float p2, float loc, float scale, uint64_t seed, void* stream) {
  if (!c || !x || n < 1 || family < 0 || family > 3) return GBS_EINVAL;
  if (family == 1 && !(p0 >= 1.f && p0 <= 64.f)) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  const long long blocks = (n + 255) / 256;
  const unsigned int grid = (unsigned int)(blocks < (long long)c->num_sms * 16 ? blocks : (long long)c->num_sms * 16);
  gen_train_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, family, p0, p1, p2, loc, scale, seed);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status gbs_bracket_features_f32(gbs_ctx* c, const float* x, int64_t n, float* feat, double* musd,
                                    void* stream) {
  if (!c || !x || !feat || !musd || n < kSample) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  features_kernel<float><<<1, kSample, 0, static_cast<cudaStream_t>(stream)>>>(x, n, feat, musd);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status gbs_bracket_model_set(gbs_ctx* c, const float* weights, int32_t count) {
  if (!c || !weights || count != kNParams) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  gbs_status st = ensure_model(c);
  if (st != GBS_OK) return st;
  if (cudaMemcpy(c->model, weights, sizeof(float) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->model + kNParams, 0, sizeof(float) * 2 * kNParams) != cudaSuccess)
    return GBS_ECUDA;
  c->model_loaded = 1;
  c->adam_t = 0;
  return GBS_OK;
}

gbs_status gbs_bracket_model_get(gbs_ctx* c, float* weights, int32_t count) {
  if (!c || !weights || count != kNParams || !c->model) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaDeviceSynchronize();
  return cudaMemcpy(weights, c->model, sizeof(float) * kNParams, cudaMemcpyDeviceToHost) == cudaSuccess
             ? GBS_OK
             : GBS_ECUDA;
}

// File: "GBSBRKT1", u32 version 1, u32 n_in, n_hid, n_out, u32 n_params, u64 adam step,
// then weights, Adam m and Adam v (float32 little-endian each).
gbs_status gbs_bracket_model_save(gbs_ctx* c, const char* path) {
  if (!c || !path || !c->model || !c->model_loaded) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  std::vector<float> buf(3 * kNParams);
  cudaDeviceSynchronize();
  if (cudaMemcpy(buf.data(), c->model, sizeof(float) * 3 * kNParams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return GBS_ECUDA;
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return GBS_EINVAL;
  const uint32_t hdr[5] = {1u, (uint32_t)kIn, (uint32_t)kHid, (uint32_t)kOut, (uint32_t)kNParams};
  const uint64_t step = (uint64_t)c->adam_t;
  bool ok = std::fwrite("GBSBRKT1", 1, 8, fp) == 8 && std::fwrite(hdr, 4, 5, fp) == 5 &&
            std::fwrite(&step, 8, 1, fp) == 1 && std::fwrite(buf.data(), 4, buf.size(), fp) == buf.size();
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? GBS_OK : GBS_EINVAL;
}

gbs_status gbs_bracket_model_load(gbs_ctx* c, const char* path) {
  if (!c || !path) return GBS_EINVAL;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return GBS_EINVAL;
  char magic[8];
  uint32_t hdr[5];
  uint64_t step = 0;
  std::vector<float> buf(3 * kNParams);
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "GBSBRKT1", 8) == 0 &&
            std::fread(hdr, 4, 5, fp) == 5 && hdr[0] == 1u && hdr[1] == (uint32_t)kIn && hdr[2] == (uint32_t)kHid &&
            hdr[3] == (uint32_t)kOut && hdr[4] == (uint32_t)kNParams && std::fread(&step, 8, 1, fp) == 1 &&
            std::fread(buf.data(), 4, buf.size(), fp) == buf.size();
  std::fclose(fp);
  if (!ok) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  gbs_status st = ensure_model(c);
  if (st != GBS_OK) return st;
  if (cudaMemcpy(c->model, buf.data(), sizeof(float) * 3 * kNParams, cudaMemcpyHostToDevice) != cudaSuccess)
    return GBS_ECUDA;
  c->model_loaded = 1;
  c->adam_t = (long long)step;
  return GBS_OK;
}

gbs_status gbs_bracket_forward(gbs_ctx* c, const float* F, int32_t B, float* out, void* stream) {
  if (!c || !F || !out || B < 1 || !c->model || !c->model_loaded) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  forward_kernel<<<B, 64, 0, static_cast<cudaStream_t>(stream)>>>(c->model, F, B, out);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status gbs_bracket_grad(gbs_ctx* c, const float* F, const float* Z, int32_t B, float* grad, double* loss,
                            void* stream) {
  if (!c || !F || !Z || !grad || !loss || B < 1 || !c->model || !c->model_loaded) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(grad, 0, sizeof(float) * kNParams, s) != cudaSuccess ||
      cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess)
    return GBS_ECUDA;
  const int grid = (B + kGradWarps - 1) / kGradWarps < 256 ? (B + kGradWarps - 1) / kGradWarps : 256;
  grad_kernel<<<grid, kGradWarps * 32, 0, s>>>(c->model, F, Z, nullptr, B, 1.0f / B, kTau, grad, loss);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status gbs_bracket_train(gbs_ctx* c, const float* F, const float* Z, int32_t N, int32_t batch, int32_t steps,
                             float lr, uint64_t seed, float* loss_hist, void* stream) {
  if (!c || !F || !Z || N < 1 || batch < 1 || batch > N || steps < 1 || !(lr > 0.f)) return GBS_EINVAL;
  if (!c->model || !c->model_loaded) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // one permutation of the rows per epoch, drawn on the host (mt19937_64, `seed`)
  int* idx = nullptr;
  double* losses = nullptr;
  if (cudaMalloc(&idx, sizeof(int) * (size_t)N) != cudaSuccess ||
      cudaMalloc(&losses, sizeof(double) * (size_t)steps) != cudaSuccess) {
    cudaGetLastError();
    if (idx) cudaFree(idx);
    return GBS_ENOMEM;
  }
  std::vector<int> perm(N);
  std::mt19937_64 rng(seed);
  int pos = N;
  gbs_status st = GBS_OK;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int it = 0; it < steps && st == GBS_OK; ++it) {
    if (pos + batch > N) {
      for (int i = 0; i < N; ++i) perm[i] = i;
      std::shuffle(perm.begin(), perm.end(), rng);
      if (cudaMemcpyAsync(idx, perm.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = GBS_ECUDA;
        break;
      }
      pos = 0;
    }
    if (cudaMemsetAsync(gradbuf(c), 0, sizeof(float) * kNParams, s) != cudaSuccess ||
        cudaMemsetAsync(losses + it, 0, sizeof(double), s) != cudaSuccess) {
      st = GBS_ECUDA;
      break;
    }
    const int grid = (batch + kGradWarps - 1) / kGradWarps < 256 ? (batch + kGradWarps - 1) / kGradWarps : 256;
    grad_kernel<<<grid, kGradWarps * 32, 0, s>>>(c->model, F, Z, idx + pos, batch, 1.0f / batch, kTau, gradbuf(c),
                                                 losses + it);
    c->adam_t += 1;
    const double c1 = 1.0 - std::pow((double)b1, (double)c->adam_t);
    const double c2 = 1.0 - std::pow((double)b2, (double)c->adam_t);
    adam_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(c->model, gradbuf(c), adam_m(c), adam_v(c), lr, b1, b2, eps,
                                                       (float)c1, (float)c2);
    if (cudaGetLastError() != cudaSuccess) st = GBS_ECUDA;
    pos += batch;
  }
  if (st == GBS_OK && loss_hist) {
    std::vector<double> h(steps);
    if (cudaMemcpyAsync(h.data(), losses, sizeof(double) * (size_t)steps, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = GBS_ECUDA;
    for (int i = 0; i < steps && st == GBS_OK; ++i) loss_hist[i] = (float)h[i];
  }
  cudaStreamSynchronize(s);
  cudaFree(idx);
  cudaFree(losses);
  return st;
}

gbs_status gbs_bracket_propose_f32(gbs_ctx* c, const float* x, int64_t n, double* out, void* stream) {
  if (!c || !x || !out) return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  return launch_propose_f32(c, x, n, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
