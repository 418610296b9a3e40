// Bracket-proposal network: sizes, parameter layout and the launch used by the select.
//
// Parameters (float32, in this order): W1 [64][36] (row = hidden unit), b1 [64],
// W2 [64][64], b2 [64], W3 [2][64], b3 [2].  Loss per example, averaged over a batch:
//   (z - c)^2 + rho_tau(|z - c| - exp(omega)),  rho_tau(u) = u (tau - [u < 0]), tau = 0.99,
// where (c, omega) are the outputs and z = (x_(k) - mu) / sd the standardised median.
#pragma once

#include "common.cuh"

namespace gbs {

constexpr int kSample = 1024;   // strided samples of the sketch
constexpr int kQuant = 32;      // sample quantiles among the features
constexpr int kIn = 36, kHid = 64, kOut = 2;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kNParams = kOffB3 + kOut;
constexpr float kTau = 0.99f;
constexpr long long kLearnMinN = 1ll << 16;   // smaller arrays start from the extremes

__device__ __forceinline__ float gelu(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }

// Features of a sorted sample (float64 values sv[0, kSample), shared memory) by one warp:
// f[0..31] the 32 quantiles sv[16 + 32 i] and f[32..34] asinh of the minimum, maximum and
// mean, all standardised by the sample mean and spread; f[35] = log(spread) / 16.  Also
// *mu and *sd (lane 0).  The training features and every proposal use this one function.
__device__ __forceinline__ void sketch_features_warp(const double* sv, float* f, double* mu, double* sd) {
  const int lane = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int i = 0; i < kSample / 32; i += 4) {
    s0 += sv[(i + 0) * 32 + lane];
    s1 += sv[(i + 1) * 32 + lane];
    s2 += sv[(i + 2) * 32 + lane];
    s3 += sv[(i + 3) * 32 + lane];
  }
  double s = (s0 + s1) + (s2 + s3);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double m = s / kSample;
  double q0 = 0.0, q1 = 0.0;
  for (int i = 0; i < kSample / 32; i += 2) {
    const double d0 = sv[i * 32 + lane] - m, d1 = sv[(i + 1) * 32 + lane] - m;
    q0 = fma(d0, d0, q0);
    q1 = fma(d1, d1, q1);
  }
  double q = q0 + q1;
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  double d = sqrt(q / kSample);
  d = d > 0.0 ? d : 1.0;
  f[lane] = (float)((sv[16 + 32 * lane] - m) / d);   // 32 quantiles (kQuant == 32)
  if (lane < 3) {
    const double z = lane == 0 ? (sv[0] - m) / d : lane == 1 ? (sv[kSample - 1] - m) / d : m / d;
    f[32 + lane] = asinhf((float)z);
  }
  if (lane == 3) f[35] = logf((float)d) * (1.0f / 16.0f);
  if (lane == 0) {
    *mu = m;
    *sd = d;
  }
}

// Dot product of a weight row (a0 at lane, a1 at lane + 32) with v[0, len), by one warp.
__device__ __forceinline__ float warp_dot(float a0, float a1, const float* v, int len) {
  const int lane = threadIdx.x & 31;
  float u = a0 * v[lane];
  if (lane + 32 < len) u = fmaf(a1, v[lane + 32], u);
  for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
  return u;
}

// Network forward of the features f (shared memory) by the NW warps of a CTA: warp w
// computes the units w, w + NW, ... of each layer, its weight rows read from W.
template <int NW>
__device__ void mlp_forward_rows(const float* __restrict__ W, const float* f, float* h1, float* h2, float* o) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < kHid; j += NW) {
    const float* r = W + kOffW1 + j * kIn;
    const float u = warp_dot(r[lane], lane + 32 < kIn ? r[lane + 32] : 0.f, f, kIn);
    if (lane == 0) h1[j] = gelu(u + W[kOffB1 + j]);
  }
  __syncthreads();
  for (int j = warp; j < kHid; j += NW) {
    const float* r = W + kOffW2 + j * kHid;
    const float u = warp_dot(r[lane], r[lane + 32], h1, kHid);
    if (lane == 0) h2[j] = gelu(u + W[kOffB2 + j]);
  }
  __syncthreads();
  for (int j = warp; j < kOut; j += NW) {
    const float* r = W + kOffW3 + j * kHid;
    const float u = warp_dot(r[lane], r[lane + 32], h2, kHid);
    if (lane == 0) o[j] = u + W[kOffB3 + j];
  }
  __syncthreads();
}

// The proposed bracket mu + sd * (c -+ exp(omega)) from the outputs o = {c, omega};
// false when it is not a finite a < b.
__device__ __forceinline__ bool proposal_from_outputs(const float* o, double mu, double sd, double* a, double* b) {
  const double c = o[0];
  const double om = fmin(fmax((double)o[1], -30.0), 30.0);
  const double w = exp(om);
  *a = mu + sd * (c - w);
  *b = mu + sd * (c + w);
  return isfinite(*a) && isfinite(*b) && *a < *b;
}

gbs_status launch_propose_f32(gbs_ctx* c, const float* x, long long n, double* prop, cudaStream_t s);
gbs_status launch_propose_f64(gbs_ctx* c, const double* x, long long n, double* prop, cudaStream_t s);

}  // namespace gbs
