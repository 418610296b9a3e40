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

gbs_status launch_propose_f32(gbs_ctx* c, const float* x, long long n, double* prop, cudaStream_t s);
gbs_status launch_propose_f64(gbs_ctx* c, const double* x, long long n, double* prop, cudaStream_t s);

}  // namespace gbs
