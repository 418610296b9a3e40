// LMS and LTS objectives of robust regression (Sec. 5) for many candidate parameter
// vectors theta_c: the residuals r_i = y_i - x_i . theta_c of the linear model
// (Eq. (model)), their squares s_i = r_i^2, and per candidate
//   LMS_c = s_(k)                                  ("Med(r_i)^2", read as s_(k))
//   LTS_c = sum of the h smallest s_i               (Eq. (med_reg): everything below
//                                                    q = s_(h) plus (h - #(s < q)) q)
//
// Squared residuals are written candidate-major (S[c][i]) by one of two kernels:
//   precision 0  float32 FMAs on the CUDA cores
//   precision 1  the product X theta on the tensor cores as three TF32 products
//                (hi*hi + hi*lo + lo*hi of a two-term TF32 split of each operand,
//                float32 accumulation), which recovers float32 accuracy
// and the orders statistics come from the segmented select (one segment per candidate)
// in its trimmed-sum mode, or, in the plain form, from one single-array select per
// candidate and rank plus a summing kernel.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <new>

#include "api_internal.h"
#include "common.cuh"
#include "segmented.cuh"
#include "select.cuh"

namespace gbs {
namespace {

constexpr int kMaxP = 16;

// ------------------------------------------------------------------ float32 CUDA cores
// CTA: 256 rows; every theta in shared memory; each thread one row, all candidates.
template <int P>
__global__ void __launch_bounds__(256) resid_fp32_kernel(const float* __restrict__ X, const float* __restrict__ y,
                                                          long long n, const float* __restrict__ theta, int C,
                                                          float* __restrict__ S) {
  extern __shared__ float th[];   // [C][P]
  for (int i = threadIdx.x; i < C * P; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  float xr[P];
#pragma unroll
  for (int j = 0; j < P; ++j) xr[j] = X[row * P + j];
  const float yr = y[row];
  for (int c = 0; c < C; ++c) {
    float acc = yr;
#pragma unroll
    for (int j = 0; j < P; ++j) acc = fmaf(-xr[j], th[c * P + j], acc);
    S[(long long)c * n + row] = acc * acc;
  }
}

// ------------------------------------------------------------------ TF32 x 3 tensor cores
__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
// v = hi + lo with both parts exactly representable in TF32 (lo rounded)
__device__ __forceinline__ void split_tf32(float v, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(v);
  lo = to_tf32(v - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Warp tile: 16 rows x 64 candidates (8 tiles of m16n8k8), KS = ceil(p/8) k-steps.
// The CTA (4 warps) owns 64 candidates (blockIdx.y) and walks row tiles.
template <int KS>
__global__ void __launch_bounds__(128) resid_tf32x3_kernel(const float* __restrict__ X, const float* __restrict__ y,
                                                            long long n, int p, const float* __restrict__ theta,
                                                            int C, float* __restrict__ S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int cbase = blockIdx.y * 64;
  // B fragments: b0 = theta(k = t, n = g), b1 = theta(k = t + 4, n = g) per n8 tile
  uint32_t bh[KS][8][2], bl[KS][8][2];
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = cbase + nt * 8 + g;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = ks * 8 + t + 4 * h;
        const float v = (c < C && j < p) ? theta[(long long)c * p + j] : 0.f;
        split_tf32(v, bh[ks][nt][h], bl[ks][nt][h]);
      }
    }
  const long long tiles = (n + 15) / 16;
  for (long long tile = (long long)blockIdx.x * 4 + warp; tile < tiles; tile += (long long)gridDim.x * 4) {
    const long long r0 = tile * 16 + g, r1 = r0 + 8;
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      // A fragments: a0 = X(r0, t), a1 = X(r1, t), a2 = X(r0, t + 4), a3 = X(r1, t + 4)
      const int j0 = ks * 8 + t, j1 = j0 + 4;
      const float x00 = (r0 < n && j0 < p) ? X[r0 * p + j0] : 0.f;
      const float x10 = (r1 < n && j0 < p) ? X[r1 * p + j0] : 0.f;
      const float x01 = (r0 < n && j1 < p) ? X[r0 * p + j1] : 0.f;
      const float x11 = (r1 < n && j1 < p) ? X[r1 * p + j1] : 0.f;
      uint32_t ah[4], al[4];
      split_tf32(x00, ah[0], al[0]);
      split_tf32(x10, ah[1], al[1]);
      split_tf32(x01, ah[2], al[2]);
      split_tf32(x11, ah[3], al[3]);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {   // small products first
        mma_tf32(acc[nt], al, bh[ks][nt]);
        mma_tf32(acc[nt], ah, bl[ks][nt]);
        mma_tf32(acc[nt], ah, bh[ks][nt]);
      }
    }
    const float y0 = r0 < n ? y[r0] : 0.f, y1 = r1 < n ? y[r1] : 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c0 = cbase + nt * 8 + 2 * t, c1 = c0 + 1;
      const float e00 = y0 - acc[nt][0], e01 = y0 - acc[nt][1];
      const float e10 = y1 - acc[nt][2], e11 = y1 - acc[nt][3];
      if (r0 < n) {
        if (c0 < C) S[(long long)c0 * n + r0] = e00 * e00;
        if (c1 < C) S[(long long)c1 * n + r0] = e01 * e01;
      }
      if (r1 < n) {
        if (c0 < C) S[(long long)c0 * n + r1] = e10 * e10;
        if (c1 < C) S[(long long)c1 * n + r1] = e11 * e11;
      }
    }
  }
}

// Plain-form LTS: per candidate, everything below q_c plus (h - #below) copies of q_c.
__global__ void __launch_bounds__(512) lts_sum_kernel(const float* __restrict__ S, long long n,
                                                       const float* __restrict__ q, long long h,
                                                       double* __restrict__ lts) {
  __shared__ double sd[16];
  __shared__ unsigned long long sc[16];
  const int c = blockIdx.x;
  const float qc = q[c];
  const float* s = S + (long long)c * n;
  float part = 0.f;
  double acc = 0.0;
  unsigned long long cnt = 0;
  int run = 0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = s[i];
    if (v < qc) { part += v; ++cnt; }
    if (++run == 256) { acc += part; part = 0.f; run = 0; }
  }
  acc += part;
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = acc; sc[threadIdx.x >> 5] = cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    unsigned long long k = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sd[w]; k += sc[w]; }
    lts[c] = a + (double)(h - (long long)k) * (double)qc;
  }
}

template <int P>
gbs_status launch_fp32(const float* X, const float* y, long long n, const float* theta, int C, float* S,
                       cudaStream_t stream) {
  const size_t smem = (size_t)C * P * sizeof(float);
  if (smem > 200 * 1024) return GBS_EINVAL;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(resid_fp32_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return GBS_ECUDA;
  }
  const unsigned int grid = (unsigned int)((n + 255) / 256);
  resid_fp32_kernel<P><<<grid, 256, smem, stream>>>(X, y, n, theta, C, S);
  return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
}

gbs_status launch_residuals(gbs_ctx* c, const float* X, const float* y, long long n, int p, const float* theta,
                            int C, float* S, int precision, cudaStream_t stream) {
  if (precision == 1) {
    const dim3 grid((unsigned int)(c->num_sms * 4 < 65535 ? c->num_sms * 4 : 65535), (unsigned int)((C + 63) / 64));
    if (p <= 8) resid_tf32x3_kernel<1><<<grid, 128, 0, stream>>>(X, y, n, p, theta, C, S);
    else resid_tf32x3_kernel<2><<<grid, 128, 0, stream>>>(X, y, n, p, theta, C, S);
    return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA;
  }
  switch (p) {
#define GBS_P(v) case v: return launch_fp32<v>(X, y, n, theta, C, S, stream);
    GBS_P(1) GBS_P(2) GBS_P(3) GBS_P(4) GBS_P(5) GBS_P(6) GBS_P(7) GBS_P(8)
    GBS_P(9) GBS_P(10) GBS_P(11) GBS_P(12) GBS_P(13) GBS_P(14) GBS_P(15) GBS_P(16)
#undef GBS_P
  }
  return GBS_EINVAL;
}

// The candidate-major residual matrix and the small per-candidate arrays live in a
// buffer of their own (grown on demand, synchronously).
gbs_status lms_buffer(gbs_ctx* c, size_t bytes, char** out) {
  if (c->lms_buf && c->lms_bytes >= bytes) {
    *out = static_cast<char*>(c->lms_buf);
    return GBS_OK;
  }
  if (c->lms_buf) {
    cudaDeviceSynchronize();
    cudaFree(c->lms_buf);
    c->lms_buf = nullptr;
    c->lms_bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GBS_ENOMEM;
  }
  c->lms_buf = p;
  c->lms_bytes = bytes;
  *out = static_cast<char*>(p);
  return GBS_OK;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace gbs

void gbs_internal_release_lms(gbs_ctx* c) {
  for (int e = 0; e < 4; ++e) {
    if (c->lms_ev[e]) {
      cudaEventDestroy(c->lms_ev[e]);
      c->lms_ev[e] = nullptr;
    }
  }
  if (c->lms_buf) {
    cudaDeviceSynchronize();
    cudaFree(c->lms_buf);
    c->lms_buf = nullptr;
    c->lms_bytes = 0;
  }
}

extern "C" {

gbs_status gbs_residual_sq_f32(gbs_ctx* c, const float* X, const float* y, int64_t n, int32_t p,
                               const float* theta, int32_t C, float* S, int32_t precision, void* stream) {
  if (!c || !X || !y || !theta || !S || n < 1 || p < 1 || p > gbs::kMaxP || C < 1) return GBS_EINVAL;
  if (precision != 0 && precision != 1) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  return gbs::launch_residuals(c, X, y, n, p, theta, C, S, precision, static_cast<cudaStream_t>(stream));
}

gbs_status gbs_lms_lts_f32(gbs_ctx* c, const float* X, const float* y, int64_t n, int32_t p, const float* theta,
                           int32_t C, int64_t k_lms, int64_t h_lts, float* lms_out, double* lts_out,
                           int32_t precision, int32_t batched, void* stream) {
  if (!c || !X || !y || !theta || !lms_out || !lts_out) return GBS_EINVAL;
  if (n < 1 || p < 1 || p > gbs::kMaxP || C < 1) return GBS_EINVAL;
  if (k_lms < 1 || k_lms > n || h_lts < 1 || h_lts > n) return GBS_EINVAL;
  if (precision != 0 && precision != 1) return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  // buffer: offsets[C+1] | q[C] | flags[C] | S[C][n]
  const size_t o_off = 0;
  const size_t o_q = gbs::up256(o_off + sizeof(long long) * (C + 1));
  const size_t o_flags = gbs::up256(o_q + sizeof(float) * C);
  const size_t o_S = gbs::up256(o_flags + sizeof(int) * C);
  const size_t bytes = o_S + sizeof(float) * (size_t)C * (size_t)n;
  char* buf = nullptr;
  gbs_status st = gbs::lms_buffer(c, bytes, &buf);
  if (st != GBS_OK) return st;
  long long* off = reinterpret_cast<long long*>(buf + o_off);
  float* q = reinterpret_cast<float*>(buf + o_q);
  int* flags = reinterpret_cast<int*>(buf + o_flags);
  float* S = reinterpret_cast<float*>(buf + o_S);
  if (c->lms_off_C != C || c->lms_off_n != n) {   // segment offsets c*n (host-built once per shape)
    long long* h = new (std::nothrow) long long[C + 1];
    if (!h) return GBS_ENOMEM;
    for (int i = 0; i <= C; ++i) h[i] = (long long)i * n;
    const bool ok = cudaMemcpy(off, h, sizeof(long long) * (C + 1), cudaMemcpyHostToDevice) == cudaSuccess;
    delete[] h;
    if (!ok) return GBS_ECUDA;
    c->lms_off_C = C;
    c->lms_off_n = n;
  }
  st = gbs::launch_residuals(c, X, y, n, p, theta, C, S, precision, strm);
  if (st != GBS_OK) return st;
  if (batched) {
    // trimmed-sum mode for rank h (LTS and q), the LMS rank k from the same bracket
    gbs::SegLaunch L;
    st = gbs::seg_attach_workspace(c, C, &L);
    if (st != GBS_OK) return st;
    L.x = S; L.off = off; L.S = C; L.kk = nullptr; L.out = q;
    L.ctrl = c->ctrl;
    L.mask = nullptr; L.kk2 = nullptr; L.out2 = lms_out; L.outsum = lts_out; L.flags = flags;
    L.k_const = h_lts; L.k2_const = k_lms;
    st = gbs::seg_launch(c, L, c->seg_variant, strm);
    if (st != GBS_OK) return st;
    // candidates whose rank k fell outside the compacted bracket: a plain select for k
    L.mask = flags; L.out = lms_out; L.out2 = nullptr; L.outsum = nullptr; L.flags = nullptr;
    L.k_const = k_lms; L.k2_const = 0;
    st = gbs::seg_launch(c, L, c->seg_variant, strm);
    if (st != GBS_OK) return st;
    c->last_segments = C;
  } else {
    for (int cc = 0; cc < C; ++cc) {
      st = gbs_select_kth_f32(c, S + (size_t)cc * n, n, k_lms, lms_out + cc, stream);
      if (st != GBS_OK) return st;
      st = gbs_select_kth_f32(c, S + (size_t)cc * n, n, h_lts, q + cc, stream);
      if (st != GBS_OK) return st;
    }
    gbs::lts_sum_kernel<<<C, 512, 0, strm>>>(S, n, q, h_lts, lts_out);
    if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  }
  c->last_stream = strm;
  return GBS_OK;
}

}  // extern "C"
