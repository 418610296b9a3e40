// The LMS / LTS estimator search (Sec. 5): computing the estimator takes many evaluations
// of F(theta), one per candidate; the library's fused objectives evaluate thousands of
// candidates at once.  LMS takes the candidate of least objective.  LTS refines the best
// candidates by concentration steps (C-steps): refit the model by least squares on the h
// observations the objective retains -- the rows weighted by the rho of Eq. (med_reg), 1
// below q = s_(h), a/b at q, 0 above -- while the objective decreases.  It cannot
// increase: the h smallest squares at the refit sum to at most its rho-weighted sum,
// which the least-squares fit makes at most the old objective.
//
// One C-step for a batch of candidates:
//   squares    s_ci = (y_i - x_i . theta_c)^2 in float32, in a stated order (no fused
//              multiply-add: acc = acc + x_ij theta_cj term by term, r = y_i - acc,
//              s = r * r), written candidate-major -- which rows are retained is an
//              integer decision taken on exactly these values;
//   select     the segmented select in its trimmed-sum mode: q_c = s_(h) and the
//              objective F_c = sum of the h smallest (float64), Eq. (med_reg);
//   counts     #(s < q_c) and #(s = q_c), so the tie weight a/b is known;
//   normal eqs the rho-weighted Gram matrix X^T diag(rho) X and X^T diag(rho) y: exact
//              products of float32 values summed as float32 pairs (the float64 pipe of
//              this GPU is narrow), CTA partials per row chunk summed in float64 in a
//              fixed order;
//   solve      Cholesky in float64, one thread per candidate; the refit is rounded to
//              float32 (coefficients are float32, as the candidates).
// A candidate stops when the objective of its latest refit is not lower than the best
// so far; it keeps the best fit.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "segmented.cuh"
#include "select.cuh"

namespace gbs {
namespace {

constexpr int kPMax = 16;
constexpr int kGT = 256;                 // threads of the Gram kernel
constexpr int kGRows = 256;              // rows per staged tile of the Gram kernel
constexpr long long kSBytes = 1ll << 30; // squares of one batch of candidates, at most

// Squared residuals of the candidates of a batch in the stated float32 order.
__global__ void cs_resid_kernel(const float* __restrict__ X, const float* __restrict__ y, long long n, int p,
                                const float* __restrict__ th, const int* __restrict__ active, float* __restrict__ S) {
  const int c = blockIdx.y;
  if (!active[c]) return;
  __shared__ float s_th[kPMax];
  if (threadIdx.x < p) s_th[threadIdx.x] = th[(long long)c * p + threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float* xr = X + i * p;
    float acc = 0.f;
    for (int j = 0; j < p; ++j) acc = __fadd_rn(acc, __fmul_rn(xr[j], s_th[j]));
    const float r = __fsub_rn(y[i], acc);
    S[(long long)c * n + i] = __fmul_rn(r, r);
  }
}

// Per CTA of a candidate: #(s < q_c) and #(s = q_c) (integer atomics: the totals are
// exact) and the sum of the squares below q_c in float64, written per CTA and summed in a
// fixed order by the update kernel, so that the objective is reproducible bit for bit.
__global__ void __launch_bounds__(256) cs_count_kernel(const float* __restrict__ S, long long n, const float* q,
                                                       const int* active, unsigned long long* cnt, double* sum_part) {
  __shared__ double s_sum[8];
  const int c = blockIdx.y;
  if (!active[c]) return;
  const float qc = q[c];
  unsigned int lt = 0, eq = 0;
  double sum = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = S[(long long)c * n + i];
    if (s < qc) { ++lt; sum += (double)s; }
    eq += s == qc;
  }
  lt = __reduce_add_sync(0xffffffffu, lt);
  eq = __reduce_add_sync(0xffffffffu, eq);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) {
    if (lt) atomicAdd(cnt + 2 * c, (unsigned long long)lt);
    if (eq) atomicAdd(cnt + 2 * c + 1, (unsigned long long)eq);
    s_sum[threadIdx.x >> 5] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_sum[w];
    sum_part[(long long)c * gridDim.x + blockIdx.x] = t;
  }
}

// CTA (chunk, candidate): the rho-weighted normal equations over the chunk's rows.  Entry
// e < p(p+1)/2 is G[j][k] (j <= k, row-major upper triangle), then p entries of X^T rho y.
// Thread t takes entry t % E over the rows t / E, t / E + P, ... of each staged tile
// (P = kGT / E phases).  The rows with weight 1 are summed exactly enough without the
// narrow float64 pipe: each product of two float32 values is split exactly into a float32
// pair (p = a b rounded, e = fma(a, b, -p)), and the pairs are added to a float32 pair
// accumulator (two-sum of the high parts, low parts added), about 2^-44 relative per add;
// the rare tied rows (weight a/b) are summed in float64.  The phases are combined in
// float64, in order.
__global__ void __launch_bounds__(kGT) cs_gram_kernel(const float* __restrict__ X, const float* __restrict__ y,
                                                     const float* __restrict__ S, long long n, int p,
                                                     long long rows_per_chunk, const float* q,
                                                     const unsigned long long* cnt, long long h, const int* active,
                                                     double* part /* [cand][chunk][E] */, int nchunks) {
  const int c = blockIdx.y;
  if (!active[c]) return;
  __shared__ float s_x[kGRows * kPMax];
  __shared__ float s_y[kGRows];
  __shared__ float s_rho[kGRows];
  __shared__ double s_acc[kGT];
  const int nE = p * (p + 1) / 2 + p;
  const int phases = kGT / nE;
  const int tid = threadIdx.x;
  const int e = tid % nE, ph = tid / nE;
  // entry e -> (j, k) or (j, y)
  int ej = 0, ek = -1;
  if (e < p * (p + 1) / 2) {
    int r = e, j = 0;
    while (r >= p - j) { r -= p - j; ++j; }
    ej = j; ek = j + r;
  } else {
    ej = e - p * (p + 1) / 2;
  }
  const float qc = q[c];
  const long long nlt = (long long)cnt[2 * c], neq = (long long)cnt[2 * c + 1];
  const double w_eq = neq > 0 ? (double)(h - nlt) / (double)neq : 0.0;
  const long long r0 = (long long)blockIdx.x * rows_per_chunk;
  const long long r1 = min(n, r0 + rows_per_chunk);
  float hi = 0.f, lo = 0.f;   // float32 pair accumulator of the weight-1 rows
  double tie = 0.0;           // the tied rows, float64
  for (long long rt = r0; rt < r1; rt += kGRows) {
    const int rows = (int)min((long long)kGRows, r1 - rt);
    __syncthreads();
    for (int i = tid; i < rows * p; i += kGT) s_x[i] = X[rt * p + i];
    for (int i = tid; i < rows; i += kGT) {
      const float s = S[(long long)c * n + rt + i];
      s_y[i] = y[rt + i];
      s_rho[i] = s < qc ? 1.f : (s == qc ? -1.f : 0.f);   // -1 marks a tie (weight w_eq)
    }
    __syncthreads();
    if (ph < phases) {
      for (int i = ph; i < rows; i += phases) {
        const float rho = s_rho[i];
        if (rho == 0.f) continue;
        const float a = s_x[i * p + ej];
        const float b = ek >= 0 ? s_x[i * p + ek] : s_y[i];
        if (rho > 0.f) {
          const float pr = __fmul_rn(a, b);
          const float pe = __fmaf_rn(a, b, -pr);           // a b = pr + pe exactly
          const float t = __fadd_rn(hi, pr);
          const float bv = __fsub_rn(t, hi);
          const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(pr, bv));   // hi + pr = t + err
          hi = t;
          lo = __fadd_rn(lo, __fadd_rn(err, pe));
        } else {
          tie += w_eq * ((double)a * (double)b);
        }
      }
    }
  }
  __syncthreads();
  s_acc[tid] = ((double)hi + (double)lo) + tie;
  __syncthreads();
  if (tid < nE) {
    double t = 0.0;
    for (int f = 0; f < phases; ++f) t += s_acc[f * nE + tid];
    part[((long long)c * nchunks + blockIdx.x) * nE + tid] = t;
  }
}

// One CTA per candidate: the objective of its current fit against the best so far (a
// refit is kept while it lowers the objective), then -- when refits continue -- the normal
// equations summed over the chunks in order (a thread per entry), solved by Cholesky in
// float64 by thread 0 and rounded to float32.  A candidate whose retained rows do not
// determine the fit (a pivot that is not positive) stops with its best fit.
__global__ void __launch_bounds__(256) cs_update_kernel(int p, int step, int max_steps, const float* q,
                                                        const unsigned long long* cnt, const double* sum_part,
                                                        int nsum, long long h, int* active, float* th,
                                                        float* th_best, double* F_best, int* refits,
                                                        const double* part, int nchunks) {
  __shared__ double s_e[kPMax * (kPMax + 1) / 2 + kPMax];
  __shared__ double s_w[8];
  __shared__ int s_go;
  const int c = blockIdx.x, tid = threadIdx.x;
  if (!active[c]) return;
  float* tc = th + (long long)c * p;
  float* bc = th_best + (long long)c * p;
  // the objective of the current fit, Eq. (med_reg): the squares below q plus (h - #(s < q)) q
  double below = 0.0;
  for (int b = tid; b < nsum; b += 256) below += sum_part[(long long)c * nsum + b];
  for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
  if ((tid & 31) == 0) s_w[tid >> 5] = below;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    const double Fc = t + (double)(h - (long long)cnt[2 * c]) * (double)q[c];
    int go = 1;
    if (step == 0) {
      F_best[c] = Fc;
      for (int j = 0; j < p; ++j) bc[j] = tc[j];
    } else if (Fc < F_best[c]) {
      F_best[c] = Fc;
      refits[c] += 1;
      for (int j = 0; j < p; ++j) bc[j] = tc[j];
    } else {
      go = 0;
    }
    if (step == max_steps) go = 0;
    if (!go) active[c] = 0;
    s_go = go;
  }
  __syncthreads();
  if (!s_go) return;
  const int nE = p * (p + 1) / 2 + p;
  for (int e = tid; e < nE; e += 256) {
    double t = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) t += part[((long long)c * nchunks + ch) * nE + e];
    s_e[e] = t;
  }
  __syncthreads();
  if (tid != 0) return;
  double G[kPMax][kPMax], v[kPMax];
  for (int e = 0; e < nE; ++e) {
    if (e < p * (p + 1) / 2) {
      int r = e, j = 0;
      while (r >= p - j) { r -= p - j; ++j; }
      G[j][j + r] = s_e[e];
      G[j + r][j] = s_e[e];
    } else {
      v[e - p * (p + 1) / 2] = s_e[e];
    }
  }
  // Cholesky G = L L^T in place (lower triangle)
  for (int j = 0; j < p; ++j) {
    double d = G[j][j];
    for (int k = 0; k < j; ++k) d -= G[j][k] * G[j][k];
    if (!(d > 0.0)) { active[c] = 0; return; }
    const double l = sqrt(d);
    G[j][j] = l;
    for (int i = j + 1; i < p; ++i) {
      double t = G[i][j];
      for (int k = 0; k < j; ++k) t -= G[i][k] * G[j][k];
      G[i][j] = t / l;
    }
  }
  double z[kPMax];
  for (int i = 0; i < p; ++i) {
    double t = v[i];
    for (int k = 0; k < i; ++k) t -= G[i][k] * z[k];
    z[i] = t / G[i][i];
  }
  for (int i = p - 1; i >= 0; --i) {
    double t = z[i];
    for (int k = i + 1; k < p; ++k) t -= G[k][i] * z[k];
    z[i] = t / G[i][i];
  }
  for (int j = 0; j < p; ++j) tc[j] = (float)z[j];
}

__global__ void cs_init_kernel(int C, int* active, int* refits, unsigned long long* cnt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  active[c] = 1;
  refits[c] = 0;
  cnt[2 * c] = 0ull;
  cnt[2 * c + 1] = 0ull;
}

__global__ void cs_offsets_kernel(long long* off, int S, long long len) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s <= S) off[s] = (long long)s * len;
}

__global__ void cs_zero_counts_kernel(int C, unsigned long long* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * C) cnt[i] = 0ull;
}

size_t up256s(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// C-steps for candidates theta[0..C) (C x p float32, device), written to theta_out (the
// best fit of each) with its objective in obj_out and the refits kept in refits_out
// (device, may be NULL).
gbs_status csteps_run(gbs_ctx* c, const float* X, const float* y, long long n, int p, const float* theta, int C,
                      long long h, int max_steps, float* theta_out, double* obj_out, int* refits_out,
                      cudaStream_t strm) {
  const int B = (int)std::max<long long>(1, std::min<long long>(C, kSBytes / (4 * n)));   // candidates per batch
  const int nE = p * (p + 1) / 2 + p;
  const int nchunks = (int)std::max<long long>(1, std::min<long long>((n + kGRows - 1) / kGRows,
                                                                      (long long)c->num_sms * 4 / B + 1));
  long long rpc = (n + nchunks - 1) / nchunks;
  rpc = (rpc + kGRows - 1) / kGRows * kGRows;
  const int nch = (int)((n + rpc - 1) / rpc);
  const unsigned int rgrid = (unsigned int)std::max<long long>(1, std::min<long long>((n + 255) / 256,
                                                                                     (long long)c->num_sms * 8 / B + 1));
  size_t o = 0;
  const size_t o_S = o; o = up256s(o + sizeof(float) * (size_t)B * n);
  const size_t o_th = o; o = up256s(o + sizeof(float) * (size_t)B * p);
  const size_t o_q = o; o = up256s(o + sizeof(float) * (size_t)B);
  const size_t o_act = o; o = up256s(o + sizeof(int) * (size_t)B);
  const size_t o_ref = o; o = up256s(o + sizeof(int) * (size_t)B);
  const size_t o_cnt = o; o = up256s(o + sizeof(unsigned long long) * 2 * (size_t)B);
  const size_t o_part = o; o = up256s(o + sizeof(double) * (size_t)B * nch * nE);
  const size_t o_sum = o; o = up256s(o + sizeof(double) * (size_t)B * rgrid);
  const size_t o_off = o; o = up256s(o + sizeof(long long) * ((size_t)B + 1));
  const size_t bytes = o;
  if (!c->search_buf || c->search_bytes < bytes) {
    if (c->search_buf) {
      cudaDeviceSynchronize();
      cudaFree(c->search_buf);
      c->search_buf = nullptr;
      c->search_bytes = 0;
    }
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ENOMEM;
    }
    c->search_buf = ptr;
    c->search_bytes = bytes;
  }
  gbs_status st = gbs_internal_ensure(c, seg_workspace_bytes(B));
  if (st != GBS_OK) return st;
  if ((st = reserve_select(c, n, 4)) != GBS_OK) return st;
  char* b = static_cast<char*>(c->search_buf);
  float* S = reinterpret_cast<float*>(b + o_S);
  float* th = reinterpret_cast<float*>(b + o_th);
  float* q = reinterpret_cast<float*>(b + o_q);
  int* active = reinterpret_cast<int*>(b + o_act);
  int* refits = reinterpret_cast<int*>(b + o_ref);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(b + o_cnt);
  double* part = reinterpret_cast<double*>(b + o_part);
  double* sum_part = reinterpret_cast<double*>(b + o_sum);
  long long* off = reinterpret_cast<long long*>(b + o_off);
  auto check = [&]() { return cudaGetLastError() == cudaSuccess ? GBS_OK : GBS_ECUDA; };
  std::vector<int> h_act((size_t)B, 1);   // host copy of the active flags of the batch
  for (int c0 = 0; c0 < C; c0 += B) {
    const int mb = std::min(B, C - c0);
    if (cudaMemcpyAsync(th, theta + (size_t)c0 * p, sizeof(float) * (size_t)mb * p, cudaMemcpyDeviceToDevice, strm) !=
        cudaSuccess)
      return GBS_ECUDA;
    cs_init_kernel<<<(mb + 255) / 256, 256, 0, strm>>>(mb, active, refits, cnt);
    cs_offsets_kernel<<<(mb + 1 + 255) / 256, 256, 0, strm>>>(off, mb, n);
    if ((st = check()) != GBS_OK) return st;
    float* th_best = theta_out + (size_t)c0 * p;
    double* F_best = obj_out + c0;
    for (int j = 0; j < mb; ++j) h_act[j] = 1;
    for (int step = 0; step <= max_steps; ++step) {
      cs_resid_kernel<<<dim3(rgrid, (unsigned)mb), 256, 0, strm>>>(X, y, n, p, th, active, S);
      if ((st = check()) != GBS_OK) return st;
      // q_c = s_(h): the single-array select kernel per candidate for a few candidates
      // (it spreads one array over every SM), the segmented select for many
      if (mb <= 16) {
        if ((st = check()) != GBS_OK) return st;
        for (int j = 0; j < mb; ++j)
          if (h_act[j] &&
              (st = run_select(c, S + (size_t)j * n, n, h, q + j, kModeSelect, 0.0, 0.0, nullptr, nullptr, strm)) !=
                  GBS_OK)
            return st;
      } else {
        SegLaunch L;
        if ((st = seg_attach_workspace(c, mb, &L)) != GBS_OK) return st;
        L.x = S; L.off = off; L.S = mb; L.kk = nullptr; L.ctrl = c->ctrl; L.mask = active; L.kk2 = nullptr;
        L.k_const = h; L.k2_const = 0; L.out = q; L.out2 = nullptr; L.outsum = nullptr; L.flags = nullptr;
        if ((st = seg_launch(c, L, c->seg_variant, strm)) != GBS_OK) return st;
      }
      cs_zero_counts_kernel<<<(2 * mb + 255) / 256, 256, 0, strm>>>(mb, cnt);
      cs_count_kernel<<<dim3(rgrid, (unsigned)mb), 256, 0, strm>>>(S, n, q, active, cnt, sum_part);
      if (step < max_steps)
        cs_gram_kernel<<<dim3((unsigned)nch, (unsigned)mb), kGT, 0, strm>>>(X, y, S, n, p, rpc, q, cnt, h, active, part,
                                                                           nch);
      cs_update_kernel<<<mb, 256, 0, strm>>>(p, step, max_steps, q, cnt, sum_part, (int)rgrid, h, active, th, th_best,
                                             F_best, refits, part, nch);
      if ((st = check()) != GBS_OK) return st;
      if (step < max_steps) {   // the candidates still refitting (none: stop)
        if (cudaMemcpyAsync(h_act.data(), active, sizeof(int) * (size_t)mb, cudaMemcpyDeviceToHost, strm) != cudaSuccess ||
            cudaStreamSynchronize(strm) != cudaSuccess)
          return GBS_ECUDA;
        bool any = false;
        for (int j = 0; j < mb; ++j) any |= h_act[j] != 0;
        if (!any) break;
      }
    }
    if (refits_out &&
        cudaMemcpyAsync(refits_out + c0, refits, sizeof(int) * (size_t)mb, cudaMemcpyDeviceToDevice, strm) !=
            cudaSuccess)
      return GBS_ECUDA;
  }
  c->last_stream = strm;
  return GBS_OK;
}

namespace {

// The candidate of least value (NaN counts as +inf), the smallest index on ties: one CTA.
template <typename V>
__global__ void cs_argmin_kernel(const V* v, int C, int* out_index) {
  __shared__ V s_v[32];
  __shared__ int s_i[32];
  V best = V(INFINITY);
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < C; i += blockDim.x) {
    const V x = v[i] == v[i] ? v[i] : V(INFINITY);
    if (x < best || (x == best && i < bi)) { best = x; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const V ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { s_v[threadIdx.x >> 5] = best; s_i[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (s_v[w] < best || (s_v[w] == best && s_i[w] < bi)) { best = s_v[w]; bi = s_i[w]; }
    *out_index = bi == 0x7fffffff ? 0 : bi;
  }
}

// Rank of every candidate by its LTS objective (NaN as +inf, the smaller index first on
// ties); the n_refine best are listed in rank order.
__global__ void cs_rank_kernel(const double* v, int C, int n_refine, int* sel) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double x = v[c] == v[c] ? v[c] : (double)INFINITY;
  int r = 0;
  for (int j = 0; j < C; ++j) {
    const double y = v[j] == v[j] ? v[j] : (double)INFINITY;
    r += (y < x) || (y == x && j < c);
  }
  if (r < n_refine) sel[r] = c;
}

__global__ void cs_gather_kernel(const float* theta, int p, const int* sel, int m, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m * p) out[i] = theta[(long long)sel[i / p] * p + i % p];
}

// Outputs of the search: the LMS candidate and value; the best refined LTS fit, its
// objective and its candidate's index.
__global__ void cs_emit_kernel(const float* theta, int p, const float* lms_all, const int* lms_idx,
                               const float* th_ref, const double* obj_ref, const int* best_ref, const int* sel,
                               float* lms_theta, float* lms_value, int* lms_index, float* lts_theta, double* lts_value,
                               int* lts_index) {
  const int j = threadIdx.x;
  const int cl = *lms_idx, r = *best_ref;
  if (j < p) {
    lms_theta[j] = theta[(long long)cl * p + j];
    lts_theta[j] = th_ref[(long long)r * p + j];
  }
  if (j == 0) {
    *lms_value = lms_all[cl];
    if (lms_index) *lms_index = cl;
    *lts_value = obj_ref[r];
    if (lts_index) *lts_index = sel[r];
  }
}

}  // namespace
}  // namespace gbs

void gbs_internal_release_search(gbs_ctx* c) {
  if (c->search_buf) {
    cudaDeviceSynchronize();
    cudaFree(c->search_buf);
    c->search_buf = nullptr;
    c->search_bytes = 0;
  }
  if (c->search_aux) {
    cudaDeviceSynchronize();
    cudaFree(c->search_aux);
    c->search_aux = nullptr;
    c->search_aux_bytes = 0;
  }
}

extern "C" gbs_status gbs_lts_csteps_f32(gbs_ctx* c, const float* X, const float* y, int64_t n, int32_t p,
                                         const float* theta, int32_t C, int64_t h, int32_t max_steps,
                                         float* theta_out, double* obj_out, int32_t* refits_out, void* stream) {
  if (!c || !X || !y || !theta || !theta_out || !obj_out) return GBS_EINVAL;
  if (n < 1 || n > (1ll << 31) || p < 1 || p > gbs::kPMax || C < 1 || h < 1 || h > n || max_steps < 0 ||
      max_steps > 1000)
    return GBS_EINVAL;
  gbs::DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  return gbs::csteps_run(c, X, y, n, p, theta, C, h, max_steps, theta_out, obj_out, refits_out,
                         static_cast<cudaStream_t>(stream));
}

extern "C" gbs_status gbs_lms_lts_search_f32(gbs_ctx* c, const float* X, const float* y, int64_t n, int32_t p,
                                             const float* theta, int32_t C, int64_t k_lms, int64_t h_lts,
                                             int32_t n_refine, int32_t max_steps, float* lms_theta, float* lms_value,
                                             int32_t* lms_index, float* lts_theta, double* lts_value,
                                             int32_t* lts_index, void* stream) {
  using namespace gbs;
  if (!c || !X || !y || !theta || !lms_theta || !lms_value || !lts_theta || !lts_value) return GBS_EINVAL;
  if (n < 1 || n > (1ll << 31) || p < 1 || p > kPMax || C < 1 || C > 65536) return GBS_EINVAL;
  if (k_lms < 1 || k_lms > n || h_lts < 1 || h_lts > n || n_refine < 1 || max_steps < 0 || max_steps > 1000)
    return GBS_EINVAL;
  DeviceGuard g(c->device);
  if (!g.ok) return GBS_ECUDA;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  const int R = std::min(n_refine, C);
  // lms_all | lts_all | idx (2) | sel | th_ref_in | th_ref | obj_ref
  size_t o = 0;
  const size_t o_lms = o; o = up256s(o + sizeof(float) * (size_t)C);
  const size_t o_lts = o; o = up256s(o + sizeof(double) * (size_t)C);
  const size_t o_idx = o; o = up256s(o + sizeof(int) * 2);
  const size_t o_sel = o; o = up256s(o + sizeof(int) * (size_t)R);
  const size_t o_tin = o; o = up256s(o + sizeof(float) * (size_t)R * p);
  const size_t o_tout = o; o = up256s(o + sizeof(float) * (size_t)R * p);
  const size_t o_obj = o; o = up256s(o + sizeof(double) * (size_t)R);
  const size_t bytes = o;
  if (!c->search_aux || c->search_aux_bytes < bytes) {
    if (c->search_aux) {
      cudaDeviceSynchronize();
      cudaFree(c->search_aux);
      c->search_aux = nullptr;
      c->search_aux_bytes = 0;
    }
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return GBS_ENOMEM;
    }
    c->search_aux = ptr;
    c->search_aux_bytes = bytes;
  }
  char* b = static_cast<char*>(c->search_aux);
  float* lms_all = reinterpret_cast<float*>(b + o_lms);
  double* lts_all = reinterpret_cast<double*>(b + o_lts);
  int* idx = reinterpret_cast<int*>(b + o_idx);
  int* sel = reinterpret_cast<int*>(b + o_sel);
  float* th_in = reinterpret_cast<float*>(b + o_tin);
  float* th_out = reinterpret_cast<float*>(b + o_tout);
  double* obj = reinterpret_cast<double*>(b + o_obj);
  // 1. both objectives of every candidate (residuals recomputed in every pass, never written)
  gbs_status st = gbs_lms_lts_fused_f32(c, X, y, n, p, theta, C, k_lms, h_lts, lms_all, lts_all, nullptr, stream);
  if (st != GBS_OK) return st;
  // 2. LMS: the least objective; LTS: the n_refine best, refined by C-steps
  cs_argmin_kernel<float><<<1, 1024, 0, strm>>>(lms_all, C, idx);
  cs_rank_kernel<<<(C + 255) / 256, 256, 0, strm>>>(lts_all, C, R, sel);
  cs_gather_kernel<<<(R * p + 255) / 256, 256, 0, strm>>>(theta, p, sel, R, th_in);
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  st = csteps_run(c, X, y, n, p, th_in, R, h_lts, max_steps, th_out, obj, nullptr, strm);
  if (st != GBS_OK) return st;
  cs_argmin_kernel<double><<<1, 1024, 0, strm>>>(obj, R, idx + 1);
  cs_emit_kernel<<<1, 32, 0, strm>>>(theta, p, lms_all, idx, th_out, obj, idx + 1, sel, lms_theta, lms_value, lms_index,
                                     lts_theta, lts_value, lts_index);
  if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA;
  c->last_stream = strm;
  return GBS_OK;
}
