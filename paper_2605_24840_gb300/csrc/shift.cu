// shift.cu -- shift policies along a sequence of slowly varying Hessians
// (Sec. 4.4, Prop. 4.2 and the shift policies of Algorithm 1): midpoint,
// damped midpoint and reuse/refresh.
//
// Reuse/refresh keeps the previous shift s while its certified margin stays
// above a threshold.  The margin is certified as in Prop. 4.2: endpoint
// estimates with error at most eps give the true margin >= m_hat - eps at the
// matrix where they were taken, and each later matrix loses at most the
// endpoint drift, which Weyl's bound limits by ||H_{n+1} - H_n||_2.  The drift
// bound is computed on the GPU as min(||D||_F, (||D||_1 + ||D||_inf) / 2) for
// D = H_{n+1} - H_n (both bound ||sym(D)||_2 from above, in one pass over the
// two matrices); a refresh re-estimates lam_k, lam_{k+1} with the GPU Lanczos
// of the automatic shift and moves to the new midpoint (damped: a blend with
// the previous shift, clipped into the certified interval).
#include "common.cuh"
#include "kernels.h"
#include "rsign.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace rsign {
namespace {

// per row i of D = Hn - Ho (leading dimension d): sum_j |D_ij| and sum_j D_ij^2
// (one warp per row)
__global__ void drift_rows_kernel(const double* __restrict__ Hn, const double* __restrict__ Ho, int d,
                                  double* __restrict__ rowabs, double* __restrict__ rowsq) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= d) return;
  const double* a = Hn + (size_t)i * d;
  const double* b = Ho + (size_t)i * d;
  double s1 = 0.0, s2 = 0.0;
  for (int j = lane; j < d; j += 32) {
    const double x = a[j] - b[j];
    s1 += fabs(x);
    s2 = fma(x, x, s2);
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    rowabs[i] = s1;
    rowsq[i] = s2;
  }
}

// per column j: sum_i |D_ij| (one thread per column, coalesced across threads)
__global__ void drift_cols_kernel(const double* __restrict__ Hn, const double* __restrict__ Ho, int d,
                                  double* __restrict__ colabs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += fabs(Hn[(size_t)i * d + j] - Ho[(size_t)i * d + j]);
  colabs[j] = s;
}

// out[0] = max rowabs, out[1] = max colabs, out[2] = sum rowsq (one block)
__global__ void drift_reduce_kernel(const double* __restrict__ rowabs, const double* __restrict__ colabs,
                                    const double* __restrict__ rowsq, int d, double* __restrict__ out) {
  __shared__ double sa[32], sb[32], sc[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    a = fmax(a, rowabs[i]);
    b = fmax(b, colabs[i]);
    c += rowsq[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  c = warp_sum(c);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
    sc[w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0, C = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      A = fmax(A, sa[q]);
      B = fmax(B, sb[q]);
      C += sc[q];
    }
    out[0] = A;
    out[1] = B;
    out[2] = C;
  }
}

// y = (Hn - Ho) x (leading dimension d), one warp per row
__global__ void diff_gemv_kernel(const double* __restrict__ Hn, const double* __restrict__ Ho, int d,
                                 const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= d) return;
  const double* a = Hn + (size_t)i * d;
  const double* b = Ho + (size_t)i * d;
  double s = 0.0;
  for (int j = lane; j < d; j += 32) s = fma(a[j] - b[j], x[j], s);
  s = warp_sum(s);
  if (lane == 0) y[i] = s;
}

__global__ void unit_start_kernel(double* x, int d) {
  const double v = 1.0 / sqrt((double)d);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
    x[i] = v * (1.0 + 0.25 * ((i * 7) % 5));
}

}  // namespace
}  // namespace rsign

extern "C" {

void rsign_shift_state_init(rsign_shift_state* st) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->shift = NAN;
  st->lam_k_est = NAN;
  st->lam_k1_est = NAN;
  st->eps = NAN;
  st->margin_cert = NAN;
}

int32_t rsign_shift_can_reuse(const rsign_shift_state* st, double drift_ub, double threshold) {
  if (!st || !std::isfinite(st->shift) || !std::isfinite(st->margin_cert)) return 0;
  if (!(drift_ub >= 0.0) || !std::isfinite(drift_ub) || !(threshold >= 0.0)) return 0;
  // Prop. 4.2: the shift stays admissible at the next matrix with margin at
  // least margin_cert - drift; reuse it while that exceeds the threshold
  const double m_next = st->margin_cert - drift_ub;
  return (m_next > 0.0 && m_next > threshold) ? 1 : 0;
}

double rsign_shift_damped(double s_prev, double lam_k_est, double lam_k1_est, double eps, double damping) {
  const double mid = 0.5 * (lam_k_est + lam_k1_est);
  if (!std::isfinite(s_prev)) return mid;
  const double theta = std::min(1.0, std::max(0.0, damping));
  double s = theta * s_prev + (1.0 - theta) * mid;
  // clip into the certified interval (lam_k_est + eps, lam_k1_est - eps),
  // keeping a quarter of its half-width as margin
  const double lo = lam_k_est + eps, hi = lam_k1_est - eps;
  if (!(hi > lo)) return mid;
  const double pad = 0.25 * 0.5 * (hi - lo);
  s = std::min(hi - pad, std::max(lo + pad, s));
  return s;
}

rsign_status rsign_shift_update(const double* H_new, const double* H_old, int64_t d64, int32_t k,
                                rsign_shift_policy policy, double threshold, double damping,
                                double drift_bound, rsign_shift_state* state, rsign_shift_report* report,
                                void* stream) {
  using namespace rsign;
  if (!H_new || !state || d64 < 2 || d64 > 16384 || k < 1 || k > d64 - 1) return RSIGN_ERR_ARG;
  if ((int)policy < RSIGN_SHIFT_MIDPOINT || (int)policy > RSIGN_SHIFT_DAMPED) return RSIGN_ERR_ARG;
  if (!(threshold >= 0.0) || !std::isfinite(threshold)) return RSIGN_ERR_ARG;
  if (!std::isnan(drift_bound) && !(drift_bound >= 0.0 && std::isfinite(drift_bound))) return RSIGN_ERR_ARG;
  int sms = 0;
  const int ds = check_device(&sms);
  if (ds != RSIGN_OK) return (rsign_status)ds;
  cudaStream_t st = (cudaStream_t)stream;
  const int d = (int)d64;
  const int dp = (d + 255) / 256 * 256;
  DevBuf mem;
  mem.st = st;
  rsign_shift_report rep;
  std::memset(&rep, 0, sizeof(rep));
  rep.drift_ub = NAN;
  rep.drift_est = NAN;
  auto fail = [&](rsign_status r) {
    mem.release();
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return r;
  };
  const size_t bytes = (size_t)d * d * 8;
  const double* Hn = H_new;
  const double* Ho = H_old;
  if (!is_device_ptr(H_new)) {
    double* p = nullptr;
    if (mem.alloc((void**)&p, bytes) != cudaSuccess ||
        cudaMemcpyAsync(p, H_new, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(RSIGN_ERR_CUDA);
    Hn = p;
  }
  if (H_old && !is_device_ptr(H_old)) {
    double* p = nullptr;
    if (mem.alloc((void**)&p, bytes) != cudaSuccess ||
        cudaMemcpyAsync(p, H_old, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(RSIGN_ERR_CUDA);
    Ho = p;
  }

  // ---- drift bound of the step H_old -> H_new (Weyl), unless the caller gave one
  if (Ho && std::isnan(drift_bound)) {
    double *rowabs = nullptr, *rowsq = nullptr, *colabs = nullptr, *red = nullptr, *x = nullptr, *y = nullptr;
    if (mem.alloc((void**)&rowabs, (size_t)d * 8) != cudaSuccess ||
        mem.alloc((void**)&rowsq, (size_t)d * 8) != cudaSuccess ||
        mem.alloc((void**)&colabs, (size_t)d * 8) != cudaSuccess ||
        mem.alloc((void**)&red, 8 * 8) != cudaSuccess || mem.alloc((void**)&x, (size_t)d * 8) != cudaSuccess ||
        mem.alloc((void**)&y, (size_t)d * 8) != cudaSuccess)
      return fail(RSIGN_ERR_CUDA);
    drift_rows_kernel<<<(d + 7) / 8, 256, 0, st>>>(Hn, Ho, d, rowabs, rowsq);
    drift_cols_kernel<<<(d + 255) / 256, 256, 0, st>>>(Hn, Ho, d, colabs);
    drift_reduce_kernel<<<1, 1024, 0, st>>>(rowabs, colabs, rowsq, d, red);
    // a few power steps on D for a (lower) estimate, reported for comparison
    constexpr int kPower = 8;
    unit_start_kernel<<<(d + 255) / 256, 256, 0, st>>>(x, d);
    double h_red[8];
    double est = 0.0;
    for (int it = 0; it < kPower; ++it) {
      diff_gemv_kernel<<<(d + 7) / 8, 256, 0, st>>>(Hn, Ho, d, x, y);
      if (normalize(y, d, x, red + 3, st) != cudaSuccess) return fail(RSIGN_ERR_CUDA);
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h_red, red, sizeof(h_red), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(RSIGN_ERR_CUDA);
    est = h_red[3];
    const double fro = std::sqrt(std::max(0.0, h_red[2]));
    const double inf1 = 0.5 * (h_red[0] + h_red[1]);
    // both are upper bounds of ||sym(D)||_2; a relative 1e-12 covers their rounding
    rep.drift_ub = std::min(fro, inf1) * (1.0 + 1e-12);
    rep.drift_est = est;
    if (!std::isfinite(rep.drift_ub)) return fail(RSIGN_ERR_ARG);
  }
  if (!std::isnan(drift_bound)) rep.drift_ub = drift_bound;  // the caller's certified bound

  const bool can_reuse = policy == RSIGN_SHIFT_REUSE_REFRESH && std::isfinite(rep.drift_ub) &&
                         rsign_shift_can_reuse(state, rep.drift_ub, threshold) != 0;
  if (can_reuse) {
    state->margin_cert -= rep.drift_ub;
    state->drift_sum += rep.drift_ub;
    state->reuses += 1;
    rep.refreshed = 0;
    rep.margin_cert = state->margin_cert;
    if (report) *report = rep;
    mem.release();
    return cudaStreamSynchronize(st) == cudaSuccess ? RSIGN_OK : RSIGN_ERR_CUDA;
  }

  // ---- refresh: Lanczos endpoint estimates at H_new, new (damped) midpoint
  double *A64 = nullptr, *rowpart = nullptr, *lw = nullptr;
  int* flags = nullptr;
  const int lmax = 600;
  if (mem.alloc((void**)&A64, (size_t)dp * dp * 8) != cudaSuccess ||
      mem.alloc((void**)&rowpart, (size_t)(dp / 32) * dp * 8) != cudaSuccess ||
      mem.alloc((void**)&flags, 4) != cudaSuccess || cudaMemsetAsync(flags, 0, 4, st) != cudaSuccess ||
      mem.alloc((void**)&lw, lanczos_work_doubles(dp, lmax) * 8) != cudaSuccess)
    return fail(RSIGN_ERR_CUDA);
  if (ingest(Hn, d, dp, 0.0, A64, rowpart, flags, st) != cudaSuccess) return fail(RSIGN_ERR_CUDA);
  LanczosResult lr{};
  int64_t launches = 0;
  if (lanczos_endpoints(A64, dp, d, k, lmax, lw, &lr, &launches, st) != cudaSuccess) return fail(RSIGN_ERR_CUDA);
  int h_flags = 0;
  if (cudaMemcpyAsync(&h_flags, flags, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(RSIGN_ERR_CUDA);
  if (h_flags & 1) return fail(RSIGN_ERR_ARG);
  const double eps = std::max(lr.eps_k, lr.eps_k1);
  double s = 0.5 * (lr.lam_k + lr.lam_k1);
  if (policy == RSIGN_SHIFT_DAMPED) s = rsign_shift_damped(state->shift, lr.lam_k, lr.lam_k1, eps, damping);
  const double m_hat = std::min(s - lr.lam_k, lr.lam_k1 - s);
  rep.refreshed = 1;
  rep.lanczos_iters = lr.iters;
  state->lam_k_est = lr.lam_k;
  state->lam_k1_est = lr.lam_k1;
  state->eps = eps;
  state->refreshes += 1;
  state->drift_sum = 0.0;
  rsign_status res = RSIGN_OK;
  if (!std::isfinite(s) || !(m_hat > eps)) {  // Prop. 4.2 margin test failed: gap not resolved
    state->shift = NAN;
    state->margin_cert = NAN;
    res = RSIGN_ERR_GAP;
  } else {
    state->shift = s;
    state->margin_cert = m_hat - eps;
  }
  rep.margin_cert = state->margin_cert;
  if (report) *report = rep;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) return RSIGN_ERR_CUDA;
  return res;
}

}  // extern "C"
