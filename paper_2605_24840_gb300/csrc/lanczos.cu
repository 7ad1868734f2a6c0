// lanczos.cu -- endpoint estimates for the automatic shift (Sec. 4.3: estimate
// lam_k, lam_{k+1} by a partial eigensolver, take the midpoint of Prop. 4.1 and
// check admissibility with the margin test of Prop. 4.2).
//
// Lanczos on A = sym(H) (FP64 vectors, full reorthogonalisation by two
// classical Gram-Schmidt passes, vectors kept on the device; the products A v
// in double-float arithmetic, ~2^-46 per term) from whichever end of the
// spectrum is closer to the target index; the tridiagonal T_m is solved on
// the host by Sturm-sequence bisection (eigenvalues) and inverse iteration
// (the last eigenvector components, which give the residual bounds
// ||A y - theta y|| = |beta_m e_m^T s|).  Each Ritz value theta has an
// eigenvalue of A within its residual bound; whether that eigenvalue carries
// the intended index is confirmed afterwards by the trace certificate of the
// reflector (trace R = d - 2k).
#include "common.cuh"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace rsign {
namespace {

// c[j] = V_j . w for j < m (one block per vector)
__global__ void dots_kernel(const double* __restrict__ V, int dp, int m, const double* __restrict__ w,
                            double* __restrict__ c) {
  const int j = blockIdx.x;
  if (j >= m) return;
  const double* v = V + (size_t)j * dp;
  double s = 0.0;
  for (int i = threadIdx.x; i < dp; i += blockDim.x) s += v[i] * w[i];
  __shared__ double sh[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) c[j] = s;
  }
}

// w -= sum_j c[j] V_j ; *alpha += c[m-1] (the projection on the newest vector
// is the diagonal entry of T; the others only remove rounding drift)
__global__ void sub_proj_kernel(const double* __restrict__ V, int dp, int m, const double* __restrict__ c,
                                double* __restrict__ w, double* alpha) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < dp; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += c[j] * V[(size_t)j * dp + i];
    w[i] -= s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *alpha += c[m - 1];
}

// start vector: v_i = 1 + (i mod 7)/8 (i < d), 0 in the padding, then normalised
__global__ void start_vec_kernel(double* y, int d, int dp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < dp; i += gridDim.x * blockDim.x)
    y[i] = (i < d) ? 1.0 + (i % 7) * 0.125 + 0.01 * ((i * 2654435761u) % 97) / 97.0 : 0.0;
}

}  // namespace

// ---------------------------------------------------------------- host solver
// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm).
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  const int n = (int)a.size();
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < n; ++i) {
    const double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
    q = (a[i] - x) - (i > 0 ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;  // a pivot exactly at zero counts as negative
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// j-th smallest eigenvalue (0-based) of the tridiagonal by bisection.
static double tridiag_eig(const std::vector<double>& a, const std::vector<double>& b, int j) {
  const int n = (int)a.size();
  double lo = 0.0, hi = 0.0;
  for (int i = 0; i < n; ++i) {  // Gershgorin interval
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(b[i]) : 0.0);
    lo = (i == 0) ? a[i] - r : std::min(lo, a[i] - r);
    hi = (i == 0) ? a[i] + r : std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo) + std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(a, b, mid) > j) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Last component of the unit eigenvector for eigenvalue theta (inverse iteration
// with a tridiagonal LU solve, two passes).
static double tridiag_last_component(const std::vector<double>& a, const std::vector<double>& b, double theta) {
  const int n = (int)a.size();
  if (n == 1) return 1.0;
  std::vector<double> x(n, 1.0), dl(n), du(n), dd(n), y(n);
  const double pert = 1e-14 * (1.0 + std::fabs(theta));
  for (int pass = 0; pass < 3; ++pass) {
    // solve (T - theta I) y = x by Gaussian elimination with partial pivoting on
    // a tridiagonal (stored densely per row as up to three bands + fill)
    std::vector<double> d0(n), d1(n), d2(n);  // row i: d0 at col i, d1 at i+1, d2 at i+2 (fill)
    std::vector<double> sub(n);                // sub-diagonal of row i (col i-1)
    for (int i = 0; i < n; ++i) {
      d0[i] = a[i] - theta;
      d1[i] = (i < n - 1) ? b[i] : 0.0;
      d2[i] = 0.0;
      sub[i] = (i > 0) ? b[i - 1] : 0.0;
    }
    std::vector<double> rhs = x;
    for (int i = 0; i < n - 1; ++i) {
      // rows i and i+1; eliminate sub[i+1]
      if (std::fabs(sub[i + 1]) > std::fabs(d0[i])) {
        std::swap(d0[i], sub[i + 1]);
        std::swap(d1[i], d0[i + 1]);
        std::swap(d2[i], d1[i + 1]);
        std::swap(rhs[i], rhs[i + 1]);
      }
      double piv = d0[i];
      if (piv == 0.0) piv = d0[i] = pert;
      const double f = sub[i + 1] / piv;
      d0[i + 1] -= f * d1[i];
      d1[i + 1] -= f * d2[i];
      rhs[i + 1] -= f * rhs[i];
      sub[i + 1] = 0.0;
    }
    if (d0[n - 1] == 0.0) d0[n - 1] = pert;
    y[n - 1] = rhs[n - 1] / d0[n - 1];
    y[n - 2] = (rhs[n - 2] - d1[n - 2] * y[n - 1]) / d0[n - 2];
    for (int i = n - 3; i >= 0; --i) y[i] = (rhs[i] - d1[i] * y[i + 1] - d2[i] * y[i + 2]) / d0[i];
    double nr = 0.0;
    for (int i = 0; i < n; ++i) nr += y[i] * y[i];
    nr = std::sqrt(nr);
    if (!(nr > 0.0) || !std::isfinite(nr)) break;
    for (int i = 0; i < n; ++i) x[i] = y[i] / nr;
  }
  return x[n - 1];
}

void tridiag_ritz(const double* alpha, const double* beta, int m, int j, double* theta, double* last) {
  std::vector<double> a(alpha, alpha + m), b(beta, beta + std::max(0, m - 1));
  *theta = tridiag_eig(a, b, j);
  *last = tridiag_last_component(a, b, *theta);
}

// ------------------------------------------------------------- Lanczos driver
cudaError_t lanczos_endpoints(const double* A, int dp, int d, int k, int max_iter, double* work,
                              LanczosResult* out, int64_t* launches, cudaStream_t st) {
  // side: smallest eigenvalues of A (k <= d/2) or of -A (k > d/2)
  const bool low = k <= d - k;
  const int kk = low ? k : d - k;   // target pair (kk-th, kk+1-th) from that end
  const int m_cap = std::min(std::min(max_iter, d), 1024);
  double* V = work;                               // [m_cap + 1][dp]
  double* w = V + (size_t)(m_cap + 1) * dp;       // [dp]
  double* c = w + dp;                             // [m_cap + 1]
  double* al = c + (m_cap + 1);                   // alpha_j
  double* be = al + (m_cap + 1);                  // beta_j (norms)
  double* tmp = be + (m_cap + 1);                 // [dp]
  // A v in double-float arithmetic on the FP32 pipe (GB300's FP64 pipe bounds
  // an FP64 GEMV): A 2^e split once into hi + lo planes, 2^e ~ 1/max|A|,
  // from a 256-byte boundary (the GEMV reads these rows with 16-byte loads)
  float* a_hi = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tmp + dp) + 255) & ~(uintptr_t)255);  // [dp][dp]
  float* a_lo = a_hi + (size_t)dp * dp;              // [dp][dp]
  float* v_hi = a_lo + (size_t)dp * dp;              // [dp]
  float* v_lo = v_hi + dp;                           // [dp]
  double* kscale = reinterpret_cast<double*>(v_lo + dp);
  unsigned long long* kbits = reinterpret_cast<unsigned long long*>(kscale + 1);
  cudaError_t e;
  int64_t nl = 0;
  if ((e = inv_maxabs(A, (size_t)dp * dp, kbits, kscale, st)) != cudaSuccess) return e;
  if ((e = split_f32(A, (size_t)dp * dp, a_hi, a_lo, 0, kscale, st)) != cudaSuccess) return e;
  nl += 3;
  start_vec_kernel<<<(dp + 255) / 256, 256, 0, st>>>(tmp, d, dp);
  e = normalize(tmp, dp, V, be + m_cap, st);  // V_0
  nl += 2;
  if (e != cudaSuccess) return e;
  std::vector<double> ha, hb;
  int m = 0;
  out->converged = 0;
  int next_check = std::min(m_cap, std::max(2 * (kk + 1) + 40, 60));
  for (int j = 0; j < m_cap; ++j) {
    // w = A v_j
    if ((e = split_f32(V + (size_t)j * dp, dp, v_hi, v_lo, 0, nullptr, st)) != cudaSuccess) return e;
    if ((e = gemv_df(a_hi, a_lo, v_hi, v_lo, w, dp, st, kscale)) != cudaSuccess) return e;
    nl += 2;
    // two passes of classical Gram-Schmidt against V_0..V_j; the coefficient on
    // V_j is alpha_j = v_j^T A v_j
    cudaMemsetAsync(al + j, 0, sizeof(double), st);
    for (int pass = 0; pass < 2; ++pass) {
      dots_kernel<<<j + 1, 256, 0, st>>>(V, dp, j + 1, w, c);
      sub_proj_kernel<<<std::max(1, std::min(1024, (dp + 255) / 256)), 256, 0, st>>>(V, dp, j + 1, c, w, al + j);
      nl += 2;
    }
    // beta_j = ||w||, V_{j+1} = w / beta_j
    if ((e = normalize(w, dp, V + (size_t)(j + 1) * dp, be + j, st)) != cudaSuccess) return e;
    ++nl;
    m = j + 1;
    if (m == next_check || m == m_cap) {
      ha.resize(m);
      hb.resize(m);
      // al accumulated the projection coefficients on all V_i; alpha_j is the j-th entry
      std::vector<double> acoef(m);
      if ((e = cudaMemcpyAsync(acoef.data(), al, m * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
      if ((e = cudaMemcpyAsync(hb.data(), be, m * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      for (int i = 0; i < m; ++i) ha[i] = acoef[i];
      // T_m: diagonal alpha_0..alpha_{m-1}, off-diagonal beta_0..beta_{m-2}
      std::vector<double> a(ha.begin(), ha.begin() + m), b(hb.begin(), hb.begin() + std::max(0, m - 1));
      if (kk + 1 <= m) {
        // Ritz indices (ascending) of the pair: low end kk-1, kk; high end
        // m-kk-1 (the (kk+1)-th largest, estimating lam_k) and m-kk (lam_{k+1})
        const int j0 = low ? kk - 1 : m - kk - 1;
        double th[2], lc[2];
        for (int q = 0; q < 2; ++q) tridiag_ritz(a.data(), b.data(), m, j0 + q, &th[q], &lc[q]);
        out->lam_k = th[0];
        out->lam_k1 = th[1];
        // residual bounds |beta_m s_m| (exact arithmetic) plus a rounding
        // allowance 16 sqrt(d) u ||T||, ||T|| <= its Gershgorin bound, with u =
        // 2^-46 the unit of the double-float products: without it a converged
        // Krylov space (beta_m ~ 0) would claim to resolve gaps below the
        // resolution of the eigenvalues
        double tn = 0.0;
        for (int i = 0; i < m; ++i)
          tn = std::max(tn, std::fabs(a[i]) + (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0));
        const double floor_r = 16.0 * std::sqrt((double)d) * std::ldexp(1.0, -46) * tn;
        out->eps_k = std::fabs(hb[m - 1] * lc[0]) + floor_r;
        out->eps_k1 = std::fabs(hb[m - 1] * lc[1]) + floor_r;
        // The pair's indices k, k+1 count the Ritz values between it and the
        // spectrum end; they are eigenvalue indices only if those Ritz values
        // have converged too.  Their largest residual bound joins both
        // errors, so an unconverged interior (k near d/2 with m < d) cannot
        // pass the margin test with a mislabelled pair.
        double worst = 0.0;
        const int q0 = low ? 0 : j0 + 2, q1 = low ? j0 : m;  // the other Ritz values up to the end
        for (int q = q0; q < q1; ++q) {
          double tq, lq;
          tridiag_ritz(a.data(), b.data(), m, q, &tq, &lq);
          worst = std::max(worst, std::fabs(hb[m - 1] * lq));
        }
        out->eps_k = std::max(out->eps_k, worst + floor_r);
        out->eps_k1 = std::max(out->eps_k1, worst + floor_r);
        out->iters = m;
        const double eps = std::max(out->eps_k, out->eps_k1);
        const double mhat = 0.5 * (out->lam_k1 - out->lam_k);
        // stop once the margin test of Prop. 4.2 passes with a factor 4 to spare
        if (mhat > 4.0 * eps || hb[m - 1] < 1e-14) {
          out->converged = 1;
          break;
        }
      }
      next_check = std::min(m_cap, m + std::max(40, m / 2));
    }
  }
  *launches += nl;
  return cudaSuccess;
}

size_t lanczos_work_doubles(int dp, int max_iter) {
  const int m_cap = std::min(max_iter, 1024);
  // V, w, c / alpha / beta, tmp; then the split A (2 dp^2 floats), the split
  // vector (2 dp floats) and two scalars
  return (size_t)(m_cap + 1) * dp + dp + 3 * (size_t)(m_cap + 1) + dp + (size_t)dp * dp + dp + 64;
}

}  // namespace rsign
