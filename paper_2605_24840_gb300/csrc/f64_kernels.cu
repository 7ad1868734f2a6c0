// f64_kernels.cu -- FP64 products (DMMA m8n8k4 on the FP64 pipe) and the
// bandwidth-bound elementwise / reduction kernels of the reflector path.
#include <type_traits>
#include "common.cuh"
#include "intconv.cuh"
#include "kernels.h"

namespace rsign {
namespace {

// ------------------------------------------------------------------ FP64 GEMM
// 64x64 output tile per 128-thread block (2x2 warps, 32x32 per warp as 4x4
// fragments of m8n8), K step 16 staged through shared memory.
constexpr int FT = 64, FK = 16, FPAD = 72;

struct F64Sched {
  int nb, sym, n;
  __host__ __device__ F64Sched(int dp, int s) : nb(dp / FT), sym(s) {
    n = s ? nb * (nb + 1) / 2 : nb * nb;
  }
  __device__ __forceinline__ void decode(int t, int& bi, int& bj) const {
    if (!sym) { bi = t / nb; bj = t % nb; return; }
    int b = 0;
    for (;;) {
      const int cnt = nb - b;
      if (t < cnt) break;
      t -= cnt;
      ++b;
    }
    bi = b;
    bj = b + t;
  }
};

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

template <int EPI>
__global__ void __launch_bounds__(128) f64_gemm_kernel(const F64GemmArgs a) {
  if (a.skip != nullptr && *a.skip != 0) return;
  __shared__ double As[2][FK][FPAD];  // As[k][m]
  __shared__ double Bs[2][FK][FPAD];  // Bs[k][n]
  int bi, bj, slot = blockIdx.x, kext = a.dp, d_real = a.d_real;
  size_t moff = 0;
  if (a.units != nullptr) {
    const int4 q = a.units[blockIdx.x];
    if (a.mat_skip != nullptr && a.mat_skip[q.x] != 0) return;  // uniform per block
    bi = q.y;
    bj = q.z;
    slot = q.w;
    kext = a.mat_dp[q.x];
    d_real = a.mat_d[q.x];
    moff = (size_t)q.x * (size_t)a.mat_stride;
  } else {
    const F64Sched sched(a.dp, a.sym);
    sched.decode(blockIdx.x, bi, bj);
  }
  const double* Ap = a.A + moff;
  const double* Bp = a.B + moff;
  double* outp = a.out + moff;
  const double* xinp = a.xin != nullptr ? a.xin + moff : nullptr;
  const int m0 = bi * FT, n0 = bj * FT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int ld = a.dp;

  double acc[4][4][2];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y][0] = acc[x][y][1] = 0.0;

  // global -> register staging: A tile 64 rows x 16 k, B tile 16 k x 64 cols
  double ra[8], rb[8];
  auto gload = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * 128;          // 0..1023
      const int am = e >> 4, ak = e & 15;   // A: row am, col k0+ak
      ra[q] = Ap[(size_t)(m0 + am) * ld + k0 + ak];
      const int bk = e >> 6, bn = e & 63;   // B: row k0+bk, col n0+bn
      rb[q] = Bp[(size_t)(k0 + bk) * ld + n0 + bn];
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * 128;
      As[buf][e & 15][e >> 4] = ra[q];
      Bs[buf][e >> 6][e & 63] = rb[q];
    }
  };

  const int nk = kext / FK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) gload((kt + 1) * FK);
#pragma unroll
    for (int kk = 0; kk < FK; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) af[x] = As[buf][kk + (lane & 3)][wm * 32 + x * 8 + (lane >> 2)];
#pragma unroll
      for (int y = 0; y < 4; ++y) bf[y] = Bs[buf][kk + (lane & 3)][wn * 32 + y * 8 + (lane >> 2)];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) dmma(acc[x][y][0], acc[x][y][1], af[x], bf[y]);
    }
    if (kt + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }

  // epilogue: thread holds rows (lane>>2) and columns 2*(lane&3)+{0,1} of each fragment
  double part = 0.0;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = m0 + wm * 32 + x * 8 + (lane >> 2);
#pragma unroll
    for (int y = 0; y < 4; ++y) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = n0 + wn * 32 + y * 8 + 2 * (lane & 3) + h;
        double v = acc[x][y][h];
        if constexpr (EPI == F64_EPI_STORE) {
          v *= a.scale;
        } else if constexpr (EPI == F64_EPI_NS_SYRK) {
          const bool real = i < d_real && j < d_real;
          if (a.ns_c2 != 0.0 && a.ns_c2 != 1.0) v *= a.ns_c2;  // E = I - a^2 X^2 (scaled step)
          v = real ? ((i == j ? 1.0 : 0.0) - v) : 0.0;
          if (real && (!a.sym || j >= i)) part += ((a.sym && j > i) ? 2.0 : 1.0) * v * v;
        } else {  // F64_EPI_NS_UPDATE
          if (a.scale != 0.0 && a.scale != 1.0) v *= a.scale;  // X_in + 1/2 scale acc
          v = xinp[(size_t)i * ld + j] + 0.5 * v;
          if (a.ns_c1 != 0.0 && a.ns_c1 != 1.0) v *= a.ns_c1;  // X+ = a (X + 1/2 X E)
          if (i == j && i < d_real) part += v;
        }
        if (!a.sym || j >= i) outp[(size_t)i * ld + j] = v;
        if (a.sym && j > i) outp[(size_t)j * ld + i] = v;
      }
    }
  }
  if constexpr (EPI != F64_EPI_STORE) {
    part = warp_sum(part);
    if (lane == 0) a.partials[(size_t)slot * 4 + warp] = part;
  }
}

// ------------------------------------------------------------------ ingest
// A = 1/2 (H + H^T) - s I (zero padded to dp), row partial sums of |A| per
// 32-column block, non-finite detection.  One block per pair of mirror tiles
// {(bi, bj), (bj, bi)}, bi <= bj: both tiles of H are read once and both
// tiles of A written from them, so every entry of H crosses the bus once
// (H may be host memory mapped for the device).  Blocks below the diagonal
// return at once.
__global__ void ingest_kernel(const double* __restrict__ H, int d, int dp, double s,
                              double* __restrict__ A, double* __restrict__ rowpart, int* flags) {
  __shared__ double t1[32][33], t2[32][33], tv[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // A tile (bi, bj): rows bi*32.., cols bj*32..
  if (bi > bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const bool mirror = bi != bj;
  // FP64 arithmetic only where it changes a value (GB300's FP64 pipe is
  // slower than the stream): the finiteness test and |v| on the bit
  // patterns, the average of a bitwise symmetric pair is the entry itself,
  // the shift only on the diagonal
  bool bad = false;
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    double h1 = 0.0, h2 = 0.0;
    if (i < d && j < d) h1 = H[(size_t)i * d + j];
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;  // the mirror tile
    if (mirror && i2 < d && j2 < d) h2 = H[(size_t)i2 * d + j2];
    if (((ic_bits(h1) >> 52) & 0x7FF) == 0x7FF || ((ic_bits(h2) >> 52) & 0x7FF) == 0x7FF) bad = true;
    t1[r][tx] = h1;
    t2[r][tx] = mirror ? h2 : h1;  // the diagonal tile holds both triangles itself
  }
  __syncthreads();
  // A(bi, bj)[r][c] from H_ij = t1[r][c] and H_ji = t2[c][r]
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    double v = 0.0;
    if (i < d && j < d) {
      const double a = t1[r][tx], b = t2[tx][r];
      if (i == j) v = a - s;
      else if (ic_bits(a) == ic_bits(b)) v = a;
      else v = 0.5 * (a + b);
    }
    A[(size_t)i * dp + j] = v;
    tv[r][tx] = v;
  }
  if (bad) atomicOr(flags, 1);
  __syncthreads();
  // A(bj, bi) = A(bi, bj)^T, the same bits: row bj*32 + r of it is column r of tv
  if (mirror)
    for (int r = ty; r < 32; r += 8) A[(size_t)(bj * 32 + r) * dp + bi * 32 + tx] = tv[tx][r];
  // row partial sums of |A| over the 32 columns of each tile, in column order
  if (ty == 0) {
    double sum = 0.0;
    for (int c = 0; c < 32; ++c) sum += ic_double(ic_bits(tv[tx][c]) & 0x7FFFFFFFFFFFFFFFull);
    rowpart[(size_t)bj * dp + bi * 32 + tx] = sum;
  } else if (ty == 1 && mirror) {
    double sum = 0.0;
    for (int r = 0; r < 32; ++r) sum += ic_double(ic_bits(tv[r][tx]) & 0x7FFFFFFFFFFFFFFFull);
    rowpart[(size_t)bi * dp + bj * 32 + tx] = sum;
  }
}

__global__ void rowsum_kernel(const double* __restrict__ rowpart, int dp, double* rowsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dp) return;
  double s = 0.0;
  const int nb = dp / 32;
  for (int b = 0; b < nb; ++b) s += rowpart[(size_t)b * dp + i];
  rowsum[i] = s;
}

__global__ void max_kernel(const double* __restrict__ x, int n, double* out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      out[0] = m;
      out[1] = m > 0.0 ? 1.0 / m : 0.0;
    }
  }
}

// Deterministic single-block sum (fixed order: strided per thread, then tree).
__global__ void sum_kernel(const double* __restrict__ x, int n, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      out[0] = s;
      out[1] = sqrt(fmax(s, 0.0));
    }
  }
}

// tr: optional trace partials of the current iterate (n_tr values); a floor
// or stagnation stop then also needs |trace - tr_target| <= tr_tol, so a
// residual that sits in the floor band while a few eigenvalues are still far
// from +-1 (the slow first phase of the iteration) cannot stop it.
__global__ void ns_check_kernel(const double* __restrict__ x, int n, double* hist, int m, double tol_abs,
                                double floor_lo, double floor_hi, double ratio, int* done, int* steps,
                                const double* __restrict__ tr, int n_tr, double tr_target, double tr_tol) {
  __shared__ double sh[32], sh2[32];
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  if (tr != nullptr)
    for (int i = threadIdx.x; i < n_tr; i += blockDim.x) t += tr[i];
  s = warp_sum(s);
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = s;
    sh2[threadIdx.x >> 5] = t;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    t = (threadIdx.x < (blockDim.x >> 5)) ? sh2[threadIdx.x] : 0.0;
    s = warp_sum(s);
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      const double r = sqrt(fmax(s, 0.0));
      if (*done == 0) {  // after a stop the partials are stale: leave hist alone
        hist[m] = r;
        const bool trace_ok = tr == nullptr || fabs(t - tr_target) <= tr_tol;
        bool stop = r < tol_abs || (trace_ok && r <= floor_lo);
        if (!stop && trace_ok && m >= 1 && r <= floor_hi && r >= ratio * hist[m - 1]) stop = true;
        if (stop) {
          *done = 1;
          *steps = m;
        }
      }
    }
  }
}

__global__ void trace_kernel(const double* __restrict__ X, int dp, int d, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) s += X[(size_t)i * dp + i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) out[0] = s;
  }
}

template <typename T>
__global__ void scale_convert_kernel(const double* __restrict__ src, size_t n, const double* scale_dev,
                                     double mult, T* __restrict__ dst) {
  const double sc = (scale_dev ? *scale_dev : 1.0) * mult;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = src[i] * sc;
    if constexpr (sizeof(T) == 8) dst[i] = v;
    else if constexpr (sizeof(T) == 4) dst[i] = (float)v;
    else dst[i] = from_f64<T>(v);
  }
}

// hi + lo = x * scale as a pair of FP16/BF16 planes without FP64 arithmetic:
// x 2^k and scale 2^-k split into float pairs by integer operations (2^k
// the scale's power of two, which keeps x 2^k inside the float range), their
// product formed in double-float (the leading product split exactly by an
// FMA), hi = T(v_hi), lo = T(v_hi - hi + v_lo).  hi + lo carries the product
// to the pair's 2^-22; hi may differ from the rounding of the exact product
// in the last place where that product lies within v_lo of a tie.
template <typename T>
__global__ void convert_split_kernel(const double* __restrict__ src, size_t n, const double* scale_dev,
                                     T* __restrict__ dst) {
  const double sc = scale_dev ? *scale_dev : 1.0;
  const int k = ic_exponent(sc);
  float ah, al;
  ic_split_f32(sc, -k, &ah, &al);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float xh, xl;
    ic_split_f32(src[i], k, &xh, &xl);
    const float p = __fmul_rn(xh, ah);
    const float c = fmaf(xh, ah, -p) + fmaf(xh, al, xl * ah);
    const float vh = __fadd_rn(p, c);
    const float vl = __fsub_rn(c, __fsub_rn(vh, p));
    const T hi = from_f32<T>(vh);
    dst[i] = hi;
    dst[n + i] = from_f32<T>(__fsub_rn(vh, to_f32<T>(hi)) + vl);
  }
}

// dst = hi + lo exactly: for FP16 by integer operations (both halves are
// multiples of 2^-24 below 2^16, so their sum is an integer count of 2^-24
// below 2^41); BF16 (a wider exponent range) in FP64
template <typename T>
__global__ void split_to_f64_kernel(const T* __restrict__ src, size_t n, double* __restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) {
      const uint16_t h = *reinterpret_cast<const uint16_t*>(src + i);
      const uint16_t l = *reinterpret_cast<const uint16_t*>(src + n + i);
      dst[i] = ic_i64_scaled(ic_f16_units(h) + ic_f16_units(l), -24);
    } else {
      dst[i] = (double)to_f32<T>(src[i]) + (double)to_f32<T>(src[n + i]);
    }
  }
}

// out[i] = sum_j x_ij^2 of the FP16/BF16 operand x = hi (+ lo) of a Newton-
// Schulz product: the exact diagonal of X^2 (row_sumsq_warp).  The tensor
// cores accumulate the diagonal's K positive terms with a downward bias that
// grows with K (about 4e-9 per term measured on this GPU: 7e-5 at K = 16384),
// which moves the fixed point of the iteration to |x| = 1 + bias/2 and the
// trace of the iterate by (d - 2k) bias/2 (0.6 at d = 16384).  Skipped (no
// writes) once *skip is set.
template <typename T>
__global__ void row_sumsq_kernel(const T* __restrict__ x, size_t plane, int split, int dp, int d,
                                 float* __restrict__ out, const int* __restrict__ skip) {
  if (skip != nullptr && *skip) return;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= dp) return;
  const double acc = row < d ? row_sumsq_warp<T>(x + (size_t)row * dp, plane, split, dp, lane) : 0.0;
  if (lane == 0) out[row] = (float)acc;
}

template <typename T>
__global__ void to_f64_kernel(const T* __restrict__ src, size_t n, double* __restrict__ dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) dst[i] = (double)src[i];
    else dst[i] = (double)to_f32<T>(src[i]);
  }
}

__global__ void normalize_kernel(double* y, int n, double* x, double* nrm) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += y[i] * y[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      const double nr = sqrt(s);
      nrm[0] = nr;
      sh[0] = nr > 0.0 ? 1.0 / nr : 0.0;  // one division for the block
    }
  }
  __syncthreads();
  const double inv = sh[0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i] * inv;
}

// G = 1/2 G + 1/2 (P1 + P1^T - P2), 32x32 tiles with a transposed read of P1
__global__ void tangent_combine_f64_kernel(double* __restrict__ G, const double* __restrict__ P1,
                                           const double* __restrict__ P2, int dp) {
  __shared__ double t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) t[r][tx] = P1[(size_t)(bj * 32 + r) * dp + bi * 32 + tx];
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const size_t e = (size_t)(bi * 32 + r) * dp + bj * 32 + tx;
    G[e] = 0.5 * G[e] + 0.5 * (P1[e] + t[tx][r] - P2[e]);
  }
}

__global__ void symmetrize_scale_kernel(const double* __restrict__ S, int dp, double scale,
                                        double* __restrict__ D) {
  __shared__ double t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) t[r][tx] = S[(size_t)(bj * 32 + r) * dp + bi * 32 + tx];
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const size_t e = (size_t)(bi * 32 + r) * dp + bj * 32 + tx;
    D[e] = 0.5 * scale * (S[e] + t[tx][r]);
  }
}

__global__ void alpha_from_rho_kernel(const double* nrm, double c, double* scal, int kscaled) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double rho = kscaled ? ldexp(nrm[0], -ic_exponent(scal[1])) : nrm[0];
    scal[3] = rho;
    scal[1] = rho > 0.0 ? 1.0 / (c * rho) : 0.0;
  }
}

__global__ void copy_unpad_kernel(const double* __restrict__ src, int dp, double* __restrict__ dst, int d) {
  const size_t n = (size_t)d * d;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / d, j = e % d;
    dst[e] = src[i * dp + j];
  }
}

__global__ void copy_pad_kernel(const double* __restrict__ src, int d, double* __restrict__ dst, int dp) {
  const size_t n = (size_t)dp * dp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / dp, j = e % dp;
    dst[e] = (i < (size_t)d && j < (size_t)d) ? src[i * d + j] : 0.0;
  }
}

int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  return (int)(g ? g : 1);
}

}  // namespace

cudaError_t copy_pad(const double* src, int d, double* dst, int dp, cudaStream_t st) {
  copy_pad_kernel<<<grid_for((size_t)dp * dp), 256, 0, st>>>(src, d, dst, dp);
  return cudaGetLastError();
}

int f64_num_tiles(int dp, int sym) { return F64Sched(dp, sym).n; }

cudaError_t f64_gemm_grouped(const F64GemmArgs& a, cudaStream_t st) {
  if (a.dp % FT || a.units == nullptr || a.n_units < 1 || !a.mat_dp || !a.mat_d) return cudaErrorInvalidValue;
  const int n = a.n_units;
  switch (a.epi) {
    case F64_EPI_STORE: f64_gemm_kernel<F64_EPI_STORE><<<n, 128, 0, st>>>(a); break;
    case F64_EPI_NS_SYRK: f64_gemm_kernel<F64_EPI_NS_SYRK><<<n, 128, 0, st>>>(a); break;
    case F64_EPI_NS_UPDATE: f64_gemm_kernel<F64_EPI_NS_UPDATE><<<n, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t f64_gemm(const F64GemmArgs& a, cudaStream_t st) {
  if (a.dp % FT || a.units != nullptr) return cudaErrorInvalidValue;
  const int n = f64_num_tiles(a.dp, a.sym);
  switch (a.epi) {
    case F64_EPI_STORE: f64_gemm_kernel<F64_EPI_STORE><<<n, 128, 0, st>>>(a); break;
    case F64_EPI_NS_SYRK: f64_gemm_kernel<F64_EPI_NS_SYRK><<<n, 128, 0, st>>>(a); break;
    case F64_EPI_NS_UPDATE: f64_gemm_kernel<F64_EPI_NS_UPDATE><<<n, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t ingest(const double* H, int d, int dp, double s, double* A, double* rowpart, int* flags,
                   cudaStream_t st) {
  dim3 grid(dp / 32, dp / 32), block(32, 8);
  ingest_kernel<<<grid, block, 0, st>>>(H, d, dp, s, A, rowpart, flags);
  return cudaGetLastError();
}

cudaError_t inf_norm_finish(const double* rowpart, int dp, double* rowsum, double* scal, cudaStream_t st) {
  rowsum_kernel<<<(dp + 255) / 256, 256, 0, st>>>(rowpart, dp, rowsum);
  max_kernel<<<1, 1024, 0, st>>>(rowsum, dp, scal);
  return cudaGetLastError();
}

cudaError_t row_sumsq(const void* x, int fmt, int split, int dp, int d, float* out, const int* skip,
                      cudaStream_t st) {
  const size_t plane = (size_t)dp * dp;
  const int blocks = (dp + 7) / 8;
  if (fmt == 0) row_sumsq_kernel<__half><<<blocks, 256, 0, st>>>((const __half*)x, plane, split, dp, d, out, skip);
  else row_sumsq_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16*)x, plane, split, dp, d, out,
                                                                  skip);
  return cudaGetLastError();
}

cudaError_t max_f64(const double* x, int n, double* out, cudaStream_t st) {
  max_kernel<<<1, 1024, 0, st>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t scale_convert(const double* src, size_t n, const double* scale_dev, double mult, void* dst,
                          int fmt, cudaStream_t st) {
  const int g = grid_for(n);
  switch (fmt) {
    case 0: scale_convert_kernel<__half><<<g, 256, 0, st>>>(src, n, scale_dev, mult, (__half*)dst); break;
    case 1: scale_convert_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(src, n, scale_dev, mult, (__nv_bfloat16*)dst); break;
    case 2: scale_convert_kernel<double><<<g, 256, 0, st>>>(src, n, scale_dev, mult, (double*)dst); break;
    case 3: scale_convert_kernel<float><<<g, 256, 0, st>>>(src, n, scale_dev, mult, (float*)dst); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t to_f64(const void* src, int fmt, size_t n, double* dst, cudaStream_t st) {
  const int g = grid_for(n);
  switch (fmt) {
    case 0: to_f64_kernel<__half><<<g, 256, 0, st>>>((const __half*)src, n, dst); break;
    case 1: to_f64_kernel<__nv_bfloat16><<<g, 256, 0, st>>>((const __nv_bfloat16*)src, n, dst); break;
    case 3: to_f64_kernel<float><<<g, 256, 0, st>>>((const float*)src, n, dst); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t scale_convert_split(const double* src, size_t n, const double* scale_dev, void* dst, int fmt,
                                cudaStream_t st) {
  const int g = grid_for(n);
  if (fmt == 0) convert_split_kernel<__half><<<g, 256, 0, st>>>(src, n, scale_dev, (__half*)dst);
  else convert_split_kernel<__nv_bfloat16><<<g, 256, 0, st>>>(src, n, scale_dev, (__nv_bfloat16*)dst);
  return cudaGetLastError();
}

cudaError_t split_to_f64(const void* src, int fmt, size_t n, double* dst, cudaStream_t st) {
  const int g = grid_for(n);
  if (fmt == 0) split_to_f64_kernel<__half><<<g, 256, 0, st>>>((const __half*)src, n, dst);
  else split_to_f64_kernel<__nv_bfloat16><<<g, 256, 0, st>>>((const __nv_bfloat16*)src, n, dst);
  return cudaGetLastError();
}

cudaError_t sum_partials(const double* partials, int n, double* out, cudaStream_t st) {
  sum_kernel<<<1, 1024, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}

cudaError_t ns_check(const double* partials, int n, double* hist, int m, double tol_abs, double floor_lo,
                     double floor_hi, double ratio, int* done, int* steps, cudaStream_t st,
                     const double* tr, int n_tr, double tr_target, double tr_tol) {
  ns_check_kernel<<<1, 1024, 0, st>>>(partials, n, hist, m, tol_abs, floor_lo, floor_hi, ratio, done, steps, tr,
                                      n_tr, tr_target, tr_tol);
  return cudaGetLastError();
}

cudaError_t trace_f64(const double* X, int dp, int d, double* out, cudaStream_t st) {
  trace_kernel<<<1, 1024, 0, st>>>(X, dp, d, out);
  return cudaGetLastError();
}

cudaError_t normalize(double* y, int n, double* x, double* nrm, cudaStream_t st) {
  normalize_kernel<<<1, 1024, 0, st>>>(y, n, x, nrm);
  return cudaGetLastError();
}

cudaError_t tangent_combine_f64(double* G, const double* P1, const double* P2, int dp, cudaStream_t st) {
  tangent_combine_f64_kernel<<<dim3(dp / 32, dp / 32), dim3(32, 8), 0, st>>>(G, P1, P2, dp);
  return cudaGetLastError();
}

cudaError_t symmetrize_scale(const double* src, int dp, double scale, double* dst, cudaStream_t st) {
  if (src == dst) return cudaErrorInvalidValue;  // tiles read transposed: out of place only
  symmetrize_scale_kernel<<<dim3(dp / 32, dp / 32), dim3(32, 8), 0, st>>>(src, dp, scale, dst);
  return cudaGetLastError();
}

cudaError_t alpha_from_rho(const double* nrm, double c, double* scal, int kscaled, cudaStream_t st) {
  alpha_from_rho_kernel<<<1, 32, 0, st>>>(nrm, c, scal, kscaled);
  return cudaGetLastError();
}

cudaError_t copy_unpad(const double* src, int dp, double* dst, int d, cudaStream_t st) {
  copy_unpad_kernel<<<grid_for((size_t)d * d), 256, 0, st>>>(src, dp, dst, d);
  return cudaGetLastError();
}

}  // namespace rsign
