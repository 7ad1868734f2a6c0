// refine.cu -- FP64-grade products on the FP16 tensor cores and the
// elementwise kernels of the commutator refinement.
//
// FP64-grade product: each operand row is written as a power-of-two scale
// times a short sum of balanced 5-bit integer digits (error-free splitting in
// the spirit of Ozaki, Ogita, Oishi and Rump's scheme, 2012).  Products of
// digit planes are integers; grouped by level t = p + q they stay below 2^24
// and therefore accumulate exactly in the FP32 TMEM accumulator of the
// tcgen05 GEMM.  The only rounding is the FP64 sum over levels in the
// epilogue and the truncation after kSlices digits (35 bits).
#include <type_traits>
#include "common.cuh"
#include "intconv.cuh"
#include "kernels.h"

#include <algorithm>
#include <cmath>

namespace rsign {
namespace {

constexpr int TILE = 32;

// ------------------------------------------------------------ digit planes
// value = mant 2^e2 exactly (mant < 2^53), for finite x
__device__ __forceinline__ void f64_parts(long long bits, unsigned long long& mant, int& e2) {
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long frac = (unsigned long long)bits & 0xFFFFFFFFFFFFFull;
  mant = E ? (frac | (1ull << 52)) : frac;
  e2 = E ? E - 1075 : -1074;
}

// E4M3 byte of a small integer |n| <= 16 (exact: at most four significant
// bits; exponent bias 7, three stored significand bits), by integer steps.
__device__ __forceinline__ uint32_t e4m3_of_int(int n) {
  const uint32_t a = (uint32_t)(n < 0 ? -n : n);
  if (a == 0) return 0u;
  const int e = 31 - __clz((int)a);  // 2^e <= a < 2^(e+1), e <= 4
  const uint32_t mant = (e <= 3 ? (a << (3 - e)) : (a >> (e - 3))) & 7u;
  return (n < 0 ? 0x80u : 0u) | ((uint32_t)(e + 7) << 3) | mant;
}

// Four digits of one plane at columns k .. k + 3 as FP16 (one 8-byte store)
// or FP8 E4M3 (one 4-byte store)
__device__ __forceinline__ void store_digit_quad(__half* planes, size_t idx, const int* dg) {
  const __half2 a = __halves2half2(__int2half_rn(dg[0]), __int2half_rn(dg[1]));
  const __half2 b = __halves2half2(__int2half_rn(dg[2]), __int2half_rn(dg[3]));
  uint2 w;
  w.x = *reinterpret_cast<const uint32_t*>(&a);
  w.y = *reinterpret_cast<const uint32_t*>(&b);
  *reinterpret_cast<uint2*>(planes + idx) = w;
}
// FP8: the E4M3 bytes of the 33 digit values -16 .. 16 come from a table in
// shared memory (filled by the block from e4m3_of_int before use)
__device__ __forceinline__ void store_digit_quad(uint8_t* planes, size_t idx, const int* dg, const uint8_t* tbl) {
  *reinterpret_cast<uint32_t*>(planes + idx) = (uint32_t)tbl[dg[0] + 16] | ((uint32_t)tbl[dg[1] + 16] << 8) |
                                               ((uint32_t)tbl[dg[2] + 16] << 16) | ((uint32_t)tbl[dg[3] + 16] << 24);
}
__device__ __forceinline__ void store_digit_quad(__half* planes, size_t idx, const int* dg, const uint8_t*) {
  store_digit_quad(planes, idx, dg);
}

// Digit planes of one row per warp (8 rows per block; grid.y = matrix).
// Everything is integer arithmetic on the FP64 bit patterns: the row scale
// sigma_i = 2^ex comes from the largest off-diagonal magnitude (compared as
// bit patterns, which order like the values), each entry becomes the
// fixed-point integer n = round(M_ik 2^(62 - ex)), |n| < 2^61, by a shift of
// its significand, and the balanced base-2^beta digits are peeled off with
// shifts; the FP64 pipe of this GPU is far slower than its integer pipe.
// Lane l handles the columns 4 l + 128 t .. 4 l + 128 t + 3 (two 16-byte
// loads, one 8- or 4-byte store per plane); row lengths are multiples of 128.
template <typename D>
__global__ void split_rows_kernel(const double* __restrict__ M, int ld, int nrows, D* __restrict__ planes,
                                  double* __restrict__ sigma, double* __restrict__ diag, int n_planes,
                                  int beta, const int* __restrict__ mat_dp, int keep_diag) {
  __shared__ uint8_t tbl[33];
  if (threadIdx.x < 33) tbl[threadIdx.x] = (uint8_t)e4m3_of_int((int)threadIdx.x - 16);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int m = blockIdx.y;
  const int ncols = mat_dp != nullptr ? mat_dp[m] : nrows;
  if (i >= ncols) return;  // outside the matrix's padded order: never read (warp-uniform)
  const size_t slot = (size_t)ld * ld;
  const long long* row = reinterpret_cast<const long long*>(M + (size_t)m * slot + (size_t)i * ld);
  long long mx = 0;
  for (int k = 4 * lane; k < ncols; k += 128) {
    const longlong2 a = *reinterpret_cast<const longlong2*>(row + k);
    const longlong2 b = *reinterpret_cast<const longlong2*>(row + k + 2);
    const long long bb[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const long long mag = bb[h] & 0x7FFFFFFFFFFFFFFFll;
      if (k + h != i || keep_diag) mx = mag > mx ? mag : mx;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  // a row without off-diagonal entries (a padding row, or a diagonal row)
  // has zero digits; its scale is the smallest normal power of two, so that
  // the largest row scale, which the refinement's level rule reads, is that
  // of the rows that have digits (a scale of 1 here made that rule depend on
  // the magnitude of H at padded orders)
  int ex = -1022;
  if (mx != 0) {
    unsigned long long mant;
    int e2;
    f64_parts(mx, mant, e2);
    const int lb = 63 - __clzll((long long)mant) + e2;  // 2^lb <= max < 2^(lb+1)
    ex = lb + 2;                                        // 2 max < 2^ex
  }
  if (lane == 0) {
    sigma[(size_t)m * ld + i] = __longlong_as_double((long long)(ex + 1023) << 52);
    diag[(size_t)m * ld + i] = __longlong_as_double(row[i]);
  }
  D* pl = planes + (size_t)m * n_planes * slot + (size_t)i * ld;
  for (int k = 4 * lane; k < ncols; k += 128) {
    const longlong2 a = *reinterpret_cast<const longlong2*>(row + k);
    const longlong2 b = *reinterpret_cast<const longlong2*>(row + k + 2);
    const long long bb[4] = {a.x, a.y, b.x, b.y};
    long long n[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const long long bits = bb[h];
      long long v = 0;
      if ((k + h != i || keep_diag) && (bits & 0x7FFFFFFFFFFFFFFFll) != 0) {  // diagonal kept apart unless keep_diag
        unsigned long long mant;
        int e2;
        f64_parts(bits, mant, e2);
        const int sh = e2 + 62 - ex;  // n = mant 2^sh, rounded to an integer
        unsigned long long q;
        if (sh >= 0) q = mant << sh;
        else if (sh > -64) q = (mant + (1ull << (-sh - 1))) >> (-sh);
        else q = 0;
        v = bits < 0 ? -(long long)q : (long long)q;
      }
      n[h] = v;
    }
    for (int p = 0; p < n_planes; ++p) {
      const int sh = 62 - beta * (p + 1);  // weight of digit p: 2^sh
      int dg[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const long long q = (n[h] + (1ll << (sh - 1))) >> sh;  // nearest, |q| <= 2^(beta-1)
        n[h] -= q * (1ll << sh);                              // |n| <= 2^(sh-1)
        dg[h] = (int)q;
      }
      store_digit_quad(pl, (size_t)p * slot + k, dg, tbl);
    }
  }
}

// ------------------------------------------------------- tiled elementwise
__device__ __forceinline__ void tile_max(float v, float* blockmax) {
  __shared__ float sm[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.y;  // blockDim = (32, 8): one warp per threadIdx.y
  if (threadIdx.x == 0) sm[w] = v;
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x == 0) {
    float m = 0.f;
    for (int q = 0; q < 8; ++q) m = fmaxf(m, sm[q]);
    blockmax[blockIdx.y * gridDim.x + blockIdx.x] = m;
  }
}

// C = N - N^T: one FP64 subtraction per element (the cancellation needs it);
// the float of the result by integer rounding, its square summed in FP32 per
// thread (four terms) and in FP64 across the tile
__global__ void antisym_kernel(const double* __restrict__ N, int dp, int k, float* __restrict__ C,
                               float* blockmax, double* part) {
  __shared__ double t[TILE][TILE + 1];
  __shared__ double sd[8];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < TILE; r += 8) t[r][tx] = N[(size_t)(bj * TILE + r) * dp + bi * TILE + tx];
  __syncthreads();
  float m = 0.f, s2f = 0.f;
  for (int r = ty; r < TILE; r += 8) {
    const size_t e = (size_t)(bi * TILE + r) * dp + bj * TILE + tx;
    float c, cl;
    ic_split_f32(N[e] - t[tx][r], k, &c, &cl);
    C[e] = c;
    m = fmaxf(m, fabsf(c));
    s2f = fmaf(c, c, s2f);
  }
  double s2 = warp_sum((double)s2f);
  if (tx == 0) sd[ty] = s2;
  tile_max(m, blockmax);  // contains __syncthreads
  if (tx == 0 && ty == 0) {
    double tt = 0.0;
    for (int q = 0; q < 8; ++q) tt += sd[q];
    part[blockIdx.y * gridDim.x + blockIdx.x] = tt;
  }
}

__global__ void newton_direction_kernel(const float* __restrict__ P, int dp, const float* sigmaC,
                                        double alpha, float* __restrict__ E, float* blockmax) {
  __shared__ float t[TILE][TILE + 1];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < TILE; r += 8) t[r][tx] = P[(size_t)(bj * TILE + r) * dp + bi * TILE + tx];
  __syncthreads();
  const float f = (float)(-0.25 * alpha) / sigmaC[0];
  float m = 0.f;
  for (int r = ty; r < TILE; r += 8) {
    const size_t e = (size_t)(bi * TILE + r) * dp + bj * TILE + tx;
    const float v = f * (P[e] + t[tx][r]);
    E[e] = v;
    m = fmaxf(m, fabsf(v));
  }
  tile_max(m, blockmax);
}

__global__ void tangent_combine_kernel(float* __restrict__ E, const float* __restrict__ P1,
                                       const float* __restrict__ P2, int dp, const float* sigma, float a,
                                       float* blockmax) {
  __shared__ float t[TILE][TILE + 1];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < TILE; r += 8) t[r][tx] = P1[(size_t)(bj * TILE + r) * dp + bi * TILE + tx];
  __syncthreads();
  const float inv = 0.5f / sigma[0];
  const float a3 = a * a * a;
  float m = 0.f;
  for (int r = ty; r < TILE; r += 8) {
    const size_t e = (size_t)(bi * TILE + r) * dp + bj * TILE + tx;
    const float v = (a == 1.0f) ? 0.5f * E[e] + inv * (P1[e] + t[tx][r] - P2[e])
                                : a * (0.5f * E[e] + inv * (P1[e] + t[tx][r])) - (a3 * inv) * P2[e];
    E[e] = v;
    m = fmaxf(m, fabsf(v));
  }
  tile_max(m, blockmax);
}

// Et = I - Y: off the diagonal -Y (a sign flip), rounded to float by integer
// operations; FP64 only on the diagonal; squares summed as in antisym_kernel
__global__ void ident_minus_kernel(const double* __restrict__ Y, int dp, int d, float* __restrict__ Et,
                                   float* blockmax, double* part) {
  __shared__ double sd[8];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  float m = 0.f, s2f = 0.f;
  for (int r = ty; r < TILE; r += 8) {
    const int i = bi * TILE + r, j = bj * TILE + tx;
    const size_t e = (size_t)i * dp + j;
    float v = 0.f, vl;
    if (i < d && j < d) {
      const double y = Y[e];
      ic_split_f32(i == j ? 1.0 - y : ic_double(ic_bits(y) ^ 0x8000000000000000ull), 0, &v, &vl);
    }
    Et[e] = v;
    m = fmaxf(m, fabsf(v));
    s2f = fmaf(v, v, s2f);
  }
  double s2 = warp_sum((double)s2f);
  if (tx == 0) sd[ty] = s2;
  tile_max(m, blockmax);  // contains __syncthreads
  if (tx == 0 && ty == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sd[q];
    part[blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void absmax_tiles_kernel(const float* __restrict__ M, int dp, float* blockmax) {
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x, ty = threadIdx.y;
  float m = 0.f;
  for (int r = ty; r < TILE; r += 8) m = fmaxf(m, fabsf(M[(size_t)(bi * TILE + r) * dp + bj * TILE + tx]));
  tile_max(m, blockmax);
}

__global__ void max_pow2_kernel(const float* __restrict__ x, int n, float* out) {
  __shared__ float sh[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, x[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, sh[w]);
    int ex = 0;
    if (mm > 0.f) frexpf(mm, &ex);  // mm = f 2^ex, f in [0.5, 1)
    out[0] = mm;
    out[1] = mm > 0.f ? ldexpf(1.f, -ex) : 1.f;  // mm * out[1] in [0.5, 1)
  }
}

template <typename T>
__global__ void scale_to_lp_kernel(const float* __restrict__ src, size_t n, const float* scale,
                                   T* __restrict__ dst) {
  // four elements per thread and iteration: one 16-byte load, one 8-byte store
  // (n is a multiple of 4)
  const float s = scale[0];
  const size_t n4 = n >> 2;
  const float4* s4 = reinterpret_cast<const float4*>(src);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = s4[i];
    const T t[4] = {from_f32<T>(v.x * s), from_f32<T>(v.y * s), from_f32<T>(v.z * s), from_f32<T>(v.w * s)};
    uint2 w;
    w.x = (uint32_t)(*reinterpret_cast<const uint16_t*>(&t[0])) |
          ((uint32_t)(*reinterpret_cast<const uint16_t*>(&t[1])) << 16);
    w.y = (uint32_t)(*reinterpret_cast<const uint16_t*>(&t[2])) |
          ((uint32_t)(*reinterpret_cast<const uint16_t*>(&t[3])) << 16);
    reinterpret_cast<uint2*>(dst)[i] = w;
  }
}

// R += E: the float converted exactly by integer operations, one FP64 add;
// ||E||_F^2 from FP32 squares (four per thread between FP64 additions)
__global__ void add_correction_kernel(double* __restrict__ R, const float* __restrict__ E, int dp, int d,
                                      double* part) {
  __shared__ double sh[32];
  double s = 0.0;
  float sf = 0.f;
  int cnt = 0;
  const size_t n = (size_t)dp * dp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float v = E[e];
    R[e] += ic_f2d(v);
    sf = fmaf(v, v, sf);
    if (++cnt == 4) {
      s += (double)sf;
      sf = 0.f;
      cnt = 0;
    }
  }
  s += (double)sf;
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// R += 1/2 P / sigma; sigma is a power of two, so the scaling is exact in
// FP32 (barring underflow); the float is converted exactly by integer
// operations: one FP64 add per element
__global__ void polish_update_kernel(double* __restrict__ R, const float* __restrict__ P, int dp,
                                     const float* sigma) {
  const float f = 0.5f / sigma[0];
  const size_t n = (size_t)dp * dp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    R[e] += ic_f2d(f * P[e]);
}

// Weight of the quintic polish step, as the FP16 operand sigma W with
// W = E + 3/4 E^2: dst = FP16(sigma E + 3/4 Q / sigma), Q = (sigma E)^2
// (FP32, from the tensor cores); four elements per thread and iteration
__global__ void polish_weight_kernel(const float* __restrict__ E, const float* __restrict__ Q, size_t n,
                                     const float* sigma, __half* __restrict__ dst) {
  const float sg = sigma[0], q = 0.75f / sigma[0];
  const size_t n4 = n >> 2;
  const float4* e4 = reinterpret_cast<const float4*>(E);
  const float4* q4 = reinterpret_cast<const float4*>(Q);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 a = e4[i], b = q4[i];
    const __half2 lo = __floats2half2_rn(fmaf(q, b.x, sg * a.x), fmaf(q, b.y, sg * a.y));
    const __half2 hi = __floats2half2_rn(fmaf(q, b.z, sg * a.z), fmaf(q, b.w, sg * a.w));
    uint2 w;
    w.x = *reinterpret_cast<const uint32_t*>(&lo);
    w.y = *reinterpret_cast<const uint32_t*>(&hi);
    reinterpret_cast<uint2*>(dst)[i] = w;
  }
}

// dst (FP16) = hi + lo of a BF16 pair of planes (plane stride n), or hi
// alone: the sum is exact in FP32, then rounded to FP16 once; two elements
// per thread and iteration
__global__ void bf16_pair_to_f16_kernel(const __nv_bfloat16* __restrict__ src, size_t n, int pair,
                                        __half* __restrict__ dst) {
  const size_t n2 = n >> 1;
  const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(src);
  const __nv_bfloat162* l2 = reinterpret_cast<const __nv_bfloat162*>(src + n);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    float2 v = __bfloat1622float2(h2[i]);
    if (pair) {
      const float2 w = __bfloat1622float2(l2[i]);
      v.x += w.x;
      v.y += w.y;
    }
    reinterpret_cast<__half2*>(dst)[i] = __floats2half2_rn(v.x, v.y);
  }
}

// The same conversion for up to kConvMax matrices in one launch (blockIdx.y
// picks the matrix): the refinement converts every stored BF16 iterate and
// residual at once.
constexpr int kConvMax = 64;
struct ConvList {
  const __nv_bfloat16* src[kConvMax];
  __half* dst[kConvMax];
};
__global__ void bf16_pairs_to_f16_kernel(const ConvList L, size_t n, int pair) {
  const size_t n2 = n >> 1;
  const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(L.src[blockIdx.y]);
  const __nv_bfloat162* l2 = reinterpret_cast<const __nv_bfloat162*>(L.src[blockIdx.y] + n);
  __half2* d2 = reinterpret_cast<__half2*>(L.dst[blockIdx.y]);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    float2 v = __bfloat1622float2(h2[i]);
    if (pair) {
      const float2 w = __bfloat1622float2(l2[i]);
      v.x += w.x;
      v.y += w.y;
    }
    d2[i] = __floats2half2_rn(v.x, v.y);
  }
}

// dst = FP16(src) by way of the nearest float (integer rounding, then the
// float -> half conversion): two elements per thread and iteration
__global__ void to_f16_kernel(const double* __restrict__ src, size_t n, __half* __restrict__ dst) {
  const size_t n2 = n >> 1;
  const double2* s2 = reinterpret_cast<const double2*>(src);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 x = s2[i];
    float a, b, al, bl;
    ic_split_f32(x.x, 0, &a, &al);
    ic_split_f32(x.y, 0, &b, &bl);
    reinterpret_cast<__half2*>(dst)[i] = __floats2half2_rn(a, b);
  }
}

// w = M v for a dp x dp FP32 matrix, one warp per row; v deterministic start
// when init != 0 (v_i = 1 + (i mod 7)/8, a vector with components along every
// eigenvector with probability one for the matrices met here).
__global__ void gemv_f32_kernel(const float* __restrict__ M, int dp, const float* __restrict__ v,
                                float* __restrict__ w, int init) {
  // FP32: a norm estimate needs no more, and the FP64 pipe is slow here.
  // One warp per row, eight 16-byte loads in flight per lane, the matrix
  // streamed past L1 (dp is a multiple of 256).
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= dp) return;
  const float4* m = reinterpret_cast<const float4*>(M + (size_t)row * dp);
  const float4* vv = reinterpret_cast<const float4*>(v);
  const int n4 = dp >> 2;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  auto chunk = [&](int j, auto n_c) {
    constexpr int NC = decltype(n_c)::value;
    float4 a[NC], b[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      const int q = j + 32 * u;
      a[u] = __ldcs(m + q);
      if (init) {
        const int e = 4 * q;
        b[u] = make_float4(1.0f + (float)(e % 7) * 0.125f, 1.0f + (float)((e + 1) % 7) * 0.125f,
                           1.0f + (float)((e + 2) % 7) * 0.125f, 1.0f + (float)((e + 3) % 7) * 0.125f);
      } else {
        b[u] = vv[q];
      }
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) {
      s0 = fmaf(a[u].x, b[u].x, s0);
      s1 = fmaf(a[u].y, b[u].y, s1);
      s2 = fmaf(a[u].z, b[u].z, s2);
      s3 = fmaf(a[u].w, b[u].w, s3);
    }
  };
  // n4 is a multiple of 64: full chunks of 256, then at most one of 128 and one of 64
  int j = lane;
  for (; j + 224 < n4; j += 256) chunk(j, std::integral_constant<int, 8>{});
  if (j + 96 < n4) { chunk(j, std::integral_constant<int, 4>{}); j += 128; }
  if (j + 32 < n4) { chunk(j, std::integral_constant<int, 2>{}); j += 64; }
  float s = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w[row] = s;
}

// v = w / ||w||; *out = ||w|| / ||v_prev|| (v_prev normalised except on the first pass)
__global__ void power_normalize_kernel(const float* __restrict__ w, int n, float* __restrict__ v, double* out,
                                       int first) {
  // squares summed in FP32 per thread (a handful of terms), then in FP64
  // across threads; one division for the block (FP64 work on one SM is slow)
  __shared__ double sh[32], sh0[32];
  __shared__ float inv_sh;
  float sf = 0.f, sf0 = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sf = fmaf(w[i], w[i], sf);
    if (first) {
      const float v0 = 1.0f + (float)(i % 7) * 0.125f;
      sf0 = fmaf(v0, v0, sf0);
    }
  }
  double s = warp_sum((double)sf), s0 = warp_sum((double)sf0);
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = s;
    sh0[threadIdx.x >> 5] = s0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0, tot0 = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      tot += sh[q];
      tot0 += sh0[q];
    }
    const double nw = sqrt(tot);
    inv_sh = nw > 0.0 ? (float)(1.0 / nw) : 0.0f;
    *out = first ? nw / sqrt(tot0) : nw;
  }
  __syncthreads();
  const float inv = inv_sh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = w[i] * inv;
}

// All the power steps of a matrix of order dp <= kPowerFusedMax in one block
// of 1024 threads: the matrix (<= 1 MB) stays in L2 between the steps and
// the call costs one launch instead of two per step (the small matrices of a
// batch run many such calls side by side, where launches, not bytes, bound
// them).  Same start vector, one warp per row as gemv_f32_kernel, and the
// same output: ||w|| / ||v0|| after a single step, else ||w|| of the last step
// (v normalised).
constexpr int kPowerFusedMax = 512;
__global__ void __launch_bounds__(1024) power_fused_kernel(const float* __restrict__ M, int dp, int iters,
                                                           double* out) {
  __shared__ float4 v4[kPowerFusedMax / 4];
  __shared__ float w[kPowerFusedMax];
  __shared__ double red[32];
  __shared__ float inv_sh;
  float* v = reinterpret_cast<float*>(v4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n4 = dp >> 2;
  float s0sq = 0.f;
  for (int i = threadIdx.x; i < dp; i += blockDim.x) {
    v[i] = 1.0f + (float)(i % 7) * 0.125f;
    s0sq = fmaf(v[i], v[i], s0sq);
  }
  double t0 = warp_sum((double)s0sq);
  if (lane == 0) red[warp] = t0;
  __syncthreads();
  double nv0 = 0.0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 32; ++q) nv0 += red[q];
    nv0 = sqrt(nv0);
  }
  for (int it = 0; it < iters; ++it) {
    for (int r = warp; r < dp; r += 32) {
      const float4* m = reinterpret_cast<const float4*>(M + (size_t)r * dp);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int q = lane; q < n4; q += 32) {
        const float4 a = m[q], b = v4[q];
        s0 = fmaf(a.x, b.x, s0);
        s1 = fmaf(a.y, b.y, s1);
        s2 = fmaf(a.z, b.z, s2);
        s3 = fmaf(a.w, b.w, s3);
      }
      float s = (s0 + s1) + (s2 + s3);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) w[r] = s;
    }
    __syncthreads();
    float sf = 0.f;
    for (int i = threadIdx.x; i < dp; i += blockDim.x) sf = fmaf(w[i], w[i], sf);
    const double t = warp_sum((double)sf);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int q = 0; q < 32; ++q) tot += red[q];
      const double nw = sqrt(tot);
      inv_sh = nw > 0.0 ? (float)(1.0 / nw) : 0.0f;
      if (it == iters - 1) *out = it == 0 ? nw / nv0 : nw;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < dp; i += blockDim.x) v[i] = w[i] * inv_sh;
    __syncthreads();
  }
}

// ---- double-float GEMVs (FP64-class products on the FP32 pipe)
// One (matrix, vectors) job: y = M x and optionally y_b = M x_b from the same
// pass over M's rows; M, x, x_b as hi + lo FP32 pairs; y in FP64 and, when
// yhi is given, also split.
struct GemvDfJob {
  const float* mhi;
  const float* mlo;
  const float* xhi;
  const float* xlo;
  const float* xbhi;  // nullable: no second vector
  const float* xblo;
  double* y;
  float* yhi;  // nullable: no split output
  float* ylo;
  double* yb;
  float* ybhi;
  float* yblo;
};
struct GemvDfArgs {
  GemvDfJob job[2];
  int n_jobs;
  int dp;
  const double* kref;  // nullable: outputs scaled by 2^-e, e the exponent of *kref
};

// s + c += (ah + al)(xh + xl): the product ah xh split exactly into p + e by
// an FMA, the cross terms ah xl + al xh (and e) added to the compensation c,
// p added to s by TwoSum with its rounding error into c (al xl, below 2^-48
// of the product, is dropped).  The _rn intrinsics keep the compiler from
// contracting the TwoSum into FMAs.
__device__ __forceinline__ void df_acc(float& s, float& c, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  const float e = fmaf(ah, xh, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c += err + fmaf(ah, xl, fmaf(al, xh, e));
}

template <bool TWO>
__device__ __forceinline__ void gemv_df_row(const GemvDfJob& J, int r, int dp, int lane, int kout) {
  const float4* mh = reinterpret_cast<const float4*>(J.mhi + (size_t)r * dp);
  const float4* ml = reinterpret_cast<const float4*>(J.mlo + (size_t)r * dp);
  const float4* xh = reinterpret_cast<const float4*>(J.xhi);
  const float4* xl = reinterpret_cast<const float4*>(J.xlo);
  const float4* bh = reinterpret_cast<const float4*>(J.xbhi);
  const float4* bl = reinterpret_cast<const float4*>(J.xblo);
  // four independent (s, c) pairs per vector, one per float4 component
  float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
  float sb[4] = {0.f, 0.f, 0.f, 0.f}, cb[4] = {0.f, 0.f, 0.f, 0.f};
  auto chunk = [&](int q0, auto n_c) {
    constexpr int U = decltype(n_c)::value;
    float4 ah[U], al[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ah[u] = __ldcs(mh + q0 + 32 * u);
      al[u] = __ldcs(ml + q0 + 32 * u);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + 32 * u;
      const float4 vh = xh[q], vl = xl[q];
      df_acc(s[0], c[0], ah[u].x, al[u].x, vh.x, vl.x);
      df_acc(s[1], c[1], ah[u].y, al[u].y, vh.y, vl.y);
      df_acc(s[2], c[2], ah[u].z, al[u].z, vh.z, vl.z);
      df_acc(s[3], c[3], ah[u].w, al[u].w, vh.w, vl.w);
      if (TWO) {
        const float4 wh = bh[q], wl = bl[q];
        df_acc(sb[0], cb[0], ah[u].x, al[u].x, wh.x, wl.x);
        df_acc(sb[1], cb[1], ah[u].y, al[u].y, wh.y, wl.y);
        df_acc(sb[2], cb[2], ah[u].z, al[u].z, wh.z, wl.z);
        df_acc(sb[3], cb[3], ah[u].w, al[u].w, wh.w, wl.w);
      }
    }
  };
  // n4 = dp / 4 is a multiple of 64: chunks of 4 float4 per lane (128 per
  // warp), then at most one chunk of 2
  const int n4 = dp >> 2;
  int q0 = lane;
  for (; q0 + 96 < n4; q0 += 128) chunk(q0, std::integral_constant<int, 4>{});
  if (q0 + 32 < n4) chunk(q0, std::integral_constant<int, 2>{});
  double t = 0.0, tb = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    t += (double)s[q] + (double)c[q];
    if (TWO) tb += (double)sb[q] + (double)cb[q];
  }
  t = warp_sum(t);
  if (TWO) tb = warp_sum(tb);
  if (kout != 0) {  // exact power-of-two rescaling
    t = ldexp(t, kout);
    if (TWO) tb = ldexp(tb, kout);
  }
  if (lane == 0) {
    J.y[r] = t;
    if (J.yhi != nullptr) {
      const float h = __double2float_rn(t);
      J.yhi[r] = h;
      J.ylo[r] = __double2float_rn(t - (double)h);
    }
    if (TWO) {
      J.yb[r] = tb;
      if (J.ybhi != nullptr) {
        const float h = __double2float_rn(tb);
        J.ybhi[r] = h;
        J.yblo[r] = __double2float_rn(tb - (double)h);
      }
    }
  }
}

// one warp per row; rows [0, dp) belong to job 0, [dp, 2 dp) to job 1
__global__ void gemv_df_kernel(const GemvDfArgs a) {
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= a.n_jobs * a.dp) return;
  const int jb = gw >= a.dp ? 1 : 0;
  const int r = gw - jb * a.dp;
  const GemvDfJob& J = a.job[jb];
  const int kout = a.kref != nullptr ? -ic_exponent(a.kref[0]) : 0;
  if (J.xbhi != nullptr) gemv_df_row<true>(J, r, a.dp, lane, kout);
  else gemv_df_row<false>(J, r, a.dp, lane, kout);
}

// ---- the same products over the upper triangle of a symmetric M
// Every 128 x 128 tile (I, J), I <= J, is read once and serves both halves:
// y_I += M_IJ x_J (its row sums) and, off the diagonal, y_J += M_IJ^T x_I
// (its column sums).  Each tile writes its partial sums, as double-float
// (s, c) pairs, to a slot of its own: the row sums of tile (I, J) to slot J
// of the rows of block I, the column sums to slot I of the rows of block J,
// so every output row gets exactly one partial per slot K = 0 .. nb-1.  A
// second pass adds the nb partials of a row in slot order (deterministic)
// and writes y like gemv_df_kernel.  Half the matrix bytes of the row
// kernel; the arithmetic per element is the same.
constexpr int kSymTile = 128;

// (s, c) += (s2, c2): TwoSum of the leading parts, the rounding error and
// the compensations into c
__device__ __forceinline__ void df_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(c2, err));
}

// tile (I, J) of the upper triangle from its linear index (row-major over I)
__host__ __device__ __forceinline__ void sym_tile(int t, int nb, int& I, int& J) {
  int r = 0;
  while (t >= nb - r) {
    t -= nb - r;
    ++r;
  }
  I = r;
  J = r + t;
}

// One CTA per (tile, job): 8 warps x 16 rows, each lane 4 columns (float4).
// Per row the lane's 4-column partial goes to shared memory (reduced over
// the 32 lanes after the loop); per column the lane accumulates over its
// warp's 16 rows in registers (reduced over the 8 warps after the loop).
// part: per job, NV vectors x nb slots x dp (s, c) pairs.
template <bool TWO>
__device__ __forceinline__ void gemv_df_sym_tile(const GemvDfJob& J_, int I, int Jt, int dp, float2* part) {
  constexpr int NV = TWO ? 2 : 1;
  // [vec][warp][row][lane] (+1 against bank conflicts), then [vec][warp][column]
  extern __shared__ float2 sym_smem[];
  float2 (*rowp)[8][16][33] = reinterpret_cast<float2 (*)[8][16][33]>(sym_smem);
  float2 (*colp)[8][kSymTile] = reinterpret_cast<float2 (*)[8][kSymTile]>(sym_smem + NV * 8 * 16 * 33);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = I * kSymTile, c0 = Jt * kSymTile;
  const bool diag = I == Jt;
  // x_J over this lane's 4 columns (row sums); x_I per row comes by broadcast
  const float4 xjh = reinterpret_cast<const float4*>(J_.xhi + c0)[lane];
  const float4 xjl = reinterpret_cast<const float4*>(J_.xlo + c0)[lane];
  float4 xbjh = make_float4(0.f, 0.f, 0.f, 0.f), xbjl = xbjh;
  if (TWO) {
    xbjh = reinterpret_cast<const float4*>(J_.xbhi + c0)[lane];
    xbjl = reinterpret_cast<const float4*>(J_.xblo + c0)[lane];
  }
  float cs[NV][4], cc[NV][4];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int q = 0; q < 4; ++q) cs[v][q] = cc[v][q] = 0.f;
#pragma unroll
  for (int rb = 0; rb < 16; rb += 4) {
    float4 mh[4], ml[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t off = (size_t)(r0 + warp * 16 + rb + u) * dp + c0;
      mh[u] = __ldcs(reinterpret_cast<const float4*>(J_.mhi + off) + lane);
      ml[u] = __ldcs(reinterpret_cast<const float4*>(J_.mlo + off) + lane);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int rl = rb + u;
      const int row = r0 + warp * 16 + rl;
      // row sum over the lane's 4 columns
      float s = 0.f, c = 0.f;
      df_acc(s, c, mh[u].x, ml[u].x, xjh.x, xjl.x);
      df_acc(s, c, mh[u].y, ml[u].y, xjh.y, xjl.y);
      df_acc(s, c, mh[u].z, ml[u].z, xjh.z, xjl.z);
      df_acc(s, c, mh[u].w, ml[u].w, xjh.w, xjl.w);
      rowp[0][warp][rl][lane] = make_float2(s, c);
      if (TWO) {
        float sb = 0.f, cb = 0.f;
        df_acc(sb, cb, mh[u].x, ml[u].x, xbjh.x, xbjl.x);
        df_acc(sb, cb, mh[u].y, ml[u].y, xbjh.y, xbjl.y);
        df_acc(sb, cb, mh[u].z, ml[u].z, xbjh.z, xbjl.z);
        df_acc(sb, cb, mh[u].w, ml[u].w, xbjh.w, xbjl.w);
        rowp[NV - 1][warp][rl][lane] = make_float2(sb, cb);
      }
      if (!diag) {
        // column sums: M_IJ^T x_I over this warp's rows
        const float xih = J_.xhi[row], xil = J_.xlo[row];
        df_acc(cs[0][0], cc[0][0], mh[u].x, ml[u].x, xih, xil);
        df_acc(cs[0][1], cc[0][1], mh[u].y, ml[u].y, xih, xil);
        df_acc(cs[0][2], cc[0][2], mh[u].z, ml[u].z, xih, xil);
        df_acc(cs[0][3], cc[0][3], mh[u].w, ml[u].w, xih, xil);
        if (TWO) {
          const float xbh = J_.xbhi[row], xbl = J_.xblo[row];
          df_acc(cs[NV - 1][0], cc[NV - 1][0], mh[u].x, ml[u].x, xbh, xbl);
          df_acc(cs[NV - 1][1], cc[NV - 1][1], mh[u].y, ml[u].y, xbh, xbl);
          df_acc(cs[NV - 1][2], cc[NV - 1][2], mh[u].z, ml[u].z, xbh, xbl);
          df_acc(cs[NV - 1][3], cc[NV - 1][3], mh[u].w, ml[u].w, xbh, xbl);
        }
      }
    }
  }
  if (!diag) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int q = 0; q < 4; ++q) colp[v][warp][4 * lane + q] = make_float2(cs[v][q], cc[v][q]);
  }
  __syncthreads();
  const int nb = dp / kSymTile;
  if (threadIdx.x < kSymTile) {
    // row t of block I: its 32 lane partials in lane order -> slot Jt
    const int t = threadIdx.x, w = t >> 4, rl = t & 15;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float s = 0.f, c = 0.f;
      for (int l = 0; l < 32; ++l) {
        const float2 p = rowp[v][w][rl][l];
        df_add(s, c, p.x, p.y);
      }
      part[((size_t)v * nb + Jt) * dp + r0 + t] = make_float2(s, c);
    }
  } else if (!diag) {
    // column t of block Jt: its 8 warp partials in warp order -> slot I
    const int t = threadIdx.x - kSymTile;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float s = 0.f, c = 0.f;
      for (int w = 0; w < 8; ++w) {
        const float2 p = colp[v][w][t];
        df_add(s, c, p.x, p.y);
      }
      part[((size_t)v * nb + I) * dp + c0 + t] = make_float2(s, c);
    }
  }
}

// grid.x = tiles of the upper triangle, grid.y = job; 256 threads
__global__ void __launch_bounds__(256) gemv_df_sym_kernel(const GemvDfArgs a, float2* part) {
  const int nb = a.dp / kSymTile;
  int I, Jt;
  sym_tile(blockIdx.x, nb, I, Jt);
  const GemvDfJob& J_ = a.job[blockIdx.y];
  float2* pj = part + (size_t)blockIdx.y * 2 * nb * a.dp;  // room for two vectors per job
  if (J_.xbhi != nullptr) gemv_df_sym_tile<true>(J_, I, Jt, a.dp, pj);
  else gemv_df_sym_tile<false>(J_, I, Jt, a.dp, pj);
}

constexpr int kSymSmem = 2 * (8 * 16 * 33 + 8 * kSymTile) * (int)sizeof(float2);  // two vectors

// y_i = the sum of its nb partials (double-float), then FP64; the outputs as
// gemv_df_row writes them.  Four consecutive lanes per (job, row), each
// adding a quarter of the slots in slot order; the quarters are combined in
// a fixed pattern ((q0 + q1) + (q2 + q3)), so the result does not depend on
// the launch.
__global__ void gemv_df_sym_reduce_kernel(const GemvDfArgs a, const float2* part) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gi = gt >> 2, q = gt & 3;
  const bool live = gi < a.n_jobs * a.dp;  // whole groups of four: the shuffles below stay in step
  const int jb = live && gi >= a.dp ? 1 : 0;
  const int r = live ? gi - jb * a.dp : 0;
  const GemvDfJob& J = a.job[jb];
  const int nb = a.dp / kSymTile;
  const int k0 = (q * nb) / 4, k1 = ((q + 1) * nb) / 4;  // the quarters cover 0 .. nb-1
  const float2* pj = part + (size_t)jb * 2 * nb * a.dp;
  const bool two = J.xbhi != nullptr;
  const int kout = live && a.kref != nullptr ? -ic_exponent(a.kref[0]) : 0;
  for (int v = 0; v < 2; ++v) {
    float s = 0.f, c = 0.f;
    if (live && (v == 0 || two))
      for (int k = k0; k < k1; ++k) {
        const float2 p = pj[((size_t)v * nb + k) * a.dp + r];
        df_add(s, c, p.x, p.y);
      }
    // (q0 + q1), (q2 + q3), then their sum, in lanes q = 0 and 2, then 0
    float s1 = __shfl_down_sync(0xffffffffu, s, 1), c1 = __shfl_down_sync(0xffffffffu, c, 1);
    if ((q & 1) == 0) df_add(s, c, s1, c1);
    s1 = __shfl_down_sync(0xffffffffu, s, 2);
    c1 = __shfl_down_sync(0xffffffffu, c, 2);
    if (q == 0) df_add(s, c, s1, c1);
    if (!live || q != 0 || (v == 1 && !two)) continue;
    double t = (double)s + (double)c;
    if (kout != 0) t = ldexp(t, kout);
    double* y = v == 0 ? J.y : J.yb;
    float* yh = v == 0 ? J.yhi : J.ybhi;
    float* yl = v == 0 ? J.ylo : J.yblo;
    y[r] = t;
    if (yh != nullptr) {
      const float h = __double2float_rn(t);
      yh[r] = h;
      yl[r] = __double2float_rn(t - (double)h);
    }
  }
}

// hi + lo = src 2^k (k = k_host, plus the exponent of *kref when given), by
// integer operations (ic_split_f32): two float2 stores per pair of elements
__global__ void split_f32_kernel(const double* __restrict__ src, size_t n, float* __restrict__ hi,
                                 float* __restrict__ lo, int k_host, const double* __restrict__ kref) {
  const int k = k_host + (kref != nullptr ? ic_exponent(kref[0]) : 0);
  const size_t n2 = n >> 1;  // n is even (dp^2 or dp)
  const double2* s2 = reinterpret_cast<const double2*>(src);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 x = s2[i];
    float2 h, l;
    ic_split_f32(x.x, k, &h.x, &l.x);
    ic_split_f32(x.y, k, &h.y, &l.y);
    reinterpret_cast<float2*>(hi)[i] = h;
    if (lo != nullptr) reinterpret_cast<float2*>(lo)[i] = l;
  }
}

// The step's two normalisations in one launch: block 0 takes w = a0 - b0
// (C v), block 1 w = a1 - b1 (N z); each writes v = w / ||w|| in FP64 and as
// hi + lo FP32 pairs and *out = ||w||.  w is formed twice (for the norm and
// for v) instead of being stored.
struct DiffNormJob {
  const double* a;
  const double* b;
  double* v;
  float* vhi;
  float* vlo;
  double* out;
};
__global__ void diff_normalize2_kernel(DiffNormJob j0, DiffNormJob j1, int n) {
  const DiffNormJob& J = blockIdx.x == 0 ? j0 : j1;
  __shared__ double sh[32];
  __shared__ double inv_sh;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double w = J.a[i] - J.b[i];
    s = fma(w, w, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += sh[q];
    const double nw = sqrt(tot);
    inv_sh = nw > 0.0 ? 1.0 / nw : 0.0;
    *J.out = nw;
  }
  __syncthreads();
  const double inv = inv_sh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = (J.a[i] - J.b[i]) * inv;
    J.v[i] = x;
    const float h = __double2float_rn(x);
    J.vhi[i] = h;
    J.vlo[i] = __double2float_rn(x - (double)h);
  }
}

// *bits = max |x_i| as the bit pattern of a non-negative double (which orders
// like an unsigned integer), by integer operations
__global__ void maxabs_bits_kernel(const double* __restrict__ x, size_t n, unsigned long long* bits) {
  unsigned long long m = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long b = ic_bits(x[i]) & 0x7FFFFFFFFFFFFFFFull;
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(bits, m);
}

// *out = 1 / max (1 when the maximum is 0 or not finite)
__global__ void inv_of_bits_kernel(const unsigned long long* bits, double* out) {
  if (threadIdx.x == 0) {
    const double m = ic_double(*bits);
    *out = (m > 0.0 && m < 1.0e300) ? 1.0 / m : 1.0;
  }
}

// v = w / ||w|| in FP64 and as hi + lo FP32 pairs; *out = ||w|| (one block)
__global__ void normalize_split_kernel(const double* __restrict__ w, int n, double* __restrict__ v,
                                       float* __restrict__ vhi, float* __restrict__ vlo, double* out) {
  __shared__ double sh[32];
  __shared__ double inv_sh;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(w[i], w[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += sh[q];
    const double nw = sqrt(tot);
    inv_sh = nw > 0.0 ? 1.0 / nw : 0.0;
    *out = nw;
  }
  __syncthreads();
  const double inv = inv_sh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = w[i] * inv;
    v[i] = x;
    const float h = __double2float_rn(x);
    vhi[i] = h;
    vlo[i] = __double2float_rn(x - (double)h);
  }
}

__global__ void scale_scalar_kernel(double* x, double f) { x[0] *= f; }

// out[0..2] = a.b, c.e, f.g over n entries (one block)
__global__ void dot3_kernel(const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ c, const double* __restrict__ e,
                            const double* __restrict__ f, const double* __restrict__ g, int n,
                            double* __restrict__ out) {
  __shared__ double sh[3][32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s0 = fma(a[i], b[i], s0);
    s1 = fma(c[i], e[i], s1);
    s2 = fma(f[i], g[i], s2);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][wid] = s0;
    sh[1][wid] = s1;
    sh[2][wid] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
    out[threadIdx.x] = t;
  }
}

__global__ void start_vec_f64_kernel(double* y, int d, int dp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < dp; i += gridDim.x * blockDim.x)
    y[i] = (i < d) ? 1.0 + (i % 7) * 0.125 : 0.0;
}

dim3 tiles_of(int dp) { return dim3(dp / TILE, dp / TILE); }
int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  return (int)(g ? g : 1);
}

}  // namespace

static bool split_ok(const SplitMat& o) {
  return o.n_planes >= 1 && o.n_planes * o.beta <= 56 && o.beta >= 2 && o.beta <= 11 && (!o.fp8 || o.beta <= 5);
}

cudaError_t split_rows(const double* M, int dp, SplitMat out, cudaStream_t st) {
  if (!split_ok(out)) return cudaErrorInvalidValue;
  const dim3 grid((dp + 7) / 8, 1);
  if (out.fp8)
    split_rows_kernel<uint8_t><<<grid, 256, 0, st>>>(M, dp, dp, (uint8_t*)out.planes, out.sigma, out.diag,
                                                     out.n_planes, out.beta, nullptr, out.keep_diag);
  else
    split_rows_kernel<__half><<<grid, 256, 0, st>>>(M, dp, dp, (__half*)out.planes, out.sigma, out.diag,
                                                    out.n_planes, out.beta, nullptr, out.keep_diag);
  return cudaGetLastError();
}

cudaError_t split_rows_grouped(const double* M, int D, int n_mat, const int* mat_dp, SplitMat out,
                               cudaStream_t st) {
  if (!split_ok(out)) return cudaErrorInvalidValue;
  const dim3 grid((D + 7) / 8, n_mat);
  if (out.fp8)
    split_rows_kernel<uint8_t><<<grid, 256, 0, st>>>(M, D, D, (uint8_t*)out.planes, out.sigma, out.diag,
                                                     out.n_planes, out.beta, mat_dp, out.keep_diag);
  else
    split_rows_kernel<__half><<<grid, 256, 0, st>>>(M, D, D, (__half*)out.planes, out.sigma, out.diag,
                                                    out.n_planes, out.beta, mat_dp, out.keep_diag);
  return cudaGetLastError();
}

int fp64e_planes(int beta) { return beta > 0 ? (54 + beta - 1) / beta : 0; }

int fp64e_beta(int k_extent) {
  // the widest digit whose pair products are exact in FP32 (2^(2 beta - 2) K
  // <= 2^24 for one pair) and whose full product fits the kernel's limits:
  // P (P + 1) / 2 pair products and one group per (level, max_pairs pairs)
  for (int b = 7; b >= 5; --b) {
    const double bound1 = std::ldexp(1.0, 2 * b - 2) * (double)k_extent;
    const int max_pairs = (int)std::floor(std::ldexp(1.0, 24) / bound1);
    if (max_pairs < 1) continue;
    const int P = fp64e_planes(b);
    if (P * (P + 1) / 2 > kTcMaxPairs) continue;
    int groups = 0;
    for (int t = 0; t < P; ++t) groups += (t + 1 + max_pairs - 1) / max_pairs;
    if (groups <= kTcMaxGroups) return b;
  }
  return 0;
}

cudaError_t fp64e_plan(TcGemmArgs* a, int n_planes, int beta, int levels, int k_extent) {
  const int L = levels < 1 ? 1 : (levels > n_planes ? n_planes : levels);
  // |digit| <= 2^(beta-1): a group of n pairs sums to at most n 2^(2 beta - 2) K
  const double bound1 = std::ldexp(1.0, 2 * beta - 2) * (double)k_extent;
  const int max_pairs = (int)std::floor(std::ldexp(1.0, 24) / bound1);
  if (max_pairs < 1) return cudaErrorInvalidValue;
  int np = 0, ng = 0;
  std::vector<int> level_groups(L, 0), group_level;
  for (int t = 0; t < L; ++t) {  // levels 0 .. L-1 (truncation after beta L bits)
    int in_group = 0;
    for (int p = 0; p <= t; ++p) {
      const int q = t - p;
      if (p >= n_planes || q >= n_planes) continue;
      if (in_group == 0) {
        if (ng >= kTcMaxGroups) return cudaErrorInvalidValue;
        a->group_start[ng] = np;
        a->group_scale[ng] = std::ldexp(1.0, -beta * (t + 2));
        group_level.push_back(t);
        ++level_groups[t];
        ++ng;
      }
      if (np >= kTcMaxPairs) return cudaErrorInvalidValue;
      a->pair_a[np] = p;
      a->pair_b[np] = q;
      ++np;
      if (++in_group == max_pairs) in_group = 0;
    }
  }
  a->n_groups = ng;
  a->group_start[ng] = np;
  // Super-groups: levels t0..t1 share one int64 sum V = sum acc_t 2^(beta (t1 - t))
  // while its bound sum_t groups_t 2^(24 + beta (t1 - t)) stays below 2^62.
  auto bound = [&](int t0, int t1) {
    double b = 0.0;
    for (int t = t0; t <= t1; ++t) b += level_groups[t] * std::ldexp(1.0, 24 + beta * (t1 - t));
    return b;
  };
  const double lim = std::ldexp(1.0, 62);
  a->oz_unit_exp = -beta * (L - 1 + 2);
  if (bound(0, L - 1) < lim) {
    a->n_sg = 0;
    for (int g = 0; g < ng; ++g) a->group_shift[g] = beta * (L - 1 - group_level[g]);
    a->final_scale = std::ldexp(1.0, -beta * (L - 1 + 2));
    // One exact int64 sum: any group order gives the same bits.  The groups
    // run from the top level down, so that the heaviest epilogue (the last
    // group's conversion to FP64) overlaps the next tile's longest group
    // (the most pair products) instead of its shortest.
    int pa[kTcMaxPairs], pb[kTcMaxPairs], gs[kTcMaxGroups + 1], sh[kTcMaxGroups];
    double sc[kTcMaxGroups];
    int q = 0;
    for (int g = ng - 1, h = 0; g >= 0; --g, ++h) {
      gs[h] = q;
      sc[h] = a->group_scale[g];
      sh[h] = a->group_shift[g];
      for (int r = a->group_start[g]; r < a->group_start[g + 1]; ++r, ++q) {
        pa[q] = a->pair_a[r];
        pb[q] = a->pair_b[r];
      }
    }
    gs[ng] = q;
    for (int g = 0; g <= ng; ++g) a->group_start[g] = gs[g];
    for (int g = 0; g < ng; ++g) {
      a->group_scale[g] = sc[g];
      a->group_shift[g] = sh[g];
    }
    for (int r = 0; r < q; ++r) {
      a->pair_a[r] = pa[r];
      a->pair_b[r] = pb[r];
    }
    return cudaSuccess;
  }
  int split = L - 1;  // super-group 1 = levels split .. L-1, as long as it fits
  while (split > 0 && bound(split - 1, L - 1) < lim) --split;
  if (!(bound(0, split - 1) < lim)) return cudaErrorInvalidValue;  // would need three sums
  a->n_sg = 2;
  for (int g = 0; g < ng; ++g) {
    const int t = group_level[g];
    const int s = t >= split ? 1 : 0;
    const int t1 = s ? L - 1 : split - 1;
    a->group_sg[g] = s;
    a->group_shift[g] = beta * (t1 - t);
    a->group_first[g] = (g == 0 || a->group_sg[g - 1] != s) ? 1 : 0;
  }
  a->sg_weight[0] = std::ldexp(1.0, -beta * (split - 1 + 2));
  a->sg_weight[1] = std::ldexp(1.0, -beta * (L - 1 + 2));
  a->oz_sh01 = beta * (L - 1 - (split - 1));
  // Within each super-group the sum is exact in any order: the groups run
  // from the top level down (super-group 0 first, as the parking of its sum
  // needs), so that the last group's conversion overlaps the next tile's
  // group with the most pair products.
  {
    int pa[kTcMaxPairs], pb[kTcMaxPairs], gs[kTcMaxGroups + 1], sh[kTcMaxGroups], sgv[kTcMaxGroups];
    double sc[kTcMaxGroups];
    int q = 0, h = 0;
    for (int s = 0; s < 2; ++s)
      for (int g = ng - 1; g >= 0; --g) {
        if (a->group_sg[g] != s) continue;
        gs[h] = q;
        sc[h] = a->group_scale[g];
        sh[h] = a->group_shift[g];
        sgv[h] = s;
        for (int r = a->group_start[g]; r < a->group_start[g + 1]; ++r, ++q) {
          pa[q] = a->pair_a[r];
          pb[q] = a->pair_b[r];
        }
        ++h;
      }
    gs[ng] = q;
    for (int g = 0; g <= ng; ++g) a->group_start[g] = gs[g];
    for (int g = 0; g < ng; ++g) {
      a->group_scale[g] = sc[g];
      a->group_shift[g] = sh[g];
      a->group_sg[g] = sgv[g];
      a->group_first[g] = (g == 0 || sgv[g - 1] != sgv[g]) ? 1 : 0;
    }
    for (int r = 0; r < q; ++r) {
      a->pair_a[r] = pa[r];
      a->pair_b[r] = pb[r];
    }
  }
  return cudaSuccess;
}

cudaError_t ozaki_gemm(const SplitMat& A, const SplitMat& B, int dp, int d_real, int sym, double* out,
                       int* status, int num_sms, cudaStream_t st, int levels, const OzTiles* tiles) {
  Fp64eExtra x{};
  if (tiles != nullptr) {  // 128 x 128 tiles, int64 level sums in TMEM (grouped mode, one matrix)
    x.units = tiles->units;
    x.n_units = tiles->n_units;
    x.n_mat = 1;
    x.bn = 128;
    x.mat_dp = tiles->dims;
    x.mat_d = tiles->dims + 1;
  }
  return fp64e_gemm(A, B, dp, d_real, sym, out, x, status, num_sms, st, levels);
}

cudaError_t fp64e_gemm(const SplitMat& A, const SplitMat& B, int dp, int d_real, int sym, double* out,
                       const Fp64eExtra& x, int* status, int num_sms, cudaStream_t st, int levels) {
  if (A.beta != B.beta || A.n_planes != B.n_planes || A.keep_diag != B.keep_diag || A.fp8 != B.fp8)
    return cudaErrorInvalidValue;
  const int fmt = A.fp8 ? 2 : 0;
  TcGemmArgs a{};
  a.dp = dp;
  a.d_real = d_real;
  a.sym = sym;
  a.epi = TC_EPI_OZAKI;
  a.scale = 1.0f;
  a.out = out;
  a.rs = A.sigma;
  a.cs = B.sigma;
  a.status = status;
  a.skip = x.skip;
  // exact diagonal terms only for diagonal-free digits
  a.a_full = A.keep_diag ? nullptr : A.full;
  a.b_full = A.keep_diag ? nullptr : B.full;
  a.a_diag = A.diag;
  a.b_diag = B.diag;
  a.acc64 = x.acc64;
  a.xin64 = x.xin64;
  a.xin_mult = x.xin_mult;
  {
    int ex = 0;
    const double f = std::frexp(x.xin_mult, &ex);
    if (f != 0.5) return cudaErrorInvalidValue;  // the multiplier must be a power of two
    a.xin_mult_exp = ex - 1;
  }
  a.oz_ident = x.ident;
  a.partials = x.partials;
  const int kext = x.k_extent > 0 ? x.k_extent : d_real;
  cudaError_t e = fp64e_plan(&a, A.n_planes, A.beta, levels, kext);
  if (e != cudaSuccess) return e;
  if (a.n_sg == 2 && a.acc64 == nullptr) return cudaErrorInvalidValue;
  if (x.units == nullptr) return tc_gemm(a, A.planes, A.n_planes, B.planes, B.n_planes, fmt, num_sms, st);
  a.units = x.units;
  a.n_units = x.n_units;
  a.mat_dp = x.mat_dp;
  a.mat_d = x.mat_d;
  a.mat_skip = x.mat_skip;
  a.mat_stride = (long long)dp * dp;
  a.mat_vec_stride = dp;
  a.a_planes = A.n_planes;
  a.b_planes = B.n_planes;
 
  return tc_gemm_grouped(a, x.bn, A.planes, x.n_mat * A.n_planes, B.planes, x.n_mat * B.n_planes, fmt, num_sms,
                         st);
}

cudaError_t antisym_part(const double* N, int dp, int k, float* C, float* blockmax, double* part,
                         cudaStream_t st) {
  antisym_kernel<<<tiles_of(dp), dim3(32, 8), 0, st>>>(N, dp, k, C, blockmax, part);
  return cudaGetLastError();
}

cudaError_t absmax_tiles(const float* M, int dp, float* blockmax, cudaStream_t st) {
  absmax_tiles_kernel<<<tiles_of(dp), dim3(32, 8), 0, st>>>(M, dp, blockmax);
  return cudaGetLastError();
}

cudaError_t max_pow2(const float* x, int n, float* out, cudaStream_t st) {
  max_pow2_kernel<<<1, 1024, 0, st>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t scale_to_lp(const float* src, size_t n, const float* scale, void* dst, int fmt, cudaStream_t st) {
  if (n & 3) return cudaErrorInvalidValue;
  if (fmt == 0) scale_to_lp_kernel<__half><<<grid_for(n / 4), 256, 0, st>>>(src, n, scale, (__half*)dst);
  else scale_to_lp_kernel<__nv_bfloat16><<<grid_for(n / 4), 256, 0, st>>>(src, n, scale, (__nv_bfloat16*)dst);
  return cudaGetLastError();
}

cudaError_t newton_direction(const float* P, int dp, const float* sigmaC, double alpha, float* E,
                             float* blockmax, cudaStream_t st) {
  newton_direction_kernel<<<tiles_of(dp), dim3(32, 8), 0, st>>>(P, dp, sigmaC, alpha, E, blockmax);
  return cudaGetLastError();
}

cudaError_t tangent_combine(float* E, const float* P1, const float* P2, int dp, const float* sigma, float a,
                            float* blockmax, cudaStream_t st) {
  tangent_combine_kernel<<<tiles_of(dp), dim3(32, 8), 0, st>>>(E, P1, P2, dp, sigma, a, blockmax);
  return cudaGetLastError();
}

cudaError_t add_correction(double* R, const float* E, int dp, int d, double* part, cudaStream_t st) {
  (void)d;
  add_correction_kernel<<<1024, 256, 0, st>>>(R, E, dp, d, part);
  return cudaGetLastError();
}

cudaError_t ident_minus(const double* Y, int dp, int d, float* Et, float* blockmax, double* part,
                        cudaStream_t st) {
  ident_minus_kernel<<<tiles_of(dp), dim3(32, 8), 0, st>>>(Y, dp, d, Et, blockmax, part);
  return cudaGetLastError();
}

int spectral_norm_launches(int dp, int iters) { return dp <= kPowerFusedMax ? 1 : 2 * iters; }

cudaError_t spectral_norm_f32(const float* M, int dp, float* v, float* w, int iters, double* out,
                              cudaStream_t st, bool per_step) {
  if (iters < 1) return cudaErrorInvalidValue;
  if (dp <= kPowerFusedMax && !per_step) {
    power_fused_kernel<<<1, 1024, 0, st>>>(M, dp, iters, out);
    return cudaGetLastError();
  }
  for (int it = 0; it < iters; ++it) {
    gemv_f32_kernel<<<(dp + 7) / 8, 256, 0, st>>>(M, dp, v, w, it == 0 ? 1 : 0);
    power_normalize_kernel<<<1, 1024, 0, st>>>(w, dp, v, out, it == 0 ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t gemv_df(const float* M_hi, const float* M_lo, const float* x_hi, const float* x_lo, double* y, int dp,
                    cudaStream_t st, const double* kref) {
  GemvDfArgs a{};
  a.n_jobs = 1;
  a.dp = dp;
  a.kref = kref;
  a.job[0] = GemvDfJob{M_hi, M_lo, x_hi, x_lo, nullptr, nullptr, y, nullptr, nullptr, nullptr, nullptr, nullptr};
  gemv_df_kernel<<<(dp + 7) / 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}

int gemv_df_sym_tiles(int dp, int* I, int* J) {
  const int nb = dp / kSymTile, n = nb * (nb + 1) / 2;
  if (I != nullptr && J != nullptr)
    for (int t = 0; t < n; ++t) sym_tile(t, nb, I[t], J[t]);
  return n;
}

size_t gemv_df_sym_part_bytes(int dp) { return (size_t)2 * 2 * (dp / kSymTile) * dp * sizeof(float2); }

// One or two jobs of y = M x (symmetric M) over the upper triangle: the tile
// pass and the slot-order reduction (two launches).
cudaError_t gemv_df_sym_run(const GemvDfArgs& a, float2* part, cudaStream_t st) {
  if (a.dp % kSymTile != 0 || a.n_jobs < 1 || a.n_jobs > 2 || part == nullptr) return cudaErrorInvalidValue;
  static cudaError_t attr = cudaFuncSetAttribute(gemv_df_sym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 kSymSmem);
  if (attr != cudaSuccess) return attr;
  const int nb = a.dp / kSymTile;
  gemv_df_sym_kernel<<<dim3(nb * (nb + 1) / 2, a.n_jobs), 256, kSymSmem, st>>>(a, part);
  gemv_df_sym_reduce_kernel<<<(4 * a.n_jobs * a.dp + 255) / 256, 256, 0, st>>>(a, part);
  return cudaGetLastError();
}

cudaError_t gemv_df_sym(const float* M_hi, const float* M_lo, const float* x_hi, const float* x_lo, double* y,
                        int dp, float2* part, cudaStream_t st) {
  GemvDfArgs a{};
  a.n_jobs = 1;
  a.dp = dp;
  a.job[0] = GemvDfJob{M_hi, M_lo, x_hi, x_lo, nullptr, nullptr, y, nullptr, nullptr, nullptr, nullptr, nullptr};
  return gemv_df_sym_run(a, part, st);
}

cudaError_t inv_maxabs(const double* x, size_t n, unsigned long long* bits, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  maxabs_bits_kernel<<<grid_for(n), 256, 0, st>>>(x, n, bits);
  inv_of_bits_kernel<<<1, 32, 0, st>>>(bits, out);
  return cudaGetLastError();
}

cudaError_t split_f32(const double* src, size_t n, float* hi, float* lo, int k, const double* kref,
                      cudaStream_t st) {
  if (n & 1) return cudaErrorInvalidValue;
  split_f32_kernel<<<grid_for(n / 2), 256, 0, st>>>(src, n, hi, lo, k, kref);
  return cudaGetLastError();
}

// Above this order the check's products read the upper triangles only (half
// the bytes, two launches per product); up to it the row kernel (one launch:
// small matrices are bound by launches, not bytes).
constexpr int kCheckSymMin = 1024;

// one double-float product pass of the check, by the form its order takes
static cudaError_t check_pass(const GemvDfArgs& a, float2* part, cudaStream_t st) {
  if (a.dp > kCheckSymMin) return gemv_df_sym_run(a, part, st);
  gemv_df_kernel<<<(a.n_jobs * a.dp + 7) / 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}

int commutator_check_launches(int dp, int iters) {
  const int per_pass = dp > kCheckSymMin ? 2 : 1;
  return 4 + iters * (2 * per_pass + 1) + per_pass + 2;
}

cudaError_t commutator_gain_norm(const float* A_hi, const float* A_lo, const double* R, float* R_hi,
                                 float* R_lo, int dp, int d, int iters, double* work, float* fwork,
                                 float2* part, double* out, cudaStream_t st) {
  if (iters < 1) return cudaErrorInvalidValue;
  // FP64 vectors
  double* vb[2] = {work, work + dp};  // unit vectors of the commutator steps (alternating)
  double* t1 = work + 2 * dp;         // A v
  double* t2 = work + 3 * dp;         // R v
  double* y1 = work + 4 * dp;         // R A v
  double* y2 = work + 5 * dp;         // A R v
  double* w = work + 6 * dp;          // C v
  double* z = work + 7 * dp;          // unit vector of the involution-residual steps
  double* t3 = work + 8 * dp;         // R z
  double* y3 = work + 9 * dp;         // R R z
  double* w3 = work + 10 * dp;        // (R^2 - I) z
  double* t4 = work + 11 * dp;        // A v_last
  // hi/lo FP32 copies of the vectors that enter a product
  float* vbh[2] = {fwork, fwork + 2 * dp};
  float* vbl[2] = {fwork + dp, fwork + 3 * dp};
  float *zh = fwork + 4 * dp, *zl = fwork + 5 * dp;
  float *t1h = fwork + 6 * dp, *t1l = fwork + 7 * dp;
  float *t2h = fwork + 8 * dp, *t2l = fwork + 9 * dp;
  float *t3h = fwork + 10 * dp, *t3l = fwork + 11 * dp;
  const size_t dd = (size_t)dp * dp;
  split_f32_kernel<<<grid_for(dd / 2), 256, 0, st>>>(R, dd, R_hi, R_lo, 0, nullptr);
  start_vec_f64_kernel<<<(dp + 255) / 256, 256, 0, st>>>(w, d, dp);
  normalize_split_kernel<<<1, 1024, 0, st>>>(w, dp, vb[0], vbh[0], vbl[0], out);
  normalize_split_kernel<<<1, 1024, 0, st>>>(w, dp, z, zh, zl, out + 1);
  // ||R C v|| = ||C v|| for the (orthogonal to working accuracy) R, so the
  // steps run on the antisymmetric C itself: v <- C v / ||C v|| turns within
  // the dominant invariant plane (eigenvalues +-i mu) and ||C v|| -> mu =
  // ||C||_2, as fast as power steps on C^2.  Power steps on the symmetric
  // N = R^2 - I ride along in the same passes over A and R.
  for (int it = 0; it < iters; ++it) {
    const int cur = it & 1, nxt = (it + 1) & 1;
    GemvDfArgs p1{};
    p1.n_jobs = 2;
    p1.dp = dp;
    p1.job[0] = GemvDfJob{A_hi, A_lo, vbh[cur], vbl[cur], nullptr, nullptr, t1, t1h, t1l, nullptr, nullptr, nullptr};
    p1.job[1] = GemvDfJob{R_hi, R_lo, vbh[cur], vbl[cur], zh, zl, t2, t2h, t2l, t3, t3h, t3l};
    cudaError_t e = check_pass(p1, part, st);  // A v; R v, R z
    if (e != cudaSuccess) return e;
    GemvDfArgs p2{};
    p2.n_jobs = 2;
    p2.dp = dp;
    p2.job[0] = GemvDfJob{R_hi, R_lo, t1h, t1l, t3h, t3l, y1, nullptr, nullptr, y3, nullptr, nullptr};
    p2.job[1] = GemvDfJob{A_hi, A_lo, t2h, t2l, nullptr, nullptr, y2, nullptr, nullptr, nullptr, nullptr, nullptr};
    e = check_pass(p2, part, st);  // R A v, R R z; A R v
    if (e != cudaSuccess) return e;
    // v <- C v / ||C v|| (C v = R A v - A R v), z <- N z / ||N z|| (N z = R R z - z)
    diff_normalize2_kernel<<<2, 1024, 0, st>>>(DiffNormJob{y1, y2, vb[nxt], vbh[nxt], vbl[nxt], out},
                                               DiffNormJob{y3, z, w3, zh, zl, out + 1}, dp);
    std::swap(z, w3);
  }
  // Rayleigh-Ritz on the last plane {v_prev, v_last = C v_prev / ||C v_prev||}
  // (orthonormal: v^T C v = 0 for the antisymmetric C): the entries of the
  // 2 x 2 projection of A, out[2..4] = v_prev.A v_prev, v_last.A v_prev,
  // v_last.A v_last
  const int last = iters & 1, prev = (iters - 1) & 1;
  GemvDfArgs p3{};
  p3.n_jobs = 1;
  p3.dp = dp;
  p3.job[0] = GemvDfJob{A_hi, A_lo, vbh[last], vbl[last], nullptr, nullptr, t4, nullptr, nullptr, nullptr, nullptr,
                        nullptr};
  cudaError_t e = check_pass(p3, part, st);
  if (e != cudaSuccess) return e;
  dot3_kernel<<<1, 1024, 0, st>>>(vb[prev], t1, vb[last], t1, vb[last], t4, dp, out + 2);
  // out[0] = ||C v_prev|| = 2 ||G v_prev|| (G = 1/2 R C): halve it
  scale_scalar_kernel<<<1, 1, 0, st>>>(out, 0.5);
  return cudaGetLastError();
}

cudaError_t to_f16(const double* src, size_t n, void* dst, cudaStream_t st) {
  if (n & 1) return cudaErrorInvalidValue;
  to_f16_kernel<<<grid_for(n / 2), 256, 0, st>>>(src, n, (__half*)dst);
  return cudaGetLastError();
}

cudaError_t bf16_pair_to_f16(const void* src, size_t n, int pair, void* dst, cudaStream_t st) {
  if (n & 1) return cudaErrorInvalidValue;
  bf16_pair_to_f16_kernel<<<grid_for(n / 2), 256, 0, st>>>((const __nv_bfloat16*)src, n, pair, (__half*)dst);
  return cudaGetLastError();
}

cudaError_t bf16_pairs_to_f16(const void* const* src, void* const* dst, int count, size_t n, int pair,
                              cudaStream_t st) {
  if (n & 1) return cudaErrorInvalidValue;
  for (int b = 0; b < count; b += kConvMax) {
    ConvList L{};
    const int m = std::min(kConvMax, count - b);
    for (int q = 0; q < m; ++q) {
      L.src[q] = (const __nv_bfloat16*)src[b + q];
      L.dst[q] = (__half*)dst[b + q];
    }
    const int gx = std::max(1, grid_for(n / 2) / std::max(1, m / 4));
    bf16_pairs_to_f16_kernel<<<dim3(gx, m), 256, 0, st>>>(L, n, pair);
  }
  return cudaGetLastError();
}

cudaError_t polish_weight(const float* E, const float* Q, size_t n, const float* sigma, void* dst, cudaStream_t st) {
  if (n & 3) return cudaErrorInvalidValue;
  polish_weight_kernel<<<grid_for(n / 4), 256, 0, st>>>(E, Q, n, sigma, (__half*)dst);
  return cudaGetLastError();
}

cudaError_t polish_update(double* R, const float* P, int dp, const float* sigma, cudaStream_t st) {
  polish_update_kernel<<<grid_for((size_t)dp * dp), 256, 0, st>>>(R, P, dp, sigma);
  return cudaGetLastError();
}

}  // namespace rsign
