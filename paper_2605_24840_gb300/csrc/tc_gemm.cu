// tc_gemm.cu -- persistent tcgen05 GEMM for the Newton-Schulz products.
//
// One CTA per SM (persistent, static round-robin over tiles), 6 warps:
//   warp 0      TMA producer: 128x64 A and BNx64 B tiles (128B swizzle) into
//               a multi-stage shared-memory ring, completion on mbarriers;
//   warp 1      TMEM allocator and MMA issuer: tcgen05.mma kind::f16,
//               M=128 N=BN K=16, FP32 accumulators in TMEM, two
//               accumulators (2 BN columns) so the epilogue of one tile
//               overlaps the main loop of the next;
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (one TMEM lane
//               quadrant per warp), fused elementwise work, global stores.
// The symmetric schedule (`sym`) visits only tiles that meet the upper
// triangle and mirrors each strictly-upper element, which halves the work
// of X^2 (SYRK) and of the symmetric product X (I - X^2) of a Newton-Schulz
// step (Eq. NS).
//
// Tile widths: BN = 256 (one matrix) and BN = 128 (grouped batches of small
// matrices, where a 256-wide tile would be mostly padding).  Every CTA loads
// its own A and B tiles: no shared-memory exchange between CTAs.  Grouped mode (args.units != nullptr) takes
// its tiles from a device table of (matrix, bm, bn, slot) entries built on
// the host: every matrix of a batch lives in its own Dmax x Dmax slot of one
// slab, each tile runs its K loop over its own matrix's padded size only, and
// tiles of matrices flagged in args.mat_skip (converged) are passed over by
// all three roles alike.
#include "common.cuh"
#include "kernels.h"

#include <cuda_fp8.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

namespace rsign {
namespace {

// One pipeline stage holds 128 bytes of K per operand row (one 128-byte
// swizzle row): BK = 64 FP16/BF16 elements, or 128 FP8 elements (kBK8).
constexpr int BM = 128, BK = 64, kBK8 = 128;
// Epilogue warps: four (one per TMEM lane quadrant), or eight for the FP8
// digit-plane products on 256-column tiles, two per quadrant, each taking
// half of the tile's 32-column chunks.  Their conversion epilogue (int64 level sums to FP64
// with the exact diagonal terms, once per element) is a long dependent
// chain per element; a second warp per quadrant doubles the instructions in
// flight.
template <int EPI, typename T, int BN>
constexpr int tc_epi_warps() { return (EPI == TC_EPI_OZAKI && sizeof(T) == 1 && BN == 256) ? 8 : 4; }
template <int EPI, typename T, int BN>
constexpr int tc_threads() { return 64 + 32 * tc_epi_warps<EPI, T, BN>(); }

template <int BN>
struct Cfg {
  static constexpr int STAGES = BN == 256 ? 4 : 6;
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr uint32_t TMEM_COLS = 2 * BN;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};

// Tile schedule of one matrix over 128 x BN output tiles (bm, bn).  In the
// triangular schedule tile row r needs the columns bn >= floor(r BM / BN).
//
// Order: blocks of 2048 rows (16 tile rows) x kBW = 8 columns (2048
// columns), block-rows top to bottom, column blocks left to right, row-major
// inside a block.  The ~150 tiles in flight then cover about one block, whose
// row and column panels (2 x 2048 rows of K) stay in L2 across all the pair
// products of the tiles, instead of one row of tiles streaming every column
// panel.
constexpr int kBW = 8;
constexpr int kBH = 16;  // tile rows per block (2048 matrix rows)

template <int BN>
struct TileSched {
  int nbm, nbn, sym, n;
  __device__ __host__ TileSched(int dp, int s) : nbm(dp / BM), nbn(dp / BN), sym(s) {
    if (!s) {
      n = nbm * nbn;
    } else {
      n = 0;
      for (int r = 0; r < nbm; ++r) n += nbn - first(r);
    }
  }
  __device__ __host__ int first(int r) const { return sym ? (r * BM) / BN : 0; }
  // unit t -> (bm, bn)
  __device__ __host__ void decode(int t, int& bm, int& bn) const {
    int r = 0, c = 0;
    for (int r0 = 0; r0 < nbm; r0 += kBH) {
      const int r1 = r0 + kBH < nbm ? r0 + kBH : nbm;
      int cnt = 0;
      for (int q = r0; q < r1; ++q) cnt += nbn - first(q);
      if (t >= cnt) {
        t -= cnt;
        continue;
      }
      // inside block-row [r0, r1): column blocks from the first needed column
      for (int c0 = first(r0);; c0 += kBW) {
        const int c1 = c0 + kBW < nbn ? c0 + kBW : nbn;
        int bc = 0;
        for (int q = r0; q < r1; ++q) {
          const int lo = c0 > first(q) ? c0 : first(q);
          bc += c1 > lo ? c1 - lo : 0;
        }
        if (t >= bc) {
          t -= bc;
          continue;
        }
        for (int q = r0; q < r1; ++q) {
          const int lo = c0 > first(q) ? c0 : first(q);
          const int w = c1 > lo ? c1 - lo : 0;
          if (t < w) {
            r = q;
            c = lo + t;
            break;
          }
          t -= w;
        }
        break;
      }
      break;
    }
    bm = r;
    bn = c;
  }
};

// One schedule unit as every role sees it.
struct Unit {
  int mat, bm, bn, slot, n_kb;
  bool skip;
};

template <int BN, int BKE>
__device__ __forceinline__ Unit unit_at(const TcGemmArgs& a, const TileSched<BN>& s, int t) {
  Unit u;
  if (a.units != nullptr) {
    const int4 q = a.units[t];
    u.mat = q.x;
    u.bm = q.y;
    u.bn = q.z;
    u.slot = q.w;
    u.n_kb = a.mat_dp[q.x] / BKE;
    u.skip = a.mat_skip != nullptr && a.mat_skip[q.x] != 0;
  } else {
    s.decode(t, u.bm, u.bn);
    u.mat = 0;
    u.slot = t;
    u.n_kb = a.dp / BKE;
    u.skip = false;
  }
  return u;
}

template <typename T>
__device__ __forceinline__ void store32_lp(T* dst, const float* v) {
  // 32 consecutive elements, 64 bytes, 16-byte aligned
  uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      T lo = from_f32<T>(v[q * 8 + 2 * h]);
      T hi = from_f32<T>(v[q * 8 + 2 * h + 1]);
      w[h] = (uint32_t)(*reinterpret_cast<uint16_t*>(&lo)) |
             ((uint32_t)(*reinterpret_cast<uint16_t*>(&hi)) << 16);
    }
    d4[q] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__device__ __forceinline__ void load_f32x32(const float* src, float* v) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 u = s4[q];
    v[4 * q] = u.x;
    v[4 * q + 1] = u.y;
    v[4 * q + 2] = u.z;
    v[4 * q + 3] = u.w;
  }
}

template <typename T>
__device__ __forceinline__ void load32_lp(const T* src, float* v) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 u = s4[q];
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      uint16_t lo = (uint16_t)(w[h] & 0xFFFFu), hi = (uint16_t)(w[h] >> 16);
      v[q * 8 + 2 * h] = to_f32<T>(*reinterpret_cast<T*>(&lo));
      v[q * 8 + 2 * h + 1] = to_f32<T>(*reinterpret_cast<T*>(&hi));
    }
  }
}

// ---- integer-pipe conversions of the digit-plane sums (the FP64 pipe of
// this GPU is ~2 FMA/clk/SM, its integer pipes are far wider)
__device__ __forceinline__ int pow2_exp(double p) {  // p an exact power of two
  return (int)((__double_as_longlong(p) >> 52) & 0x7FF) - 1023;
}

// v 2^e rounded to the nearest binary64 (ties to even), from integer ops only
__device__ __forceinline__ double i128_scaled(__int128 v, int e) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 m = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
  int top = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading bit index
  unsigned long long sig;
  if (top <= 52) {
    sig = lo << (52 - top);
  } else {
    const int sh = top - 52;
    unsigned __int128 q = m >> sh;
    const unsigned __int128 rem = m & ((((unsigned __int128)1) << sh) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q >> 53) {
      q >>= 1;
      ++top;
    }
    sig = (unsigned long long)q;
  }
  const int eb = top + e + 1023;
  if (eb <= 0 || eb >= 2047) {  // outside the normal range: let the FP64 pipe handle it
    const double f = (double)sig;
    return ldexp(neg ? -f : f, top - 52 + e);
  }
  const unsigned long long bits =
      ((unsigned long long)eb << 52) | (sig & 0xFFFFFFFFFFFFFull) | (neg ? (1ull << 63) : 0ull);
  return __longlong_as_double((long long)bits);
}

// v 2^e rounded to the nearest binary64 (ties to even) for a 64-bit v: one
// hardware conversion (correctly rounded), then the exponent moved by e with
// integer operations; the same value as i128_scaled((__int128)v, e), at a
// small fraction of its instructions (the conversion epilogue of a tile runs
// once per element on four warps, so its instruction count is what shows).
__device__ __forceinline__ double i64_scaled(long long v, int e) {
  if (v == 0) return 0.0;
  const double f = __ll2double_rn(v);
  const long long b = __double_as_longlong(f);
  const int eb = (int)((b >> 52) & 0x7FF) + e;
  if (eb <= 0 || eb >= 2047) return ldexp(f, e);  // outside the normal range
  return __longlong_as_double(b + ((long long)e << 52));
}

// Final value of one element: the super-group sums V1 (last) and V0 combined
// exactly in 128 bits (one sum: 64 bits), converted, scaled by
// sigma_i sigma_j 2^unit_exp (and xin_mult when an FP64 input is added)
// through the exponent.
// F8: FP8 digit planes (5-bit digits, at most seven levels), whose launches
// have one sum and no FP64 input (checked on the host).
template <bool F8>
__device__ __forceinline__ double oz_value(const TcGemmArgs& a, long long V1, long long V0, int e_ij) {
  const int e = e_ij + a.oz_unit_exp + (!F8 && a.xin64 != nullptr ? a.xin_mult_exp : 0);
  if (F8 || a.n_sg != 2) return i64_scaled(V1, e);
  const __int128 t = (__int128)V1 + (((__int128)V0) << a.oz_sh01);
  return i128_scaled(t, e);
}

// Epilogue for one 32-column chunk held by one thread (row i, columns j0..j0+31).
// moff: element offset of the tile's matrix in out / xin (grouped mode),
// voff: its offset in the per-row vectors of TC_EPI_OZAKI;
// d_real: that matrix's logical size.  With the symmetric schedule the warp's
// 32 rows and the chunk's 32 columns are either disjoint with every column
// above every row (`above`: row-vector stores plus the mirrored column
// stores, which are coalesced across the warp) or the same index range (the
// diagonal block: row-vector stores of the whole block, then, ordered after
// them by __syncwarp, the mirrors of the strictly-upper part overwrite its
// lower part).  Chunks wholly below the warp's rows are never passed here.
template <int EPI, typename T>
__device__ __forceinline__ void epilogue_chunk(const TcGemmArgs& a, int i, int j0, int g,
                                               float* v, bool above, double& acc1, size_t moff,
                                               size_t voff, int d_real) {
  const int ld = a.dp;
  const size_t row = (size_t)i * ld;
  if constexpr (EPI == TC_EPI_STORE_F32) {
    float* out = reinterpret_cast<float*>(a.out) + moff;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) v[jj] *= a.scale;
    float4* d4 = reinterpret_cast<float4*>(out + row + j0);
#pragma unroll
    for (int q = 0; q < 8; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    if (a.sym) {
      if (!above) __syncwarp();
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        if (above || j0 + jj > i) out[(size_t)(j0 + jj) * ld + i] = v[jj];
    }
  } else if constexpr (EPI == TC_EPI_STORE_LP) {
    T* out = reinterpret_cast<T*>(a.out) + moff;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) v[jj] *= a.scale;
    store32_lp<T>(out + row + j0, v);
    if (a.sym) {
      if (!above) __syncwarp();
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        if (above || j0 + jj > i) out[(size_t)(j0 + jj) * ld + i] = from_f32<T>(v[jj]);
    }
  } else if constexpr (EPI == TC_EPI_NS_SYRK || EPI == TC_EPI_NS_UPDATE) {
    // SYRK:   E  = I - X^2 restricted to the logical d x d block, with the
    //         residual ||X^2 - I||_F^2 accumulated in acc1;
    // UPDATE: X+ = X + 1/2 X (I - X^2), trace of the stored iterate in acc1.
    // With a.split the value is stored as hi = T(v), lo = T(v - hi) in two
    // planes (and X is read back as hi + lo).
    T* out = reinterpret_cast<T*>(a.out) + moff;
    const size_t plane = (size_t)ld * ld;
    if constexpr (EPI == TC_EPI_NS_SYRK) {
      const bool row_real = i < d_real;
      // the chunk's squares are summed in FP32 (32 terms, relative error
      // below 2e-6, ample for the stop rule) and added to the FP64 tile sum
      // once: FP64 arithmetic per element would cost far more than the MMAs
      // of a small-K tile on this GPU
      float accf = 0.0f;
      const float c2 = a.ns_c2 != 0.0f ? a.ns_c2 : 1.0f;  // E = I - a^2 X^2 (scaled step)
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int j = j0 + jj;
        const bool real = row_real && (j < d_real);
        // the diagonal from the exact row norms when given (the tensor-core
        // sum of its K positive terms is biased low)
        const float xx = (i == j && a.ns_diag != nullptr) ? a.ns_diag[voff + i] : v[jj];
        const float e = real ? ((i == j ? 1.0f : 0.0f) - (c2 == 1.0f ? xx : c2 * xx)) : 0.0f;
        v[jj] = e;
        if (real && j >= i) accf = fmaf((j > i ? 2.0f : 1.0f) * e, e, accf);
      }
      acc1 += (double)accf;
    } else {
      const T* xin = reinterpret_cast<const T*>(a.xin) + moff;
      float x[32];
      load32_lp<T>(xin + row + j0, x);
      if (a.split) {
        float xl[32];
        load32_lp<T>(xin + plane + row + j0, xl);
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) x[jj] += xl[jj];
      }
      const float c1 = a.ns_c1 != 0.0f ? a.ns_c1 : 1.0f;  // X+ = a (X + 1/2 X E) (scaled step)
      if (a.scale != 1.0f && a.scale != 0.0f) {  // X_in + 1/2 scale acc
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) v[jj] *= a.scale;
      }
      if (c1 == 1.0f) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) v[jj] = x[jj] + 0.5f * v[jj];
      } else {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) v[jj] = c1 * (x[jj] + 0.5f * v[jj]);
      }
      if (i >= j0 && i < j0 + 32 && i < d_real) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
          if (j0 + jj == i) {
            const T h = from_f32<T>(v[jj]);
            acc1 += (double)to_f32<T>(h);
            if ((a.split && !a.single_out) || a.pair_out)
              acc1 += (double)to_f32<T>(from_f32<T>(v[jj] - to_f32<T>(h)));
          }
      }
    }
    // the result is written as a hi/lo pair when the operands were (unless
    // single_out asks for the hi plane alone) or when pair_out asks for it
    const bool lo_out = (a.split && !a.single_out) || a.pair_out;
    float lo[32];
    if (lo_out) {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) lo[jj] = v[jj] - to_f32<T>(from_f32<T>(v[jj]));
    }
    store32_lp<T>(out + row + j0, v);
    if (lo_out) store32_lp<T>(out + plane + row + j0, lo);
    if (!above) __syncwarp();
    {
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        if (!above && j0 + jj <= i) continue;
        out[(size_t)(j0 + jj) * ld + i] = from_f32<T>(v[jj]);
        if (lo_out) out[plane + (size_t)(j0 + jj) * ld + i] = from_f32<T>(lo[jj]);
      }
    }
  } else if constexpr (EPI == TC_EPI_TANGENT) {
    // tangent step fused with the product sigma X E X (symmetric schedule):
    // every element read here is upper (j >= i) and written only by this
    // thread (its mirror goes to a lower position nobody reads), except in
    // the diagonal 32 x 32 block, where the warp's reads are ordered before
    // its stores by __syncwarp
    float* E = a.tg_E;
    const float* P = a.tg_P;
    const float inv = 0.5f / a.tg_sigma[0];
    const float am = a.tg_a, a3 = am * am * am;
    float e_old[32], p1[32];
    load_f32x32(E + row + j0, e_old);
    load_f32x32(P + row + j0, p1);
    float vn[32];
    float mx = 0.0f;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const float pt = P[(size_t)(j0 + jj) * ld + i];  // (P^T)_ij, coalesced across the warp
      vn[jj] = (am == 1.0f) ? 0.5f * e_old[jj] + inv * (p1[jj] + pt - v[jj])
                            : am * (0.5f * e_old[jj] + inv * (p1[jj] + pt)) - (a3 * inv) * v[jj];
      if (above || j0 + jj >= i) mx = fmaxf(mx, fabsf(vn[jj]));
    }
    acc1 = fmax(acc1, (double)mx);
    if (!above) __syncwarp();
    float4* d4 = reinterpret_cast<float4*>(E + row + j0);
#pragma unroll
    for (int q = 0; q < 8; ++q) d4[q] = make_float4(vn[4 * q], vn[4 * q + 1], vn[4 * q + 2], vn[4 * q + 3]);
    // the next step's operand, E sigma in the operand type (nothing in this
    // launch reads it), stored in the same order as E: rows, then mirrors
    T* el = reinterpret_cast<T*>(a.tg_Elp);
    const float sg = el != nullptr ? a.tg_sigma[0] : 0.0f;
    if (el != nullptr) {
      float vs[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) vs[jj] = vn[jj] * sg;
      store32_lp<T>(el + row + j0, vs);
    }
    if (!above) __syncwarp();
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
      if (above || j0 + jj > i) {
        E[(size_t)(j0 + jj) * ld + i] = vn[jj];
        if (el != nullptr) el[(size_t)(j0 + jj) * ld + i] = from_f32<T>(vn[jj] * sg);
      }
  } else {  // TC_EPI_OZAKI
    // The group sums are exact integers (< 2^24).  They are combined as
    // int64 fixed-point values V = sum_g acc_g 2^(group_shift[g]) (one per
    // super-group of levels) kept in memory between groups; the last group
    // converts to FP64 once, applies the row/column scales, adds the exact
    // diagonal terms and, optionally, the FP64 input xin64.  Only the direct
    // (upper) element is carried between groups; the mirror is written once.
    double* out = reinterpret_cast<double*>(a.out) + moff;
    long long* outi = reinterpret_cast<long long*>(out);
    constexpr bool F8 = sizeof(T) == 1;
    const bool two = !F8 && a.n_sg == 2;
    const bool use_xin = !F8 && a.xin64 != nullptr;
    const int sg = two ? a.group_sg[g] : 0;
    long long* accp = (two && sg == 0) ? a.acc64 + moff : outi;
    const bool first = two ? (a.group_first[g] != 0) : (g == 0);
    const bool last = (g == a.n_groups - 1);
    const int shift = a.group_shift[g];
    const bool with_diag = last && a.a_full != nullptr;
    const double* rs = a.rs + voff;
    const double* cs = a.cs + voff;
    const int ei = last ? pow2_exp(rs[i]) : 0;
    const double dai = with_diag ? a.a_diag[voff + i] : 0.0;
    const double* a_full = with_diag ? a.a_full + moff : nullptr;
    const double* b_full = with_diag ? a.b_full + moff : nullptr;
    float accf = 0.0f;
    // The int64 partial sums move in halves of 16 elements: all loads of a
    // half are issued before any use (16-byte loads where the whole chunk is
    // direct, i.e. not in the diagonal block of a symmetric product; there
    // only the upper elements are touched), so their latency overlaps.
    const bool full_chunk = !a.sym || above;
#pragma unroll
    for (int hh = 0; hh < 32; hh += 16) {
      long long pv[16], pk[16];
      if (!first) {
        if (full_chunk) {
          const longlong2* p2 = reinterpret_cast<const longlong2*>(accp + row + j0 + hh);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const longlong2 t = p2[q];
            pv[2 * q] = t.x;
            pv[2 * q + 1] = t.y;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) pv[q] = (j0 + hh + q >= i) ? accp[row + j0 + hh + q] : 0ll;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) pv[q] = 0ll;
      }
      if (last && two) {
        const long long* pp = a.acc64 + moff + row + j0 + hh;
        if (full_chunk) {
          const longlong2* p2 = reinterpret_cast<const longlong2*>(pp);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const longlong2 t = p2[q];
            pk[2 * q] = t.x;
            pk[2 * q + 1] = t.y;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) pk[q] = (j0 + hh + q >= i) ? pp[q] : 0ll;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) pk[q] = 0ll;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) pv[q] += (long long)__float2int_rn(v[hh + q]) * (1ll << shift);
      if (!last) {
        if (full_chunk) {
          longlong2* p2 = reinterpret_cast<longlong2*>(accp + row + j0 + hh);
#pragma unroll
          for (int q = 0; q < 8; ++q) p2[q] = make_longlong2(pv[2 * q], pv[2 * q + 1]);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (j0 + hh + q >= i) accp[row + j0 + hh + q] = pv[q];
        }
        continue;
      }
      // Last group, eight elements at a time: every input of the eight is
      // loaded before the first of their stores.  The stores go to `out`,
      // which the compiler cannot tell apart from the FP64 inputs, so it
      // would not move a later element's loads above an earlier store; here
      // the eight loads are in flight together.
#pragma unroll
      for (int o = 0; o < 16; o += 8) {
        const int jb = j0 + hh + o;
        const size_t eb = row + jb;
        int ce[8];
        double af[8], bf[8], db[8], xi[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          ce[q] = pow2_exp(cs[jb + q]);
          af[q] = with_diag ? a_full[eb + q] : 0.0;
          bf[q] = with_diag ? b_full[eb + q] : 0.0;
          db[q] = with_diag ? a.b_diag[voff + jb + q] : 0.0;
          xi[q] = use_xin ? a.xin64[moff + eb + q] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = jb + q;
          const bool mirror = a.sym && j > i;
          if (a.sym && j < i) continue;
          const size_t e = eb + q;
          double x = oz_value<F8>(a, pv[o + q], pk[o + q], ei + ce[q]);
          // exact diagonal terms: d^A_i B_ij + A_ij d^B_j - [i == j] d^A_i d^B_j
          if (with_diag) x += dai * bf[q] + af[q] * db[q] - (i == j ? dai * db[q] : 0.0);
          if (use_xin) x = xi[q] + x;
          if (!F8 && a.oz_ident) {
            const bool real = i < d_real && j < d_real;
            x = real ? ((i == j) ? 1.0 - x : -x) : 0.0;
            const float xf = (float)x;
            if (real) accf = fmaf(mirror ? 2.0f * xf : xf, xf, accf);
          }
          out[e] = x;
          if (mirror) out[(size_t)j * ld + i] = x;
        }
      }
    }
    acc1 += (double)accf;
  }
}

// TC_EPI_OZAKI on 128-column tiles: the int64 level sums stay in TMEM
// (columns 256..511, unused by the two 128-column accumulators), so the
// groups of a tile never touch global memory until the last one.  For the
// 32-column chunk q of the tile the low words sit at columns 256 + 64 q + jj
// and the high words at 256 + 64 q + 32 + jj (vaddr = the warp's lanes at
// column 256 + 64 q).  Super-group 0's sum, once complete, is converted to
// FP64 (times its weight) and parked in acc64 (as FP64) for the last group.
// The TMEM loads and stores are warp-collective; every flag that selects
// them depends on the group only.
template <bool F8>
__device__ __forceinline__ void epilogue_oz_tmem(const TcGemmArgs& a, int i, int j0, int g, const float* v,
                                                 double& acc1, size_t moff, size_t voff, int d_real,
                                                 uint32_t vaddr) {
  const int ld = a.dp;
  const size_t row = (size_t)i * ld;
  const bool two = !F8 && a.n_sg == 2;
  const bool use_xin = !F8 && a.xin64 != nullptr;
  const int sg = two ? a.group_sg[g] : 0;
  const bool first = two ? (a.group_first[g] != 0) : (g == 0);
  const bool last = (g == a.n_groups - 1);
  const bool sg_end = last || (two && a.group_sg[g + 1] != sg);
  const int shift = a.group_shift[g];
  uint32_t lo[32], hi[32];
  if (!first) {
    tmem_ld32u(vaddr, lo);
    tmem_ld32u(vaddr + 32, hi);
  }
  long long V[32];
#pragma unroll
  for (int jj = 0; jj < 32; ++jj) {
    V[jj] = (long long)__float2int_rn(v[jj]) * (1ll << shift);
    if (!first) V[jj] += (long long)(((uint64_t)hi[jj] << 32) | (uint64_t)lo[jj]);
  }
  if (!sg_end) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      lo[jj] = (uint32_t)((uint64_t)V[jj] & 0xFFFFFFFFull);
      hi[jj] = (uint32_t)((uint64_t)V[jj] >> 32);
    }
    tmem_st32u(vaddr, lo);
    tmem_st32u(vaddr + 32, hi);
    return;
  }
  long long* park = a.acc64 + moff;
  if (!last) {  // end of super-group 0: park its sum
#pragma unroll 4
    for (int jj = 0; jj < 32; ++jj) {
      const int j = j0 + jj;
      if (a.sym && j < i) continue;
      park[row + j] = V[jj];
    }
    return;
  }
  double* out = reinterpret_cast<double*>(a.out) + moff;
  const bool with_diag = a.a_full != nullptr;
  const double* rs = a.rs + voff;
  const double* cs = a.cs + voff;
  const int ei = pow2_exp(rs[i]);
  const double dai = with_diag ? a.a_diag[voff + i] : 0.0;
  const double* a_full = with_diag ? a.a_full + moff : nullptr;
  const double* b_full = with_diag ? a.b_full + moff : nullptr;
  float accf = 0.0f;
  // eight elements at a time, every input loaded before the first of their
  // stores (the compiler would not move a load above a store to `out`)
#pragma unroll
  for (int o = 0; o < 32; o += 8) {
    const int jb = j0 + o;
    const size_t eb = row + jb;
    int ce[8];
    long long pk[8];
    double af[8], bf[8], db[8], xi[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ce[q] = pow2_exp(cs[jb + q]);
      pk[q] = two ? park[eb + q] : 0ll;
      af[q] = with_diag ? a_full[eb + q] : 0.0;
      bf[q] = with_diag ? b_full[eb + q] : 0.0;
      db[q] = with_diag ? a.b_diag[voff + jb + q] : 0.0;
      xi[q] = use_xin ? a.xin64[moff + eb + q] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = jb + q;
      const bool mirror = a.sym && j > i;
      if (a.sym && j < i) continue;
      const size_t e = eb + q;
      double x = oz_value<F8>(a, V[o + q], pk[q], ei + ce[q]);
      if (with_diag) x += dai * bf[q] + af[q] * db[q] - (i == j ? dai * db[q] : 0.0);
      if (use_xin) x = xi[q] + x;
      if (!F8 && a.oz_ident) {
        const bool real = i < d_real && j < d_real;
        x = real ? ((i == j) ? 1.0 - x : -x) : 0.0;
        const float xf = (float)x;
        if (real) accf = fmaf(mirror ? 2.0f * xf : xf, xf, accf);
      }
      out[e] = x;
      if (mirror) out[(size_t)j * ld + i] = x;
    }
  }
  acc1 += (double)accf;
}

template <int EPI, typename T, int BN>
__global__ void __launch_bounds__(tc_threads<EPI, T, BN>(), 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ TcGemmArgs args, const uint32_t idesc) {
  using C = Cfg<BN>;
  constexpr int STAGES = C::STAGES, A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES;
  // FP8 (E4M3) digit planes: the same 128-byte rows per stage hold 128
  // elements of K, four kind::f8f6f4 MMAs of K = 32 each
  constexpr bool F8 = sizeof(T) == 1;
  constexpr int BKE = F8 ? kBK8 : BK;
  static_assert(!F8 || EPI == TC_EPI_OZAKI, "FP8 operands only for the digit-plane products");
  constexpr int NEPI = tc_epi_warps<EPI, T, BN>();
  static_assert(NEPI == 4 || !(EPI == TC_EPI_NS_SYRK || EPI == TC_EPI_NS_UPDATE || EPI == TC_EPI_TANGENT),
                "per-tile partials assume one epilogue warp per quadrant");
  // 128-column digit-plane products keep their int64 sums in TMEM columns 256..511
  constexpr bool OZ_TMEM = (EPI == TC_EPI_OZAKI && BN == 128);
  constexpr uint32_t TMEM_ALLOC = OZ_TMEM ? 512u : C::TMEM_COLS;
  if (args.skip != nullptr && *args.skip != 0) return;  // uniform across the grid
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  uint64_t* full = bars;                 // [STAGES]
  uint64_t* empty = bars + STAGES;       // [STAGES]
  uint64_t* tfull = bars + 2 * STAGES;   // [2]
  uint64_t* tempty = bars + 2 * STAGES + 2;  // [2]
  uint64_t* drain = bars + 2 * STAGES + 4;   // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 6);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* status = args.status;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&tfull[s]), 1);
      mbar_init(smem_u32(&tempty[s]), 32 * NEPI);
    }
    mbar_init(smem_u32(drain), 1);
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    prefetch_tensormap(&tmA);
    prefetch_tensormap(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_ALLOC);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const TileSched<BN> sched(args.dp, args.sym);
  const int n_units = args.units != nullptr ? args.n_units : sched.n;
  const int unit0 = blockIdx.x, unit_step = gridDim.x;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = unit0; ok && t < n_units; t += unit_step) {
        const Unit u = unit_at<BN, BKE>(args, sched, t);
        if (u.skip) continue;
        const int sa = u.mat * args.a_planes, sb = u.mat * args.b_planes;
        for (int g = 0; ok && g < args.n_groups; ++g) {
          for (int pi = args.group_start[g]; ok && pi < args.group_start[g + 1]; ++pi) {
            for (int kb = 0; kb < u.n_kb; ++kb) {
              if (!mbar_wait(smem_u32(&empty[stage]), phase ^ 1u, status)) { ok = false; break; }
              const uint32_t fb = smem_u32(&full[stage]);
              mbar_arrive_expect_tx(fb, C::STAGE_BYTES);
              tma_load_3d(smem_u32(sA + stage * A_BYTES), &tmA, fb, kb * BKE, u.bm * BM, sa + args.pair_a[pi]);
              tma_load_3d(smem_u32(sB + stage * B_BYTES), &tmB, fb, kb * BKE, u.bn * BN, sb + args.pair_b[pi]);
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
          }
        }
      }
      // make sure no bulk copy is still writing shared memory when the CTA
      // leaves: wait (bounded) for the last fill of every stage
      for (int s = 0; s < STAGES; ++s) {
        // the most recent fill of slot s used parity (phase ^ 1) if s >= stage, else phase
        const uint32_t par = (s >= stage) ? (phase ^ 1u) : phase;
        mbar_wait_drain(smem_u32(&full[s]), par);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------- MMA issue
      int stage = 0;
      uint32_t phase = 0;
      int acc_it = 0;
      bool ok = true;
      for (int t = unit0; ok && t < n_units; t += unit_step) {
        const Unit u = unit_at<BN, BKE>(args, sched, t);
        if (u.skip) continue;
        for (int g = 0; ok && g < args.n_groups; ++g) {
          const int acc = acc_it & 1;
          const uint32_t aph = (acc_it >> 1) & 1;
          if (!mbar_wait(smem_u32(&tempty[acc]), aph ^ 1u, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
          uint32_t accumulate = 0;
          for (int pi = args.group_start[g]; ok && pi < args.group_start[g + 1]; ++pi) {
            for (int kb = 0; kb < u.n_kb; ++kb) {
              if (!mbar_wait(smem_u32(&full[stage]), phase, status)) { ok = false; break; }
              tc_fence_after();
              const uint64_t ad = smem_desc_k128(smem_u32(sA + stage * A_BYTES));
              const uint64_t bd = smem_desc_k128(smem_u32(sB + stage * B_BYTES));
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                // advance 32 bytes along K inside the swizzle atom (16 FP16 or 32 FP8 elements)
                if constexpr (F8) tc_mma_f8(d_tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accumulate);
                else tc_mma_f16(d_tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, accumulate);
                accumulate = 1;
              }
              tc_commit(smem_u32(&empty[stage]));
              if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
          }
          if (ok) tc_commit(smem_u32(&tfull[acc]));
          ++acc_it;
        }
      }
      // retire every MMA issued by this thread before TMEM is released
      tc_commit(smem_u32(drain));
      mbar_wait_drain(smem_u32(drain), 0);
    }
  } else {
    // -------------------------------------------------------------- epilogue
    const int quad = warp & 3;  // the TMEM lane quadrant this warp may access
    // chunks of this warp: all of them, or one half with two warps per quadrant
    constexpr int CPW = (BN / 32) / (NEPI / 4);
    const int c_lo = ((warp - 2) >> 2) * CPW;
    const int r = quad * 32 + lane;
    int acc_it = 0;
    bool ok = true;
    for (int t = unit0; ok && t < n_units; t += unit_step) {
      const Unit u = unit_at<BN, BKE>(args, sched, t);
      if (u.skip) continue;
      const int i = u.bm * BM + r;
      const size_t moff = (size_t)u.mat * (size_t)args.mat_stride;
      const size_t voff = (size_t)u.mat * (size_t)args.mat_vec_stride;
      const int d_real = args.units != nullptr ? args.mat_d[u.mat] : args.d_real;
      double acc1 = 0.0;
      for (int g = 0; g < args.n_groups; ++g) {
        const int acc = acc_it & 1;
        const uint32_t aph = (acc_it >> 1) & 1;
        // one lane waits, the warp follows: the TMEM loads below are warp-collective
        int got = 1;
        if (lane == 0) got = mbar_wait(smem_u32(&tfull[acc]), aph, status) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        if (!got) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * BN);
        const int wrow0 = u.bm * BM + quad * 32;  // first row of this warp
        for (int c = c_lo; c < c_lo + CPW; ++c) {
          const int j0 = u.bn * BN + c * 32;
          // symmetric schedule: a chunk wholly below this warp's rows is the
          // mirror image of elements that their row owners write
          if (args.sym && j0 + 31 < wrow0) continue;
          float v[32];
          tmem_ld32(taddr + (uint32_t)(c * 32), v);
          // chunk lies strictly above the diagonal for every row of this warp
          const bool above = j0 > wrow0 + 31;
          if constexpr (OZ_TMEM) {
            const uint32_t vaddr = tmem_base + ((uint32_t)(quad * 32) << 16) + 256u + (uint32_t)(c * 64);
            epilogue_oz_tmem<F8>(args, i, j0, g, v, acc1, moff, voff, d_real, vaddr);
          } else {
            epilogue_chunk<EPI, T>(args, i, j0, g, v, above, acc1, moff, voff, d_real);
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&tempty[acc]));
        ++acc_it;
      }
      if (!ok) break;
      if (EPI == TC_EPI_NS_SYRK || EPI == TC_EPI_NS_UPDATE || (EPI == TC_EPI_OZAKI && args.oz_ident)) {
        const double s = warp_sum(acc1);
        if (lane == 0) args.partials[(size_t)u.slot * 4 + quad] = s;
      }
      if constexpr (EPI == TC_EPI_TANGENT) {
        double m = acc1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) args.tg_max[(size_t)u.slot * 4 + quad] = (float)m;
      }
    }
  }

  tc_fence_before();
  // every role has drained its own asynchronous work (bounded waits above)
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_ALLOC);
  }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// lp_fmt: 0 FP16, 1 BF16, 2 FP8 E4M3 (bytes)
bool make_map(CUtensorMap* m, const void* ptr, int dp, int slices, int box_rows, int lp_fmt) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t esz = lp_fmt == 2 ? 1 : 2;
  const cuuint64_t dims[3] = {(cuuint64_t)dp, (cuuint64_t)dp, (cuuint64_t)slices};
  const cuuint64_t strides[2] = {(cuuint64_t)dp * esz, (cuuint64_t)dp * dp * esz};
  const cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = lp_fmt == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : (lp_fmt ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  const CUresult r = enc(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int EPI, typename T, int BN>
cudaError_t launch(const TcGemmArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, int grid,
                   uint32_t idesc, cudaStream_t st) {
  constexpr int SMEM_BYTES = Cfg<BN>::SMEM_BYTES;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(tc_gemm_kernel<EPI, T, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SMEM_BYTES);
  });
  if (attr_err != cudaSuccess) return attr_err;
  tc_gemm_kernel<EPI, T, BN><<<grid, tc_threads<EPI, T, BN>(), SMEM_BYTES, st>>>(ma, mb, a, idesc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const TcGemmArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, int grid,
                     uint32_t idesc, cudaStream_t st) {
  switch (a.epi) {
    case TC_EPI_STORE_F32: return launch<TC_EPI_STORE_F32, T, 256>(a, ma, mb, grid, idesc, st);
    case TC_EPI_STORE_LP: return launch<TC_EPI_STORE_LP, T, 256>(a, ma, mb, grid, idesc, st);
    case TC_EPI_NS_SYRK: return launch<TC_EPI_NS_SYRK, T, 256>(a, ma, mb, grid, idesc, st);
    case TC_EPI_NS_UPDATE: return launch<TC_EPI_NS_UPDATE, T, 256>(a, ma, mb, grid, idesc, st);
    case TC_EPI_OZAKI: return launch<TC_EPI_OZAKI, T, 256>(a, ma, mb, grid, idesc, st);
    case TC_EPI_TANGENT: return launch<TC_EPI_TANGENT, T, 256>(a, ma, mb, grid, idesc, st);
    default: return cudaErrorInvalidValue;
  }
}

// grouped launches: one CTA per SM at most, BN = 128 or 256
template <typename T, int BN>
cudaError_t dispatch_grouped(const TcGemmArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, int grid,
                             uint32_t idesc, cudaStream_t st) {
  switch (a.epi) {
    case TC_EPI_STORE_F32: return launch<TC_EPI_STORE_F32, T, BN>(a, ma, mb, grid, idesc, st);
    case TC_EPI_STORE_LP: return launch<TC_EPI_STORE_LP, T, BN>(a, ma, mb, grid, idesc, st);
    case TC_EPI_NS_SYRK: return launch<TC_EPI_NS_SYRK, T, BN>(a, ma, mb, grid, idesc, st);
    case TC_EPI_NS_UPDATE: return launch<TC_EPI_NS_UPDATE, T, BN>(a, ma, mb, grid, idesc, st);
    case TC_EPI_OZAKI:
      if constexpr (std::is_same<T, __half>::value)
        return launch<TC_EPI_OZAKI, T, BN>(a, ma, mb, grid, idesc, st);
      else
        return cudaErrorInvalidValue;  // digit planes are FP16 or FP8 (dispatched apart)
    default: return cudaErrorInvalidValue;
  }
}

// Both conversions of the digit-plane epilogue side by side (debug entry):
// a[i] = i64_scaled(v[i], e[i]), b[i] = i128_scaled(v[i], e[i]).
__global__ void oz_convert_kernel(const long long* v, const int* e, int n, double* a, double* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  a[i] = i64_scaled(v[i], e[i]);
  b[i] = i128_scaled((__int128)v[i], e[i]);
}

}  // namespace

cudaError_t oz_convert_pair(const long long* v, const int* e, int n, double* a, double* b, cudaStream_t st) {
  if (n < 1) return cudaErrorInvalidValue;
  oz_convert_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, e, n, a, b);
  return cudaGetLastError();
}

int tc_num_tiles(int dp, int sym) { return TileSched<256>(dp, sym).n; }

int tc_tile_order(int dp, int sym, int* bm, int* bn) {
  const TileSched<256> sc(dp, sym);
  for (int t = 0; t < sc.n; ++t) sc.decode(t, bm[t], bn[t]);
  return sc.n;
}

cudaError_t tc_gemm(const TcGemmArgs& args, const void* A, int a_slices, const void* B, int b_slices,
                    int lp_fmt, int num_sms, cudaStream_t st) {
  if (args.units != nullptr || args.dp % 256 != 0 || args.n_groups < 1 || args.n_groups > kTcMaxGroups ||
      args.group_start[args.n_groups] > kTcMaxPairs || lp_fmt < 0 || lp_fmt > 2)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, args.dp, a_slices, BM, lp_fmt) || !make_map(&mb, B, args.dp, b_slices, 256, lp_fmt))
    return cudaErrorInvalidValue;
  const int units = TileSched<256>(args.dp, args.sym).n;
  const int grid = units < num_sms ? units : num_sms;
  // FP8 E4M3 digit planes (format field 0 of kind::f8f6f4); their kernel has
  // two epilogue warps per quadrant, no per-tile partials (no oz_ident), one
  // level sum and no FP64 input
  if (lp_fmt == 2)
    return args.epi == TC_EPI_OZAKI && !args.oz_ident && args.n_sg != 2 && args.xin64 == nullptr
               ? launch<TC_EPI_OZAKI, __nv_fp8_e4m3, 256>(args, ma, mb, grid, idesc_f16(0u, BM, 256), st)
               : cudaErrorInvalidValue;
  const uint32_t idesc = idesc_f16(lp_fmt ? 1u : 0u, BM, 256);
  return lp_fmt ? dispatch<__nv_bfloat16>(args, ma, mb, grid, idesc, st)
                : dispatch<__half>(args, ma, mb, grid, idesc, st);
}

cudaError_t tc_gemm_grouped(const TcGemmArgs& args, int bn, const void* A, int a_slices, const void* B,
                            int b_slices, int lp_fmt, int num_sms, cudaStream_t st) {
  if (args.units == nullptr || args.n_units < 1 || args.mat_dp == nullptr || args.mat_d == nullptr ||
      (bn != 128 && bn != 256) || args.dp % 256 != 0 || args.n_groups < 1 || args.n_groups > kTcMaxGroups ||
      args.group_start[args.n_groups] > kTcMaxPairs || (args.epi == TC_EPI_OZAKI && lp_fmt == 1) ||
      (args.epi != TC_EPI_OZAKI && lp_fmt == 2) || (lp_fmt == 2 && (args.oz_ident || args.n_sg == 2 || args.xin64 != nullptr)) || lp_fmt < 0 || lp_fmt > 2)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, args.dp, a_slices, BM, lp_fmt) || !make_map(&mb, B, args.dp, b_slices, bn, lp_fmt))
    return cudaErrorInvalidValue;
  const int grid = args.n_units < num_sms ? args.n_units : num_sms;
  if (lp_fmt == 2)
    return bn == 128 ? launch<TC_EPI_OZAKI, __nv_fp8_e4m3, 128>(args, ma, mb, grid, idesc_f16(0u, BM, 128), st)
                     : launch<TC_EPI_OZAKI, __nv_fp8_e4m3, 256>(args, ma, mb, grid, idesc_f16(0u, BM, 256), st);
  const uint32_t idesc = idesc_f16(lp_fmt ? 1u : 0u, BM, bn);
  if (bn == 128)
    return lp_fmt ? dispatch_grouped<__nv_bfloat16, 128>(args, ma, mb, grid, idesc, st)
                  : dispatch_grouped<__half, 128>(args, ma, mb, grid, idesc, st);
  return lp_fmt ? dispatch_grouped<__nv_bfloat16, 256>(args, ma, mb, grid, idesc, st)
                : dispatch_grouped<__half, 256>(args, ma, mb, grid, idesc, st);
}

// Host-side tile table of a batch (grouped mode): every tile of matrix m
// with padded size dp[m] on a 128 x bn grid (upper-triangle tiles only when
// sym), ordered by decreasing K extent so that the large tiles start first
// and the small ones fill the tail of the persistent schedule; slot numbers
// are contiguous per matrix (slot_begin[m] .. slot_begin[m + 1]).
void tc_build_units(int n, const int* dp, int bn, int sym, int order, std::vector<int4>* units,
                    std::vector<int>* slot_begin) {
  units->clear();
  slot_begin->assign(n + 1, 0);
  std::vector<int4> all;
  for (int m = 0; m < n; ++m) {
    (*slot_begin)[m] = (int)all.size();
    const int nbm = dp[m] / BM, nbn = dp[m] / bn;
    for (int r = 0; r < nbm; ++r)
      for (int c = sym ? (r * BM) / bn : 0; c < nbn; ++c) all.push_back(make_int4(m, r, c, (int)all.size()));
  }
  (*slot_begin)[n] = (int)all.size();
  if (order == 0) {
    std::stable_sort(all.begin(), all.end(), [&](const int4& x, const int4& y) { return dp[x.x] > dp[y.x]; });
  }
  *units = all;
}

}  // namespace rsign
