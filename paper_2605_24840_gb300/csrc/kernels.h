// kernels.h -- internal host-side interface of the rsign CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsign {

// ---------------------------------------------------------------------------
// Tensor-core GEMM (tcgen05, FP16/BF16 operands, FP32 accumulation in TMEM).
// C (dp x dp) = sum over (a_slice, b_slice) pairs of A[a_slice] * B[b_slice]^T,
// where A and B are [slices][dp][dp] row-major arrays (K contiguous).  For a
// symmetric right factor the row-major storage of B is already B^T.
// Tiles are 128 rows x 256 columns; `sym` restricts the schedule to tiles
// that meet the upper triangle and mirrors every strictly-upper element.
// ---------------------------------------------------------------------------
enum TcEpi : int {
  TC_EPI_STORE_F32 = 0,  // out_f32 = scale * acc
  TC_EPI_STORE_LP = 1,   // out_lp  = scale * acc (rounded to the operand type)
  TC_EPI_NS_SYRK = 2,    // acc = X^2: out_lp = I - acc (masked to d), residual partials
  TC_EPI_NS_UPDATE = 3,  // acc = X E: out_lp = X_in + 1/2 acc, trace partials
  TC_EPI_OZAKI = 4,      // out_f64 (+)= rs_i cs_j group_scale_g acc (exact integer groups)
};

constexpr int kTcMaxPairs = 64;
constexpr int kTcMaxGroups = 16;

struct TcGemmArgs {
  int dp;          // padded order: rows of A/B, K extent, leading dimension of outputs
  int d_real;      // logical order (masking of identity / residual / trace)
  int sym;         // 1: upper-triangle tile schedule with mirrored writes
  int epi;         // TcEpi (selects the kernel instantiation)
  int n_groups;    // accumulation groups per tile (one TMEM accumulator each)
  int group_start[kTcMaxGroups + 1];
  int pair_a[kTcMaxPairs];
  int pair_b[kTcMaxPairs];
  double group_scale[kTcMaxGroups];
  float scale;
  void* out;
  const void* xin;         // TC_EPI_NS_UPDATE: current iterate (operand type)
  double* partials;        // TC_EPI_NS_*: one double per (tile, epilogue warp)
  const double* rs;        // TC_EPI_OZAKI: per-row scale of the left operand
  const double* cs;        // TC_EPI_OZAKI: per-row scale of the right operand
  int* status;             // device status word of the call
  const int* skip;         // optional: kernel returns at once when *skip != 0
};

// Number of tiles of the schedule (needed to size `partials`: 4 per tile).
int tc_num_tiles(int dp, int sym);

// Launch.  A/B point to [a_slices][dp][dp] / [b_slices][dp][dp] arrays of
// the operand type; lp_fmt 0 = FP16, 1 = BF16.  dp must be a multiple of 256.
cudaError_t tc_gemm(const TcGemmArgs& args, const void* A, int a_slices, const void* B,
                    int b_slices, int lp_fmt, int num_sms, cudaStream_t st);

// ---------------------------------------------------------------------------
// FP64 kernels (native FP64 pipe, DMMA m8n8k4).
// ---------------------------------------------------------------------------
enum F64Epi : int {
  F64_EPI_STORE = 0,      // out = scale * acc
  F64_EPI_NS_SYRK = 1,    // acc = X^2: out = I - acc (masked to d), residual partials
  F64_EPI_NS_UPDATE = 2,  // acc = X E: out = X_in + 1/2 acc, trace partials
};

struct F64GemmArgs {
  int dp, d_real, sym, epi;
  double scale;
  const double* A;   // left operand, dp x dp row-major
  const double* B;   // right operand, dp x dp row-major (B itself, not transposed)
  double* out;
  const double* xin;
  double* partials;  // one double per (tile, warp): 4 per tile
  const int* skip;   // optional: kernel returns at once when *skip != 0
};
int f64_num_tiles(int dp, int sym);
cudaError_t f64_gemm(const F64GemmArgs& a, cudaStream_t st);

// ---------------------------------------------------------------------------
// Elementwise / reduction kernels.
// ---------------------------------------------------------------------------
// A = 1/2 (H + H^T) - s I into the zero-padded dp x dp buffer; per-(column
// block, row) partial sums of |A| into rowpart[dp/32][dp]; non-finite entries
// of H set bit 1 of *flags.
cudaError_t ingest(const double* H, int d, int dp, double s, double* A, double* rowpart,
                   int* flags, cudaStream_t st);
// rowsum[i] = sum_b rowpart[b][i]; scal[0] = ||A||_inf = max_i rowsum[i].
cudaError_t inf_norm_finish(const double* rowpart, int dp, double* rowsum, double* scal,
                            cudaStream_t st);
// dst = scale * src (FP64 -> FP64/FP16/BF16), scale = *scale_dev * mult.
cudaError_t scale_convert(const double* src, size_t n, const double* scale_dev, double mult,
                          void* dst, int dst_fmt /*0 f16, 1 bf16, 2 f64, 3 f32*/, cudaStream_t st);
// dst(FP64) = src(fmt) converted.
cudaError_t to_f64(const void* src, int src_fmt, size_t n, double* dst, cudaStream_t st);
// Deterministic sum of n partials -> out[0]; out[1] = sqrt(out[0]) when sqrt_out.
cudaError_t sum_partials(const double* partials, int n, double* out, cudaStream_t st);
// y = A x for dp x dp FP64 A (row-major), x,y length dp.
cudaError_t gemv_f64(const double* A, int dp, const double* x, double* y, cudaStream_t st);
// Copy the leading d x d block of src (ld dp) into dst (ld d), and back.
cudaError_t copy_unpad(const double* src, int dp, double* dst, int d, cudaStream_t st);
// Newton-Schulz step check (one block, deterministic): r = sqrt(sum of
// partials) is stored in hist[m]; if *done == 0 the stop rule is applied:
//   r < tol_abs                                   (converged), or
//   r <= floor_lo, or (m >= 1 && r <= floor_hi && r >= ratio * hist[m-1])
//                                                 (low-precision floor reached)
// and on a stop *done = 1, *steps = m.
cudaError_t ns_check(const double* partials, int n, double* hist, int m, double tol_abs,
                     double floor_lo, double floor_hi, double ratio, int* done, int* steps,
                     cudaStream_t st);
// out[0] = sum_{i<d} X[i*dp + i] (FP64 X).
cudaError_t trace_f64(const double* X, int dp, int d, double* out, cudaStream_t st);
// Power-iteration helpers: x <- y / ||y||_2, norm stored in *nrm.
cudaError_t normalize(double* y, int n, double* x, double* nrm, cudaStream_t st);

}  // namespace rsign
