// kernels.h -- internal host-side interface of the rsign CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace rsign {

// ---------------------------------------------------------------------------
// Runtime helpers shared by the entry points (defined in rsign_api.cu).
// ---------------------------------------------------------------------------
// Library-owned stream-ordered pool of the current device (unlimited release
// threshold: the memory stays mapped between calls), or nullptr.
cudaMemPool_t library_pool();
// Workspace of one call: stream-ordered allocations from library_pool(),
// all released (stream-ordered) by release().
struct DevBuf {
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  int64_t bytes = 0;
  cudaError_t alloc(void** p, size_t n);
  void release();
};
bool is_device_ptr(const void* p);
// RSIGN_OK when the current device is sm_103 (fills the SM count), else an
// rsign_status error value.
int check_device(int* num_sms);

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
  TC_EPI_NS_UPDATE = 3,  // acc = X E: out_lp = X_in + 1/2 scale acc, trace partials
  TC_EPI_OZAKI = 4,      // out_f64 (+)= rs_i cs_j group_scale_g acc (exact integer groups)
  TC_EPI_TANGENT = 5,    // acc = sigma X E X (symmetric): the tangent step of the refinement,
                         // E <- a (1/2 E + inv (P + P^T)) - a^3 inv acc, inv = 1/(2 sigma),
                         // in place on the FP32 E (both triangles), P = sigma E Et (FP32,
                         // full); per (tile, warp) max |E| into tg_max
};

constexpr int kTcMaxPairs = 72;
constexpr int kTcMaxGroups = 32;

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
  int group_shift[kTcMaxGroups];  // TC_EPI_OZAKI: group weight 2^shift in its int64 sum
  double final_scale;             // TC_EPI_OZAKI (n_sg == 0): weight of one unit of that sum
  // TC_EPI_OZAKI with two super-groups of levels (n_sg == 2, for products of
  // more than ~37 bits, whose fixed-point sum would overflow one int64):
  // super-group 0 accumulates in acc64, super-group 1 in out (as int64); the
  // last group combines V0 sg_weight[0] + V1 sg_weight[1] in FP64.
  int n_sg;                        // 0: one sum in out (first group = group 0); 2: as above
  int group_sg[kTcMaxGroups];      // super-group of each group
  int group_first[kTcMaxGroups];   // 1: first group of its super-group (writes, no read)
  double sg_weight[2];
  long long* acc64;                // dp x dp (per matrix) int64 scratch of super-group 0
  const double* xin64;             // optional: out = xin64 + xin_mult * (product)
  double xin_mult;                 // a power of two
  int xin_mult_exp;                // log2(xin_mult)
  int oz_unit_exp;                 // log2 of the weight of one unit of the (last) int64 sum
  int oz_sh01;                     // n_sg == 2: super-group 0's unit over super-group 1's, log2
  int oz_ident;                    // 1: out = I - (product) on the logical d x d block (0
                                   // outside) with ||out||_F^2 partials in `partials`
  float scale;
  void* out;
  const void* xin;         // TC_EPI_NS_UPDATE: current iterate (operand type)
  double* partials;        // TC_EPI_NS_*: one double per (tile, epilogue warp)
  const double* rs;        // TC_EPI_OZAKI: per-row scale of the left operand
  const double* cs;        // TC_EPI_OZAKI: per-row scale of the right operand
  int* status;             // device status word of the call
  const int* skip;         // optional: kernel returns at once when *skip != 0
  int split;               // TC_EPI_NS_*: operands/outputs are hi/lo pairs of planes
                           // (plane stride dp*dp); out = hi + lo carries ~2x the bits
  int single_out;          // with split: write the result's hi plane only (the step
                           // after this one runs on single planes)
  int pair_out;            // TC_EPI_NS_UPDATE without split: write the result as a hi/lo
                           // pair all the same (the next step reads hi only; the pair
                           // keeps the FP32 value if this is the last iterate)
  // TC_EPI_OZAKI with diagonal-free digit planes: the first group adds the
  // exact FP64 diagonal terms d^A_i B_ij + A_ij d^B_j - [i == j] d^A_i d^B_j
  const double* a_full;    // FP64 A (dp x dp), or nullptr
  const double* b_full;    // FP64 B (dp x dp, symmetric)
  const double* a_diag;
  const double* b_diag;
  // Grouped mode (tc_gemm_grouped): a batch of matrices, matrix m in slot m of
  // a slab (A/B slices m * a_planes + pair_a[.], outputs at out + m * mat_stride
  // elements, each slot dp x dp with leading dimension dp = Dmax).
  const int4* units;       // device table of (matrix, bm, bn, slot), n_units entries
  int n_units;
  const int* mat_dp;       // per matrix: padded order (K extent), a multiple of the tile width
  const int* mat_d;        // per matrix: logical order
  const int* mat_skip;     // per matrix: nonzero = converged, its tiles are skipped
  long long mat_stride;    // elements of the output type between consecutive matrices
  int a_planes, b_planes;  // slices per matrix in A / B
  int mat_vec_stride;      // TC_EPI_OZAKI: elements between matrices in rs / cs / a_diag / b_diag
  // TC_EPI_TANGENT operands
  float* tg_E;             // FP32 E (dp x dp), read and rewritten
  const float* tg_P;       // FP32 sigma E Et (dp x dp, full)
  const float* tg_sigma;   // device scalar sigma
  float tg_a;              // step scaling a (1 = plain)
  float* tg_max;           // 4 per tile
  void* tg_Elp;            // nullable: also store the new E times tg_sigma in the operand
                           // type (both triangles), the next step's operand
  // scaled Newton-Schulz step X+ = 1/2 a X (3I - a^2 X^2): TC_EPI_NS_SYRK stores
  // E = I - ns_c2 X^2 (ns_c2 = a^2), TC_EPI_NS_UPDATE stores ns_c1 (X + 1/2 X E)
  // (ns_c1 = a); 0 means 1 (the plain step)
  float ns_c1, ns_c2;
  // TC_EPI_NS_SYRK: exact squared row norms of the operand X (nullable): the
  // diagonal of X^2 is taken from here instead of the tensor-core sum
  const float* ns_diag;
};

// The two int64 -> FP64 conversions of the digit-plane epilogue on n device
// values: a = the correctly rounded conversion moved by 2^e, b = the 128-bit
// integer path (debug comparison).
cudaError_t oz_convert_pair(const long long* v, const int* e, int n, double* a, double* b, cudaStream_t st);

// Number of tiles of the schedule (needed to size `partials`: 4 per tile).
int tc_num_tiles(int dp, int sym);
// Host copy of the single-matrix tile order (128 x 256 tiles): (bm, bn) of
// schedule unit t at index t; returns the number of entries.
int tc_tile_order(int dp, int sym, int* bm, int* bn);

// Launch.  A/B point to [a_slices][dp][dp] / [b_slices][dp][dp] arrays of
// the operand type; lp_fmt 0 = FP16, 1 = BF16, 2 = FP8 E4M3 (digit-plane
// products only: TC_EPI_OZAKI).  dp must be a multiple of 256.
cudaError_t tc_gemm(const TcGemmArgs& args, const void* A, int a_slices, const void* B,
                    int b_slices, int lp_fmt, int num_sms, cudaStream_t st);
// Grouped launch over args.units (tile width bn = 128 or 256);
// a_slices / b_slices count all slices of the slab (matrices x planes).
// The digit-plane epilogue has no grouped form.
cudaError_t tc_gemm_grouped(const TcGemmArgs& args, int bn, const void* A, int a_slices, const void* B,
                            int b_slices, int lp_fmt, int num_sms, cudaStream_t st);
// Tile table of a batch with padded orders dp[0..n) (multiples of bn):
// order 0 = largest matrices first, 1 = matrix order; slot_begin has n + 1
// entries (the tiles of matrix m own partial slots slot_begin[m] ..).
void tc_build_units(int n, const int* dp, int bn, int sym, int order, std::vector<int4>* units,
                    std::vector<int>* slot_begin);

// ---------------------------------------------------------------------------
// FP64 kernels (native FP64 pipe, DMMA m8n8k4).
// ---------------------------------------------------------------------------
enum F64Epi : int {
  F64_EPI_STORE = 0,      // out = scale * acc
  F64_EPI_NS_SYRK = 1,    // acc = X^2: out = I - acc (masked to d), residual partials
  F64_EPI_NS_UPDATE = 2,  // acc = X E: out = X_in + 1/2 scale acc (scale 0 = 1), trace partials
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
  // grouped mode (f64_gemm_grouped): one block per entry of a device table of
  // (matrix, bi, bj, slot) 64 x 64 tiles; matrix m at A/B/out/xin + m * mat_stride
  const int4* units;
  int n_units;
  const int* mat_dp;
  const int* mat_d;
  const int* mat_skip;
  long long mat_stride;
  double ns_c1, ns_c2;  // scaled step factors as in TcGemmArgs (0 = 1)
};
int f64_num_tiles(int dp, int sym);
// Grouped FP64 products over a.units (64 x 64 tiles, dp = slot leading dimension).
cudaError_t f64_gemm_grouped(const F64GemmArgs& a, cudaStream_t st);
constexpr int kF64Tile = 64;
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
// Split FP64 into a hi/lo pair of FP16/BF16 planes (plane stride n):
// hi = T(x s), lo = T(x s - hi), s = *scale_dev (or 1); and back: dst = hi + lo.
cudaError_t scale_convert_split(const double* src, size_t n, const double* scale_dev, void* dst,
                                int fmt, cudaStream_t st);
cudaError_t split_to_f64(const void* src, int fmt, size_t n, double* dst, cudaStream_t st);
// out[i] = sum_j x_ij^2 (FP32 result, FP64 accumulation) of the dp x dp
// FP16/BF16 operand x (hi + lo planes when split), rows >= d get 0; no work
// once *skip (nullable) is set.
cudaError_t row_sumsq(const void* x, int fmt, int split, int dp, int d, float* out, const int* skip,
                      cudaStream_t st);
// Deterministic sum of n partials -> out[0]; out[1] = sqrt(out[0]) when sqrt_out.
cudaError_t sum_partials(const double* partials, int n, double* out, cudaStream_t st);
// Copy the leading d x d block of src (ld dp) into dst (ld d), and back
// (copy_pad writes the whole dp x dp destination, zeros outside d x d).
cudaError_t copy_unpad(const double* src, int dp, double* dst, int d, cudaStream_t st);
cudaError_t copy_pad(const double* src, int d, double* dst, int dp, cudaStream_t st);
// Newton-Schulz step check (one block, deterministic): r = sqrt(sum of
// partials) is stored in hist[m]; if *done == 0 the stop rule is applied:
//   r < tol_abs                                   (converged), or
//   r <= floor_lo, or (m >= 1 && r <= floor_hi && r >= ratio * hist[m-1])
//                                                 (low-precision floor reached)
// where the two floor stops also need |sum(tr) - tr_target| <= tr_tol when
// trace partials tr are given; on a stop *done = 1, *steps = m.
cudaError_t ns_check(const double* partials, int n, double* hist, int m, double tol_abs,
                     double floor_lo, double floor_hi, double ratio, int* done, int* steps,
                     cudaStream_t st, const double* tr = nullptr, int n_tr = 0, double tr_target = 0.0,
                     double tr_tol = 0.0);
// Adjoint helpers (FP64): G <- 1/2 G + 1/2 (P1 + P1^T - P2) (the transposed
// Frechet step of X + 1/2 X (I - X^2), P1 = G E, P2 = X G X); dst = scale/2 (src + src^T).
cudaError_t tangent_combine_f64(double* G, const double* P1, const double* P2, int dp, cudaStream_t st);
cudaError_t symmetrize_scale(const double* src, int dp, double scale, double* dst, cudaStream_t st);
// out[0] = sum_{i<d} X[i*dp + i] (FP64 X).
cudaError_t trace_f64(const double* X, int dp, int d, double* out, cudaStream_t st);
// Power-iteration helpers: x <- y / ||y||_2, norm stored in *nrm.
cudaError_t normalize(double* y, int n, double* x, double* nrm, cudaStream_t st);

// ---------------------------------------------------------------------------
// Automatic shift (lanczos.cu).
// ---------------------------------------------------------------------------
struct LanczosResult {
  double lam_k, lam_k1;  // Ritz estimates of lam_k, lam_{k+1}
  double eps_k, eps_k1;  // their residual bounds (an eigenvalue lies within each), each
                         // plus a rounding allowance 16 sqrt(d) u ||T_m||
  int iters;             // Lanczos steps taken
  int converged;         // 1 when (lam_k1 - lam_k)/2 > 4 max(eps) was reached
};
// Lanczos with full reorthogonalisation on the symmetric dp x dp FP64 A (rows
// and columns >= d zero) from the spectrum end nearer to k; `work` holds
// lanczos_work_doubles(dp, max_iter) doubles.
cudaError_t lanczos_endpoints(const double* A, int dp, int d, int k, int max_iter, double* work,
                              LanczosResult* out, int64_t* launches, cudaStream_t st);
size_t lanczos_work_doubles(int dp, int max_iter);
// Host: j-th smallest eigenvalue (0-based) of the m x m symmetric tridiagonal
// (diagonal alpha, off-diagonal beta) and the last component of its unit eigenvector.
void tridiag_ritz(const double* alpha, const double* beta, int m, int j, double* theta, double* last);

// ---------------------------------------------------------------------------
// FP64-grade products on the FP16 tensor cores (refine.cu).
// A symmetric FP64 matrix M is split row by row into S digit planes:
//   M_ik = sigma_i * sum_p d_p(i,k) 2^(-beta (p+1)) + O(sigma_i 2^(-beta S - 1)),
//   sigma_i = 2^e_i >= 2 max_k |M_ik|, d_p integers in [-2^(beta-1), 2^(beta-1)],
// stored exactly as FP16.  A product of two split matrices is a sum of digit
// plane products grouped by level t = p + q; each group sum is an integer
// bounded by (#pairs) 2^(2 beta - 2) K and is exact in the FP32 accumulator
// while that bound stays <= 2^24.  The epilogue adds
// sigma_i sigma_j 2^(-beta (t+2)) acc_t into an FP64 output.
// ---------------------------------------------------------------------------
constexpr int kSliceBeta = 5;   // bits per digit plane
constexpr int kSlices = 7;      // digit planes per operand (35 bits)

// The diagonal is kept out of the digit planes (rows are scaled by their
// off-diagonal maximum, which is far below the diagonal for the reflector
// and for diagonally heavy Hessians) and re-enters exactly in the epilogue.
struct SplitMat {
  void* planes;        // [n_planes][dp][dp] FP16 (or FP8) digits of M - diag(M)
                       // (grouped: [n_mat][n_planes][dp][dp], dp = slot order)
  double* sigma;       // [dp] row scales (powers of two)
  double* diag;        // [dp] diag(M)
  const double* full;  // the FP64 matrix itself (dp x dp), not owned
  int n_planes = kSlices;   // digit planes (n_planes * beta <= 56)
  int beta = kSliceBeta;    // bits per digit
  int keep_diag = 0;        // 1: the diagonal is in the digits (no exact diagonal terms)
  int fp8 = 0;              // 1: digits stored as FP8 E4M3 bytes (beta <= 5: |digit| <= 16,
                            // exact in E4M3), multiplied on the kind::f8f6f4 tensor cores
};
// Split the FP64 matrix M (dp x dp, symmetric) into digit planes; out.full = M.
cudaError_t split_rows(const double* M, int dp, SplitMat out, cudaStream_t st);
// The same for every matrix of a slab (matrix m in slot m, D x D, rows and
// columns below mat_dp[m]).
cudaError_t split_rows_grouped(const double* M, int D, int n_mat, const int* mat_dp, SplitMat out,
                               cudaStream_t st);

// FP64-emulating products (Ozaki scheme with 53+ bits): digits of beta bits,
// beta the widest for which one pair product over K terms is exact in the
// FP32 accumulator (fp64e_beta), and fp64e_planes(beta) planes (>= 54 bits).
// Products of more than ~37 bits use two int64 fixed-point sums (scratch acc64).
int fp64e_beta(int k_extent);
int fp64e_planes(int beta);
struct Fp64eExtra {
  long long* acc64 = nullptr;       // int64 scratch (dp x dp per matrix) when two sums are needed
  const double* xin64 = nullptr;    // out = xin64 + xin_mult * product
  double xin_mult = 1.0;            // a power of two
  int ident = 0;                    // out = I - product (logical block) with residual partials
  double* partials = nullptr;       // 4 per tile (ident)
  const int* skip = nullptr;
  int k_extent = 0;                 // nonzero K terms (default d_real)
  // grouped launch (slab of n_mat matrices, dp = slot order)
  const int4* units = nullptr;
  int n_units = 0, n_mat = 0, bn = 128;
  const int* mat_dp = nullptr;
  const int* mat_d = nullptr;
  const int* mat_skip = nullptr;
};
cudaError_t fp64e_plan(TcGemmArgs* a, int n_planes, int beta, int levels, int k_extent);
cudaError_t fp64e_gemm(const SplitMat& A, const SplitMat& B, int dp, int d_real, int sym, double* out,
                       const Fp64eExtra& x, int* status, int num_sms, cudaStream_t st, int levels);
// out (FP64, dp x dp) = A * B for split symmetric A, B (K = d_real nonzeros);
// sym = 1 when the product is symmetric (A == B): upper tiles + mirror.
// `levels` (<= kSlices) truncates the digit-plane product after levels
// 0 .. levels-1 (5 bits each, relative to the off-diagonal row maxima).
// With `tiles` the product runs on 128 x 128 tiles from that device table
// (one matrix in the grouped mode): the int64 level sums then stay in TMEM
// instead of a global read-modify-write per level group.
struct OzTiles {
  const int4* units = nullptr;  // (0, row tile, column tile, slot)
  int n_units = 0;
  const int* dims = nullptr;    // device {dp, d_real}
};
cudaError_t ozaki_gemm(const SplitMat& A, const SplitMat& B, int dp, int d_real, int sym,
                       double* out, int* status, int num_sms, cudaStream_t st, int levels = kSlices,
                       const OzTiles* tiles = nullptr);

// Elementwise kernels of the refinement sweep.  `scal` is a small device
// array of scalars: each kernel documents the slots it reads and writes.
// C = (N - N^T) 2^k (FP32; the power of two keeps C inside the float range
// whatever the scale of N), block maxima of |C| -> blockmax and FP64 sums of
// C^2 -> part (one each per 32x32 tile).
cudaError_t antisym_part(const double* N, int dp, int k, float* C, float* blockmax, double* part,
                         cudaStream_t st);
// Per-32x32-tile maxima of |M| for an FP32 dp x dp matrix.
cudaError_t absmax_tiles(const float* M, int dp, float* blockmax, cudaStream_t st);
// out[0] = max of n floats; out[1] = 2^-ceil(log2 out[0]) (1 if out[0] == 0).
cudaError_t max_pow2(const float* x, int n, float* out, cudaStream_t st);
// out[0] = max(0, max_i x_i), out[1] = 1 / out[0] (0 if the max is 0); one block
cudaError_t max_f64(const double* x, int n, double* out, cudaStream_t st);
// dst (FP16/BF16) = src * scale[0]   (scale a device float)
cudaError_t scale_to_lp(const float* src, size_t n, const float* scale, void* dst, int fmt,
                        cudaStream_t st);
// Direction of the Newton correction from the commutator product:
// P = R C_lp^T (= -sigmaC R C); E0 = alpha * 1/4 (RC + (RC)^T) = -alpha/4 (P + P^T)/sigmaC,
// written as FP32 with per-tile maxima (alpha pairs with the C given: alpha 2^-k
// for a C scaled by 2^k).
cudaError_t newton_direction(const float* P, int dp, const float* sigmaC, double alpha, float* E,
                             float* blockmax, cudaStream_t st);
// Tangent Newton-Schulz step (Frechet derivative of X + 1/2 X (I - X^2)):
// E <- 1/2 E + 1/2 (P1 + P1^T)/sigma - 1/2 P2/sigma, P1 = E_lp Et, P2 = X E_lp X,
// with per-tile maxima of the new E.
// tangent step of the (scaled) Newton-Schulz map:
// E <- a (1/2 E + 1/2 (P1 + P1^T)/sigma) - 1/2 a^3 P2/sigma  (a = 1: the plain step)
cudaError_t tangent_combine(float* E, const float* P1, const float* P2, int dp, const float* sigma, float a,
                            float* blockmax, cudaStream_t st);
// R += E (FP64 += FP32, masked to d) and per-block sums of E^2 -> part.
cudaError_t add_correction(double* R, const float* E, int dp, int d, double* part, cudaStream_t st);
// Et = I - Y (FP64 -> FP32, masked to d), per-tile maxima, per-tile sums of
// (I - Y)^2 in FP64 -> part (one per 32x32 tile).
cudaError_t ident_minus(const double* Y, int dp, int d, float* Et, float* blockmax, double* part,
                        cudaStream_t st);
// Largest |eigenvalue| of a symmetric FP32 dp x dp matrix by `iters` power
// steps (a lower bound that converges from below) -> *out (device double).
// v, w: dp-float work vectors (unused for dp <= 512, where all the steps run
// in one launch; per_step forces one GEMV and one normalisation launch per
// step at any order, the same arithmetic).  spectral_norm_launches: the
// kernels it launches.
int spectral_norm_launches(int dp, int iters);
cudaError_t spectral_norm_f32(const float* M, int dp, float* v, float* w, int iters, double* out,
                              cudaStream_t st, bool per_step = false);
// hi + lo = x 2^k to 2^-47 relative (lo nullable), by integer operations
// (GB300's FP64 conversions run at the FP64 rate): the operand form of the
// double-float GEMVs below.  k = k_host plus, when kref is given, the
// exponent of the device scalar *kref (a power-of-two scaling that keeps the
// data inside the float range; values below 2^-126 after scaling become 0).
// n even.
cudaError_t split_f32(const double* src, size_t n, float* hi, float* lo, int k_host, const double* kref,
                      cudaStream_t st);
// y = M x in double-float arithmetic (M, x as hi + lo FP32 pairs; dp a
// multiple of 256), y in FP64; with kref, M is the split of M0 2^e (e the
// exponent of *kref) and y = M0 x (the result is scaled back by 2^-e).
cudaError_t gemv_df(const float* M_hi, const float* M_lo, const float* x_hi, const float* x_lo, double* y, int dp,
                    cudaStream_t st, const double* kref = nullptr);
// The same product for a symmetric M from its upper triangle only (half the
// bytes): every 128 x 128 tile (I, J), I <= J, adds M_IJ x_J to y_I and, off
// the diagonal, M_IJ^T x_I to y_J; per-tile partial sums land in slots of
// `part` and are added in slot order (deterministic).  dp a multiple of 128;
// part: gemv_df_sym_part_bytes(dp) bytes of device scratch.
size_t gemv_df_sym_part_bytes(int dp);
// Host copy of the tile order of gemv_df_sym: block t of the launch handles
// tile (I[t], J[t]); returns the tile count (fills I/J when both are given).
int gemv_df_sym_tiles(int dp, int* I, int* J);
cudaError_t gemv_df_sym(const float* M_hi, const float* M_lo, const float* x_hi, const float* x_lo, double* y,
                        int dp, float2* part, cudaStream_t st);
// *out = 1 / max_i |x_i| (1 when that is 0 or not finite), a device scalar
// for split_f32's kref; bits: one device word of scratch.
cudaError_t inv_maxabs(const double* x, size_t n, unsigned long long* bits, double* out, cudaStream_t st);
// Matrix-free estimate of ||G||_2, G = 1/2 R C, C = R A - A R: power steps on
// the antisymmetric C, v -> R (A v) - A (R v), and in the same passes power
// steps on N = R^2 - I.  The matrix-vector products run on the FP32 pipe in
// double-float arithmetic (matrices and vectors as hi + lo FP32 pairs, exact
// product splitting and TwoSum accumulation per lane, lanes combined in
// FP64): ~2^-46 relative per term, FP64-class, at HBM speed (GB300's FP64
// pipe would bound FP64 GEMVs at ~0.6 T FMA/s).
// A and R are symmetric: above order 1024 the products read their upper
// triangles only (gemv_df_sym), up to it whole rows (gemv_df, one launch per
// product); commutator_check_launches gives the kernels it launches.  A_hi/A_lo: split of A (split_f32); R_hi/R_lo: dp^2-float
// buffers that receive the split of R.  work: 12 dp doubles; fwork: 12 dp
// floats; part: gemv_df_sym_part_bytes(dp) bytes.
// out[0] = ||G||_2 estimate, out[1] = ||N||_2 estimate, out[2..4] = the 2 x 2
// Rayleigh-Ritz projection of A on the last plane of the commutator steps.
int commutator_check_launches(int dp, int iters);
cudaError_t commutator_gain_norm(const float* A_hi, const float* A_lo, const double* R, float* R_hi,
                                 float* R_lo, int dp, int d, int iters, double* work, float* fwork,
                                 float2* part, double* out, cudaStream_t st);
// Scaling by power steps (Sec. 4.3: alpha close to 1/||H - sI||_2 enlarges the
// scaled margin gamma): with rho_est = nrm[0] from power steps (a lower bound
// of rho(A) converging from below), scal[3] = rho_est and scal[1] = alpha =
// 1 / (c rho_est).  alpha rho < sqrt(3) keeps every sign (f(t) = t(3 - t^2)/2
// > 0 on (0, sqrt(3))) as long as rho_est > rho / (c sqrt(3)); the trace
// certificate checks it.
// With kscaled, nrm[0] came from A 2^k, k the exponent of the Gershgorin alpha
// in scal[1] on entry: rho_est = nrm[0] 2^-k.
cudaError_t alpha_from_rho(const double* nrm, double c, double* scal, int kscaled, cudaStream_t st);
// dst (FP16) = src (FP64) rounded by way of the nearest float (integer
// operations; may differ from a direct rounding at exact FP16 ties); n even.
cudaError_t to_f16(const double* src, size_t n, void* dst, cudaStream_t st);
// dst (FP16) = hi + lo of a BF16 pair of planes (plane stride n; hi alone when
// pair == 0), summed in FP32 and rounded once; n even.
cudaError_t bf16_pair_to_f16(const void* src, size_t n, int pair, void* dst, cudaStream_t st);
// The same for `count` matrices of n elements (src[i] -> dst[i]) in
// ceil(count / 64) launches.
cudaError_t bf16_pairs_to_f16(const void* const* src, void* const* dst, int count, size_t n, int pair,
                              cudaStream_t st);
// dst (FP16) = sigma E + 3/4 Q / sigma, Q = (sigma E)^2: sigma W, W = E + 3/4 E^2,
// the weight of the quintic polish step R <- R + 1/2 R W; n a multiple of 4.
cudaError_t polish_weight(const float* E, const float* Q, size_t n, const float* sigma, void* dst, cudaStream_t st);
// R += 1/2 P / sigma (P FP32 symmetric product R_lp Et_lp).
cudaError_t polish_update(double* R, const float* P, int dp, const float* sigma, cudaStream_t st);

}  // namespace rsign
