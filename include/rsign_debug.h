/*
 * rsign_debug.h -- kernel-level entry points of librsign, for testing the
 * individual GPU products against a reference.  They are not part of the
 * reflector method itself; the paper has no counterpart of them.
 *
 * All pointers are device pointers; `stream` is a cudaStream_t as void*.
 * The calls are asynchronous on `stream` and return RSIGN_ERR_CUDA when a
 * launch fails, RSIGN_ERR_ARG for bad sizes.
 */
#ifndef RSIGN_DEBUG_H
#define RSIGN_DEBUG_H

#include <stdint.h>
#include "rsign.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Tensor-core product on the tcgen05 path: out = A * B^T (FP32 accumulate),
 * A, B dp x dp row-major FP16 (fmt 0) or BF16 (fmt 1), out dp x dp FP32.
 * dp must be a multiple of 256.  sym = 1 computes only the tiles that meet
 * the upper triangle and mirrors them (valid when A B^T is symmetric).
 * `status` is a device int (initialised to 0 by the caller) that receives
 * RSIGN_ERR_TIMEOUT if a bounded pipeline wait gave up.
 */
rsign_status rsign_dbg_tc_gemm(const void* A, const void* B, int64_t dp, int32_t fmt, int32_t sym,
                               float* out, int* status, void* stream);

/*
 * Host routine of the automatic shift (runs on the CPU, no GPU needed): the
 * j-th smallest eigenvalue (0-based) of the m x m symmetric tridiagonal with
 * diagonal alpha[0..m-1] and off-diagonal beta[0..m-2] (Sturm bisection), and
 * the last component of its unit eigenvector (inverse iteration), which gives
 * the Lanczos residual bound |beta_m * last|.
 */
rsign_status rsign_dbg_tridiag_ritz(const double* alpha, const double* beta, int32_t m, int32_t j,
                                    double* theta, double* last);

/*
 * Host routine of the scaled steps (runs on the CPU, no GPU needed): the step
 * scalings a_0, a_1, ... that rsign_reflector_ex uses with ns_scaling = 1 for
 * alpha_margin = alpha * margin (clipped to 1) and u0 the bound on the largest
 * |eigenvalue| of X_0 (1 for the Gershgorin alpha, 1.04 for the power-step
 * alpha).  For l = alpha_margin / u0, a = sqrt(3 / (1 + l + l^2)) and
 * l <- 1/2 a l (3 - a^2 l^2), until a = 1 to 1e-15; a_0 is divided by u0.
 * *n receives the count; the first min(cap, *n) are written to out.
 */
rsign_status rsign_dbg_scaled_coeffs(double alpha_margin, double u0, int32_t cap, double* out, int32_t* n);

/*
 * Host routine of the refinement (CPU, no GPU needed): the lower bound of the
 * scaled margin gamma that a plain low-precision trajectory stopping after m
 * steps implies, the root of p_m(gamma) = 0.9 (Eq. pm; p_m increases on
 * [0, 1]) by bisection.
 */
rsign_status rsign_dbg_gamma_from_steps(int32_t m, double* gamma);

/*
 * Host routines of the FP64-grade products (CPU, no GPU needed).
 * rsign_dbg_fp64e_beta: the digit width (bits) that the FP64-emulating
 * products use for an inner extent k_extent (the widest with one pair product
 * exact in the FP32 accumulator and the plan within the kernel's limits);
 * 0 when none fits.
 * rsign_dbg_fp64e_plan: the accumulation plan of a product of two operands
 * split into n_planes digit planes of beta bits, truncated after `levels`
 * digit levels (level t = p + q for the pair of planes p, q), over k_extent
 * terms.  meta[0..4] = number of groups G, number of pair products, number of
 * int64 super-group sums (0 = one sum, 2 = two), log2 of the weight of one
 * unit of the (last) sum, log2 of super-group 0's unit over super-group 1's.
 * group_start[0..G] (pairs of group g: group_start[g] .. group_start[g+1]-1),
 * pair_a / pair_b (plane of each operand, up to 72), group_shift[G] (log2 of
 * the group's weight in its int64 sum), group_sg[G] (super-group of each
 * group, 0 with one sum).  Groups appear in the kernel's execution order.
 * RSIGN_ERR_ARG when the plan does not fit the kernel's limits.
 */
int32_t rsign_dbg_fp64e_beta(int64_t k_extent);

/*
 * Host routine of the refinement (CPU, no GPU needed): the digit levels the
 * refinement chooses by rule.  Low 16 bits: levels L of the first sweep's
 * R A product, the smallest L in 5..7 with 2^(-5L) s_a s_r sqrt(d) <= tol mu / 2
 * (7 when none), s_a and s_r the largest row scales of the digit splits of A
 * and R, mu the margin.  High bits: levels of the polish product R^2 (5 when
 * tol >= 1e-6 and 32 min(k, d - k) <= d, else 6).  -1 for bad arguments.
 */
int32_t rsign_dbg_refine_levels(double tol, double s_a, double s_r, int64_t d, double mu, int32_t k);

/*
 * Host routine of the grouped batched launches (CPU, no GPU needed): the tile
 * table of a batch of n matrices with padded orders dp[0..n) (multiples of
 * bn, bn = 128 or 256), 128-row tiles of width bn, upper-triangle tiles only
 * when sym; order 0 = largest matrices first, 1 = matrix order.  Entry i is
 * units[4i .. 4i+3] = (matrix, tile row, tile column, partial slot); the first
 * min(cap, count) entries are written, slot_begin (n + 1 entries, may be NULL)
 * gets each matrix's first slot.  Returns the count, -1 for bad arguments.
 */
int32_t rsign_dbg_batch_units(int32_t n, const int32_t* dp, int32_t bn, int32_t sym, int32_t order, int32_t cap,
                              int32_t* units, int32_t* slot_begin);
rsign_status rsign_dbg_fp64e_plan(int32_t n_planes, int32_t beta, int32_t levels, int64_t k_extent, int32_t* meta,
                                  int32_t* group_start, int32_t* pair_a, int32_t* pair_b, int32_t* group_shift,
                                  int32_t* group_sg);

/*
 * FP64 product on the FP64 pipe: out = A * B, all dp x dp row-major FP64,
 * dp a multiple of 64; sym = 1 as above.
 */
rsign_status rsign_dbg_f64_gemm(const double* A, const double* B, int64_t dp, int32_t sym,
                                double* out, void* stream);

/*
 * FP64-grade product on the FP16 tensor cores: out = A * B for symmetric
 * FP64 A, B (dp x dp, dp a multiple of 256, rows/columns >= d_real zero),
 * through 5-bit integer digit planes whose level sums are exact in FP32.
 * Blocking: allocates and frees its own workspace, synchronises `stream`.
 */
rsign_status rsign_dbg_fp64grade_gemm(const double* A, const double* B, int64_t dp, int64_t d_real,
                                      int32_t sym, double* out, void* stream);

/*
 * Storage of the 5-bit digit planes of the FP64-grade products (the
 * refinement's R A and R^2, and rsign_dbg_fp64grade_gemm): 1 (the default)
 * = FP8 E4M3 bytes multiplied on the kind::f8f6f4 tensor cores, 0 = FP16 on
 * kind::f16.
 * The digits (|d| <= 16) are exact in both formats and every level sum is
 * the same integer, so the two settings give the same bits.  Other values
 * leave the setting unchanged.  Process-wide; returns the previous setting.
 */
int32_t rsign_dbg_set_digit_fp8(int32_t on);

/*
 * Low-precision stage of the *_REFINE policies: the iterates X_0 .. X_{n-1}
 * are carried as hi/lo pairs of FP16/BF16 planes (three pair products per
 * launch), later ones as single planes (one product per launch, the plain
 * format's rounding).  n = -1 (the default): every iterate; n = -2: by rule,
 * FP16_REFINE only, pairs while the known lower end of the iterate's
 * spectrum (from alpha times the margin) is below the threshold of
 * rsign_dbg_set_split_until, and every iterate when no margin is known;
 * n >= 0: the first n.  Values below -2 leave the setting unchanged.
 * Process-wide; returns the previous setting.  For measurements of the
 * trade-off between the stage's cost and the refinement sweeps its rounding
 * leaves to do.
 */
int32_t rsign_dbg_set_split_steps(int32_t n);

/*
 * Tangent solve of the refinement: 1 leaves out the tangent steps at stored
 * iterates whose known lower end of the spectrum (from alpha times the
 * margin) is within 1e-3 of 1, where the step's derivative is the identity
 * on the error's anticommuting part; 0 (the default) runs a tangent step for
 * every stored iterate.  Other values leave the setting unchanged.
 * Process-wide; returns the previous setting.
 */
int32_t rsign_dbg_set_tangent_cut(int32_t on);

/*
 * Host buffers of rsign_reflector[_ex]: 0 (the default) copies H in and R
 * out through staging device buffers on the copy engines; 1 lets the ingest
 * and output kernels read and write page-locked host buffers (cudaHostAlloc
 * or cudaHostRegister memory) in place over the CPU-GPU link (other host
 * memory is still staged).  Other values leave the setting unchanged.
 * Process-wide; returns the previous setting.
 */
int32_t rsign_dbg_set_host_mapped(int32_t on);

/*
 * Staged host copies of rsign_reflector[_ex] (H in, R out, each at least
 * 64 MiB) split over n streams (1 .. 8) that fork from and join back into
 * the call's stream, so that several copy engines share the link; 1 (the
 * default) copies on the call's stream alone.  Other values leave the
 * setting unchanged.  Process-wide; returns the previous setting.
 */
int32_t rsign_dbg_set_copy_streams(int32_t n);

/*
 * Threshold of the stage-1 split rule (rsign_dbg_set_split_steps(-2)): the
 * iterates whose known lower end of the spectrum is below l are carried as
 * hi/lo pairs.  l in (0, 1]; other values leave it unchanged.  Process-wide;
 * returns the previous threshold.
 */
double rsign_dbg_set_split_until(double l);

/*
 * Host routine of the REFINE stage plan (runs on the CPU, no GPU needed):
 * the lower end l_m of the normalised spectrum of X_m, m = 0 .. max_steps
 * (l_0 = min(1, alpha_margin) / u0, then the scaled steps' map when scaled,
 * the map of Eq. NS beyond them or when not scaled) into lower_end
 * (nullable, max_steps + 1 doubles); *n_split = the number of leading
 * iterates carried as hi/lo pairs (first m with l_m >= 1/2); *m_tangent = the
 * number of tangent steps run for a stage of steps_low steps (first m with
 * l_m >= 1 - 1e-3, at least 1, else steps_low).
 */
rsign_status rsign_dbg_stage_plan(double alpha_margin, double u0, int32_t scaled, int32_t max_steps,
                                  int32_t steps_low, double* lower_end, int32_t* n_split, int32_t* m_tangent);

/*
 * Failure path of the bounded pipeline waits (the mbarrier waits of every
 * tcgen05 kernel, which give up after a wall-clock limit instead of hanging):
 * one kernel initialises an mbarrier for one arrival and waits for its first
 * phase with the limit limit_ns (1 ns .. 2 s).  With arrive = 1 it arrives
 * first and the wait succeeds; with arrive = 0 nothing completes the phase,
 * the wait gives up after limit_ns and writes RSIGN_ERR_TIMEOUT into the
 * device int *status (which the caller initialises to 0), and the kernel
 * returns normally: the context stays usable.  Blocks until the kernel ends;
 * returns RSIGN_ERR_ARG for a bad limit or a non-device status pointer.
 */
rsign_status rsign_dbg_bounded_wait(int32_t arrive, int64_t limit_ns, int* status, void* stream);

/*
 * Digit levels (5 bits each, at most 7) of the refinement's FP64-grade
 * products: the polish SYRK R^2, the first sweep's R A and the later sweeps'
 * R A (defaults 0, 0, 7; 0 = chosen by the tolerance: 5 levels for tol >= 1e-6,
 * else 6).  Values outside 0..7 leave a setting unchanged.  Process-wide;
 * returns the previous settings as 100 p + 10 f + l.
 */
int32_t rsign_dbg_set_refine_levels(int32_t polish, int32_t ra_first, int32_t ra_later);

/*
 * Tile width of the digit-plane products of one-matrix calls (refinement and
 * FP64 polish): 128 (the int64 level
 * sums stay in TMEM), 256 (sums in global memory) or 0 (the
 * default: 128 up to order 3072, else 256).  Other values leave it unchanged.
 * Process-wide; returns the previous setting.
 */
int32_t rsign_dbg_set_ozaki_tile(int32_t bn);

/*
 * The digit-plane products' final conversion of an exact int64 level sum v to
 * FP64, v 2^e rounded to the nearest (ties to even), computed two ways on the
 * device for n values: a[i] by one correctly rounded int64 -> FP64 conversion
 * whose exponent is then moved by e[i] (the way the products' epilogue does
 * it), b[i] by 128-bit integer arithmetic (shift, round to 53 bits, compose
 * the exponent).  Results outside the normal range go through ldexp on both
 * sides.  v, e, a, b: device arrays of n entries.  Blocking.  RSIGN_ERR_ARG
 * for null pointers or n outside 1 .. 2^30.
 */
rsign_status rsign_dbg_oz_convert(const int64_t* v, const int32_t* e, int64_t n, double* a, double* b,
                                  void* stream);

/*
 * The tiles of the check's symmetric double-float product (host computation,
 * no GPU): block t of its launch handles the 128 x 128 tile (I[t], J[t]) of
 * the upper triangle, I <= J; its row sums fill slot J of block I's rows and,
 * off the diagonal, its column sums slot I of block J's rows.  With I == NULL
 * returns the tile count; otherwise fills I/J and returns it; -1 for a bad dp.
 */
int32_t rsign_dbg_sym_gemv_tiles(int64_t dp, int32_t* I, int32_t* J);

/*
 * The order in which the persistent tcgen05 GEMM visits the 128 x 256 tiles of
 * one dp x dp product (host computation, no GPU): entry t is the (bm, bn) of
 * schedule unit t; sym selects the upper triangle.  With bm == NULL returns
 * the entry count; otherwise fills bm/bn and returns the count; -1 for a bad
 * dp.
 */
int32_t rsign_dbg_tile_order(int64_t dp, int32_t sym, int32_t* bm, int32_t* bn);

/*
 * FP64-emulating product on the FP16 tensor cores (the products of the FP64
 * polish steps): as rsign_dbg_fp64grade_gemm with digit planes of beta bits
 * (the widest for which a pair product over d_real terms is exact in FP32:
 * 7 for d_real <= 4096, 6 up to 16384) and ceil(54 / beta) planes, so each
 * operand carries at least 54 bits relative to its off-diagonal row maxima
 * (diagonal exact); level sums in two int64 fixed-point accumulators.
 */
rsign_status rsign_dbg_fp64e_gemm(const double* A, const double* B, int64_t dp, int64_t d_real, int32_t sym,
                                  double* out, void* stream);

/*
 * y = M x for device FP64 M (dp x dp, dp a multiple of 256) and x (dp) in the
 * double-float arithmetic of the refinement's a-posteriori check: M and x
 * split into hi + lo FP32 pairs, exact product splitting and TwoSum
 * accumulation on the FP32 pipe, lanes combined in FP64.  y: device FP64.
 */
rsign_status rsign_dbg_gemv_df(const double* M, const double* x, int64_t dp, double* y, void* stream);

/*
 * The same product for a symmetric M, read from its upper triangle only (the
 * form the a-posteriori check uses): every 128 x 128 tile (I, J), I <= J,
 * adds M_IJ x_J to y_I and, off the diagonal, M_IJ^T x_I to y_J; the partial
 * sums of each output row are added in a fixed order.  The tiles below the
 * diagonal tiles are not read (the diagonal tiles are read whole).  Same
 * arguments and errors as rsign_dbg_gemv_df.
 */
rsign_status rsign_dbg_gemv_df_sym(const double* M, const double* x, int64_t dp, double* y, void* stream);

/*
 * The power-step estimate of ||M||_2 that the alpha rule and the refinement's
 * norms use: M (device FP64, symmetric, dp x dp, dp a multiple of 256) is
 * rounded to FP32, `iters` power steps from the fixed start vector
 * v_i = 1 + (i mod 7)/8 give *out (host double): ||M v|| / ||v|| after one
 * step, else ||M v|| of the last step with v normalised.  Up to order 512 the
 * steps run in one launch; per_step != 0 forces one GEMV and one
 * normalisation launch per step (the same arithmetic, so the same bits).
 * Blocking.  RSIGN_ERR_ARG for bad sizes or iters outside 1 .. 1000.
 */
rsign_status rsign_dbg_spectral_norm(const double* M, int64_t dp, int32_t iters, int32_t per_step, double* out,
                                     void* stream);

/*
 * The matrix-free check of the refinement on device FP64 A, R (dp x dp, dp a
 * multiple of 256, logical order d): `iters` power steps on C = R A - A R and
 * on N = R^2 - I from the check's fixed start vector.  out (host, 5 doubles):
 * ||C v||/2 at the last step (the estimate of ||G||_2), ||N z|| at the last
 * step, and the 2 x 2 projection of A on the last commutator plane
 * (v_prev.A v_prev, v_last.A v_prev, v_last.A v_last).
 */
rsign_status rsign_dbg_commutator_check(const double* A, const double* R, int64_t dp, int64_t d, int32_t iters,
                                        double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSIGN_DEBUG_H */
