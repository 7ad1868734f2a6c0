// batched.cu -- many reflectors of uneven size through grouped launches (the
// batched regime of Sec. 4.5: many Hessians of modest order, each with its
// own index k, shift s and scaling alpha).
//
// Layout.  The matrices of a group share slabs of n_g slots; slot m is a
// Dmax x Dmax row-major block (Dmax = the largest order rounded up to 256)
// holding matrix m in its leading d_m x d_m corner and zeros elsewhere.  The
// FP64 slab of A_m = 1/2 (H_m + H_m^T) - s_m I, the FP16/BF16 iterate slabs
// X (two, ping-pong) and E, and the FP64 iterate slabs all use this layout,
// so one TMA descriptor (a 3-D map over [slot][row][col]) serves the whole
// group and one tile table drives every grouped launch.
//
// Step.  Every Newton-Schulz step (Eq. NS, update form X + 1/2 X (I - X^2))
// of the group is three launches:
//   1. grouped SYRK   E_m = I - X_m^2 for every unconverged m (upper-triangle
//                     tiles of each matrix, K loop over that matrix's padded
//                     order only), residual partials per tile;
//   2. stop test      per matrix: ||X_m^2 - I||_F from its tiles' partials and
//                     the one-matrix stop rule; retired matrices are flagged
//                     (their tiles are skipped by every later launch) and a
//                     group flag turns the remaining launches into no-ops
//                     once every matrix has retired;
//   3. grouped update X_m <- X_m + 1/2 X_m E_m (symmetric output tiles).
// Eight steps form a chunk.  The first chunk runs eagerly; the chunk is then
// captured once as a CUDA graph and replayed until the group flag is set.
// The tile width of the tensor-core launches (128 or 256 columns) and the
// tile order are chosen by timing the candidates on the group's first SYRK;
// the choice is cached per batch shape.
#include "common.cuh"
#include "kernels.h"
#include "rsign.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace rsign {
namespace {

constexpr int kBatchMaxD = 1024;  // larger matrices take the one-matrix path
constexpr int kRestWorkers = 16;  // host threads running one-matrix calls concurrently
constexpr int kBatchChunk = 8;    // steps per chunk (even: the ping-pong parity repeats)
constexpr double kEps64 = 2.220446049250313e-16;

// ------------------------------------------------------------------ kernels
// A_m = 1/2 (H_m + H_m^T) - s_m I into slot m (zeros outside d_m x d_m),
// per-(32-column block, row) sums of |A_m| into rowpart[m][D/32][D],
// non-finite entries of H_m set bit 0 of flags[m].  Block (32, 8) per 32 x 32
// tile; grid (D/32, D/32, n).
__global__ void batch_ingest_kernel(const double* const* __restrict__ H, const int* __restrict__ dv,
                                    const double* __restrict__ sv, int D, double* __restrict__ A,
                                    double* __restrict__ rowpart, int* __restrict__ flags) {
  __shared__ double t1[32][33], t2[32][33];
  const int m = blockIdx.z, bi = blockIdx.y, bj = blockIdx.x;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int d = dv[m];
  const double s = sv[m];
  const double* Hm = H[m];
  double* Am = A + (size_t)m * D * D;
  const int nbj = D / 32;
  const bool inside = bi * 32 < d && bj * 32 < d;
  if (!inside) {  // padding block: zeros, no arithmetic (block-uniform)
    for (int r = ty; r < 32; r += 8) Am[(size_t)(bi * 32 + r) * D + bj * 32 + tx] = 0.0;
    if (ty == 0) rowpart[((size_t)m * nbj + bj) * D + bi * 32 + tx] = 0.0;
    return;
  }
  bool bad = false;
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    double h1 = 0.0, h2 = 0.0;
    if (inside && i < d && j < d) h1 = Hm[(size_t)i * d + j];
    const int i2 = bj * 32 + r, j2 = bi * 32 + tx;  // transposed tile
    if (inside && i2 < d && j2 < d) h2 = Hm[(size_t)i2 * d + j2];
    if (!isfinite(h1) || !isfinite(h2)) bad = true;
    t1[r][tx] = h1;
    t2[r][tx] = h2;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + tx;
    double v = 0.0;
    if (i < d && j < d) v = 0.5 * (t1[r][tx] + t2[tx][r]) - (i == j ? s : 0.0);
    Am[(size_t)i * D + j] = v;
    t1[r][tx] = fabs(v);
  }
  if (bad) atomicOr(&flags[m], 1);
  __syncthreads();
  if (ty == 0) {
    double sum = 0.0;
    for (int c = 0; c < 32; ++c) sum += t1[tx][c];
    rowpart[((size_t)m * nbj + bj) * D + bi * 32 + tx] = sum;
  }
}

// alpha_m = 1/||A_m||_inf (Gershgorin bound on rho, Sec. 4.3); 0 when A_m = 0
// or non-finite.  One block of 1024 threads per matrix.
__global__ void batch_alpha_kernel(const double* __restrict__ rowpart, int D, double* __restrict__ alpha) {
  __shared__ double sh[32];
  const int m = blockIdx.x, nbj = D / 32;
  double mx = 0.0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nbj; ++b) s += rowpart[((size_t)m * nbj + b) * D + i];
    mx = fmax(mx, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) alpha[m] = (mx > 0.0 && isfinite(mx)) ? 1.0 / mx : 0.0;
  }
}

// dst (slot m) = alpha_m * A (slot m), rounded to T.
template <typename T>
__global__ void batch_scale_kernel(const double* __restrict__ A, const double* __restrict__ alpha, int D,
                                   size_t n, T* __restrict__ dst) {
  const size_t slot = (size_t)D * D;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double v = A[e] * (alpha[e / slot] * 1.0);
    if constexpr (sizeof(T) == 8) dst[e] = v;
    else dst[e] = from_f64<T>(v);
  }
}

// FP64 copy of each matrix's final low-precision iterate, X_m in slab
// (steps[m] & 1) of the ping-pong pair.
template <typename T>
__global__ void batch_to_f64_kernel(const T* __restrict__ X0, const T* __restrict__ X1,
                                    const int* __restrict__ steps, int D, size_t n, double* __restrict__ dst) {
  const size_t slot = (size_t)D * D;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const T* src = (steps[e / slot] & 1) ? X1 : X0;
    dst[e] = (double)to_f32<T>(src[e]);
  }
}

// Stop test of one group step.  mode 0: low-precision stage (stop on the
// residual floor or its stagnation, as the one-matrix stage); mode 1: FP64
// stage (stop when ||X^2 - I||_F < max(tol, 16 d u_64)); mode 2: fixed-depth
// FP64 polish (stop only at the budget).  u > 0 enables the floor rule with
// floor_lo = 2 u sqrt(d), floor_hi = 16 u sqrt(d).  done[m]: 0 active,
// 1 stopped, 2 budget exhausted; steps[m]: index of the current iterate.
// One warp per matrix over many blocks (the FP64 arithmetic of the test is
// slow on this GPU, so it is spread over the SMs); ctr[0] counts the
// matrices that stay active and ctr[1] the finished blocks: the last block
// sets all_done (1 once no matrix is active) and clears both counters.
constexpr int kCheckWarps = 4;
// trp (nullable): trace partials of the current iterates (from the grouped
// update, same slots); a floor or stagnation stop of matrix m then also needs
// |trace X_m - (d_m - 2 k_m)| <= 1/2 + 2 u sqrt(d_m).
__global__ void batch_check_kernel(const double* __restrict__ partials, const int* __restrict__ slot_begin,
                                   int n, const int* __restrict__ dv, int mode, double tol, double u,
                                   int max_steps, int* __restrict__ done, int* __restrict__ steps,
                                   double* __restrict__ prev, double* __restrict__ resid,
                                   int* __restrict__ all_done, int* __restrict__ ctr,
                                   const double* __restrict__ trp, const int* __restrict__ kv) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * kCheckWarps + (threadIdx.x >> 5);
  if (m < n && done[m] == 0) {  // uniform across the warp
    const int q0 = slot_begin[m] * 4, q1 = slot_begin[m + 1] * 4;
    double s = 0.0, tr = 0.0;
    for (int q = q0 + lane; q < q1; q += 32) {
      s += partials[q];
      if (trp != nullptr) tr += trp[q];
    }
    s = warp_sum(s);
    tr = warp_sum(tr);
    if (lane == 0) {
      const double r = sqrt(fmax(s, 0.0));
      const double d = (double)dv[m];
      const int mm = steps[m];
      const double tol_abs = mode == 0 ? 0.0 : (mode == 1 ? fmax(tol, 16.0 * d * kEps64) : -1.0);
      bool stop = r < tol_abs;
      const bool trace_ok = trp == nullptr || mm == 0 ||
                            fabs(tr - (d - 2.0 * kv[m])) <= 0.5 + 2.0 * u * sqrt(d);
      if (u > 0.0 && trace_ok) {
        const double flo = 2.0 * u * sqrt(d), fhi = 16.0 * u * sqrt(d);
        if (r <= flo) stop = true;
        if (mm >= 1 && r <= fhi && r >= 0.5 * prev[m]) stop = true;
      }
      resid[m] = r;
      prev[m] = r;
      if (stop) {
        done[m] = 1;
      } else if (mm >= max_steps) {
        done[m] = 2;
      } else {
        steps[m] = mm + 1;
        atomicAdd(&active, 1);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (active) atomicAdd(&ctr[0], active);
    __threadfence();
    const int ticket = atomicAdd(&ctr[1], 1);
    if (ticket == (int)gridDim.x - 1) {  // every block has published its count
      __threadfence();
      const int total = atomicAdd(&ctr[0], 0);
      *all_done = total == 0 ? 1 : 0;
      ctr[0] = 0;
      ctr[1] = 0;
    }
  }
}

// trace of each matrix's result (FP64 slab pair, parity steps[m] & 1, or one
// slab when X1 == nullptr).  One block of 1024 threads per matrix.
__global__ void batch_trace_kernel(const double* __restrict__ X0, const double* __restrict__ X1,
                                   const int* __restrict__ steps, const int* __restrict__ dv, int D,
                                   double* __restrict__ trace) {
  __shared__ double sh[32];
  const int m = blockIdx.x, d = dv[m];
  const double* X = ((X1 != nullptr && (steps[m] & 1)) ? X1 : X0) + (size_t)m * D * D;
  double s = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) s += X[(size_t)i * D + i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) trace[m] = s;
  }
}

// R_m (d_m x d_m, leading dimension d_m) <- slot m of the result slab.
// Block (32, 8) per 32 x 32 tile; grid (D/32, D/32, n).
__global__ void batch_scatter_kernel(const double* __restrict__ X0, const double* __restrict__ X1,
                                     const int* __restrict__ steps, const int* __restrict__ dv, int D,
                                     double* const* __restrict__ R) {
  const int m = blockIdx.z, d = dv[m];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi * 32 >= d || bj * 32 >= d) return;
  const double* X = ((X1 != nullptr && (steps[m] & 1)) ? X1 : X0) + (size_t)m * D * D;
  double* Rm = R[m];
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + threadIdx.x;
    if (i < d && j < d) Rm[(size_t)i * d + j] = X[(size_t)i * D + j];
  }
}

int grid_of(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)std::min<size_t>(g, 152 * 16);
}

// 64 x 64 FP64 tiles of a batch (upper triangle), largest matrices first.
void f64_units(int n, const int* dp64, std::vector<int4>* units, std::vector<int>* slot_begin) {
  units->clear();
  slot_begin->assign(n + 1, 0);
  std::vector<int4> all;
  for (int m = 0; m < n; ++m) {
    (*slot_begin)[m] = (int)all.size();
    const int nb = dp64[m] / kF64Tile;
    for (int r = 0; r < nb; ++r)
      for (int c = r; c < nb; ++c) all.push_back(make_int4(m, r, c, (int)all.size()));
  }
  (*slot_begin)[n] = (int)all.size();
  std::stable_sort(all.begin(), all.end(), [&](const int4& x, const int4& y) { return dp64[x.x] > dp64[y.x]; });
  *units = all;
}

// ------------------------------------------------------------- autotuner
// Cache of the tile choice per (format, Dmax, multiset of padded orders).
struct TileChoice {
  int bn, order;
};
std::mutex g_tune_mu;
std::map<std::vector<int>, TileChoice> g_tune_cache;

int round_up(int x, int q) { return (x + q - 1) / q * q; }

struct Group {
  int n = 0, D = 0;
  std::vector<int> idx;  // caller indices
  std::vector<int> d, k;
  std::vector<double> s;
};

}  // namespace

// ---------------------------------------------------------------- host path
rsign_status batched_impl(int32_t n, const double* const* H, const int64_t* d, const int32_t* k,
                          const double* s, double tol, rsign_policy policy, const rsign_options* opt_in,
                          double* const* R, rsign_info* infos, cudaStream_t st) {
  rsign_options opt;
  rsign_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (n < 0 || (n > 0 && (!H || !d || !k || !s || !R))) return RSIGN_ERR_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol)) return RSIGN_ERR_ARG;
  if ((int)policy < RSIGN_FP64 || (int)policy > RSIGN_FP32) return RSIGN_ERR_ARG;
  if (opt.max_steps < 1 || opt.max_steps > 1000 || opt.polish_steps < 0) return RSIGN_ERR_ARG;
  if (opt.batch_tile != 0 && opt.batch_tile != 128 && opt.batch_tile != 256) return RSIGN_ERR_ARG;
  if (opt.engine != RSIGN_ENGINE_NS3) return RSIGN_ERR_ARG;  // the grouped launches run Eq. NS
  if (n == 0) return RSIGN_OK;
  std::vector<rsign_status> stat(n, RSIGN_OK);
  if (infos) std::memset(infos, 0, sizeof(rsign_info) * (size_t)n);

  // ---- partition: grouped matrices and the one-by-one rest
  // refinement and the hi/lo FP32-class trajectory take the one-matrix path
  const bool refine = policy == RSIGN_FP16_REFINE || policy == RSIGN_BF16_REFINE || policy == RSIGN_FP32;
  Group g;
  std::vector<int> rest;
  for (int i = 0; i < n; ++i) {
    if (!H[i] || !R[i] || d[i] < 2 || k[i] < 1 || k[i] > d[i] - 1 || std::isinf(s[i])) {
      stat[i] = RSIGN_ERR_ARG;
      continue;
    }
    if (!refine && std::isfinite(s[i]) && d[i] <= kBatchMaxD) {
      g.idx.push_back(i);
      g.d.push_back((int)d[i]);
      g.k.push_back(k[i]);
      g.s.push_back(s[i]);
    } else {
      rest.push_back(i);
    }
  }
  g.n = (int)g.idx.size();

  if (g.n > 0) {
    int num_sms = 0;
    const int dst = check_device(&num_sms);
    if (dst != RSIGN_OK) return (rsign_status)dst;
    const bool low = policy != RSIGN_FP64;
    const bool polish = policy == RSIGN_FP16_POLISH || policy == RSIGN_BF16_POLISH;
    const int fmt = (policy == RSIGN_BF16 || policy == RSIGN_BF16_POLISH) ? 1 : 0;
    const int ng = g.n;
    int dmax = 0;
    for (int x : g.d) dmax = std::max(dmax, x);
    g.D = round_up(dmax, 256);
    const int D = g.D;
    const size_t slot = (size_t)D * D, nel = (size_t)ng * slot;

    DevBuf mem;
    mem.st = st;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0;
    auto cleanup = [&]() {
      if (gexec) cudaGraphExecDestroy(gexec);
      if (graph) cudaGraphDestroy(graph);
      mem.release();
      cudaStreamSynchronize(st);
      if (cap) cudaStreamDestroy(cap);
      for (auto& e : ev) if (e) cudaEventDestroy(e);
    };
    auto fail_cuda = [&]() {
      cleanup();
      cudaGetLastError();
      return RSIGN_ERR_CUDA;
    };
    if (opt.timing)
      for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda();
    if (opt.timing) cudaEventRecord(ev[0], st);

    // ---- per-matrix control arrays (one int and one double allocation)
    // ints: d, dp_lp(128), dp_lp(256), dp64, done, steps, flags, done64, steps64,
    //       slot_begin (lp: n+1, f64: n+1), status, all_done, all_done64
    enum { I_D = 0, I_DP128, I_DP256, I_DP64, I_DONE, I_STEPS, I_FLAGS, I_DONE64, I_STEPS64, I_K, I_N };
    const size_t n_int = (size_t)I_N * ng + 3 * (size_t)(ng + 1) + 6;
    int* ib = nullptr;
    double* db = nullptr;
    enum { D_S = 0, D_ALPHA, D_PREV, D_RESID, D_TRACE, D_N };
    const double** hptr = nullptr;
    double** rptr = nullptr;
    if (mem.alloc((void**)&ib, n_int * 4) != cudaSuccess ||
        mem.alloc((void**)&db, (size_t)D_N * ng * 8) != cudaSuccess ||
        mem.alloc((void**)&hptr, (size_t)ng * 8) != cudaSuccess ||
        mem.alloc((void**)&rptr, (size_t)ng * 8) != cudaSuccess)
      return fail_cuda();
    auto ia = [&](int which) { return ib + (size_t)which * ng; };
    int* slot_lp = ib + (size_t)I_N * ng;            // ng + 1 (filled after tuning)
    int* slot_lp2 = slot_lp + (ng + 1);              // ng + 1 (second candidate, tuning)
    int* slot_64 = slot_lp2 + (ng + 1);              // ng + 1
    int* status = slot_64 + (ng + 1);
    int* all_done = status + 1;
    int* all_done64 = status + 2;
    int* ctr = status + 3;  // two counters of the stop test (zero between launches)
    const int check_blocks = (ng + kCheckWarps - 1) / kCheckWarps;
    auto da = [&](int which) { return db + (size_t)which * ng; };

    std::vector<int> h_int(n_int, 0);
    std::vector<int> dp128(ng), dp256(ng), dp64(ng);
    for (int m = 0; m < ng; ++m) {
      h_int[(size_t)I_D * ng + m] = g.d[m];
      h_int[(size_t)I_K * ng + m] = g.k[m];
      dp128[m] = round_up(g.d[m], 128);
      dp256[m] = round_up(g.d[m], 256);
      dp64[m] = round_up(g.d[m], kF64Tile);
      h_int[(size_t)I_DP128 * ng + m] = dp128[m];
      h_int[(size_t)I_DP256 * ng + m] = dp256[m];
      h_int[(size_t)I_DP64 * ng + m] = dp64[m];
    }
    std::vector<int4> u64;
    std::vector<int> sb64;
    f64_units(ng, dp64.data(), &u64, &sb64);
    std::copy(sb64.begin(), sb64.end(), h_int.begin() + (slot_64 - ib));
    std::vector<double> h_dbl((size_t)D_N * ng, 0.0);
    for (int m = 0; m < ng; ++m) h_dbl[(size_t)D_S * ng + m] = g.s[m];

    // ---- inputs: device pointers as given, host matrices staged
    std::vector<const double*> hp(ng);
    std::vector<double*> rp(ng);
    std::vector<int> r_host;
    for (int m = 0; m < ng; ++m) {
      const int i = g.idx[m];
      const size_t bytes = (size_t)g.d[m] * g.d[m] * 8;
      if (is_device_ptr(H[i])) {
        hp[m] = H[i];
      } else {
        double* p = nullptr;
        if (mem.alloc((void**)&p, bytes) != cudaSuccess ||
            cudaMemcpyAsync(p, H[i], bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
          return fail_cuda();
        hp[m] = p;
      }
      if (is_device_ptr(R[i])) {
        rp[m] = R[i];
      } else {
        double* p = nullptr;
        if (mem.alloc((void**)&p, bytes) != cudaSuccess) return fail_cuda();
        rp[m] = p;
        r_host.push_back(m);
      }
    }
    int4* units64 = nullptr;
    if (mem.alloc((void**)&units64, u64.size() * sizeof(int4)) != cudaSuccess) return fail_cuda();
    if (cudaMemcpyAsync(ib, h_int.data(), n_int * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(db, h_dbl.data(), h_dbl.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(hptr, hp.data(), (size_t)ng * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(rptr, rp.data(), (size_t)ng * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(units64, u64.data(), u64.size() * sizeof(int4), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return fail_cuda();

    // ---- ingest, alpha, X_0
    double *A64 = nullptr, *rowpart = nullptr, *partials = nullptr;
    size_t n_slots_max = u64.size();
    std::vector<int4> ulp[2];
    std::vector<int> sblp[2];
    int cand_bn[2] = {128, 256};
    if (low) {
      for (int c = 0; c < 2; ++c) {
        tc_build_units(ng, c == 0 ? dp128.data() : dp256.data(), cand_bn[c], 1, 0, &ulp[c], &sblp[c]);
        n_slots_max = std::max(n_slots_max, ulp[c].size());
      }
    }
    double* trpart = nullptr;  // trace partials of the grouped updates
    if (mem.alloc((void**)&A64, nel * 8) != cudaSuccess ||
        mem.alloc((void**)&rowpart, (size_t)ng * (D / 32) * D * 8) != cudaSuccess ||
        mem.alloc((void**)&partials, n_slots_max * 4 * 8) != cudaSuccess ||
        mem.alloc((void**)&trpart, n_slots_max * 4 * 8) != cudaSuccess)
      return fail_cuda();
    {
      dim3 grid(D / 32, D / 32, ng), block(32, 8);
      batch_ingest_kernel<<<grid, block, 0, st>>>(hptr, ia(I_D), da(D_S), D, A64, rowpart, ia(I_FLAGS));
      batch_alpha_kernel<<<ng, 1024, 0, st>>>(rowpart, D, da(D_ALPHA));
      launches += 2;
      if (cudaGetLastError() != cudaSuccess) return fail_cuda();
    }

    int tile_bn = 64;
    // 128-column tile table of the low-precision stage (reused by the polish)
    int4* units_sel = nullptr;
    int n_units_sel = 0;
    int* slot_sel = nullptr;
    const int* mat_dp_sel = nullptr;
    void* xlp[2] = {nullptr, nullptr};
    void* elp = nullptr;
    double* x64[2] = {nullptr, nullptr};
    double* e64 = nullptr;
    if (mem.alloc((void**)&x64[0], nel * 8) != cudaSuccess) return fail_cuda();
    if (!low || polish) {
      if (mem.alloc((void**)&x64[1], nel * 8) != cudaSuccess || mem.alloc((void**)&e64, nel * 8) != cudaSuccess)
        return fail_cuda();
    }

    // Runs the NS loop of one stage: `step(gstep, parity)` enqueues the
    // SYRK / check / update of global step gstep; chunks of kBatchChunk
    // steps, the first eager, the later ones one graph launch each.
    auto run_stage = [&](int max_steps, int* flag, int per_step, auto&& step) -> bool {
      if (cudaMemsetAsync(flag, 0, 4, st) != cudaSuccess) return false;
      const int total = max_steps + 1;  // SYRK/check launches: steps 0 .. max_steps
      int gstep = 0;
      bool use_graph = opt.batch_graphs != 0;
      while (gstep < total) {
        const int n_here = std::min(kBatchChunk, total - gstep);
        if (gstep > 0 && use_graph && n_here == kBatchChunk) {
          if (!gexec) {
            if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return false;
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
            bool ok = true;
            for (int q = 0; q < kBatchChunk && ok; ++q) ok = step(q, cap, false);
            cudaGraph_t gr = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(cap, &gr);
            if (!ok || ce != cudaSuccess || gr == nullptr) {
              if (gr) cudaGraphDestroy(gr);
              cudaGetLastError();
              use_graph = false;  // fall back to eager launches
              continue;
            }
            graph = gr;
            if (cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
              cudaGetLastError();
              gexec = nullptr;
              use_graph = false;
              continue;
            }
          }
          if (cudaGraphLaunch(gexec, st) != cudaSuccess) return false;
          launches += (int64_t)per_step * kBatchChunk;
        } else {
          for (int q = 0; q < n_here; ++q)
            if (!step(gstep + q, st, gstep + q == max_steps)) return false;
        }
        gstep += n_here;
        int h_flag = 0, h_status = 0;
        if (cudaMemcpyAsync(&h_flag, flag, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
          return false;
        if (h_flag != 0 || h_status != 0) break;
      }
      if (gexec) {
        cudaGraphExecDestroy(gexec);
        gexec = nullptr;
      }
      if (graph) {
        cudaGraphDestroy(graph);
        graph = nullptr;
      }
      return true;
    };

    if (opt.timing) cudaEventRecord(ev[1], st);
    if (low) {
      // ------------------------------------------------ low-precision stage
      for (int b = 0; b < 2; ++b)
        if (mem.alloc(&xlp[b], nel * 2) != cudaSuccess) return fail_cuda();
      if (mem.alloc(&elp, nel * 2) != cudaSuccess) return fail_cuda();
      if (fmt == 0)
        batch_scale_kernel<__half><<<grid_of(nel), 256, 0, st>>>(A64, da(D_ALPHA), D, nel, (__half*)xlp[0]);
      else
        batch_scale_kernel<__nv_bfloat16><<<grid_of(nel), 256, 0, st>>>(A64, da(D_ALPHA), D, nel,
                                                                          (__nv_bfloat16*)xlp[0]);
      ++launches;
      int4* units_c[2] = {nullptr, nullptr};
      for (int c = 0; c < 2; ++c) {
        if (mem.alloc((void**)&units_c[c], ulp[c].size() * sizeof(int4)) != cudaSuccess ||
            cudaMemcpyAsync(units_c[c], ulp[c].data(), ulp[c].size() * sizeof(int4), cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
          return fail_cuda();
      }
      if (cudaMemcpyAsync(slot_lp, sblp[0].data(), (ng + 1) * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(slot_lp2, sblp[1].data(), (ng + 1) * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail_cuda();
      auto syrk_args = [&](int c) {
        TcGemmArgs a{};
        a.dp = D; a.d_real = 0; a.sym = 1; a.epi = TC_EPI_NS_SYRK; a.n_groups = 1;
        a.group_start[0] = 0; a.group_start[1] = 1; a.pair_a[0] = 0; a.pair_b[0] = 0;
        a.group_scale[0] = 1.0; a.scale = 1.0f; a.out = elp; a.partials = partials; a.status = status;
        a.skip = all_done; a.units = units_c[c]; a.n_units = (int)ulp[c].size();
        a.mat_dp = c == 0 ? ia(I_DP128) : ia(I_DP256); a.mat_d = ia(I_D); a.mat_skip = ia(I_DONE);
        a.mat_stride = (long long)slot; a.a_planes = 1; a.b_planes = 1;
        return a;
      };
      // tile choice: forced, cached, or timed on the first SYRK (which
      // writes only E and the partials; the stage recomputes both)
      int choice = opt.batch_tile == 128 ? 0 : (opt.batch_tile == 256 ? 1 : -1);
      std::vector<int> key;
      if (choice < 0) {
        key.push_back(fmt);
        key.push_back(D);
        std::vector<int> sorted_dp = dp128;
        std::sort(sorted_dp.begin(), sorted_dp.end());
        key.insert(key.end(), sorted_dp.begin(), sorted_dp.end());
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) choice = it->second.bn == 128 ? 0 : 1;
      }
      if (choice < 0) {
        float best = 1e30f;
        for (int c = 0; c < 2; ++c) {
          const TcGemmArgs a = syrk_args(c);
          float t_c = 0.f;
          for (int rep = 0; rep < 3; ++rep) {
            if (opt.timing == 0 && !ev[0]) {
              for (auto& e : ev)
                if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda();
            }
            cudaEventRecord(ev[2], st);
            if (tc_gemm_grouped(a, cand_bn[c], xlp[0], ng, xlp[0], ng, fmt, num_sms, st) != cudaSuccess)
              return fail_cuda();
            cudaEventRecord(ev[3], st);
            if (cudaEventSynchronize(ev[3]) != cudaSuccess) return fail_cuda();
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[2], ev[3]);
            if (rep > 0) t_c += t;  // the first launch pays the one-time set-up
            ++launches;
          }
          if (t_c < best) {
            best = t_c;
            choice = c;
          }
        }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = TileChoice{cand_bn[choice], 0};
      }
      tile_bn = cand_bn[choice];
      int* slot_use = choice == 0 ? slot_lp : slot_lp2;
      const TcGemmArgs sy = syrk_args(choice);
      // the FP64 polish uses the 128-column tiles (its int64 sums live in
      // TMEM next to two 128-column accumulators)
      units_sel = units_c[0];
      n_units_sel = (int)ulp[0].size();
      slot_sel = slot_lp;
      mat_dp_sel = ia(I_DP128);
      TcGemmArgs up = sy;
      up.epi = TC_EPI_NS_UPDATE;
      up.partials = trpart;
      const double u = fmt ? 0.00390625 : 0.00048828125;  // unit roundoff of the operand type
      const int max_steps = opt.max_steps;
      auto step = [&](int gs, cudaStream_t s2, bool last) -> bool {
        void* xm = xlp[gs & 1];
        void* xn = xlp[(gs + 1) & 1];
        if (tc_gemm_grouped(sy, tile_bn, xm, ng, xm, ng, fmt, num_sms, s2) != cudaSuccess) return false;
        batch_check_kernel<<<check_blocks, 32 * kCheckWarps, 0, s2>>>(
            partials, slot_use, ng, ia(I_D), 0, tol, u, max_steps, ia(I_DONE), ia(I_STEPS), da(D_PREV),
            da(D_RESID), all_done, ctr, trpart, ia(I_K));
        if (cudaGetLastError() != cudaSuccess) return false;
        if (last) return true;
        TcGemmArgs a = up;
        a.out = xn;
        a.xin = xm;
        if (tc_gemm_grouped(a, tile_bn, xm, ng, elp, ng, fmt, num_sms, s2) != cudaSuccess) return false;
        if (s2 == st) launches += 3;
        return true;
      };
      if (!run_stage(max_steps, all_done, 3, step)) return fail_cuda();
      // FP64 copy of each matrix's final iterate
      if (fmt == 0)
        batch_to_f64_kernel<__half><<<grid_of(nel), 256, 0, st>>>((const __half*)xlp[0], (const __half*)xlp[1],
                                                                  ia(I_STEPS), D, nel, x64[0]);
      else
        batch_to_f64_kernel<__nv_bfloat16><<<grid_of(nel), 256, 0, st>>>(
            (const __nv_bfloat16*)xlp[0], (const __nv_bfloat16*)xlp[1], ia(I_STEPS), D, nel, x64[0]);
      ++launches;
      if (cudaGetLastError() != cudaSuccess) return fail_cuda();
    } else {
      batch_scale_kernel<double><<<grid_of(nel), 256, 0, st>>>(A64, da(D_ALPHA), D, nel, x64[0]);
      ++launches;
      if (cudaGetLastError() != cudaSuccess) return fail_cuda();
    }
    if (opt.timing) cudaEventRecord(ev[2], st);

    const bool run64 = !low || polish;
    if (polish) {
      // ---------------------------------------------------------- FP64 polish
      // X+ = X + 1/2 X (I - X^2) with FP64-emulating digit-plane products on
      // the tensor cores (>= 54-bit digits; see fp64e_gemm), grouped over the
      // slab with the tile table of the low-precision stage: per step one
      // digit split of X, one fused I - X^2 product with residual partials,
      // the stop test, one split of E and one fused update product.
      int dmax = 0;
      for (int x : g.d) dmax = std::max(dmax, x);
      const int beta = fp64e_beta(dmax);
      const int P = fp64e_planes(beta);
      SplitMat Xs{}, Es{};
      Xs.n_planes = Es.n_planes = P;
      Xs.beta = Es.beta = beta;
      Xs.keep_diag = Es.keep_diag = 1;  // 54-bit digits of the whole rows: no exact diagonal terms needed
      long long* acc64 = nullptr;
      if (beta == 0 || mem.alloc(&Xs.planes, nel * 2 * P) != cudaSuccess ||
          mem.alloc(&Es.planes, nel * 2 * P) != cudaSuccess ||
          mem.alloc((void**)&Xs.sigma, (size_t)ng * D * 8) != cudaSuccess ||
          mem.alloc((void**)&Xs.diag, (size_t)ng * D * 8) != cudaSuccess ||
          mem.alloc((void**)&Es.sigma, (size_t)ng * D * 8) != cudaSuccess ||
          mem.alloc((void**)&Es.diag, (size_t)ng * D * 8) != cudaSuccess ||
          mem.alloc((void**)&acc64, nel * 8) != cudaSuccess)
        return fail_cuda();
      Fp64eExtra base{};
      base.acc64 = acc64;
      base.skip = all_done64;
      base.k_extent = dmax;
      base.units = units_sel;
      base.n_units = n_units_sel;
      base.n_mat = ng;
      base.bn = 128;
      base.mat_dp = mat_dp_sel;
      base.mat_d = ia(I_D);
      base.mat_skip = ia(I_DONE64);
      const int max_steps = opt.polish_steps;
      auto step = [&](int gs, cudaStream_t s2, bool last) -> bool {
        double* X = x64[gs & 1];
        Xs.full = X;
        if (split_rows_grouped(X, D, ng, mat_dp_sel, Xs, s2) != cudaSuccess) return false;
        Fp64eExtra sq = base;
        sq.ident = 1;
        sq.partials = partials;
        if (fp64e_gemm(Xs, Xs, D, dmax, 1, e64, sq, status, num_sms, s2, P) != cudaSuccess) return false;
        batch_check_kernel<<<check_blocks, 32 * kCheckWarps, 0, s2>>>(
            partials, slot_sel, ng, ia(I_D), 2, tol, 0.0, max_steps, ia(I_DONE64), ia(I_STEPS64),
            da(D_PREV), da(D_RESID), all_done64, ctr, nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) return false;
        if (last) return true;
        Es.full = e64;
        if (split_rows_grouped(e64, D, ng, mat_dp_sel, Es, s2) != cudaSuccess) return false;
        Fp64eExtra up = base;
        up.xin64 = X;
        up.xin_mult = 0.5;
        if (fp64e_gemm(Xs, Es, D, dmax, 1, x64[(gs + 1) & 1], up, status, num_sms, s2, P) != cudaSuccess)
          return false;
        if (s2 == st) launches += 5;
        return true;
      };
      if (!run_stage(max_steps, all_done64, 5, step)) return fail_cuda();
    } else if (run64) {
      // --------------------------------------------- FP64 stage / FP64 polish
      F64GemmArgs sy{};
      sy.dp = D; sy.d_real = 0; sy.sym = 1; sy.epi = F64_EPI_NS_SYRK; sy.out = e64; sy.partials = partials;
      sy.skip = all_done64; sy.units = units64; sy.n_units = (int)u64.size(); sy.mat_dp = ia(I_DP64);
      sy.mat_d = ia(I_D); sy.mat_skip = ia(I_DONE64); sy.mat_stride = (long long)slot;
      const int mode = polish ? 2 : 1;
      const int max_steps = polish ? opt.polish_steps : opt.max_steps;
      auto step = [&](int gs, cudaStream_t s2, bool last) -> bool {
        F64GemmArgs a = sy;
        a.A = x64[gs & 1];
        a.B = x64[gs & 1];
        if (f64_gemm_grouped(a, s2) != cudaSuccess) return false;
        batch_check_kernel<<<check_blocks, 32 * kCheckWarps, 0, s2>>>(
            partials, slot_64, ng, ia(I_D), mode, tol, 0.0, max_steps, ia(I_DONE64), ia(I_STEPS64),
            da(D_PREV), da(D_RESID), all_done64, ctr, nullptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) return false;
        if (last) return true;
        F64GemmArgs b = sy;
        b.epi = F64_EPI_NS_UPDATE;
        b.A = x64[gs & 1];
        b.B = e64;
        b.xin = x64[gs & 1];
        b.out = x64[(gs + 1) & 1];
        if (f64_gemm_grouped(b, s2) != cudaSuccess) return false;
        if (s2 == st) launches += 3;
        return true;
      };
      if (!run_stage(max_steps, all_done64, 3, step)) return fail_cuda();
    }

    // ---- certificate and output
    const double* res0 = x64[0];
    const double* res1 = run64 ? x64[1] : nullptr;
    const int* par = run64 ? ia(I_STEPS64) : ia(I_STEPS);
    batch_trace_kernel<<<ng, 1024, 0, st>>>(res0, res1, par, ia(I_D), D, da(D_TRACE));
    {
      dim3 grid(D / 32, D / 32, ng), block(32, 8);
      batch_scatter_kernel<<<grid, block, 0, st>>>(res0, res1, par, ia(I_D), D, rptr);
    }
    launches += 2;
    if (cudaGetLastError() != cudaSuccess) return fail_cuda();
    for (int m : r_host) {
      const int i = g.idx[m];
      if (cudaMemcpyAsync(R[i], rp[m], (size_t)g.d[m] * g.d[m] * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail_cuda();
    }
    if (opt.timing) cudaEventRecord(ev[3], st);
    if (cudaMemcpyAsync(h_int.data(), ib, n_int * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(h_dbl.data(), db, h_dbl.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail_cuda();
    float ms_total = 0.f, ms_low = 0.f, ms_64 = 0.f;
    if (opt.timing) {
      cudaEventElapsedTime(&ms_total, ev[0], ev[3]);
      cudaEventElapsedTime(&ms_low, ev[1], ev[2]);
      cudaEventElapsedTime(&ms_64, ev[2], ev[3]);
    }
    const int dev_status = h_int[(size_t)(status - ib)];
    for (int m = 0; m < ng; ++m) {
      const int i = g.idx[m];
      const int dm = g.d[m];
      const int flags = h_int[(size_t)I_FLAGS * ng + m];
      const double alpha = h_dbl[(size_t)D_ALPHA * ng + m];
      const double trace = h_dbl[(size_t)D_TRACE * ng + m];
      const double resid = h_dbl[(size_t)D_RESID * ng + m];
      const int done_low = h_int[(size_t)I_DONE * ng + m];
      const int done64 = h_int[(size_t)I_DONE64 * ng + m];
      const int steps_low = low ? h_int[(size_t)I_STEPS * ng + m] : 0;
      const int steps64 = run64 ? h_int[(size_t)I_STEPS64 * ng + m] : 0;
      const double tol_fro = std::max(tol, 16.0 * dm * kEps64);
      const bool trace_ok = std::fabs(trace - (double)(dm - 2 * g.k[m])) < 0.5;
      const bool resid_ok = policy == RSIGN_FP64 ? (resid <= tol_fro) : true;
      rsign_status r = RSIGN_OK;
      if (dev_status != 0) r = (rsign_status)dev_status;
      else if ((flags & 1) || !(alpha > 0.0)) r = RSIGN_ERR_ARG;
      else if (policy == RSIGN_FP64 && done64 != 1) r = RSIGN_ERR_NOCONV;
      else if (low && !polish && done_low != 1) r = RSIGN_ERR_NOCONV;
      else if (!trace_ok) r = RSIGN_ERR_CERT;
      stat[i] = r;
      if (infos) {
        rsign_info* inf = &infos[i];
        inf->steps_low = steps_low;
        inf->steps_fp64 = steps64;
        inf->cert_ok = (trace_ok && resid_ok) ? 1 : 0;
        inf->alpha = alpha;
        inf->shift = g.s[m];
        inf->gamma_est = NAN;
        inf->resid_fro = resid;
        inf->trace = trace;
        inf->correction_fro = NAN;
        inf->commutator_norm = NAN;
        inf->err_est = NAN;
        inf->err_bound = NAN;
        inf->tol_fro = tol_fro;
        inf->ms_total = ms_total;
        inf->ms_low = low ? ms_low : 0.0;
        inf->ms_fp64 = ms_64;
        inf->flops_low = low ? (double)dm * dm * dm * (2.0 * steps_low + 1.0) : 0.0;
        inf->launches = launches;
        inf->workspace_bytes = mem.bytes;
        inf->steps_pred = -1;
        inf->batch_grouped = 1;
        inf->batch_tile = low ? tile_bn : kF64Tile;
      }
    }
    cleanup();
    if (cudaGetLastError() != cudaSuccess) return RSIGN_ERR_CUDA;
  }

  // ---- the rest: one-matrix calls (the refinement policies, automatic
  // shifts, orders above kBatchMaxD), run concurrently by worker threads,
  // each on a stream of its own that first waits for the caller's stream.
  // Each call is the same computation as a lone rsign_reflector_ex call on
  // that matrix (same kernels, same order: the same bits); small matrices
  // leave most SMs idle, so several calls in flight fill the GPU.
  if (!rest.empty()) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RSIGN_ERR_CUDA;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nw = (int)std::min<size_t>({rest.size(), (size_t)kRestWorkers, (size_t)hw});
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, st) != cudaSuccess) {
      if (ready) cudaEventDestroy(ready);
      cudaGetLastError();
      return RSIGN_ERR_CUDA;
    }
    std::atomic<size_t> next(0);
    auto worker = [&]() {
      cudaStream_t ws = nullptr;
      if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) {
        cudaGetLastError();
        if (ws) cudaStreamDestroy(ws);
        return;
      }
      for (size_t q; (q = next++) < rest.size();) {
        const int i = rest[q];
        stat[i] = rsign_reflector_ex(H[i], d[i], k[i], s[i], tol, policy, &opt, R[i],
                                     infos ? &infos[i] : nullptr, (void*)ws);
      }
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
    };
    if (nw <= 1) {
      for (int i : rest)
        stat[i] = rsign_reflector_ex(H[i], d[i], k[i], s[i], tol, policy, &opt, R[i],
                                     infos ? &infos[i] : nullptr, (void*)st);
    } else {
      std::vector<std::thread> pool;
      pool.reserve(nw);
      for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
      for (auto& t : pool) t.join();
      // a worker that could not set up its stream left matrices undone: the
      // caller's stream finishes them
      for (size_t q; (q = next++) < rest.size();) {
        const int i = rest[q];
        stat[i] = rsign_reflector_ex(H[i], d[i], k[i], s[i], tol, policy, &opt, R[i],
                                     infos ? &infos[i] : nullptr, (void*)st);
      }
    }
    cudaEventDestroy(ready);
  }
  for (int i = 0; i < n; ++i)
    if (stat[i] != RSIGN_OK) return stat[i];
  return RSIGN_OK;
}

}  // namespace rsign

extern "C" {

rsign_status rsign_reflector_batched_ex(int32_t n, const double* const* H, const int64_t* d,
                                        const int32_t* k, const double* s, double tol,
                                        rsign_policy policy, const rsign_options* opt,
                                        double* const* R, rsign_info* infos, void* stream) {
  return rsign::batched_impl(n, H, d, k, s, tol, policy, opt, R, infos, (cudaStream_t)stream);
}

rsign_status rsign_reflector_batched(int32_t n, const double* const* H, const int64_t* d,
                                     const int32_t* k, const double* s, double tol,
                                     rsign_policy policy, double* const* R, rsign_info* infos,
                                     void* stream) {
  return rsign::batched_impl(n, H, d, k, s, tol, policy, nullptr, R, infos, (cudaStream_t)stream);
}

}  // extern "C"
