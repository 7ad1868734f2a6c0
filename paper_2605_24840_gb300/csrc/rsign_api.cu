// rsign_api.cu -- C ABI of the shifted matrix-sign reflector (see include/rsign.h).
//
// Host orchestration of one call:
//   1. ingest: A = 1/2 (H + H^T) - sI (FP64, zero padded to dp, a multiple
//      of 256), row sums of |A| -> alpha = 1/||A||_inf (Sec. 4.3);
//   2. Newton-Schulz X_{m+1} = X_m + 1/2 X_m (I - X_m^2) (Eq. NS, written in
//      update form), each step as a SYRK-style product E = I - X^2 with a
//      fused residual ||X^2 - I||_F and a symmetric product X + 1/2 X E;
//      the low-precision stage runs on the tcgen05 tensor cores, the FP64
//      stage on the FP64 pipe; the stop test runs on the device and later
//      launches of the chunk return at once (no host round trip per step);
//   3. certificate: trace(R) = d - 2k (Prop. 2.1, Lemma 3.4) and the residual.
#include "common.cuh"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace rsign {

// Library-owned stream-ordered memory pool per device.  Its release threshold
// is unlimited, so the workspace of one call stays mapped for the next call
// (re-mapping tens of GB per call costs tens of milliseconds);
// rsign_trim_workspace() returns the cached memory to the driver.
namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};
}  // namespace

cudaMemPool_t library_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxPoolDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (g_pools[dev] == nullptr) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

cudaError_t DevBuf::alloc(void** p, size_t n) {
  n = (n + 255) & ~size_t(255);
  cudaMemPool_t pool = library_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, n, pool, st) : cudaMallocAsync(p, n, st);
  if (e == cudaSuccess) {
    ptrs.push_back(*p);
    bytes += (int64_t)n;
  }
  return e;
}

void DevBuf::release() {
  for (void* p : ptrs) cudaFreeAsync(p, st);
  ptrs.clear();
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// In-place access of page-locked host buffers by the kernels (1) instead of
// staging copies (0, the default).  Measured end to end at d = 8192 with
// pinned buffers: about 0.6 ms faster than the staged copies on two GB300
// boxes, ~150 ms slower on a third; the copy engines are the steadier path.
int g_host_mapped = 0;

// Staged host copies of H and R split over this many streams (1 = one copy
// on the call's stream; more lets several copy engines share the link).
int g_copy_streams = 1;

// dst <- src (bytes, a staged host copy) on `st`: split over g_copy_streams
// streams that fork from and join back into `st` (stream-ordered for every
// caller of `st`).  Parts are whole multiples of 1 MiB but the last.
cudaError_t staged_copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
  const int n = std::max(1, std::min(g_copy_streams, 8));
  if (n == 1 || bytes < ((size_t)64 << 20)) return cudaMemcpyAsync(dst, src, bytes, kind, st);
  cudaStream_t hs[8] = {};
  cudaEvent_t fork = nullptr, join[8] = {};
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(fork, st);
  const size_t part = ((bytes / n) + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
  for (int q = 1; q < n && e == cudaSuccess; ++q) {
    const size_t off = part * q;
    if (off >= bytes) break;
    const size_t len = std::min(part, bytes - off);
    if ((e = cudaStreamCreateWithFlags(&hs[q], cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&join[q], cudaEventDisableTiming)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(hs[q], fork, 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, len, kind,
                             hs[q])) != cudaSuccess)
      break;
    e = cudaEventRecord(join[q], hs[q]);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, std::min(part, bytes), kind, st);
  for (int q = 1; q < n; ++q)
    if (join[q] && e == cudaSuccess) e = cudaStreamWaitEvent(st, join[q], 0);
  for (int q = 1; q < n; ++q) {
    if (join[q]) cudaEventDestroy(join[q]);
    if (hs[q]) cudaStreamDestroy(hs[q]);  // released once its work is done
  }
  if (fork) cudaEventDestroy(fork);
  return e;
}

// Device address of page-locked host memory (cudaHostAlloc / cudaHostRegister:
// mapped into the device's address space), or nullptr for any other pointer.
// Kernels read and write such memory directly over the CPU-GPU link, with
// no staging copy (on GB300 the NVLink-C2C link to the Grace CPU).
const void* mapped_host_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int check_device(int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return RSIGN_ERR_CUDA; }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (major != 10 || minor != 3) return RSIGN_ERR_UNSUPPORTED;
  return RSIGN_OK;
}

namespace {

constexpr int kChunk = 8;  // NS steps enqueued between host checks of the stop flag
// Low-precision stage: the first chunk reaches three steps past m_min (the
// step from which the floor tests apply; the stop follows within a step or
// two when the margin is known), later chunks are shorter, so that fewer
// launches are enqueued past the device-side stop (they return at once, but
// each still costs a launch).
constexpr int kChunkLate = 4;

// Control block kept in device memory (one allocation, read back with one copy).
struct Ctl {
  int status;     // device status word (RSIGN_ERR_TIMEOUT on a failed bounded wait)
  int flags;      // bit 0: non-finite input
  int done_low, steps_low;
  int done64, steps64;
  int pad[2];
  double scal[8];  // [0] ||A||_inf  [1] alpha  [2] trace  [3..4] scratch
};

struct Ctx {
  cudaStream_t st;
  int num_sms = 0;
  int64_t launches = 0;
  cudaError_t err = cudaSuccess;
  bool ok(cudaError_t e) {
    ++launches;
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    return err == cudaSuccess;
  }
};

bool is_low(rsign_policy p) { return p != RSIGN_FP64; }
int lp_fmt_of(rsign_policy p) {
  return (p == RSIGN_BF16 || p == RSIGN_BF16_POLISH || p == RSIGN_BF16_REFINE) ? 1 : 0;
}
double unit_roundoff(int fmt) { return fmt ? 0.00390625 /* 2^-8 */ : 0.00048828125 /* 2^-11 */; }

// FP64 Newton-Schulz on buffers xb[0], xb[1] (X_0 in xb[0]); stops on the
// device when ||X_m^2 - I||_F < tol_abs (tol_abs < 0: run exactly max_steps
// updates).  Returns the index m of the returned iterate X_m (in xb[m % 2])
// and whether the stop test fired.
struct F64Loop {
  double* xb[2];
  double* E;
  double* partials;
  double* hist;
  int* done;
  int* steps;
  double* W = nullptr;  // NS5 engine: W = E + 3/4 E^2 (nullptr: Eq. NS)
};

bool f64_ns(Ctx& c, const F64Loop& L, int dp, int d, double tol_abs, int max_steps, Ctl* ctl_dev,
            Ctl& ctl_host, int* m_out, bool* conv, const std::vector<double>* coef = nullptr) {
  const int nt = f64_num_tiles(dp, 1);
  int m = 0;
  bool stopped = false;
  for (; m <= max_steps && !stopped; ) {
    const int m_end = std::min(m + kChunk, max_steps + 1);
    for (int mm = m; mm < m_end; ++mm) {
      F64GemmArgs sy{};
      sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = F64_EPI_NS_SYRK;
      sy.A = L.xb[mm & 1]; sy.B = L.xb[mm & 1]; sy.out = L.E; sy.partials = L.partials;
      sy.skip = L.done;
      const double am = (coef != nullptr && mm < (int)coef->size()) ? (*coef)[mm] : 1.0;
      sy.ns_c2 = am * am;
      if (!c.ok(f64_gemm(sy, c.st))) return false;
      if (!c.ok(ns_check(L.partials, nt * 4, L.hist, mm, tol_abs, -1.0, -1.0, 0.0, L.done, L.steps, c.st)))
        return false;
      if (mm == max_steps) break;  // residual of the last iterate only
      if (L.W != nullptr) {
        // NS5: W = E + 3/4 E^2 (the update epilogue with scale 3/2 on E E),
        // then X+ = X + 1/2 X W = 1/8 X (15I - 10X^2 + 3X^4)
        F64GemmArgs w{};
        w.dp = dp; w.d_real = d; w.sym = 1; w.epi = F64_EPI_NS_UPDATE; w.scale = 1.5;
        w.A = L.E; w.B = L.E; w.xin = L.E; w.out = L.W; w.partials = L.partials; w.skip = L.done;
        if (!c.ok(f64_gemm(w, c.st))) return false;
      }
      F64GemmArgs up{};
      up.dp = dp; up.d_real = d; up.sym = 1; up.epi = F64_EPI_NS_UPDATE;
      up.A = L.xb[mm & 1]; up.B = L.W != nullptr ? L.W : L.E; up.xin = L.xb[mm & 1];
      up.out = L.xb[(mm + 1) & 1];
      up.partials = L.partials; up.skip = L.done;
      up.ns_c1 = am;
      if (!c.ok(f64_gemm(up, c.st))) return false;
    }
    if (!c.ok(cudaMemcpyAsync(&ctl_host, ctl_dev, sizeof(Ctl), cudaMemcpyDeviceToHost, c.st))) return false;
    if (!c.ok(cudaStreamSynchronize(c.st))) return false;
    c.launches -= 2;  // the copy and the sync are not kernels
    stopped = (L.done == &ctl_dev->done64) ? ctl_host.done64 != 0 : ctl_host.done_low != 0;
    m = m_end;
  }
  const int steps = (L.done == &ctl_dev->done64) ? ctl_host.steps64 : ctl_host.steps_low;
  *conv = stopped;
  *m_out = stopped ? steps : max_steps;
  return true;
}

// Tile width of the digit-plane products of one-matrix calls (the
// refinement's FP64-grade products and the FP64-emulating polish): 128 keeps
// the int64 level sums in TMEM (grouped-mode launch over a one-matrix tile
// table), 256 keeps them in global memory between level groups; 0 = by order.
// Short K loops favour the TMEM sums (a level group's MMAs do not hide the
// read-modify-write of its sums), long ones the 256-wide tiles (each A panel
// load serves twice the columns, so less operand traffic per product).
int g_oz_tile = 0;
int oz_tile_for(int dp) { return g_oz_tile != 0 ? g_oz_tile : (dp <= 3072 ? 128 : 256); }

// Tile table of one dp x dp product on 128 x 128 tiles (upper triangle when
// sym), visited in blocks of 16 x 16 tiles so that the CTAs in flight share
// row and column panels in L2.
std::vector<int4> oz_tile_table(int dp, int sym) {
  const int nb = dp / 128, bh = 16, bw = 16;
  std::vector<int4> u;
  for (int cb = 0; cb < nb; cb += bw)
    for (int rb = 0; rb < nb; rb += bh)
      for (int r = rb; r < std::min(rb + bh, nb); ++r)
        for (int c = cb; c < std::min(cb + bw, nb); ++c)
          if (!sym || c >= r) u.push_back(make_int4(0, r, c, (int)u.size()));
  return u;
}

// Device tile table (and {dp, d}) of one product on 128 x 128 tiles, from the
// call's workspace.
cudaError_t make_oz_tiles(DevBuf& mem, int dp, int d, int sym, cudaStream_t st, OzTiles* out) {
  const std::vector<int4> u = oz_tile_table(dp, sym);
  int4* du = nullptr;
  int* dims = nullptr;
  const int h_dims[2] = {dp, d};
  cudaError_t e;
  if ((e = mem.alloc((void**)&du, u.size() * sizeof(int4))) != cudaSuccess) return e;
  if ((e = mem.alloc((void**)&dims, 2 * sizeof(int))) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(du, u.data(), u.size() * sizeof(int4), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(dims, h_dims, 2 * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;  // the host table goes out of scope
  out->units = du;
  out->n_units = (int)u.size();
  out->dims = dims;
  return cudaSuccess;
}

// FP64 polish steps X+ = X + 1/2 X (I - X^2) (Eq. NS, update form) on the
// tensor cores: both products are FP64-emulating digit-plane products
// (fp64e: >= 54-bit digits, FP32-exact group sums, int64 fixed point), the
// first one fused with I - X^2 and its residual, the second with the update.
// Runs exactly `steps` updates and a final residual product, as the FP64
// polish of the one-matrix FP64 loop does; X_0 in xb[0], the result in
// xb[steps & 1], residuals in hist[0..steps].
cudaError_t fp64e_polish(Ctx& c, DevBuf& mem, double* xb[2], double* E, int dp, int d, int steps,
                         double* partials, double* hist, Ctl* ctl) {
  const size_t dd = (size_t)dp * dp;
  const int beta = fp64e_beta(d);
  if (beta == 0) return cudaErrorInvalidValue;
  const int P = fp64e_planes(beta);
  SplitMat Xs{}, Es{};
  Xs.n_planes = Es.n_planes = P;
  Xs.beta = Es.beta = beta;
  Xs.keep_diag = Es.keep_diag = 1;  // 54-bit digits of the whole rows: no exact diagonal terms needed
  long long* acc64 = nullptr;
  cudaError_t e;
  if ((e = mem.alloc(&Xs.planes, dd * 2 * P)) != cudaSuccess) return e;
  if ((e = mem.alloc(&Es.planes, dd * 2 * P)) != cudaSuccess) return e;
  if ((e = mem.alloc((void**)&Xs.sigma, (size_t)dp * 8)) != cudaSuccess) return e;
  if ((e = mem.alloc((void**)&Xs.diag, (size_t)dp * 8)) != cudaSuccess) return e;
  if ((e = mem.alloc((void**)&Es.sigma, (size_t)dp * 8)) != cudaSuccess) return e;
  if ((e = mem.alloc((void**)&Es.diag, (size_t)dp * 8)) != cudaSuccess) return e;
  if ((e = mem.alloc((void**)&acc64, dd * 8)) != cudaSuccess) return e;
  // up to order 4096 the products run on 128 x 128 tiles with the int64 sums
  // in TMEM (as the refinement's products); the residual partials then come
  // per tile of that table
  OzTiles tz{};
  int nt = tc_num_tiles(dp, 1);
  const bool t128 = oz_tile_for(dp) == 128;
  if (t128) {
    if ((e = make_oz_tiles(mem, dp, d, 1, c.st, &tz)) != cudaSuccess) return e;
    nt = tz.n_units;
  }
  auto tiles = [&](Fp64eExtra& x) {
    if (!t128) return;
    x.units = tz.units;
    x.n_units = tz.n_units;
    x.n_mat = 1;
    x.bn = 128;
    x.mat_dp = tz.dims;
    x.mat_d = tz.dims + 1;
  };
  for (int m = 0; m <= steps; ++m) {
    double* X = xb[m & 1];
    Xs.full = X;
    if (!c.ok(split_rows(X, dp, Xs, c.st))) return c.err;
    Fp64eExtra sq{};
    sq.acc64 = acc64;
    sq.ident = 1;
    sq.partials = partials;
    tiles(sq);
    if (!c.ok(fp64e_gemm(Xs, Xs, dp, d, 1, E, sq, &ctl->status, c.num_sms, c.st, P))) return c.err;
    if (!c.ok(ns_check(partials, nt * 4, hist, m, -1.0, -1.0, -1.0, 0.0, &ctl->done64, &ctl->steps64, c.st)))
      return c.err;
    if (m == steps) break;
    Es.full = E;
    if (!c.ok(split_rows(E, dp, Es, c.st))) return c.err;
    Fp64eExtra up{};
    up.acc64 = acc64;
    up.xin64 = X;
    up.xin_mult = 0.5;
    tiles(up);
    if (!c.ok(fp64e_gemm(Xs, Es, dp, d, 1, xb[(m + 1) & 1], up, &ctl->status, c.num_sms, c.st, P)))
      return c.err;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Commutator refinement (beyond the paper's plain iteration; needed because
// Newton-Schulz forgets A after X_0: an error that anticommutes with sign(A)
// is a fixed point of the update, so low-precision subspace errors persist
// through any number of FP64 steps).  With R ~ S = sign(A) an involution and
// C = R A - A R, the off-block error F = S - R solves |A| F + F |A| = R C
// (eigen-basis: F_ij = (RC)_ij / (|lam_i| + |lam_j|)), i.e. F = L_sign(A, G)
// with G = 1/4 (R C + (R C)^T), the Frechet derivative of the sign function.
// L_sign(A, G) is evaluated by the tangent recursion of Eq. NS along the
// stored low-precision iterates:
//   E_0 = alpha G,  E_{m+1} = 1/2 E_m + 1/2 (E_m Et_m + Et_m E_m) - 1/2 X_m E_m X_m,
// (Et_m = I - X_m^2), then R <- R + E_M and one update-form polish step
// R <- R + 1/2 R (I - R^2) restores R^2 = I.  N = R A and R^2 are FP64-grade
// products; everything else is FP16/BF16 with FP32 accumulation.
// ---------------------------------------------------------------------------
struct RefineIn {
  int dp, d, k, fmt, M, max_sweeps;
  int M_tangent;        // tangent steps run: m = 0 .. M_tangent - 1 (<= M)
  double alpha, tol;
  double* A64;          // A = sym(H) - sI, FP64, zero padded
  double* R64;          // in: stage-1 result; out: refined reflector
  void* const* X;       // X_0 .. X_{M-1} (operand type)
  void* const* Et;      // I - a_m^2 X_m^2, m = 0 .. M-1 (operand type)
  bool pairs;           // X and Et slots hold hi/lo pairs of planes (plane stride dp^2)
  const double* a;      // step scalings a_m of the stage-1 trajectory (nullptr: all 1)
  int n_a;              // entries of a (steps beyond use 1)
  double margin;        // lower bound of min |lam_i(A)| (NaN: unknown)
  double mu_lb;         // margin, or a lower bound from the stage-1 step count
  bool stop_on_bound;   // stop test on the bound (needs margin) instead of the estimate
};
struct RefineOut {
  int sweeps = 0, polish_steps = 0;
  bool converged = false;
  double resid = NAN, corr = NAN, comm = NAN, err_est = NAN, err_bound = NAN, rho = NAN;
  int levels_ra0 = 0;
};

// Order above which the Newton-Schulz SYRK takes the diagonal of X^2 from
// exact row norms (row_sumsq) instead of the tensor-core sums.
constexpr int kExactDiagMin = 1024;

// Digit levels of the refinement's FP64-grade products (5 bits each): the
// polish SYRK R^2, the first sweep's R A and the later sweeps' R A; 0 = by
// rule.  Polish: the truncation error scales with the off-diagonal row maxima
// of R = I - 2 P_k, which grow like sqrt(min(k, d - k))/d; five levels when
// the index is small against d (measured at d = 8192, k = 16), else six.
int g_levels_polish = 0, g_levels_ra0 = 0, g_levels_ra = kSlices;
// Digit planes of the refinement's FP64-grade products as FP8 E4M3 bytes on
// the kind::f8f6f4 tensor cores (1, the default) or as FP16 (0).  The 5-bit
// balanced digits (|digit| <= 16) are exact in E4M3 and the level sums are
// the same integers either way, so both give the same bits; FP8 has twice
// the tensor rate and half the operand bytes (measured at d = 8192: the two
// products of a FP16_REFINE call 18.4 -> 12.1 ms).
int g_digit_fp8 = 1;
// Stage-1 iterates carried as hi/lo pairs by the *_REFINE policies: every
// iterate (g_split_steps = -1, the default), the first n (n >= 0), or by
// rule (-2): while the known lower end l_m of the iterate's spectrum (the
// scaled or plain recurrence from alpha * margin) is below g_split_until,
// FP16_REFINE only; later steps then run on single FP16 planes, one pair
// product per launch instead of three.  Rounding made while the eigenvalues
// next to the gap are small is what the tangent solve cannot undo in one
// sweep (its relative error there is ~u / l_m); later single-plane steps
// add cross-eigenspace noise of ~u that the sweep must remove.  Measured at
// d = 8192, k = 16, half-gap 1e-2 the rule with threshold 1/2 saved 9 ms of
// 63 in one sweep, but its error estimate sat at 0.9 of the tolerance and
// the gain did not hold over the sweep of controlled spectra (27 points at
// d = 8192: 3043 ms in total with every iterate a pair, 2968 / 2898 ms with
// thresholds 0.99 / 0.9; at d = 2048 every iterate a pair was fastest).
int g_split_steps = -1;
double g_split_until = 0.5;
// safety factor of the refinement's a-posteriori error estimate (see the check)
constexpr double kEstSafety = 2.5;
// Tangent steps of the refinement at iterates whose known lower end is within
// kTangentCut of 1 are left out with g_tangent_cut = 1; 0, the default, runs
// them all (measured at d = 8192: leaving out the last step made the error
// estimate after the first sweep miss the tolerance, 56 -> 95 ms per call).
constexpr double kTangentCut = 1e-3;
int g_tangent_cut = 0;
int levels_for(int set, double tol, int d, int k) {
  if (set > 0) return set;
  const bool few = 32 * std::min(k, d - k) <= d;
  return (tol >= 1e-6 && few) ? kSlices - 2 : kSlices - 1;
}

// First sweep's R A: the commutator's truncation error reaches the
// correction through the gain of L_sign, up to 1/(2 mu) on the components
// between the two eigenspaces (and largest there when the spectrum next to
// the gap is sparse).  Model: error after the sweep ~ 2^(-5L) s_A s_R sqrt(d)
// / mu, s the largest power-of-two row scales of the two digit splits.
// Measured at L = 5: it over-predicts 7x..14x on the Allen-Cahn Hessian
// (d = 1024, 4096; k = 1, 2, 4) and matches within 1.5x on controlled
// spectra (d = 8192, k = 16; d = 768, k = 384, which needs six levels).  The
// smallest L in 5..7 with a predicted error <= tol / 2.
int levels_ra0(double tol, double sA, double sR, int d, double mu) {
  for (int L = kSlices - 2; L < kSlices; ++L)
    if (std::ldexp(1.0, -5 * L) * sA * sR * std::sqrt((double)d) <= 0.5 * tol * mu) return L;
  return kSlices;
}

// Lower bound of the scaled margin from a plain trajectory that stopped
// after m steps: an eigenvalue x_0 = gamma reaches p_m(gamma) >= 0.9 only for
// gamma above the root of p_m(gamma) = 0.9 (the map is increasing on [0, 1]).
// Step scalings of the scaled iteration for a spectrum of X_0 in
// [-u0, -l0] U [l0, u0] with l0 = min(1, alpha margin) (Sec. 3.5, the stable
// scalings of the cited GPU sign iteration): with l = l0 / u0, each step's
// a = sqrt(3 / (1 + l + l^2)) and l <- 1/2 a l (3 - a^2 l^2), until a is 1
// to 1e-15; the first factor absorbs 1/u0.  Host only.
std::vector<double> scaled_ns_coeffs(double alpha_margin, double u0) {
  std::vector<double> coef;
  double l = std::min(1.0, alpha_margin) / u0;
  for (int m = 0; m < 200; ++m) {
    const double a = std::sqrt(3.0 / (1.0 + l + l * l));
    if (std::fabs(a - 1.0) <= 1e-15) break;
    coef.push_back(m == 0 ? a / u0 : a);
    l = 0.5 * a * l * (3.0 - a * a * l * l);
  }
  return coef;
}

// Lower end l_m of the normalised spectrum of X_m, m = 0 .. max_steps: the
// eigenvalues of X_0 = alpha A lie in [-u0, -l] U [l, u0] with l = alpha
// margin, so l_0 = min(1, alpha margin) / u0, and each step maps the lower
// end by its scaled cubic l <- 1/2 a l (3 - a^2 l^2) (coef[0] carries the
// 1/u0 normalisation; a = 1 beyond the scalings: Eq. NS).  Host only.
std::vector<double> lower_end_sequence(double alpha_margin, double u0, const std::vector<double>& coef,
                                       int max_steps) {
  std::vector<double> out;
  double l = std::min(1.0, alpha_margin) / u0;
  for (int mi = 0; mi <= max_steps; ++mi) {
    out.push_back(l);
    const double a = mi < (int)coef.size() ? coef[mi] * (mi == 0 ? u0 : 1.0) : 1.0;
    l = 0.5 * a * l * (3.0 - a * a * l * l);
  }
  return out;
}

// Stage plan of the *_REFINE policies from the lower ends: the number of
// leading iterates carried as hi/lo pairs (first m with l_m >= kSplitUntil)
// and the number of tangent steps run (first m with l_m >= 1 - kTangentCut,
// at least 1), given steps_low stage-1 steps.
void refine_stage_plan(const std::vector<double>& lower_end, int steps_low, int* n_split, int* m_tangent) {
  int ns = 0;
  while (ns < (int)lower_end.size() && lower_end[ns] < g_split_until) ++ns;
  *n_split = ns;
  int mt = steps_low;
  for (int mi = 0; mi < steps_low && mi < (int)lower_end.size(); ++mi)
    if (lower_end[mi] >= 1.0 - kTangentCut) {
      mt = std::max(1, mi);
      break;
    }
  *m_tangent = mt;
}

double gamma_from_steps(int m) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double g = 0.5 * (lo + hi);
    double x = g;
    for (int q = 0; q < m; ++q) x = 0.5 * x * (3.0 - x * x);
    (x >= 0.9 ? hi : lo) = g;
  }
  return hi;
}

cudaError_t refine_sweeps(Ctx& c, DevBuf& mem, const RefineIn& in, Ctl* ctl, RefineOut* o) {
  const int dp = in.dp, d = in.d;
  const size_t dd = (size_t)dp * dp;
  const int ntile = (dp / 32) * (dp / 32);
  cudaStream_t st = c.st;
  SplitMat As{}, Rs{};
  double *N64 = nullptr, *part = nullptr, *red = nullptr;
  float *C32 = nullptr, *P32 = nullptr, *Q32 = nullptr, *E32 = nullptr, *bmax = nullptr, *fs = nullptr;
  void *Clp = nullptr, *Rlp = nullptr, *Elp = nullptr, *Qlp = nullptr;
  cudaError_t e;
#define RS_TRY(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
  As.fp8 = Rs.fp8 = g_digit_fp8;
  const size_t digit_bytes = g_digit_fp8 ? 1 : 2;
  RS_TRY(mem.alloc(&As.planes, dd * digit_bytes * kSlices));
  RS_TRY(mem.alloc((void**)&As.sigma, (size_t)dp * 8));
  RS_TRY(mem.alloc((void**)&As.diag, (size_t)dp * 8));
  RS_TRY(mem.alloc(&Rs.planes, dd * digit_bytes * kSlices));
  RS_TRY(mem.alloc((void**)&Rs.sigma, (size_t)dp * 8));
  RS_TRY(mem.alloc((void**)&Rs.diag, (size_t)dp * 8));
  As.full = in.A64;
  Rs.full = in.R64;
  RS_TRY(mem.alloc((void**)&N64, dd * 8));
  RS_TRY(mem.alloc((void**)&C32, dd * 4));
  RS_TRY(mem.alloc((void**)&P32, dd * 4));
  RS_TRY(mem.alloc((void**)&Q32, dd * 4));
  RS_TRY(mem.alloc((void**)&E32, dd * 4));
  RS_TRY(mem.alloc(&Clp, dd * 2));
  RS_TRY(mem.alloc(&Rlp, dd * 2));
  RS_TRY(mem.alloc(&Elp, dd * 2));
  RS_TRY(mem.alloc(&Qlp, dd * 2));
  RS_TRY(mem.alloc((void**)&bmax, (size_t)ntile * 4));
  RS_TRY(mem.alloc((void**)&part, (size_t)std::max(ntile, 1024) * 8));
  RS_TRY(mem.alloc((void**)&fs, 16 * 4));
  RS_TRY(mem.alloc((void**)&red, 24 * 8));
  OzTiles oz_full{}, oz_sym{};
  const OzTiles* tz_full = nullptr;
  const OzTiles* tz_sym = nullptr;
  if (oz_tile_for(dp) == 128) {
    RS_TRY(make_oz_tiles(mem, dp, d, 0, st, &oz_full));
    RS_TRY(make_oz_tiles(mem, dp, d, 1, st, &oz_sym));
    tz_full = &oz_full;
    tz_sym = &oz_sym;
  }
  int* status = &ctl->status;

  auto tc = [&](const void* A, const void* B, int fmt, int sym, int epi, void* out) {
    TcGemmArgs a{};
    a.dp = dp; a.d_real = d; a.sym = sym; a.epi = epi; a.n_groups = 1;
    a.group_start[0] = 0; a.group_start[1] = 1; a.pair_a[0] = 0; a.pair_b[0] = 0;
    a.group_scale[0] = 1.0; a.scale = 1.0f; a.out = out; a.status = status; a.skip = nullptr;
    return tc_gemm(a, A, 1, B, 1, fmt, c.num_sms, st);
  };
  // One update-form polish step of the quintic Newton-Schulz filter:
  // R <- R + 1/2 R W, W = E + 3/4 E^2, E = I - R^2 (R (15I - 10R^2 + 3R^4)/8).
  // An eigenvalue 1 + eta of R goes to 1 + O(eta^3); the cubic step
  // R + 1/2 R E leaves 1 - 3/2 eta^2, a one-sided bias that adds up over the
  // d eigenvalues in the trace when eta is at the FP16 level (single-plane
  // stage-1 iterates).  E comes from an FP64-grade product; E^2 and R W,
  // both small corrections, from FP16 products.  Residual -> red[0..1].
  auto polish = [&]() -> cudaError_t {
    cudaError_t r;
    if (!c.ok(r = split_rows(in.R64, dp, Rs, st))) return r;
    // R^2 to ~1e-9 absolute suffices for the polish: 6 levels (30 bits of the
    // off-diagonal part, the diagonal exact)
    if (!c.ok(r = ozaki_gemm(Rs, Rs, dp, d, 1, N64, status, c.num_sms, st,
                             levels_for(g_levels_polish, in.tol, d, in.k), tz_sym)))
      return r;
    if (!c.ok(r = ident_minus(N64, dp, d, C32, bmax, part, st))) return r;
    if (!c.ok(r = sum_partials(part, ntile, red + 0, st))) return r;
    if (!c.ok(r = max_pow2(bmax, ntile, fs + 0, st))) return r;
    if (!c.ok(r = scale_to_lp(C32, dd, fs + 1, Clp, 0, st))) return r;        // sigma E
    if (!c.ok(r = tc(Clp, Clp, 0, 1, TC_EPI_STORE_F32, P32))) return r;        // (sigma E)^2
    if (!c.ok(r = polish_weight(C32, P32, dd, fs + 1, Clp, st))) return r;     // sigma W
    if (!c.ok(r = to_f16(in.R64, dd, Rlp, st))) return r;
    if (!c.ok(r = tc(Rlp, Clp, 0, 1, TC_EPI_STORE_F32, P32))) return r;        // sigma R W
    if (!c.ok(r = polish_update(in.R64, P32, dp, fs + 1, st))) return r;
    o->polish_steps++;
    return cudaSuccess;
  };

  // No polish before the first sweep: the stage-1 result is an involution to
  // the split trajectory's floor, and the sweep's own polish step follows the
  // correction (measured: the same error after one sweep with or without it).
  RS_TRY(c.ok(split_rows(in.A64, dp, As, st)) ? cudaSuccess : c.err);
  RS_TRY(c.ok(max_f64(As.sigma, dp, red + 16, st)) ? cudaSuccess : c.err);  // s_A
  double h_red[24];
  if (in.M == 0) {
    // X_0 was already at the low-precision floor (A a scaled near-involution):
    // there is no trajectory to differentiate; the polish alone finishes R.
    RS_TRY(polish());
    RS_TRY(polish());
    RS_TRY(cudaMemcpyAsync(h_red, red, sizeof(h_red), cudaMemcpyDeviceToHost, st));
    RS_TRY(cudaStreamSynchronize(st));
    o->resid = h_red[1];
    o->converged = h_red[1] <= in.tol;
    return cudaSuccess;
  }
  // A-posteriori stop test.  The error of the current R is the correction the
  // next sweep would add, F = L_sign(A, G).  Its 2-norm is estimated as
  // kappa * ||alpha G||_2 with kappa = ||E||_2 / ||E_0||_2 measured on the
  // previous tangent solve (the gain of L_sign on the error directions),
  // times a safety factor of 1.5 (measured: the unscaled estimate exceeds the
  // true error by 1.2x to 3x at errors of 1e-7 .. 1e-6).  ||G||_2 is taken
  // matrix free: to first order G = 1/2 R C, and C v = R (A v) - A (R v) needs
  // only FP64 matrix-vector products, so a passed test costs a few GEMV sweeps
  // over A and R instead of an FP64-grade matrix product.
  float *pv = nullptr, *pw = nullptr;
  RS_TRY(mem.alloc((void**)&pv, (size_t)dp * 4));
  RS_TRY(mem.alloc((void**)&pw, (size_t)dp * 4));
  // side stream for the 2-norm estimates of the tangent solve; joined before
  // every readback, and synchronised before the workspace can be released
  struct Side {
    cudaStream_t s = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    ~Side() {
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
      for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    }
  } side;
  RS_TRY(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
  for (int q = 0; q < 3; ++q) RS_TRY(cudaEventCreateWithFlags(&side.ev[q], cudaEventDisableTiming));
  constexpr int kPowerIters = 16;
  // power steps of the check: ||C v|| after 8 steps lies within 1 % of the
  // value after 40 on the controlled spectrum (d = 8192) and the Allen-Cahn
  // Hessian (d = 4096, k = 1, 4), after one and after two sweeps (6 steps:
  // up to 7 % low); the ||R^2 - I|| steps, which enter the bound only, are up
  // to 16 % low after 8
  constexpr int kCheckIters = 8;
  double* cwork = nullptr;
  float *cfwork = nullptr, *A_hi = nullptr, *A_lo = nullptr, *R_hi = nullptr, *R_lo = nullptr;
  RS_TRY(mem.alloc((void**)&cwork, (size_t)12 * dp * 8));
  RS_TRY(mem.alloc((void**)&cfwork, (size_t)12 * dp * 4));
  float2* cpart = nullptr;
  RS_TRY(mem.alloc((void**)&cpart, gemv_df_sym_part_bytes(dp)));
  RS_TRY(mem.alloc((void**)&A_hi, dd * 4));
  RS_TRY(mem.alloc((void**)&A_lo, dd * 4));
  RS_TRY(mem.alloc((void**)&R_hi, dd * 4));
  RS_TRY(mem.alloc((void**)&R_lo, dd * 4));
  // operand of the checks: A 2^kA, 2^kA ~ alpha ~ 1/||A|| (results scaled back)
  const int kA = std::ilogb(in.alpha);
  RS_TRY(c.ok(split_f32(in.A64, dd, A_hi, A_lo, kA, nullptr, st)) ? cudaSuccess : c.err);
  // Operands of the tangent solve, always FP16 (11-bit significands): the
  // stored FP16 iterates themselves (their hi planes), or, for BF16 stage-1
  // iterates, FP16 copies of hi + lo made once here.  The BF16 tangent solve
  // (8-bit significands) stopped contracting once the margin fell to ~2e-4
  // of ||H||; its relative error there is ~u / (scaled margin).
  std::vector<void*> X_t(in.X, in.X + in.M), Et_t(in.Et, in.Et + in.M);
  if (in.fmt == 1 && in.M_tangent > 0) {
    std::vector<const void*> src;
    std::vector<void*> dst;
    for (int m = 0; m < in.M_tangent; ++m) {
      void *xc = nullptr, *ec = nullptr;
      RS_TRY(mem.alloc(&xc, dd * 2));
      RS_TRY(mem.alloc(&ec, dd * 2));
      src.push_back(in.X[m]);
      dst.push_back(xc);
      src.push_back(in.Et[m]);
      dst.push_back(ec);
      X_t[m] = xc;
      Et_t[m] = ec;
    }
    // all of them in one launch (64 matrices per launch)
    RS_TRY(c.ok(bf16_pairs_to_f16(src.data(), dst.data(), (int)src.size(), dd, in.pairs ? 1 : 0, st)) ? cudaSuccess
                                                                                                    : c.err);
    c.launches += ((int)src.size() + 63) / 64 - 1;  // c.ok counted one
  }
  double kappa = NAN;
  for (int sw = 0; sw <= in.max_sweeps; ++sw) {
    if (sw >= 1) {
      // a-posteriori check of the current R (matrix free, FP64 GEMVs):
      // err ~ 1.5 kappa alpha ||G||_2 with kappa the gain of the last tangent solve
      if (!c.ok(commutator_gain_norm(A_hi, A_lo, in.R64, R_hi, R_lo, dp, d, kCheckIters, cwork, cfwork, cpart,
                                     red + 9, st)))
        return c.err;
      c.launches += commutator_check_launches(dp, kCheckIters) - 1;  // c.ok counted one
      RS_TRY(cudaMemcpyAsync(h_red, red, sizeof(h_red), cudaMemcpyDeviceToHost, st));
      RS_TRY(cudaStreamSynchronize(st));
      const double g2 = std::ldexp(h_red[9], -kA);
      o->comm = 2.0 * g2;  // ||R A - A R||_2 = 2 ||G||_2 for an orthogonal R
      o->rho = h_red[10];
      const bool mu_known = std::isfinite(in.margin) && in.margin > 0.0;
      // Estimate: the larger of two gains applied to the commutator.  kappa,
      // the gain ||E||_2 / ||E_0||_2 of the last tangent solve, follows the
      // previous error's directions; the Rayleigh-Ritz gap g of A on the
      // dominant plane of C (the 2 x 2 projection from the check) gives the
      // gain 1/g of the component that dominates C now: a single error
      // component F between eigenpairs i, j has ||C||_2 = |lam_i - lam_j| ||F||_2.
      // The second catches errors that the last solve left between
      // eigenvalues next to the gap (clustered spectra).
      const double a11 = std::ldexp(h_red[11], -kA), a12 = std::ldexp(h_red[12], -kA),
                   a22 = std::ldexp(h_red[13], -kA);
      double g_rr = std::sqrt((a11 - a22) * (a11 - a22) + 4.0 * a12 * a12);
      if (mu_known) g_rr = std::max(g_rr, 2.0 * in.margin);
      const double est_rr = g_rr > 0.0 ? o->comm / g_rr : INFINITY;
      // The two gains are estimates, not bounds: over the controlled-spectrum
      // sweep (d = 1024 .. 16384, k in {1, 16, d/2}, half-gap 1e-3 .. 1e-1,
      // shifts at 10/50/90 % of the gap) and the 512-matrix batch, the true
      // error reached up to 2.1 times the unscaled maximum (and exceeded the
      // tolerance once, 1.6e-6, under BF16_REFINE), so the estimate carries a
      // factor kEstSafety = 2.5 on both terms.
      o->err_est = kEstSafety * std::max(1.5 * kappa * in.alpha * g2, est_rr);
      // With a known margin mu the error is bounded outright (Sylvester
      // argument): F = R - sign(A) has its blocks between the two eigenspaces
      // of A bounded by ||C||_2 / (2 mu) and its blocks within them by
      // (||R^2 - I||_2 + ||F||^2) / 2, so ||F||_2 <= 1 - sqrt(1 - 2c) with
      // c = ||C||_2 / (2 mu) + ||R^2 - I||_2 / 2, both 2-norms from the power
      // steps of the check.
      if (mu_known) {
        const double cb = o->comm / (2.0 * in.margin) + 0.5 * o->rho;
        o->err_bound = 2.0 * cb < 1.0 ? 2.0 * cb / (1.0 + std::sqrt(1.0 - 2.0 * cb)) : INFINITY;
      }
      const bool stop = in.stop_on_bound ? (mu_known && o->err_bound <= in.tol) : o->err_est <= in.tol;
      if (!(g2 > 0.0) || stop) {
        o->converged = true;
        break;
      }
      if (sw == in.max_sweeps) break;
    }
    // commutator C = R A - A R from the FP64-grade product N = R A
    if (!c.ok(split_rows(in.R64, dp, Rs, st))) return c.err;
    // the first sweep's levels from the truncation model; later sweeps use all 7
    int lev = g_levels_ra;
    if (sw == 0) {
      lev = g_levels_ra0;
      if (lev <= 0) {
        if (!c.ok(max_f64(Rs.sigma, dp, red + 18, st))) return c.err;  // s_R
        RS_TRY(cudaMemcpyAsync(h_red + 16, red + 16, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
        RS_TRY(cudaStreamSynchronize(st));
        lev = levels_ra0(in.tol, h_red[16], h_red[18], d, in.mu_lb);
      }
    }
    o->levels_ra0 = sw == 0 ? lev : o->levels_ra0;
    if (!c.ok(ozaki_gemm(Rs, As, dp, d, 0, N64, status, c.num_sms, st, lev, tz_full))) return c.err;
    // C in the units of alpha A (2^kA ~ alpha, exact): the FP32 copy and the
    // direction's factor alpha 2^-kA in [1, 2) stay in range for any scale of H
    if (!c.ok(antisym_part(N64, dp, kA, C32, bmax, part, st))) return c.err;
    if (!c.ok(sum_partials(part, ntile, red + 4, st))) return c.err;
    if (!c.ok(max_pow2(bmax, ntile, fs + 2, st))) return c.err;
    if (!c.ok(scale_to_lp(C32, dd, fs + 3, Clp, 0, st))) return c.err;
    if (!c.ok(to_f16(in.R64, dd, Rlp, st))) return c.err;
    // P = R C_lp^T = -sigma_C R C;  E_0 = alpha/4 (R C + (R C)^T)
    if (!c.ok(tc(Rlp, Clp, 0, 0, TC_EPI_STORE_F32, P32))) return c.err;
    if (!c.ok(newton_direction(P32, dp, fs + 3, std::ldexp(in.alpha, -kA), E32, bmax, st))) return c.err;
    if (!c.ok(max_pow2(bmax, ntile, fs + 4, st))) return c.err;
    // ||E_0||_2 on the side stream, beside the tangent products (tensor-bound,
    // with HBM and SM slots to spare): a copy first, since the tangent steps
    // update E in place
    RS_TRY(cudaMemcpyAsync(Q32, E32, dd * 4, cudaMemcpyDeviceToDevice, st));
    RS_TRY(cudaEventRecord(side.ev[0], st));
    RS_TRY(cudaStreamWaitEvent(side.s, side.ev[0], 0));
    if (!c.ok(spectral_norm_f32(Q32, dp, pv, pw, kPowerIters, red + 6, side.s))) return c.err;  // ||E_0||_2
    c.launches += spectral_norm_launches(dp, kPowerIters) - 1;
    // tangent recursion along the stored iterates.  The operand scale sigma
    // (fs[5], a power of two with |E_0| sigma <= 1) stays fixed along the
    // recursion: E grows by at most ~2.6 per step, well inside the FP16 range
    // (FP16's relative precision does not depend on the scale), so each
    // step's epilogue writes the next step's operand directly.
    if (!c.ok(scale_to_lp(E32, dd, fs + 5, Elp, 0, st))) return c.err;
    for (int m = 0; m < in.M_tangent; ++m) {
      if (!c.ok(tc(Elp, Et_t[m], 0, 0, TC_EPI_STORE_F32, P32))) return c.err;   // E Et
      if (!c.ok(tc(X_t[m], Elp, 0, 0, TC_EPI_STORE_LP, Qlp))) return c.err;     // X E
      // (X E) X with the tangent step fused into its epilogue (E updated in place)
      TcGemmArgs tg{};
      tg.dp = dp; tg.d_real = d; tg.sym = 1; tg.epi = TC_EPI_TANGENT; tg.n_groups = 1;
      tg.group_start[0] = 0; tg.group_start[1] = 1; tg.pair_a[0] = 0; tg.pair_b[0] = 0;
      tg.group_scale[0] = 1.0; tg.scale = 1.0f; tg.status = status;
      tg.tg_E = E32; tg.tg_P = P32; tg.tg_sigma = fs + 5; tg.tg_max = bmax;
      tg.tg_a = (in.a != nullptr && m < in.n_a) ? (float)in.a[m] : 1.0f;
      tg.tg_Elp = (m + 1 < in.M_tangent) ? Elp : nullptr;
      if (!c.ok(tc_gemm(tg, Qlp, 1, X_t[m], 1, 0, c.num_sms, st))) return c.err;
    }
    // ||E||_2 on the side stream (after ||E_0||_2 there), beside the
    // correction and the polish, which only read E
    RS_TRY(cudaEventRecord(side.ev[1], st));
    RS_TRY(cudaStreamWaitEvent(side.s, side.ev[1], 0));
    if (!c.ok(spectral_norm_f32(E32, dp, pv, pw, kPowerIters, red + 7, side.s))) return c.err;
    RS_TRY(cudaEventRecord(side.ev[2], side.s));
    c.launches += spectral_norm_launches(dp, kPowerIters) - 1;
    if (!c.ok(add_correction(in.R64, E32, dp, d, part, st))) return c.err;
    if (!c.ok(sum_partials(part, 1024, red + 2, st))) return c.err;
    RS_TRY(polish());
    RS_TRY(cudaStreamWaitEvent(st, side.ev[2], 0));  // join before E and red are reused
    RS_TRY(cudaMemcpyAsync(h_red, red, sizeof(h_red), cudaMemcpyDeviceToHost, st));
    RS_TRY(cudaStreamSynchronize(st));
    o->sweeps = sw + 1;
    o->resid = h_red[1];
    o->corr = h_red[3];
    kappa = (h_red[6] > 0.0) ? h_red[7] / h_red[6] : 1.0;  // gain ||E||_2 / ||E_0||_2 of this solve
  }
#undef RS_TRY
  return cudaSuccess;
}

rsign_status reflector_impl(const double* H, int64_t d64, int32_t k, double s, double tol,
                            rsign_policy policy, const rsign_options* opt_in, double* R,
                            rsign_info* info, cudaStream_t st) {
  rsign_options opt;
  rsign_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (!H || !R) return RSIGN_ERR_ARG;
  if (d64 < 2 || d64 > 16384) return d64 > 16384 ? RSIGN_ERR_UNSUPPORTED : RSIGN_ERR_ARG;
  if (k < 1 || k > d64 - 1) return RSIGN_ERR_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol)) return RSIGN_ERR_ARG;
  if ((int)policy < RSIGN_FP64 || (int)policy > RSIGN_FP32) return RSIGN_ERR_ARG;
  if (opt.max_steps < 1 || opt.max_steps > 1000 || opt.polish_steps < 0 || opt.max_sweeps < 0)
    return RSIGN_ERR_ARG;
  if (!std::isnan(opt.margin) && !(opt.margin > 0.0 && std::isfinite(opt.margin))) return RSIGN_ERR_ARG;
  if (std::isinf(s)) return RSIGN_ERR_ARG;
  const bool auto_shift = std::isnan(s);
  const bool refine = policy == RSIGN_FP16_REFINE || policy == RSIGN_BF16_REFINE;
  if (opt.refine_stop != RSIGN_STOP_ESTIMATE && opt.refine_stop != RSIGN_STOP_BOUND) return RSIGN_ERR_ARG;
  if (opt.engine != RSIGN_ENGINE_NS3 && opt.engine != RSIGN_ENGINE_NS5) return RSIGN_ERR_ARG;
  const bool ns5 = opt.engine == RSIGN_ENGINE_NS5;
  if (ns5 && refine) return RSIGN_ERR_ARG;  // the tangent recursion differentiates Eq. NS
  if (refine && opt.refine_stop == RSIGN_STOP_BOUND && !auto_shift && std::isnan(opt.margin)) return RSIGN_ERR_ARG;

  Ctx c;
  c.st = st;
  rsign_status dst = (rsign_status)check_device(&c.num_sms);
  if (dst != RSIGN_OK) return dst;

  const int d = (int)d64;
  const int dp = (d + 255) / 256 * 256;
  const size_t dd = (size_t)dp * dp;
  const double eps64 = 2.220446049250313e-16;
  const double tol_fro = std::max(tol, 16.0 * d * eps64);

  DevBuf mem;
  mem.st = st;
  rsign_status result = RSIGN_OK;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  Ctl ctl_h;
  std::memset(&ctl_h, 0, sizeof(ctl_h));
  int steps_low = 0, steps64 = 0, sweeps_done = 0;
  double corr_fro = NAN, comm_norm = NAN, err_est = NAN, err_bound = NAN;
  int refine_levels = 0;
  bool conv64 = true;
  double resid = NAN;
  std::vector<double> hist_h;

  auto fail_cuda = [&]() {
    mem.release();
    cudaStreamSynchronize(st);
    cudaGetLastError();
    for (auto& e : ev) if (e) cudaEventDestroy(e);
    return RSIGN_ERR_CUDA;
  };

  if (opt.timing)
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail_cuda();
  if (opt.timing) cudaEventRecord(ev[0], st);

  // ---- buffers
  const bool h_dev = is_device_ptr(H), r_dev = is_device_ptr(R);
  double *Hd = const_cast<double*>(H), *Rd = R;
  Ctl* ctl = nullptr;
  double *A64 = nullptr, *rowpart = nullptr, *rowsum = nullptr, *partials = nullptr, *hist = nullptr;
  const int n_part = std::max(tc_num_tiles(dp, 1), f64_num_tiles(dp, 1)) * 4;
  const int hist_len = 2 * (opt.max_steps + 2);
  if (mem.alloc((void**)&ctl, sizeof(Ctl)) != cudaSuccess ||
      mem.alloc((void**)&A64, dd * 8) != cudaSuccess ||
      mem.alloc((void**)&rowpart, (size_t)(dp / 32) * dp * 8) != cudaSuccess ||
      mem.alloc((void**)&rowsum, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&partials, (size_t)n_part * 8) != cudaSuccess ||
      mem.alloc((void**)&hist, (size_t)hist_len * 8) != cudaSuccess)
    return fail_cuda();
  // host buffers go through staging copies on the copy engines; with
  // g_host_mapped, page-locked ones are read and written in place by the
  // ingest and output kernels instead
  const double* h_map = (h_dev || !g_host_mapped) ? nullptr : static_cast<const double*>(mapped_host_ptr(H));
  double* r_map =
      (r_dev || !g_host_mapped) ? nullptr : const_cast<double*>(static_cast<const double*>(mapped_host_ptr(R)));
  if (!h_dev) {
    if (h_map) {
      Hd = const_cast<double*>(h_map);
    } else {
      if (mem.alloc((void**)&Hd, (size_t)d * d * 8) != cudaSuccess) return fail_cuda();
      if (staged_copy(Hd, H, (size_t)d * d * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail_cuda();
    }
  }
  if (r_map) Rd = r_map;
  else if (!r_dev && mem.alloc((void**)&Rd, (size_t)d * d * 8) != cudaSuccess) return fail_cuda();
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) != cudaSuccess) return fail_cuda();
  double* hist_low = hist;
  double* hist64 = hist + opt.max_steps + 2;

  // ---- automatic shift (Sec. 4.3): Lanczos endpoint estimates of lam_k and
  // lam_{k+1}, the midpoint (Prop. 4.1), and the margin test m_hat > eps of
  // Prop. 4.2 (the shift is then admissible with true margin >= m_hat - eps)
  LanczosResult lr{};
  double margin_lb = NAN;
  auto fill_shift_info = [&](rsign_info* inf) {
    if (!inf || !auto_shift) return;
    inf->lam_k_est = lr.lam_k;
    inf->lam_k1_est = lr.lam_k1;
    inf->shift_eps = std::max(lr.eps_k, lr.eps_k1);
    inf->margin_lb = margin_lb;
    inf->lanczos_iters = lr.iters;
  };
  if (auto_shift) {
    if (!c.ok(ingest(Hd, d, dp, 0.0, A64, rowpart, &ctl->flags, st))) return fail_cuda();
    const int lmax = opt.lanczos_max > 0 ? opt.lanczos_max : 600;
    double* lw = nullptr;
    if (mem.alloc((void**)&lw, lanczos_work_doubles(dp, lmax) * 8) != cudaSuccess) return fail_cuda();
    if (lanczos_endpoints(A64, dp, d, k, lmax, lw, &lr, &c.launches, st) != cudaSuccess) return fail_cuda();
    if (cudaMemcpyAsync(&ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail_cuda();
    const double eps = std::max(lr.eps_k, lr.eps_k1);
    const double m_hat = 0.5 * (lr.lam_k1 - lr.lam_k);
    s = 0.5 * (lr.lam_k + lr.lam_k1);
    margin_lb = m_hat - eps;
    if ((ctl_h.flags & 1) || !std::isfinite(s) || !(m_hat > eps)) {
      if (info) {
        std::memset(info, 0, sizeof(*info));
        info->shift = s;
        info->steps_pred = -1;
        fill_shift_info(info);
      }
      mem.release();
      cudaStreamSynchronize(st);
      for (auto& e : ev) if (e) cudaEventDestroy(e);
      return (ctl_h.flags & 1) ? RSIGN_ERR_ARG : RSIGN_ERR_GAP;
    }
  }

  // ---- ingest and scaling (Sec. 4.3: alpha = 1/||H - sI||_inf)
  if (!c.ok(ingest(Hd, d, dp, s, A64, rowpart, &ctl->flags, st))) return fail_cuda();
  if (!c.ok(inf_norm_finish(rowpart, dp, rowsum, ctl->scal, st))) return fail_cuda();
  ++c.launches;  // inf_norm_finish issues two kernels
  if (opt.alpha_mode == RSIGN_ALPHA_POWER) {
    // alpha = 1/(1.02 rho_est) from power steps on A (overwrites the Gershgorin
    // value); an estimate within a few percent is all it needs, so the steps
    // run on an FP32 copy of A: half the bytes and the FP32 pipe (FP64 FMAs
    // would bound the GEMV on this GPU)
    float *a32 = nullptr, *pv = nullptr, *pw = nullptr;
    if (mem.alloc((void**)&a32, dd * 4) != cudaSuccess || mem.alloc((void**)&pv, (size_t)dp * 4) != cudaSuccess ||
        mem.alloc((void**)&pw, (size_t)dp * 4) != cudaSuccess)
      return fail_cuda();
    const int ps = std::max(1, opt.power_steps);
    // (A scaled by 2^k, 2^k the Gershgorin alpha's power of two, so that any
    // scale of H stays inside the float range)
    if (!c.ok(split_f32(A64, dd, a32, nullptr, 0, ctl->scal + 1, st)) ||
        !c.ok(spectral_norm_f32(a32, dp, pv, pw, ps, ctl->scal + 4, st)) ||
        !c.ok(alpha_from_rho(ctl->scal + 4, 1.02, ctl->scal, 1, st)))
      return fail_cuda();
    c.launches += spectral_norm_launches(dp, ps) - 1;  // c.ok counted one per helper
  }
  if (cudaMemcpyAsync(&ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail_cuda();
  if (ctl_h.flags & 1) {
    mem.release();
    cudaStreamSynchronize(st);
    for (auto& e : ev) if (e) cudaEventDestroy(e);
    return RSIGN_ERR_ARG;
  }
  const double alpha = ctl_h.scal[1];
  if (!(alpha > 0.0) || !std::isfinite(alpha)) {
    mem.release();
    cudaStreamSynchronize(st);
    for (auto& e : ev) if (e) cudaEventDestroy(e);
    return RSIGN_ERR_ARG;  // H - sI == 0
  }

  // ---- scaled Newton-Schulz steps (Sec. 3.5: the stable step scalings of the
  // cited GPU sign iteration) when a lower bound of the spectral margin is
  // known -- the caller's opt.margin or the certified margin of the automatic
  // shift: for the spectrum of X in [-1, -l] U [l, 1] the step
  // X <- 1/2 a X (3I - a^2 X^2), a = sqrt(3 / (1 + l + l^2)), maps [l, 1] into
  // [l', 1] with l' = 1/2 a l (3 - a^2 l^2), about 2.6 l for small l (1.5 l
  // for the plain step).  The upper end is 1 for the Gershgorin alpha; for
  // the power-step alpha, whose rho estimate is not a certified bound, the
  // first factor is divided by 1.04 (a rho estimate down to 0.94 rho stays
  // sign-safe; below that the trace certificate fails and the call is redone
  // with the Gershgorin alpha).
  std::vector<double> coef;
  {
    const double mk = auto_shift ? margin_lb : opt.margin;
    if (opt.ns_scaling && !ns5 && std::isfinite(mk) && mk > 0.0)
      coef = scaled_ns_coeffs(alpha * mk, opt.alpha_mode == RSIGN_ALPHA_POWER ? 1.04 : 1.0);
  }

  // Known lower end l_m of the spectrum of X_m, when a margin is known
  std::vector<double> lower_end;
  {
    const double mk = auto_shift ? margin_lb : opt.margin;
    if (std::isfinite(mk) && mk > 0.0)
      lower_end = lower_end_sequence(alpha * mk, opt.alpha_mode == RSIGN_ALPHA_POWER ? 1.04 : 1.0, coef,
                                     opt.max_steps);
  }

  double* Rfinal = nullptr;  // dp x dp FP64 result
  double* xb64[2] = {nullptr, nullptr};
  double* E64 = nullptr;
  double* W64 = nullptr;  // NS5 engine, FP64 policy
  const bool need64 = policy == RSIGN_FP64 || policy == RSIGN_FP16_POLISH || policy == RSIGN_BF16_POLISH;
  if (ns5 && policy == RSIGN_FP64 && mem.alloc((void**)&W64, dd * 8) != cudaSuccess) return fail_cuda();
  if (mem.alloc((void**)&xb64[0], dd * 8) != cudaSuccess) return fail_cuda();
  if (need64 && (mem.alloc((void**)&xb64[1], dd * 8) != cudaSuccess ||
                 mem.alloc((void**)&E64, dd * 8) != cudaSuccess))
    return fail_cuda();

  if (opt.timing) cudaEventRecord(ev[1], st);
  if (is_low(policy)) {
    // ---------------------------------------------- low-precision stage (tcgen05)
    const int fmt = lp_fmt_of(policy);
    // Iterates X_m and E_m = I - X_m^2: two ping-pong slots, or (refinement)
    // one slot per step, kept for the tangent recursion.  For refinement the
    // iterates are carried as hi/lo pairs of planes (X = X_hi + X_lo, about
    // twice the bits of the operand type): every product is the fused sum of
    // the pair products hi*hi + hi*lo + lo*hi, so the stored trajectory is an
    // accurate one and its derivative (the tangent recursion) is accurate too.
    const bool split = (refine && opt.low_split != 0) || policy == RSIGN_FP32;
    const int planes = split ? 2 : 1;
    std::vector<void*> xs, es;
    auto slot_x = [&](int m) -> void* {
      const int idx = refine ? m : (m & 1);
      while ((int)xs.size() <= idx) {
        void* p = nullptr;
        if (mem.alloc(&p, dd * 2 * planes) != cudaSuccess) return nullptr;
        xs.push_back(p);
      }
      return xs[idx];
    };
    auto slot_e = [&](int m) -> void* {
      const int idx = refine ? m : 0;
      while ((int)es.size() <= idx) {
        void* p = nullptr;
        if (mem.alloc(&p, dd * 2 * planes) != cudaSuccess) return nullptr;
        es.push_back(p);
      }
      return es[idx];
    };
    if (!slot_x(0)) return fail_cuda();
    if (split) {
      if (!c.ok(scale_convert_split(A64, dd, ctl->scal + 1, slot_x(0), fmt, st))) return fail_cuda();
    } else {
      if (!c.ok(scale_convert(A64, dd, ctl->scal + 1, 1.0, slot_x(0), fmt, st))) return fail_cuda();
    }
    // the split trajectory reaches a floor near u^2 (FP32 accumulation)
    const double u = split ? 4.0 * unit_roundoff(fmt) * unit_roundoff(fmt) : unit_roundoff(fmt);
    const double floor_lo = 2.0 * u * std::sqrt((double)d);
    const double floor_hi = 16.0 * u * std::sqrt((double)d);
    const int nt = tc_num_tiles(dp, 1);
    // With the scaled steps the floor tests wait until the recurrence of
    // the interval's bottom end has come within u of 1: before that a small
    // residual is no sign of convergence.
    int m_min = 0;
    {
      double l = std::min(1.0, alpha * (auto_shift ? margin_lb : opt.margin));
      for (size_t q = 0; q < coef.size() && 1.0 - l > u; ++q) {
        l = 0.5 * coef[q] * l * (3.0 - coef[q] * coef[q] * l * l);
        m_min = (int)q + 1;
      }
    }
    // trace guard of the floor tests: the trace of the iterate (from the
    // update epilogue, in its own partials) within 1/2 + 2 u sqrt(d) of d - 2k
    double* tr_part = nullptr;
    if (mem.alloc((void**)&tr_part, (size_t)nt * 4 * 8) != cudaSuccess) return fail_cuda();
    const double tr_tol = 0.5 + 2.0 * u * std::sqrt((double)d);
    void* wlp = nullptr;  // NS5 engine: W = E + 3/4 E^2
    if (ns5 && mem.alloc(&wlp, dd * 2 * planes) != cudaSuccess) return fail_cuda();
    // exact squared row norms of each iterate for the SYRK's diagonal above
    // d = 1024 (kExactDiagMin): below, the tensor cores' accumulation bias moves
    // the trace by less than 3e-3 (and the grouped launches of the batched
    // calls, d <= 1024, stay bitwise equal to one-matrix calls)
    float* rowsq = nullptr;
    if (d > kExactDiagMin && mem.alloc((void**)&rowsq, (size_t)dp * 4) != cudaSuccess) return fail_cuda();
    // iterate X_m as a hi/lo pair (refinement: the leading n_split only),
    // and the floors of the stop test for its format
    int n_split = -1;  // -1: every iterate
    if (refine && g_split_steps >= 0) {
      n_split = g_split_steps;
    } else if (refine && g_split_steps == -2 && fmt == 0 && !lower_end.empty()) {
      // FP16 only: a single BF16 plane (8-bit significand) leaves a floor,
      // u sqrt(d) ~ 0.35 at d = 8192, that the trace guard of the stop test
      // never passes (measured: stage 1 ran to its step limit)
      int mt_unused = 0;
      refine_stage_plan(lower_end, opt.max_steps, &n_split, &mt_unused);
    }
    auto x_split = [&](int mi) { return split && (!refine || n_split < 0 || mi < n_split); };
    const double u1 = unit_roundoff(fmt);
    int m = 0;
    bool stopped = false;
    while (m <= opt.max_steps && !stopped) {
      const int chunk = m == 0 ? std::max(kChunk, m_min + 3) : kChunkLate;
      const int m_end = std::min(m + chunk, opt.max_steps + 1);
      for (int mm = m; mm < m_end; ++mm) {
        void* xm = slot_x(mm);
        void* em = slot_e(mm);
        void* xn = (mm < opt.max_steps) ? slot_x(mm + 1) : xm;
        if (!xm || !em || !xn) return fail_cuda();
        const bool sp = x_split(mm);
        const double um = sp ? u : u1;
        TcGemmArgs sy{};
        sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = TC_EPI_NS_SYRK; sy.n_groups = 1;
        sy.group_start[0] = 0; sy.pair_a[0] = 0; sy.pair_b[0] = 0;
        if (sp) {  // hi*hi + hi*lo + lo*hi in one accumulator
          sy.pair_a[1] = 0; sy.pair_b[1] = 1; sy.pair_a[2] = 1; sy.pair_b[2] = 0;
          sy.group_start[1] = 3;
        } else {
          sy.group_start[1] = 1;
        }
        sy.split = sp ? 1 : 0;
        sy.group_scale[0] = 1.0; sy.scale = 1.0f; sy.out = em; sy.partials = partials;
        sy.status = &ctl->status; sy.skip = &ctl->done_low;
        const double am = mm < (int)coef.size() ? coef[mm] : 1.0;
        sy.ns_c2 = (float)(am * am);
        sy.ns_c1 = (float)am;
        sy.ns_diag = rowsq;
        if (rowsq && !c.ok(row_sumsq(xm, fmt, sp ? 1 : 0, dp, d, rowsq, &ctl->done_low, st))) return fail_cuda();
        if (!c.ok(tc_gemm(sy, xm, planes, xm, planes, fmt, c.num_sms, st))) return fail_cuda();
        const bool floors = mm >= m_min;
        const double fl_lo = sp ? floor_lo : 2.0 * um * std::sqrt((double)d);
        const double fl_hi = sp ? floor_hi : 16.0 * um * std::sqrt((double)d);
        const double tr_tol_m = sp ? tr_tol : 0.5 + 2.0 * um * std::sqrt((double)d);
        if (!c.ok(ns_check(partials, nt * 4, hist_low, mm, 0.0, floors ? fl_lo : -1.0, floors ? fl_hi : -1.0,
                           0.5, &ctl->done_low, &ctl->steps_low, st, mm >= 1 ? tr_part : nullptr, nt * 4,
                           (double)(d - 2 * k), tr_tol_m)))
          return fail_cuda();
        if (mm == opt.max_steps) break;
        void* bm = em;
        if (ns5) {
          // W = E + 3/4 E^2 (update epilogue, scale 3/2 on E E), then X+ = X + 1/2 X W
          TcGemmArgs w = sy;
          w.epi = TC_EPI_NS_UPDATE; w.out = wlp; w.xin = em; w.partials = partials; w.scale = 1.5f;
          w.ns_c1 = 0.0f; w.ns_diag = nullptr;
          if (!c.ok(tc_gemm(w, em, planes, em, planes, fmt, c.num_sms, st))) return fail_cuda();
          bm = wlp;
        }
        TcGemmArgs up = sy;
        up.epi = TC_EPI_NS_UPDATE; up.out = xn; up.xin = xm; up.partials = tr_part;
        // single-plane steps of a split policy still store the lo plane of
        // their result: the next step reads the hi plane only, but the
        // iterate the stage ends on keeps its FP32 value (an FP16 rounding of
        // the last iterate would leave noise ~u16 inside the eigenspaces,
        // which the polish's FP16 products can only reduce to ~u16^2)
        up.single_out = 0;
        up.pair_out = (split && !sp) ? 1 : 0;
        if (!c.ok(tc_gemm(up, xm, planes, bm, planes, fmt, c.num_sms, st))) return fail_cuda();
      }
      if (cudaMemcpyAsync(&ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail_cuda();
      if (ctl_h.status != 0) break;
      stopped = ctl_h.done_low != 0;
      m = m_end;
    }
    steps_low = stopped ? ctl_h.steps_low : opt.max_steps;
    if (split) {  // every iterate of a split policy keeps a lo plane (X_0 and the pairs, pair_out after)
      if (!c.ok(split_to_f64(slot_x(steps_low), fmt, dd, xb64[0], st))) return fail_cuda();
    } else {
      if (!c.ok(to_f64(slot_x(steps_low), fmt, dd, xb64[0], st))) return fail_cuda();
    }
    Rfinal = xb64[0];
    hist_h.resize(opt.max_steps + 2);
    if (cudaMemcpyAsync(hist_h.data(), hist_low, hist_h.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail_cuda();
    resid = hist_h[steps_low];
    if (!stopped && ctl_h.status == 0) result = RSIGN_ERR_NOCONV;
    if (opt.timing) cudaEventRecord(ev[2], st);
    if (refine && ctl_h.status == 0 && result == RSIGN_OK) {
      // ------------------------------------------- commutator refinement sweeps
      RefineIn in{};
      in.dp = dp; in.d = d; in.k = k; in.fmt = fmt; in.M = steps_low; in.alpha = alpha; in.tol = tol;
      // Tangent steps at iterates already within kTangentCut of the sign
      // (known lower end l_m >= 1 - kTangentCut) are left out: there the
      // Frechet derivative of the step is the identity on the error's part
      // that anticommutes with the sign (factor (3a - a^3 (x_i^2 + x_i x_j +
      // x_j^2)) / 2 = 1 + O(1 - l_m) for x_i ~ -x_j ~ +-1) and only damps the
      // commuting part, which the polish step removes.
      in.M_tangent = steps_low;
      if (g_tangent_cut && !lower_end.empty()) {
        int ns_unused = 0;
        refine_stage_plan(lower_end, steps_low, &ns_unused, &in.M_tangent);
      }
      in.A64 = A64; in.R64 = xb64[0]; in.X = xs.data(); in.Et = es.data(); in.pairs = split;
      in.a = coef.empty() ? nullptr : coef.data(); in.n_a = (int)coef.size();
      in.max_sweeps = std::max(1, opt.max_sweeps);
      in.margin = auto_shift ? margin_lb : opt.margin;
      in.stop_on_bound = opt.refine_stop == RSIGN_STOP_BOUND;
      in.mu_lb = (std::isfinite(in.margin) && in.margin > 0.0)
                     ? in.margin
                     : (coef.empty() ? gamma_from_steps(steps_low) / alpha : NAN);
      RefineOut ro{};
      const cudaError_t re = refine_sweeps(c, mem, in, ctl, &ro);
      if (re != cudaSuccess) return fail_cuda();
      sweeps_done = ro.sweeps;
      steps64 = ro.polish_steps;
      resid = ro.resid;
      corr_fro = ro.corr;
      comm_norm = ro.comm;
      err_est = ro.err_est;
      err_bound = ro.err_bound;
      refine_levels = ro.levels_ra0;
      if (!ro.converged && result == RSIGN_OK) result = RSIGN_ERR_NOCONV;
    }
  } else {
    if (!c.ok(scale_convert(A64, dd, ctl->scal + 1, 1.0, xb64[0], 2, st))) return fail_cuda();
    if (opt.timing) cudaEventRecord(ev[2], st);
  }

  if (need64 && ctl_h.status == 0) {
    // ------------------------------------------------------------- FP64 stage
    F64Loop L{{xb64[0], xb64[1]}, E64, partials, hist64, &ctl->done64, &ctl->steps64, W64};
    int m_ret = 0;
    const bool polish = policy != RSIGN_FP64;
    if (polish) {
      // FP64 polish on the tensor cores (FP64-emulating digit-plane products)
      if (fp64e_polish(c, mem, xb64, E64, dp, d, opt.polish_steps, partials, hist64, ctl) != cudaSuccess)
        return fail_cuda();
      m_ret = opt.polish_steps;
    } else if (!f64_ns(c, L, dp, d, tol_fro, opt.max_steps, ctl, ctl_h, &m_ret, &conv64, &coef)) {
      return fail_cuda();
    }
    steps64 = m_ret;
    Rfinal = xb64[m_ret & 1];
    hist_h.resize(opt.max_steps + 2);
    if (cudaMemcpyAsync(hist_h.data(), hist64, hist_h.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail_cuda();
    resid = hist_h[m_ret];
    if (!polish && !conv64) result = RSIGN_ERR_NOCONV;
    if (polish) result = RSIGN_OK;  // the polish depth is fixed; the residual is reported
  }

  // ---- certificate and output
  if (!c.ok(trace_f64(Rfinal, dp, d, ctl->scal + 2, st))) return fail_cuda();
  if (!c.ok(copy_unpad(Rfinal, dp, Rd, d, st))) return fail_cuda();
  if (!r_dev && !r_map && staged_copy(R, Rd, (size_t)d * d * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail_cuda();
  if (opt.timing) cudaEventRecord(ev[3], st);
  if (cudaMemcpyAsync(&ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail_cuda();
  const double trace = ctl_h.scal[2];
  const bool trace_ok = std::fabs(trace - (double)(d - 2 * k)) < 0.5;
  const bool resid_ok = policy == RSIGN_FP64 ? (resid <= tol_fro) : true;
  if (ctl_h.status != 0) result = (rsign_status)ctl_h.status;
  else if (!trace_ok) result = RSIGN_ERR_CERT;

  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->steps_low = steps_low;
    info->steps_fp64 = steps64;
    info->sweeps_refine = sweeps_done;
    info->cert_ok = (trace_ok && resid_ok) ? 1 : 0;
    info->alpha = alpha;
    info->shift = s;
    info->gamma_est = auto_shift ? alpha * margin_lb : NAN;
    info->steps_pred = -1;
    info->ns_scaled_steps = (int32_t)coef.size();
    if (auto_shift && info->gamma_est > 0.0) {
      // smallest m with eps_m(gamma) <= tol, eps_0 = 1 - gamma, eps_{m+1} = eps_m^2 (3 - eps_m)/2
      double e = 1.0 - std::min(1.0, info->gamma_est);
      int m = 0;
      while (e > tol && m < 10000) {
        e = 0.5 * e * e * (3.0 - e);
        ++m;
      }
      info->steps_pred = m;
    }
    fill_shift_info(info);
    info->resid_fro = resid;
    info->trace = trace;
    info->correction_fro = corr_fro;
    info->commutator_norm = comm_norm;
    info->err_est = err_est;
    info->err_bound = err_bound;
    info->refine_levels = refine_levels;
    info->tol_fro = tol_fro;
    if (opt.timing) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[0], ev[3]); info->ms_total = t;
      cudaEventElapsedTime(&t, ev[1], ev[2]); info->ms_low = is_low(policy) ? t : 0.0;
      cudaEventElapsedTime(&t, ev[2], ev[3]); info->ms_fp64 = t;
    }
    const double dd3 = (double)d * d * d;
    info->flops_low = is_low(policy) ? dd3 * ((ns5 ? 3.0 : 2.0) * steps_low + 1.0) : 0.0;
    info->launches = c.launches;
    info->workspace_bytes = mem.bytes;
  }
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); result = RSIGN_ERR_CUDA; }
  for (auto& e : ev) if (e) cudaEventDestroy(e);
  return result;
}

// ---------------------------------------------------------------------------
// Adjoint of R = p_M(alpha (H - sI)) (Eq. NS unrolled M times) with s and alpha
// held fixed.  The Frechet derivative of f(X) = 3/2 X - 1/2 X^3 at a symmetric
// X, L_f(X, E) = 3/2 E - 1/2 (E X^2 + X E X + X^2 E), is self-adjoint for the
// Frobenius inner product, so with G_M = sym(Rbar) the backward sweep is
//   G_m = L_f(X_m, G_{m+1}) = 1/2 G + 1/2 (G E_m + E_m G) - 1/2 X_m G X_m,
// E_m = I - X_m^2, and Hbar = alpha sym(G_0) (A = sym(H) - sI).
// FP64 policy: FP64 products; the forward keeps X every `ckpt_every` steps
// and each backward segment recomputes its iterates from its checkpoint.
// Low-precision policies: the stage-1 trajectory (hi/lo for *_REFINE) is kept
// whole and the sweep uses the FP16/BF16 tangent products of the refinement.
// ---------------------------------------------------------------------------
rsign_status backward_impl(const double* H, int64_t d64, int32_t k, double s, rsign_policy policy,
                           const double* Rbar, double* Hbar, int32_t ckpt_every, cudaStream_t st) {
  if (!H || !Rbar || !Hbar) return RSIGN_ERR_ARG;
  if (d64 < 2 || d64 > 16384) return d64 > 16384 ? RSIGN_ERR_UNSUPPORTED : RSIGN_ERR_ARG;
  if (k < 1 || k > d64 - 1 || !std::isfinite(s)) return RSIGN_ERR_ARG;
  if ((int)policy < RSIGN_FP64 || (int)policy > RSIGN_FP32) return RSIGN_ERR_ARG;
  const bool polish = policy == RSIGN_FP16_POLISH || policy == RSIGN_BF16_POLISH;
  const int ck = ckpt_every > 0 ? ckpt_every : 4;
  Ctx c;
  c.st = st;
  rsign_status dst = (rsign_status)check_device(&c.num_sms);
  if (dst != RSIGN_OK) return dst;
  const int d = (int)d64, dp = (d + 255) / 256 * 256;
  const size_t dd = (size_t)dp * dp;
  const int max_steps = 100;
  DevBuf mem;
  mem.st = st;
  auto fail = [&]() {
    mem.release();
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return RSIGN_ERR_CUDA;
  };
  Ctl* ctl = nullptr;
  Ctl h;
  std::memset(&h, 0, sizeof(h));
  double *A64 = nullptr, *rowpart = nullptr, *rowsum = nullptr, *partials = nullptr, *hist = nullptr;
  double *G = nullptr, *Gs = nullptr;
  const int n_part = std::max(tc_num_tiles(dp, 1), f64_num_tiles(dp, 1)) * 4;
  if (mem.alloc((void**)&ctl, sizeof(Ctl)) != cudaSuccess || mem.alloc((void**)&A64, dd * 8) != cudaSuccess ||
      mem.alloc((void**)&rowpart, (size_t)(dp / 32) * dp * 8) != cudaSuccess ||
      mem.alloc((void**)&rowsum, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&partials, (size_t)n_part * 8) != cudaSuccess ||
      mem.alloc((void**)&hist, (size_t)(max_steps + 2) * 8) != cudaSuccess ||
      mem.alloc((void**)&G, dd * 8) != cudaSuccess || mem.alloc((void**)&Gs, dd * 8) != cudaSuccess)
    return fail();
  // inputs may live on the host
  const double *Hd = H, *Rb = Rbar;
  double* Hb = Hbar;
  if (!is_device_ptr(H)) {
    double* t = nullptr;
    if (mem.alloc((void**)&t, (size_t)d * d * 8) != cudaSuccess ||
        cudaMemcpyAsync(t, H, (size_t)d * d * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail();
    Hd = t;
  }
  if (!is_device_ptr(Rbar)) {
    double* t = nullptr;
    if (mem.alloc((void**)&t, (size_t)d * d * 8) != cudaSuccess ||
        cudaMemcpyAsync(t, Rbar, (size_t)d * d * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail();
    Rb = t;
  }
  const bool hb_dev = is_device_ptr(Hbar);
  if (!hb_dev && mem.alloc((void**)&Hb, (size_t)d * d * 8) != cudaSuccess) return fail();
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) != cudaSuccess) return fail();
  if (!c.ok(ingest(Hd, d, dp, s, A64, rowpart, &ctl->flags, st)) ||
      !c.ok(inf_norm_finish(rowpart, dp, rowsum, ctl->scal, st)))
    return fail();
  if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail();
  const double alpha = h.scal[1];
  if ((h.flags & 1) || !(alpha > 0.0)) {
    mem.release();
    cudaStreamSynchronize(st);
    return RSIGN_ERR_ARG;
  }
  // G_M = sym(Rbar), zero padded
  if (!c.ok(copy_pad(Rb, d, Gs, dp, st)) || !c.ok(symmetrize_scale(Gs, dp, 1.0, G, st))) return fail();
  const int nt64 = f64_num_tiles(dp, 1);
  const double tol_fro = 16.0 * d * 2.220446049250313e-16;

  if (policy == RSIGN_FP64) {
    // -------- forward: Newton-Schulz to convergence, checkpoints every ck steps
    double *xb[2] = {nullptr, nullptr}, *E = nullptr;
    if (mem.alloc((void**)&xb[0], dd * 8) != cudaSuccess || mem.alloc((void**)&xb[1], dd * 8) != cudaSuccess ||
        mem.alloc((void**)&E, dd * 8) != cudaSuccess)
      return fail();
    std::vector<double*> ckpt;
    auto checkpoint = [&](int j, const double* src) -> bool {
      while ((int)ckpt.size() <= j) {
        double* p = nullptr;
        if (mem.alloc((void**)&p, dd * 8) != cudaSuccess) return false;
        ckpt.push_back(p);
      }
      return cudaMemcpyAsync(ckpt[j], src, dd * 8, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    };
    if (!c.ok(scale_convert(A64, dd, ctl->scal + 1, 1.0, xb[0], 2, st)) || !checkpoint(0, xb[0])) return fail();
    int M = max_steps;
    for (int m = 0; m <= max_steps; ++m) {
      F64GemmArgs sy{};
      sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = F64_EPI_NS_SYRK;
      sy.A = xb[m & 1]; sy.B = xb[m & 1]; sy.out = E; sy.partials = partials;
      if (!c.ok(f64_gemm(sy, st)) ||
          !c.ok(ns_check(partials, nt64 * 4, hist, m, tol_fro, -1.0, -1.0, 0.0, &ctl->done64, &ctl->steps64, st)))
        return fail();
      if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail();
      if (h.done64 || m == max_steps) {
        M = m;
        break;
      }
      F64GemmArgs up{};
      up.dp = dp; up.d_real = d; up.sym = 1; up.epi = F64_EPI_NS_UPDATE;
      up.A = xb[m & 1]; up.B = E; up.xin = xb[m & 1]; up.out = xb[(m + 1) & 1]; up.partials = partials;
      if (!c.ok(f64_gemm(up, st))) return fail();
      if ((m + 1) % ck == 0 && !checkpoint((m + 1) / ck, xb[(m + 1) & 1])) return fail();
    }
    // -------- backward over segments [c0, c1), iterates recomputed from checkpoints
    std::vector<double*> segX(ck, nullptr), segE(ck, nullptr);
    for (int q = 0; q < ck; ++q)
      if (mem.alloc((void**)&segX[q], dd * 8) != cudaSuccess || mem.alloc((void**)&segE[q], dd * 8) != cudaSuccess)
        return fail();
    double *P1 = nullptr, *Q = nullptr, *P2 = nullptr;
    if (mem.alloc((void**)&P1, dd * 8) != cudaSuccess || mem.alloc((void**)&Q, dd * 8) != cudaSuccess ||
        mem.alloc((void**)&P2, dd * 8) != cudaSuccess)
      return fail();
    const int nseg = (M + ck - 1) / ck;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int c0 = seg * ck, c1 = std::min(c0 + ck, M);
      if (cudaMemcpyAsync(segX[0], ckpt[seg], dd * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return fail();
      for (int m = c0; m < c1; ++m) {
        const int q = m - c0;
        F64GemmArgs sy{};
        sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = F64_EPI_NS_SYRK;
        sy.A = segX[q]; sy.B = segX[q]; sy.out = segE[q]; sy.partials = partials;
        if (!c.ok(f64_gemm(sy, st))) return fail();
        if (m + 1 < c1) {
          F64GemmArgs up{};
          up.dp = dp; up.d_real = d; up.sym = 1; up.epi = F64_EPI_NS_UPDATE;
          up.A = segX[q]; up.B = segE[q]; up.xin = segX[q]; up.out = segX[q + 1]; up.partials = partials;
          if (!c.ok(f64_gemm(up, st))) return fail();
        }
      }
      for (int m = c1 - 1; m >= c0; --m) {
        const int q = m - c0;
        F64GemmArgs g1{};
        g1.dp = dp; g1.d_real = d; g1.sym = 0; g1.epi = F64_EPI_STORE; g1.scale = 1.0;
        g1.A = G; g1.B = segE[q]; g1.out = P1;                      // G E_m
        F64GemmArgs g2 = g1;
        g2.A = segX[q]; g2.B = G; g2.out = Q;                       // X_m G
        F64GemmArgs g3 = g1;
        g3.sym = 1; g3.A = Q; g3.B = segX[q]; g3.out = P2;          // X_m G X_m (symmetric)
        if (!c.ok(f64_gemm(g1, st)) || !c.ok(f64_gemm(g2, st)) || !c.ok(f64_gemm(g3, st)) ||
            !c.ok(tangent_combine_f64(G, P1, P2, dp, st)))
          return fail();
      }
    }
  } else {
    // -------- low precision: the stage-1 trajectory kept whole, tangent products in FP16/BF16
    const int fmt = lp_fmt_of(policy);
    const bool split = policy == RSIGN_FP16_REFINE || policy == RSIGN_BF16_REFINE || policy == RSIGN_FP32;
    const int planes = split ? 2 : 1;
    std::vector<void*> xs, es;
    auto slot = [&](std::vector<void*>& v, int m) -> void* {
      while ((int)v.size() <= m) {
        void* p = nullptr;
        if (mem.alloc(&p, dd * 2 * planes) != cudaSuccess) return nullptr;
        v.push_back(p);
      }
      return v[m];
    };
    if (!slot(xs, 0)) return fail();
    if (split) {
      if (!c.ok(scale_convert_split(A64, dd, ctl->scal + 1, xs[0], fmt, st))) return fail();
    } else if (!c.ok(scale_convert(A64, dd, ctl->scal + 1, 1.0, xs[0], fmt, st))) {
      return fail();
    }
    const double u = split ? 4.0 * unit_roundoff(fmt) * unit_roundoff(fmt) : unit_roundoff(fmt);
    const int nt = tc_num_tiles(dp, 1);
    float* rowsq = nullptr;
    if (d > kExactDiagMin && mem.alloc((void**)&rowsq, (size_t)dp * 4) != cudaSuccess) return fail();
    int M = max_steps;
    for (int m = 0; m <= max_steps; ++m) {
      void* xm = slot(xs, m);
      void* em = slot(es, m);
      if (!xm || !em) return fail();
      TcGemmArgs sy{};
      sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = TC_EPI_NS_SYRK; sy.n_groups = 1;
      sy.group_start[0] = 0; sy.pair_a[0] = 0; sy.pair_b[0] = 0;
      if (split) {
        sy.pair_a[1] = 0; sy.pair_b[1] = 1; sy.pair_a[2] = 1; sy.pair_b[2] = 0; sy.group_start[1] = 3;
      } else {
        sy.group_start[1] = 1;
      }
      sy.split = split ? 1 : 0; sy.group_scale[0] = 1.0; sy.scale = 1.0f; sy.out = em; sy.partials = partials;
      sy.status = &ctl->status;
      sy.ns_diag = rowsq;
      if ((rowsq && !c.ok(row_sumsq(xm, fmt, split ? 1 : 0, dp, d, rowsq, nullptr, st))) ||
          !c.ok(tc_gemm(sy, xm, planes, xm, planes, fmt, c.num_sms, st)) ||
          !c.ok(ns_check(partials, nt * 4, hist, m, 0.0, 2.0 * u * std::sqrt((double)d), 16.0 * u * std::sqrt((double)d),
                         0.5, &ctl->done_low, &ctl->steps_low, st)))
        return fail();
      if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail();
      if (h.status != 0) {
        mem.release();
        cudaStreamSynchronize(st);
        return (rsign_status)h.status;
      }
      if (h.done_low || m == max_steps) {
        M = m;
        break;
      }
      void* xn = slot(xs, m + 1);
      if (!xn) return fail();
      TcGemmArgs up = sy;
      up.epi = TC_EPI_NS_UPDATE; up.out = xn; up.xin = xm;
      if (!c.ok(tc_gemm(up, xm, planes, em, planes, fmt, c.num_sms, st))) return fail();
    }
    if (polish) {
      // -------- the FP64 polish steps after stage 1 (the default depth of the
      // forward, rsign_options.polish_steps = 2): recomputed in FP64 from the
      // stage-1 result, then G is taken back through them in FP64
      constexpr int kPolish = 2;
      std::vector<double*> xp(kPolish + 1, nullptr), ep(kPolish, nullptr);
      for (auto& p : xp)
        if (mem.alloc((void**)&p, dd * 8) != cudaSuccess) return fail();
      for (auto& p : ep)
        if (mem.alloc((void**)&p, dd * 8) != cudaSuccess) return fail();
      double *P1 = nullptr, *Q = nullptr, *P2 = nullptr;
      if (mem.alloc((void**)&P1, dd * 8) != cudaSuccess || mem.alloc((void**)&Q, dd * 8) != cudaSuccess ||
          mem.alloc((void**)&P2, dd * 8) != cudaSuccess)
        return fail();
      if (!c.ok(to_f64(xs[M], fmt, dd, xp[0], st))) return fail();
      for (int j = 0; j < kPolish; ++j) {
        F64GemmArgs sy{};
        sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = F64_EPI_NS_SYRK;
        sy.A = xp[j]; sy.B = xp[j]; sy.out = ep[j]; sy.partials = partials;
        F64GemmArgs up{};
        up.dp = dp; up.d_real = d; up.sym = 1; up.epi = F64_EPI_NS_UPDATE;
        up.A = xp[j]; up.B = ep[j]; up.xin = xp[j]; up.out = xp[j + 1]; up.partials = partials;
        if (!c.ok(f64_gemm(sy, st)) || !c.ok(f64_gemm(up, st))) return fail();
      }
      for (int j = kPolish - 1; j >= 0; --j) {
        F64GemmArgs g1{};
        g1.dp = dp; g1.d_real = d; g1.sym = 0; g1.epi = F64_EPI_STORE; g1.scale = 1.0;
        g1.A = G; g1.B = ep[j]; g1.out = P1;                        // G E_j
        F64GemmArgs g2 = g1;
        g2.A = xp[j]; g2.B = G; g2.out = Q;                         // X_j G
        F64GemmArgs g3 = g1;
        g3.sym = 1; g3.A = Q; g3.B = xp[j]; g3.out = P2;            // X_j G X_j
        if (!c.ok(f64_gemm(g1, st)) || !c.ok(f64_gemm(g2, st)) || !c.ok(f64_gemm(g3, st)) ||
            !c.ok(tangent_combine_f64(G, P1, P2, dp, st)))
          return fail();
      }
    }
    // backward tangent sweep in the operand type (hi planes), FP32 master G
    const int ntile = (dp / 32) * (dp / 32);
    float *G32 = nullptr, *P32 = nullptr, *Q32 = nullptr, *bmax = nullptr, *fs = nullptr;
    void *Glp = nullptr, *Qlp = nullptr;
    if (mem.alloc((void**)&G32, dd * 4) != cudaSuccess || mem.alloc((void**)&P32, dd * 4) != cudaSuccess ||
        mem.alloc((void**)&Q32, dd * 4) != cudaSuccess || mem.alloc(&Glp, dd * 2) != cudaSuccess ||
        mem.alloc(&Qlp, dd * 2) != cudaSuccess || mem.alloc((void**)&bmax, (size_t)ntile * 4) != cudaSuccess ||
        mem.alloc((void**)&fs, 16 * 4) != cudaSuccess)
      return fail();
    auto tc = [&](const void* Aop, const void* Bop, int sym, int epi, void* out) {
      TcGemmArgs a{};
      a.dp = dp; a.d_real = d; a.sym = sym; a.epi = epi; a.n_groups = 1;
      a.group_start[0] = 0; a.group_start[1] = 1; a.pair_a[0] = 0; a.pair_b[0] = 0;
      a.group_scale[0] = 1.0; a.scale = 1.0f; a.out = out; a.status = &ctl->status;
      return tc_gemm(a, Aop, 1, Bop, 1, fmt, c.num_sms, st);
    };
    if (!c.ok(scale_convert(G, dd, nullptr, 1.0, G32, 3, st))) return fail();
    if (!c.ok(absmax_tiles(G32, dp, bmax, st)) || !c.ok(max_pow2(bmax, ntile, fs + 4, st))) return fail();
    for (int m = M - 1; m >= 0; --m) {
      if (!c.ok(scale_to_lp(G32, dd, fs + 5, Glp, fmt, st))) return fail();
      if (!c.ok(tc(Glp, es[m], 0, TC_EPI_STORE_F32, P32))) return fail();     // G E_m
      if (!c.ok(tc(xs[m], Glp, 0, TC_EPI_STORE_LP, Qlp))) return fail();      // X_m G
      if (!c.ok(tc(Qlp, xs[m], 1, TC_EPI_STORE_F32, Q32))) return fail();     // X_m G X_m
      if (!c.ok(tangent_combine(G32, P32, Q32, dp, fs + 5, 1.0f, bmax, st))) return fail();
      if (!c.ok(max_pow2(bmax, ntile, fs + 4, st))) return fail();
    }
    if (!c.ok(to_f64(G32, 3, dd, G, st))) return fail();
  }
  // Hbar = alpha sym(G_0), unpadded
  if (!c.ok(symmetrize_scale(G, dp, alpha, Gs, st)) || !c.ok(copy_unpad(Gs, dp, Hb, d, st))) return fail();
  if (!hb_dev && cudaMemcpyAsync(Hbar, Hb, (size_t)d * d * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail();
  if (cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail();
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return RSIGN_ERR_CUDA;
  }
  return h.status != 0 ? (rsign_status)h.status : RSIGN_OK;
}

// out = R V, FP64; one warp per row of R, 8 columns of V per pass.
__global__ void apply_kernel(const double* __restrict__ R, int64_t d, const double* __restrict__ V,
                             int64_t nv, double* __restrict__ out) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= d) return;
  const double* r = R + row * d;
  for (int64_t c0 = 0; c0 < nv; c0 += 8) {
    const int nc = (int)std::min<int64_t>(8, nv - c0);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t kk = lane; kk < d; kk += 32) {
      const double a = r[kk];
      const double* v = V + kk * nv + c0;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < nc) acc[c] += a * v[c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double t = warp_sum(acc[c]);
      if (lane == 0 && c < nc) out[row * nv + c0 + c] = t;
    }
  }
}

// One bounded mbarrier wait with a caller-chosen limit: thread 0 initialises a
// barrier for one arrival and waits for its first phase, arriving itself first
// when `arrive` is set.  Without the arrival nothing completes the phase, so
// the wait gives up after limit_ns and records RSIGN_ERR_TIMEOUT in *status:
// the failure path of every pipeline wait in the library, exercised without a
// broken pipeline.
__global__ void bounded_wait_kernel(int* status, unsigned long long limit_ns, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(smem_u32(&bar));
    mbar_wait_for(smem_u32(&bar), 0, status, limit_ns);
  }
}

}  // namespace
}  // namespace rsign

using namespace rsign;

extern "C" {

void rsign_options_default(rsign_options* opt) {
  if (!opt) return;
  opt->max_steps = 100;
  opt->polish_steps = 2;
  opt->max_sweeps = 4;
  opt->alpha_mode = RSIGN_ALPHA_INF;
  opt->power_steps = 20;
  opt->timing = 1;
  opt->low_split = 1;
  opt->lanczos_max = 600;
  opt->batch_graphs = 1;
  opt->batch_tile = 0;
  opt->ns_scaling = 0;
  opt->margin = NAN;
  opt->refine_stop = RSIGN_STOP_ESTIMATE;
  opt->engine = RSIGN_ENGINE_NS3;
}

rsign_status rsign_reflector_ex(const double* H, int64_t d, int32_t k, double s, double tol,
                                rsign_policy policy, const rsign_options* opt, double* R,
                                rsign_info* info, void* stream) {
  rsign_status st = reflector_impl(H, d, k, s, tol, policy, opt, R, info, (cudaStream_t)stream);
  if (st == RSIGN_ERR_CERT && opt && opt->alpha_mode == RSIGN_ALPHA_POWER) {
    // the power estimate of rho came out too low (alpha rho >= sqrt(3) flips
    // signs): redo the call with the Gershgorin scaling, which is always safe
    rsign_options o = *opt;
    o.alpha_mode = RSIGN_ALPHA_INF;
    st = reflector_impl(H, d, k, s, tol, policy, &o, R, info, (cudaStream_t)stream);
  }
  return st;
}

rsign_status rsign_reflector(const double* H, int64_t d, int32_t k, double s, double tol,
                             rsign_policy policy, double* R, rsign_info* info, void* stream) {
  return reflector_impl(H, d, k, s, tol, policy, nullptr, R, info, (cudaStream_t)stream);
}

rsign_status rsign_apply(const double* R, int64_t d, const double* V, int64_t nv, double* out,
                         void* stream) {
  if (!R || !V || !out || d < 1 || nv < 1) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const double *Rd = R, *Vd = V;
  double* Od = out;
  const bool rd = is_device_ptr(R), vd = is_device_ptr(V), od = is_device_ptr(out);
  auto fail = [&]() { mem.release(); cudaStreamSynchronize(st); cudaGetLastError(); return RSIGN_ERR_CUDA; };
  if (!rd) {
    if (mem.alloc((void**)&Rd, (size_t)d * d * 8) != cudaSuccess ||
        cudaMemcpyAsync((void*)Rd, R, (size_t)d * d * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail();
  }
  if (!vd) {
    if (mem.alloc((void**)&Vd, (size_t)d * nv * 8) != cudaSuccess ||
        cudaMemcpyAsync((void*)Vd, V, (size_t)d * nv * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail();
  }
  if (!od && mem.alloc((void**)&Od, (size_t)d * nv * 8) != cudaSuccess) return fail();
  apply_kernel<<<(unsigned)((d + 7) / 8), 256, 0, st>>>(Rd, d, Vd, nv, Od);
  if (cudaGetLastError() != cudaSuccess) return fail();
  if (!od && cudaMemcpyAsync(out, Od, (size_t)d * nv * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail();
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return RSIGN_ERR_CUDA; }
  return RSIGN_OK;
}

rsign_status rsign_reflector_backward(const double* H, int64_t d, int32_t k, double s,
                                      rsign_policy policy, const double* Rbar, double* Hbar,
                                      int32_t ckpt_every, void* stream) {
  return backward_impl(H, d, k, s, policy, Rbar, Hbar, ckpt_every, (cudaStream_t)stream);
}

const char* rsign_status_str(rsign_status st) {
  switch (st) {
    case RSIGN_OK: return "ok";
    case RSIGN_ERR_ARG: return "invalid argument";
    case RSIGN_ERR_NOCONV: return "step budget exhausted before the tolerance was met";
    case RSIGN_ERR_CERT: return "trace certificate failed (shift not admissible)";
    case RSIGN_ERR_GAP: return "target gap not resolved";
    case RSIGN_ERR_CUDA: return "CUDA error";
    case RSIGN_ERR_TIMEOUT: return "device-side wait timed out";
    case RSIGN_ERR_UNSUPPORTED: return "unsupported device, size or mode";
    default: return "unknown status";
  }
}

const char* rsign_version(void) { return "rsign 0.1 sm_103a"; }

rsign_status rsign_trim_workspace(void) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (int i = 0; i < kMaxPoolDevices; ++i) {
    if (g_pools[i] == nullptr) continue;
    if (cudaMemPoolTrimTo(g_pools[i], 0) != cudaSuccess) {
      cudaGetLastError();
      return RSIGN_ERR_CUDA;
    }
  }
  return RSIGN_OK;
}

}  // extern "C"

// ------------------------------------------------------------ debug entry points
#include "../../include/rsign_debug.h"

extern "C" {

rsign_status rsign_dbg_tc_gemm(const void* A, const void* B, int64_t dp, int32_t fmt, int32_t sym,
                               float* out, int* status, void* stream) {
  if (!A || !B || !out || !status || dp < 256 || dp % 256 || dp > 16384 || (fmt != 0 && fmt != 1))
    return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  TcGemmArgs a{};
  a.dp = (int)dp; a.d_real = (int)dp; a.sym = sym ? 1 : 0; a.epi = TC_EPI_STORE_F32; a.n_groups = 1;
  a.group_start[0] = 0; a.group_start[1] = 1; a.pair_a[0] = 0; a.pair_b[0] = 0; a.group_scale[0] = 1.0;
  a.scale = 1.0f; a.out = out; a.status = status; a.skip = nullptr;
  return tc_gemm(a, A, 1, B, 1, fmt, sms, (cudaStream_t)stream) == cudaSuccess ? RSIGN_OK : RSIGN_ERR_CUDA;
}

rsign_status rsign_dbg_scaled_coeffs(double alpha_margin, double u0, int32_t cap, double* out, int32_t* n) {
  if (!out || !n || cap < 0 || !(alpha_margin > 0.0) || !(u0 >= 1.0) || !std::isfinite(u0)) return RSIGN_ERR_ARG;
  const std::vector<double> coef = scaled_ns_coeffs(alpha_margin, u0);
  *n = (int32_t)coef.size();
  for (int32_t i = 0; i < cap && i < *n; ++i) out[i] = coef[i];
  return RSIGN_OK;
}

rsign_status rsign_dbg_gamma_from_steps(int32_t m, double* gamma) {
  if (!gamma || m < 0 || m > 1000) return RSIGN_ERR_ARG;
  *gamma = gamma_from_steps(m);
  return RSIGN_OK;
}

rsign_status rsign_dbg_tridiag_ritz(const double* alpha, const double* beta, int32_t m, int32_t j, double* theta,
                                    double* last) {
  if (!alpha || (m > 1 && !beta) || !theta || !last || m < 1 || j < 0 || j >= m) return RSIGN_ERR_ARG;
  tridiag_ritz(alpha, beta, m, j, theta, last);
  return RSIGN_OK;
}

rsign_status rsign_dbg_f64_gemm(const double* A, const double* B, int64_t dp, int32_t sym, double* out,
                                void* stream) {
  if (!A || !B || !out || dp < 64 || dp % 64 || dp > 16384) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  F64GemmArgs a{};
  a.dp = (int)dp; a.d_real = (int)dp; a.sym = sym ? 1 : 0; a.epi = F64_EPI_STORE; a.scale = 1.0;
  a.A = A; a.B = B; a.out = out;
  return f64_gemm(a, (cudaStream_t)stream) == cudaSuccess ? RSIGN_OK : RSIGN_ERR_CUDA;
}

rsign_status rsign_dbg_fp64grade_gemm(const double* A, const double* B, int64_t dp, int64_t d_real,
                                      int32_t sym, double* out, void* stream) {
  if (!A || !B || !out || dp < 256 || dp % 256 || dp > 16384 || d_real < 1 || d_real > dp)
    return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const size_t dd = (size_t)dp * dp;
  SplitMat sa{}, sb{};
  int* status = nullptr;
  rsign_status res = RSIGN_OK;
  sa.full = A;
  sb.full = B;
  sa.fp8 = sb.fp8 = g_digit_fp8;
  const size_t digit_bytes = g_digit_fp8 ? 1 : 2;
  if (mem.alloc(&sa.planes, dd * digit_bytes * kSlices) != cudaSuccess ||
      mem.alloc((void**)&sa.sigma, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&sa.diag, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc(&sb.planes, dd * digit_bytes * kSlices) != cudaSuccess ||
      mem.alloc((void**)&sb.sigma, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&sb.diag, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&status, 4) != cudaSuccess || cudaMemsetAsync(status, 0, 4, st) != cudaSuccess ||
      split_rows(A, (int)dp, sa, st) != cudaSuccess || split_rows(B, (int)dp, sb, st) != cudaSuccess ||
      ozaki_gemm(sa, sb, (int)dp, (int)d_real, sym ? 1 : 0, out, status, sms, st) != cudaSuccess)
    res = RSIGN_ERR_CUDA;
  int hs = 0;
  if (res == RSIGN_OK && (cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                          cudaStreamSynchronize(st) != cudaSuccess))
    res = RSIGN_ERR_CUDA;
  if (res == RSIGN_OK && hs != 0) res = (rsign_status)hs;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

rsign_status rsign_dbg_stage_plan(double alpha_margin, double u0, int32_t scaled, int32_t max_steps,
                                  int32_t steps_low, double* lower_end, int32_t* n_split, int32_t* m_tangent) {
  if (!(alpha_margin > 0.0) || !(u0 >= 1.0) || !std::isfinite(u0) || max_steps < 1 || max_steps > 1000 ||
      steps_low < 0 || steps_low > max_steps || !n_split || !m_tangent)
    return RSIGN_ERR_ARG;
  const std::vector<double> coef = scaled ? scaled_ns_coeffs(alpha_margin, u0) : std::vector<double>();
  const std::vector<double> le = lower_end_sequence(alpha_margin, u0, coef, max_steps);
  if (lower_end)
    for (size_t q = 0; q < le.size(); ++q) lower_end[q] = le[q];
  int ns = 0, mt = 0;
  refine_stage_plan(le, steps_low, &ns, &mt);
  *n_split = ns;
  *m_tangent = mt;
  return RSIGN_OK;
}

double rsign_dbg_set_split_until(double l) {
  const double prev = g_split_until;
  if (l > 0.0 && l <= 1.0) g_split_until = l;
  return prev;
}

int32_t rsign_dbg_set_copy_streams(int32_t n) {
  const int prev = g_copy_streams;
  if (n >= 1 && n <= 8) g_copy_streams = n;
  return prev;
}

int32_t rsign_dbg_set_host_mapped(int32_t on) {
  const int prev = g_host_mapped;
  if (on == 0 || on == 1) g_host_mapped = on;
  return prev;
}

int32_t rsign_dbg_set_tangent_cut(int32_t on) {
  const int prev = g_tangent_cut;
  if (on == 0 || on == 1) g_tangent_cut = on;
  return prev;
}

int32_t rsign_dbg_set_split_steps(int32_t n) {
  const int prev = g_split_steps;
  if (n >= -2) g_split_steps = n;
  return prev;
}

int32_t rsign_dbg_set_digit_fp8(int32_t on) {
  const int prev = g_digit_fp8;
  if (on == 0 || on == 1) g_digit_fp8 = on;
  return prev;
}

rsign_status rsign_dbg_bounded_wait(int32_t arrive, int64_t limit_ns, int* status, void* stream) {
  if (!status || limit_ns < 1 || limit_ns > (int64_t)kWaitLimitNs || !is_device_ptr(status)) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  bounded_wait_kernel<<<1, 32, 0, st>>>(status, (unsigned long long)limit_ns, arrive ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return RSIGN_ERR_CUDA;
  }
  return RSIGN_OK;
}

int32_t rsign_dbg_set_refine_levels(int32_t polish, int32_t ra_first, int32_t ra_later) {
  const int prev = g_levels_polish * 100 + g_levels_ra0 * 10 + g_levels_ra;
  auto ok = [](int v) { return v >= 0 && v <= kSlices; };
  if (ok(polish)) g_levels_polish = polish;
  if (ok(ra_first)) g_levels_ra0 = ra_first;
  if (ok(ra_later)) g_levels_ra = ra_later;
  return prev;
}

int32_t rsign_dbg_set_ozaki_tile(int32_t bn) {
  const int prev = g_oz_tile;
  if (bn == 0 || bn == 128 || bn == 256) g_oz_tile = bn;
  return prev;
}

int32_t rsign_dbg_batch_units(int32_t n, const int32_t* dp, int32_t bn, int32_t sym, int32_t order, int32_t cap,
                              int32_t* units, int32_t* slot_begin) {
  if (n < 0 || (n > 0 && !dp) || (bn != 128 && bn != 256) || cap < 0 || (cap > 0 && !units)) return -1;
  std::vector<int> d(dp, dp + n);
  for (int m = 0; m < n; ++m)
    if (d[m] < bn || d[m] % bn || d[m] > 16384) return -1;
  std::vector<int4> u;
  std::vector<int> sb;
  tc_build_units(n, d.data(), bn, sym ? 1 : 0, order ? 1 : 0, &u, &sb);
  for (int i = 0; i < (int)u.size() && i < cap; ++i) {
    units[4 * i] = u[i].x;
    units[4 * i + 1] = u[i].y;
    units[4 * i + 2] = u[i].z;
    units[4 * i + 3] = u[i].w;
  }
  if (slot_begin)
    for (int m = 0; m <= n; ++m) slot_begin[m] = sb[m];
  return (int32_t)u.size();
}

int32_t rsign_dbg_refine_levels(double tol, double s_a, double s_r, int64_t d, double mu, int32_t k) {
  if (!(tol > 0.0) || !(s_a > 0.0) || !(s_r > 0.0) || d < 2 || d > 16384 || !(mu > 0.0) || k < 1 || k >= d)
    return -1;
  // low 16 bits: the first sweep's R A levels; high bits: the polish levels
  return levels_ra0(tol, s_a, s_r, (int)d, mu) | (levels_for(0, tol, (int)d, k) << 16);
}

int32_t rsign_dbg_fp64e_beta(int64_t k_extent) {
  if (k_extent < 1 || k_extent > 16384) return 0;
  return fp64e_beta((int)k_extent);
}

rsign_status rsign_dbg_fp64e_plan(int32_t n_planes, int32_t beta, int32_t levels, int64_t k_extent, int32_t* meta,
                                  int32_t* group_start, int32_t* pair_a, int32_t* pair_b, int32_t* group_shift,
                                  int32_t* group_sg) {
  if (!meta || !group_start || !pair_a || !pair_b || !group_shift || !group_sg || n_planes < 1 || beta < 2 ||
      beta > 11 || n_planes * beta > 77 || levels < 1 || k_extent < 1 || k_extent > 16384)
    return RSIGN_ERR_ARG;
  TcGemmArgs a{};
  if (fp64e_plan(&a, n_planes, beta, levels, (int)k_extent) != cudaSuccess) return RSIGN_ERR_ARG;
  meta[0] = a.n_groups;
  meta[1] = a.group_start[a.n_groups];
  meta[2] = a.n_sg;
  meta[3] = a.oz_unit_exp;
  meta[4] = a.oz_sh01;
  for (int g = 0; g <= a.n_groups; ++g) group_start[g] = a.group_start[g];
  for (int r = 0; r < a.group_start[a.n_groups]; ++r) {
    pair_a[r] = a.pair_a[r];
    pair_b[r] = a.pair_b[r];
  }
  for (int g = 0; g < a.n_groups; ++g) {
    group_shift[g] = a.group_shift[g];
    group_sg[g] = a.n_sg == 2 ? a.group_sg[g] : 0;
  }
  return RSIGN_OK;
}

rsign_status rsign_dbg_oz_convert(const int64_t* v, const int32_t* e, int64_t n, double* a, double* b,
                                  void* stream) {
  if (!v || !e || !a || !b || n < 1 || n > (int64_t)1 << 30) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  rsign_status res = RSIGN_OK;
  if (oz_convert_pair((const long long*)v, (const int*)e, (int)n, a, b, st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

int32_t rsign_dbg_sym_gemv_tiles(int64_t dp, int32_t* I, int32_t* J) {
  if (dp < 256 || dp % 256 || dp > 16384) return -1;
  return gemv_df_sym_tiles((int)dp, I, J);
}

int32_t rsign_dbg_tile_order(int64_t dp, int32_t sym, int32_t* bm, int32_t* bn) {
  if (dp < 256 || dp % 256 || dp > 16384) return -1;
  const int n = tc_num_tiles((int)dp, sym ? 1 : 0);
  if (!bm || !bn) return n;
  return tc_tile_order((int)dp, sym ? 1 : 0, bm, bn);
}

rsign_status rsign_dbg_fp64e_gemm(const double* A, const double* B, int64_t dp, int64_t d_real, int32_t sym,
                                  double* out, void* stream) {
  if (!A || !B || !out || dp < 256 || dp % 256 || dp > 16384 || d_real < 1 || d_real > dp)
    return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const size_t dd = (size_t)dp * dp;
  const int beta = fp64e_beta((int)d_real);
  const int P = fp64e_planes(beta);
  SplitMat sa{}, sb{};
  sa.n_planes = sb.n_planes = P;
  sa.beta = sb.beta = beta;
  int* status = nullptr;
  Fp64eExtra x{};
  rsign_status res = RSIGN_OK;
  sa.full = A;
  sb.full = B;
  if (beta == 0 || mem.alloc(&sa.planes, dd * 2 * P) != cudaSuccess ||
      mem.alloc((void**)&sa.sigma, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&sa.diag, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc(&sb.planes, dd * 2 * P) != cudaSuccess ||
      mem.alloc((void**)&sb.sigma, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&sb.diag, (size_t)dp * 8) != cudaSuccess ||
      mem.alloc((void**)&x.acc64, dd * 8) != cudaSuccess ||
      mem.alloc((void**)&status, 4) != cudaSuccess || cudaMemsetAsync(status, 0, 4, st) != cudaSuccess ||
      split_rows(A, (int)dp, sa, st) != cudaSuccess || split_rows(B, (int)dp, sb, st) != cudaSuccess ||
      fp64e_gemm(sa, sb, (int)dp, (int)d_real, sym ? 1 : 0, out, x, status, sms, st, P) != cudaSuccess)
    res = RSIGN_ERR_CUDA;
  int hs = 0;
  if (res == RSIGN_OK && (cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                          cudaStreamSynchronize(st) != cudaSuccess))
    res = RSIGN_ERR_CUDA;
  if (res == RSIGN_OK && hs != 0) res = (rsign_status)hs;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

rsign_status rsign_dbg_spectral_norm(const double* M, int64_t dp, int32_t iters, int32_t per_step, double* out,
                                     void* stream) {
  if (!M || !out || dp < 256 || dp % 256 || dp > 16384 || iters < 1 || iters > 1000) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const size_t dd = (size_t)dp * dp;
  float *m32 = nullptr, *v = nullptr, *w = nullptr;
  double* o = nullptr;
  rsign_status res = RSIGN_OK;
  if (mem.alloc((void**)&m32, dd * 4) != cudaSuccess || mem.alloc((void**)&v, (size_t)dp * 4) != cudaSuccess ||
      mem.alloc((void**)&w, (size_t)dp * 4) != cudaSuccess || mem.alloc((void**)&o, 8) != cudaSuccess ||
      split_f32(M, dd, m32, nullptr, 0, nullptr, st) != cudaSuccess ||
      spectral_norm_f32(m32, (int)dp, v, w, iters, o, st, per_step != 0) != cudaSuccess ||
      cudaMemcpyAsync(out, o, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    res = RSIGN_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

rsign_status rsign_dbg_gemv_df_sym(const double* M, const double* x, int64_t dp, double* y, void* stream) {
  if (!M || !x || !y || dp < 256 || dp % 256 || dp > 16384) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const size_t dd = (size_t)dp * dp;
  float *mh = nullptr, *ml = nullptr, *xh = nullptr, *xl = nullptr;
  float2* pt = nullptr;
  rsign_status res = RSIGN_OK;
  if (mem.alloc((void**)&mh, dd * 4) != cudaSuccess || mem.alloc((void**)&ml, dd * 4) != cudaSuccess ||
      mem.alloc((void**)&xh, (size_t)dp * 4) != cudaSuccess || mem.alloc((void**)&xl, (size_t)dp * 4) != cudaSuccess ||
      mem.alloc((void**)&pt, gemv_df_sym_part_bytes((int)dp)) != cudaSuccess ||
      split_f32(M, dd, mh, ml, 0, nullptr, st) != cudaSuccess ||
      split_f32(x, (size_t)dp, xh, xl, 0, nullptr, st) != cudaSuccess ||
      gemv_df_sym(mh, ml, xh, xl, y, (int)dp, pt, st) != cudaSuccess)
    res = RSIGN_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

rsign_status rsign_dbg_gemv_df(const double* M, const double* x, int64_t dp, double* y, void* stream) {
  if (!M || !x || !y || dp < 256 || dp % 256 || dp > 16384) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const size_t dd = (size_t)dp * dp;
  float *mh = nullptr, *ml = nullptr, *xh = nullptr, *xl = nullptr;
  rsign_status res = RSIGN_OK;
  if (mem.alloc((void**)&mh, dd * 4) != cudaSuccess || mem.alloc((void**)&ml, dd * 4) != cudaSuccess ||
      mem.alloc((void**)&xh, (size_t)dp * 4) != cudaSuccess || mem.alloc((void**)&xl, (size_t)dp * 4) != cudaSuccess ||
      split_f32(M, dd, mh, ml, 0, nullptr, st) != cudaSuccess ||
      split_f32(x, (size_t)dp, xh, xl, 0, nullptr, st) != cudaSuccess ||
      gemv_df(mh, ml, xh, xl, y, (int)dp, st) != cudaSuccess)
    res = RSIGN_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

rsign_status rsign_dbg_commutator_check(const double* A, const double* R, int64_t dp, int64_t d, int32_t iters,
                                        double* out, void* stream) {
  if (!A || !R || !out || dp < 256 || dp % 256 || dp > 16384 || d < 1 || d > dp || iters < 1 || iters > 1000)
    return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = (rsign_status)check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf mem;
  mem.st = st;
  const size_t dd = (size_t)dp * dp;
  float *ah = nullptr, *al = nullptr, *rh = nullptr, *rl = nullptr, *fw = nullptr;
  float2* pt = nullptr;
  double *w = nullptr, *o = nullptr;
  rsign_status res = RSIGN_OK;
  if (mem.alloc((void**)&ah, dd * 4) != cudaSuccess || mem.alloc((void**)&al, dd * 4) != cudaSuccess ||
      mem.alloc((void**)&rh, dd * 4) != cudaSuccess || mem.alloc((void**)&rl, dd * 4) != cudaSuccess ||
      mem.alloc((void**)&fw, (size_t)12 * dp * 4) != cudaSuccess ||
      mem.alloc((void**)&w, (size_t)12 * dp * 8) != cudaSuccess || mem.alloc((void**)&o, 8 * 8) != cudaSuccess ||
      split_f32(A, dd, ah, al, 0, nullptr, st) != cudaSuccess ||
      mem.alloc((void**)&pt, gemv_df_sym_part_bytes((int)dp)) != cudaSuccess ||
      commutator_gain_norm(ah, al, R, rh, rl, (int)dp, (int)d, iters, w, fw, pt, o, st) != cudaSuccess ||
      cudaMemcpyAsync(out, o, 5 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    res = RSIGN_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) res = RSIGN_ERR_CUDA;
  cudaGetLastError();
  return res;
}

}  // extern "C"
