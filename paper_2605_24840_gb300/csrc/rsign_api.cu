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
#include <vector>

namespace rsign {
namespace {

constexpr int kChunk = 8;  // NS steps enqueued between host checks of the stop flag

struct DevBuf {
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  int64_t bytes = 0;
  cudaError_t alloc(void** p, size_t n) {
    n = (n + 255) & ~size_t(255);
    cudaError_t e = cudaMallocAsync(p, n, st);
    if (e == cudaSuccess) {
      ptrs.push_back(*p);
      bytes += (int64_t)n;
    }
    return e;
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

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

rsign_status check_device(int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return RSIGN_ERR_CUDA; }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (major != 10 || minor != 3) return RSIGN_ERR_UNSUPPORTED;
  return RSIGN_OK;
}

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
};

bool f64_ns(Ctx& c, const F64Loop& L, int dp, int d, double tol_abs, int max_steps, Ctl* ctl_dev,
            Ctl& ctl_host, int* m_out, bool* conv) {
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
      if (!c.ok(f64_gemm(sy, c.st))) return false;
      if (!c.ok(ns_check(L.partials, nt * 4, L.hist, mm, tol_abs, -1.0, -1.0, 0.0, L.done, L.steps, c.st)))
        return false;
      if (mm == max_steps) break;  // residual of the last iterate only
      F64GemmArgs up{};
      up.dp = dp; up.d_real = d; up.sym = 1; up.epi = F64_EPI_NS_UPDATE;
      up.A = L.xb[mm & 1]; up.B = L.E; up.xin = L.xb[mm & 1]; up.out = L.xb[(mm + 1) & 1];
      up.partials = L.partials; up.skip = L.done;
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
  if ((int)policy < RSIGN_FP64 || (int)policy > RSIGN_BF16_REFINE) return RSIGN_ERR_ARG;
  if (opt.max_steps < 1 || opt.max_steps > 1000 || opt.polish_steps < 0 || opt.max_sweeps < 0)
    return RSIGN_ERR_ARG;
  if (std::isinf(s)) return RSIGN_ERR_ARG;
  if (std::isnan(s)) return RSIGN_ERR_UNSUPPORTED;  // automatic shift: not in this build
  if (policy == RSIGN_FP16_REFINE || policy == RSIGN_BF16_REFINE) return RSIGN_ERR_UNSUPPORTED;

  Ctx c;
  c.st = st;
  rsign_status dst = check_device(&c.num_sms);
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
  int steps_low = 0, steps64 = 0;
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
  if (!h_dev) {
    if (mem.alloc((void**)&Hd, (size_t)d * d * 8) != cudaSuccess) return fail_cuda();
    if (cudaMemcpyAsync(Hd, H, (size_t)d * d * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail_cuda();
  }
  if (!r_dev && mem.alloc((void**)&Rd, (size_t)d * d * 8) != cudaSuccess) return fail_cuda();
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) != cudaSuccess) return fail_cuda();
  double* hist_low = hist;
  double* hist64 = hist + opt.max_steps + 2;

  // ---- ingest and scaling (Sec. 4.3: alpha = 1/||H - sI||_inf)
  if (!c.ok(ingest(Hd, d, dp, s, A64, rowpart, &ctl->flags, st))) return fail_cuda();
  if (!c.ok(inf_norm_finish(rowpart, dp, rowsum, ctl->scal, st))) return fail_cuda();
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

  double* Rfinal = nullptr;  // dp x dp FP64 result
  double* xb64[2] = {nullptr, nullptr};
  double* E64 = nullptr;
  const bool need64 = policy == RSIGN_FP64 || policy == RSIGN_FP16_POLISH || policy == RSIGN_BF16_POLISH;
  if (mem.alloc((void**)&xb64[0], dd * 8) != cudaSuccess) return fail_cuda();
  if (need64 && (mem.alloc((void**)&xb64[1], dd * 8) != cudaSuccess ||
                 mem.alloc((void**)&E64, dd * 8) != cudaSuccess))
    return fail_cuda();

  if (opt.timing) cudaEventRecord(ev[1], st);
  if (is_low(policy)) {
    // ---------------------------------------------- low-precision stage (tcgen05)
    const int fmt = lp_fmt_of(policy);
    void* xs[2] = {nullptr, nullptr};
    void* es = nullptr;
    if (mem.alloc(&xs[0], dd * 2) != cudaSuccess || mem.alloc(&xs[1], dd * 2) != cudaSuccess ||
        mem.alloc(&es, dd * 2) != cudaSuccess)
      return fail_cuda();
    if (!c.ok(scale_convert(A64, dd, ctl->scal + 1, 1.0, xs[0], fmt, st))) return fail_cuda();
    const double u = unit_roundoff(fmt);
    const double floor_lo = 2.0 * u * std::sqrt((double)d);
    const double floor_hi = 16.0 * u * std::sqrt((double)d);
    const int nt = tc_num_tiles(dp, 1);
    int m = 0;
    bool stopped = false;
    while (m <= opt.max_steps && !stopped) {
      const int m_end = std::min(m + kChunk, opt.max_steps + 1);
      for (int mm = m; mm < m_end; ++mm) {
        TcGemmArgs sy{};
        sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = TC_EPI_NS_SYRK; sy.n_groups = 1;
        sy.group_start[0] = 0; sy.group_start[1] = 1; sy.pair_a[0] = 0; sy.pair_b[0] = 0;
        sy.group_scale[0] = 1.0; sy.scale = 1.0f; sy.out = es; sy.partials = partials;
        sy.status = &ctl->status; sy.skip = &ctl->done_low;
        if (!c.ok(tc_gemm(sy, xs[mm & 1], 1, xs[mm & 1], 1, fmt, c.num_sms, st))) return fail_cuda();
        if (!c.ok(ns_check(partials, nt * 4, hist_low, mm, 0.0, floor_lo, floor_hi, 0.5, &ctl->done_low,
                           &ctl->steps_low, st)))
          return fail_cuda();
        if (mm == opt.max_steps) break;
        TcGemmArgs up = sy;
        up.epi = TC_EPI_NS_UPDATE; up.out = xs[(mm + 1) & 1]; up.xin = xs[mm & 1];
        if (!c.ok(tc_gemm(up, xs[mm & 1], 1, es, 1, fmt, c.num_sms, st))) return fail_cuda();
      }
      if (cudaMemcpyAsync(&ctl_h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return fail_cuda();
      if (ctl_h.status != 0) break;
      stopped = ctl_h.done_low != 0;
      m = m_end;
    }
    steps_low = stopped ? ctl_h.steps_low : opt.max_steps;
    if (!c.ok(to_f64(xs[steps_low & 1], fmt, dd, xb64[0], st))) return fail_cuda();
    Rfinal = xb64[0];
    hist_h.resize(opt.max_steps + 2);
    if (cudaMemcpyAsync(hist_h.data(), hist_low, hist_h.size() * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail_cuda();
    resid = hist_h[steps_low];
    if (!stopped && ctl_h.status == 0) result = RSIGN_ERR_NOCONV;
  } else {
    if (!c.ok(scale_convert(A64, dd, ctl->scal + 1, 1.0, xb64[0], 2, st))) return fail_cuda();
  }
  if (opt.timing) cudaEventRecord(ev[2], st);

  if (need64 && ctl_h.status == 0) {
    // ------------------------------------------------------------- FP64 stage
    F64Loop L{{xb64[0], xb64[1]}, E64, partials, hist64, &ctl->done64, &ctl->steps64};
    int m_ret = 0;
    const bool polish = policy != RSIGN_FP64;
    const double tol_abs = polish ? -1.0 : tol_fro;
    const int budget = polish ? opt.polish_steps : opt.max_steps;
    if (!f64_ns(c, L, dp, d, tol_abs, budget, ctl, ctl_h, &m_ret, &conv64)) return fail_cuda();
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
  if (!r_dev && cudaMemcpyAsync(R, Rd, (size_t)d * d * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
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
    info->sweeps_refine = 0;
    info->cert_ok = (trace_ok && resid_ok) ? 1 : 0;
    info->alpha = alpha;
    info->shift = s;
    info->gamma_est = NAN;
    info->resid_fro = resid;
    info->trace = trace;
    info->correction_fro = NAN;
    info->commutator_fro = NAN;
    info->tol_fro = tol_fro;
    if (opt.timing) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[0], ev[3]); info->ms_total = t;
      cudaEventElapsedTime(&t, ev[1], ev[2]); info->ms_low = is_low(policy) ? t : 0.0;
      cudaEventElapsedTime(&t, ev[2], ev[3]); info->ms_fp64 = t;
    }
    const double dd3 = (double)d * d * d;
    info->flops_low = is_low(policy) ? dd3 * (2.0 * steps_low + 1.0) : 0.0;
    info->launches = c.launches;
    info->workspace_bytes = mem.bytes;
  }
  mem.release();
  if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); result = RSIGN_ERR_CUDA; }
  for (auto& e : ev) if (e) cudaEventDestroy(e);
  return result;
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
  opt->power_steps = 12;
  opt->timing = 1;
}

rsign_status rsign_reflector_ex(const double* H, int64_t d, int32_t k, double s, double tol,
                                rsign_policy policy, const rsign_options* opt, double* R,
                                rsign_info* info, void* stream) {
  return reflector_impl(H, d, k, s, tol, policy, opt, R, info, (cudaStream_t)stream);
}

rsign_status rsign_reflector(const double* H, int64_t d, int32_t k, double s, double tol,
                             rsign_policy policy, double* R, rsign_info* info, void* stream) {
  return reflector_impl(H, d, k, s, tol, policy, nullptr, R, info, (cudaStream_t)stream);
}

rsign_status rsign_apply(const double* R, int64_t d, const double* V, int64_t nv, double* out,
                         void* stream) {
  if (!R || !V || !out || d < 1 || nv < 1) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = check_device(&sms);
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

rsign_status rsign_reflector_batched(int32_t n, const double* const* H, const int64_t* d,
                                     const int32_t* k, const double* s, double tol,
                                     rsign_policy policy, double* const* R, rsign_info* infos,
                                     void* stream) {
  if (n < 0 || (n > 0 && (!H || !d || !k || !s || !R))) return RSIGN_ERR_ARG;
  rsign_status first = RSIGN_OK;
  for (int32_t i = 0; i < n; ++i) {
    const rsign_status st = rsign_reflector(H[i], d[i], k[i], s[i], tol, policy, R[i],
                                            infos ? &infos[i] : nullptr, stream);
    if (st != RSIGN_OK && first == RSIGN_OK) first = st;
  }
  return first;
}

rsign_status rsign_reflector_backward(const double* H, int64_t d, int32_t k, double s,
                                      rsign_policy policy, const double* Rbar, double* Hbar,
                                      int32_t ckpt_every, void* stream) {
  (void)H; (void)d; (void)k; (void)s; (void)policy; (void)Rbar; (void)Hbar; (void)ckpt_every;
  (void)stream;
  return RSIGN_ERR_UNSUPPORTED;
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

}  // extern "C"

// ------------------------------------------------------------ debug entry points
#include "../../include/rsign_debug.h"

extern "C" {

rsign_status rsign_dbg_tc_gemm(const void* A, const void* B, int64_t dp, int32_t fmt, int32_t sym,
                               float* out, int* status, void* stream) {
  if (!A || !B || !out || !status || dp < 256 || dp % 256 || dp > 16384 || (fmt != 0 && fmt != 1))
    return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  TcGemmArgs a{};
  a.dp = (int)dp; a.d_real = (int)dp; a.sym = sym ? 1 : 0; a.epi = TC_EPI_STORE_F32; a.n_groups = 1;
  a.group_start[0] = 0; a.group_start[1] = 1; a.pair_a[0] = 0; a.pair_b[0] = 0; a.group_scale[0] = 1.0;
  a.scale = 1.0f; a.out = out; a.status = status; a.skip = nullptr;
  return tc_gemm(a, A, 1, B, 1, fmt, sms, (cudaStream_t)stream) == cudaSuccess ? RSIGN_OK : RSIGN_ERR_CUDA;
}

rsign_status rsign_dbg_f64_gemm(const double* A, const double* B, int64_t dp, int32_t sym, double* out,
                                void* stream) {
  if (!A || !B || !out || dp < 64 || dp % 64 || dp > 16384) return RSIGN_ERR_ARG;
  int sms = 0;
  rsign_status ds = check_device(&sms);
  if (ds != RSIGN_OK) return ds;
  F64GemmArgs a{};
  a.dp = (int)dp; a.d_real = (int)dp; a.sym = sym ? 1 : 0; a.epi = F64_EPI_STORE; a.scale = 1.0;
  a.A = A; a.B = B; a.out = out;
  return f64_gemm(a, (cudaStream_t)stream) == cudaSuccess ? RSIGN_OK : RSIGN_ERR_CUDA;
}

}  // extern "C"
