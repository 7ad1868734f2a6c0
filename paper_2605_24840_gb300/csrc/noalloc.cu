// noalloc.cu -- rsign_reflector_noalloc: the FP64-policy reflector for small
// matrices without any device allocation.
//
// Some callers cannot call cudaMalloc (or let a library call it) inside their
// own work: code running inside a stream-ordered region whose allocations are
// planned up front, embedders whose memory budget is fixed at start-up, or
// host threads that must not synchronise with the allocator.  For them this
// entry point takes its workspace from one statically sized device array,
// defined in this file, instead of allocating.
//
// Ownership and limits:
//  - the array `g_noalloc_scratch` (kNoallocScratchBytes bytes) is part of
//    the library image: every GPU that loads librsign holds it until the
//    process exits;
//  - orders up to kNoallocMaxD (512) fit: the FP64 path needs A = H - sI,
//    two iterate buffers, E = I - X^2 (each dp x dp FP64, dp = d rounded up
//    to a multiple of 256) plus small reduction arrays;
//  - every call reuses the same array and the array keeps the previous
//    call's contents; the control block that must start at zero is cleared
//    by each call, and every other region is fully rewritten before it is
//    read;
//  - calls that overlap on the GPU (concurrent streams, several host
//    threads, several calls in flight on different streams) share the array
//    and race: serialise them.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current (host code may not
// use the symbol itself: in host code it is only a stand-in).  That first
// call should come before any stream capture begins.
#include "common.cuh"
#include "kernels.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace rsign {
namespace {

constexpr int kNoallocMaxD = 512;
constexpr int kNoallocMaxDp = 512;
constexpr int kNoallocMaxSteps = 100;
constexpr size_t kNoallocDd = (size_t)kNoallocMaxDp * kNoallocMaxDp;

struct NoallocCtl {
  int status, flags, done, steps;
  double scal[8];  // [0] ||A||_inf  [1] alpha  [2] trace
};

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// layout of the scratch array (offsets in bytes)
constexpr size_t kOffCtl = 0;
constexpr size_t kOffHist = align256(kOffCtl + sizeof(NoallocCtl));
constexpr size_t kOffPart = align256(kOffHist + (kNoallocMaxSteps + 2) * sizeof(double));
constexpr size_t kOffRowsum = align256(kOffPart + 64 * 1024);
constexpr size_t kOffRowpart = align256(kOffRowsum + kNoallocMaxDp * sizeof(double));
constexpr size_t kOffA = align256(kOffRowpart + (kNoallocMaxDp / 32) * kNoallocMaxDp * sizeof(double));
constexpr size_t kOffX0 = align256(kOffA + kNoallocDd * sizeof(double));
constexpr size_t kOffX1 = align256(kOffX0 + kNoallocDd * sizeof(double));
constexpr size_t kOffE = align256(kOffX1 + kNoallocDd * sizeof(double));
constexpr size_t kNoallocScratchBytes = align256(kOffE + kNoallocDd * sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

bool device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace rsign

using namespace rsign;

extern "C" rsign_status rsign_reflector_noalloc(const double* H, int64_t d64, int32_t k, double s,
                                                double tol, double* R, rsign_info* info, void* stream) {
  if (!H || !R) return RSIGN_ERR_ARG;
  if (d64 < 2) return RSIGN_ERR_ARG;
  if (d64 > kNoallocMaxD) return RSIGN_ERR_UNSUPPORTED;  // larger than the static workspace
  if (k < 1 || k > d64 - 1) return RSIGN_ERR_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol) || !std::isfinite(s)) return RSIGN_ERR_ARG;
  if (!device_pointer(H) || !device_pointer(R)) return RSIGN_ERR_ARG;  // no host staging buffers
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return RSIGN_ERR_CUDA; }
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return RSIGN_ERR_UNSUPPORTED;

  unsigned char* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) { cudaGetLastError(); return RSIGN_ERR_CUDA; }
  cudaStream_t st = (cudaStream_t)stream;
  const int d = (int)d64;
  const int dp = (d + 255) / 256 * 256;
  const size_t dd = (size_t)dp * dp;
  const double tol_fro = std::fmax(tol, 16.0 * d * 2.220446049250313e-16);

  NoallocCtl* ctl = reinterpret_cast<NoallocCtl*>(base + kOffCtl);
  double* hist = reinterpret_cast<double*>(base + kOffHist);
  double* partials = reinterpret_cast<double*>(base + kOffPart);
  double* rowsum = reinterpret_cast<double*>(base + kOffRowsum);
  double* rowpart = reinterpret_cast<double*>(base + kOffRowpart);
  double* A = reinterpret_cast<double*>(base + kOffA);
  double* xb[2] = {reinterpret_cast<double*>(base + kOffX0), reinterpret_cast<double*>(base + kOffX1)};
  double* E = reinterpret_cast<double*>(base + kOffE);

  NoallocCtl h;
  std::memset(&h, 0, sizeof(h));
  auto fail = [&]() {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return RSIGN_ERR_CUDA;
  };
  // the control block is the only region read before it is written
  if (cudaMemsetAsync(ctl, 0, sizeof(NoallocCtl), st) != cudaSuccess) return fail();
  if (ingest(H, d, dp, s, A, rowpart, &ctl->flags, st) != cudaSuccess) return fail();
  if (inf_norm_finish(rowpart, dp, rowsum, ctl->scal, st) != cudaSuccess) return fail();
  if (cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail();
  if ((h.flags & 1) || !(h.scal[1] > 0.0) || !std::isfinite(h.scal[1])) return RSIGN_ERR_ARG;
  if (scale_convert(A, dd, ctl->scal + 1, 1.0, xb[0], 2, st) != cudaSuccess) return fail();

  // FP64 Newton-Schulz (Eq. NS, update form) with the device-side stop test
  const int nt = f64_num_tiles(dp, 1);
  int m = 0;
  bool stopped = false;
  while (m <= kNoallocMaxSteps && !stopped) {
    const int m_end = (m + 8 < kNoallocMaxSteps + 1) ? m + 8 : kNoallocMaxSteps + 1;
    for (int mm = m; mm < m_end; ++mm) {
      F64GemmArgs sy{};
      sy.dp = dp; sy.d_real = d; sy.sym = 1; sy.epi = F64_EPI_NS_SYRK;
      sy.A = xb[mm & 1]; sy.B = xb[mm & 1]; sy.out = E; sy.partials = partials; sy.skip = &ctl->done;
      if (f64_gemm(sy, st) != cudaSuccess) return fail();
      if (ns_check(partials, nt * 4, hist, mm, tol_fro, -1.0, -1.0, 0.0, &ctl->done, &ctl->steps, st) !=
          cudaSuccess)
        return fail();
      if (mm == kNoallocMaxSteps) break;
      F64GemmArgs up{};
      up.dp = dp; up.d_real = d; up.sym = 1; up.epi = F64_EPI_NS_UPDATE;
      up.A = xb[mm & 1]; up.B = E; up.xin = xb[mm & 1]; up.out = xb[(mm + 1) & 1];
      up.partials = partials; up.skip = &ctl->done;
      if (f64_gemm(up, st) != cudaSuccess) return fail();
    }
    if (cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail();
    stopped = h.done != 0;
    m = m_end;
  }
  const int steps = stopped ? h.steps : kNoallocMaxSteps;
  double* X = xb[steps & 1];
  if (trace_f64(X, dp, d, ctl->scal + 2, st) != cudaSuccess) return fail();
  if (copy_unpad(X, dp, R, d, st) != cudaSuccess) return fail();
  double resid = NAN;
  if (cudaMemcpyAsync(&resid, hist + steps, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail();
  const double trace = h.scal[2];
  const bool trace_ok = std::fabs(trace - (double)(d - 2 * k)) < 0.5;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->steps_fp64 = steps;
    info->cert_ok = (trace_ok && stopped && resid <= tol_fro) ? 1 : 0;
    info->alpha = h.scal[1];
    info->shift = s;
    info->gamma_est = NAN;
    info->resid_fro = resid;
    info->trace = trace;
    info->correction_fro = NAN;
    info->commutator_norm = NAN;
    info->err_est = NAN;
    info->err_bound = NAN;
    info->tol_fro = tol_fro;
    // kernels issued: ingest, the two of the inf-norm reduction, the FP64
    // copy of X_0, three per step of every 8-step chunk enqueued (the ones
    // after the device-side stop return at once), trace and output copy
    info->launches = 6 + 3 * (int64_t)m;
    info->workspace_bytes = 0;
  }
  if (!stopped) return RSIGN_ERR_NOCONV;
  if (!trace_ok) return RSIGN_ERR_CERT;
  return RSIGN_OK;
}
