// csp_aggregate_noalloc: overlap-add aggregation that allocates no memory.
//
// csp_aggregate keeps the synthesized patches x_hat_p in a workspace buffer
// that the context grows with cudaMalloc on first use.  Some callers cannot
// allocate device memory at the point where they aggregate: code running
// while a CUDA stream is being captured into a graph, allocators that own all
// of the device memory and forbid other allocations after start-up, or
// real-time loops that must not stall on the driver.  This entry point does
// the same two launches (synthesis, then per-pixel average) with the scratch
// held in a fixed array in the library's device image instead.
//
// The array holds kNoAllocScratchFloats floats (16 MiB) and exists on every
// GPU that loads this library, until the process exits.  Its device address is
// looked up when a context is created on the device (csp_create), which is also
// when the driver loads the array's module and reserves the memory; if that
// lookup failed, the entry point's first call on the device repeats it, and
// such a first call should then come before any stream capture.  Calls are limited to
// B * N0 <= kNoAllocScratchFloats.  All calls share the array: calls whose
// work overlaps on the GPU (different streams, or different contexts on the
// same device) race on it.  The array keeps the last call's contents; every
// entry a call reads is first written by that call (the synthesis kernel
// writes all B * N0 values before the average reads them), so nothing needs
// clearing.
#include <string>

#include "csp_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchFloats = size_t(4) << 20;  // 16 MiB of float32

__device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

// Device address of the scratch array, looked up once per device with that
// device current (host code cannot use the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices] = {};

// Looks up (once per device, with `dev` current) the device address of the
// scratch array.  Looking it up loads the array's module, which is when the
// driver reserves its 16 MiB; csp_create calls this so that the memory is
// taken at set-up and no later call of the entry point allocates anything.
cudaError_t scratch_lookup(int dev) {
  if (g_scratch_addr[dev]) return cudaSuccess;
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaSuccess && p) g_scratch_addr[dev] = static_cast<float *>(p);
  return e == cudaSuccess && !p ? cudaErrorInvalidSymbol : e;
}

}  // namespace

namespace csp {
void noalloc_setup(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return;
  if (scratch_lookup(dev) != cudaSuccess) cudaGetLastError();  // the entry point retries and reports
}
}  // namespace csp

extern "C" csp_status csp_aggregate_noalloc(csp_ctx *ctx, const int32_t *support, const float *coef,
                                           const int8_t *k_eff, int64_t B, int Kmax, float *image_out,
                                           void *stream) {
  if (!ctx) return CSP_ERR_INVALID;
  auto fail = [&](csp_status st, const std::string &m) {
    ctx->err = m;
    return st;
  };
  if (!ctx->has_geom) return fail(CSP_ERR_NOT_READY, "geometry not set");
  if (!ctx->lv[0].D) return fail(CSP_ERR_NOT_READY, "fine dictionary not loaded");
  if (B != ctx->B) return fail(CSP_ERR_INVALID, "B must equal the geometry's patch count");
  if (Kmax < 1 || Kmax > CSP_MAX_K) return fail(CSP_ERR_INVALID, "Kmax must be in 1..CSP_MAX_K");
  if (!support || !coef || !k_eff || !image_out) return fail(CSP_ERR_INVALID, "NULL buffer");
  const int N0 = ctx->lv[0].N;
  if ((size_t)B * (size_t)N0 > kNoAllocScratchFloats)
    return fail(CSP_ERR_INVALID, "csp_aggregate_noalloc: B * N0 = " + std::to_string((size_t)B * N0) +
                                     " exceeds the fixed scratch of " + std::to_string(kNoAllocScratchFloats) +
                                     " floats; use csp_aggregate");
  const int dev = ctx->device;
  if (dev < 0 || dev >= kMaxDevices) return fail(CSP_ERR_UNSUPPORTED, "device index beyond the scratch table");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fail(CSP_ERR_CUDA, "cudaGetDevice failed");
  if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return fail(CSP_ERR_CUDA, "cudaSetDevice failed");
  csp_status st = CSP_OK;
  if (!g_scratch_addr[dev]) {  // normally done by csp_create; retried here if that lookup failed
    const cudaError_t e = scratch_lookup(dev);
    if (e != cudaSuccess) st = fail(CSP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  }
  if (st == CSP_OK) {
    csp::launch_aggregate(ctx->gd, ctx->lv[0].D, N0, support, coef, k_eff, Kmax, ctx->cover_y, ctx->cover_x,
                          g_scratch_addr[dev], image_out, (cudaStream_t)stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(CSP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    else ctx->launches[csp::KK_AGGREGATE] += 1;
  }
  if (prev != dev) cudaSetDevice(prev);
  return st;
}
