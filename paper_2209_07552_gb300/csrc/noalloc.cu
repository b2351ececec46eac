// msrep_spmv_noalloc: msrep_spmv with its workspace taken from a scratch
// array compiled into the library, for callers that cannot allocate device
// memory (see include/msrep.h).  The SpMV itself is msrep_spmv's.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"

namespace msrep {

// The scratch array: one per GPU that loads the library, alive until exit.
// Host code must not take its address directly (on the host the name is
// only a stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MSREP_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[128] = {nullptr};

// Device address of the scratch array on the current device.  It is looked
// up again on every call made outside a stream capture, so a context that
// was destroyed and recreated (cudaDeviceReset) never leaves a stale address
// behind; during a capture (where the call must not depend on a runtime
// query) the address from the device's last uncaptured call is used, so the
// first call on a device must come before any capture.
static msrep_status noalloc_scratch(cudaStream_t st, void **out) {
  int dev = 0;
  MSREP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(MSREP_ERR_CUDA, "device ordinal %d out of range", dev);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MSREP_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(MSREP_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  } else if (!g_noalloc_addr[dev]) {
    return fail(MSREP_ERR_INVALID_ARG,
                "msrep_spmv_noalloc was first called on device %d inside a stream capture; "
                "call it once before capturing",
                dev);
  }
  *out = g_noalloc_addr[dev];
  return MSREP_OK;
}

}  // namespace msrep

using namespace msrep;

extern "C" {

msrep_status msrep_spmv_noalloc(const msrep_matrix *A, const msrep_partition *part,
                                double alpha, const void *x, double beta, void *y,
                                int32_t xy_dtype, unsigned flags, void *stream) {
  // The permuted CSC accumulator is used when it fits in the scratch array;
  // otherwise a CSC SpMV scatters into y directly (same result up to the
  // order of additions), so the limit below is the one without it.
  size_t full = 0, need = 0;
  MSREP_TRY(spmv_workspace_bytes(A, part, true, &full));
  const bool perm_ok = full <= MSREP_NOALLOC_SCRATCH_BYTES;
  MSREP_TRY(spmv_workspace_bytes(A, part, perm_ok, &need));
  if (need > MSREP_NOALLOC_SCRATCH_BYTES)
    return fail(MSREP_ERR_WORKSPACE,
                "this SpMV needs %zu bytes of scratch; the built-in array holds %u "
                "(use msrep_spmv with a caller workspace, or a larger tile)",
                need, MSREP_NOALLOC_SCRATCH_BYTES);
  void *scratch = nullptr;
  MSREP_TRY(noalloc_scratch(as_stream(stream), &scratch));
  return spmv_run(A, part, alpha, x, beta, y, xy_dtype, flags, scratch, stream, perm_ok);
}

}  // extern "C"
