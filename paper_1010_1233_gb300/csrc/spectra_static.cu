// Correlator sampling for callers that cannot allocate device memory.
//
// flb_spectra_accumulate needs a scratch block from its caller.  Some callers
// cannot provide one: a host application whose framework owns the whole device
// memory budget through its own pool and forbids direct allocations, a service
// running under a fixed per-process memory cap, or a latency-critical loop that
// must not pay for cudaMalloc / cudaFree and the device-wide synchronisation
// they imply.  flb_spectra_accumulate_static does the same work with its scratch
// in a file-scope device array of fixed size (kStaticScratchBytes), so the
// caller only passes the fields and the output sums.
//
// The array is part of the library image: every GPU that loads the library holds
// it until the process exits.  All calls on a device share it, and it keeps the
// contents of the last call; each call rewrites everything it reads (plan,
// twiddles, row transforms), so nothing needs clearing between calls.  Calls
// whose work overlaps on the GPU (different streams, or other threads) race on
// the array and give wrong results: serialise them.
#include <mutex>

#include "flb_internal.cuh"
#include "spectra_plan.cuh"

namespace flb {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_spectra_scratch[kStaticScratchBytes];

// Device address of g_spectra_scratch on the current device.  In host code the
// symbol names a host-side stand-in, so the address is looked up with that device
// current: on the first call there, and again on every call made outside a stream
// capture (after a cudaDeviceReset the module is loaded again, possibly elsewhere);
// a call made while its stream is being captured uses the address found last.
static int static_scratch(cudaStream_t st, char** out) {
  static std::mutex mu;
  static char* addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FLB_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(FLB_EINVAL, "device %d beyond the %d supported", dev, kMaxDevices);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return set_error(FLB_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev] || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_spectra_scratch);
    if (e != cudaSuccess || !p)
      return set_error(FLB_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    addr[dev] = static_cast<char*>(p);
  }
  *out = addr[dev];
  return FLB_OK;
}

}  // namespace flb

using namespace flb;

extern "C" int flb_spectra_accumulate_static(int precision, int nx, int ny, int n_fields, const void* fields_dev,
                                             double* pair_sums_dev, double* mean0_dev, void* cuda_stream) {
  SpectraPlan P;
  int rc = spectra_plan(precision, nx, ny, n_fields, P);
  if (rc) return rc;
  if (!fields_dev || !pair_sums_dev || !mean0_dev) return set_error(FLB_EINVAL, "NULL pointer");
  if (P.scratch_bytes > kStaticScratchBytes)
    return set_error(FLB_EINVAL,
                     "%d fields of %d x %d need %zu bytes of scratch, more than the %zu-byte static array of "
                     "flb_spectra_accumulate_static; use flb_spectra_accumulate with caller scratch",
                     n_fields, nx, ny, P.scratch_bytes, kStaticScratchBytes);
  char* scratch = nullptr;
  rc = static_scratch(static_cast<cudaStream_t>(cuda_stream), &scratch);
  if (rc) return rc;
  return spectra_launch(precision, P, scratch, fields_dev, pair_sums_dev, mean0_dev,
                        static_cast<cudaStream_t>(cuda_stream));
}
