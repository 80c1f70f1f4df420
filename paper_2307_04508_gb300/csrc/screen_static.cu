// Allocation-free variant of the screening step: C_j = [1 - Pi_j]^-1 - 1 with
// the sweep operator, its two ping-pong buffers and its error flag held in a
// fixed file-scope device array instead of memory obtained from cudaMalloc.
//
// For callers that cannot allocate device memory at the point of the call:
// processes whose device memory is already claimed in full by another
// allocator (a framework's caching allocator, a pre-reserved pool), and
// latency-sensitive callers that cannot afford cudaMalloc/cudaFree, which may
// block and synchronise the device.  The caller still provides Pi and C.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

// Two sweep buffers of LTGW_SCREEN_STATIC_MAX_ELEMS doubles each, then flags.
constexpr size_t kMaxElems = LTGW_SCREEN_STATIC_MAX_ELEMS;
constexpr size_t kFlagDoubles = 8;  // room for ltgw::FLAG_COUNT ints
static_assert(ltgw::FLAG_COUNT * sizeof(int) <= kFlagDoubles * sizeof(double),
              "the flag tail of the scratch array must hold every device flag");
static __device__ __align__(256) double g_screen_scratch[2 * kMaxElems + kFlagDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};  // device address of g_screen_scratch, per device

// Device address of the scratch array on the current device.  The array's
// name in host code is only a stand-in, so the address is looked up with
// cudaGetSymbolAddress: on every call made outside stream capture (a device
// reset or a re-created primary context reloads the module and moves the
// array), and from the per-device cache while `s` is capturing, where the
// lookup's implicit module load must not run.
cudaError_t scratch_address(int dev, cudaStream_t s, double **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return cudaGetLastError();
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_screen_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ltgw_status ltgw_screen_static(int N, int n_omega, const double *Pi, double *C,
                                          void *stream) {
  if (N < 1 || n_omega < 1 || !Pi || !C || Pi == C) return LTGW_ERR_BAD_ARG;
  if ((size_t)n_omega * (size_t)N * (size_t)N > kMaxElems) return LTGW_ERR_BAD_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *base = nullptr;
  if (scratch_address(dev, s, &base) != cudaSuccess) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  double *X0 = base, *X1 = base + kMaxElems;
  int *flags = reinterpret_cast<int *>(base + 2 * kMaxElems);
  // the array keeps the previous call's contents: the flags must start at zero
  if (cudaMemsetAsync(flags, 0, ltgw::FLAG_COUNT * sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  int launches = 0;
  if (ltgw::launch_screen(Pi, N, n_omega, X0, X1, C, flags, s, &launches) != cudaSuccess) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  int h[ltgw::FLAG_COUNT];
  if (cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return LTGW_ERR_DEVICE;
  }
  return h[ltgw::FLAG_NOT_SPD] ? LTGW_ERR_NOT_SPD : LTGW_OK;
}
