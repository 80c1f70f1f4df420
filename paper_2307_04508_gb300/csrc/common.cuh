// Shared helpers for the LT-GW CUDA library: status plumbing, launch
// accounting and the per-context workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/ltgw.h"

namespace ltgw {

// Kernel launches issued by this process (host-side counter, read per solve).
extern int g_launch_count;

inline void count_launch() { ++g_launch_count; }

struct Status {
  ltgw_status code = LTGW_OK;
  std::string msg;
};

// Record a CUDA error (if any) as LTGW_ERR_DEVICE with the call site.
#define LTGW_CUDA(ctx, call)                                                        \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess) {                                                        \
      (ctx)->fail(LTGW_ERR_DEVICE, std::string(#call) + ": " + cudaGetErrorString(_e)); \
      return (ctx)->status();                                                       \
    }                                                                               \
  } while (0)

#define LTGW_LAUNCHED(ctx)                                                          \
  do {                                                                              \
    ::ltgw::count_launch();                                                         \
    cudaError_t _e = cudaGetLastError();                                            \
    if (_e != cudaSuccess) {                                                        \
      (ctx)->fail(LTGW_ERR_DEVICE, std::string("kernel launch at ") + __FILE__ + ":" + \
                                       std::to_string(__LINE__) + ": " + cudaGetErrorString(_e)); \
      return (ctx)->status();                                                       \
    }                                                                               \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Device-side error flags written by kernels (one int each, zeroed per solve).
enum DeviceFlag { FLAG_NOT_SPD = 0, FLAG_EIG = 1, FLAG_NONFINITE = 2, FLAG_TC_TIMEOUT = 3, FLAG_COUNT = 8 };

}  // namespace ltgw
