// Scope of one call of the C ABI (internal to libqcd).
//
// Every entry point that takes a context opens one: it names the call in an NVTX range (seen by
// Nsight Systems and by `ncu --nvtx`; a no-op when no tool is attached), makes the context's device
// current for the duration of the call and restores the caller's current device when the call
// returns, so that a caller driving several GPUs from one thread keeps its own device selection.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "qcd.h"

namespace qcd {

qcd_status set_error(qcd_status s, const char* msg);

class ApiScope {
 public:
  // device < 0: no context (the call fails with QCD_ERR_ARG "null context")
  ApiScope(const char* name, int device) {
    nvtxRangePushA(name);
    if (device < 0) {
      status_ = set_error(QCD_ERR_ARG, "null context");
      return;
    }
    if (cudaGetDevice(&prev_) != cudaSuccess) {
      cudaGetLastError();
      prev_ = -1;
    }
    if (prev_ != device) {
      const cudaError_t e = cudaSetDevice(device);
      if (e != cudaSuccess) {
        status_ = set_error(QCD_ERR_CUDA, cudaGetErrorString(e));
        return;
      }
      restore_ = prev_ >= 0;
    }
  }
  ~ApiScope() {
    if (restore_ && cudaSetDevice(prev_) != cudaSuccess) cudaGetLastError();
    nvtxRangePop();
  }
  ApiScope(const ApiScope&) = delete;
  ApiScope& operator=(const ApiScope&) = delete;
  qcd_status status() const { return status_; }

 private:
  int prev_ = -1;
  bool restore_ = false;
  qcd_status status_ = QCD_OK;
};

}  // namespace qcd
