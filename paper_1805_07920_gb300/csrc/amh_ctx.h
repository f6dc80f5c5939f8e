// amh_ctx.h -- the context behind the opaque amh_ctx handle of amh.h
// (private to the library's translation units).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "amh.h"
#include "amh_device.cuh"

struct amh_ctx {
  amh_params p;
  int W = 0, H = 0, N = 0, ref = 0;
  int device = 0;                         // the CUDA device current at amh_create
  int src[AMH_MAX_SRC];
  cudaStream_t stream = nullptr;
  cudaArray_t arr[AMH_MAX_SRC] = {};      // source views, uint8 texture arrays
  cudaTextureObject_t tex[AMH_MAX_SRC] = {};
  void* d_ref = nullptr;                  // reference image (uint8 or FP16)
  float4* d_plane = nullptr;
  float* d_cost = nullptr;
  uint32_t* d_sel = nullptr;
  uint8_t* d_vbest = nullptr;
  uint32_t* d_wmask = nullptr;
  uint8_t* d_choice = nullptr;
  unsigned long long* d_pairs = nullptr;  // amh::kPairCounters striped counters
  float4* d_prop = nullptr;               // caller-set proposals (amh_set_proposal)
  unsigned int* d_status = nullptr;       // bounds-check status word (bounds-checked builds)
  size_t prop_cap = 0;                    // cells d_prop holds
  amh::PhaseArgs args;
  int t = 0;
  bool initialized = false;
  std::string err;
};

namespace amh {
// Message for amh_last_error(NULL): the last failure of a call that has no
// context (amh_create, amh_median4, amh_fuse, amh_select_sources) on this
// host thread.  Returns code.
int fail_no_context(int code, const char* fmt, ...);
}  // namespace amh

