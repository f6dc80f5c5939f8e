// amh_noalloc.cu -- map read-back into host buffers that allocates nothing.
//
// amh_read_maps() with host buffers stages the depth and normal maps in a
// device buffer it allocates for the call.  Some callers cannot allocate
// device memory at that point: hosts that hand the GPU to a pooling allocator
// and forbid any other device allocation, and real-time loops that must not
// allocate after start-up.  This variant stages through one fixed scratch
// array that is part of the library's device image instead.  It blocks (it
// synchronises the context's stream and copies into pageable host memory), so
// it is called outside stream capture.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "amh.h"
#include "amh_ctx.h"

namespace {

constexpr int64_t kMaxPixels = AMH_NOALLOC_MAX_PIXELS;

// Scratch: depth of up to kMaxPixels pixels, then their normals (3 floats
// each): 4 MB held on every GPU that loads this library, until exit.
static __device__ __align__(256) float g_noalloc_scratch[4 * kMaxPixels];

// Device address of g_noalloc_scratch, per device (looked up once, with that
// device current; host code cannot use the symbol itself as an address).
constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// pixels first .. first + n - 1 in row-major order, read from the state
// (amh::state_index layout)
__global__ void split_maps_to_scratch(const float4* __restrict__ plane, int W, int64_t first, int64_t n,
                                      float* __restrict__ scratch) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t px = first + i;
    const float4 p = plane[amh::state_index((int)(px % W), (int)(px / W), W)];
    scratch[i] = p.w;
    scratch[kMaxPixels + 3 * i] = p.x;
    scratch[kMaxPixels + 3 * i + 1] = p.y;
    scratch[kMaxPixels + 3 * i + 2] = p.z;
  }
}

int set_err(amh_ctx* c, int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "%s", msg);
  c->err = buf;
  return code;
}

}  // namespace

extern "C" AMH_API int amh_read_maps_noalloc(amh_ctx* c, float* depth, float* normal3, int64_t first_pixel,
                                             int64_t n_pixels) {
  if (!c) return AMH_EINVAL;
  const int64_t np = (int64_t)c->W * c->H;
  if (!depth && !normal3) return set_err(c, AMH_EINVAL, "amh_read_maps_noalloc: depth and normal3 are both NULL");
  if (first_pixel < 0 || n_pixels < 0 || first_pixel > np || n_pixels > np - first_pixel)
    return set_err(c, AMH_EINVAL, "amh_read_maps_noalloc: pixel range outside the image");
  if (n_pixels > kMaxPixels)
    return set_err(c, AMH_EINVAL,
                   "amh_read_maps_noalloc: at most AMH_NOALLOC_MAX_PIXELS (262144) pixels per call; "
                   "read larger maps in slices");
  if (n_pixels == 0) return AMH_OK;

  // the context's device (recorded at amh_create), made current for the
  // set-up and the launch
  const int dev = c->device;
  if (dev < 0 || dev >= kMaxDevices) return set_err(c, AMH_EINVAL, "amh_read_maps_noalloc: device index too large");
  cudaError_t e;
  int prev = 0;
  e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: cudaGetDevice", e);
  if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
    return set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: cudaSetDevice", e);

  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        if (prev != dev) cudaSetDevice(prev);
        return set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: cudaGetSymbolAddress of the scratch array", e);
      }
      g_scratch_ptr[dev] = (float*)p;
    }
    scratch = g_scratch_ptr[dev];
  }

  int rc = AMH_OK;
  const int blocks = (int)((n_pixels + 255) / 256 < 1024 ? (n_pixels + 255) / 256 : 1024);
  split_maps_to_scratch<<<blocks, 256, 0, c->stream>>>(c->d_plane, c->W, first_pixel, n_pixels, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) rc = set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: launch", e);
  if (!rc && depth) {
    e = cudaMemcpyAsync(depth, scratch, (size_t)n_pixels * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) rc = set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: depth copy", e);
  }
  if (!rc && normal3) {
    e = cudaMemcpyAsync(normal3, scratch + kMaxPixels, (size_t)n_pixels * 3 * sizeof(float),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) rc = set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: normal copy", e);
  }
  if (!rc) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = set_err(c, AMH_ECUDA, "amh_read_maps_noalloc: synchronize", e);
  }
  if (prev != dev) cudaSetDevice(prev);
  return rc;
}
