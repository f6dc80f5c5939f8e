// amh_gather_peak.cu -- the texture-gather ceiling of the GPU, measured: a
// loop that does nothing but gather (one tex2Dgather of a uint8 texture per
// "window sample" and two additions) over windows laid out like the update's
// (lanes of a warp on neighbouring pixels, 36 samples at stride 2), with 16
// warps per SM.  Its sample rate is the denominator of the update's fetch
// roofline: the update needs one gather per window sample.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "amh.h"

namespace amh {
namespace {

constexpr int kPairsPerThread = 64;

__global__ void __launch_bounds__(512) gather_loop_kernel(cudaTextureObject_t t, int W, int H, float* out) {
  const int l = threadIdx.x & 31, w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nbx = (W - 200) / 8;
  const float x = (float)((w % nbx) * 8 + 80 + (l & 1) * 6 + ((l >> 2) & 7) / 3);
  const float y = (float)(((w / nbx) * 2) % (H - 200) + 80 + ((l >> 1) & 1) * 6 + ((l >> 2) & 7) % 3);
  float acc = 0.f, acc2 = 0.f;
  for (int p = 0; p < kPairsPerThread; p++) {
    const float bx = x + (float)(p & 7), by = y + (float)(p >> 3);
#pragma unroll
    for (int k = 0; k < 36; k++) {
      const float4 g = tex2Dgather<float4>(t, bx + (float)(2 * (k % 6)), by + (float)(2 * (k / 6)), 0);
      acc += g.x;
      acc2 += g.w;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc + acc2;
}

}  // namespace
}  // namespace amh

using namespace amh;

extern "C" AMH_API int amh_gather_peak(double* samples_per_s) {
  if (!samples_per_s) return AMH_EINVAL;
  *samples_per_s = 0.0;
  const int W = 3200, H = 2112;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return AMH_ECUDA;
  std::vector<uint8_t> img((size_t)W * H);
  uint32_t s = 12345u;
  for (auto& v : img) {
    s = s * 1664525u + 1013904223u;
    v = (uint8_t)(s >> 24);
  }
  cudaArray_t arr = nullptr;
  cudaTextureObject_t tex = 0;
  float* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  const int threads = 512, blocks = sms * 4;
  int rc = AMH_ECUDA;
  cudaChannelFormatDesc fd = cudaCreateChannelDesc<uint8_t>();
  cudaResourceDesc rd;
  cudaTextureDesc td;
  std::memset(&rd, 0, sizeof rd);
  std::memset(&td, 0, sizeof td);
  float ms = 0.f;
  if (cudaMallocArray(&arr, &fd, W, H, cudaArrayTextureGather) != cudaSuccess) goto done;
  if (cudaMemcpy2DToArray(arr, 0, 0, img.data(), W, W, H, cudaMemcpyHostToDevice) != cudaSuccess) goto done;
  rd.resType = cudaResourceTypeArray;
  rd.res.array.array = arr;
  td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
  td.filterMode = cudaFilterModePoint;
  td.readMode = cudaReadModeNormalizedFloat;
  if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) != cudaSuccess) goto done;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) goto done;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) goto done;
  gather_loop_kernel<<<blocks, threads>>>(tex, W, H, out);   // warm-up
  cudaEventRecord(a);
  for (int r = 0; r < 3; r++) gather_loop_kernel<<<blocks, threads>>>(tex, W, H, out);
  cudaEventRecord(b);
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f) goto done;
  *samples_per_s = 3.0 * blocks * threads * (double)kPairsPerThread * 36.0 / (ms * 1e-3);
  rc = AMH_OK;
done:
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (tex) cudaDestroyTextureObject(tex);
  if (arr) cudaFreeArray(arr);
  return rc;
}
