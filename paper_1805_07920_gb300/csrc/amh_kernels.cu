// amh_kernels.cu -- kernels of the single-reference context: random
// initialisation and one colour phase over a 16 x 16 tile per block (the
// update itself is in amh_update.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "amh_device.cuh"
#include "amh_kernels.h"
#include "amh_update.cuh"

namespace amh {
namespace {
using namespace upd;

constexpr int kTile = 16;
constexpr int kThreads = 128;
constexpr int kPhaseBlocksPerSM = 3;          // 168 registers per thread

// npairs: evaluations of this thread, plus 2^16 for each one sampled from a
// shared-memory box (fewer than 2^11 per thread and launch); the two totals
// go to the first and the second kPairCounters counters
__device__ __forceinline__ void count_pairs(const PhaseArgs& a, int npairs) {
  const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)npairs & 0xFFFFu);
  const unsigned hi = __reduce_add_sync(0xffffffffu, (unsigned)npairs >> 16);
  const int k = (blockIdx.x * 4 + (threadIdx.x >> 5) + blockIdx.y * 7) % kPairCounters;
  if ((threadIdx.x & 31) == 0 && lo) atomicAdd(&a.pairs[k], (unsigned long long)lo);
  if ((threadIdx.x & 31) == 0 && hi) atomicAdd(&a.pairs[kPairCounters + k], (unsigned long long)hi);
}

template <bool kHalf, int kMode>
__global__ void __launch_bounds__(kThreads, kPhaseBlocksPerSM) phase_kernel(const __grid_constant__ PhaseArgs a) {
  PixelArrays sm;
  const int tid = threadIdx.x;
  int npairs = 0;
  if constexpr ((kMode & kStage) != 0) {
    // Warp w updates rows 4w .. 4w + 3 of the tile (8 pixels of the colour
    // per row); each quarter-warp takes 4 pixels of two neighbouring rows, so
    // the 8 lanes of a 16-byte shared load sample 8 distinct columns modulo
    // 8 of the box where the view maps the tile at unit scale.
    const int lane = tid & 31, q = lane >> 3;
    const int y = blockIdx.y * kTile + 4 * (tid >> 5) + 2 * (q >> 1) + ((lane >> 2) & 1);
    const int x = blockIdx.x * kTile + 2 * (4 * (q & 1) + (lane & 3)) + ((y + a.color) & 1);
    // the whole block takes part in the staged sweep, pixels outside the image too
    __shared__ StageShared ss;
    update_pixel<kHalf, kMode>(a, sm, x, y, &npairs, &ss, x < a.W && y < a.H);
  } else {
    const int y = blockIdx.y * kTile + (tid >> 3);
    const int x = blockIdx.x * kTile + 2 * (tid & 7) + ((y + a.color) & 1);
    if (x < a.W && y < a.H) update_pixel<kHalf, kMode>(a, sm, x, y, &npairs);
  }
  count_pairs(a, npairs);
}

// Random initialisation: one thread per pixel over the whole image.
template <bool kHalf, bool kTex>
__global__ void __launch_bounds__(kThreads) init_kernel(const __grid_constant__ PhaseArgs a) {
  PixelArrays sm;
  const int x = blockIdx.x * kTile + (threadIdx.x & 15), y = blockIdx.y * 8 + (threadIdx.x >> 4);
  int npairs = 0;
  if (x < a.W && y < a.H) init_pixel<kHalf, kTex>(a, sm, x, y, &npairs);
  count_pairs(a, npairs);
}


}  // namespace

// Both kernels use no shared memory: ask for the largest L1 (texture cache).
// The preference is per device, so it is set once for each device that
// launches the kernel.
template <typename K>
void prefer_l1(K kernel, std::once_flag* once) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::call_once(once[dev & 63], [kernel] {
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  });
}

template <bool kHalf, bool kTex>
int launch_init_t(const PhaseArgs& a, cudaStream_t s) {
  static std::once_flag once[64];
  prefer_l1(init_kernel<kHalf, kTex>, once);
  dim3 grid((a.W + kTile - 1) / kTile, (a.H + 7) / 8);
  init_kernel<kHalf, kTex><<<grid, kThreads, 0, s>>>(a);
  return (int)cudaGetLastError();
}
// the texture-filter form exists for uint8 images only (the context refuses
// it with FP16 images and with the ablations)
int launch_init(const PhaseArgs& a, cudaStream_t s) {
  if (a.tex_filter) return launch_init_t<false, true>(a, s);
  return a.img_half ? launch_init_t<true, false>(a, s) : launch_init_t<false, false>(a, s);
}

template <bool kHalf, int kMode>
int launch_phase_t(const PhaseArgs& a, cudaStream_t s) {
  static std::once_flag once[64];
  if ((kMode & kStage) == 0) {
    prefer_l1(phase_kernel<kHalf, kMode>, once);
  } else {
    // the smallest carve-out that holds the staged blocks' shared memory: the
    // rest of the unified L1 stays texture and local-memory cache
    int dev = 0;
    cudaGetDevice(&dev);
    std::call_once(once[dev & 63], [] {
      int d = 0, smem_sm = 0;
      cudaGetDevice(&d);
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
      const int need = kPhaseBlocksPerSM * (int)(sizeof(StageShared) + 1024);
      const int pct = smem_sm > 0 ? std::min(100, (100 * need + smem_sm - 1) / smem_sm) : 100;
      cudaFuncSetAttribute(phase_kernel<kHalf, kMode>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    });
  }
  dim3 grid((a.W + kTile - 1) / kTile, (a.H + kTile - 1) / kTile);
  phase_kernel<kHalf, kMode><<<grid, kThreads, 0, s>>>(a);
  return (int)cudaGetLastError();
}
template <int kMode>
int launch_phase_m(const PhaseArgs& a, cudaStream_t s) {
  // staged sweep on request; at t = 0 the planes are the random ones of the
  // initialisation and no window set fits a box, so those phases fetch
  // through the texture unit
  if (a.staged && a.t > 0)
    return a.img_half ? launch_phase_t<true, kMode | kStage>(a, s) : launch_phase_t<false, kMode | kStage>(a, s);
  return a.img_half ? launch_phase_t<true, kMode>(a, s) : launch_phase_t<false, kMode>(a, s);
}
// the method, or one of the ablations of Sec. 4 (a.ablation: bit 0 symmetric
// propagation, bit 1 heuristic view selection)
int launch_phase(const PhaseArgs& a, cudaStream_t s) {
  if (a.tex_filter) return launch_phase_t<false, kTexture>(a, s);
  switch (a.ablation & 3) {
    case kSymmetric: return launch_phase_m<kSymmetric>(a, s);
    case kHeuristic: return launch_phase_m<kHeuristic>(a, s);
    case kSymmetric | kHeuristic: return launch_phase_m<kSymmetric | kHeuristic>(a, s);
    default: return launch_phase_m<0>(a, s);
  }
}

namespace {
// conversion between the state layout and row-major maps
template <class T>
__global__ void state_to_rows_kernel(const T* __restrict__ st, T* __restrict__ rows, int W, int H) {
  const size_t n = (size_t)W * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    rows[i] = st[state_index((int)(i % W), (int)(i / W), W)];
}
template <class T>
__global__ void rows_to_state_kernel(const T* __restrict__ rows, T* __restrict__ st, int W, int H) {
  const size_t n = (size_t)W * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    st[state_index((int)(i % W), (int)(i / W), W)] = rows[i];
}
template <class T>
void launch_convert(const void* src, void* dst, int W, int H, bool to_rows, cudaStream_t s) {
  if (to_rows)
    state_to_rows_kernel<T><<<1024, 256, 0, s>>>(static_cast<const T*>(src), static_cast<T*>(dst), W, H);
  else
    rows_to_state_kernel<T><<<1024, 256, 0, s>>>(static_cast<const T*>(src), static_cast<T*>(dst), W, H);
}
cudaError_t convert(const void* src, void* dst, int W, int H, int elem, bool to_rows, cudaStream_t s) {
  switch (elem) {
    case 16: launch_convert<float4>(src, dst, W, H, to_rows, s); break;
    case 4: launch_convert<uint32_t>(src, dst, W, H, to_rows, s); break;
    case 1: launch_convert<uint8_t>(src, dst, W, H, to_rows, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t export_state_field(const void* state, void* rows, int W, int H, int elem, bool host, cudaStream_t s) {
  if (!host) return convert(state, rows, W, H, elem, true, s);
  const size_t bytes = (size_t)W * H * elem;
  void* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&tmp, bytes, s);
  if (e != cudaSuccess) return e;
  e = convert(state, tmp, W, H, elem, true, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rows, tmp, bytes, cudaMemcpyDeviceToHost, s);
  const cudaError_t f = cudaFreeAsync(tmp, s);
  return e != cudaSuccess ? e : f;
}
cudaError_t import_state_field(const void* rows, void* state, int W, int H, int elem, bool host, cudaStream_t s) {
  if (!host) return convert(rows, state, W, H, elem, false, s);
  const size_t bytes = (size_t)W * H * elem;
  void* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&tmp, bytes, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(tmp, rows, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = convert(tmp, state, W, H, elem, false, s);
  const cudaError_t f = cudaFreeAsync(tmp, s);
  return e != cudaSuccess ? e : f;
}
}  // namespace amh
