// amh_batch.cu -- the batched form: every listed view of a scene in turn the
// reference, each with its own source list and its own size, resident
// together; one persistent launch per colour phase updates all references;
// the iteration loop is replayed from a CUDA graph; the tile shape is picked
// by timing the candidates on the batch itself.
//
// Work items are tiles of one reference, ordered reference by reference; a
// persistent grid (a few blocks per SM) takes them in order from one counter,
// so every block stays busy until the last item (the result of each pixel
// depends only on its reference's state, not on which block updates it).  A
// block loads the argument block of
// its item's reference (sizes, intrinsics, state pointers, view table) into
// shared memory and runs the same per-pixel update as the single-reference
// kernels (amh_update.cuh).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "amh.h"
#include "amh_device.cuh"
#include "amh_kernels.h"
#include "amh_update.cuh"

namespace amh {
namespace {
using namespace upd;

constexpr int kBThreads = 128;
constexpr int kMaxRefs = 256;
constexpr int kViewWords = (int)(sizeof(ViewConst) / sizeof(float));   // a view table entry in 4-byte words
static_assert(sizeof(ViewConst) % sizeof(float) == 0, "view table entries are whole words");

// the fields update_pixel reads, for one reference of the batch
struct RefArgs {
  int W, H, N, t;
  float Kinv[9];
  float tau, tau_up;
  int n1, n2, k;
  float inv2beta2, wI, wX;
  int squared, img_half;
  float dmin, dmax;
  uint32_t key0, key1;
  const void* ref;
  float4* plane;
  float* cost;
  uint32_t* sel;
  uint8_t* vbest;
  uint32_t* wmask;
  uint8_t* choice;
  const float4* prop;    // no learned proposals in the batched form (null)
  int prop_w, prop_h;
  unsigned int* status;  // bounds-check status word of the batch
  const ViewConst* vt;   // N views in global memory
  int tile0, tiles_x, tiles;
  ViewConst v[kMaxSrc];  // copied from vt into shared memory per item
};

struct BatchArgs {
  const RefArgs* refs;   // global memory, n_refs entries (v[] unused there)
  int n_refs, n_items, color, t;
  float tau;
  unsigned long long* pairs;
  unsigned int* queue;   // next work item; zeroed before every launch
};

// The next work item of this block: blocks take items in order from one
// counter (balanced to the last item, whatever each item costs).  The whole
// block calls it; it returns the same item to every thread.
__device__ __forceinline__ int next_item(const BatchArgs& b, int* slot) {
  __syncthreads();                       // every thread is done with the previous item
  if (threadIdx.x == 0) *slot = (int)atomicAdd(b.queue, 1u);
  __syncthreads();
  return *slot;
}

// Tile of TW x TH pixels per 128-thread block, one colour updated: TW / 2
// pixels of the colour per row, TH = 256 / TW rows.  Each warp takes a
// sub-tile of WC pixels of the colour per row and 32 / WC rows (its 32
// pixels laid out WC x 32 / WC), so the tile shape and the warp's pixel
// layout are chosen independently.
template <int TW, int WC>
struct TileShape {
  static constexpr int cols = TW / 2, rows = kBThreads / cols;
  static constexpr int wrows = 32 / WC, wpr = cols / WC;
  static_assert(cols % WC == 0 && (cols / WC) * (rows / wrows) == kBThreads / 32, "4 warps tile the block");
  // (row within the tile, pixel of the colour within the row) of this thread
  static __device__ __forceinline__ int row(int tid) { return (tid >> 5) / wpr * wrows + (tid & 31) / WC; }
  static __device__ __forceinline__ int col(int tid) { return (tid >> 5) % wpr * WC + (tid & 31) % WC; }
};

template <bool kHalf, int TW, int WC, int kMode>
__global__ void __launch_bounds__(kBThreads, 3) batch_phase_kernel(const __grid_constant__ BatchArgs b) {
  __shared__ RefArgs ra;
  __shared__ int cur_ref, item_slot;
  using T = TileShape<TW, WC>;
  int npairs = 0;
  if (threadIdx.x == 0) cur_ref = -1;
  for (int item = next_item(b, &item_slot); item < b.n_items; item = next_item(b, &item_slot)) {
    // the reference of this item: items are ordered reference by reference
    int r = 0;
    while (r + 1 < b.n_refs && b.refs[r + 1].tile0 <= item) r++;
    if (r != cur_ref) {
      const int words = (int)(offsetof(RefArgs, v) / sizeof(int));
      for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<int*>(&ra)[i] = reinterpret_cast<const int*>(&b.refs[r])[i];
      __syncthreads();
      for (int i = threadIdx.x; i < ra.N * kViewWords; i += blockDim.x)
        reinterpret_cast<float*>(ra.v)[i] = reinterpret_cast<const float*>(ra.vt)[i];
      if (threadIdx.x == 0) {
        ra.t = b.t;
        ra.tau = b.tau;
        cur_ref = r;
      }
      __syncthreads();
    }
    const int local = item - ra.tile0;
    const int ty = local / ra.tiles_x, tx = local % ra.tiles_x;
    const int y = ty * T::rows + T::row(threadIdx.x);
    const int x = tx * TW + 2 * T::col(threadIdx.x) + ((y + b.color) & 1);
    if (x < ra.W && y < ra.H) {
      PixelArrays sm;
      update_pixel<kHalf, kMode>(ra, sm, x, y, &npairs);
    }
  }
  const int tot = __reduce_add_sync(0xffffffffu, npairs);
  if ((threadIdx.x & 31) == 0 && tot)
    atomicAdd(&b.pairs[(blockIdx.x * 4 + (threadIdx.x >> 5)) % kPairCounters], (unsigned long long)tot);
}

// random initialisation of every pixel of every reference: 16 x 8 pixel tiles
template <bool kHalf, bool kTex>
__global__ void __launch_bounds__(kBThreads) batch_init_kernel(const __grid_constant__ BatchArgs b) {
  __shared__ RefArgs ra;
  __shared__ int cur_ref, item_slot;
  int npairs = 0;
  if (threadIdx.x == 0) cur_ref = -1;
  for (int item = next_item(b, &item_slot); item < b.n_items; item = next_item(b, &item_slot)) {
    int r = 0;
    while (r + 1 < b.n_refs && b.refs[r + 1].tile0 <= item) r++;
    if (r != cur_ref) {
      const int words = (int)(offsetof(RefArgs, v) / sizeof(int));
      for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<int*>(&ra)[i] = reinterpret_cast<const int*>(&b.refs[r])[i];
      __syncthreads();
      for (int i = threadIdx.x; i < ra.N * kViewWords; i += blockDim.x)
        reinterpret_cast<float*>(ra.v)[i] = reinterpret_cast<const float*>(ra.vt)[i];
      if (threadIdx.x == 0) cur_ref = r;
      __syncthreads();
    }
    const int local = item - ra.tile0;
    const int ty = local / ra.tiles_x, tx = local % ra.tiles_x;
    const int x = tx * 16 + (threadIdx.x & 15), y = ty * 8 + (threadIdx.x >> 4);
    if (x < ra.W && y < ra.H) {
      PixelArrays sm;
      init_pixel<kHalf, kTex>(ra, sm, x, y, &npairs);
    }
  }
  const int tot = __reduce_add_sync(0xffffffffu, npairs);
  if ((threadIdx.x & 31) == 0 && tot)
    atomicAdd(&b.pairs[(blockIdx.x * 4 + (threadIdx.x >> 5)) % kPairCounters], (unsigned long long)tot);
}

}  // namespace
}  // namespace amh

using namespace amh;

// ===========================================================================
// host side
// ===========================================================================
struct amh_batch {
  amh_params p;
  int n_views = 0, n_refs = 0;
  bool half = false;
  bool tex_filter = false;   // AMH_FLAG_TEXTURE_BILINEAR
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<cudaArray_t> arr;
  std::vector<cudaTextureObject_t> tex;
  std::vector<void*> img;                 // linear copies of the views (reference windows)
  std::vector<int> refs, W, H, N, tiles_x, tile0;
  size_t total_px = 0;
  float4* d_plane = nullptr;
  float* d_cost = nullptr;
  uint32_t* d_sel = nullptr;
  uint8_t* d_vbest = nullptr;
  uint32_t* d_wmask = nullptr;
  uint8_t* d_choice = nullptr;
  std::vector<size_t> px0;                // first entry of each reference in the state arrays (state_index layout)
  ViewConst* d_views = nullptr;
  RefArgs* d_refs[AMH_BATCH_VARIANTS] = {};   // work lists, per variant (by its tile width)
  int items[AMH_BATCH_VARIANTS] = {};
  int init_items = 0;
  RefArgs* d_refs_init = nullptr;
  unsigned long long* d_pairs = nullptr;
  unsigned int* d_status = nullptr;       // bounds-check status word (bounds-checked builds)
  unsigned int* d_queue = nullptr;        // work-item counter of the running launch
  int variant = 0;                        // index into kVariants
  int t = 0;
  bool initialized = false;
  int grid_blocks = 0;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_iters = -1, graph_variant = -1;
  std::string err;
};

namespace {
// the phase kernel's variants: (tile width in pixels, warp width in pixels of
// the colour); the block is always 128 threads, 256 pixels
struct Variant { int tw, wc; };
const Variant kVariants[AMH_BATCH_VARIANTS] = {{16, 8}, {32, 16}, {64, 32}, {16, 4}, {32, 8}};
thread_local std::string g_batch_create_err;

int bfail(amh_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf; else g_batch_create_err = buf;
  return code;
}

#define BTRY(b, call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                    \
  } while (0)

bool binv3(const double* A, double* I) {
  const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8],
               c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
  const double id = 1.0 / det;
  I[0] = c00 * id; I[1] = (A[2] * A[7] - A[1] * A[8]) * id; I[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  I[3] = c01 * id; I[4] = (A[0] * A[8] - A[2] * A[6]) * id; I[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  I[6] = c02 * id; I[7] = (A[1] * A[6] - A[0] * A[7]) * id; I[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return true;
}
void bmul3(const double* A, const double* B, double* C) {
  double T[9];
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) T[3 * r + q] = A[3 * r] * B[q] + A[3 * r + 1] * B[3 + q] + A[3 * r + 2] * B[6 + q];
  std::memcpy(C, T, sizeof T);
}
bool bcam_ok(const amh_camera& c) {
  for (double v : c.K) if (!std::isfinite(v)) return false;
  for (double v : c.R) if (!std::isfinite(v)) return false;
  for (double v : c.t) if (!std::isfinite(v)) return false;
  if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768) return false;
  return c.K[6] == 0.0 && c.K[7] == 0.0 && c.K[8] == 1.0;
}

void free_batch(amh_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  for (auto t : b->tex) if (t) cudaDestroyTextureObject(t);
  for (auto a : b->arr) if (a) cudaFreeArray(a);
  for (auto p : b->img) cudaFree(p);
  cudaFree(b->d_plane);
  cudaFree(b->d_cost);
  cudaFree(b->d_sel);
  cudaFree(b->d_vbest);
  cudaFree(b->d_wmask);
  cudaFree(b->d_choice);
  cudaFree(b->d_views);
  for (auto r : b->d_refs) cudaFree(r);
  cudaFree(b->d_refs_init);
  cudaFree(b->d_pairs);
  cudaFree(b->d_status);
  cudaFree(b->d_queue);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

float tau_at(const amh_params& p, int t) { return (float)(p.tau_mc_init * std::exp(-(double)t * t / (double)p.alpha)); }

BatchArgs make_args(amh_batch* b, const RefArgs* refs, int n_items, int color) {
  BatchArgs a;
  a.refs = refs;
  a.n_refs = b->n_refs;
  a.n_items = n_items;
  a.color = color;
  a.t = b->t;
  a.tau = tau_at(b->p, b->t);
  a.pairs = b->d_pairs;
  a.queue = b->d_queue;
  return a;
}

template <bool kHalf, int kMode>
void launch_batch_phase(amh_batch* b, int color) {
  const BatchArgs a = make_args(b, b->d_refs[b->variant], b->items[b->variant], color);
  cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), b->stream);
  const dim3 g(b->grid_blocks), t(kBThreads);
  switch (b->variant) {
    case 0: batch_phase_kernel<kHalf, 16, 8, kMode><<<g, t, 0, b->stream>>>(a); break;
    case 1: batch_phase_kernel<kHalf, 32, 16, kMode><<<g, t, 0, b->stream>>>(a); break;
    case 2: batch_phase_kernel<kHalf, 64, 32, kMode><<<g, t, 0, b->stream>>>(a); break;
    case 3: batch_phase_kernel<kHalf, 16, 4, kMode><<<g, t, 0, b->stream>>>(a); break;
    default: batch_phase_kernel<kHalf, 32, 8, kMode><<<g, t, 0, b->stream>>>(a); break;
  }
}
// FP16 images, uint8 images, or uint8 images through the texture unit's
// linear filter (AMH_FLAG_TEXTURE_BILINEAR; not combined with FP16)
int batch_phase(amh_batch* b, int color) {
  if (b->tex_filter) launch_batch_phase<false, kTexture>(b, color);
  else if (b->half) launch_batch_phase<true, 0>(b, color);
  else launch_batch_phase<false, 0>(b, color);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, AMH_ECUDA, "batch phase launch: %s", cudaGetErrorString(e));
  if (color == 1) b->t++;
  return AMH_OK;
}
int batch_init(amh_batch* b) {
  b->t = 0;
  const BatchArgs a = make_args(b, b->d_refs_init, b->init_items, 0);
  cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), b->stream);
  if (b->tex_filter) batch_init_kernel<false, true><<<b->grid_blocks, kBThreads, 0, b->stream>>>(a);
  else if (b->half) batch_init_kernel<true, false><<<b->grid_blocks, kBThreads, 0, b->stream>>>(a);
  else batch_init_kernel<false, false><<<b->grid_blocks, kBThreads, 0, b->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, AMH_ECUDA, "batch init launch: %s", cudaGetErrorString(e));
  b->initialized = true;
  return AMH_OK;
}
}  // namespace

extern "C" {

AMH_API int amh_batch_create(amh_batch** out, const amh_params* p, int32_t n_views, const amh_camera* cams,
                             const uint8_t* const* images, int32_t images_mem, int32_t n_refs, const int32_t* refs,
                             const int32_t* src_offsets, const int32_t* src_lists, void* stream) {
  g_batch_create_err.clear();
  if (!out) return bfail(nullptr, AMH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p || !cams || !images || !refs || !src_offsets || !src_lists) return bfail(nullptr, AMH_EINVAL, "NULL argument");
  if (images_mem != AMH_MEM_HOST && images_mem != AMH_MEM_DEVICE) return bfail(nullptr, AMH_EINVAL, "bad memory kind");
  if (n_views < 2 || n_refs < 1 || n_refs > kMaxRefs) return bfail(nullptr, AMH_EINVAL, "n_views >= 2, 1 <= n_refs <= 256");
  if (p->win_radius != kWinR || p->win_stride != kWinStride)
    return bfail(nullptr, AMH_EINVAL, "only the 11x11 stride-2 window (radius 5, stride 2) is built");
  if (!(p->k >= 1) || p->n1 < 0 || p->n2 < 0 || !(p->beta > 0) || !(p->sigma_I > 0) || !(p->sigma_x > 0) ||
      !(p->alpha > 0) || !(p->depth_min > 0) || !(p->depth_max > p->depth_min))
    return bfail(nullptr, AMH_EINVAL, "invalid parameters");
  if (p->flags & (AMH_FLAG_SYMMETRIC_PROPAGATION | AMH_FLAG_HEURISTIC_VIEWS))
    return bfail(nullptr, AMH_EINVAL, "the ablation flags apply to single contexts only");
  if ((p->flags & AMH_FLAG_TEXTURE_BILINEAR) && (p->flags & AMH_FLAG_IMAGES_F16))
    return bfail(nullptr, AMH_EINVAL, "AMH_FLAG_TEXTURE_BILINEAR takes uint8 images");
  if (src_offsets[0] != 0) return bfail(nullptr, AMH_EINVAL, "src_offsets[0] must be 0");
  for (int r = 0; r < n_refs; r++) {
    const int ref = refs[r];
    if (ref < 0 || ref >= n_views) return bfail(nullptr, AMH_EINVAL, "refs[%d] = %d invalid", r, ref);
    const int n = src_offsets[r + 1] - src_offsets[r];
    if (n < 1 || n > AMH_MAX_SRC) return bfail(nullptr, AMH_EINVAL, "reference %d: 1..32 sources", r);
    for (int j = 0; j < n; j++) {
      const int v = src_lists[src_offsets[r] + j];
      if (v < 0 || v >= n_views || v == ref) return bfail(nullptr, AMH_EINVAL, "reference %d: source %d invalid", r, v);
      for (int q = 0; q < j; q++)
        if (src_lists[src_offsets[r] + q] == v) return bfail(nullptr, AMH_EINVAL, "reference %d repeats view %d", r, v);
    }
  }
  for (int v = 0; v < n_views; v++) {
    if (!bcam_ok(cams[v])) return bfail(nullptr, AMH_EINVAL, "camera %d invalid", v);
    if (!images[v]) return bfail(nullptr, AMH_EINVAL, "image %d is NULL", v);
  }

  amh_batch* b = new (std::nothrow) amh_batch();
  if (!b) return bfail(nullptr, AMH_ENOMEM, "host allocation failed");
  auto bail = [&](int code) {
    g_batch_create_err = b->err;
    free_batch(b);
    delete b;
    return code;
  };
#define CB(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      bfail(b, e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA, "%s: %s", #call,           \
            cudaGetErrorString(e_));                                                                \
      return bail(e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA);                        \
    }                                                                                               \
  } while (0)
  b->p = *p;
  b->n_views = n_views;
  b->n_refs = n_refs;
  b->half = (p->flags & AMH_FLAG_IMAGES_F16) != 0;
  b->tex_filter = (p->flags & AMH_FLAG_TEXTURE_BILINEAR) != 0;
  if (stream) b->stream = (cudaStream_t)stream;
  else {  // graph capture needs a stream other than the legacy default stream
    CB(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  const size_t es = b->half ? 2 : 1;
  const cudaMemcpyKind kind = images_mem == AMH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  // every view once: a texture (as a source) and a linear copy (as a reference)
  b->arr.assign(n_views, nullptr);
  b->tex.assign(n_views, 0);
  b->img.assign(n_views, nullptr);
  std::vector<bool> used(n_views, false);
  for (int r = 0; r < n_refs; r++) {
    used[refs[r]] = true;
    for (int j = src_offsets[r]; j < src_offsets[r + 1]; j++) used[src_lists[j]] = true;
  }
  for (int v = 0; v < n_views; v++) {
    if (!used[v]) continue;
    const amh_camera& c = cams[v];
    const size_t np = (size_t)c.width * c.height;
    CB(cudaMalloc(&b->img[v], np * es));
    CB(cudaMemcpyAsync(b->img[v], images[v], np * es, kind, b->stream));
    cudaChannelFormatDesc fd = b->half ? cudaCreateChannelDescHalf() : cudaCreateChannelDesc<uint8_t>();
    CB(cudaMallocArray(&b->arr[v], &fd, c.width, c.height, cudaArrayTextureGather));
    CB(cudaMemcpy2DToArrayAsync(b->arr[v], 0, 0, images[v], c.width * es, c.width * es, c.height, kind, b->stream));
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = b->arr[v];
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = b->tex_filter ? cudaFilterModeLinear : cudaFilterModePoint;
    td.readMode = b->half ? cudaReadModeElementType : cudaReadModeNormalizedFloat;
    CB(cudaCreateTextureObject(&b->tex[v], &rd, &td, nullptr));
  }
  // references: sizes, state offsets, view tables
  std::vector<ViewConst> views;
  std::vector<RefArgs> host_refs(n_refs);
  b->refs.assign(refs, refs + n_refs);
  b->px0.resize(n_refs);
  for (int r = 0; r < n_refs; r++) {
    const amh_camera& cr = cams[refs[r]];
    b->W.push_back(cr.width);
    b->H.push_back(cr.height);
    b->N.push_back(src_offsets[r + 1] - src_offsets[r]);
    b->px0[r] = b->total_px;
    b->total_px += state_size(cr.width, cr.height);
  }
  const size_t NP = b->total_px;
  CB(cudaMalloc(&b->d_plane, NP * sizeof(float4)));
  CB(cudaMalloc(&b->d_cost, NP * sizeof(float)));
  CB(cudaMalloc(&b->d_sel, NP * sizeof(uint32_t)));
  CB(cudaMalloc(&b->d_vbest, NP));
  CB(cudaMalloc(&b->d_wmask, NP * sizeof(uint32_t)));
  CB(cudaMalloc(&b->d_choice, NP));
  CB(cudaMalloc(&b->d_pairs, kPairCounters * sizeof(unsigned long long)));
  CB(cudaMemsetAsync(b->d_pairs, 0, kPairCounters * sizeof(unsigned long long), b->stream));
  CB(cudaMalloc(&b->d_status, sizeof(unsigned int)));
  CB(cudaMemsetAsync(b->d_status, 0, sizeof(unsigned int), b->stream));
  CB(cudaMalloc(&b->d_queue, sizeof(unsigned int)));
  for (int r = 0; r < n_refs; r++) {
    const amh_camera& cr = cams[refs[r]];
    double Kri[9];
    if (!binv3(cr.K, Kri)) {
      bfail(b, AMH_EINVAL, "K of view %d singular", refs[r]);
      return bail(AMH_EINVAL);
    }
    RefArgs& ra = host_refs[r];
    std::memset(&ra, 0, sizeof ra);
    ra.W = cr.width;
    ra.H = cr.height;
    ra.N = b->N[r];
    for (int i = 0; i < 9; i++) ra.Kinv[i] = (float)Kri[i];
    ra.tau_up = p->tau_up;
    ra.n1 = p->n1;
    ra.n2 = p->n2;
    ra.k = p->k;
    ra.inv2beta2 = (float)(1.0 / (2.0 * (double)p->beta * p->beta));
    ra.wI = (float)(1.0 / (2.0 * (double)p->sigma_I * p->sigma_I));
    ra.wX = (float)(1.0 / (2.0 * (double)p->sigma_x * p->sigma_x));
    ra.squared = (p->flags & AMH_FLAG_BILATERAL_SQUARED) ? 1 : 0;
    ra.img_half = b->half ? 1 : 0;
    ra.dmin = p->depth_min;
    ra.dmax = p->depth_max;
    // reference r draws with the key seed + r
    const uint64_t key = p->seed + (uint64_t)r;
    ra.key0 = (uint32_t)(key & 0xFFFFFFFFu);
    ra.key1 = (uint32_t)(key >> 32);
    ra.ref = b->img[refs[r]];
    const size_t o = b->px0[r];
    ra.plane = b->d_plane + o;
    ra.cost = b->d_cost + o;
    ra.sel = b->d_sel + o;
    ra.vbest = b->d_vbest + o;
    ra.wmask = b->d_wmask + o;
    ra.choice = b->d_choice + o;
    ra.status = b->d_status;
    ra.tile0 = (int)views.size();   // temporarily: first view-table entry
    double RrT[9];
    for (int i = 0; i < 3; i++)
      for (int q = 0; q < 3; q++) RrT[3 * i + q] = cr.R[3 * q + i];
    for (int jj = src_offsets[r]; jj < src_offsets[r + 1]; jj++) {
      const int v = src_lists[jj];
      const amh_camera& cj = cams[v];
      double Rjr[9], tjr[3], A[9], KR[9], bb[3];
      bmul3(cj.R, RrT, Rjr);
      for (int i = 0; i < 3; i++)
        tjr[i] = cj.t[i] - (Rjr[3 * i] * cr.t[0] + Rjr[3 * i + 1] * cr.t[1] + Rjr[3 * i + 2] * cr.t[2]);
      bmul3(cj.K, Rjr, KR);
      bmul3(KR, Kri, A);
      for (int i = 0; i < 3; i++) bb[i] = cj.K[3 * i] * tjr[0] + cj.K[3 * i + 1] * tjr[1] + cj.K[3 * i + 2] * tjr[2];
      for (int q = 0; q < 3; q++) {
        A[q] += A[6 + q]; A[3 + q] += A[6 + q];
        KR[q] += KR[6 + q]; KR[3 + q] += KR[6 + q];
      }
      bb[0] += bb[2];
      bb[1] += bb[2];
      ViewConst V;
      std::memset(&V, 0, sizeof V);
      for (int i = 0; i < 9; i++) V.A[i] = (float)A[i];
      for (int i = 0; i < 9; i++) V.P[i] = (float)KR[i];
      for (int i = 0; i < 3; i++) V.b[i] = (float)bb[i];
      V.xmax = (float)cj.width;
      V.ymax = (float)cj.height;
      V.tex = b->tex[v];
      views.push_back(V);
    }
  }
  CB(cudaMalloc(&b->d_views, views.size() * sizeof(ViewConst)));
  CB(cudaMemcpyAsync(b->d_views, views.data(), views.size() * sizeof(ViewConst), cudaMemcpyHostToDevice, b->stream));
  for (int r = 0; r < n_refs; r++) host_refs[r].vt = b->d_views + host_refs[r].tile0;
  // work lists: one per tile width for the phases, one for the initialisation
  auto upload = [&](int tw, int th, RefArgs** dst, int* n_items) -> cudaError_t {
    std::vector<RefArgs> h = host_refs;
    int items = 0;
    for (int r = 0; r < n_refs; r++) {
      h[r].tiles_x = (h[r].W + tw - 1) / tw;
      h[r].tiles = h[r].tiles_x * ((h[r].H + th - 1) / th);
      h[r].tile0 = items;
      items += h[r].tiles;
    }
    *n_items = items;
    cudaError_t e = cudaMalloc(dst, n_refs * sizeof(RefArgs));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(*dst, h.data(), n_refs * sizeof(RefArgs), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(b->stream);   // h goes out of scope
  };
  for (int vi = 0; vi < AMH_BATCH_VARIANTS; vi++)
    CB(upload(kVariants[vi].tw, 2 * kBThreads / kVariants[vi].tw, &b->d_refs[vi], &b->items[vi]));
  CB(upload(16, 8, &b->d_refs_init, &b->init_items));
  int dev = 0, sms = 0;
  CB(cudaGetDevice(&dev));
  CB(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->grid_blocks = sms * 3;   // persistent: three 128-thread blocks per SM
  CB(cudaStreamSynchronize(b->stream));
#undef CB
  *out = b;
  return AMH_OK;
}

AMH_API int amh_batch_init_random(amh_batch* b) {
  if (!b) return AMH_EINVAL;
  return batch_init(b);
}

AMH_API int amh_batch_step_phase(amh_batch* b, int32_t color) {
  if (!b) return AMH_EINVAL;
  if (color != 0 && color != 1) return bfail(b, AMH_EINVAL, "color must be 0 or 1");
  if (!b->initialized) return bfail(b, AMH_ESTATE, "batch not initialised");
  return batch_phase(b, color);
}

AMH_API int amh_batch_iterate(amh_batch* b, int32_t k) {
  if (!b) return AMH_EINVAL;
  if (k < 0) return bfail(b, AMH_EINVAL, "k < 0");
  if (!b->initialized) return bfail(b, AMH_ESTATE, "batch not initialised");
  for (int i = 0; i < k; i++) {
    int rc = batch_phase(b, 0);
    if (!rc) rc = batch_phase(b, 1);
    if (rc) return rc;
  }
  return AMH_OK;
}

AMH_API int amh_batch_run(amh_batch* b, int32_t iters) {
  if (!b) return AMH_EINVAL;
  if (iters < 0) return bfail(b, AMH_EINVAL, "iters < 0");
  if (!b->graph_exec || b->graph_iters != iters || b->graph_variant != b->variant) {
    if (b->graph_exec) {
      cudaGraphExecDestroy(b->graph_exec);
      b->graph_exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    BTRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_init(b);
    for (int i = 0; i < iters && !rc; i++) {
      rc = batch_phase(b, 0);
      if (!rc) rc = batch_phase(b, 1);
    }
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return bfail(b, AMH_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, AMH_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    b->graph_iters = iters;
    b->graph_variant = b->variant;
  }
  BTRY(b, cudaGraphLaunch(b->graph_exec, b->stream));
  b->t = iters;
  b->initialized = true;
  return AMH_OK;
}

AMH_API int amh_batch_set_variant(amh_batch* b, int32_t variant) {
  if (!b) return AMH_EINVAL;
  if (variant < 0 || variant >= AMH_BATCH_VARIANTS)
    return bfail(b, AMH_EINVAL, "variant must be 0 .. %d", AMH_BATCH_VARIANTS - 1);
  b->variant = variant;
  return AMH_OK;
}

AMH_API int amh_batch_autotune(amh_batch* b, int32_t iters, int32_t* chosen, float* ms_out) {
  if (!b) return AMH_EINVAL;
  if (iters < 1) return bfail(b, AMH_EINVAL, "iters >= 1");
  cudaEvent_t e0, e1;
  BTRY(b, cudaEventCreate(&e0));
  BTRY(b, cudaEventCreate(&e1));
  float best = 0.f;
  int bi = 0;
  for (int vi = 0; vi < AMH_BATCH_VARIANTS; vi++) {
    b->variant = vi;
    int rc = batch_init(b);
    for (int i = 0; i < iters && !rc; i++) rc = batch_phase(b, i & 1);   // warm-up
    if (rc) return rc;
    BTRY(b, cudaEventRecord(e0, b->stream));
    rc = batch_init(b);
    for (int i = 0; i < iters && !rc; i++) {
      rc = batch_phase(b, 0);
      if (!rc) rc = batch_phase(b, 1);
    }
    if (rc) return rc;
    BTRY(b, cudaEventRecord(e1, b->stream));
    BTRY(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    BTRY(b, cudaEventElapsedTime(&ms, e0, e1));
    if (ms_out) ms_out[vi] = ms;
    if (vi == 0 || ms < best) { best = ms; bi = vi; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->variant = bi;
  b->initialized = false;   // the state holds a tuning run: initialise again
  if (chosen) *chosen = bi;
  return AMH_OK;
}

AMH_API int amh_batch_info(const amh_batch* b, int32_t r, int32_t* width, int32_t* height, int32_t* n_src,
                           int32_t* n_refs) {
  if (!b) return AMH_EINVAL;
  if (n_refs) *n_refs = b->n_refs;
  if (r < 0 || r >= b->n_refs) return (width || height || n_src) ? AMH_EINVAL : AMH_OK;
  if (width) *width = b->W[r];
  if (height) *height = b->H[r];
  if (n_src) *n_src = b->N[r];
  return AMH_OK;
}

AMH_API int amh_batch_get_state(amh_batch* b, int32_t r, amh_state* o, int32_t mem) {
  if (!b || !o) return AMH_EINVAL;
  if (r < 0 || r >= b->n_refs) return bfail(b, AMH_EINVAL, "reference index out of range");
  if (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE) return bfail(b, AMH_EINVAL, "bad memory kind");
  const size_t o0 = b->px0[r];
  const int W = b->W[r], H = b->H[r];
  const bool host = mem == AMH_MEM_HOST;
  if (o->plane) BTRY(b, export_state_field(b->d_plane + o0, o->plane, W, H, 16, host, b->stream));
  if (o->cost) BTRY(b, export_state_field(b->d_cost + o0, o->cost, W, H, 4, host, b->stream));
  if (o->sel) BTRY(b, export_state_field(b->d_sel + o0, o->sel, W, H, 4, host, b->stream));
  if (o->vbest) BTRY(b, export_state_field(b->d_vbest + o0, o->vbest, W, H, 1, host, b->stream));
  if (o->wmask) BTRY(b, export_state_field(b->d_wmask + o0, o->wmask, W, H, 4, host, b->stream));
  if (o->choice) BTRY(b, export_state_field(b->d_choice + o0, o->choice, W, H, 1, host, b->stream));
  o->t = b->t;
  if (mem == AMH_MEM_HOST) BTRY(b, cudaStreamSynchronize(b->stream));
  return AMH_OK;
}

AMH_API int amh_batch_pair_count(amh_batch* b, uint64_t* count, int32_t reset) {
  if (!b) return AMH_EINVAL;
  unsigned long long v[kPairCounters];
  BTRY(b, cudaMemcpyAsync(v, b->d_pairs, sizeof v, cudaMemcpyDeviceToHost, b->stream));
  BTRY(b, cudaStreamSynchronize(b->stream));
  unsigned long long tot = 0;
  for (int i = 0; i < kPairCounters; i++) tot += v[i];
  if (count) *count = tot;
  if (reset) BTRY(b, cudaMemsetAsync(b->d_pairs, 0, sizeof v, b->stream));
  return AMH_OK;
}

AMH_API int amh_batch_synchronize(amh_batch* b) {
  if (!b) return AMH_EINVAL;
  BTRY(b, cudaStreamSynchronize(b->stream));
#ifdef AMH_BOUNDS_CHECK
  unsigned int st = 0;
  BTRY(b, cudaMemcpy(&st, b->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (st) return bfail(b, AMH_EDEVICE, "bounds check: index out of range in the update (status 0x%x)", st);
#endif
  return AMH_OK;
}

AMH_API const char* amh_batch_last_error(const amh_batch* b) {
  if (!b) return g_batch_create_err.c_str();
  return b->err.c_str();
}

AMH_API void amh_batch_destroy(amh_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
}

}  // extern "C"
