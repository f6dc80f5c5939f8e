// amh_learned.cu -- the learned proposal network (this project's extension):
// a 4-level convolutional encoder-decoder that reads the half-resolution
// state of the checkerboard update (reference intensity, log depth, normal,
// cost) and proposes one plane per pixel; the phase kernel scores that plane
// with the unchanged matching cost (Eq. 8) and view weights (Eqs. 2-7) as one
// more candidate, so the plain method stays the arbiter.
//
// Kernels: 3x3 convolution forward on the fifth-generation tensor cores
// (tcgen05.mma, FP32 accumulator in tensor memory, BF16 operands brought in by
// the tensor memory accelerator; fused bias / ReLU / skip add), the data
// gradient as the same convolution with flipped, transposed weights, the
// weight gradient on the same tensor-core path, reading the pixel-major
// operands directly (amh_conv_tc.cuh; bias gradients in FP32), 2x2 average pooling,
// nearest upsampling, the L1 loss, Adam, and the feature / head / proposal
// conversions.
//
// Layout: activations (H, W, C) with C a multiple of 16, BF16 between
// layers; conv weights (9, Cout, Cin) BF16 (FP32 master copy for Adam), tap
// t = 3 (dy + 1) + (dx + 1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "amh.h"
#include "amh_conv_tc.cuh"
#include "amh_ctx.h"
#include "amh_device.cuh"

namespace amh {
namespace {

constexpr int kLayers = 8;
struct LayerDef { int cin, cout, relu; };
// e1 e2 e3 e4 d3 d2 d1 out
constexpr LayerDef kNet[kLayers] = {{16, 32, 1}, {32, 64, 1}, {64, 96, 1}, {96, 128, 1},
                                    {128, 96, 1}, {96, 64, 1}, {64, 32, 1}, {32, 16, 0}};

// bias gradient in FP32: db[c] += sum over pixels of dy(p, c), C a multiple
// of 16 (at most 128), in two passes without atomics.  Pass 1: a thread sums
// four channels (one float4) of every k-th pixel of its block's range,
// k = 256 / (C / 4), and the block writes its per-channel sums to part[block].
// Pass 2: one block per channel adds the partial sums into db.
constexpr int kBiasBlocks = 2048;     // most pass-1 blocks (rows of the partial sums)
__global__ void __launch_bounds__(256) bias_grad_kernel(const float* __restrict__ dy, int np, int C,
                                                        int per_block, float* __restrict__ part) {
  __shared__ float4 red[256];
  const int g4 = C >> 2, k = 256 / g4, t = threadIdx.x, g = t % g4, j = t / g4;
  const int p0 = blockIdx.x * per_block, p1 = min(np, p0 + per_block);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j < k) {
#pragma unroll 4
    for (int p = p0 + j; p < p1; p += k) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(dy + (size_t)p * C) + g);
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
  }
  red[t] = s;
  __syncthreads();
  if (j == 0) {
    for (int q = 1; q < k; q++) {
      const float4 v = red[q * g4 + g];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    reinterpret_cast<float4*>(part + (size_t)blockIdx.x * C)[g] = s;
  }
}
__global__ void __launch_bounds__(256) bias_sum_kernel(const float* __restrict__ part, int nb, int C, float* db) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < nb; b += 256) s += part[(size_t)b * C + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] += red[0];
}

// weights (9, Cout, Cin) -> data-gradient weights (9, Cin, Cout), taps flipped
__global__ void flip_transpose_kernel(const __nv_bfloat16* w, __nv_bfloat16* wd, int Cin, int Cout) {
  const int n = 9 * Cin * Cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int t = i / (Cin * Cout), ci = (i / Cout) % Cin, co = i % Cout;
    wd[i] = w[((size_t)(8 - t) * Cout + co) * Cin + ci];
  }
}

// The elementwise kernels below take four channels per thread and step (C is
// a multiple of 16, so a group of four never crosses a pixel): 16-byte FP32
// and 8-byte BF16 accesses.
struct bf16x4 { __nv_bfloat162 a, b; };
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const bf16x4 v = *reinterpret_cast<const bf16x4*>(p);
  const float2 lo = __bfloat1622float2(v.a), hi = __bfloat1622float2(v.b);
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
  bf16x4 o;
  o.a = __floats2bfloat162_rn(v.x, v.y);
  o.b = __floats2bfloat162_rn(v.z, v.w);
  *reinterpret_cast<bf16x4*>(p) = o;
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 scale4(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }

__global__ void pool2_kernel(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  const size_t n = (size_t)Ho * Wo * C / 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(4 * i % C), p = (int)(4 * i / C), oy = p / Wo, ox = p % Wo;
    const size_t b = ((size_t)(2 * oy) * W + 2 * ox) * C + c;
    const float4 s = add4(add4(add4(ld4(x + b), ld4(x + b + C)), ld4(x + b + (size_t)W * C)), ld4(x + b + (size_t)W * C + C));
    st4(y + 4 * i, scale4(0.25f, s));
  }
}
__global__ void pool2_bwd_add_kernel(const float* __restrict__ d, float* __restrict__ dx, int H, int W, int C) {   // dx += pool'^T d
  const size_t n = (size_t)H * W * C / 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(4 * i % C), p = (int)(4 * i / C), yy = p / W, xx = p % W;
    float4* o = reinterpret_cast<float4*>(dx) + i;
    *o = add4(*o, scale4(0.25f, *reinterpret_cast<const float4*>(d + ((size_t)(yy / 2) * (W / 2) + xx / 2) * C + c)));
  }
}
__global__ void up2_kernel(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ y, int Ho, int Wo, int C) {  // (Ho, Wo) output
  const size_t n = (size_t)Ho * Wo * C / 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(4 * i % C), p = (int)(4 * i / C), yy = p / Wo, xx = p % Wo;
    *reinterpret_cast<bf16x4*>(y + 4 * i) =
        *reinterpret_cast<const bf16x4*>(x + ((size_t)(yy / 2) * (Wo / 2) + xx / 2) * C + c);
  }
}
__global__ void up2_bwd_kernel(const float* __restrict__ d, float* __restrict__ dx, int H, int W, int C) {   // (H, W) = input size
  const size_t n = (size_t)H * W * C / 4;
  const int Wo = 2 * W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(4 * i % C), p = (int)(4 * i / C), yy = p / W, xx = p % W;
    const float* b = d + ((size_t)(2 * yy) * Wo + 2 * xx) * C + c;
    const float4 s = add4(add4(add4(*reinterpret_cast<const float4*>(b), *reinterpret_cast<const float4*>(b + C)),
                               *reinterpret_cast<const float4*>(b + (size_t)Wo * C)),
                          *reinterpret_cast<const float4*>(b + (size_t)Wo * C + C));
    reinterpret_cast<float4*>(dx)[i] = s;
  }
}
// g (FP32) times the ReLU mask of r, optionally also into a BF16 copy; n a
// multiple of 4
__global__ void relu_mask_kernel(const float* __restrict__ g, const __nv_bfloat16* __restrict__ r, float* __restrict__ out,
                                 __nv_bfloat16* __restrict__ out16, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 gv = reinterpret_cast<const float4*>(g)[i], rv = ld4(r + 4 * i);
    const float4 v = make_float4(rv.x > 0.f ? gv.x : 0.f, rv.y > 0.f ? gv.y : 0.f, rv.z > 0.f ? gv.z : 0.f,
                                 rv.w > 0.f ? gv.w : 0.f);
    reinterpret_cast<float4*>(out)[i] = v;
    if (out16) st4(out16 + 4 * i, v);
  }
}
__global__ void bf16_to_f32_kernel(const __nv_bfloat16* g, float* o, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    o[i] = __bfloat162float(g[i]);
}
__global__ void to_bf16_kernel(const float* g, __nv_bfloat16* o, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    o[i] = __float2bfloat16(g[i]);
}

// L1 loss over the 4 used output channels of the masked pixels and its
// gradient (zero on the other 12 channels); loss accumulated in *loss (sum;
// the host divides by the count)
__global__ void l1_loss_kernel(const float* __restrict__ out, const float* __restrict__ target,
                               const uint8_t* __restrict__ mask, float* __restrict__ dout, float* loss, int np,
                               float inv_n) {
  float s = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const float4 o = reinterpret_cast<const float4*>(out)[(size_t)p * 4];
    const float4 t = reinterpret_cast<const float4*>(target)[p];
    const bool on = mask[p] != 0;
    const float d[4] = {o.x - t.x, o.y - t.y, o.z - t.z, o.w - t.w};
    float g[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      g[c] = 0.f;
      if (on) {
        s += fabsf(d[c]);
        g[c] = (d[c] > 0.f ? 1.f : (d[c] < 0.f ? -1.f : 0.f)) * inv_n;
      }
    }
    float4* dp = reinterpret_cast<float4*>(dout) + (size_t)p * 4;
    dp[0] = make_float4(g[0], g[1], g[2], g[3]);
    dp[1] = dp[2] = dp[3] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_n);
}

__global__ void adam_kernel(float* w, float* m, float* v, const float* g, __nv_bfloat16* w16, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16(wi);
  }
}

// Features of half-resolution pixel (X, Y), read at full-resolution pixel
// (2X, 2Y): intensity / 255 - 0.5, normalised log depth, normal, cost / 2,
// zeros up to 16 channels.  Also keeps the input plane for the head.  The
// plane and cost come from the context's state (state_index layout).
__global__ void features_kernel(const void* ref, int ref_half, const float4* plane, const float* cost, int W, int H,
                                int w2, int h2, float lmid, float lscale, __nv_bfloat16* x0, float4* pin) {
  const int n = w2 * h2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int X = p % w2, Y = p / w2;
    const int x = min(2 * X, W - 1), y = min(2 * Y, H - 1);
    const size_t q = (size_t)y * W + x, qs = state_index(x, y, W);   // image, state
    const float I = ref_half ? __half2float(reinterpret_cast<const __half*>(ref)[q])
                             : (float)reinterpret_cast<const uint8_t*>(ref)[q];
    const float4 pl = plane[qs];
    const float f[6] = {I / 255.f - 0.5f, (logf(fmaxf(pl.w, 1e-6f)) - lmid) * lscale, pl.x, pl.y, pl.z,
                        cost[qs] * 0.5f};
    for (int c = 0; c < 16; c++) x0[(size_t)p * 16 + c] = __float2bfloat16(c < 6 ? f[c] : 0.f);
    pin[p] = pl;
  }
}
// one training example, mirrored: output pixel (X, Y) reads source pixel
// (w2 - 1 - X or X, h2 - 1 - Y or Y); an x mirror negates the normal's x
// (feature 2, target 1), a y mirror its y (feature 3, target 2); features
// padded to 16 channels and stored as BF16
__global__ void example_kernel(const float* __restrict__ x, int C, const float* __restrict__ t,
                               const uint8_t* __restrict__ m, int w2, int h2, int mirror, __nv_bfloat16* x0,
                               float* target, uint8_t* mask) {
  const int n = w2 * h2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int X = p % w2, Y = p / w2;
    const int sx = (mirror & 1) ? w2 - 1 - X : X, sy = (mirror & 2) ? h2 - 1 - Y : Y;
    const size_t q = (size_t)sy * w2 + sx;
    __align__(16) __nv_bfloat16 row[16];
#pragma unroll
    for (int c = 0; c < 16; c++) {
      float v = c < C ? x[q * C + c] : 0.f;
      if ((c == 2 && (mirror & 1)) || (c == 3 && (mirror & 2))) v = -v;
      row[c] = __float2bfloat16(v);
    }
    reinterpret_cast<uint4*>(x0)[(size_t)p * 2] = reinterpret_cast<const uint4*>(row)[0];
    reinterpret_cast<uint4*>(x0)[(size_t)p * 2 + 1] = reinterpret_cast<const uint4*>(row)[1];
    float4 tv = reinterpret_cast<const float4*>(t)[q];
    if (mirror & 1) tv.y = -tv.y;
    if (mirror & 2) tv.z = -tv.z;
    reinterpret_cast<float4*>(target)[p] = tv;
    mask[p] = m[q];
  }
}
// targets: (log D_final - log D_in, n_final - n_in) where the final cost is
// below cmax (confident pixels)
__global__ void targets_kernel(const float4* plane, const float* cost, const float4* pin, int W, int H, int w2,
                               int h2, float cmax, float* target, uint8_t* mask) {
  const int n = w2 * h2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int X = p % w2, Y = p / w2;
    const int x = min(2 * X, W - 1), y = min(2 * Y, H - 1);
    const size_t q = state_index(x, y, W);
    const float4 pf = plane[q], pi = pin[p];
    const bool ok = cost[q] < cmax && pf.w > 0.f && pi.w > 0.f;
    target[(size_t)p * 4 + 0] = ok ? logf(pf.w) - logf(pi.w) : 0.f;
    target[(size_t)p * 4 + 1] = ok ? pf.x - pi.x : 0.f;
    target[(size_t)p * 4 + 2] = ok ? pf.y - pi.y : 0.f;
    target[(size_t)p * 4 + 3] = ok ? pf.z - pi.z : 0.f;
    mask[p] = ok ? 1 : 0;
  }
}
// head: proposal plane of half-resolution pixel (X, Y) as (n, d) with
// n . X + d = 0, from the input plane and the predicted residuals, valid when
// it faces the camera at full-resolution pixel (2X, 2Y)
__global__ void head_kernel(const float* out, const float4* pin, int W, int H, int w2, int h2, PhaseArgs geo,
                            float4* prop) {
  const int n = w2 * h2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int X = p % w2, Y = p / w2;
    const float x = (float)min(2 * X, W - 1), y = (float)min(2 * Y, H - 1);
    const float4 pi = pin[p];
    const float* o = out + (size_t)p * 16;
    const float D = pi.w * expf(fminf(fmaxf(o[0], -3.f), 3.f));
    float3 nn = make_float3(pi.x + o[1], pi.y + o[2], pi.z + o[3]);
    const float l = sqrtf(dot3(nn, nn));
    const float3 ray = ref_ray(geo.Kinv, x, y);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l > 1e-6f && pi.w > 0.f && isfinite(D)) {
      nn = face_camera(make_float3(nn.x / l, nn.y / l, nn.z / l), ray);
      const float d = -D * dot3(nn, ray);
      if (d > 0.f && isfinite(d)) r = make_float4(nn.x, nn.y, nn.z, d);
    }
    prop[p] = r;
  }
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

}  // namespace
}  // namespace amh

using namespace amh;

// ===========================================================================
// host side
// ===========================================================================
struct amh_net {
  int w2 = 0, h2 = 0;                     // network input size (half resolution)
  cudaStream_t stream = nullptr;
  // parameters per layer: FP32 master, BF16 copy, Adam moments, gradients
  float* wm[kLayers] = {};
  float* bm[kLayers] = {};
  __nv_bfloat16* w16[kLayers] = {};
  __nv_bfloat16* wd16[kLayers] = {};      // data-gradient weights
  float *mw[kLayers] = {}, *vw[kLayers] = {}, *mb[kLayers] = {}, *vb[kLayers] = {};
  float *gw[kLayers] = {}, *gb[kLayers] = {};
  float* bpart = nullptr;                 // per-block partial sums of the bias gradients
  int step = 0;
  // activations (BF16) and gradient buffers (FP32)
  __nv_bfloat16 *x0 = nullptr, *e1 = nullptr, *in_e2 = nullptr, *e2 = nullptr, *in_e3 = nullptr, *e3 = nullptr,
                *in_e4 = nullptr, *e4 = nullptr, *in_d3 = nullptr, *r3 = nullptr, *d3 = nullptr, *in_d2 = nullptr,
                *r2 = nullptr, *d2 = nullptr, *in_d1 = nullptr, *r1 = nullptr, *d1 = nullptr, *g16 = nullptr;
  float* out = nullptr;
  float* target = nullptr;
  uint8_t* mask = nullptr;
  float4* pin = nullptr;
  float4* prop = nullptr;
  // backward: dy[L] = gradient at layer L's output after its ReLU mask (FP32),
  // gA / gB scratch, gE1..gE3 gradients arriving at e1..e3 through the skips
  float* dy[kLayers] = {};
  float *gA = nullptr, *gB = nullptr, *gE1 = nullptr, *gE2 = nullptr, *gE3 = nullptr;
  float* loss = nullptr;
  unsigned int* status = nullptr;         // bit 0: a convolution's barrier wait gave up
  size_t maxel = 0;
  std::vector<void*> allocs;
  std::string err;
};

namespace {
thread_local std::string g_net_err;
int nfail(amh_net* n, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (n) n->err = buf; else g_net_err = buf;
  return code;
}
template <typename T>
cudaError_t nalloc(amh_net* n, T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) {
    n->allocs.push_back((void*)*p);
    e = cudaMemsetAsync(*p, 0, count * sizeof(T), n->stream);
  }
  return e;
}
#define NTRY(n, call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return nfail(n, e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                    \
  } while (0)

// the driver's tensor-map encoder, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
// tensor map of a BF16 tensor of dims (d0, d1, d2), d0 contiguous, rows of
// pitch0 elements (>= d0), read in boxes of (b0, b1, b2); reads outside the
// tensor return zeros
bool bf16_map(CUtensorMap* m, const void* p, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b0, uint32_t b1,
              uint32_t b2 = 1, uint64_t pitch0 = 0, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  if (!pitch0) pitch0 = d0;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {pitch0 * 2, pitch0 * d1 * 2};
  cuuint32_t box[3] = {b0, b1, b2};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(p), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
// the swizzle of a channel block of conv3x3_tc_kernel: rows of 2 x nch bytes
CUtensorMapSwizzle block_swizzle(int nch) {
  return nch == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : nch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}

// 3x3 convolution on the tensor cores (amh_conv_tc.cuh): x (H, W, Cin), w (9,
// Cout, Cin), Cin and Cout multiples of 16, Cout at most 128
int conv(amh_net* n, const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, const __nv_bfloat16* skip,
         __nv_bfloat16* y16, __nv_bfloat16* r16, float* y32, int H, int W, int Cin, int Cout, int relu) {
  if (Cin % 16 || Cin > 128 || Cin % 64 == 48 || Cout % 16 || Cout > tc::kMaxCout)
    return nfail(n, AMH_EINVAL, "conv: channel counts");
  const tc::ConvPlan p = tc::conv_plan(Cin, Cout);
  // one map per kind of channel block (64 channels; the 16 or 32 of the
  // tail); a kind the layer lacks gets a copy of the other
  CUtensorMap mx[2], mw[2];
  const int tail = Cin % 64;
  bool ok = true;
  if (Cin >= 64)
    ok = bf16_map(&mx[0], x, Cin, W, H, 64, tc::kHalo, 1, 0, block_swizzle(64)) &&
         bf16_map(&mw[0], w, Cin, Cout, 9, 64, p.Nb, 1, 0, block_swizzle(64));
  if (ok && tail)
    ok = bf16_map(&mx[1], x, Cin, W, H, tail, tc::kHalo, 1, 0, block_swizzle(tail)) &&
         bf16_map(&mw[1], w, Cin, Cout, 9, tail, p.Nb, 1, 0, block_swizzle(tail));
  if (!ok) return nfail(n, AMH_ECUDA, "conv: tensor map encoding failed");
  if (Cin < 64) mx[0] = mx[1], mw[0] = mw[1];
  if (!tail) mx[1] = mx[0], mw[1] = mw[0];
  const tc::ConvTcArgs a{bias, skip, y16, r16, y32, n->status, H, W, Cin, Cout, relu, p.Nb, p.S};
  // persistent grid: per channel block, as many CTAs as fit on the SMs at
  // once (every CTA holds its tensor memory until it exits), at most one per
  // tile
  static int n_sm[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!n_sm[dev & 63]) cudaDeviceGetAttribute(&n_sm[dev & 63], cudaDevAttrMultiProcessorCount, dev);
  // the decoder layers (skip input, two BF16 outputs) write their outputs
  // in whole sectors through lane pairs (tc::store_sector_pair)
  const int pair = skip ? 1 : 0;
  static std::once_flag once[64];
  static cudaError_t attr_err[64] = {};
  static int regs[64][2] = {};
  std::call_once(once[dev & 63], [dev] {
    cudaError_t e = cudaSuccess;
    cudaFuncAttributes fa;
    const void* kerns[2] = {reinterpret_cast<const void*>(tc::conv3x3_tc_kernel<false>),
                            reinterpret_cast<const void*>(tc::conv3x3_tc_kernel<true>)};
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
      e = cudaFuncSetAttribute(kerns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kConvSmemCap);
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kerns[k]);
      if (e == cudaSuccess) regs[dev & 63][k] = fa.numRegs;
    }
    attr_err[dev & 63] = e;
  });
  if (attr_err[dev & 63] != cudaSuccess)
    return nfail(n, AMH_ECUDA, "conv: shared-memory attribute: %s", cudaGetErrorString(attr_err[dev & 63]));
  if (p.smem > tc::kConvSmemCap) return nfail(n, AMH_EINVAL, "conv: shared memory plan too large");
  // CTAs resident per SM: the plan's, and what the register file holds
  const int threads = tc::conv_threads(p.Nb);
  const int by_regs = 65536 / (((regs[dev & 63][pair] + 7) & ~7) * threads);
  const int cps = std::max(1, std::min(p.ctas_per_sm, by_regs));
  const int nblk = Cout / p.Nb, ntiles = H * ((W + tc::kM - 1) / tc::kM);
  const int gx = std::max(1, std::min(ntiles, n_sm[dev & 63] * cps / nblk));
  if (pair)
    tc::conv3x3_tc_kernel<true><<<dim3(gx, nblk), threads, p.smem, n->stream>>>(mx[0], mx[1], mw[0], mw[1], a);
  else
    tc::conv3x3_tc_kernel<false><<<dim3(gx, nblk), threads, p.smem, n->stream>>>(mx[0], mx[1], mw[0], mw[1], a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(n, AMH_ECUDA, "conv launch: %s", cudaGetErrorString(e));
  return AMH_OK;
}
// weight gradient of layer L from its input x and its output gradient (FP32
// dy for the bias, its BF16 copy dy16 for the weights): the tensor-core
// kernel reads both pixel-major and sums a band of rows per CTA (all nine
// taps when Cout <= 32, else the three of one vertical tap) into gw
int wgrad(amh_net* n, int L, const __nv_bfloat16* x, const float* dy, const __nv_bfloat16* dy16, int H, int W) {
  const int Cin = kNet[L].cin, Cout = kNet[L].cout, np = H * W;
  const int stacked = Cout <= 32 ? 1 : 0, cba = stacked ? Cout : 64, cbb = tc::wgrad_xbox(Cin);
  CUtensorMap mdy, mx;
  if (!bf16_map(&mdy, dy16, Cout, W, H, cba, 64, 1, 0, block_swizzle(cba)) ||
      !bf16_map(&mx, x, Cin, W, H, cbb, 66, 1, 0, block_swizzle(cbb)))
    return nfail(n, AMH_ECUDA, "wgrad: tensor map encoding failed");
  const int S = tc::wgrad_stages(Cin);
  const size_t smem = (size_t)S * tc::wgrad_stage_bytes(Cin) + tc::kWgSlack;
  int dev = 0;
  cudaGetDevice(&dev);
  static std::once_flag once[64];
  static cudaError_t attr_err[64] = {};
  std::call_once(once[dev & 63], [dev] {
    attr_err[dev & 63] = cudaFuncSetAttribute(tc::wgrad3x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(tc::kWgSmemCap + tc::kWgSlack));
  });
  if (attr_err[dev & 63] != cudaSuccess)
    return nfail(n, AMH_ECUDA, "wgrad: shared-memory attribute: %s", cudaGetErrorString(attr_err[dev & 63]));
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per SM (the ring takes most of the shared memory), each an equal
  // share of the (row, 64-pixel chunk) steps
  const int gy = stacked ? 1 : 3, steps = H * ((W + 63) / 64);
  const int per_cta = (steps + std::max(1, n_sm / gy) - 1) / std::max(1, n_sm / gy);
  const tc::WgradTcArgs a{n->gw[L], n->status, H, W, Cin, Cout, per_cta, stacked, S};
  tc::wgrad3x3_tc_kernel<<<dim3((steps + per_cta - 1) / per_cta, gy), tc::kThreads, smem, n->stream>>>(mdy, mx, a);
  // about eight blocks per SM (at most kBiasBlocks), each a whole number of
  // the block's pixel steps
  const int step = 256 / (Cout / 4), want = std::min(kBiasBlocks, 8 * n_sm), per = (np + want - 1) / want;
  const int per_block = std::max(step, (per + step - 1) / step * step), nb = (np + per_block - 1) / per_block;
  bias_grad_kernel<<<nb, 256, 0, n->stream>>>(dy, np, Cout, per_block, n->bpart);
  bias_sum_kernel<<<Cout, 256, 0, n->stream>>>(n->bpart, nb, Cout, n->gb[L]);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(n, AMH_ECUDA, "wgrad launch: %s", cudaGetErrorString(e));
  return AMH_OK;
}
// data gradient of layer L: dx (FP32, H x W x Cin) from dy (BF16 copy in g16)
int dgrad(amh_net* n, int L, const __nv_bfloat16* dy16, float* dx, int H, int W) {
  return conv(n, dy16, n->wd16[L], nullptr, nullptr, nullptr, nullptr, dx, H, W, kNet[L].cout, kNet[L].cin, 0);
}
}  // namespace

extern "C" {

AMH_API int amh_net_create(amh_net** out, int32_t width2, int32_t height2, uint64_t seed, void* stream) {
  g_net_err.clear();
  if (!out) return nfail(nullptr, AMH_EINVAL, "out is NULL");
  *out = nullptr;
  if (width2 < 8 || height2 < 8 || width2 % 8 || height2 % 8 || (size_t)width2 * height2 > (1u << 24))
    return nfail(nullptr, AMH_EINVAL, "network size must be positive multiples of 8 (at most 2^24 pixels)");
  amh_net* n = new (std::nothrow) amh_net();
  if (!n) return nfail(nullptr, AMH_ENOMEM, "host allocation failed");
  n->w2 = width2;
  n->h2 = height2;
  n->stream = (cudaStream_t)stream;
  auto bail = [&](int code) {
    g_net_err = n->err;
    for (void* p : n->allocs) cudaFree(p);
    delete n;
    return code;
  };
#define NA(p, c)                                                  \
  do {                                                            \
    cudaError_t e_ = nalloc(n, &(p), (c));                        \
    if (e_ != cudaSuccess) {                                      \
      nfail(n, AMH_ENOMEM, "allocation: %s", cudaGetErrorString(e_)); \
      return bail(AMH_ENOMEM);                                    \
    }                                                             \
  } while (0)
  // He-normal initial weights from a seeded host generator (Box-Muller over
  // a 64-bit LCG), zero biases
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (int L = 0; L < kLayers; L++) {
    const int Cin = kNet[L].cin, Cout = kNet[L].cout;
    const size_t nw = (size_t)9 * Cin * Cout;
    NA(n->wm[L], nw); NA(n->w16[L], nw); NA(n->wd16[L], nw); NA(n->mw[L], nw); NA(n->vw[L], nw); NA(n->gw[L], nw);
    NA(n->bm[L], Cout); NA(n->mb[L], Cout); NA(n->vb[L], Cout); NA(n->gb[L], Cout);
    std::vector<float> w(nw);
    const double sd = std::sqrt(2.0 / (9.0 * Cin)) * (L == kLayers - 1 ? 0.1 : 1.0);
    for (size_t i = 0; i < nw; i++) w[i] = (float)(sd * std::sqrt(-2.0 * std::log(uni())) * std::cos(6.283185307179586 * uni()));
    cudaMemcpyAsync(n->wm[L], w.data(), nw * sizeof(float), cudaMemcpyHostToDevice, n->stream);
    cudaStreamSynchronize(n->stream);
  }
  NA(n->bpart, (size_t)kBiasBlocks * 128);
  NA(n->status, 1);
  const size_t P0 = (size_t)width2 * height2, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  NA(n->x0, P0 * 16); NA(n->e1, P0 * 32); NA(n->in_e2, P1 * 32); NA(n->e2, P1 * 64); NA(n->in_e3, P2 * 64);
  NA(n->e3, P2 * 96); NA(n->in_e4, P3 * 96); NA(n->e4, P3 * 128); NA(n->in_d3, P2 * 128); NA(n->r3, P2 * 96);
  NA(n->d3, P2 * 96); NA(n->in_d2, P1 * 96); NA(n->r2, P1 * 64); NA(n->d2, P1 * 64); NA(n->in_d1, P0 * 64);
  NA(n->r1, P0 * 32); NA(n->d1, P0 * 32);
  n->maxel = P0 * 64;
  NA(n->g16, n->maxel); NA(n->gA, n->maxel); NA(n->gB, n->maxel);
  {
    const size_t lp[kLayers] = {P0, P1, P2, P3, P2, P1, P0, P0};   // output size of each layer
    for (int L = 0; L < kLayers; L++) NA(n->dy[L], lp[L] * kNet[L].cout);
  }
  NA(n->gE1, P0 * 32); NA(n->gE2, P1 * 64); NA(n->gE3, P2 * 96);
  NA(n->out, P0 * 16); NA(n->target, P0 * 4); NA(n->mask, P0); NA(n->pin, P0); NA(n->prop, P0); NA(n->loss, 1);
#undef NA
  for (int L = 0; L < kLayers; L++) {
    const size_t nw = (size_t)9 * kNet[L].cin * kNet[L].cout;
    to_bf16_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->wm[L], n->w16[L], nw);
    flip_transpose_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->w16[L], n->wd16[L], kNet[L].cin, kNet[L].cout);
  }
  cudaError_t e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    nfail(n, AMH_ECUDA, "net init: %s", cudaGetErrorString(e));
    return bail(AMH_ECUDA);
  }
  *out = n;
  return AMH_OK;
}

AMH_API int amh_net_params(amh_net* n, int32_t layer, float* w, float* b, int32_t set) {
  if (!n || layer < 0 || layer >= kLayers) return AMH_EINVAL;
  const size_t nw = (size_t)9 * kNet[layer].cin * kNet[layer].cout, nb = kNet[layer].cout;
  if (set) {
    if (w) NTRY(n, cudaMemcpyAsync(n->wm[layer], w, nw * 4, cudaMemcpyHostToDevice, n->stream));
    if (b) NTRY(n, cudaMemcpyAsync(n->bm[layer], b, nb * 4, cudaMemcpyHostToDevice, n->stream));
    to_bf16_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->wm[layer], n->w16[layer], nw);
    flip_transpose_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->w16[layer], n->wd16[layer], kNet[layer].cin,
                                                                kNet[layer].cout);
  } else {
    if (w) NTRY(n, cudaMemcpyAsync(w, n->wm[layer], nw * 4, cudaMemcpyDeviceToHost, n->stream));
    if (b) NTRY(n, cudaMemcpyAsync(b, n->bm[layer], nb * 4, cudaMemcpyDeviceToHost, n->stream));
  }
  NTRY(n, cudaStreamSynchronize(n->stream));
  return AMH_OK;
}

AMH_API int amh_net_grads(amh_net* n, int32_t layer, float* gw, float* gb) {
  if (!n || layer < 0 || layer >= kLayers) return AMH_EINVAL;
  const size_t nw = (size_t)9 * kNet[layer].cin * kNet[layer].cout, nb = kNet[layer].cout;
  if (gw) NTRY(n, cudaMemcpyAsync(gw, n->gw[layer], nw * 4, cudaMemcpyDeviceToHost, n->stream));
  if (gb) NTRY(n, cudaMemcpyAsync(gb, n->gb[layer], nb * 4, cudaMemcpyDeviceToHost, n->stream));
  NTRY(n, cudaStreamSynchronize(n->stream));
  return AMH_OK;
}

// input features (H2 x W2 x 16) from the host (tests), or from a context
AMH_API int amh_net_set_input(amh_net* n, const float* x0_host) {
  if (!n || !x0_host) return AMH_EINVAL;
  const size_t ne = (size_t)n->w2 * n->h2 * 16;
  std::vector<__nv_bfloat16> h(ne);
  for (size_t i = 0; i < ne; i++) h[i] = __float2bfloat16(x0_host[i]);
  NTRY(n, cudaMemcpyAsync(n->x0, h.data(), ne * 2, cudaMemcpyHostToDevice, n->stream));
  NTRY(n, cudaStreamSynchronize(n->stream));
  return AMH_OK;
}

AMH_API int amh_net_set_example(amh_net* n, const float* x, int32_t channels, const float* target,
                                const uint8_t* mask, int32_t mirror, int32_t mem) {
  if (!n || !x || !target || !mask) return AMH_EINVAL;
  if (channels < 1 || channels > 16) return nfail(n, AMH_EINVAL, "channels must be 1..16");
  if (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE) return nfail(n, AMH_EINVAL, "bad memory kind");
  const size_t np = (size_t)n->w2 * n->h2;
  const float *dx = x, *dt = target;
  const uint8_t* dm = mask;
  if (mem == AMH_MEM_HOST) {   // into the scratch buffers (gA: features, gB: targets, then the mask)
    NTRY(n, cudaMemcpyAsync(n->gA, x, np * channels * 4, cudaMemcpyHostToDevice, n->stream));
    NTRY(n, cudaMemcpyAsync(n->gB, target, np * 16, cudaMemcpyHostToDevice, n->stream));
    uint8_t* mb = reinterpret_cast<uint8_t*>(n->gB + np * 4);
    NTRY(n, cudaMemcpyAsync(mb, mask, np, cudaMemcpyHostToDevice, n->stream));
    dx = n->gA;
    dt = n->gB;
    dm = mb;
  }
  if (reinterpret_cast<uintptr_t>(dt) & 15) {   // the kernel reads each pixel's targets as one float4
    NTRY(n, cudaMemcpyAsync(n->gB, dt, np * 16, cudaMemcpyDeviceToDevice, n->stream));
    dt = n->gB;
  }
  example_kernel<<<blocks_for(np), 256, 0, n->stream>>>(dx, channels, dt, dm, n->w2, n->h2, mirror & 3, n->x0,
                                                        n->target, n->mask);
  NTRY(n, cudaGetLastError());
  return AMH_OK;
}

AMH_API int amh_net_features(amh_net* n, amh_ctx* c) {
  if (!n || !c) return AMH_EINVAL;
  if ((c->W + 1) / 2 > n->w2 || (c->H + 1) / 2 > n->h2) return nfail(n, AMH_EINVAL, "context larger than the network");
  const float lmid = 0.5f * (std::log(c->p.depth_min) + std::log(c->p.depth_max));
  const float lscale = 2.f / std::max(1e-6f, std::log(c->p.depth_max / c->p.depth_min));
  NTRY(n, cudaMemsetAsync(n->x0, 0, (size_t)n->w2 * n->h2 * 16 * 2, n->stream));
  features_kernel<<<blocks_for((size_t)n->w2 * n->h2), 256, 0, n->stream>>>(
      c->d_ref, c->args.img_half, c->d_plane, c->d_cost, c->W, c->H, n->w2, n->h2, lmid, lscale, n->x0, n->pin);
  NTRY(n, cudaGetLastError());
  return AMH_OK;
}

AMH_API int amh_net_targets(amh_net* n, amh_ctx* c, float cost_max) {
  if (!n || !c) return AMH_EINVAL;
  targets_kernel<<<blocks_for((size_t)n->w2 * n->h2), 256, 0, n->stream>>>(
      c->d_plane, c->d_cost, n->pin, c->W, c->H, n->w2, n->h2, cost_max, n->target, n->mask);
  NTRY(n, cudaGetLastError());
  return AMH_OK;
}

AMH_API int amh_net_set_targets(amh_net* n, const float* target_host, const uint8_t* mask_host) {
  if (!n || !target_host || !mask_host) return AMH_EINVAL;
  const size_t np = (size_t)n->w2 * n->h2;
  NTRY(n, cudaMemcpyAsync(n->target, target_host, np * 16, cudaMemcpyHostToDevice, n->stream));
  NTRY(n, cudaMemcpyAsync(n->mask, mask_host, np, cudaMemcpyHostToDevice, n->stream));
  NTRY(n, cudaStreamSynchronize(n->stream));
  return AMH_OK;
}

AMH_API int amh_net_forward(amh_net* n, float* out_host) {
  if (!n) return AMH_EINVAL;
  const int W0 = n->w2, H0 = n->h2, W1 = W0 / 2, H1 = H0 / 2, W2 = W1 / 2, H2 = H1 / 2, W3 = W2 / 2, H3 = H2 / 2;
  const cudaStream_t s = n->stream;
  int rc = conv(n, n->x0, n->w16[0], n->bm[0], nullptr, n->e1, nullptr, nullptr, H0, W0, 16, 32, 1);
  pool2_kernel<<<blocks_for((size_t)H1 * W1 * 32), 256, 0, s>>>(n->e1, n->in_e2, H0, W0, 32);
  if (!rc) rc = conv(n, n->in_e2, n->w16[1], n->bm[1], nullptr, n->e2, nullptr, nullptr, H1, W1, 32, 64, 1);
  pool2_kernel<<<blocks_for((size_t)H2 * W2 * 64), 256, 0, s>>>(n->e2, n->in_e3, H1, W1, 64);
  if (!rc) rc = conv(n, n->in_e3, n->w16[2], n->bm[2], nullptr, n->e3, nullptr, nullptr, H2, W2, 64, 96, 1);
  pool2_kernel<<<blocks_for((size_t)H3 * W3 * 96), 256, 0, s>>>(n->e3, n->in_e4, H2, W2, 96);
  if (!rc) rc = conv(n, n->in_e4, n->w16[3], n->bm[3], nullptr, n->e4, nullptr, nullptr, H3, W3, 96, 128, 1);
  up2_kernel<<<blocks_for((size_t)H2 * W2 * 128), 256, 0, s>>>(n->e4, n->in_d3, H2, W2, 128);
  if (!rc) rc = conv(n, n->in_d3, n->w16[4], n->bm[4], n->e3, n->d3, n->r3, nullptr, H2, W2, 128, 96, 1);
  up2_kernel<<<blocks_for((size_t)H1 * W1 * 96), 256, 0, s>>>(n->d3, n->in_d2, H1, W1, 96);
  if (!rc) rc = conv(n, n->in_d2, n->w16[5], n->bm[5], n->e2, n->d2, n->r2, nullptr, H1, W1, 96, 64, 1);
  up2_kernel<<<blocks_for((size_t)H0 * W0 * 64), 256, 0, s>>>(n->d2, n->in_d1, H0, W0, 64);
  if (!rc) rc = conv(n, n->in_d1, n->w16[6], n->bm[6], n->e1, n->d1, n->r1, nullptr, H0, W0, 64, 32, 1);
  if (!rc) rc = conv(n, n->d1, n->w16[7], n->bm[7], nullptr, nullptr, nullptr, n->out, H0, W0, 32, 16, 0);
  if (rc) return rc;
  NTRY(n, cudaGetLastError());
  if (out_host) {
    NTRY(n, cudaMemcpyAsync(out_host, n->out, (size_t)H0 * W0 * 16 * 4, cudaMemcpyDeviceToHost, s));
    NTRY(n, cudaStreamSynchronize(s));
  }
  return AMH_OK;
}

// loss of the last forward against the targets, and all gradients
AMH_API int amh_net_backward(amh_net* n, float* loss_out) {
  if (!n) return AMH_EINVAL;
  const int W0 = n->w2, H0 = n->h2, W1 = W0 / 2, H1 = H0 / 2, W2 = W1 / 2, H2 = H1 / 2, W3 = W2 / 2, H3 = H2 / 2;
  const size_t P0 = (size_t)W0 * H0, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  const cudaStream_t s = n->stream;
  // mask count on the host side of the stream
  std::vector<uint8_t> mk(P0);
  NTRY(n, cudaMemcpyAsync(mk.data(), n->mask, P0, cudaMemcpyDeviceToHost, s));
  NTRY(n, cudaStreamSynchronize(s));
  size_t cnt = 0;
  for (uint8_t m : mk) cnt += m;
  const float inv_n = 1.f / (float)std::max<size_t>(1, cnt);
  for (int L = 0; L < kLayers; L++) {
    NTRY(n, cudaMemsetAsync(n->gw[L], 0, (size_t)9 * kNet[L].cin * kNet[L].cout * 4, s));
    NTRY(n, cudaMemsetAsync(n->gb[L], 0, (size_t)kNet[L].cout * 4, s));
  }
  NTRY(n, cudaMemsetAsync(n->loss, 0, 4, s));
  float* const* dy = n->dy;
  l1_loss_kernel<<<blocks_for(P0), 256, 0, s>>>(n->out, n->target, n->mask, dy[7], n->loss, (int)P0, inv_n);
  // out = conv(d1)
  to_bf16_kernel<<<blocks_for(P0 * 16), 256, 0, s>>>(dy[7], n->g16, P0 * 16);
  int rc = wgrad(n, 7, n->d1, dy[7], n->g16, H0, W0);
  if (!rc) rc = dgrad(n, 7, n->g16, n->gA, H0, W0);                  // gA = d d1 (P0 x 32)
  // d1 = relu(conv(in_d1)) + e1
  NTRY(n, cudaMemcpyAsync(n->gE1, n->gA, P0 * 32 * 4, cudaMemcpyDeviceToDevice, s));
  relu_mask_kernel<<<blocks_for(P0 * 32), 256, 0, s>>>(n->gA, n->r1, dy[6], n->g16, P0 * 32);
  if (!rc) rc = wgrad(n, 6, n->in_d1, dy[6], n->g16, H0, W0);
  if (!rc) rc = dgrad(n, 6, n->g16, n->gA, H0, W0);                  // d in_d1 (P0 x 64)
  up2_bwd_kernel<<<blocks_for(P1 * 64), 256, 0, s>>>(n->gA, n->gE2, H1, W1, 64);  // d d2 (P1 x 64)
  relu_mask_kernel<<<blocks_for(P1 * 64), 256, 0, s>>>(n->gE2, n->r2, dy[5], n->g16, P1 * 64);
  if (!rc) rc = wgrad(n, 5, n->in_d2, dy[5], n->g16, H1, W1);
  if (!rc) rc = dgrad(n, 5, n->g16, n->gA, H1, W1);                  // d in_d2 (P1 x 96)
  up2_bwd_kernel<<<blocks_for(P2 * 96), 256, 0, s>>>(n->gA, n->gE3, H2, W2, 96);  // d d3 (P2 x 96)
  relu_mask_kernel<<<blocks_for(P2 * 96), 256, 0, s>>>(n->gE3, n->r3, dy[4], n->g16, P2 * 96);
  if (!rc) rc = wgrad(n, 4, n->in_d3, dy[4], n->g16, H2, W2);
  if (!rc) rc = dgrad(n, 4, n->g16, n->gA, H2, W2);                  // d in_d3 (P2 x 128)
  up2_bwd_kernel<<<blocks_for(P3 * 128), 256, 0, s>>>(n->gA, n->gB, H3, W3, 128); // d e4 (P3 x 128)
  // e4 = relu(conv(in_e4))
  relu_mask_kernel<<<blocks_for(P3 * 128), 256, 0, s>>>(n->gB, n->e4, dy[3], n->g16, P3 * 128);
  if (!rc) rc = wgrad(n, 3, n->in_e4, dy[3], n->g16, H3, W3);
  if (!rc) rc = dgrad(n, 3, n->g16, n->gA, H3, W3);                  // d in_e4 (P3 x 96)
  pool2_bwd_add_kernel<<<blocks_for(P2 * 96), 256, 0, s>>>(n->gA, n->gE3, H2, W2, 96);
  // e3 = relu(conv(in_e3)), read by d3 (skip) and by the pooling
  relu_mask_kernel<<<blocks_for(P2 * 96), 256, 0, s>>>(n->gE3, n->e3, dy[2], n->g16, P2 * 96);
  if (!rc) rc = wgrad(n, 2, n->in_e3, dy[2], n->g16, H2, W2);
  if (!rc) rc = dgrad(n, 2, n->g16, n->gA, H2, W2);                  // d in_e3 (P2 x 64)
  pool2_bwd_add_kernel<<<blocks_for(P1 * 64), 256, 0, s>>>(n->gA, n->gE2, H1, W1, 64);
  relu_mask_kernel<<<blocks_for(P1 * 64), 256, 0, s>>>(n->gE2, n->e2, dy[1], n->g16, P1 * 64);
  if (!rc) rc = wgrad(n, 1, n->in_e2, dy[1], n->g16, H1, W1);
  if (!rc) rc = dgrad(n, 1, n->g16, n->gA, H1, W1);                  // d in_e2 (P1 x 32)
  pool2_bwd_add_kernel<<<blocks_for(P0 * 32), 256, 0, s>>>(n->gA, n->gE1, H0, W0, 32);
  relu_mask_kernel<<<blocks_for(P0 * 32), 256, 0, s>>>(n->gE1, n->e1, dy[0], n->g16, P0 * 32);
  if (!rc) rc = wgrad(n, 0, n->x0, dy[0], n->g16, H0, W0);
  if (rc) return rc;
  NTRY(n, cudaGetLastError());
  if (loss_out) {
    NTRY(n, cudaMemcpyAsync(loss_out, n->loss, 4, cudaMemcpyDeviceToHost, s));
    NTRY(n, cudaStreamSynchronize(s));
  }
  return AMH_OK;
}

AMH_API int amh_net_adam(amh_net* n, float lr) {
  if (!n) return AMH_EINVAL;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
  for (int L = 0; L < kLayers; L++) {
    const size_t nw = (size_t)9 * kNet[L].cin * kNet[L].cout;
    adam_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->wm[L], n->mw[L], n->vw[L], n->gw[L], n->w16[L], (int)nw,
                                                     lr, b1, b2, 1e-8f, c1, c2);
    adam_kernel<<<1, 256, 0, n->stream>>>(n->bm[L], n->mb[L], n->vb[L], n->gb[L], nullptr, kNet[L].cout, lr, b1, b2,
                                         1e-8f, c1, c2);
    flip_transpose_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->w16[L], n->wd16[L], kNet[L].cin, kNet[L].cout);
  }
  NTRY(n, cudaGetLastError());
  return AMH_OK;
}

// the proposal planes of the last forward, handed to the context's phases
AMH_API int amh_net_propose(amh_net* n, amh_ctx* c) {
  if (!n || !c) return AMH_EINVAL;
  head_kernel<<<blocks_for((size_t)n->w2 * n->h2), 256, 0, n->stream>>>(n->out, n->pin, c->W, c->H, n->w2, n->h2,
                                                                        c->args, n->prop);
  NTRY(n, cudaGetLastError());
  c->args.prop = n->prop;
  c->args.prop_w = n->w2;
  c->args.prop_h = n->h2;
  return AMH_OK;
}

AMH_API int amh_clear_proposal(amh_ctx* c) {
  if (!c) return AMH_EINVAL;
  c->args.prop = nullptr;
  return AMH_OK;
}

// internal tensors for element-wise checks of every operation
AMH_API int amh_net_read(amh_net* n, int32_t which, float* out, int64_t* count) {
  if (!n || !count) return AMH_EINVAL;
  const size_t P0 = (size_t)n->w2 * n->h2, P1 = P0 / 4, P2 = P0 / 16, P3 = P0 / 64;
  struct B { const __nv_bfloat16* b; const float* f; size_t n; };
  const B act[] = {{n->x0, nullptr, P0 * 16},   {n->e1, nullptr, P0 * 32},    {n->in_e2, nullptr, P1 * 32},
                   {n->e2, nullptr, P1 * 64},   {n->in_e3, nullptr, P2 * 64}, {n->e3, nullptr, P2 * 96},
                   {n->in_e4, nullptr, P3 * 96}, {n->e4, nullptr, P3 * 128},  {n->in_d3, nullptr, P2 * 128},
                   {n->r3, nullptr, P2 * 96},   {n->d3, nullptr, P2 * 96},    {n->in_d2, nullptr, P1 * 96},
                   {n->r2, nullptr, P1 * 64},   {n->d2, nullptr, P1 * 64},    {n->in_d1, nullptr, P0 * 64},
                   {n->r1, nullptr, P0 * 32},   {n->d1, nullptr, P0 * 32},    {nullptr, n->out, P0 * 16}};
  constexpr int kAct = (int)(sizeof(act) / sizeof(act[0]));
  const size_t lp[kLayers] = {P0, P1, P2, P3, P2, P1, P0, P0};
  B src{};
  if (which == 65) {   // the mask, as 0 / 1
    if (!out) {
      *count = (int64_t)P0;
      return AMH_OK;
    }
    if (*count != (int64_t)P0) return nfail(n, AMH_EINVAL, "the mask has %zu elements", P0);
    std::vector<uint8_t> h(P0);
    NTRY(n, cudaMemcpyAsync(h.data(), n->mask, P0, cudaMemcpyDeviceToHost, n->stream));
    NTRY(n, cudaStreamSynchronize(n->stream));
    for (size_t i = 0; i < P0; i++) out[i] = (float)h[i];
    return AMH_OK;
  }
  if (which >= 0 && which < kAct) src = act[which];
  else if (which >= 32 && which < 32 + kLayers) src = B{nullptr, n->dy[which - 32], lp[which - 32] * kNet[which - 32].cout};
  else if (which == 64) src = B{nullptr, n->target, P0 * 4};
  else return nfail(n, AMH_EINVAL, "unknown tensor %d", which);
  if (!out) {
    *count = (int64_t)src.n;
    return AMH_OK;
  }
  if (*count != (int64_t)src.n) return nfail(n, AMH_EINVAL, "tensor %d has %zu elements, not %lld", which, src.n, (long long)*count);
  const float* dev = src.f;
  if (src.b) {   // BF16 -> FP32 in the scratch buffer (the largest tensor fits)
    bf16_to_f32_kernel<<<blocks_for(src.n), 256, 0, n->stream>>>(src.b, n->gB, src.n);
    NTRY(n, cudaGetLastError());
    dev = n->gB;
  }
  NTRY(n, cudaMemcpyAsync(out, dev, src.n * 4, cudaMemcpyDeviceToHost, n->stream));
  NTRY(n, cudaStreamSynchronize(n->stream));
  return AMH_OK;
}

AMH_API int amh_net_synchronize(amh_net* n) {
  if (!n) return AMH_EINVAL;
  NTRY(n, cudaStreamSynchronize(n->stream));
  unsigned int st = 0;
  NTRY(n, cudaMemcpy(&st, n->status, sizeof st, cudaMemcpyDeviceToHost));
  if (st) return nfail(n, AMH_EDEVICE, "a convolution's barrier wait gave up (status 0x%x)", st);
  return AMH_OK;
}

AMH_API const char* amh_net_last_error(const amh_net* n) { return n ? n->err.c_str() : g_net_err.c_str(); }

AMH_API void amh_net_destroy(amh_net* n) {
  if (!n) return;
  cudaStreamSynchronize(n->stream);
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

}  // extern "C"
