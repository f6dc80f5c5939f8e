// amh_device.cuh -- device building blocks of the checkerboard update:
// Philox4x32-10, random planes, the plane-induced homography and the kernel
// argument block.
//
// Written for sm_103a.  FP32 arithmetic throughout; every source view is a
// uint8 texture read with tex2Dgather (four texels per fetch, clamp-to-edge
// addressing in the texture unit) and interpolated in FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amh {

constexpr int kMaxSrc = 32;
constexpr int kRegions = 8;
constexpr int kWinR = 5;                 // 11 x 11 window ...
constexpr int kWinStride = 2;            // ... every other row and column
constexpr int kWinN = 2 * kWinR / kWinStride + 1;   // 6 samples per axis
constexpr int kWinS = kWinN * kWinN;                // 36 samples
constexpr float kWorst = 2.0f;           // cost of an invalid (hypothesis, view)
constexpr int kMaxRefine = 6;
constexpr int kPairCounters = 64;        // striped evaluation counters

// Layout of the per-pixel state (plane, cost, S, v, selected views, winning
// row): each row holds its pixels of colour 0 ((x + y) even), then its
// pixels of colour 1, each run W2 = ceil(W / 2) entries long.  A checkerboard
// phase then reads and writes whole sectors of its own colour and leaves the
// other colour's sectors clean, where a row-major layout would dirty every
// sector with half of its bytes.  The library's calls take and return
// row-major maps; only the kernels see this layout.
__host__ __device__ __forceinline__ size_t state_size(int W, int H) { return (size_t)H * 2 * (size_t)((W + 1) >> 1); }
__host__ __device__ __forceinline__ size_t state_index(int x, int y, int W) {
  const size_t w2 = (size_t)((W + 1) >> 1);
  return (size_t)y * 2 * w2 + (((x + y) & 1) ? w2 : 0) + (size_t)(x >> 1);
}

// One source view.  A and b give the homography of a plane (n, d) as
// H = A - b c^T with c = K_ref^-T n / d (Sec. 2: planes in scene space), where
// A = K_j R_jr K_ref^-1 and b = K_j t_jr; P = K_j R_jr.  Rows 0 and 1 of A, b
// and P already hold row 2 added once, so H maps reference pixels to source
// coordinates + (1, 1): with integer part f of such a coordinate, tex2Dgather
// at f fetches the texels (f - 1, f) = (floor(x), floor(x) + 1).
// The image of a window centre is taken from the plane's 3-D point there,
// H (x, y, 1) = P ray + b / D (ray = K_ref^-1 (x, y, 1), D its depth), which
// in FP32 stays accurate for planes seen nearly edge-on, where the terms of
// H (x, y, 1) nearly cancel; the window offsets use H's first two columns.
struct ViewConst {
  float A[9];
  float b[3];
  float P[9];
  float xmax, ymax;          // width, height: valid shifted centres in [1, W] x [1, H]
  cudaTextureObject_t tex;   // point sampling, clamp; uint8 read as value / 255, or FP16
};
static_assert(sizeof(ViewConst) == 104, "ViewConst is 104 bytes");

struct PhaseArgs {
  int W, H, N, color, t;
  float Kinv[9];
  float tau;                 // tau_mc(t), Eq. (2)
  float tau_up;
  int n1, n2, k;
  float inv2beta2;           // 1 / (2 beta^2), Eq. (3)
  float wI, wX;              // 1 / (2 sigma_I^2), 1 / (2 sigma_x^2), Eq. (8)
  int squared;               // bilateral weight on squared differences
  int img_half;              // images are FP16 (else uint8)
  int ablation;              // bit 0: symmetric propagation, bit 1: heuristic views (Sec. 4)
  int tex_filter;            // samples through the texture unit's linear filter
  int staged;                // shared-memory staged matrix sweep (AMH_FLAG_STAGED_FETCH)
  float dmin, dmax;
  uint32_t key0, key1;       // Philox key (seed)
  const void* ref;           // reference image, W x H (uint8 or FP16)
  float4* plane;
  float* cost;
  uint32_t* sel;
  uint8_t* vbest;
  uint32_t* wmask;
  uint8_t* choice;
  unsigned long long* pairs; // kPairCounters striped (hypothesis, view) evaluation counters
  const float4* prop;        // learned proposals (n, d) on the (x/2, y/2) grid, or null
  int prop_w, prop_h;
  unsigned int* status;      // bounds-check status word (see checked_index)
  ViewConst v[kMaxSrc];
};

// Bounds-checked builds (compiled with -DAMH_BOUNDS_CHECK): every index the
// update computes into the state, the reference image or the proposals is
// checked; one out of range sets its bit in the status word and is replaced
// by 0, so the access stays inside the array, and the host turns the word
// into AMH_EDEVICE.  Other builds take the index as it is.
enum : unsigned { kBadPixel = 1u, kBadNeighbour = 2u, kBadReference = 4u, kBadProposal = 8u };
template <class A>
__device__ __forceinline__ size_t checked_index(const A& a, size_t i, size_t n, unsigned code) {
#ifdef AMH_BOUNDS_CHECK
  if (i >= n) {
    atomicOr(a.status, code);
    return 0;
  }
#else
  (void)a; (void)n; (void)code;
#endif
  return i;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32
// multiplications with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}
// uniform in [0, 1) from the top 24 bits (exact in FP32)
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// hardware reciprocal (MUFU), about 1 ulp
// Two FP32 lanes in one 64-bit register pair, for the packed f32x2
// arithmetic of sm_100-class SMs (one instruction issues both lanes; each lane
// rounds exactly as the scalar instruction would).
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 pack2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(f2 p, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
// floor of both lanes for |x| < 2^22: x + 2^23 rounded towards -inf is
// 2^23 + floor(x) exactly (the spacing there is 1), and removing 2^23 is exact
__device__ __forceinline__ f2 floor2(f2 x) {
  const f2 M = pack2(8388608.f, 8388608.f);
  f2 t;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(t.v) : "l"(x.v), "l"(M.v));
  return sub2(t, M);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------------------
// planes
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 ref_ray(const float* Ki, float x, float y) {
  return make_float3(fmaf(Ki[0], x, fmaf(Ki[1], y, Ki[2])), fmaf(Ki[3], x, fmaf(Ki[4], y, Ki[5])),
                     fmaf(Ki[6], x, fmaf(Ki[7], y, Ki[8])));
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

__device__ __forceinline__ float3 face_camera(float3 n, float3 ray) {
  if (!(dot3(n, ray) < 0.f)) { n.x = -n.x; n.y = -n.y; n.z = -n.z; }
  return n;
}
// unit normal: z uniform in [-1, 1), azimuth 2 pi u2
__device__ __forceinline__ float3 normal_from_uniforms(float u1, float u2) {
  float z = 2.f * u1 - 1.f;
  float r = sqrtf(fmaxf(0.f, 1.f - z * z));
  float s, c;
  sincospif(2.f * u2, &s, &c);
  return make_float3(r * c, r * s, z);
}

// The cost needs c = K_ref^-T n / d (Sec. 2) with d = -D (n . ray) the plane
// offset, and 1 / D (the window centre's image, see ViewConst); the plane is
// usable when it faces the pixel (d > 0) at D > 0.  c.w = 1 / D.
__device__ __forceinline__ bool plane_c(const float* Ki, float4 pl, float3 ray, float4* c) {
  const float3 n = make_float3(pl.x, pl.y, pl.z);
  const float d = -pl.w * dot3(n, ray);
  const bool ok = (pl.w > 0.f) && (d > 0.f) && isfinite(d);
  const float id = ok ? 1.f / d : 0.f;
  *c = make_float4((Ki[0] * n.x + Ki[3] * n.y + Ki[6] * n.z) * id,
                   (Ki[1] * n.x + Ki[4] * n.y + Ki[7] * n.z) * id,
                   (Ki[2] * n.x + Ki[5] * n.y + Ki[8] * n.z) * id, ok ? 1.f / pl.w : 0.f);
  return ok;
}

}  // namespace amh
