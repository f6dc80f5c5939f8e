// amh_device.cuh -- device building blocks of the checkerboard update:
// Philox4x32-10, random planes, the plane-induced homography, the warped
// bilateral weighted NCC over the skipping window (Eq. 8) and the
// multi-hypothesis joint view selection (Eqs. 2-7).
//
// Written for sm_103a.  FP32 arithmetic throughout; the source images are
// uint8 textures read with tex2Dgather (four texels per fetch, clamp-to-edge
// addressing done by the texture unit) and interpolated in FP32.
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

// One source view.  A and b give the homography of a plane (n, d) as
// H = A - b c^T with c = K_ref^-T n / d (Sec. 2: planes in scene space), where
// A = K_j R_jr K_ref^-1 and b = K_j t_jr; rows 0 and 1 already hold row 2
// added once, so that H maps reference pixels to source coordinates + (1, 1),
// the coordinate tex2Dgather needs to fetch texels (floor(x), floor(x) + 1).
struct ViewConst {
  float A[9];
  float b[3];
  float xmax, ymax;          // width, height (valid shifted centre: [1, W] x [1, H])
  cudaTextureObject_t tex;   // uint8, point sampling, clamp, normalised float
};

struct PhaseArgs {
  int W, H, N, color, t;
  float Kinv[9];
  float tau;                 // tau_mc(t), Eq. (2)
  float tau_up;
  int n1, n2, k;
  float inv2beta2;           // 1 / (2 beta^2), Eq. (3)
  float wI, wX;              // 1 / (2 sigma_I^2), 1 / (2 sigma_x^2), Eq. (8)
  int squared;               // bilateral weight on squared differences
  float dmin, dmax;
  uint32_t key0, key1;       // Philox key (seed)
  const uint8_t* ref;        // reference image, W x H
  float4* plane;
  float* cost;
  uint32_t* sel;
  uint8_t* vbest;
  uint32_t* wmask;
  uint8_t* choice;
  unsigned long long* pairs; // (hypothesis, view) evaluations
  ViewConst v[kMaxSrc];
};

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

// A hypothesis in the form the cost needs: c = K_ref^-T n / d (Sec. 2), with
// d = -D (n . ray) the plane offset; valid when the plane faces the pixel.
struct Hyp {
  float4 pl;    // (n, D at this pixel)
  float3 c;
  bool ok;
};
__device__ __forceinline__ Hyp make_hyp(const float* Ki, float4 pl, float3 ray) {
  Hyp h;
  h.pl = pl;
  float3 n = make_float3(pl.x, pl.y, pl.z);
  float d = -pl.w * dot3(n, ray);
  h.ok = (pl.w > 0.f) && (d > 0.f) && isfinite(d);
  float id = h.ok ? 1.f / d : 0.f;
  h.c = make_float3((Ki[0] * n.x + Ki[3] * n.y + Ki[6] * n.z) * id,
                    (Ki[1] * n.x + Ki[4] * n.y + Ki[7] * n.z) * id,
                    (Ki[2] * n.x + Ki[5] * n.y + Ki[8] * n.z) * id);
  return h;
}

// ---------------------------------------------------------------------------
// Reference window of one pixel (Sec. 3.3): 36 samples at offsets
// {-5,-3,-1,1,3,5}^2 clamped to the image, bilateral weights
// w = exp(-|I - I_c| / (2 sigma_I^2) - |dx| / (2 sigma_x^2)), and the
// weighted-centred reference values so that cov(r, s) = sum w r^ s / sum w.
// ---------------------------------------------------------------------------
struct RefWin {
  float w[kWinS];
  float wr[kWinS];    // w * (r - E_w r)
  float inv_sw;       // 1 / sum w
  float sum_wr;       // sum w (r - E_w r), ~0
  float var_r;        // weighted variance of r (0..255 units)
};

__device__ __forceinline__ void load_ref_window(const PhaseArgs& a, int x, int y, RefWin& rw) {
  const uint8_t* I = a.ref;
  const float Ic = (float)__ldg(&I[(size_t)y * a.W + x]);
  float rv[kWinS];
  float sw = 0.f, s1 = 0.f;
#pragma unroll
  for (int k = 0; k < kWinS; k++) {
    const int du = -kWinR + kWinStride * (k % kWinN), dv = -kWinR + kWinStride * (k / kWinN);
    const int xr = min(max(x + du, 0), a.W - 1), yr = min(max(y + dv, 0), a.H - 1);
    const float r = (float)__ldg(&I[(size_t)yr * a.W + xr]) - Ic;   // exact
    const float dist = sqrtf((float)(du * du + dv * dv));
    float dI = fabsf(r), dx = dist;
    if (a.squared) { dI = r * r; dx = (float)(du * du + dv * dv); }
    const float w = expf(-dI * a.wI - dx * a.wX);
    rv[k] = r;
    rw.w[k] = w;
    sw += w;
    s1 = fmaf(w, r, s1);
  }
  const float inv = 1.f / sw;
  const float mr = s1 * inv;
  float s2 = 0.f, swr = 0.f;
#pragma unroll
  for (int k = 0; k < kWinS; k++) {
    const float rc = rv[k] - mr;
    const float wr = rw.w[k] * rc;
    rw.wr[k] = wr;
    swr += wr;
    s2 = fmaf(wr, rc, s2);
  }
  rw.inv_sw = inv;
  rw.sum_wr = swr;
  rw.var_r = s2 * inv - (swr * inv) * (swr * inv);
}

// ---------------------------------------------------------------------------
// Eq. (8): cost of one hypothesis against one source view.  Returns 2 when
// the plane is invalid, lies behind view j over the window, or projects the
// centre outside view j, or when a patch has no variance; else clamps to
// [0, 2].  *evaluated is set when the 36 samples were taken.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ncc_cost(const ViewConst& V, const Hyp& h, float x, float y,
                                          const RefWin& rw, int* evaluated) {
  if (!h.ok) return kWorst;
  // H = A - b c^T
  const float H0 = fmaf(-V.b[0], h.c.x, V.A[0]), H1 = fmaf(-V.b[0], h.c.y, V.A[1]),
              H2 = fmaf(-V.b[0], h.c.z, V.A[2]);
  const float H3 = fmaf(-V.b[1], h.c.x, V.A[3]), H4 = fmaf(-V.b[1], h.c.y, V.A[4]),
              H5 = fmaf(-V.b[1], h.c.z, V.A[5]);
  const float H6 = fmaf(-V.b[2], h.c.x, V.A[6]), H7 = fmaf(-V.b[2], h.c.y, V.A[7]),
              H8 = fmaf(-V.b[2], h.c.z, V.A[8]);
  // homogeneous depth is affine over the window: check its minimum corner
  const float pz = fmaf(H6, x, fmaf(H7, y, H8));
  const float zmin = pz - (float)kWinR * (fabsf(H6) + fabsf(H7));
  if (!(zmin > 0.f)) return kWorst;
  const float px = fmaf(H0, x, fmaf(H1, y, H2)), py = fmaf(H3, x, fmaf(H4, y, H5));
  const float iz = 1.f / pz;
  const float cx = px * iz, cy = py * iz;
  if (!(cx >= 1.f && cx <= V.xmax && cy >= 1.f && cy <= V.ymax)) return kWorst;
  *evaluated = 1;
  // window corner (-R, -R) and the steps between samples
  const float sx0 = px - (float)kWinR * (H0 + H1), sy0 = py - (float)kWinR * (H3 + H4),
              sz0 = pz - (float)kWinR * (H6 + H7);
  const float cxs = (float)kWinStride * H0, cys = (float)kWinStride * H3, czs = (float)kWinStride * H6;
  const float rxs = (float)kWinStride * H1, rys = (float)kWinStride * H4, rzs = (float)kWinStride * H7;
  float s0 = 0.f, m1 = 0.f, m2 = 0.f, mrs = 0.f;
#pragma unroll
  for (int a = 0; a < kWinN; a++) {
    const float ax = fmaf((float)a, rxs, sx0), ay = fmaf((float)a, rys, sy0), az = fmaf((float)a, rzs, sz0);
#pragma unroll
    for (int b = 0; b < kWinN; b++) {
      const int k = a * kWinN + b;
      const float qx = fmaf((float)b, cxs, ax), qy = fmaf((float)b, cys, ay), qz = fmaf((float)b, czs, az);
      const float iq = rcp_approx(qz);
      const float gx = qx * iq, gy = qy * iq;
      const float fx0 = floorf(gx), fy0 = floorf(gy);
      const float fx = gx - fx0, fy = gy - fy0;
      // texels: w (x0, y0), z (x0+1, y0), x (x0, y0+1), y (x0+1, y0+1)
      const float4 g = tex2Dgather<float4>(V.tex, fx0, fy0, 0);
      const float top = fmaf(fx, g.z - g.w, g.w);
      const float bot = fmaf(fx, g.y - g.x, g.x);
      const float s = fmaf(fy, bot - top, top);
      if (k == 0) s0 = s;
      const float sc = s - s0;
      const float ws = rw.w[k] * sc;
      m1 += ws;
      m2 = fmaf(ws, sc, m2);
      mrs = fmaf(rw.wr[k], sc, mrs);
    }
  }
  const float es = m1 * rw.inv_sw;
  const float var_s = fmaf(m2, rw.inv_sw, -es * es);
  const float cov = fmaf(mrs, rw.inv_sw, -(rw.sum_wr * rw.inv_sw) * es);
  // variances in (0..255)^2 units: the texture returns intensities / 255
  const float vv = rw.var_r * var_s * (255.f * 255.f);
  if (!(vv >= 1e-10f)) return kWorst;
  float m = 1.f - cov * (255.f * rsqrtf(vv));
  return fminf(fmaxf(m, 0.f), 2.f);
}

}  // namespace amh
