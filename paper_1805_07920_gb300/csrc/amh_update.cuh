// amh_update.cuh -- one pixel's checkerboard update and its parts, shared by
// the single-reference kernels (amh_kernels.cu) and the batched persistent
// kernels (amh_batch.cu).  The argument block is a template parameter: any
// struct with the fields of PhaseArgs (sizes, parameters, state pointers and
// an indexable view table v) works.
//
// Work mapping: one thread per reference pixel; a warp updates 32 pixels of
// one colour of a compact tile, so the lanes of every texture gather sample
// neighbouring windows of the same source view.  Every (hypothesis, view)
// loop runs with a warp-uniform view index (uniform texture handle).  Each
// thread keeps its 36 bilateral weights in registers and its cost matrix and
// view weights in local memory (L1); no shared memory is needed, so the whole
// L1 serves the texture gathers.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "amh_device.cuh"

namespace amh {
namespace upd {


// Sec. 3.1, Fig. 2(d): candidate c of the 72 in scan order.  Regions 0..3
// (near up/down/left/right) hold 7 candidates: the axis pixel at distance 1
// and the pairs at lateral offset -+a, distance a + 1 (a = 1..3); regions
// 4..7 (far) hold the axis pixels at distances 3, 5, ..., 23.
__host__ __device__ constexpr int acp_region(int c) { return c < 28 ? c / 7 : 4 + (c - 28) / 11; }
__host__ __device__ constexpr int acp_index(int c) { return c < 28 ? c % 7 : (c - 28) % 11; }
__host__ __device__ constexpr int acp_start(int g) { return g < 4 ? 7 * g : 28 + 11 * (g - 4); }
__host__ __device__ constexpr int acp_depth(int c) {
  return acp_region(c) < 4 ? (acp_index(c) + 1) / 2 + 1 : 3 + 2 * acp_index(c);
}
__host__ __device__ constexpr int acp_lateral(int c) {
  return acp_region(c) < 4 && acp_index(c) > 0 ? ((acp_index(c) & 1) ? -1 : 1) * ((acp_index(c) + 1) / 2) : 0;
}
__host__ __device__ constexpr int acp_dx(int c) {
  return (acp_region(c) & 3) == 2 ? -acp_depth(c) : (acp_region(c) & 3) == 3 ? acp_depth(c) : acp_lateral(c);
}
__host__ __device__ constexpr int acp_dy(int c) {
  return (acp_region(c) & 3) == 0 ? -acp_depth(c) : (acp_region(c) & 3) == 1 ? acp_depth(c) : acp_lateral(c);
}
static_assert(acp_dx(0) == 0 && acp_dy(0) == -1, "near up starts at (0, -1)");
static_assert(acp_dx(1) == -1 && acp_dy(1) == -2 && acp_dx(2) == 1 && acp_dy(2) == -2, "V arms");
static_assert(acp_dx(6) == 3 && acp_dy(6) == -4, "near up ends at (3, -4)");
static_assert(acp_dx(15) == -2 && acp_dy(15) == -1, "near left (-2, -1)");
static_assert(acp_dx(28) == 0 && acp_dy(28) == -3 && acp_dy(38) == -23, "far up strip 3..23");
static_assert(acp_dx(71) == 23 && acp_dy(71) == 0, "far right ends at (23, 0)");
// every candidate lies on the other colour of the checkerboard (odd dx + dy)
__host__ __device__ constexpr bool acp_other_colour(int c = 0) {
  return c == 72 ? true : (((acp_dx(c) + acp_dy(c)) & 1) != 0 && acp_other_colour(c + 1));
}
static_assert(acp_other_colour(), "propagation candidates lie on the other colour");

// Reference window of one pixel (Sec. 3.3): 36 samples at offsets
// {-5,-3,-1,1,3,5}^2 clamped to the image; w = exp(-|I - I_c| / (2 sigma_I^2)
// - |dx| / (2 sigma_x^2)); the values centred on their weighted mean so that
// cov(r, s) = sum w r^ s / sum w.
// Stored as lane pairs (samples 2m, 2m + 1) for the packed moment updates.
struct RefWin {
  f2 w2[kWinS / 2];
  f2 wr2[kWinS / 2];
  float inv_sw, sum_wr, var_r;
};
static_assert(kWinS % 2 == 0 && kWinN % 2 == 0, "window samples are processed in pairs along a row");

// intensity of reference pixel i (uint8 or FP16 images)
template <bool kHalf, class A>
__device__ __forceinline__ float ref_at(const A& a, size_t i) {
  i = checked_index(a, i, (size_t)a.W * a.H, kBadReference);
  if (kHalf) return __half2float(__ldg(reinterpret_cast<const __half*>(a.ref) + i));
  return (float)__ldg(reinterpret_cast<const uint8_t*>(a.ref) + i);
}
// Source textures return intensity / 255 for uint8 images (normalised read)
// and the intensity itself for FP16 images.
template <bool kHalf>
__host__ __device__ constexpr float tex_scale() { return kHalf ? 1.f : 255.f; }

template <bool kHalf, class A>
__device__ __forceinline__ void load_ref_window(const A& a, int x, int y, RefWin& rw) {
  const float Ic = ref_at<kHalf, A>(a, (size_t)y * a.W + x);
  // w = exp(-e) relative to the largest weight: the statistics of Eq. (8) are
  // ratios of weighted sums, so the common factor cancels, and no weight
  // underflows (squared 8-bit differences reach e = 3600)
  float rv[kWinS], wv[kWinS];
  float emin = 3.4e38f;
#pragma unroll
  for (int k = 0; k < kWinS; k++) {
    const int du = -kWinR + kWinStride * (k % kWinN), dv = -kWinR + kWinStride * (k / kWinN);
    const int xr = min(max(x + du, 0), a.W - 1), yr = min(max(y + dv, 0), a.H - 1);
    const float r = ref_at<kHalf, A>(a, (size_t)yr * a.W + xr) - Ic;   // exact
    float dI = fabsf(r), dx = sqrtf((float)(du * du + dv * dv));
    if (a.squared) { dI = r * r; dx = (float)(du * du + dv * dv); }
    const float e = fmaf(dI, a.wI, dx * a.wX);
    rv[k] = r;
    wv[k] = e;
    emin = fminf(emin, e);
  }
  float sw = 0.f, s1 = 0.f;
#pragma unroll
  for (int k = 0; k < kWinS; k++) {
    const float w = expf(emin - wv[k]);
    wv[k] = w;
    sw += w;
    s1 = fmaf(w, rv[k], s1);
  }
  const float inv = 1.f / sw;
  const float mr = s1 * inv;
  float s2 = 0.f, swr = 0.f, wrv[kWinS];
#pragma unroll
  for (int k = 0; k < kWinS; k++) {
    const float rc = rv[k] - mr;
    const float wr = wv[k] * rc;
    wrv[k] = wr;
    swr += wr;
    s2 = fmaf(wr, rc, s2);
  }
#pragma unroll
  for (int m = 0; m < kWinS / 2; m++) {
    rw.w2[m] = pack2(wv[2 * m], wv[2 * m + 1]);
    rw.wr2[m] = pack2(wrv[2 * m], wrv[2 * m + 1]);
  }
  rw.inv_sw = inv;
  rw.sum_wr = swr;
  rw.var_r = s2 * inv - (swr * inv) * (swr * inv);
}

// ---------------------------------------------------------------------------
// Eq. (8): cost of the plane c = K^-T n / d against view V at pixel (x, y).
// 2 when the plane is unusable (ok false), lies behind view j over the window
// (homogeneous depth <= 0 at a window corner; it is affine over the window),
// projects the centre outside view j, or when a patch has no variance;
// otherwise clamped to [0, 2].  Window samples outside the view are clamped to
// its edge by the texture unit (or, in a shared-memory box, by the gathers
// that filled it).
// ---------------------------------------------------------------------------

// The homography of one (hypothesis, view) pair at one pixel: its linear part
// (output shifted by (+1, +1), see ViewConst), the window centre's image
// (px, py, pz) and (cx, cy), and the smallest homogeneous depth over the
// window.
struct PairGeom {
  float H0, H1, H3, H4, H6, H7;
  float px, py, pz, cx, cy, zmin;
};

// false: the pair costs 2 (behind the view over the window, or the centre
// outside the view).  c = (K_ref^-T n / d, 1 / D), ray = K_ref^-1 (x, y, 1).
__device__ __forceinline__ bool pair_geometry(const ViewConst& V, float4 c, float3 ray, PairGeom& G) {
  const float H0 = fmaf(-V.b[0], c.x, V.A[0]), H1 = fmaf(-V.b[0], c.y, V.A[1]);
  const float H3 = fmaf(-V.b[1], c.x, V.A[3]), H4 = fmaf(-V.b[1], c.y, V.A[4]);
  const float H6 = fmaf(-V.b[2], c.x, V.A[6]), H7 = fmaf(-V.b[2], c.y, V.A[7]);
  // H (x, y, 1) = P ray + b / D: the window centre's 3-D point projected
  const float pz = fmaf(V.P[6], ray.x, fmaf(V.P[7], ray.y, fmaf(V.P[8], ray.z, V.b[2] * c.w)));
  const float zmin = pz - (float)kWinR * (fabsf(H6) + fabsf(H7));
  if (!(zmin > 0.f)) return false;
  const float px = fmaf(V.P[0], ray.x, fmaf(V.P[1], ray.y, fmaf(V.P[2], ray.z, V.b[0] * c.w)));
  const float py = fmaf(V.P[3], ray.x, fmaf(V.P[4], ray.y, fmaf(V.P[5], ray.z, V.b[1] * c.w)));
  const float iz = rcp_approx(pz);
  const float cx = px * iz, cy = py * iz;
  if (!(cx >= 1.f && cx <= V.xmax && cy >= 1.f && cy <= V.ymax)) return false;
  G.H0 = H0; G.H1 = H1; G.H3 = H3; G.H4 = H4; G.H6 = H6; G.H7 = H7;
  G.px = px; G.py = py; G.pz = pz; G.cx = cx; G.cy = cy; G.zmin = zmin;
  return true;
}

// Where the 36 window samples fetch their 2 x 2 texels: the texture unit's
// gather (kFetchGather), its linear filter (kFetchFilter, the
// AMH_FLAG_TEXTURE_BILINEAR form), or a shared-memory box of bilinear cells
// built from the same gathers (kFetchBox).
constexpr int kFetchGather = 0, kFetchFilter = 1, kFetchBox = 2;

// Shared-memory sample box: kBoxW x kBoxH bilinear cells of one source view.
// Cell (c, r) covers the texels (ox + c .. ox + c + 1, oy + r .. oy + r + 1)
// and holds the coefficients of their bilinear interpolant,
// (a, b, c', d) = (T00, T10 - T00, T01 - T00, T11 - T01 - T10 + T00), so that
// a sample at fractions (fx, fy) inside the cell is a + fx b + fy (c' + fx d):
// one 16-byte load and three FMAs.
constexpr int kBoxW = 40, kBoxH = 40;
struct SampleBox {
  float4 q[kBoxH * kBoxW];
};
// Placement of one view's box for a block: its texel origin and the range
// the (shifted) sample positions must stay in, with a quarter-texel margin
// for rounding: floor(p) - 1 - ox in [0, kBoxW - 1], floor(p) - 1 - oy in
// [0, kBoxH - 1].
struct BoxPlace {
  int ox, oy;
  float bx0, bx1, by0, by1;
};
__device__ __forceinline__ BoxPlace make_place(int ox, int oy) {
  BoxPlace b;
  b.ox = ox;
  b.oy = oy;
  b.bx0 = (float)ox + 1.25f;
  b.bx1 = (float)(ox + kBoxW) + 0.75f;
  b.by0 = (float)oy + 1.25f;
  b.by1 = (float)(oy + kBoxH) + 0.75f;
  return b;
}
// Every sample of the window lies in the box: |x(u, v) - cx| <= 5 (|H0 - cx
// H6| + |H1 - cx H7|) / zmin over the window offsets u, v in [-5, 5] (the
// numerator of x - cx is linear in (u, v), the denominator at least zmin), and
// likewise for y.
__device__ __forceinline__ bool window_in_box(const PairGeom& G, const BoxPlace& b) {
  const float izm = rcp_approx(G.zmin);
  const float R = (float)kWinR;
  const float ex = R * (fabsf(fmaf(-G.cx, G.H6, G.H0)) + fabsf(fmaf(-G.cx, G.H7, G.H1))) * izm;
  const float ey = R * (fabsf(fmaf(-G.cy, G.H6, G.H3)) + fabsf(fmaf(-G.cy, G.H7, G.H4))) * izm;
  return G.cx - ex >= b.bx0 && G.cx + ex <= b.bx1 && G.cy - ey >= b.by0 && G.cy + ey <= b.by1;
}
// floor of both lanes (as floor2) and the integer parts as the bits of
// x + 2^23 rounded towards -inf: 0x4B000000 + floor(x) for 0 <= x < 2^23
__device__ __forceinline__ f2 floor2_bits(f2 x, uint32_t& bx, uint32_t& by) {
  const f2 M = pack2(8388608.f, 8388608.f);
  f2 t;
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(t.v) : "l"(x.v), "l"(M.v));
  float tx, ty;
  unpack2(t, tx, ty);
  bx = __float_as_uint(tx);
  by = __float_as_uint(ty);
  return sub2(t, M);
}

// The 36 samples of one pair and the NCC of Eq. (8).  kFetchBox: box_cells
// is the box's cell array and box_adj its box_adjust(), so that the cell of
// a sample whose floored positions have the bits (bx, by) is
// by kBoxW + bx - box_adj.
template <bool kHalf, int kFetch>
__device__ __forceinline__ float ncc_window(const ViewConst& V, const PairGeom& G, const RefWin& rw,
                                            const void* box_cells = nullptr, uint32_t box_adj = 0u) {
  const float H0 = G.H0, H1 = G.H1, H3 = G.H3, H4 = G.H4, H6 = G.H6, H7 = G.H7;
  const float px = G.px, py = G.py, pz = G.pz;
  const float R = (float)kWinR, St = (float)kWinStride;
  const float sx0 = fmaf(-R, H0 + H1, px), sy0 = fmaf(-R, H3 + H4, py), sz0 = fmaf(-R, H6 + H7, pz);
  const float cxs = St * H0, cys = St * H3, czs = St * H6;
  const float rxs = St * H1, rys = St * H4, rzs = St * H7;
  // Packed f32x2 arithmetic: the (x, y) position, floor and fraction of each
  // sample form one lane pair (the gather takes them as a pair), the depths
  // and the three moments of samples (cb, cb + 1) of a row another; the
  // fetches and the bilinear blends are per sample.
  const float4* box = reinterpret_cast<const float4*>(box_cells);
  if (kFetch == kFetchBox) __builtin_assume(__isShared(box) != 0);
  const f2 cxy = pack2(cxs, cys), cz2 = pack2(czs, czs);
  f2 acc1 = pack2(0.f, 0.f), acc2 = pack2(0.f, 0.f), accr = pack2(0.f, 0.f);
  f2 s0p = pack2(0.f, 0.f);
#pragma unroll
  for (int ra = 0; ra < kWinN; ra++) {
    const float bx = fmaf((float)ra, rxs, sx0), by = fmaf((float)ra, rys, sy0), bz = fmaf((float)ra, rzs, sz0);
    const f2 bxy = pack2(bx, by), bz2 = pack2(bz, bz);
#pragma unroll
    for (int cb = 0; cb < kWinN; cb += 2) {
      const int m = (ra * kWinN + cb) / 2;
      // (x, y) of each sample in one lane pair (the gather takes them as a pair)
      const f2 qa = fma2(pack2((float)cb, (float)cb), cxy, bxy);
      const f2 qb = fma2(pack2((float)(cb + 1), (float)(cb + 1)), cxy, bxy);
      const f2 qz = fma2(pack2((float)cb, (float)(cb + 1)), cz2, bz2);
      float qz0, qz1, qxa, qya, qxb, qyb;
      unpack2(qz, qz0, qz1);
      unpack2(qa, qxa, qya);
      unpack2(qb, qxb, qyb);
      const float ia = rcp_approx(qz0), ib = rcp_approx(qz1);
      const f2 pa = pack2(qxa * ia, qya * ia), pb = pack2(qxb * ib, qyb * ib);
      f2 sp;
      if (kFetch == kFetchFilter) {
        // the texture unit's linear filter (AMH_FLAG_TEXTURE_BILINEAR): its
        // texel centres sit at +0.5, the positions here at +1
        const f2 ha = sub2(pa, pack2(0.5f, 0.5f)), hb = sub2(pb, pack2(0.5f, 0.5f));
        float hxa, hya, hxb, hyb;
        unpack2(ha, hxa, hya);
        unpack2(hb, hxb, hyb);
        sp = pack2(tex2D<float>(V.tex, hxa, hya), tex2D<float>(V.tex, hxb, hyb));
      } else if (kFetch == kFetchBox) {
        // cell index (floor(p) - 1 - o) from the bits of the floored
        // positions; box_adj folds in the origin and the 2^23 offsets
        uint32_t bxa, bya, bxb, byb;
        const f2 fla = floor2_bits(pa, bxa, bya), flb = floor2_bits(pb, bxb, byb);
        const f2 fra = sub2(pa, fla), frb = sub2(pb, flb);
        const float4 ca = box[bya * (uint32_t)kBoxW + bxa - box_adj];
        const float4 cb4 = box[byb * (uint32_t)kBoxW + bxb - box_adj];
        float fxa, fya, fxb, fyb;
        unpack2(fra, fxa, fya);
        unpack2(frb, fxb, fyb);
        sp = pack2(fmaf(fya, fmaf(fxa, ca.w, ca.z), fmaf(fxa, ca.y, ca.x)),
                   fmaf(fyb, fmaf(fxb, cb4.w, cb4.z), fmaf(fxb, cb4.y, cb4.x)));
      } else {
        const f2 fla = floor2(pa), flb = floor2(pb);
        const f2 fra = sub2(pa, fla), frb = sub2(pb, flb);
        float x0a, x0b, y0a, y0b, fxa, fxb, fya, fyb;
        unpack2(fla, x0a, y0a);
        unpack2(flb, x0b, y0b);
        unpack2(fra, fxa, fya);
        unpack2(frb, fxb, fyb);
        // texels: w (x0, y0), z (x0+1, y0), x (x0, y0+1), y (x0+1, y0+1)
        const float4 ga = tex2Dgather<float4>(V.tex, x0a, y0a, 0);
        const float4 gb = tex2Dgather<float4>(V.tex, x0b, y0b, 0);
        const float ta = fmaf(fxa, ga.z - ga.w, ga.w), ba = fmaf(fxa, ga.y - ga.x, ga.x);
        const float tb = fmaf(fxb, gb.z - gb.w, gb.w), bb = fmaf(fxb, gb.y - gb.x, gb.x);
        sp = pack2(fmaf(fya, ba - ta, ta), fmaf(fyb, bb - tb, tb));
      }
      // moments about the first sample: exact zero variance for constant
      // patches in FP32
      if (m == 0) {
        float s0, s1_;
        unpack2(sp, s0, s1_);
        s0p = pack2(s0, s0);
      }
      const f2 sc = sub2(sp, s0p);
      const f2 ws = mul2(rw.w2[m], sc);
      acc1 = add2(acc1, ws);
      acc2 = fma2(ws, sc, acc2);
      accr = fma2(rw.wr2[m], sc, accr);
    }
  }
  float m1a, m1b, m2a, m2b, mra, mrb;
  unpack2(acc1, m1a, m1b);
  unpack2(acc2, m2a, m2b);
  unpack2(accr, mra, mrb);
  const float m1 = m1a + m1b, m2 = m2a + m2b, mrs = mra + mrb;
  const float es = m1 * rw.inv_sw;
  const float var_s = fmaf(m2, rw.inv_sw, -es * es);
  const float cov = fmaf(mrs, rw.inv_sw, -(rw.sum_wr * rw.inv_sw) * es);
  // variances in squared intensity units (the threshold is 1e-10 there)
  constexpr float S = tex_scale<kHalf>();
  const float vv = rw.var_r * var_s * (S * S);
  if (!(vv >= 1e-10f)) return kWorst;
  return fminf(fmaxf(1.f - cov * (S * rsqrtf(vv)), 0.f), 2.f);
}

template <bool kHalf, bool kTex = false>
__device__ __forceinline__ float ncc_cost(const ViewConst& V, float4 c, bool ok, float3 ray,
                                          const RefWin& rw, int* evaluated) {
  if (!ok) return kWorst;
  PairGeom G;
  if (!pair_geometry(V, c, ray, G)) return kWorst;
  *evaluated += 1;
  return ncc_window<kHalf, kTex ? kFetchFilter : kFetchGather>(V, G, rw);
}

// The same cost inside the staged matrix sweep, where the whole warp calls
// it together: when every lane that evaluates the pair has its window inside
// the block's box of this view, the warp samples the box, otherwise the
// texture unit (the two interpolate the same texels in FP32, in a different
// order of operations).
template <bool kHalf>
__device__ __forceinline__ float ncc_cost_boxed(const ViewConst& V, float4 c, bool ok, float3 ray,
                                                const RefWin& rw, int* evaluated, const BoxPlace& bp,
                                                const SampleBox& box, uint32_t box_adj) {
  PairGeom G;
  const bool act = ok && pair_geometry(V, c, ray, G);
  const bool fits = act && window_in_box(G, bp);
  const bool all_fit = __all_sync(0xffffffffu, fits || !act);
  float m = kWorst;
  if (act) {
    *evaluated += all_fit ? 0x10001 : 1;      // the high half counts box-sampled evaluations
    m = all_fit ? ncc_window<kHalf, kFetchBox>(V, G, rw, box.q, box_adj) : ncc_window<kHalf, kFetchGather>(V, G, rw);
  }
  return m;
}

// ---------------------------------------------------------------------------
// Staged matrix sweep: per block and source view, one shared-memory box of
// texel pairs around where the block's pixels' own planes put their windows;
// every warp whose windows of a (hypothesis, view) pair all lie in it samples
// the box instead of the texture unit.
// ---------------------------------------------------------------------------
constexpr int kStageWarps = 8;          // blocks of up to 256 threads
constexpr int kStageLane = 12;          // the lane whose own plane places its warp's candidate
struct StageShared {
  SampleBox box;
  BoxPlace place[kMaxSrc];
  float2 wcen[kStageWarps][kMaxSrc];    // per warp and view: window centre of lane kStageLane, NaN if none
};

// Box origins of every view for this block (block-wide; ends synchronised):
// each warp proposes the window centre its lane kStageLane's own plane
// projects to; the box is centred on the median of the proposals.
template <class A>
__device__ __forceinline__ void place_boxes(const A& a, StageShared& ss, float4 c_own, bool own_ok, float3 ray) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == kStageLane) {
    for (int j = 0; j < a.N; j++) {
      PairGeom G;
      const bool ok = own_ok && pair_geometry(a.v[j], c_own, ray, G);
      ss.wcen[warp][j] = ok ? make_float2(G.cx, G.cy) : make_float2(__int_as_float(0x7fc00000), 0.f);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < a.N; j += blockDim.x) {
    float xs[kStageWarps], ys[kStageWarps];
    int n = 0;
    for (int w = 0; w < nw; w++) {
      const float2 m = ss.wcen[w][j];
      if (m.x == m.x) {                     // insertion into the sorted lists
        int i = n++;
        while (i > 0 && xs[i - 1] > m.x) { xs[i] = xs[i - 1]; i--; }
        xs[i] = m.x;
        i = n - 1;
        while (i > 0 && ys[i - 1] > m.y) { ys[i] = ys[i - 1]; i--; }
        ys[i] = m.y;
      }
    }
    int ox = -1, oy = -1;
    if (n > 0) {
      // (shifted) centre c sits on real texel c - 1 at the middle of the box
      const float cx = 0.5f * (xs[(n - 1) >> 1] + xs[n >> 1]), cy = 0.5f * (ys[(n - 1) >> 1] + ys[n >> 1]);
      ox = max(-1, (int)floorf(cx - 1.f - 0.5f * (float)(kBoxW - 1)));
      oy = max(-1, (int)floorf(cy - 1.f - 0.5f * (float)(kBoxH - 1)));
    }
    ss.place[j] = make_place(ox, oy);
  }
  __syncthreads();
}

// The box of view V at bp: one gather per cell (its four texels; the texture
// unit clamps coordinates outside the view, exactly as for the samples it
// serves directly), turned into the cell's coefficients.
__device__ __forceinline__ void fill_box(const ViewConst& V, SampleBox& B, const BoxPlace& bp) {
  for (int i = threadIdx.x; i < kBoxH * kBoxW; i += blockDim.x) {
    const int r = i / kBoxW, cc = i - r * kBoxW;
    const float4 g = tex2Dgather<float4>(V.tex, (float)(bp.ox + cc + 1), (float)(bp.oy + r + 1), 0);
    const float b = g.z - g.w;
    B.q[i] = make_float4(g.w, b, g.x - g.w, (g.y - g.x) - b);
  }
}

// Cell index of the sample whose floored positions have the bits (bx, by):
// by kBoxW + bx - box_adjust(bp)  (mod 2^32)
__device__ __forceinline__ uint32_t box_adjust(const BoxPlace& bp) {
  const uint32_t K = 0x4B000000u;
  return (K + 1u + (uint32_t)bp.oy) * (uint32_t)kBoxW + K + 1u + (uint32_t)bp.ox;
}

// Refinement candidate idx (Sec. 3.3): rho_t = 2^-(t+1); 0: depth and normal
// perturbed (bisection); from t = 3 on also 1: (random D, n), 2: (D, random
// n), 3: (random D, random n), 4: (perturbed D, n), 5: (D, perturbed n).
// Draws (pixel, t, 0, 1) and (pixel, t, 1, 1).
template <class A>
__device__ __forceinline__ float4 refine_candidate(const A& a, int x, int y, float4 pl, float3 ray,
                                                   int idx) {
  const uint32_t pix = (uint32_t)(y * a.W + x);
  const float rho = ldexpf(1.f, -(a.t + 1));
  float Dp = pl.w;
  float3 np = make_float3(pl.x, pl.y, pl.z);
  if (idx == 0 || idx == 4 || idx == 5) {
    const uint4 r0 = philox4x32_10(make_uint4(pix, (uint32_t)a.t, 0u, 1u), a.key0, a.key1);
    Dp = pl.w * (1.f + rho * (2.f * u01(r0.x) - 1.f));
    np = make_float3(pl.x + rho * (2.f * u01(r0.y) - 1.f), pl.y + rho * (2.f * u01(r0.z) - 1.f),
                     pl.z + rho * (2.f * u01(r0.w) - 1.f));
    const float inn = 1.f / sqrtf(dot3(np, np));
    np = face_camera(make_float3(np.x * inn, np.y * inn, np.z * inn), ray);
  }
  float Dr = pl.w;
  float3 nr = make_float3(pl.x, pl.y, pl.z);
  if (idx >= 1 && idx <= 3) {
    const uint4 r1 = philox4x32_10(make_uint4(pix, (uint32_t)a.t, 1u, 1u), a.key0, a.key1);
    Dr = a.dmin + (a.dmax - a.dmin) * u01(r1.x);
    nr = face_camera(normal_from_uniforms(u01(r1.y), u01(r1.z)), ray);
  }
  switch (idx) {
    case 0: return make_float4(np.x, np.y, np.z, Dp);
    case 1: return make_float4(pl.x, pl.y, pl.z, Dr);
    case 2: return make_float4(nr.x, nr.y, nr.z, pl.w);
    case 3: return make_float4(nr.x, nr.y, nr.z, Dr);
    case 4: return make_float4(pl.x, pl.y, pl.z, Dp);
    default: return make_float4(np.x, np.y, np.z, pl.w);
  }
}

// Per-pixel working arrays of one thread (local memory, cached in L1): the
// 8 x N cost matrix of Eq. (1), the N view weights and the 8 propagated planes
// as (c = K^-T n / d, 1 / D).  Shared memory stays unused so that L1 serves the texture
// gathers.
struct PixelArrays {
  float M[kRegions * kMaxSrc];
  float w[kMaxSrc];
  float4 C[kRegions];
  __device__ float& m(int g, int j, int) { return M[g * kMaxSrc + j]; }
  __device__ float& wt(int j) { return w[j]; }
  __device__ float4& cc(int g) { return C[g]; }
};

// Eqs. (2)-(6): weights of the N views from the 8 x N matrix (rows of invalid
// regions are left out of the counts and of the mean of Eq. (4)).
template <class A>
__device__ __forceinline__ void joint_view_selection(const A& a, PixelArrays& sm, uint32_t valid,
                                                     uint32_t S_prev, int v_prev, uint32_t* S_out, int* v_out) {
  const int N = a.N;
  const int nvalid = __popc(valid);
  const int k = a.k < N ? a.k : N;
  uint32_t S = 0;
  for (int j = 0; j < N; j++) {         // psi_mod of the good views into w
    int ng = 0, nb = 0;
    float psi = 0.f;
#pragma unroll
    for (int i = 0; i < kRegions; i++) {
      if (!(valid >> i & 1u)) continue;
      const float m = sm.m(i, j, N);
      ng += m < a.tau;
      nb += m > a.tau_up;
      psi += expf(-m * m * a.inv2beta2);          // Eq. (3)
    }
    float pm = 0.f;
    if (ng > a.n1 && nb < a.n2) {                  // good view
      S |= 1u << j;
      psi = psi / (float)nvalid;                   // Eq. (4)
      pm = (j == v_prev) ? 2.f * psi : psi;        // Eqs. (5), (6)
    }
    sm.wt(j) = pm;
  }
  uint32_t kept = 0;
  int v = -1;
  for (int j = 0; j < N; j++) {
    if (!(S >> j & 1u)) continue;
    const float pj = sm.wt(j);
    int rank = 0;
    for (int q = 0; q < N; q++) {
      const float pq = sm.wt(q);
      rank += (S >> q & 1u) && (pq > pj || (pq == pj && q < j));
    }
    if (rank < k) kept |= 1u << j;                 // at most k views keep weight
    if (rank == 0) v = j;
  }
  bool any = false;
  for (int j = 0; j < N; j++) {
    float wj;
    if (S >> j & 1u) wj = (kept >> j & 1u) ? sm.wt(j) : 0.f;
    else wj = (S_prev >> j & 1u) ? 0.2f : 0.f;   // selected at t - 1, not at t
    sm.wt(j) = wj;
    any = any || wj > 0.f;
  }
  if (!any) {  // no weight at all: the k views of smallest mean cost get 1
    for (int j = 0; j < N; j++) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < kRegions; i++)
        if (valid >> i & 1u) s += sm.m(i, j, N);
      sm.wt(j) = nvalid ? s / (float)nvalid : 0.f;
    }
    uint32_t low = 0;
    for (int j = 0; j < N; j++) {
      const float cj = sm.wt(j);
      int rank = 0;
      for (int q = 0; q < N; q++) {
        const float cq = sm.wt(q);
        rank += cq < cj || (cq == cj && q < j);
      }
      if (rank < k) low |= 1u << j;
    }
    for (int j = 0; j < N; j++) sm.wt(j) = (low >> j & 1u) ? 1.f : 0.f;
  }
  *S_out = S;
  *v_out = v;
}


// mean of the k smallest of m[0..N), summed in ascending order (ties: lower
// index) -- the heuristic view selection of Sec. 2
__device__ __forceinline__ float kbest_mean(const float* m, int N, int k) {
  uint32_t used = 0;
  float acc = 0.f;
  for (int r = 0; r < k; r++) {
    int bj = -1;
    float bmv = 0.f;
    for (int j = 0; j < N; j++) {
      const float mj = m[j];
      if (!(used >> j & 1u) && (bj < 0 || mj < bmv)) { bj = j; bmv = mj; }
    }
    used |= 1u << bj;
    acc += bmv;
  }
  return acc / (float)k;
}

// Ablations of Sec. 4 (template bits of update_pixel): kSymmetric -- each of
// the 8 regions is one fixed candidate, the axis neighbour at distance 1
// (regions 0-3) or 5 (regions 4-7) up, down, left, right, instead of the
// lowest-cost pick of ACP; kHeuristic -- every hypothesis (rows, own plane,
// refinement candidates) is scored by the mean of its own k smallest
// per-view costs instead of MHJ, and no S_t / v_t is kept.
constexpr int kSymmetric = 1, kHeuristic = 2;
// kTexture: window samples through the texture unit's linear filter
// (AMH_FLAG_TEXTURE_BILINEAR) instead of gathers and FP32 blends.
constexpr int kTexture = 4;
// kStage: the 8 x N matrix sweep stages shared-memory sample boxes (the whole
// block calls update_pixel together, pixels outside the image included)
constexpr int kStage = 8;

// ---------------------------------------------------------------------------
// one pixel's checkerboard update
// ---------------------------------------------------------------------------
template <bool kHalf, int kMode = 0, class A>
__device__ __forceinline__ void update_pixel(const A& a, PixelArrays& sm, int x, int y,
                                             int* npairs, StageShared* ss = nullptr, bool live = true) {
  constexpr bool kTex = (kMode & kTexture) != 0;
  constexpr bool kStaged = (kMode & kStage) != 0;
  static_assert(!(kStaged && kTex), "the staged sweep gathers; the texture-filter form does not stage");
  const int N = a.N;
  // the pixel's state index (32-bit: a state holds fewer than 2^31 entries)
  const int pi = live ? (int)checked_index(a, (size_t)(y * (2 * ((a.W + 1) >> 1)) + (((x + y) & 1) ? (a.W + 1) >> 1 : 0) +
                                                       (x >> 1)),
                                           state_size(a.W, a.H), kBadPixel)
                      : 0;
  const float fx = (float)x, fy = (float)y;
  const float3 ray = ref_ray(a.Kinv, fx, fy);

  // --- Sec. 3.1: asymmetric checkerboard propagation ---------------------------
  // pick[g]: pixel offset of region g's candidate from (x, y), packed as
  // (dx + 32) | (dy + 32) << 8 (-1: none).  Every candidate offset has odd
  // dx + dy, so every candidate lies on the other colour: its state index is
  // the pixel's base, y S + (the other colour's run) + x / 2, plus
  // dy S + ((x mod 2) + dx) / 2 (S = entries per state row).
  const int srow = 2 * ((a.W + 1) >> 1), xodd = x & 1;
  const int qbase = y * srow + (((x + y) & 1) ? 0 : (srow >> 1)) + (x >> 1);
  auto pick_index = [&](int off) {
    return checked_index(a, state_index(x + (off & 255) - 32, y + (off >> 8) - 32, a.W), state_size(a.W, a.H),
                         kBadNeighbour);
  };
  int pick[kRegions];
#pragma unroll
  for (int g = 0; g < kRegions; g++) pick[g] = -1;
  if (live) {
#pragma unroll
  for (int g = 0; g < kRegions; g++) {
    int best = -1;
    if (kMode & kSymmetric) {
      const int dist = g < 4 ? 1 : 5, dir = g & 3;
      const int dx = dir == 2 ? -dist : dir == 3 ? dist : 0, dy = dir == 0 ? -dist : dir == 1 ? dist : 0;
      const int qx = x + dx, qy = y + dy;
      if (qx >= 0 && qy >= 0 && qx < a.W && qy < a.H) best = (dx + 32) | (dy + 32) << 8;
    } else {
      float bc = 0.f;
#pragma unroll
      for (int c = acp_start(g); c < acp_start(g + 1); c++) {
        const int qx = x + acp_dx(c), qy = y + acp_dy(c);
        if (qx < 0 || qy < 0 || qx >= a.W || qy >= a.H) continue;
        const int q = (int)checked_index(a, (size_t)(qbase + acp_dy(c) * srow + ((xodd + acp_dx(c)) >> 1)),
                                         state_size(a.W, a.H), kBadNeighbour);
        const float cq = __ldg(&a.cost[q]);
        if (best < 0 || cq < bc) { best = (acp_dx(c) + 32) | (acp_dy(c) + 32) << 8; bc = cq; }
      }
    }
    pick[g] = best;
  }
  }
  float hD[kRegions];
  uint32_t valid = 0;
#pragma unroll
  for (int g = 0; g < kRegions; g++) {
    hD[g] = 0.f;
    if (pick[g] < 0) continue;
    const float4 pq = a.plane[pick_index(pick[g])];
    const float3 nq = make_float3(pq.x, pq.y, pq.z);
    const int qx = x + (pick[g] & 255) - 32, qy = y + (pick[g] >> 8) - 32;
    const float3 rq = ref_ray(a.Kinv, (float)qx, (float)qy);
    const float d = -pq.w * dot3(nq, rq);          // plane offset, the same at q and x
    const float den = dot3(nq, ray);
    if (!(den < 0.f)) continue;
    const float Dx = -d / den;
    if (!(Dx > 0.f) || !isfinite(Dx)) continue;
    float4 c;
    if (!plane_c(a.Kinv, make_float4(nq.x, nq.y, nq.z, Dx), ray, &c)) continue;
    sm.cc(g) = c;
    hD[g] = Dx;
    valid |= 1u << g;
  }

  RefWin rw;
  if (live) load_ref_window<kHalf>(a, x, y, rw);

  // --- Eq. (1): the 8 x N cost matrix (views outer: the 8 hypotheses of a view
  // fetch neighbouring texels) -------------------------------------------------------
  if constexpr (kStaged) {
    // one shared-memory box per view for the whole block, placed where a few
    // of the pixels' own planes put their windows
    float4 c_own = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool own_ok = live && plane_c(a.Kinv, a.plane[pi], ray, &c_own);
    place_boxes(a, *ss, c_own, own_ok, ray);
    for (int j = 0; j < N; j++) {
      const ViewConst& V = a.v[j];
      const BoxPlace bp = ss->place[j];
      __syncthreads();                      // the previous view's box is no longer read
      fill_box(V, ss->box, bp);
      __syncthreads();
      const uint32_t adj = box_adjust(bp);
#pragma unroll 1
      for (int g = 0; g < kRegions; g++) {
        const bool ok = valid >> g & 1u;
        const float4 c = ok ? sm.cc(g) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float m = ncc_cost_boxed<kHalf>(V, c, ok, ray, rw, npairs, bp, ss->box, adj);
        if (live) sm.m(g, j, N) = m;
      }
    }
    if (!live) return;
  } else {
    for (int j = 0; j < N; j++) {
      const ViewConst& V = a.v[j];
#pragma unroll 1
      for (int g = 0; g < kRegions; g++) {
        const bool ok = valid >> g & 1u;
        const float4 c = ok ? sm.cc(g) : make_float4(0.f, 0.f, 0.f, 0.f);
        sm.m(g, j, N) = ncc_cost<kHalf, kTex>(V, c, ok, ray, rw, npairs);
      }
    }
  }

  if (kMode & kHeuristic) {
    const int k = a.k < N ? a.k : N;
    float4 best = a.plane[pi];
    float4 c;
    bool ok = plane_c(a.Kinv, best, ray, &c);
    for (int j = 0; j < N; j++) sm.wt(j) = ncc_cost<kHalf, kTex>(a.v[j], c, ok, ray, rw, npairs);
    float bm = kbest_mean(sm.w, N, k);
    int choice = 8;
    float bestD = 0.f;
#pragma unroll 1
    for (int g = 0; g < kRegions; g++) {
      if (!(valid >> g & 1u)) continue;
      const float r = kbest_mean(&sm.M[g * kMaxSrc], N, k);
      if (r < bm) { bm = r; choice = g; }
    }
    if (choice < 8) {
#pragma unroll
      for (int g = 0; g < kRegions; g++) if (g == choice) bestD = hD[g];
      const float4 pq = a.plane[pick_index(pick[choice])];
      best = make_float4(pq.x, pq.y, pq.z, bestD);
    }
    const int nc = a.t < 3 ? 1 : kMaxRefine;
    int bc = -1;
    float bcm = 0.f;
#pragma unroll 1
    for (int ci = 0; ci < nc; ci++) {
      ok = plane_c(a.Kinv, refine_candidate(a, x, y, best, ray, ci), ray, &c);
      for (int j = 0; j < N; j++) sm.wt(j) = ncc_cost<kHalf, kTex>(a.v[j], c, ok, ray, rw, npairs);
      const float m = kbest_mean(sm.w, N, k);
      if (bc < 0 || m < bcm) { bc = ci; bcm = m; }
    }
    if (bc >= 0 && bcm < bm) {
      bm = bcm;
      best = refine_candidate(a, x, y, best, ray, bc);
      choice = 9 + bc;
    }
    a.plane[pi] = best;
    a.cost[pi] = bm;
    a.sel[pi] = 0;
    a.vbest[pi] = 255;
    a.wmask[pi] = 0;
    a.choice[pi] = (uint8_t)choice;
    return;
  }

  // --- Eqs. (2)-(6) ------------------------------------------------------------------
  uint32_t St;
  int v;
  const uint8_t vb = a.vbest[pi];
  joint_view_selection(a, sm, valid, a.sel[pi], vb == 255 ? -1 : (int)vb, &St, &v);
  float sw = 0.f;
  uint32_t wm = 0;
  for (int j = 0; j < N; j++) {
    const float wj = sm.wt(j);
    sw += wj;
    wm |= (wj > 0.f ? 1u : 0u) << j;
  }
  const float inv_sw = 1.f / sw;

  // --- Eq. (7): unified cost; the own plane competes and wins ties -------------------
  float4 best = a.plane[pi];
  float4 c;
  bool ok = plane_c(a.Kinv, best, ray, &c);
  float bm = 0.f;
  for (int j = 0; j < N; j++) {   // views with weight 0 are skipped (per-lane predicate)
    const float wj = sm.wt(j);
    if (wj > 0.f) bm = fmaf(wj, ncc_cost<kHalf, kTex>(a.v[j], c, ok, ray, rw, npairs), bm);
  }
  bm *= inv_sw;
  int choice = 8;
  float bestD = 0.f;
#pragma unroll 1
  for (int g = 0; g < kRegions; g++) {
    if (!(valid >> g & 1u)) continue;
    float r = 0.f;
    for (int j = 0; j < N; j++) {
      const float wj = sm.wt(j);
      if (wj > 0.f) r = fmaf(wj, sm.m(g, j, N), r);
    }
    r *= inv_sw;
    if (r < bm) { bm = r; choice = g; }
  }
  if (choice < 8) {
#pragma unroll
    for (int g = 0; g < kRegions; g++) if (g == choice) bestD = hD[g];
    const float4 pq = a.plane[pick_index(pick[choice])];
    best = make_float4(pq.x, pq.y, pq.z, bestD);
  }

  // --- Sec. 3.3: refinement with the same weights -------------------------------------
  // A learned proposal (n, d) of this pixel's 2 x 2 block, when present, is one
  // more candidate after the refinement ones, scored with the same weights.
  const int nc = a.t < 3 ? 1 : kMaxRefine;
  float4 prop = make_float4(0.f, 0.f, 0.f, 0.f);
  bool has_prop = false;
  if (a.prop) {
    const float4 pr = a.prop[checked_index(a, (size_t)min(y / 2, a.prop_h - 1) * a.prop_w + min(x / 2, a.prop_w - 1),
                                           (size_t)a.prop_w * a.prop_h, kBadProposal)];
    const float den = pr.x * ray.x + pr.y * ray.y + pr.z * ray.z;
    const float Dx = den < 0.f ? -pr.w / den : 0.f;
    has_prop = pr.w > 0.f && Dx > 0.f && isfinite(Dx);
    prop = make_float4(pr.x, pr.y, pr.z, Dx);
  }
  const int ncand = nc + (has_prop ? 1 : 0);
  // The outcome is the candidate of least cost strictly below the current
  // best (ties: the lower index).  The candidates are scored view by view:
  // for each view (warp-uniform: one texture per gather) a lane runs only its
  // own live candidates, so the warp pays for its busiest lane rather than
  // for every candidate some lane still needs.  A candidate's weighted sum
  // runs over the views in the same order as alone and only grows (w_j >= 0,
  // m_j >= 0, rounding is monotone), so one that reaches the current best
  // has lost and is dropped: every sum that is kept, and so the outcome, is
  // exactly that of scoring each candidate in full.  The candidates' planes
  // take the propagated rows' slots and their sums the first matrix row,
  // both no longer read.
  uint32_t okm = 0u;
#pragma unroll 1
  for (int ci = 0; ci < ncand; ci++) {
    float4 cc;
    if (plane_c(a.Kinv, ci < nc ? refine_candidate(a, x, y, best, ray, ci) : prop, ray, &cc)) okm |= 1u << ci;
    sm.cc(ci) = cc;
    sm.m(0, ci, N) = 0.f;
  }
  uint32_t cand_live = (1u << ncand) - 1u;
#pragma unroll 1
  for (int j = 0; j < N; j++) {
    const float wj = sm.wt(j);
    uint32_t todo = wj > 0.f ? cand_live : 0u;
    while (todo) {
      const int ci = __ffs(todo) - 1;
      todo &= todo - 1u;
      const float m = fmaf(wj, ncc_cost<kHalf, kTex>(a.v[j], sm.cc(ci), (okm >> ci) & 1u, ray, rw, npairs),
                           sm.m(0, ci, N));
      sm.m(0, ci, N) = m;
      if (!(m * inv_sw < bm)) cand_live &= ~(1u << ci);
    }
  }
  int bc = -1;
  float bcm = 0.f;
  for (int ci = 0; ci < ncand; ci++) {
    if (!(cand_live >> ci & 1u)) continue;
    const float m = sm.m(0, ci, N) * inv_sw;
    if (bc < 0 || m < bcm) { bc = ci; bcm = m; }
  }
  if (bc >= 0 && bcm < bm) {
    bm = bcm;
    best = bc < nc ? refine_candidate(a, x, y, best, ray, bc) : prop;
    choice = bc < nc ? 9 + bc : 15;
  }
  // the pixel's new state: streaming stores, nothing reads it again in this
  // phase
  __stcs(&a.plane[pi], best);
  __stcs(&a.cost[pi], bm);
  __stcs(&a.sel[pi], St);
  __stcs(&a.vbest[pi], v < 0 ? (uint8_t)255 : (uint8_t)v);
  __stcs(&a.wmask[pi], wm);
  __stcs(&a.choice[pi], (uint8_t)choice);
}

// Random initialisation of one pixel (Sec. 2, Gipuma-style random planes):
// depth uniform in [d_min, d_max], normal uniform on the sphere flipped to
// face the camera, draws (pixel, 0, 0, 0); the initial cost is the mean of the
// k smallest per-view costs, summed in ascending order (ties: lower view).
template <bool kHalf, bool kTex, class A>
__device__ __forceinline__ void init_pixel(const A& a, PixelArrays& sm, int x, int y, int* npairs) {
  const int N = a.N;
  const size_t pi = checked_index(a, state_index(x, y, a.W), state_size(a.W, a.H), kBadPixel);
  const float fx = (float)x, fy = (float)y;
  const float3 ray = ref_ray(a.Kinv, fx, fy);
  const uint4 r = philox4x32_10(make_uint4((uint32_t)(y * a.W + x), 0u, 0u, 0u), a.key0, a.key1);
  const float3 n = face_camera(normal_from_uniforms(u01(r.y), u01(r.z)), ray);
  const float4 pl = make_float4(n.x, n.y, n.z, a.dmin + (a.dmax - a.dmin) * u01(r.x));
  float4 c;
  const bool ok = plane_c(a.Kinv, pl, ray, &c);
  RefWin rw;
  load_ref_window<kHalf>(a, x, y, rw);
  for (int j = 0; j < N; j++) sm.wt(j) = ncc_cost<kHalf, kTex>(a.v[j], c, ok, ray, rw, npairs);
  // mean of the k smallest per-view costs, summed in ascending order (ties:
  // lower view index)
  const int k = a.k < N ? a.k : N;
  uint32_t used = 0;
  float acc = 0.f;
  for (int r2 = 0; r2 < k; r2++) {
    int bj = -1;
    float bmv = 0.f;
    for (int j = 0; j < N; j++) {
      const float mj = sm.wt(j);
      if (!(used >> j & 1u) && (bj < 0 || mj < bmv)) { bj = j; bmv = mj; }
    }
    used |= 1u << bj;
    acc += bmv;
  }
  a.plane[pi] = pl;
  a.cost[pi] = acc / (float)k;
  a.sel[pi] = 0;
  a.vbest[pi] = 255;
  a.wmask[pi] = 0;
  a.choice[pi] = 8;
}

}  // namespace upd
}  // namespace amh
