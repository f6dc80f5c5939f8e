// amh_api.cu -- the C-ABI of include/amh.h and the kernels of the
// checkerboard update: random initialisation, one colour phase (ACP + cost
// matrix + joint view selection + weighted choice + refinement) and the map
// read-back.  All method arithmetic runs in the kernels below; the host code
// validates arguments, converts the cameras once (in FP64) and launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "amh.h"
#include "amh_device.cuh"
#include "amh_ctx.h"

using namespace amh;

// ===========================================================================
// Sec. 3.1: the eight ACP regions.  Near V-shaped regions (7 candidates): the
// axis pixel at distance 1 and the pairs at lateral offset +-a, distance a+1;
// far strips (11 candidates): the axis pixels at distances 3, 5, ..., 23.
// Scan order nearest first, negative lateral side first; every offset has odd
// |dx| + |dy| (opposite checkerboard colour).
// ===========================================================================
namespace {
// candidate c of the 72: regions 0..3 hold 7 each, regions 4..7 hold 11 each
__host__ __device__ constexpr int acp_region(int c) { return c < 28 ? c / 7 : 4 + (c - 28) / 11; }
__host__ __device__ constexpr int acp_index(int c) { return c < 28 ? c % 7 : (c - 28) % 11; }
__host__ __device__ constexpr int acp_start(int g) { return g < 4 ? 7 * g : 28 + 11 * (g - 4); }
// axis distance and signed lateral offset of candidate c
__host__ __device__ constexpr int acp_depth(int c) {
  return acp_region(c) < 4 ? (acp_index(c) + 1) / 2 + 1 : 3 + 2 * acp_index(c);
}
__host__ __device__ constexpr int acp_lateral(int c) {
  return acp_region(c) < 4 && acp_index(c) > 0 ? ((acp_index(c) & 1) ? -1 : 1) * ((acp_index(c) + 1) / 2) : 0;
}
// directions: up (0,-1), down (0,1), left (-1,0), right (1,0); the lateral
// axis is x for up/down and y for left/right
__host__ __device__ constexpr int acp_dx(int c) {
  return (acp_region(c) & 3) == 2 ? -acp_depth(c) : (acp_region(c) & 3) == 3 ? acp_depth(c) : acp_lateral(c);
}
__host__ __device__ constexpr int acp_dy(int c) {
  return (acp_region(c) & 3) == 0 ? -acp_depth(c) : (acp_region(c) & 3) == 1 ? acp_depth(c) : acp_lateral(c);
}
static_assert(acp_dx(0) == 0 && acp_dy(0) == -1, "near up starts at (0, -1)");
static_assert(acp_dx(1) == -1 && acp_dy(1) == -2 && acp_dx(2) == 1 && acp_dy(2) == -2, "V arms");
static_assert(acp_dx(6) == 3 && acp_dy(6) == -4, "near up ends at (3, -4)");
static_assert(acp_dx(7 * 2 + 1) == -2 && acp_dy(7 * 2 + 1) == -1, "near left (-2, -1)");
static_assert(acp_dx(28) == 0 && acp_dy(28) == -3 && acp_dy(38) == -23, "far up strip 3..23");
static_assert(acp_dx(71) == 23 && acp_dy(71) == 0, "far right ends at (23, 0)");
}  // namespace

namespace amh {

// ---------------------------------------------------------------------------
// Refinement candidates (Sec. 3.3).  rho_t = 2^-(t+1) halves every iteration;
// the bisection candidate perturbs depth and normal; from t = 3 on the five
// other combinations of {own, perturbed, random} depth and normal follow:
// (random D, n), (D, random n), (random D, random n), (perturbed D, n),
// (D, perturbed n).  Draws (pixel, t, 0, 1) and (pixel, t, 1, 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int refine_candidates(const PhaseArgs& a, int x, int y, float4 pl,
                                                 float3 ray, float4* cand) {
  const uint32_t pix = (uint32_t)(y * a.W + x);
  const float rho = ldexpf(1.f, -(a.t + 1));
  const uint4 r0 = philox4x32_10(make_uint4(pix, (uint32_t)a.t, 0u, 1u), a.key0, a.key1);
  const float Dp = pl.w * (1.f + rho * (2.f * u01(r0.x) - 1.f));
  float3 np = make_float3(pl.x + rho * (2.f * u01(r0.y) - 1.f), pl.y + rho * (2.f * u01(r0.z) - 1.f),
                          pl.z + rho * (2.f * u01(r0.w) - 1.f));
  const float inn = 1.f / sqrtf(dot3(np, np));
  np = face_camera(make_float3(np.x * inn, np.y * inn, np.z * inn), ray);
  cand[0] = make_float4(np.x, np.y, np.z, Dp);
  if (a.t < 3) return 1;
  const uint4 r1 = philox4x32_10(make_uint4(pix, (uint32_t)a.t, 1u, 1u), a.key0, a.key1);
  const float Dr = a.dmin + (a.dmax - a.dmin) * u01(r1.x);
  const float3 nr = face_camera(normal_from_uniforms(u01(r1.y), u01(r1.z)), ray);
  cand[1] = make_float4(pl.x, pl.y, pl.z, Dr);
  cand[2] = make_float4(nr.x, nr.y, nr.z, pl.w);
  cand[3] = make_float4(nr.x, nr.y, nr.z, Dr);
  cand[4] = make_float4(pl.x, pl.y, pl.z, Dp);
  cand[5] = make_float4(np.x, np.y, np.z, pl.w);
  return 6;
}

// ---------------------------------------------------------------------------
// Eqs. (2)-(6): weights of the N views from the 8 x N cost matrix M (rows of
// invalid regions are left out of the counts and of the mean of Eq. (4)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void joint_view_selection(const PhaseArgs& a, const float* M, uint32_t valid,
                                                     uint32_t S_prev, int v_prev, float* w,
                                                     uint32_t* S_out, int* v_out) {
  const int N = a.N;
  const int nvalid = __popc(valid);
  const int k = a.k < N ? a.k : N;
  uint32_t S = 0;
  float psim[kMaxSrc];
  for (int j = 0; j < N; j++) {
    int ng = 0, nb = 0;
    float psi = 0.f;
#pragma unroll
    for (int i = 0; i < kRegions; i++) {
      if (!(valid >> i & 1u)) continue;
      const float m = M[i * kMaxSrc + j];
      ng += m < a.tau;
      nb += m > a.tau_up;
      psi += expf(-m * m * a.inv2beta2);          // Eq. (3)
    }
    psim[j] = 0.f;
    if (ng > a.n1 && nb < a.n2) {                  // good view
      S |= 1u << j;
      psi = psi / (float)nvalid;                   // Eq. (4)
      psim[j] = (j == v_prev) ? 2.f * psi : psi;   // Eqs. (5), (6)
    }
  }
  int v = -1;
  for (int j = 0; j < N; j++) {
    float wj = 0.f;
    if (S >> j & 1u) {
      int rank = 0;
      for (int q = 0; q < N; q++)
        rank += (S >> q & 1u) && (psim[q] > psim[j] || (psim[q] == psim[j] && q < j));
      if (rank < k) wj = psim[j];                  // at most k views keep weight
      if (rank == 0) v = j;
    } else if (S_prev >> j & 1u) {
      wj = 0.2f;                                   // dropped since t - 1, Eq. (5)
    }
    w[j] = wj;
  }
  float sw = 0.f;
  for (int j = 0; j < N; j++) sw += w[j];
  if (sw == 0.f) {  // no view at all: the k views of smallest mean cost
    float cm[kMaxSrc];
    for (int j = 0; j < N; j++) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < kRegions; i++)
        if (valid >> i & 1u) s += M[i * kMaxSrc + j];
      cm[j] = nvalid ? s / (float)nvalid : 0.f;
    }
    for (int j = 0; j < N; j++) {
      int rank = 0;
      for (int q = 0; q < N; q++) rank += cm[q] < cm[j] || (cm[q] == cm[j] && q < j);
      w[j] = rank < k ? 1.f : 0.f;
    }
  }
  *S_out = S;
  *v_out = v;
}

// cost of one plane under the weights w (Eq. 7), views with w = 0 skipped
__device__ __forceinline__ float weighted_cost(const PhaseArgs& a, const Hyp& h, float fx, float fy,
                                               const RefWin& rw, const float* w, float inv_sw,
                                               int* npairs) {
  float acc = 0.f;
  for (int j = 0; j < a.N; j++) {
    const float wj = w[j];
    if (wj > 0.f) {
      int ev = 0;
      acc = fmaf(wj, ncc_cost(a.v[j], h, fx, fy, rw, &ev), acc);
      *npairs += ev;
    }
  }
  return acc * inv_sw;
}

// ---------------------------------------------------------------------------
// One pixel's checkerboard update.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void update_pixel(const PhaseArgs& a, int x, int y, int* npairs) {
  const size_t pi = (size_t)y * a.W + x;
  const float fx = (float)x, fy = (float)y;
  const float3 ray = ref_ray(a.Kinv, fx, fy);

  // --- Sec. 3.1: asymmetric checkerboard propagation -----------------------
  int pick[kRegions];
#pragma unroll
  for (int g = 0; g < kRegions; g++) {
    int best = -1;
    float bc = 0.f;
#pragma unroll
    for (int c = acp_start(g); c < acp_start(g + 1); c++) {
      const int qx = x + acp_dx(c), qy = y + acp_dy(c);
      if (qx < 0 || qy < 0 || qx >= a.W || qy >= a.H) continue;
      const int q = qy * a.W + qx;
      const float cq = __ldg(&a.cost[q]);
      if (best < 0 || cq < bc) { best = q; bc = cq; }
    }
    pick[g] = best;
  }
  float4 hpl[kRegions];
  float3 hc[kRegions];
  uint32_t valid = 0;
#pragma unroll
  for (int g = 0; g < kRegions; g++) {
    hpl[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    hc[g] = make_float3(0.f, 0.f, 0.f);
    if (pick[g] < 0) continue;
    const int q = pick[g];
    const float4 pq = a.plane[q];
    const float3 nq = make_float3(pq.x, pq.y, pq.z);
    const float3 rq = ref_ray(a.Kinv, (float)(q % a.W), (float)(q / a.W));
    const float d = -pq.w * dot3(nq, rq);        // plane offset, same for q and x
    const float den = dot3(nq, ray);
    if (!(den < 0.f)) continue;
    const float Dx = -d / den;
    if (!(Dx > 0.f) || !isfinite(Dx)) continue;
    const Hyp h = make_hyp(a.Kinv, make_float4(nq.x, nq.y, nq.z, Dx), ray);
    if (!h.ok) continue;
    hpl[g] = h.pl;
    hc[g] = h.c;
    valid |= 1u << g;
  }

  // --- reference window -----------------------------------------------------
  RefWin rw;
  load_ref_window(a, x, y, rw);

  // --- Eq. (1): the 8 x N cost matrix ---------------------------------------
  float M[kRegions * kMaxSrc];
  for (int j = 0; j < a.N; j++) {
    const ViewConst& V = a.v[j];
#pragma unroll 1
    for (int g = 0; g < kRegions; g++) {
      float m = kWorst;
      if (valid >> g & 1u) {
        Hyp h;
        h.pl = hpl[g];
        h.c = hc[g];
        h.ok = true;
        int ev = 0;
        m = ncc_cost(V, h, fx, fy, rw, &ev);
        *npairs += ev;
      }
      M[g * kMaxSrc + j] = m;
    }
  }

  // --- Eqs. (2)-(6) -----------------------------------------------------------
  float w[kMaxSrc];
  uint32_t S;
  int v;
  const uint8_t vb = a.vbest[pi];
  joint_view_selection(a, M, valid, a.sel[pi], vb == 255 ? -1 : (int)vb, w, &S, &v);
  float sw = 0.f;
  uint32_t wm = 0;
  for (int j = 0; j < a.N; j++) {
    sw += w[j];
    wm |= (w[j] > 0.f ? 1u : 0u) << j;
  }
  const float inv_sw = 1.f / sw;

  // --- Eq. (7): unified cost; the own plane competes and wins ties ----------
  float4 best = a.plane[pi];
  const Hyp own = make_hyp(a.Kinv, best, ray);
  float bm = weighted_cost(a, own, fx, fy, rw, w, inv_sw, npairs);
  int choice = 8;
#pragma unroll 1
  for (int g = 0; g < kRegions; g++) {
    if (!(valid >> g & 1u)) continue;
    float acc = 0.f;
    for (int j = 0; j < a.N; j++)
      if (w[j] > 0.f) acc = fmaf(w[j], M[g * kMaxSrc + j], acc);
    acc *= inv_sw;
    if (acc < bm) { bm = acc; best = hpl[g]; choice = g; }
  }

  // --- Sec. 3.3: refinement, same weights --------------------------------------
  float4 cand[6];
  const int nc = refine_candidates(a, x, y, best, ray, cand);
  int bc = -1;
  float bcm = 0.f;
#pragma unroll 1
  for (int c = 0; c < nc; c++) {
    const Hyp h = make_hyp(a.Kinv, cand[c], ray);
    const float m = weighted_cost(a, h, fx, fy, rw, w, inv_sw, npairs);
    if (bc < 0 || m < bcm) { bc = c; bcm = m; }
  }
  if (bc >= 0 && bcm < bm) { bm = bcm; best = cand[bc]; choice = 9 + bc; }

  a.plane[pi] = best;
  a.cost[pi] = bm;
  a.sel[pi] = S;
  a.vbest[pi] = v < 0 ? (uint8_t)255 : (uint8_t)v;
  a.wmask[pi] = wm;
  a.choice[pi] = (uint8_t)choice;
}

// 16 x 16 pixel tile per block: 16 rows of 8 same-coloured pixels; a warp
// covers 4 rows (a 16 x 4 footprint).
constexpr int kTile = 16;
constexpr int kPhaseThreads = 128;

__global__ void __launch_bounds__(kPhaseThreads) phase_kernel(const __grid_constant__ PhaseArgs a) {
  const int tid = threadIdx.x;
  const int y = blockIdx.y * kTile + (tid >> 3);
  const int x = blockIdx.x * kTile + 2 * (tid & 7) + ((y + a.color) & 1);
  int npairs = 0;
  if (x < a.W && y < a.H) update_pixel(a, x, y, &npairs);
  const int tot = __reduce_add_sync(0xffffffffu, npairs);
  if ((tid & 31) == 0 && tot) atomicAdd(a.pairs, (unsigned long long)tot);
}

// Random initialisation: one thread per pixel over the whole image.
__global__ void __launch_bounds__(256) init_kernel(const __grid_constant__ PhaseArgs a) {
  const int x = blockIdx.x * 16 + (threadIdx.x & 15), y = blockIdx.y * 16 + (threadIdx.x >> 4);
  int npairs = 0;
  if (x < a.W && y < a.H) {
    const size_t pi = (size_t)y * a.W + x;
    const float fx = (float)x, fy = (float)y;
    const float3 ray = ref_ray(a.Kinv, fx, fy);
    const uint4 r = philox4x32_10(make_uint4((uint32_t)pi, 0u, 0u, 0u), a.key0, a.key1);
    const float3 n = face_camera(normal_from_uniforms(u01(r.y), u01(r.z)), ray);
    const float D = a.dmin + (a.dmax - a.dmin) * u01(r.x);
    const float4 pl = make_float4(n.x, n.y, n.z, D);
    const Hyp h = make_hyp(a.Kinv, pl, ray);
    RefWin rw;
    load_ref_window(a, x, y, rw);
    float m[kMaxSrc];
    for (int j = 0; j < a.N; j++) {
      int ev = 0;
      m[j] = ncc_cost(a.v[j], h, fx, fy, rw, &ev);
      npairs += ev;
    }
    // mean of the k smallest per-view costs (ties: lower view index)
    const int k = a.k < a.N ? a.k : a.N;
    uint32_t used = 0;
    float acc = 0.f;
    for (int r2 = 0; r2 < k; r2++) {
      int bj = -1;
      for (int j = 0; j < a.N; j++)
        if (!(used >> j & 1u) && (bj < 0 || m[j] < m[bj])) bj = j;
      used |= 1u << bj;
      acc += m[bj];
    }
    a.plane[pi] = pl;
    a.cost[pi] = acc / (float)k;
    a.sel[pi] = 0;
    a.vbest[pi] = 255;
    a.wmask[pi] = 0;
    a.choice[pi] = 8;
  }
  const int tot = __reduce_add_sync(0xffffffffu, npairs);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(a.pairs, (unsigned long long)tot);
}

// depth / normal split of the plane array
__global__ void split_maps_kernel(const float4* __restrict__ plane, size_t n, float* depth, float* normal3) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float4 p = plane[i];
    if (depth) depth[i] = p.w;
    if (normal3) { normal3[3 * i] = p.x; normal3[3 * i + 1] = p.y; normal3[3 * i + 2] = p.z; }
  }
}

}  // namespace amh

// ===========================================================================
// host side
// ===========================================================================
// struct amh_ctx is defined in amh_ctx.h

namespace {
thread_local std::string g_create_err;

int fail(amh_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_err = buf;
  return code;
}

#define CUDA_TRY(ctx, call)                                                                 \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA, "%s: %s",  \
                  #call, cudaGetErrorString(e_));                                           \
  } while (0)

bool inv3(const double* A, double* I) {
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
void mul3(const double* A, const double* B, double* C) {
  double T[9];
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) T[3 * r + q] = A[3 * r] * B[q] + A[3 * r + 1] * B[3 + q] + A[3 * r + 2] * B[6 + q];
  std::memcpy(C, T, sizeof T);
}
bool camera_ok(const amh_camera& c) {
  for (double v : c.K) if (!std::isfinite(v)) return false;
  for (double v : c.R) if (!std::isfinite(v)) return false;
  for (double v : c.t) if (!std::isfinite(v)) return false;
  if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768) return false;
  return c.K[6] == 0.0 && c.K[7] == 0.0 && c.K[8] == 1.0;
}

void free_ctx(amh_ctx* c) {
  for (int j = 0; j < AMH_MAX_SRC; j++) {
    if (c->tex[j]) cudaDestroyTextureObject(c->tex[j]);
    if (c->arr[j]) cudaFreeArray(c->arr[j]);
  }
  cudaFree(c->d_ref);
  cudaFree(c->d_plane);
  cudaFree(c->d_cost);
  cudaFree(c->d_sel);
  cudaFree(c->d_vbest);
  cudaFree(c->d_wmask);
  cudaFree(c->d_choice);
  cudaFree(c->d_pairs);
}

void fill_step_args(amh_ctx* c, int color) {
  PhaseArgs& a = c->args;
  a.color = color;
  a.t = c->t;
  a.tau = (float)(c->p.tau_mc_init * std::exp(-(double)c->t * c->t / (double)c->p.alpha));
}

int launch_check(amh_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, AMH_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
  return AMH_OK;
}
}  // namespace

extern "C" {

AMH_API int amh_default_params(amh_params* o) {
  if (!o) return AMH_EINVAL;
  std::memset(o, 0, sizeof *o);
  o->iters = 6;
  o->tau_mc_init = 0.8f;
  o->alpha = 90.f;
  o->beta = 0.3f;
  o->tau_up = 1.2f;
  o->n1 = 2;
  o->n2 = 3;
  o->k = 4;
  o->sigma_I = 3.f;
  o->sigma_x = 30.f;
  o->win_radius = 5;
  o->win_stride = 2;
  o->depth_min = 1.f;
  o->depth_max = 10.f;
  o->seed = 0;
  o->flags = 0;
  return AMH_OK;
}

AMH_API int amh_create(amh_ctx** out, const amh_params* p, int32_t n_views, const amh_camera* cams,
                       const uint8_t* const* images, int32_t images_mem, int32_t ref, const int32_t* src,
                       int32_t n_src, void* stream) {
  g_create_err.clear();
  if (!out) return fail(nullptr, AMH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p || !cams || !images || !src) return fail(nullptr, AMH_EINVAL, "NULL argument");
  if (images_mem != AMH_MEM_HOST && images_mem != AMH_MEM_DEVICE)
    return fail(nullptr, AMH_EINVAL, "images_mem must be AMH_MEM_HOST or AMH_MEM_DEVICE");
  if (n_views < 2 || ref < 0 || ref >= n_views) return fail(nullptr, AMH_EINVAL, "bad ref / n_views");
  if (n_src < 1 || n_src > AMH_MAX_SRC) return fail(nullptr, AMH_EINVAL, "n_src must be 1..32");
  if (p->win_radius != kWinR || p->win_stride != kWinStride)
    return fail(nullptr, AMH_EINVAL, "only the 11x11 stride-2 window (radius 5, stride 2) is built");
  if (!(p->k >= 1) || p->n1 < 0 || p->n2 < 0 || !(p->beta > 0) || !(p->sigma_I > 0) || !(p->sigma_x > 0) ||
      !(p->alpha > 0) || !(p->depth_min > 0) || !(p->depth_max > p->depth_min))
    return fail(nullptr, AMH_EINVAL, "invalid parameters");
  for (int j = 0; j < n_src; j++) {
    const int v = src[j];
    if (v < 0 || v >= n_views || v == ref) return fail(nullptr, AMH_EINVAL, "src[%d] = %d invalid", j, v);
    for (int q = 0; q < j; q++)
      if (src[q] == v) return fail(nullptr, AMH_EINVAL, "src[%d] repeats view %d", j, v);
  }
  if (!camera_ok(cams[ref])) return fail(nullptr, AMH_EINVAL, "reference camera invalid");
  for (int j = 0; j < n_src; j++)
    if (!camera_ok(cams[src[j]])) return fail(nullptr, AMH_EINVAL, "camera %d invalid", src[j]);
  for (int j = 0; j < n_src; j++)
    if (!images[src[j]]) return fail(nullptr, AMH_EINVAL, "image %d is NULL", src[j]);
  if (!images[ref]) return fail(nullptr, AMH_EINVAL, "reference image is NULL");

  amh_ctx* c = new (std::nothrow) amh_ctx();
  if (!c) return fail(nullptr, AMH_ENOMEM, "host allocation failed");
  c->p = *p;
  c->ref = ref;
  c->N = n_src;
  c->stream = (cudaStream_t)stream;
  const amh_camera& cr = cams[ref];
  c->W = cr.width;
  c->H = cr.height;
  double Kri[9];
  if (!inv3(cr.K, Kri)) { delete c; return fail(nullptr, AMH_EINVAL, "reference K singular"); }
  const size_t np = (size_t)c->W * c->H;
  const cudaMemcpyKind kind = images_mem == AMH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;

  auto bail = [&](int code) {
    g_create_err = c->err;
    free_ctx(c);
    delete c;
    return code;
  };
#define CTRY(call)                                                                              \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      fail(c, e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA, "%s: %s", #call,        \
           cudaGetErrorString(e_));                                                             \
      return bail(e_ == cudaErrorMemoryAllocation ? AMH_ENOMEM : AMH_ECUDA);                    \
    }                                                                                           \
  } while (0)

  CTRY(cudaMalloc(&c->d_ref, np));
  CTRY(cudaMemcpyAsync(c->d_ref, images[ref], np, kind, c->stream));
  CTRY(cudaMalloc(&c->d_plane, np * sizeof(float4)));
  CTRY(cudaMalloc(&c->d_cost, np * sizeof(float)));
  CTRY(cudaMalloc(&c->d_sel, np * sizeof(uint32_t)));
  CTRY(cudaMalloc(&c->d_vbest, np));
  CTRY(cudaMalloc(&c->d_wmask, np * sizeof(uint32_t)));
  CTRY(cudaMalloc(&c->d_choice, np));
  CTRY(cudaMalloc(&c->d_pairs, sizeof(unsigned long long)));
  CTRY(cudaMemsetAsync(c->d_pairs, 0, sizeof(unsigned long long), c->stream));

  PhaseArgs& a = c->args;
  std::memset(&a, 0, sizeof a);
  a.W = c->W;
  a.H = c->H;
  a.N = c->N;
  for (int i = 0; i < 9; i++) a.Kinv[i] = (float)Kri[i];
  a.tau_up = p->tau_up;
  a.n1 = p->n1;
  a.n2 = p->n2;
  a.k = p->k;
  a.inv2beta2 = (float)(1.0 / (2.0 * (double)p->beta * p->beta));
  a.wI = (float)(1.0 / (2.0 * (double)p->sigma_I * p->sigma_I));
  a.wX = (float)(1.0 / (2.0 * (double)p->sigma_x * p->sigma_x));
  a.squared = (p->flags & AMH_FLAG_BILATERAL_SQUARED) ? 1 : 0;
  a.dmin = p->depth_min;
  a.dmax = p->depth_max;
  a.key0 = (uint32_t)(p->seed & 0xFFFFFFFFu);
  a.key1 = (uint32_t)(p->seed >> 32);
  a.ref = c->d_ref;
  a.plane = c->d_plane;
  a.cost = c->d_cost;
  a.sel = c->d_sel;
  a.vbest = c->d_vbest;
  a.wmask = c->d_wmask;
  a.choice = c->d_choice;
  a.pairs = c->d_pairs;

  double RrT[9];
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) RrT[3 * r + q] = cr.R[3 * q + r];
  for (int j = 0; j < n_src; j++) {
    const int v = src[j];
    c->src[j] = v;
    const amh_camera& cj = cams[v];
    // relative pose ref -> j, then A = K_j R_jr K_ref^-1, b = K_j t_jr
    double Rjr[9], tjr[3], A[9], KR[9], b[3];
    mul3(cj.R, RrT, Rjr);
    for (int i = 0; i < 3; i++)
      tjr[i] = cj.t[i] - (Rjr[3 * i] * cr.t[0] + Rjr[3 * i + 1] * cr.t[1] + Rjr[3 * i + 2] * cr.t[2]);
    mul3(cj.K, Rjr, KR);
    mul3(KR, Kri, A);
    for (int i = 0; i < 3; i++) b[i] = cj.K[3 * i] * tjr[0] + cj.K[3 * i + 1] * tjr[1] + cj.K[3 * i + 2] * tjr[2];
    // shift the output by (+1, +1): rows 0 and 1 gain row 2
    for (int q = 0; q < 3; q++) { A[q] += A[6 + q]; A[3 + q] += A[6 + q]; }
    b[0] += b[2];
    b[1] += b[2];
    ViewConst& V = a.v[j];
    for (int i = 0; i < 9; i++) V.A[i] = (float)A[i];
    for (int i = 0; i < 3; i++) V.b[i] = (float)b[i];
    V.xmax = (float)cj.width;
    V.ymax = (float)cj.height;
    // texture array
    cudaChannelFormatDesc fd = cudaCreateChannelDesc<uint8_t>();
    CTRY(cudaMallocArray(&c->arr[j], &fd, cj.width, cj.height, cudaArrayTextureGather));
    CTRY(cudaMemcpy2DToArrayAsync(c->arr[j], 0, 0, images[v], cj.width, cj.width, cj.height, kind, c->stream));
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = c->arr[j];
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = cudaAddressModeClamp;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeNormalizedFloat;
    td.normalizedCoords = 0;
    CTRY(cudaCreateTextureObject(&c->tex[j], &rd, &td, nullptr));
    V.tex = c->tex[j];
  }
  CTRY(cudaStreamSynchronize(c->stream));
#undef CTRY
  *out = c;
  return AMH_OK;
}

AMH_API int amh_set_stream(amh_ctx* c, void* stream) {
  if (!c) return AMH_EINVAL;
  c->stream = (cudaStream_t)stream;
  return AMH_OK;
}

AMH_API int amh_init_random(amh_ctx* c) {
  if (!c) return AMH_EINVAL;
  c->t = 0;
  fill_step_args(c, 0);
  dim3 grid((c->W + 15) / 16, (c->H + 15) / 16);
  init_kernel<<<grid, 256, 0, c->stream>>>(c->args);
  int rc = launch_check(c, "init");
  if (rc) return rc;
  c->initialized = true;
  return AMH_OK;
}

AMH_API int amh_step_phase(amh_ctx* c, int32_t color) {
  if (!c) return AMH_EINVAL;
  if (color != 0 && color != 1) return fail(c, AMH_EINVAL, "color must be 0 or 1");
  if (!c->initialized) return fail(c, AMH_ESTATE, "state not initialised (amh_init_random or amh_set_state)");
  fill_step_args(c, color);
  dim3 grid((c->W + kTile - 1) / kTile, (c->H + kTile - 1) / kTile);
  phase_kernel<<<grid, kPhaseThreads, 0, c->stream>>>(c->args);
  int rc = launch_check(c, "phase");
  if (rc) return rc;
  if (color == 1) c->t++;
  return AMH_OK;
}

AMH_API int amh_iterate(amh_ctx* c, int32_t k) {
  if (!c) return AMH_EINVAL;
  if (k < 0) return fail(c, AMH_EINVAL, "k < 0");
  for (int i = 0; i < k; i++) {
    int rc = amh_step_phase(c, 0);
    if (rc) return rc;
    rc = amh_step_phase(c, 1);
    if (rc) return rc;
  }
  return AMH_OK;
}

AMH_API int amh_get_state(amh_ctx* c, amh_state* o, int32_t mem) {
  if (!c || !o) return AMH_EINVAL;
  if (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE) return fail(c, AMH_EINVAL, "bad memory kind");
  const size_t np = (size_t)c->W * c->H;
  const cudaMemcpyKind k = mem == AMH_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (o->plane) CUDA_TRY(c, cudaMemcpyAsync(o->plane, c->d_plane, np * sizeof(float4), k, c->stream));
  if (o->cost) CUDA_TRY(c, cudaMemcpyAsync(o->cost, c->d_cost, np * sizeof(float), k, c->stream));
  if (o->sel) CUDA_TRY(c, cudaMemcpyAsync(o->sel, c->d_sel, np * sizeof(uint32_t), k, c->stream));
  if (o->vbest) CUDA_TRY(c, cudaMemcpyAsync(o->vbest, c->d_vbest, np, k, c->stream));
  if (o->wmask) CUDA_TRY(c, cudaMemcpyAsync(o->wmask, c->d_wmask, np * sizeof(uint32_t), k, c->stream));
  if (o->choice) CUDA_TRY(c, cudaMemcpyAsync(o->choice, c->d_choice, np, k, c->stream));
  o->t = c->t;
  if (mem == AMH_MEM_HOST) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return AMH_OK;
}

AMH_API int amh_set_state(amh_ctx* c, const amh_state* in, int32_t mem) {
  if (!c || !in) return AMH_EINVAL;
  if (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE) return fail(c, AMH_EINVAL, "bad memory kind");
  if (!in->plane) return fail(c, AMH_EINVAL, "plane is required");
  if (in->t < 0) return fail(c, AMH_EINVAL, "t < 0");
  const size_t np = (size_t)c->W * c->H;
  const cudaMemcpyKind k = mem == AMH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_plane, in->plane, np * sizeof(float4), k, c->stream));
  if (in->cost) CUDA_TRY(c, cudaMemcpyAsync(c->d_cost, in->cost, np * sizeof(float), k, c->stream));
  if (in->sel) CUDA_TRY(c, cudaMemcpyAsync(c->d_sel, in->sel, np * sizeof(uint32_t), k, c->stream));
  if (in->vbest) CUDA_TRY(c, cudaMemcpyAsync(c->d_vbest, in->vbest, np, k, c->stream));
  if (in->wmask) CUDA_TRY(c, cudaMemcpyAsync(c->d_wmask, in->wmask, np * sizeof(uint32_t), k, c->stream));
  if (in->choice) CUDA_TRY(c, cudaMemcpyAsync(c->d_choice, in->choice, np, k, c->stream));
  if (!c->initialized) {  // fields not given start empty
    if (!in->cost) CUDA_TRY(c, cudaMemsetAsync(c->d_cost, 0, np * sizeof(float), c->stream));
    if (!in->sel) CUDA_TRY(c, cudaMemsetAsync(c->d_sel, 0, np * sizeof(uint32_t), c->stream));
    if (!in->vbest) CUDA_TRY(c, cudaMemsetAsync(c->d_vbest, 0xFF, np, c->stream));
    if (!in->wmask) CUDA_TRY(c, cudaMemsetAsync(c->d_wmask, 0, np * sizeof(uint32_t), c->stream));
    if (!in->choice) CUDA_TRY(c, cudaMemsetAsync(c->d_choice, 8, np, c->stream));
  }
  c->t = in->t;
  c->initialized = true;
  if (mem == AMH_MEM_HOST) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return AMH_OK;
}

AMH_API int amh_read_maps(amh_ctx* c, float* depth, float* normal3, float* cost, uint32_t* selected,
                          int32_t mem) {
  if (!c) return AMH_EINVAL;
  if (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE) return fail(c, AMH_EINVAL, "bad memory kind");
  const size_t np = (size_t)c->W * c->H;
  if (depth || normal3) {
    if (mem == AMH_MEM_DEVICE) {
      split_maps_kernel<<<1024, 256, 0, c->stream>>>(c->d_plane, np, depth, normal3);
      int rc = launch_check(c, "split_maps");
      if (rc) return rc;
    } else {
      float* dd = nullptr;
      float* dn = nullptr;
      if (depth) CUDA_TRY(c, cudaMallocAsync(&dd, np * sizeof(float), c->stream));
      if (normal3) CUDA_TRY(c, cudaMallocAsync(&dn, np * 3 * sizeof(float), c->stream));
      split_maps_kernel<<<1024, 256, 0, c->stream>>>(c->d_plane, np, dd, dn);
      int rc = launch_check(c, "split_maps");
      if (!rc && depth) CUDA_TRY(c, cudaMemcpyAsync(depth, dd, np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      if (!rc && normal3)
        CUDA_TRY(c, cudaMemcpyAsync(normal3, dn, np * 3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      if (dd) cudaFreeAsync(dd, c->stream);
      if (dn) cudaFreeAsync(dn, c->stream);
      if (rc) return rc;
    }
  }
  const cudaMemcpyKind k = mem == AMH_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (cost) CUDA_TRY(c, cudaMemcpyAsync(cost, c->d_cost, np * sizeof(float), k, c->stream));
  if (selected) CUDA_TRY(c, cudaMemcpyAsync(selected, c->d_wmask, np * sizeof(uint32_t), k, c->stream));
  if (mem == AMH_MEM_HOST) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return AMH_OK;
}

AMH_API int amh_get_info(const amh_ctx* c, int32_t* w, int32_t* h, int32_t* n, int32_t* t) {
  if (!c) return AMH_EINVAL;
  if (w) *w = c->W;
  if (h) *h = c->H;
  if (n) *n = c->N;
  if (t) *t = c->t;
  return AMH_OK;
}

AMH_API int amh_pair_count(amh_ctx* c, uint64_t* count, int32_t reset) {
  if (!c) return AMH_EINVAL;
  unsigned long long v = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&v, c->d_pairs, sizeof v, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (count) *count = v;
  if (reset) CUDA_TRY(c, cudaMemsetAsync(c->d_pairs, 0, sizeof(unsigned long long), c->stream));
  return AMH_OK;
}

AMH_API int amh_synchronize(amh_ctx* c) {
  if (!c) return AMH_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return AMH_OK;
}

AMH_API const char* amh_last_error(const amh_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}

AMH_API void amh_destroy(amh_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  delete c;
}

}  // extern "C"
