// amh_api.cu -- the C-ABI of include/amh.h (host side).  It validates
// arguments, converts the cameras once (in FP64), uploads the source views as
// textures and launches the kernels of amh_kernels.cu; all method arithmetic
// runs in those kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "amh.h"
#include "amh_device.cuh"
#include "amh_ctx.h"
#include "amh_kernels.h"

using namespace amh;

namespace amh {
// depth / normal split of the plane array into row-major maps
__global__ void split_maps_kernel(const float4* __restrict__ plane, int W, int H, float* depth, float* normal3) {
  const size_t n = (size_t)W * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float4 p = plane[state_index((int)(i % W), (int)(i / W), W)];
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

}  // namespace

int amh::fail_no_context(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_create_err = buf;
  return code;
}

namespace {
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
  cudaFree(c->d_prop);
  cudaFree(c->d_status);
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
  if ((p->flags & AMH_FLAG_TEXTURE_BILINEAR) &&
      (p->flags & (AMH_FLAG_IMAGES_F16 | AMH_FLAG_SYMMETRIC_PROPAGATION | AMH_FLAG_HEURISTIC_VIEWS)))
    return fail(nullptr, AMH_EINVAL, "AMH_FLAG_TEXTURE_BILINEAR takes uint8 images and the method's own propagation and view selection");
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
  {
    const cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, AMH_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
  }
  c->N = n_src;
  c->stream = (cudaStream_t)stream;
  const amh_camera& cr = cams[ref];
  c->W = cr.width;
  c->H = cr.height;
  double Kri[9];
  if (!inv3(cr.K, Kri)) { delete c; return fail(nullptr, AMH_EINVAL, "reference K singular"); }
  const size_t np = (size_t)c->W * c->H;
  const cudaMemcpyKind kind = images_mem == AMH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const bool half = (p->flags & AMH_FLAG_IMAGES_F16) != 0;
  const size_t es = half ? 2 : 1;   // bytes per image element

  auto bail = [&](int code) {
    g_create_err = c->err;
    free_ctx(c);
    delete c;
    return code;
  };
  // Fault injection for tests: with AMH_FAIL_ALLOC_AT=k in the environment,
  // the k-th device allocation of this call reports an out-of-memory error
  // without allocating, so the cleanup path of a real failure runs.
  int alloc_n = 0, alloc_fail_at = 0;
  if (const char* e = std::getenv("AMH_FAIL_ALLOC_AT")) alloc_fail_at = std::atoi(e);
  auto injected = [&]() { return alloc_fail_at > 0 && ++alloc_n == alloc_fail_at; };
  auto dev_alloc = [&](void** ptr, size_t bytes) {
    return injected() ? cudaErrorMemoryAllocation : cudaMalloc(ptr, bytes);
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

  CTRY(dev_alloc((void**)&c->d_ref, np * es));
  CTRY(cudaMemcpyAsync(c->d_ref, images[ref], np * es, kind, c->stream));
  // the state, in the kernels' layout (state_index)
  const size_t ns = state_size(c->W, c->H);
  CTRY(dev_alloc((void**)&c->d_plane, ns * sizeof(float4)));
  CTRY(dev_alloc((void**)&c->d_cost, ns * sizeof(float)));
  CTRY(dev_alloc((void**)&c->d_sel, ns * sizeof(uint32_t)));
  CTRY(dev_alloc((void**)&c->d_vbest, ns));
  CTRY(dev_alloc((void**)&c->d_wmask, ns * sizeof(uint32_t)));
  CTRY(dev_alloc((void**)&c->d_choice, ns));
  CTRY(dev_alloc((void**)&c->d_pairs, 2 * kPairCounters * sizeof(unsigned long long)));
  CTRY(cudaMemsetAsync(c->d_pairs, 0, 2 * kPairCounters * sizeof(unsigned long long), c->stream));
  CTRY(dev_alloc((void**)&c->d_status, sizeof(unsigned int)));
  CTRY(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned int), c->stream));

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
  a.img_half = half ? 1 : 0;
  a.ablation = ((p->flags & AMH_FLAG_SYMMETRIC_PROPAGATION) ? 1 : 0) | ((p->flags & AMH_FLAG_HEURISTIC_VIEWS) ? 2 : 0);
  a.tex_filter = (p->flags & AMH_FLAG_TEXTURE_BILINEAR) ? 1 : 0;
  a.staged = (p->flags & AMH_FLAG_STAGED_FETCH) ? 1 : 0;
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
  a.status = c->d_status;
  a.pairs = c->d_pairs;

  double RrT[9];
  for (int r = 0; r < 3; r++)
    for (int q = 0; q < 3; q++) RrT[3 * r + q] = cr.R[3 * q + r];
  for (int j = 0; j < n_src; j++) {
    const int v = src[j];
    c->src[j] = v;
    const amh_camera& cj = cams[v];
    // relative pose ref -> j, then P = K_j R_jr, A = P K_ref^-1, b = K_j t_jr
    double Rjr[9], tjr[3], A[9], KR[9], b[3];
    mul3(cj.R, RrT, Rjr);
    for (int i = 0; i < 3; i++)
      tjr[i] = cj.t[i] - (Rjr[3 * i] * cr.t[0] + Rjr[3 * i + 1] * cr.t[1] + Rjr[3 * i + 2] * cr.t[2]);
    mul3(cj.K, Rjr, KR);
    mul3(KR, Kri, A);
    for (int i = 0; i < 3; i++) b[i] = cj.K[3 * i] * tjr[0] + cj.K[3 * i + 1] * tjr[1] + cj.K[3 * i + 2] * tjr[2];
    // shift the output by (+1, +1): rows 0 and 1 gain row 2
    for (int q = 0; q < 3; q++) {
      A[q] += A[6 + q]; A[3 + q] += A[6 + q];
      KR[q] += KR[6 + q]; KR[3 + q] += KR[6 + q];
    }
    b[0] += b[2];
    b[1] += b[2];
    ViewConst& V = a.v[j];
    for (int i = 0; i < 9; i++) V.A[i] = (float)A[i];
    for (int i = 0; i < 9; i++) V.P[i] = (float)KR[i];
    for (int i = 0; i < 3; i++) V.b[i] = (float)b[i];
    V.xmax = (float)cj.width;
    V.ymax = (float)cj.height;
    // the view as a texture: clamp to edge; uint8 read as value / 255, FP16
    // read as the value; point sampling (the kernels gather 2 x 2 texels and
    // blend in FP32) or, for AMH_FLAG_TEXTURE_BILINEAR, the linear filter
    cudaChannelFormatDesc fd = half ? cudaCreateChannelDescHalf() : cudaCreateChannelDesc<uint8_t>();
    CTRY(injected() ? cudaErrorMemoryAllocation
                    : cudaMallocArray(&c->arr[j], &fd, cj.width, cj.height, cudaArrayTextureGather));
    CTRY(cudaMemcpy2DToArrayAsync(c->arr[j], 0, 0, images[v], cj.width * es, cj.width * es, cj.height, kind,
                                  c->stream));
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = c->arr[j];
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = cudaAddressModeClamp;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = a.tex_filter ? cudaFilterModeLinear : cudaFilterModePoint;
    td.readMode = half ? cudaReadModeElementType : cudaReadModeNormalizedFloat;
    td.normalizedCoords = 0;
    CTRY(cudaCreateTextureObject(&c->tex[j], &rd, &td, nullptr));
    V.tex = c->tex[j];
  }
  CTRY(cudaStreamSynchronize(c->stream));
#undef CTRY
  *out = c;
  return AMH_OK;
}

AMH_API int amh_select_sources(int32_t n_views, const amh_camera* cams, int32_t ref, double depth,
                               int32_t n_src, double min_angle_deg, double max_angle_deg,
                               int32_t* src_out, int32_t* n_out) {
  if (!cams || !src_out || !n_out || n_views < 2 || ref < 0 || ref >= n_views || !(depth > 0) || n_src < 1 ||
      !(min_angle_deg >= 0) || !(max_angle_deg >= min_angle_deg))
    return fail(nullptr, AMH_EINVAL, "invalid source-selection arguments");
  if (!camera_ok(cams[ref])) return fail(nullptr, AMH_EINVAL, "reference camera invalid");
  const amh_camera& cr = cams[ref];
  auto centre = [](const amh_camera& c, double C[3]) {   // -R^T t
    for (int r = 0; r < 3; r++) C[r] = -(c.R[r] * c.t[0] + c.R[3 + r] * c.t[1] + c.R[6 + r] * c.t[2]);
  };
  double Cr[3], P[3];
  centre(cr, Cr);
  // optical axis in world coordinates: the third row of R
  for (int r = 0; r < 3; r++) P[r] = Cr[r] + depth * cr.R[6 + r];
  std::vector<std::pair<double, int>> cand;
  for (int v = 0; v < n_views; v++) {
    if (v == ref || !camera_ok(cams[v])) continue;
    const amh_camera& c = cams[v];
    double Xc[3];
    for (int r = 0; r < 3; r++) Xc[r] = c.R[3 * r] * P[0] + c.R[3 * r + 1] * P[1] + c.R[3 * r + 2] * P[2] + c.t[r];
    if (!(Xc[2] > 0)) continue;
    const double u = (c.K[0] * Xc[0] + c.K[1] * Xc[1] + c.K[2] * Xc[2]) / Xc[2];
    const double w = (c.K[3] * Xc[0] + c.K[4] * Xc[1] + c.K[5] * Xc[2]) / Xc[2];
    if (!(u >= 0 && u <= c.width - 1 && w >= 0 && w <= c.height - 1)) continue;
    double Cv[3], a[3], b[3];
    centre(c, Cv);
    for (int r = 0; r < 3; r++) { a[r] = Cr[r] - P[r]; b[r] = Cv[r] - P[r]; }
    const double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double nb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    if (!(na > 0 && nb > 0)) continue;
    const double cosang = std::max(-1.0, std::min(1.0, (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (na * nb)));
    const double ang = std::acos(cosang) * 180.0 / 3.14159265358979323846;
    if (ang >= min_angle_deg && ang <= max_angle_deg) cand.push_back({ang, v});
  }
  std::stable_sort(cand.begin(), cand.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first < y.first || (x.first == y.first && x.second < y.second);
  });
  const int n = std::min<int>(n_src, (int)cand.size());
  for (int i = 0; i < n; i++) src_out[i] = cand[i].second;
  *n_out = n;
  return AMH_OK;
}

AMH_API int amh_set_proposal(amh_ctx* c, const float* plane4, int32_t width2, int32_t height2, int32_t mem) {
  if (!c) return fail(nullptr, AMH_EINVAL, "amh_set_proposal: NULL context");
  if (!plane4 || width2 < 1 || height2 < 1 || (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE))
    return fail(c, AMH_EINVAL, "amh_set_proposal: NULL planes, empty grid or bad memory kind");
  const size_t cells = (size_t)width2 * height2;
  if (cells > c->prop_cap) {
    cudaFree(c->d_prop);
    c->d_prop = nullptr;
    c->prop_cap = 0;
    const cudaError_t e = cudaMalloc(&c->d_prop, cells * sizeof(float4));
    if (e != cudaSuccess) return fail(c, AMH_ENOMEM, "amh_set_proposal: %s", cudaGetErrorString(e));
    c->prop_cap = cells;
  }
  const cudaError_t e = cudaMemcpyAsync(c->d_prop, plane4, cells * sizeof(float4),
                                        mem == AMH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                        c->stream);
  if (e != cudaSuccess) return fail(c, AMH_ECUDA, "amh_set_proposal: %s", cudaGetErrorString(e));
  c->args.prop = c->d_prop;
  c->args.prop_w = width2;
  c->args.prop_h = height2;
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
  launch_init(c->args, c->stream);
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
  launch_phase(c->args, c->stream);
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
  const bool host = mem == AMH_MEM_HOST;
  const int W = c->W, H = c->H;
  if (o->plane) CUDA_TRY(c, export_state_field(c->d_plane, o->plane, W, H, 16, host, c->stream));
  if (o->cost) CUDA_TRY(c, export_state_field(c->d_cost, o->cost, W, H, 4, host, c->stream));
  if (o->sel) CUDA_TRY(c, export_state_field(c->d_sel, o->sel, W, H, 4, host, c->stream));
  if (o->vbest) CUDA_TRY(c, export_state_field(c->d_vbest, o->vbest, W, H, 1, host, c->stream));
  if (o->wmask) CUDA_TRY(c, export_state_field(c->d_wmask, o->wmask, W, H, 4, host, c->stream));
  if (o->choice) CUDA_TRY(c, export_state_field(c->d_choice, o->choice, W, H, 1, host, c->stream));
  o->t = c->t;
  if (mem == AMH_MEM_HOST) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return AMH_OK;
}

AMH_API int amh_set_state(amh_ctx* c, const amh_state* in, int32_t mem) {
  if (!c || !in) return AMH_EINVAL;
  if (mem != AMH_MEM_HOST && mem != AMH_MEM_DEVICE) return fail(c, AMH_EINVAL, "bad memory kind");
  if (!in->plane) return fail(c, AMH_EINVAL, "plane is required");
  if (in->t < 0) return fail(c, AMH_EINVAL, "t < 0");
  const bool host = mem == AMH_MEM_HOST;
  const int W = c->W, H = c->H;
  const size_t ns = state_size(W, H);
  CUDA_TRY(c, import_state_field(in->plane, c->d_plane, W, H, 16, host, c->stream));
  if (in->cost) CUDA_TRY(c, import_state_field(in->cost, c->d_cost, W, H, 4, host, c->stream));
  if (in->sel) CUDA_TRY(c, import_state_field(in->sel, c->d_sel, W, H, 4, host, c->stream));
  if (in->vbest) CUDA_TRY(c, import_state_field(in->vbest, c->d_vbest, W, H, 1, host, c->stream));
  if (in->wmask) CUDA_TRY(c, import_state_field(in->wmask, c->d_wmask, W, H, 4, host, c->stream));
  if (in->choice) CUDA_TRY(c, import_state_field(in->choice, c->d_choice, W, H, 1, host, c->stream));
  if (!c->initialized) {  // fields not given start empty
    if (!in->cost) CUDA_TRY(c, cudaMemsetAsync(c->d_cost, 0, ns * sizeof(float), c->stream));
    if (!in->sel) CUDA_TRY(c, cudaMemsetAsync(c->d_sel, 0, ns * sizeof(uint32_t), c->stream));
    if (!in->vbest) CUDA_TRY(c, cudaMemsetAsync(c->d_vbest, 0xFF, ns, c->stream));
    if (!in->wmask) CUDA_TRY(c, cudaMemsetAsync(c->d_wmask, 0, ns * sizeof(uint32_t), c->stream));
    if (!in->choice) CUDA_TRY(c, cudaMemsetAsync(c->d_choice, 8, ns, c->stream));
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
      split_maps_kernel<<<1024, 256, 0, c->stream>>>(c->d_plane, c->W, c->H, depth, normal3);
      int rc = launch_check(c, "split_maps");
      if (rc) return rc;
    } else {
      float* dd = nullptr;
      float* dn = nullptr;
      if (depth) CUDA_TRY(c, cudaMallocAsync(&dd, np * sizeof(float), c->stream));
      if (normal3) CUDA_TRY(c, cudaMallocAsync(&dn, np * 3 * sizeof(float), c->stream));
      split_maps_kernel<<<1024, 256, 0, c->stream>>>(c->d_plane, c->W, c->H, dd, dn);
      int rc = launch_check(c, "split_maps");
      if (!rc && depth) CUDA_TRY(c, cudaMemcpyAsync(depth, dd, np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      if (!rc && normal3)
        CUDA_TRY(c, cudaMemcpyAsync(normal3, dn, np * 3 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      if (dd) cudaFreeAsync(dd, c->stream);
      if (dn) cudaFreeAsync(dn, c->stream);
      if (rc) return rc;
    }
  }
  if (cost) CUDA_TRY(c, export_state_field(c->d_cost, cost, c->W, c->H, 4, mem == AMH_MEM_HOST, c->stream));
  if (selected) CUDA_TRY(c, export_state_field(c->d_wmask, selected, c->W, c->H, 4, mem == AMH_MEM_HOST, c->stream));
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

AMH_API int amh_pair_counts(amh_ctx* c, uint64_t* total, uint64_t* staged, int32_t reset) {
  if (!c) return AMH_EINVAL;
  unsigned long long v[2 * kPairCounters];
  CUDA_TRY(c, cudaMemcpyAsync(v, c->d_pairs, sizeof v, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  unsigned long long tot = 0, st = 0;
  for (int i = 0; i < kPairCounters; i++) {
    tot += v[i];
    st += v[kPairCounters + i];
  }
  if (total) *total = tot;
  if (staged) *staged = st;
  if (reset) CUDA_TRY(c, cudaMemsetAsync(c->d_pairs, 0, sizeof v, c->stream));
  return AMH_OK;
}

AMH_API int amh_pair_count(amh_ctx* c, uint64_t* count, int32_t reset) {
  return amh_pair_counts(c, count, nullptr, reset);
}

AMH_API int amh_synchronize(amh_ctx* c) {
  if (!c) return AMH_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
#ifdef AMH_BOUNDS_CHECK
  unsigned int st = 0;
  CUDA_TRY(c, cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
  if (st) return fail(c, AMH_EDEVICE, "bounds check: index out of range in the update (status 0x%x: 1 pixel, 2 neighbour, "
                                      "4 reference image, 8 proposal)", st);
#endif
  return AMH_OK;
}

AMH_API int amh_bounds_checked(void) {
#ifdef AMH_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
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
