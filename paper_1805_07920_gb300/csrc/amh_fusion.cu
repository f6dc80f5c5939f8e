// amh_fusion.cu -- post-processing of the depth maps (Sec. 3.3, last two
// paragraphs): the 4x4 median filter, and the fusion of several views'
// depth / normal maps by Gipuma's consistency check (the paper's reference
// [9]) with the thresholds f_eps (disparity difference), f_ang (normal
// difference) and f_con (consistent views).  Readings (the paper leaves the
// details to [9]):
//   median: offsets -2..+1 in x and y, clamped borders, mean of the 8th and
//     9th smallest of the 16 values;
//   fusion: pixel p of view i with depth D > 0 back-projects to the world
//     point X with world normal n; view j agrees when X is in front of it,
//     projects to the pixel q = floor(u + 0.5), floor(v + 0.5) inside it with
//     D_j(q) > 0, f_j |C_i - C_j| |1 / z_j(X) - 1 / D_j(q)| <= f_eps and the
//     angle between n and view j's world normal at q is <= f_ang; with at
//     least f_con agreeing views the point is the mean of X and their
//     back-projected points, the normal the normalised sum of the normals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "amh.h"
#include "amh_ctx.h"

namespace amh {
namespace {

constexpr int kFuseMaxViews = 32;

__global__ void median4_kernel(const float* __restrict__ in, float* __restrict__ out, int W, int H) {
  const size_t n = (size_t)W * H;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % W), y = (int)(i / W);
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int xx = min(max(x + (k & 3) - 2, 0), W - 1), yy = min(max(y + (k >> 2) - 2, 0), H - 1);
      v[k] = __ldg(&in[(size_t)yy * W + xx]);
    }
    // insertion sort in registers (the loops unroll: no local memory)
#pragma unroll
    for (int a = 1; a < 16; a++) {
#pragma unroll
      for (int b = a; b > 0; b--) {
        const float lo = fminf(v[b - 1], v[b]), hi = fmaxf(v[b - 1], v[b]);
        v[b - 1] = lo;
        v[b] = hi;
      }
    }
    // both halves are exact: one rounding, as the exact mean rounded to FP32
    out[i] = 0.5f * v[7] + 0.5f * v[8];
  }
}

struct FuseView {
  float Kinv[9];
  float K[9];
  float R[9];
  float t[3];
  float C[3];
  int W, H;
  const float* depth;
  const float* normal;
  float* points;
  uint8_t* count;
};

struct FuseArgs {
  int n;
  float f_eps, cos_ang;
  int f_con;
  FuseView v[kFuseMaxViews];
};

__global__ void __launch_bounds__(256) fuse_kernel(const __grid_constant__ FuseArgs a) {
  const int i = blockIdx.y;
  const FuseView& Vi = a.v[i];
  const size_t np = (size_t)Vi.W * Vi.H;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < np; p += (size_t)gridDim.x * blockDim.x) {
    const float x = (float)(p % Vi.W), y = (float)(p / Vi.W);
    const float D = Vi.depth[p];
    float out[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int cnt = 0;
    if (D > 0.f) {
      // X = R^T (D K^-1 [x y 1] - t), n = R^T n_cam
      const float rx = Vi.Kinv[0] * x + Vi.Kinv[1] * y + Vi.Kinv[2];
      const float ry = Vi.Kinv[3] * x + Vi.Kinv[4] * y + Vi.Kinv[5];
      const float rz = Vi.Kinv[6] * x + Vi.Kinv[7] * y + Vi.Kinv[8];
      const float cx = D * rx - Vi.t[0], cy = D * ry - Vi.t[1], cz = D * rz - Vi.t[2];
      float X[3], n[3];
      const float* nc = Vi.normal + 3 * p;
      for (int r = 0; r < 3; r++) {
        X[r] = Vi.R[r] * cx + Vi.R[3 + r] * cy + Vi.R[6 + r] * cz;
        n[r] = Vi.R[r] * nc[0] + Vi.R[3 + r] * nc[1] + Vi.R[6 + r] * nc[2];
      }
      const float nn = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      float sX[3] = {X[0], X[1], X[2]}, sN[3] = {n[0], n[1], n[2]};
      for (int j = 0; j < a.n; j++) {
        if (j == i) continue;
        const FuseView& Vj = a.v[j];
        float Xc[3];
        for (int r = 0; r < 3; r++) Xc[r] = Vj.R[3 * r] * X[0] + Vj.R[3 * r + 1] * X[1] + Vj.R[3 * r + 2] * X[2] + Vj.t[r];
        const float z = Xc[2];
        if (!(z > 0.f)) continue;
        const float u = (Vj.K[0] * Xc[0] + Vj.K[1] * Xc[1] + Vj.K[2] * Xc[2]) / z;
        const float v = (Vj.K[3] * Xc[0] + Vj.K[4] * Xc[1] + Vj.K[5] * Xc[2]) / z;
        const float uf = floorf(u + 0.5f), vf = floorf(v + 0.5f);
        if (!(uf >= 0.f && uf < (float)Vj.W && vf >= 0.f && vf < (float)Vj.H)) continue;
        const size_t q = (size_t)vf * Vj.W + (size_t)uf;
        const float Dj = Vj.depth[q];
        if (!(Dj > 0.f)) continue;
        const float bx = Vi.C[0] - Vj.C[0], by = Vi.C[1] - Vj.C[1], bz = Vi.C[2] - Vj.C[2];
        const float disp = Vj.K[0] * sqrtf(bx * bx + by * by + bz * bz) * fabsf(1.f / z - 1.f / Dj);
        if (!(disp <= a.f_eps)) continue;
        const float* ncj = Vj.normal + 3 * q;
        float nj[3];
        for (int r = 0; r < 3; r++) nj[r] = Vj.R[r] * ncj[0] + Vj.R[3 + r] * ncj[1] + Vj.R[6 + r] * ncj[2];
        const float dn = sqrtf(nj[0] * nj[0] + nj[1] * nj[1] + nj[2] * nj[2]) * nn;
        const float dot = (n[0] * nj[0] + n[1] * nj[1] + n[2] * nj[2]) / fmaxf(dn, 1e-30f);
        if (!(dot >= a.cos_ang)) continue;
        // the agreeing view's own point at q
        const float qx = Vj.Kinv[0] * uf + Vj.Kinv[1] * vf + Vj.Kinv[2];
        const float qy = Vj.Kinv[3] * uf + Vj.Kinv[4] * vf + Vj.Kinv[5];
        const float qz = Vj.Kinv[6] * uf + Vj.Kinv[7] * vf + Vj.Kinv[8];
        const float ex = Dj * qx - Vj.t[0], ey = Dj * qy - Vj.t[1], ez = Dj * qz - Vj.t[2];
        for (int r = 0; r < 3; r++) {
          sX[r] += Vj.R[r] * ex + Vj.R[3 + r] * ey + Vj.R[6 + r] * ez;
          sN[r] += nj[r];
        }
        cnt++;
      }
      if (cnt >= a.f_con) {
        const float inv = 1.f / (float)(1 + cnt);
        const float ln = sqrtf(sN[0] * sN[0] + sN[1] * sN[1] + sN[2] * sN[2]);
        for (int r = 0; r < 3; r++) {
          out[r] = sX[r] * inv;
          out[3 + r] = sN[r] / fmaxf(ln, 1e-30f);
        }
      }
    }
    float* o = Vi.points + 6 * p;
    for (int r = 0; r < 6; r++) o[r] = out[r];
    Vi.count[p] = (uint8_t)cnt;
  }
}

bool inv3f(const double* A, double* I) {
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

int launch_status(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AMH_OK : fail_no_context(AMH_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
}

}  // namespace
}  // namespace amh

using namespace amh;

extern "C" {

AMH_API int amh_median4(const float* depth_in, float* depth_out, int32_t width, int32_t height, void* stream) {
  if (!depth_in || !depth_out || width < 1 || height < 1 || depth_in == depth_out)
    return fail_no_context(AMH_EINVAL, "amh_median4: NULL or aliased buffers, or an empty image");
  const size_t n = (size_t)width * height;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 65535);
  median4_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(depth_in, depth_out, width, height);
  return launch_status("amh_median4");
}

AMH_API int amh_fuse(int32_t n_views, const amh_camera* cams, const float* const* depth, const float* const* normal3,
                     float f_eps, float f_ang_deg, int32_t f_con, float* const* points6, uint8_t* const* count,
                     void* stream) {
  if (n_views < 2 || n_views > kFuseMaxViews || !cams || !depth || !normal3 || !points6 || !count)
    return fail_no_context(AMH_EINVAL, "amh_fuse: 2..%d views with non-NULL arrays required", kFuseMaxViews);
  if (!(f_eps >= 0.f) || !(f_ang_deg >= 0.f && f_ang_deg <= 180.f) || f_con < 1)
    return fail_no_context(AMH_EINVAL, "amh_fuse: thresholds out of range");
  FuseArgs a;
  std::memset(&a, 0, sizeof a);
  a.n = n_views;
  a.f_eps = f_eps;
  a.cos_ang = (float)std::cos((double)f_ang_deg * 3.14159265358979323846 / 180.0);
  a.f_con = f_con;
  size_t most = 0;
  for (int v = 0; v < n_views; v++) {
    const amh_camera& c = cams[v];
    if (!depth[v] || !normal3[v] || !points6[v] || !count[v] || c.width < 1 || c.height < 1)
      return fail_no_context(AMH_EINVAL, "amh_fuse: view %d has a NULL array or an empty image", v);
    double Ki[9];
    if (!inv3f(c.K, Ki)) return fail_no_context(AMH_EINVAL, "amh_fuse: K of view %d is singular", v);
    FuseView& F = a.v[v];
    for (int k = 0; k < 9; k++) {
      F.Kinv[k] = (float)Ki[k];
      F.K[k] = (float)c.K[k];
      F.R[k] = (float)c.R[k];
    }
    for (int r = 0; r < 3; r++) {
      F.t[r] = (float)c.t[r];
      F.C[r] = (float)-(c.R[r] * c.t[0] + c.R[3 + r] * c.t[1] + c.R[6 + r] * c.t[2]);   // -R^T t
    }
    F.W = c.width;
    F.H = c.height;
    F.depth = depth[v];
    F.normal = normal3[v];
    F.points = points6[v];
    F.count = count[v];
    most = std::max(most, (size_t)c.width * c.height);
  }
  dim3 grid((unsigned)std::min<size_t>((most + 255) / 256, 4096), (unsigned)n_views);
  fuse_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  return launch_status("amh_fuse");
}

}  // extern "C"
