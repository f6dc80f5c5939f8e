/*
 * scenegen.c -- seeded synthetic multi-view scenes for the checkerboard
 * update: a ray caster over planes, bounded quads and spheres with a 3-D
 * Perlin-noise albedo evaluated at the hit point (so every view sees the same
 * surface texture), 2x2 supersampling, per-view gain and bias, and uint8
 * quantisation.  It also writes the ground-truth z-depth and normal of every
 * pixel.
 *
 * This is an input generator only: it holds none of the stereo method's
 * arithmetic (no homographies, no matching cost, no view selection) and is
 * shared by the tests, the benchmark and the examples.
 *
 * Noise: "improved noise" (K. Perlin, "Improving noise", SIGGRAPH 2002):
 * quintic fade 6t^5 - 15t^4 + 10t^3 and gradients along the twelve cube-edge
 * directions, with a permutation table shuffled from the scene seed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double K[9], R[9], t[3];
  int width, height;
} syn_camera;

/* primitive kinds */
enum { SYN_PLANE = 0, SYN_QUAD = 1, SYN_SPHERE = 2, SYN_SKY = 3 };

typedef struct {
  int kind;
  int flat;          /* 1: constant albedo (textureless surface)              */
  double a[3];       /* plane: normal; quad/sphere/sky: centre               */
  double b[3];       /* plane: (d, 0, 0); quad: half-axis u; sphere: (r,0,0) */
  double c[3];       /* quad: half-axis v                                      */
  double albedo;     /* base albedo in [0, 1]                                  */
  double tex_freq;   /* noise frequency (1 / world units)                      */
  double tex_amp;    /* noise amplitude                                        */
  double tex_off;    /* offset into the noise field                            */
} syn_prim;

typedef struct {
  int perm[512];
  double flat_freq;      /* frequency of the textureless-patch mask (0: none) */
  double flat_thresh;    /* mask threshold: noise above it is textureless     */
  double flat_albedo;
} syn_noise;

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }
static double lerp(double t, double a, double b) { return a + t * (b - a); }
static double grad(int h, double x, double y, double z) {
  switch (h & 15) {
    case 0: return x + y;   case 1: return -x + y;  case 2: return x - y;   case 3: return -x - y;
    case 4: return x + z;   case 5: return -x + z;  case 6: return x - z;   case 7: return -x - z;
    case 8: return y + z;   case 9: return -y + z;  case 10: return y - z;  case 11: return -y - z;
    case 12: return x + y;  case 13: return -x + y; case 14: return -y + z; default: return -y - z;
  }
}
static double perlin(const int* P, double x, double y, double z) {
  double fx = floor(x), fy = floor(y), fz = floor(z);
  int X = (int)fx & 255, Y = (int)fy & 255, Z = (int)fz & 255;
  x -= fx; y -= fy; z -= fz;
  double u = fade(x), v = fade(y), w = fade(z);
  int A = P[X] + Y, AA = P[A] + Z, AB = P[A + 1] + Z;
  int B = P[X + 1] + Y, BA = P[B] + Z, BB = P[B + 1] + Z;
  return lerp(w, lerp(v, lerp(u, grad(P[AA], x, y, z), grad(P[BA], x - 1, y, z)),
                       lerp(u, grad(P[AB], x, y - 1, z), grad(P[BB], x - 1, y - 1, z))),
              lerp(v, lerp(u, grad(P[AA + 1], x, y, z - 1), grad(P[BA + 1], x - 1, y, z - 1)),
                   lerp(u, grad(P[AB + 1], x, y - 1, z - 1), grad(P[BB + 1], x - 1, y - 1, z - 1))));
}
/* four octaves of fractal noise, roughly in [-1, 1] */
static double fbm(const int* P, double x, double y, double z) {
  double s = 0, amp = 1.0, f = 1.0;
  for (int o = 0; o < 4; o++) {
    s += amp * perlin(P, x * f, y * f, z * f);
    f *= 2.03; amp *= 0.5;
  }
  return s;
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* nearest hit along o + s d (s > 1e-9); returns primitive index or -1 */
static int intersect(const syn_prim* pr, int np, const double* o, const double* d,
                     double* s_out, double* n_out) {
  int best = -1;
  double bs = INFINITY, bn[3] = {0, 0, 0};
  for (int i = 0; i < np; i++) {
    const syn_prim* p = &pr[i];
    if (p->kind == SYN_PLANE || p->kind == SYN_QUAD) {
      double n[3];
      if (p->kind == SYN_PLANE) { n[0] = p->a[0]; n[1] = p->a[1]; n[2] = p->a[2]; }
      else {
        n[0] = p->b[1] * p->c[2] - p->b[2] * p->c[1];
        n[1] = p->b[2] * p->c[0] - p->b[0] * p->c[2];
        n[2] = p->b[0] * p->c[1] - p->b[1] * p->c[0];
        double l = sqrt(dot3(n, n)); n[0] /= l; n[1] /= l; n[2] /= l;
      }
      double den = dot3(n, d);
      if (fabs(den) < 1e-12) continue;
      double s;
      if (p->kind == SYN_PLANE) s = -(dot3(n, o) + p->b[0]) / den;
      else {
        double oc[3] = {p->a[0] - o[0], p->a[1] - o[1], p->a[2] - o[2]};
        s = dot3(n, oc) / den;
      }
      if (!(s > 1e-9) || s >= bs) continue;
      if (p->kind == SYN_QUAD) {
        double X[3] = {o[0] + s * d[0] - p->a[0], o[1] + s * d[1] - p->a[1], o[2] + s * d[2] - p->a[2]};
        double cu = dot3(X, p->b) / dot3(p->b, p->b), cv = dot3(X, p->c) / dot3(p->c, p->c);
        if (fabs(cu) > 1.0 || fabs(cv) > 1.0) continue;
      }
      bs = s; best = i; bn[0] = n[0]; bn[1] = n[1]; bn[2] = n[2];
    } else {  /* sphere (outside) or sky (inside, far root) */
      double oc[3] = {o[0] - p->a[0], o[1] - p->a[1], o[2] - p->a[2]};
      double r = p->b[0];
      double B = dot3(oc, d), C = dot3(oc, oc) - r * r, A = dot3(d, d);
      double disc = B * B - A * C;
      if (disc < 0) continue;
      double sq = sqrt(disc);
      double s = p->kind == SYN_SPHERE ? (-B - sq) / A : (-B + sq) / A;
      if (!(s > 1e-9) || s >= bs) continue;
      bs = s; best = i;
      for (int k = 0; k < 3; k++) bn[k] = (o[k] + s * d[k] - p->a[k]) / r;
    }
  }
  if (best >= 0) { *s_out = bs; n_out[0] = bn[0]; n_out[1] = bn[1]; n_out[2] = bn[2]; }
  return best;
}

static double albedo_at(const syn_prim* p, const syn_noise* nz, const double* X) {
  if (p->flat) return p->albedo;
  if (nz->flat_freq > 0) {
    double m = perlin(nz->perm, X[0] * nz->flat_freq + 17.3, X[1] * nz->flat_freq + 5.1,
                      X[2] * nz->flat_freq + 9.7);
    if (m > nz->flat_thresh) return nz->flat_albedo;
  }
  double f = p->tex_freq, o = p->tex_off;
  double a = p->albedo + p->tex_amp * fbm(nz->perm, X[0] * f + o, X[1] * f + 0.5 * o, X[2] * f - o);
  return a < 0 ? 0 : (a > 1 ? 1 : a);
}

static int inv3(const double* A, double* I) {
  double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (det == 0) return 0;
  double id = 1.0 / det;
  I[0] = c00 * id; I[1] = (A[2] * A[7] - A[1] * A[8]) * id; I[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  I[3] = c01 * id; I[4] = (A[0] * A[8] - A[2] * A[6]) * id; I[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  I[6] = c02 * id; I[7] = (A[1] * A[6] - A[0] * A[7]) * id; I[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return 1;
}

/* Shuffle 0..255 with a 64-bit LCG seeded by `seed` (Fisher-Yates). */
void syn_make_perm(uint64_t seed, int* perm512) {
  int p[256];
  for (int i = 0; i < 256; i++) p[i] = i;
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  for (int i = 255; i > 0; i--) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    int j = (int)((s >> 33) % (uint64_t)(i + 1));
    int tmp = p[i]; p[i] = p[j]; p[j] = tmp;
  }
  for (int i = 0; i < 512; i++) perm512[i] = p[i & 255];
}

/* Render one view: uint8 image (gain * albedo * 255 + bias, rounded and
 * clamped), z-depth (0 where nothing is hit) and unit normal facing the
 * camera (camera coordinates).  Supersampling ss x ss per pixel for the
 * image; depth and normal come from the pixel-centre ray and are skipped
 * when depth is NULL. */
int syn_render_view(const syn_camera* cam, const syn_prim* prims, int n_prims,
                    const int* perm512, double flat_freq, double flat_thresh,
                    double flat_albedo, double gain, double bias, int ss,
                    uint8_t* image, float* depth, float* normal) {
  syn_noise nz;
  memcpy(nz.perm, perm512, sizeof nz.perm);
  nz.flat_freq = flat_freq; nz.flat_thresh = flat_thresh; nz.flat_albedo = flat_albedo;
  double Kinv[9];
  if (!inv3(cam->K, Kinv)) return -1;
  const double* R = cam->R;
  /* camera centre C = -R^T t */
  double C[3];
  for (int i = 0; i < 3; i++) C[i] = -(R[i] * cam->t[0] + R[3 + i] * cam->t[1] + R[6 + i] * cam->t[2]);
  const int W = cam->width, H = cam->height;
  if (ss < 1) ss = 1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      double acc = 0;
      for (int sy = 0; sy < ss; sy++)
        for (int sx = 0; sx < ss; sx++) {
          double px = x + (sx + 0.5) / ss - 0.5, py = y + (sy + 0.5) / ss - 0.5;
          double rc[3] = {Kinv[0] * px + Kinv[1] * py + Kinv[2], Kinv[3] * px + Kinv[4] * py + Kinv[5],
                          Kinv[6] * px + Kinv[7] * py + Kinv[8]};
          double d[3];
          for (int i = 0; i < 3; i++) d[i] = R[i] * rc[0] + R[3 + i] * rc[1] + R[6 + i] * rc[2];
          double s, n[3];
          int h = intersect(prims, n_prims, C, d, &s, n);
          double a = 0;
          if (h >= 0) {
            double X[3] = {C[0] + s * d[0], C[1] + s * d[1], C[2] + s * d[2]};
            a = albedo_at(&prims[h], &nz, X);
          }
          acc += a;
        }
      acc /= (double)(ss * ss);
      double v = floor(gain * acc * 255.0 + bias + 0.5);
      image[(size_t)y * W + x] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
      if (!depth) continue;
      /* ground truth at the pixel centre */
      double rc[3] = {Kinv[0] * x + Kinv[1] * y + Kinv[2], Kinv[3] * x + Kinv[4] * y + Kinv[5],
                      Kinv[6] * x + Kinv[7] * y + Kinv[8]};
      double d[3];
      for (int i = 0; i < 3; i++) d[i] = R[i] * rc[0] + R[3 + i] * rc[1] + R[6 + i] * rc[2];
      double s, n[3];
      int h = intersect(prims, n_prims, C, d, &s, n);
      size_t pi = (size_t)y * W + x;
      if (h < 0) {
        depth[pi] = 0; normal[3 * pi] = 0; normal[3 * pi + 1] = 0; normal[3 * pi + 2] = 0;
        continue;
      }
      /* z-depth: the camera-space z of the hit point is s * rc_z (rc_z = 1 for
       * a K with last row 0 0 1) */
      depth[pi] = (float)(s * rc[2]);
      double nc[3];
      for (int i = 0; i < 3; i++) nc[i] = R[3 * i] * n[0] + R[3 * i + 1] * n[1] + R[3 * i + 2] * n[2];
      if (nc[0] * rc[0] + nc[1] * rc[1] + nc[2] * rc[2] > 0) { nc[0] = -nc[0]; nc[1] = -nc[1]; nc[2] = -nc[2]; }
      normal[3 * pi] = (float)nc[0]; normal[3 * pi + 1] = (float)nc[1]; normal[3 * pi + 2] = (float)nc[2];
    }
  }
  return 0;
}
