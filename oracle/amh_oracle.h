/*
 * amh_oracle.h -- plain, single-threaded FP64 CPU oracle of the AMHMVS
 * red/black checkerboard update (Xu & Tao, "Multi-View Stereo with Asymmetric
 * Checkerboard Propagation and Multi-Hypothesis Joint View Selection",
 * arXiv 1805.07920).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no source with the CUDA library.
 *
 * Every function follows one passage of the paper (cited beside it) and the
 * written readings of the passages the paper leaves open (window geometry,
 * region shapes, Eq. (5) as printed, refinement details).  Equation numbers
 * are those of the compiled paper: (1) cost matrix M, (2) tau_mc(t),
 * (3) confidence C, (4) view importance psi, (5) psi_mod, (6) epsilon,
 * (7) m_final, (8) bilateral weighted NCC.
 *
 * Conventions
 *   image      : W x H row-major intensities (0..255 as double); pixel (x, y)
 *                has its centre at integer coordinates.
 *   camera     : K (3x3, last row 0 0 1), R (3x3), t (3), row-major;
 *                x_cam = R X_world + t.
 *   plane      : (nx, ny, nz, D) per pixel: unit normal in reference-camera
 *                coordinates facing the camera (n . ray < 0) and the z-depth D
 *                of the plane along this pixel's ray.
 *   state      : plane[4*W*H], cost[W*H], sel[W*H] (bit j = source view j in
 *                S_{t-1}), vprev[W*H] (most important view v_{t-1}, -1 none),
 *                choice[W*H] (which row won the last update: 0..7 region,
 *                8 own plane, 9+c refinement candidate c), t (iteration).
 */
#ifndef AMH_ORACLE_H
#define AMH_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SRC 32
#define ORC_NREGION 8
#define ORC_MAX_REFINE 6

typedef struct {
  double K[9], R[9], t[3];
  int width, height;
} orc_camera;

typedef struct {
  int iters;                 /* 6 (Sec. 4)                                    */
  double tau_mc_init, alpha; /* 0.8, 90 (Eq. 2)                               */
  double beta;               /* 0.3 (Eq. 3)                                   */
  double tau_up;             /* 1.2 (Sec. 3.2)                                */
  int n1, n2, k;             /* 2, 3, 4 (Sec. 3.2)                            */
  double sigma_I, sigma_x;   /* 3.0, 30.0 (Eq. 8)                             */
  int win_radius, win_stride;/* 5, 2: 11x11 window, every other row/column    */
  double depth_min, depth_max;
  uint64_t seed;
  int flags;                 /* bit 0: squared bilateral differences;
                                bit 2: symmetric propagation (ablation
                                "\\ACP" of Sec. 4); bit 3: heuristic view
                                selection (ablation "\\MHJ" of Sec. 4);
                                bit 4: texture-unit bilinear interpolation
                                (orc_bilinear_texture)                      */
} orc_params;

#define ORC_FLAG_SYMMETRIC 4
#define ORC_FLAG_HEURISTIC 8
#define ORC_FLAG_TEXTURE_BILINEAR 16

typedef struct orc_ctx orc_ctx;

void orc_default_params(orc_params* p);

/* images[v] is a W_v x H_v double image for every camera v; ref and src[]
 * index into cams/images.  Returns NULL on invalid input. */
orc_ctx* orc_create(const orc_params* p, int n_views, const orc_camera* cams,
                    const double* const* images, int ref, const int* src, int n_src);
void orc_destroy(orc_ctx* c);

int  orc_width(const orc_ctx* c);
int  orc_height(const orc_ctx* c);

void orc_set_state(orc_ctx* c, const double* plane, const double* cost,
                   const uint32_t* sel, const int32_t* vprev, int t);
void orc_get_state(const orc_ctx* c, double* plane, double* cost, uint32_t* sel,
                   int32_t* vprev, int32_t* choice, int* t);

/* Random initialisation (Sec. 2 / Sec. 3: Gipuma-style random scene planes). */
void orc_init_random(orc_ctx* c);
/* One colour phase at the current t (color 0 = black: (x+y) even).  After
 * the red phase (color 1) t advances by one. */
/* threads of the pixel loops of orc_step_phase / orc_init_random (default
 * 1; the results do not depend on it) */
void orc_set_threads(int n);
void orc_step_phase(orc_ctx* c, int color);
void orc_iterate(orc_ctx* c, int k);
/* One pixel's update from the current state, without writing it. */
void orc_update_pixel(const orc_ctx* c, int x, int y, double plane_out[4],
                      double* cost_out, uint32_t* sel_out, int32_t* v_out,
                      int32_t* choice_out);
/* Unified cost (Eq. 7) of any plane at (x, y) under the view weights that
 * pixel's update would use (for judging near-ties). */
double orc_score_plane(const orc_ctx* c, int x, int y, const double plane[4]);
/* Update only the listed pixels (all of one colour) and write them back. */
void orc_update_pixels(orc_ctx* c, int n, const int32_t* xs, const int32_t* ys);

/* ---- building blocks, exposed for the oracle's own pin tests ---- */
void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);
double orc_tau_mc(const orc_params* p, int t);
double orc_confidence(const orc_params* p, double m);
/* plane-induced homography of source view j (index into src[]) */
void   orc_homography(const orc_ctx* c, int j, const double n[3], double d, double H[9]);
double orc_bilinear(const double* img, int W, int H, double x, double y);
double orc_bilinear_texture(const double* img, int W, int H, double x, double y);
/* matching cost m of one plane (n, D at pixel x) against source view j (Eq. 8) */
double orc_cost(const orc_ctx* c, int x, int y, const double plane[4], int j);
/* multi-hypothesis joint view selection on an 8 x N matrix (Eqs. 2-6) */
void   orc_mhj(const orc_params* p, int t, const double* M, const int* row_valid,
               int N, uint32_t S_prev, int v_prev, double* w_out,
               uint32_t* S_out, int32_t* v_out);
/* candidate offsets of ACP region g (0..3 near up/down/left/right, 4..7 far) */
int    orc_acp_offsets(int g, int* dx, int* dy);
int    orc_scp_offsets(int g, int* dx, int* dy);
/* index y*W+x of the picked candidate of region g, or -1 if none in image */
int    orc_acp_pick(const orc_ctx* c, int x, int y, int g);
/* propagated hypothesis of region g at pixel (x, y); 0 if the row is invalid */
int    orc_acp_row(const orc_ctx* c, int x, int y, int g, double plane_out[4]);
int    orc_refine_candidates(const orc_ctx* c, int x, int y, const double plane[4],
                             int t, double cand[][4]);
void   orc_random_plane(const orc_ctx* c, int x, int y, double plane_out[4]);

#ifdef __cplusplus
}
#endif
#endif
