/*
 * amh.h -- C-ABI of the GB300 (sm_103a) implementation of the AMHMVS
 * red/black checkerboard update (Xu & Tao, "Multi-View Stereo with Asymmetric
 * Checkerboard Propagation and Multi-Hypothesis Joint View Selection",
 * arXiv 1805.07920).
 *
 * One context holds one reference view with up to 32 source views, all
 * resident on one GPU.  Every step of the update runs in this library's own
 * CUDA kernels; there is no CPU path.  The signatures use plain pointers and
 * sizes only.
 *
 * Conventions shared by all entry points
 *   - Return value: AMH_OK (0) on success, a negative AMH_E* code on failure.
 *     No call aborts the process; amh_last_error() returns a message for the
 *     last failure of a context (or of a failed amh_create when ctx is NULL).
 *   - Images: uint8 grayscale, row-major, width x height, tightly packed.
 *     Pixel (x, y) has its centre at integer coordinates (x, y).
 *   - Cameras: pinhole K (3x3, last row 0 0 1), R (3x3), t (3), row-major,
 *     world-to-camera: x_cam = R X_world + t (Sec. 2: calibrated cameras).
 *   - Planes (Sec. 2, scene-space planes): per pixel (nx, ny, nz, D): unit
 *     normal in reference-camera coordinates facing the camera (n . ray < 0)
 *     and the z-depth D of the plane along the pixel's ray.
 *   - Memory kinds: AMH_MEM_HOST buffers are ordinary host memory (pinned or
 *     not); AMH_MEM_DEVICE buffers are device pointers on the context's GPU
 *     (e.g. from torch.Tensor.data_ptr()).  The caller owns every buffer it
 *     passes; the library copies inputs at create time and never keeps a
 *     caller pointer.
 *   - Streams: all work of a context is enqueued on its stream (the one given
 *     at create time or by amh_set_stream; NULL = the legacy default stream).
 *     Calls that take device buffers are asynchronous with respect to the
 *     host; calls that take host buffers synchronise the stream before they
 *     return.  A context must not be used from two host threads at once.
 */
#ifndef AMH_H
#define AMH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(_WIN32)
#define AMH_API
#else
#define AMH_API __attribute__((visibility("default")))
#endif

#define AMH_MAX_SRC 32

enum {
  AMH_OK = 0,
  AMH_EINVAL = -1,      /* invalid argument (null pointer, size, camera, ...)   */
  AMH_ECUDA = -2,       /* a CUDA runtime call failed                            */
  AMH_ENOMEM = -3,      /* device or host allocation failed                      */
  AMH_EDEVICE = -4,     /* a kernel reported an error through its status word
                           (bounds-checked builds, see amh_bounds_checked)        */
  AMH_ESTATE = -5       /* call out of order (e.g. iterate before init)          */
};

enum { AMH_MEM_HOST = 0, AMH_MEM_DEVICE = 1 };

/* parameter flags */
enum {
  AMH_FLAG_BILATERAL_SQUARED = 1, /* use dI^2 and dx^2 in the bilateral weight  */
  AMH_FLAG_IMAGES_F16 = 2,        /* images are IEEE binary16 (2 bytes/pixel,
                                     intensities in any unit) instead of uint8;
                                     they are stored as FP16 textures, the
                                     interpolation and NCC moments stay FP32   */
  /* The ablations of Sec. 4 (Table 2, columns "\ACP" and "\MHJ"); single
   * contexts only (amh_batch_create rejects them). */
  AMH_FLAG_SYMMETRIC_PROPAGATION = 4, /* instead of ACP (Sec. 3.1): region g
                                     is one fixed candidate, the axis
                                     neighbour at distance 1 (g = 0..3) or 5
                                     (g = 4..7) up / down / left / right    */
  AMH_FLAG_HEURISTIC_VIEWS = 8,   /* instead of MHJ (Sec. 3.2): every
                                     hypothesis is scored by the mean of its
                                     own k smallest per-view costs; no S_t or
                                     v_t is kept (sel 0, vbest 255)           */
  /* Precision form of the warped samples of Eq. (8) (the paper does not fix
   * the interpolation): the texture unit's linear filter interpolates, with
   * its fractions and their product rounded half up to 1/256, instead of
   * FP32 blends of gathered texels (fewer instructions per sample).  uint8
   * images and the method's own propagation / view selection only (amh_create
   * and amh_batch_create reject other combinations). */
  AMH_FLAG_TEXTURE_BILINEAR = 16,
  /* Fetch path of the 8 x N matrix of Eq. (1) in single contexts (a
   * measured alternative; the default fetches every window sample through
   * the texture unit): from t = 1 on, per block of pixels and source view, a
   * shared-memory box of 40 x 40 bilinear cells is filled from the texture
   * and serves the samples of every warp whose windows of a (hypothesis,
   * view) pair all fit inside; the other samples use the texture unit.  The
   * interpolation is FP32 either way, in a different order of operations, so
   * results agree with the default path to rounding, not bit for bit. */
  AMH_FLAG_STAGED_FETCH = 32
};

typedef struct amh_ctx amh_ctx;

typedef struct {
  double K[9];
  double R[9];
  double t[3];
  int32_t width;
  int32_t height;
} amh_camera;

/* Method parameters.  amh_default_params() fills the values of Sec. 4:
 * 6 iterations, tau_mc_init 0.8, alpha 90 (Eq. 2), beta 0.3 (Eq. 3),
 * tau_up 1.2, n1 2, n2 3, k 4 (Sec. 3.2), sigma_I 3, sigma_x 30 (Eq. 8), and
 * the 11x11 window with every other row and column (radius 5, stride 2,
 * Sec. 3.3).  This build supports radius 5 / stride 2 only. */
typedef struct {
  int32_t iters;
  float tau_mc_init, alpha, beta, tau_up;
  int32_t n1, n2, k;
  float sigma_I, sigma_x;
  int32_t win_radius, win_stride;
  float depth_min, depth_max;   /* range of random depths (init, refinement) */
  uint64_t seed;                /* Philox4x32-10 key                          */
  int32_t flags;                /* AMH_FLAG_*                                 */
} amh_params;

/* Per-pixel state, W x H arrays in the memory kind given to get/set:
 *   plane[4 W H]  float  (nx, ny, nz, D) per pixel
 *   cost[W H]     float  current unified cost m_final of the kept plane (Eq. 7)
 *   sel[W H]      uint32 S_t: bit j set when source view j was a good view at
 *                        the pixel's last update (Sec. 3.2)
 *   vbest[W H]    uint8  v_t: most important view of the last update, 255 none
 *   wmask[W H]    uint32 views with a nonzero weight psi_mod at the last update
 *   choice[W H]   uint8  row that won the last update: 0..7 ACP region
 *                        (near up/down/left/right, far up/down/left/right),
 *                        8 own plane, 9 + c refinement candidate c,
 *                        15 a proposal (amh_net_propose / amh_set_proposal)
 *   t             iteration index of the next update (0-based)
 * Any pointer except plane may be NULL in amh_get_state (not read back) and
 * in amh_set_state (left unchanged; plane is required there). */
typedef struct {
  float* plane;
  float* cost;
  uint32_t* sel;
  uint8_t* vbest;
  uint32_t* wmask;
  uint8_t* choice;
  int32_t t;
} amh_state;

/* Fill *out with the parameters of Sec. 4.  Returns AMH_EINVAL on NULL. */
AMH_API int amh_default_params(amh_params* out);

/* Create a context for reference view `ref` and source views src[0..n_src-1]
 * (indices into cams/images, n_src in 1..32, no repeats, none equal to ref).
 * images[v] points to a cams[v].height x cams[v].width uint8 image in the
 * memory kind `images_mem`; only ref and the listed sources are read.  The
 * images are copied into device-resident texture arrays.  Fails with
 * AMH_EINVAL on bad sizes, singular or non-pinhole K, or unsupported window
 * parameters; with AMH_ENOMEM when the device is full, after freeing what
 * it had allocated.  `stream` is a cudaStream_t (NULL = legacy default
 * stream).  Test facility: with AMH_FAIL_ALLOC_AT=k in the environment the
 * k-th device allocation of the call reports out-of-memory without
 * allocating. */
AMH_API int amh_create(amh_ctx** out, const amh_params* params, int32_t n_views,
                       const amh_camera* cams, const uint8_t* const* images,
                       int32_t images_mem, int32_t ref, const int32_t* src,
                       int32_t n_src, void* stream);

/* Change the stream later work is enqueued on. */
AMH_API int amh_set_stream(amh_ctx* ctx, void* stream);

/* Random initialisation (Sec. 2, Gipuma-style random scene planes): depth
 * uniform in [depth_min, depth_max], normal uniform on the sphere flipped to
 * face the camera, from Philox4x32-10 draws keyed by (seed) with counter
 * (pixel, 0, 0, 0); the initial cost is the mean of the k smallest per-view
 * costs (the heuristic view selection of Sec. 2); S = {}, v = none, t = 0. */
AMH_API int amh_init_random(amh_ctx* ctx);

/* One colour phase of the red/black checkerboard (Sec. 3.1, Fig. 2(a)) at the
 * current t: every pixel with (x + y) % 2 == color is updated from pixels of
 * the other colour -- asymmetric checkerboard propagation (8 hypotheses),
 * the 8 x N cost matrix of bilateral weighted NCC (Eqs. 1, 8), the
 * multi-hypothesis joint view selection (Eqs. 2-6), the weighted best
 * hypothesis (Eq. 7) and refinement (Sec. 3.3).  After color 1, t advances. */
AMH_API int amh_step_phase(amh_ctx* ctx, int32_t color);

/* k full iterations (black phase then red phase each). */
AMH_API int amh_iterate(amh_ctx* ctx, int32_t k);

/* Copy the state out / in (see amh_state). */
AMH_API int amh_get_state(amh_ctx* ctx, amh_state* out, int32_t mem);
AMH_API int amh_set_state(amh_ctx* ctx, const amh_state* in, int32_t mem);

/* Read back the depth map (D), normals (3 floats per pixel), the cost and the
 * selected-view masks (wmask).  Any pointer may be NULL. */
AMH_API int amh_read_maps(amh_ctx* ctx, float* depth, float* normal3, float* cost,
                          uint32_t* selected, int32_t mem);

/* ------------------------------------------------------------------------
 * Batched form.  The paper computes "the depth map for every reference image
 * in turn" (Sec. 3, overview figure); here several references -- each with
 * its own source list and its own image size -- are resident together and
 * every colour phase of all of them is one persistent launch.  Reference r of
 * a batch draws its random numbers with the key seed + r, so it reproduces a
 * single-reference context created with that seed bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct amh_batch amh_batch;

/* refs[0..n_refs-1] index cams/images (1..256 references); the sources of
 * reference r are src_lists[src_offsets[r] .. src_offsets[r+1]-1]
 * (src_offsets[0] = 0, 1..32 per reference, none equal to refs[r]).  Every
 * view used is uploaded once (texture + linear copy).  stream NULL: the batch
 * creates its own stream (CUDA graphs cannot be captured on the legacy
 * default stream). */
AMH_API int amh_batch_create(amh_batch** out, const amh_params* params, int32_t n_views,
                             const amh_camera* cams, const uint8_t* const* images,
                             int32_t images_mem, int32_t n_refs, const int32_t* refs,
                             const int32_t* src_offsets, const int32_t* src_lists,
                             void* stream);
/* random initialisation of every reference (one launch; see amh_init_random) */
AMH_API int amh_batch_init_random(amh_batch* batch);
/* one colour phase of every reference (one persistent launch) */
AMH_API int amh_batch_step_phase(amh_batch* batch, int32_t color);
/* k iterations (2 launches each) */
AMH_API int amh_batch_iterate(amh_batch* batch, int32_t k);
/* initialisation + iters iterations replayed from a CUDA graph; the graph is
 * captured on the first call for a given iters / tile variant and reused. */
AMH_API int amh_batch_run(amh_batch* batch, int32_t iters);
/* Variant of the phase kernel: the block's tile and each warp's pixel
 * layout (a warp updates 32 pixels of one colour, laid out in its own
 * sub-tile of the block's tile; the layout sets how far apart its lanes'
 * windows fall in every source view):
 *   0: 16 x 16 tile, warps of 8 x 4 pixels of the colour (16 x 4 pixels)
 *   1: 32 x 8 tile,  warps of 16 x 2 (32 x 2 pixels)
 *   2: 64 x 4 tile,  warps of 32 x 1 (64 x 1 pixels)
 *   3: 16 x 16 tile, warps of 4 x 8 (8 x 8 pixels)
 *   4: 32 x 8 tile,  warps of 8 x 4 (16 x 4 pixels)
 * Results do not depend on the variant. */
#define AMH_BATCH_VARIANTS 5
AMH_API int amh_batch_set_variant(amh_batch* batch, int32_t variant);
/* Times initialisation + iters iterations with each variant on this batch
 * and keeps the fastest; *chosen gets its index and ms_out[0 ..
 * AMH_BATCH_VARIANTS - 1] (may be NULL) the times.  The state afterwards is
 * a tuning run: initialise again before use. */
AMH_API int amh_batch_autotune(amh_batch* batch, int32_t iters, int32_t* chosen, float* ms_out);
/* size and number of sources of reference r; *n_refs the batch size */
AMH_API int amh_batch_info(const amh_batch* batch, int32_t r, int32_t* width, int32_t* height,
                           int32_t* n_src, int32_t* n_refs);
/* state of reference r (see amh_state) */
AMH_API int amh_batch_get_state(amh_batch* batch, int32_t r, amh_state* out, int32_t mem);
/* (hypothesis, view) evaluations since the last reset (see amh_pair_count) */
AMH_API int amh_batch_pair_count(amh_batch* batch, uint64_t* count, int32_t reset);
AMH_API int amh_batch_synchronize(amh_batch* batch);
AMH_API const char* amh_batch_last_error(const amh_batch* batch);
AMH_API void amh_batch_destroy(amh_batch* batch);


/* ------------------------------------------------------------------------
 * Learned proposal (this project's extension; the paper trains no network
 * and proposes planes only by propagation (Sec. 3.1) and refinement
 * (Sec. 3.4)).  A 4-level convolutional encoder-decoder (3x3 convolutions
 * 16-32-64-96-128 channels, 2x2 average pooling, nearest upsampling,
 * additive skips; BF16 weights and activations, FP32 accumulation on tensor
 * cores) reads a context's state on the half-resolution grid (X, Y) =
 * (x/2, y/2) -- intensity, log depth, normal and cost of pixel (2X, 2Y) --
 * and predicts the residuals (log-depth change, normal change) towards the
 * converged plane.  amh_net_propose hands the predicted plane of each 2 x 2
 * block to the context: its phases then score it with the unchanged
 * matching cost (Eq. 8) under the pixel's view weights (Eqs. 2-7) as one
 * more refinement candidate (winning choice code 15), so the plain method
 * stays the arbiter.  Training runs on the same kernels: amh_net_features
 * (inputs) -> more plain iterations -> amh_net_targets -> amh_net_forward
 * -> amh_net_backward (L1 loss, every gradient) -> amh_net_adam.
 *
 * Layouts: features height2 x width2 x 16 floats (6 used); outputs height2
 * x width2 x 16 floats (4 used); targets height2 x width2 x 4 floats plus a
 * uint8 mask; weights of layer L (0..7 = e1 e2 e3 e4 d3 d2 d1 out) 9 x Cout
 * x Cin floats, tap 3 (dy + 1) + (dx + 1), biases Cout floats.  Host
 * buffers are the caller's.  Calls run on the stream given at creation;
 * those that return host data synchronise it.  Errors: AMH_EINVAL for NULL
 * handles / buffers, an unknown layer or a context larger than the network;
 * AMH_ENOMEM / AMH_ECUDA from the runtime, with amh_net_last_error.
 * ------------------------------------------------------------------------ */
typedef struct amh_net amh_net;

/* Network for half-resolution inputs of width2 x height2 (positive
 * multiples of 8, at most 2^24 pixels); a W x H reference needs at least
 * ceil(W/2) x ceil(H/2).  He-normal weights drawn from the seed (output
 * layer scaled by 0.1), zero biases, zero Adam moments. */
AMH_API int amh_net_create(amh_net** out, int32_t width2, int32_t height2, uint64_t seed,
                           void* stream);
/* FP32 master weights w and biases b of one layer: read into the host
 * buffers (set = 0) or written from them (set != 0; either may be NULL). */
AMH_API int amh_net_params(amh_net* net, int32_t layer, float* w, float* b, int32_t set);
/* Weight and bias gradients of the last amh_net_backward, same layout. */
AMH_API int amh_net_grads(amh_net* net, int32_t layer, float* gw, float* gb);
/* Features from host memory (stored as BF16). */
AMH_API int amh_net_set_input(amh_net* net, const float* x0);
/* One training example in a single call, from host or device memory (mem:
 * AMH_MEM_HOST / AMH_MEM_DEVICE): features x (h2, w2, channels) FP32,
 * channels 1..16 (the rest are zero; stored as BF16), targets (h2, w2, 4)
 * FP32 and mask (h2, w2) u8, the layouts amh_net_features /
 * amh_net_targets produce.  mirror bit 0 mirrors the example along x
 * (columns reversed, the normal's x negated: feature 2 and target 1), bit 1
 * along y (rows reversed, feature 3 and target 2): the augmentation of
 * training.  The mirroring, padding and conversion run on the device; host
 * inputs are copied first.  The call does not synchronise; the inputs must
 * stay valid until the network's stream reaches it.  Errors: AMH_EINVAL for
 * NULL pointers, channels outside 1..16 or a bad memory kind. */
AMH_API int amh_net_set_example(amh_net* net, const float* x, int32_t channels, const float* target,
                                const uint8_t* mask, int32_t mirror, int32_t mem);
/* Features from the context's current state; also keeps that state's planes
 * as the base the outputs are residuals of. */
AMH_API int amh_net_features(amh_net* net, amh_ctx* ctx);
/* Targets: the context's current planes minus the kept base planes, where
 * the current cost is below cost_max (mask 1), else 0 (mask 0). */
AMH_API int amh_net_targets(amh_net* net, amh_ctx* ctx, float cost_max);
/* Targets and mask from host memory. */
AMH_API int amh_net_set_targets(amh_net* net, const float* target, const uint8_t* mask);
/* Forward pass; out (may be NULL) receives the outputs. */
AMH_API int amh_net_forward(amh_net* net, float* out);
/* L1 loss of the last forward against the targets (sum over the 4 used
 * channels, mean over masked pixels) into *loss (may be NULL), and every
 * weight and bias gradient. */
AMH_API int amh_net_backward(amh_net* net, float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. */
AMH_API int amh_net_adam(amh_net* net, float lr);
/* Proposals from the last forward for the context's following phases; the
 * network must outlive their use (or call amh_clear_proposal first). */
AMH_API int amh_net_propose(amh_net* net, amh_ctx* ctx);
/* Stop scoring proposals in the context. */
AMH_API int amh_clear_proposal(amh_ctx* ctx);
/* Proposals from any source (another network, a prior reconstruction): one
 * plane per cell of a width2 x height2 grid, cell (X, Y) serving the pixels
 * (2X .. 2X+1, 2Y .. 2Y+1) (cells past the grid's edge repeat its last row /
 * column; width2 = ceil(W/2), height2 = ceil(H/2) covers the image).  Layout
 * height2 x width2 x 4 floats (nx, ny, nz, d): the plane n . X + d = 0 in
 * reference-camera coordinates, n facing the camera.  At each pixel it is
 * scored like amh_net_propose's planes (one more refinement candidate under
 * the pixel's view weights, winning choice code 15; not under the
 * AMH_FLAG_HEURISTIC_VIEWS ablation, which has no view weights); a cell with d <= 0, or
 * whose plane does not meet the pixel's ray in front of the camera, proposes
 * nothing.  The planes are copied (mem: AMH_MEM_HOST or AMH_MEM_DEVICE) on
 * the context's stream into a buffer the context owns; they stay in use
 * until amh_clear_proposal, another amh_set_proposal or amh_net_propose.
 * Errors: AMH_EINVAL for a NULL context / buffer, an empty grid or a bad mem;
 * AMH_ENOMEM / AMH_ECUDA from the runtime. */
AMH_API int amh_set_proposal(amh_ctx* ctx, const float* plane4, int32_t width2, int32_t height2,
                             int32_t mem);
/* Internal tensors, for element-wise checks of every operation: which =
 * 0..17 the forward tensors x0 e1 in_e2 e2 in_e3 e3 in_e4 e4 in_d3 r3 d3
 * in_d2 r2 d2 in_d1 r1 d1 out (in_* = pooled / upsampled inputs, r* = a
 * decoder layer's ReLU output before its skip; BF16 ones widened to FP32),
 * 32 + L the gradient at layer L's output after its ReLU mask (FP32, from the
 * last amh_net_backward).  Layout (H, W, C) of that level.  which = 64: the
 * targets (h2, w2, 4); 65: the mask (h2, w2) as 0 / 1.  With out = NULL the
 * element count is written to *count; otherwise *count must equal it. */
AMH_API int amh_net_read(amh_net* net, int32_t which, float* out, int64_t* count);
/* Wait for the network's work. */
AMH_API int amh_net_synchronize(amh_net* net);
/* Message of the last failure (NULL net: of the last failed create). */
AMH_API const char* amh_net_last_error(const amh_net* net);
/* Free everything; NULL is allowed. */
AMH_API void amh_net_destroy(amh_net* net);

#define AMH_NOALLOC_MAX_PIXELS 262144

/* amh_read_maps without any allocation (the paper has no counterpart: this
 * is a service for callers that cannot allocate device memory when they read
 * results -- hosts whose pooling allocator owns the GPU and forbids any other
 * device allocation, and loops that must not allocate after start-up, where
 * amh_read_maps with host buffers would allocate a staging buffer per call).
 * It is a plain blocking read: it synchronises the context's stream and copies
 * into pageable host memory, so it must be called outside stream capture.
 *
 * Copies the depth (float per pixel) and/or the normal (3 floats per pixel)
 * of the pixels [first_pixel, first_pixel + n_pixels) in row-major order into
 * HOST buffers of n_pixels (depth) and 3 * n_pixels (normal3) floats; either
 * may be NULL, not both.  At most AMH_NOALLOC_MAX_PIXELS pixels per call
 * (read larger maps in slices); more, or a range outside the image, returns
 * AMH_EINVAL with a message and touches nothing.
 *
 * The data is staged through one fixed scratch array that is part of the
 * library's device image (4 MB, held on every GPU that loads the library
 * until the process exits); the call itself makes no cudaMalloc/cudaFree or
 * other allocating call.  The first call on a device looks up the array's
 * device address (once per device, on the device the context was created
 * on); that first call may also load the library's kernels onto the device,
 * which the CUDA runtime does lazily and which can reserve device memory of
 * its own.  Every call on a device shares the one array: calls whose GPU work
 * can overlap (other streams, other host threads) race on it, so serialise
 * them.  The call synchronises the context's stream before it returns. */
AMH_API int amh_read_maps_noalloc(amh_ctx* ctx, float* depth, float* normal3,
                                  int64_t first_pixel, int64_t n_pixels);

/* ------------------------------------------------------------------------
 * Post-processing of depth maps (Sec. 3.3, last two paragraphs; the details
 * follow Gipuma, the paper's reference [9], under these readings).  Both
 * calls take DEVICE buffers the caller owns and run asynchronously on
 * `stream`; errors: AMH_EINVAL for NULL / aliased buffers or bad sizes,
 * AMH_ECUDA for a failed launch, each with a message in amh_last_error(NULL).
 * ------------------------------------------------------------------------ */
/* 4x4 median of a width x height depth map: the window holds the offsets
 * -2..+1 in x and y (clamped at the borders), the value is the mean of its
 * 8th and 9th smallest entries (exact to FP32 rounding).  depth_in and
 * depth_out must differ. */
AMH_API int amh_median4(const float* depth_in, float* depth_out, int32_t width, int32_t height, void* stream);
/* Consistency fusion of n_views (2..32) depth maps: depth[v] (W_v x H_v
 * z-depths, <= 0 = none) and normal3[v] (W_v x H_v x 3, view v's camera
 * coordinates) of camera cams[v] (host array of device pointers).  Pixel p of
 * view i back-projects to the world point X with world normal n; view j
 * agrees when X lies in front of it and projects to the pixel q = (floor(u +
 * 0.5), floor(v + 0.5)) inside it with depth D_j(q) > 0, the disparity
 * difference f_j |C_i - C_j| |1/z_j(X) - 1/D_j(q)| (f_j = K_j[0], C the camera
 * centres, z_j(X) the depth of X in view j) is at most f_eps, and the angle
 * between n and view j's normal at q is at most f_ang_deg.  count[v] (W_v x
 * H_v uint8) receives the number of agreeing views; where it reaches f_con,
 * points6[v] (W_v x H_v x 6 floats) receives the mean of X and the agreeing
 * views' back-projected points and the normalised sum of the normals (world
 * coordinates), else zeros.  The paper fixes f_eps 0.3, f_ang 30, f_con 2. */
AMH_API int amh_fuse(int32_t n_views, const amh_camera* cams, const float* const* depth,
                     const float* const* normal3, float f_eps, float f_ang_deg, int32_t f_con,
                     float* const* points6, uint8_t* const* count, void* stream);

/* Source-view preselection (Sec. 2 / Sec. 4: the N source views are chosen
 * "according to viewing angle and baseline"; host-only, no GPU needed).
 * Reading: P is the point at z-depth `depth` on the reference's optical
 * axis; a view qualifies when P lies in front of it and projects inside its
 * image, and the triangulation angle between the rays from P to the two
 * camera centres lies in [min_angle_deg, max_angle_deg] (the lower bound asks
 * for baseline, the upper for similar appearance).  Qualifying views are
 * ranked by increasing angle (ties: lower index); the first n_src go to
 * src_out (capacity n_src), their number to *n_out.  AMH_EINVAL for a bad
 * reference, non-positive depth, n_src < 1 or an empty angle range. */
AMH_API int amh_select_sources(int32_t n_views, const amh_camera* cams, int32_t ref, double depth,
                               int32_t n_src, double min_angle_deg, double max_angle_deg,
                               int32_t* src_out, int32_t* n_out);

/* The texture-gather ceiling of the current GPU, measured (this project's
 * measurement utility, not part of the method): a loop of nothing but 2x2
 * gathers of a uint8 texture laid out like the update's windows, 16 warps per
 * SM; *samples_per_s receives gathers per second (one gather serves one
 * window sample of Eq. (8)).  Synchronises the device; allocates and frees
 * its own buffers. */
AMH_API int amh_gather_peak(double* samples_per_s);

/* Reference size, number of sources, current t. */
AMH_API int amh_get_info(const amh_ctx* ctx, int32_t* width, int32_t* height,
                         int32_t* n_src, int32_t* t);

/* Number of (hypothesis, view) cost evaluations the kernels have performed
 * since the last reset (each is one 36-sample warped bilateral NCC).  The
 * count is kept on the device; reading it synchronises the stream. */
AMH_API int amh_pair_count(amh_ctx* ctx, uint64_t* count, int32_t reset);
/* The same count (total, may be NULL) and, of those, the evaluations whose 36
 * samples were read from a shared-memory box instead of the texture unit
 * (staged, may be NULL; see AMH_FLAG_STAGED_FETCH).  reset clears both. */
AMH_API int amh_pair_counts(amh_ctx* ctx, uint64_t* total, uint64_t* staged, int32_t reset);

/* Wait for all work of the context; reports kernel status errors. */
AMH_API int amh_synchronize(amh_ctx* ctx);

/* Message of the last failure (never NULL). */
AMH_API const char* amh_last_error(const amh_ctx* ctx);

/* Free everything; NULL is allowed. */
AMH_API void amh_destroy(amh_ctx* ctx);

/* 1 in a bounds-checked build of the library (compiled with
 * -DAMH_BOUNDS_CHECK), else 0.  There every index the update computes into
 * the state, the reference image or the proposals is checked; an index out
 * of range is replaced by 0 and recorded in the context's (or batch's)
 * status word, and amh_synchronize / amh_batch_synchronize return
 * AMH_EDEVICE with the status in amh_last_error.  Results are otherwise the
 * same as the normal build's. */
AMH_API int amh_bounds_checked(void);

#ifdef __cplusplus
}
#endif
#endif /* AMH_H */
