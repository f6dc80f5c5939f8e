// amh_conv_tc.cuh -- 3x3 convolution (stride 1, zero padding) of the learned
// proposal network on the fifth-generation tensor cores: tcgen05.mma with the
// FP32 accumulator in tensor memory, BF16 operands brought into shared memory
// by the tensor memory accelerator (cp.async.bulk.tensor).
//
// Implicit GEMM: D (128 pixels x Cout) = sum over the 9 taps t and the input
// channels ci of X (pixel + off(t), ci) W (t, co, ci).  A CTA owns 128
// consecutive pixels of one row and every output channel; one K step is one
// tap and 16 input channels.  Per step, four TMA boxes land in a stage of the
// shared-memory ring: the activations of the 128 pixels shifted by the tap
// (two boxes of 8 channels; rows or columns outside the image read as zeros,
// which is the convolution's padding) and the tap's weights (two boxes of 8
// channels x Cout).  Each box is 16 bytes per row, so a stage holds both
// operands in the tensor cores' K-major layout without swizzling: 8 x 16-byte
// core matrices, 128 bytes apart along M / N, the second 8 channels 2048
// bytes after the first.  A producer warp keeps the ring full, an MMA warp
// consumes it and recycles each stage once the MMA that read it has
// committed, and the epilogue warps read the accumulator with tcgen05.ld and
// apply bias, ReLU, skip addition and the BF16 / FP32 stores.
//
// Layout: activations (H, W, C) BF16 with C a multiple of 16; weights (9,
// Cout, Cin) BF16, tap t = 3 (dy + 1) + (dx + 1); Cout a multiple of 16, at
// most 128.  Every wait on a barrier gives up after a bounded number of
// tries and sets the status word instead of hanging.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace amh {
namespace tc {

constexpr int kM = 128;          // pixels per CTA (rows of the accumulator)
constexpr int kStages = 6;       // shared-memory ring
constexpr int kMaxCout = 128;
constexpr uint32_t kWaitTries = 1u << 24;

// one ring stage: the activation and weight boxes of one K step, each as two
// halves of 8 channels x 16 bytes per row
struct alignas(1024) Stage {
  uint8_t a[2][kM * 16];
  uint8_t b[2][kMaxCout * 16];
};
constexpr size_t kSmemBytes = kStages * sizeof(Stage) + 1024;   // + alignment slack

struct ConvTcArgs {
  const float* bias;          // Cout or null
  const __nv_bfloat16* skip;  // (H, W, Cout) added after the ReLU, or null
  __nv_bfloat16* y16;         // (H, W, Cout) BF16 output (after ReLU + skip), or null
  __nv_bfloat16* r16;         // (H, W, Cout) ReLU output before the skip, or null
  float* y32;                 // (H, W, Cout) FP32 output, or null
  unsigned int* status;       // bit 0: a barrier wait gave up
  int H, W, Cin, Cout, relu;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// true once the barrier's phase with the given parity has completed; false
// after kWaitTries unsuccessful tries
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitTries && !done; it++) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
  }
  return done != 0;
}
// TMA: one box of a 3-D tensor into shared memory, completion counted on bar
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor, K-major, no swizzle: start address,
// leading byte offset (between the two 8-element core matrices along K),
// stride byte offset (between 8-row groups along M / N), descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Persistent, warp-specialised: warps 0-3 drain the accumulator (warp w owns
// TMEM lanes 32 w .. 32 w + 31, i.e. pixels 32 w .. 32 w + 31 of the tile),
// warp 4 produces (TMA into the ring), warp 5 allocates the tensor memory and
// issues the MMAs.  Two accumulators in tensor memory let the epilogue of one
// tile overlap the MMAs of the next.  The CTA walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; tile = (row y, 128-pixel segment).
constexpr int kThreads = 192;

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__global__ void __launch_bounds__(kThreads) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tx,
                                                              const __grid_constant__ CUtensorMap tw,
                                                              const ConvTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  Stage* st = reinterpret_cast<Stage*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nc = a.Cin / 16, nk = 9 * nc;
  const int nseg = (a.W + kM - 1) / kM, ntiles = a.H * nseg;
  const uint32_t ncols = a.Cout <= 32 ? 32u : a.Cout <= 64 ? 64u : 128u;   // one accumulator

  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);    // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == 4) {
    // producer: a stage is refilled once the MMA that read it has committed
    if (lane == 0) {
      const uint32_t bytes = 2u * kM * 16u + 2u * (uint32_t)a.Cout * 16u;
      uint32_t g = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int y = tile / nseg, x0 = (tile % nseg) * kM;
        for (int k = 0; k < nk && ok; k++, g++) {
          const int s = (int)(g % kStages);
          if (!(ok = mbar_wait(&empty[s], ((g / kStages) & 1u) ^ 1u))) break;
          const int t = k / nc, ci0 = (k % nc) * 16, dy = t / 3 - 1, dx = t % 3 - 1;
          mbar_expect_tx(&full[s], bytes);
#pragma unroll
          for (int h = 0; h < 2; h++) {
            tma_load_3d(st[s].a[h], &tx, ci0 + 8 * h, x0 + dx, y + dy, &full[s]);
            tma_load_3d(st[s].b[h], &tw, ci0 + 8 * h, 0, t, &full[s]);
          }
        }
      }
    }
  } else if (warp == 5) {
    // MMA issuer: K steps of a tile accumulate in buffer i % 2
    if (lane == 0) {
      const uint32_t idesc = mma_idesc(kM, a.Cout);
      uint32_t g = 0, i = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, i++) {
        const uint32_t b = i & 1u;
        if (!(ok = mbar_wait(&acc_empty[b], ((i >> 1) & 1u) ^ 1u))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + b * ncols;
        for (int k = 0; k < nk; k++, g++) {
          const int s = (int)(g % kStages);
          if (!(ok = mbar_wait(&full[s], (g / kStages) & 1u))) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          mma_bf16(d, smem_desc(smem_u32(st[s].a[0]), kM * 16, 128), smem_desc(smem_u32(st[s].b[0]), kMaxCout * 16, 128),
                   idesc, k > 0 ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[b]);
      }
    }
  } else {
    // epilogue: warp w drains TMEM lanes 32 w .. 32 w + 31 of each tile
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, i++) {
      const uint32_t b = i & 1u;
      if (!(ok = mbar_wait(&acc_full[b], (i >> 1) & 1u))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int y = tile / nseg, x0 = (tile % nseg) * kM;
      const int r = warp * 32 + lane, px = x0 + r;
      const size_t o0 = ((size_t)y * a.W + px) * a.Cout;
      for (int c0 = 0; c0 < a.Cout; c0 += 8) {
        uint32_t v[8];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
            : "r"(tmem + b * ncols + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (px >= a.W) continue;
        const size_t o = o0 + c0;
        float f[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
          const float val = __uint_as_float(v[e]) + (a.bias ? a.bias[c0 + e] : 0.f);
          f[e] = a.relu ? fmaxf(val, 0.f) : val;
        }
        __align__(16) __nv_bfloat16 hb[8];
        if (a.r16) {
#pragma unroll
          for (int e = 0; e < 8; e++) hb[e] = __float2bfloat16(f[e]);
          *reinterpret_cast<uint4*>(a.r16 + o) = *reinterpret_cast<const uint4*>(hb);
        }
        if (a.skip) {
          __align__(16) __nv_bfloat16 sk[8];
          *reinterpret_cast<uint4*>(sk) = *reinterpret_cast<const uint4*>(a.skip + o);
#pragma unroll
          for (int e = 0; e < 8; e++) f[e] = __bfloat162float(__float2bfloat16(f[e])) + __bfloat162float(sk[e]);
        }
        if (a.y16) {
#pragma unroll
          for (int e = 0; e < 8; e++) hb[e] = __float2bfloat16(f[e]);
          *reinterpret_cast<uint4*>(a.y16 + o) = *reinterpret_cast<const uint4*>(hb);
        }
        if (a.y32) {
          reinterpret_cast<float4*>(a.y32 + o)[0] = make_float4(f[0], f[1], f[2], f[3]);
          reinterpret_cast<float4*>(a.y32 + o)[1] = make_float4(f[4], f[5], f[6], f[7]);
        }
      }
      // this warp's lanes of buffer b may be overwritten by the next tile's MMAs
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  if (!ok && (lane == 0)) atomicOr(a.status, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ncols));
  }
}

// Weight gradient of a 3x3 convolution on the tensor cores:
// dW (t, co, ci) = sum over pixels p of dy (p, co) x (p + off(t), ci), one
// tap per blockIdx.y and a band of rows per blockIdx.x, as a GEMM with M =
// Cout (the accumulator's rows; rows past Cout are left over and ignored), N
// = Cin and K = the band's pixels, 16 per step.  The operands come
// transposed, channel-major: dyT (Cout, H, Wp) and three copies of x,
// xT_s (Cin, H, Wp) with xT_s (c, y, x) = x (y, x + s, c) for s = -1, 0, 1
// (zero where x + s leaves the row), BF16, rows padded to Wp (a multiple of
// 8).  A K step is two TMA boxes of 8 pixels x the channels per operand, in
// the same K-major layout as the forward kernel.  The tap's column offset is
// taken by the copy xT_dx, so every box starts at a pixel index that is a
// multiple of 8 (a TMA box must start on a 16-byte boundary in its innermost
// dimension); its row offset shifts the box's row coordinate, and rows
// outside the image read zeros, as do pixels past the row's end.  The band's
// sum is added into dw (FP32) by the epilogue warps.
struct WgradTcArgs {
  float* dw;                 // (9, Cout, Cin), accumulated into
  unsigned int* status;      // bit 0: a barrier wait gave up
  int H, W, Cin, Cout, rows_per_band;
};

__global__ void __launch_bounds__(kThreads) wgrad3x3_tc_kernel(const __grid_constant__ CUtensorMap tdy,
                                                               const __grid_constant__ CUtensorMap tx_m1,
                                                               const __grid_constant__ CUtensorMap tx_0,
                                                               const __grid_constant__ CUtensorMap tx_p1,
                                                               const WgradTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  Stage* st = reinterpret_cast<Stage*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t = blockIdx.y, dy = t / 3 - 1, dx = t % 3 - 1;
  const int y0 = blockIdx.x * a.rows_per_band, y1 = min(a.H, y0 + a.rows_per_band);
  const int nseg = (a.W + 15) / 16, nk = (y1 > y0 ? y1 - y0 : 0) * nseg;
  const uint32_t ncols = a.Cin <= 32 ? 32u : a.Cin <= 64 ? 64u : 128u;

  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == 4) {
    if (lane == 0) {
      const uint32_t bytes = 2u * (uint32_t)(a.Cout + a.Cin) * 16u;
      const CUtensorMap* tx = dx < 0 ? &tx_m1 : dx > 0 ? &tx_p1 : &tx_0;
      for (int k = 0; k < nk && ok; k++) {
        const int s = k % kStages;
        if (!(ok = mbar_wait(&empty[s], ((uint32_t)(k / kStages) & 1u) ^ 1u))) break;
        const int y = y0 + k / nseg, x0 = (k % nseg) * 16;
        mbar_expect_tx(&full[s], bytes);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          tma_load_3d(st[s].a[h], &tdy, x0 + 8 * h, y, 0, &full[s]);
          tma_load_3d(st[s].b[h], tx, x0 + 8 * h, y + dy, 0, &full[s]);
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = mma_idesc(kM, a.Cin);
      for (int k = 0; k < nk && ok; k++) {
        const int s = k % kStages;
        if (!(ok = mbar_wait(&full[s], (uint32_t)(k / kStages) & 1u))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        mma_bf16(tmem, smem_desc(smem_u32(st[s].a[0]), kM * 16, 128), smem_desc(smem_u32(st[s].b[0]), kMaxCout * 16, 128),
                 idesc, k > 0 ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&acc_full);
    }
  } else if (nk > 0) {
    if ((ok = mbar_wait(&acc_full, 0))) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int co = warp * 32 + lane;
      for (int c0 = 0; c0 < a.Cin; c0 += 8) {
        uint32_t v[8];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (co >= a.Cout) continue;
        float* d = a.dw + ((size_t)t * a.Cout + co) * a.Cin + c0;
#pragma unroll
        for (int e = 0; e < 8; e++) atomicAdd(d + e, __uint_as_float(v[e]));
      }
    }
  }
  if (!ok && lane == 0) atomicOr(a.status, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

// (P, C) -> (C, H, Wp) BF16 transpose of an activation or gradient map (P = H
// W pixels; rows padded to Wp), shifted along the row by `shift`:
// out (c, y, x) = in (y, x + shift, c), zero where x + shift leaves the row
__global__ void __launch_bounds__(256) to_channel_major_kernel(const __nv_bfloat16* __restrict__ in,
                                                               __nv_bfloat16* __restrict__ out, int H, int W, int Wp,
                                                               int C, int shift) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32, P = H * W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int p = p0 + r, c = c0 + tx;
    tile[r][tx] = (p < P && c < C) ? in[(size_t)p * C + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, p = p0 + tx;
    if (c >= C || p >= P) continue;
    // the output pixel whose shifted source is pixel p, and the row ends the
    // shift uncovers
    const int y = p / W, x = p % W - shift;
    if (x >= 0 && x < W) out[((size_t)c * H + y) * Wp + x] = tile[tx][r];
    if (shift > 0 && p % W == 0) out[((size_t)c * H + y) * Wp + W - 1] = __float2bfloat16(0.f);
    if (shift < 0 && p % W == W - 1) out[((size_t)c * H + y) * Wp + 0] = __float2bfloat16(0.f);
  }
}

// CTAs of conv3x3_tc_kernel that fit on one SM: the shared-memory ring and
// the tensor memory (512 columns, two accumulators per CTA) both bound it
__host__ __device__ constexpr int ctas_per_sm(int cout) {
  const int cols = 2 * (cout <= 32 ? 32 : cout <= 64 ? 64 : 128);
  const int by_tmem = 512 / cols, by_smem = (int)((228u * 1024u) / (kSmemBytes + 1024u));
  return by_tmem < by_smem ? by_tmem : by_smem;
}

}  // namespace tc
}  // namespace amh
