// amh_conv_tc.cuh -- 3x3 convolution (stride 1, zero padding) of the learned
// proposal network on the fifth-generation tensor cores: tcgen05.mma with the
// FP32 accumulator in tensor memory, BF16 operands brought into shared memory
// by the tensor memory accelerator (cp.async.bulk.tensor).
//
// Implicit GEMM: D (pixels x Cout) = sum over the 9 taps t and the input
// channels ci of X (pixel + off(t), ci) W (t, co, ci), one MMA per tap and 16
// input channels (M = 128 pixels of one row, N = a block of output channels,
// K = 16).  Both operands sit in shared memory in the tensor cores' K-major
// layout, in blocks of 64 channels (128-byte rows, 128-byte swizzle; a 16- or
// 32-channel remainder in 32- or 64-byte rows).  The forward / data-gradient
// kernel keeps its block of weights resident and streams input rows with a
// one-pixel halo, each row loaded once per run of vertically adjacent tiles
// (its comment below gives the schedule); the weight-gradient kernel streams
// 64-pixel chunks of the same pixel-major tensors as MN-major operands.  A
// producer warp issues the TMA copies, an MMA warp consumes them and recycles
// each buffer once the MMAs that read it have committed, and the epilogue
// warps read the accumulator with tcgen05.ld and apply bias, ReLU, skip
// addition and the BF16 / FP32 stores.
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
constexpr int kMaxCout = 128;
constexpr uint32_t kWaitTries = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// true once the barrier's phase with the given parity has completed; false
// after kWaitTries unsuccessful tries.  A waiter that is not on the critical
// path passes sleep_ns, so that between tries it leaves the issue slots of its
// SM sub-partition to the warps that are.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint32_t sleep_ns = 0) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitTries; it++) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (done) break;
    if (sleep_ns) __nanosleep(sleep_ns);
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
// Shared-memory matrix descriptor of a tcgen05 operand, as two 32-bit words.
// Low word: start address >> 4 (bits 0-13) and the leading byte offset >> 4
// (bits 16-29; ignored for swizzled K-major operands, set to 16 bytes;
// for MN-major operands the step between blocks along M / N, see
// desc_lo_mn).  High word: the stride byte offset >> 4 (between 8-row groups:
// along M / N for K-major, along K for MN-major; 8 rows of `pitch` bytes
// either way), descriptor version 1 (bit 46 of the whole), base offset 0 and
// the layout in bits 61-63 (2, 4, 6: rows of 128, 64, 32 bytes with the
// matching swizzle).  The swizzle pattern follows the shared-memory address
// bits, so a start moved by whole rows stays consistent with what the TMA
// wrote.  The low word moves with the operand; the high word is fixed per
// channel block.
__host__ __device__ constexpr uint32_t swizzle_layout(int pitch) { return pitch == 128 ? 2u : pitch == 64 ? 4u : 6u; }
__device__ __forceinline__ uint32_t desc_lo(uint32_t addr) { return ((addr >> 4) & 0x3FFFu) | (1u << 16); }
__device__ __forceinline__ uint32_t desc_hi(uint32_t pitch) {
  return ((8u * pitch) >> 4) | (1u << 14) | (swizzle_layout((int)pitch) << 29);
}
__device__ __forceinline__ uint64_t desc_pack(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; }

// position in a ring of S buffers: the slot and the parity of its current use
struct RingPos {
  uint32_t slot, phase;
  __device__ __forceinline__ RingPos next(uint32_t S) const {
    return slot + 1 == S ? RingPos{0u, phase ^ 1u} : RingPos{slot + 1, phase};
  }
};
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// The MMA warps run their issue loops with all 32 lanes converged, so that
// the descriptor arithmetic is warp-uniform; one lane chosen by elect.sync
// (the same lane every time, the warp being converged) issues each MMA and
// each commit.  Measured: 39-48 cycles per M = 128, K = 16 MMA (N <= 64)
// with the descriptors computed in the loop this way, 63-68 cycles when a
// single lane runs the loop.
__device__ __forceinline__ void mma_bf16_elect(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit_elect(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}
// a barrier wait by the whole warp, with one answer for all its lanes
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity) {
  return __all_sync(0xffffffffu, mbar_wait(b, parity));
}
// 16 consecutive accumulator columns of this thread's TMEM lane (the warp
// reads its lane quarter); the caller waits with tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Both kernels are persistent and warp-specialised: epilogue warps drain the
// accumulator (a warp reads the TMEM lanes of its SM sub-partition, lanes
// 32 (w % 4) .. 32 (w % 4) + 31), one warp produces (TMA), one allocates the
// tensor memory and issues the MMAs.  Two accumulators in tensor memory let
// the epilogue of one tile overlap the MMAs of the next.  The weight-gradient
// kernel has 4 epilogue warps (kThreads); the convolution kernel has 4 per
// 16 output channels of its block (conv_threads), so that the chunks of a
// tile drain in parallel.
constexpr int kThreads = 192;

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Store one 32-byte sector per pixel (16 BF16 or 8 FP32 channels, as two
// 16-byte halves lo, hi) for the pixels of lane pairs (2k, 2k + 1), which
// are neighbours, so that each store instruction writes whole sectors: the
// first writes the even pixel's sector (its lo from the even lane, its hi
// from the odd one), the second the odd pixel's.  self / partner point at
// this lane's and the pair partner's sector; st_self / st_partner say
// whether those pixels are stored.  All 32 lanes call it together.
__device__ __forceinline__ void store_sector_pair(uint4* self, uint4* partner, uint4 lo, uint4 hi, bool odd,
                                                  bool st_self, bool st_partner) {
  const uint4 send = odd ? lo : hi;    // the half the partner stores for this lane's pixel
  uint4 recv;
  recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
  recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
  recv.z = __shfl_xor_sync(0xffffffffu, send.z, 1);
  recv.w = __shfl_xor_sync(0xffffffffu, send.w, 1);
  uint4* const pa = odd ? partner + 1 : self;      // the even pixel's sector
  uint4* const pb = odd ? self + 1 : partner;      // the odd pixel's sector
  const uint4 va = odd ? recv : lo, vb = odd ? hi : recv;
  const bool sa = odd ? st_partner : st_self, sb = odd ? st_self : st_partner;
  if (sa) *pa = va;
  if (sb) *pb = vb;
}

// Forward / data-gradient kernel.  A tile is 128 consecutive pixels of one
// output row and one block of Nb output channels; CTA (bx, by) owns channel
// block by and a contiguous range of the tiles ordered (128-pixel column
// segment, row), i.e. runs of vertically adjacent tiles.  Its Nb x Cin x 9
// weights are loaded into shared memory once.  The input enters as slabs:
// one input row, 130 pixels (the tile's 128 and one halo pixel on each side)
// x all Cin channels.  Channels are split into blocks of 64 (128-byte rows)
// and a tail of 16 or 32 (32- or 64-byte rows); each block is one TMA box
// with the swizzle of its row length, 1024-byte aligned, and the weights of
// a tap use the same blocks.  Output row y reads the slabs of input rows
// y - 1, y, y + 1, and the tap (dx, dy) of slab y + dy is the same block seen
// from row 1 + dx: its matrix descriptor starts 1 + dx rows later (the
// swizzle pattern follows the address, so the shifted view reads what the
// TMA wrote).  So each input row of a run is loaded once and feeds
// 9 Cin / 16 MMAs (M = 128, N = Nb, K = 16) for three output rows.  The slabs
// sit in a ring of S stages; slab k is released when output row k + 1 (the
// last one reading it) has committed its MMAs.
constexpr int kHalo = kM + 2;               // pixels per slab row
constexpr int kMaxStages = 8;
constexpr int kConvMaxNb = 64;              // output channels per CTA
// threads of conv3x3_tc_kernel: 4 epilogue warps per 16 output channels of the
// block (one per TMEM lane quarter and 16-channel chunk), the producer and the
// MMA warp
__host__ __device__ constexpr int conv_threads(int nb) { return 32 * (4 * (nb / 16) + 2); }
constexpr int kConvMaxThreads = 32 * (4 * (kConvMaxNb / 16) + 2);

struct ConvTcArgs {
  const float* bias;          // Cout or null
  const __nv_bfloat16* skip;  // (H, W, Cout) added after the ReLU, or null
  __nv_bfloat16* y16;         // (H, W, Cout) BF16 output (after ReLU + skip), or null
  __nv_bfloat16* r16;         // (H, W, Cout) ReLU output before the skip, or null
  float* y32;                 // (H, W, Cout) FP32 output, or null
  unsigned int* status;       // bit 0: a barrier wait gave up
  int H, W, Cin, Cout, relu;
  int Nb;                     // output channels per CTA (a multiple of 16 dividing Cout, at most kConvMaxNb)
  int S;                      // slab stages (3 .. kMaxStages)
};

// channel blocks of a Cin-channel operand: cin / 64 blocks of 64 channels,
// then a tail of cin % 64 (0, 16 or 32) channels; each block's region is
// rows x (2 x its channels) bytes rounded up to 1 KB
__host__ __device__ constexpr size_t round_1k(size_t b) { return (b + 1023) & ~(size_t)1023; }
__host__ __device__ constexpr size_t conv_block_bytes(int cin, int rows) {
  return (size_t)(cin / 64) * round_1k((size_t)rows * 128) + (cin % 64 ? round_1k((size_t)rows * 2 * (cin % 64)) : 0);
}
// dynamic shared memory of conv3x3_tc_kernel: alignment slack, the weights
// (9 taps of Nb rows), the slab ring (rows of kHalo pixels)
__host__ __device__ constexpr size_t conv_wtap_bytes(int cin, int nb) { return conv_block_bytes(cin, nb); }
__host__ __device__ constexpr size_t conv_weight_bytes(int cin, int nb) { return 9 * conv_wtap_bytes(cin, nb); }
__host__ __device__ constexpr size_t conv_slab_bytes(int cin) { return conv_block_bytes(cin, kHalo); }
__host__ __device__ constexpr size_t conv_smem_bytes(int cin, int nb, int s) {
  return 1024 + conv_weight_bytes(cin, nb) + (size_t)s * conv_slab_bytes(cin);
}
// tensor-memory columns of one accumulator (allocations are powers of two >= 32)
__host__ __device__ constexpr uint32_t conv_acc_cols(int nb) { return nb <= 32 ? 32u : nb <= 64 ? 64u : 128u; }

// run r of the CTA's tile range: tiles u .. u + len - 1 of one column segment
struct TileRun {
  int seg, y0, len;
};
__device__ __forceinline__ bool next_run(int& u, int hi, int H, TileRun& r) {
  if (u >= hi) return false;
  r.seg = u / H;
  r.y0 = u % H;
  r.len = min(hi - u, H - r.y0);
  u += r.len;
  return true;
}

// tx_main / tw_main: boxes of 64 channels x (kHalo pixels | Nb output
// channels), 128-byte swizzle; tx_tail / tw_tail: the same for the tail
// channels (unused when Cin is a multiple of 64)
// kPairStores: the epilogue writes whole 32-byte sectors through lane pairs
// (store_sector_pair); it pays where the stores bound the layer (the decoder
// layers with a skip input and two BF16 outputs) and costs registers and
// shuffles elsewhere
template <bool kPairStores>
__global__ void __launch_bounds__(kConvMaxThreads, 1) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tx_main,
                                                              const __grid_constant__ CUtensorMap tx_tail,
                                                              const __grid_constant__ CUtensorMap tw_main,
                                                              const __grid_constant__ CUtensorMap tw_tail,
                                                              const ConvTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* wsm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = a.S, Nb = a.Nb, nmain = a.Cin / 64, tail = a.Cin % 64, nblk = nmain + (tail ? 1 : 0);
  uint8_t* slabs = wsm + conv_weight_bytes(a.Cin, Nb);
  const uint32_t slab_bytes = (uint32_t)conv_slab_bytes(a.Cin), wtap_bytes = (uint32_t)conv_wtap_bytes(a.Cin, Nb);
  // per channel block: byte offset in a slab / a tap's weights
  const uint32_t sblk = (uint32_t)round_1k((size_t)kHalo * 128), wblk = (uint32_t)round_1k((size_t)Nb * 128);
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2], wbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float bias_s[kMaxCout];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int w_prod = 4 * (Nb / 16), w_mma = w_prod + 1;
  const int co0 = blockIdx.y * Nb;
  const int nseg = (a.W + kM - 1) / kM, ntiles = a.H * nseg;
  const int lo = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
  const int hi = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x);
  const uint32_t ncols = conv_acc_cols(Nb);

  if (warp == w_mma) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2 * ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < S; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], (uint32_t)w_prod);    // one arrival per epilogue warp
    }
    mbar_init(&wbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int c = tid; c < Nb; c += (int)blockDim.x) bias_s[c] = a.bias ? a.bias[co0 + c] : 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == w_prod) {
    // producer: the weights once, then the slabs of every run in order
    if (lane == 0) {
      mbar_expect_tx(&wbar, 9u * (uint32_t)Nb * 2u * (uint32_t)a.Cin);
      for (int t = 0; t < 9; t++)
        for (int bk = 0; bk < nblk; bk++)
          tma_load_3d(wsm + (size_t)t * wtap_bytes + (size_t)bk * wblk, bk < nmain ? &tw_main : &tw_tail, 64 * bk, co0, t,
                      &wbar);
      RingPos q{0u, 0u};
      TileRun r;
      for (int u = lo; ok && next_run(u, hi, a.H, r);) {
        const int x0 = r.seg * kM;
        for (int k = 0; k < r.len + 2 && ok; k++, q = q.next((uint32_t)S)) {
          if (!(ok = mbar_wait(&empty[q.slot], q.phase ^ 1u))) break;
          mbar_expect_tx(&full[q.slot], (uint32_t)kHalo * 2u * (uint32_t)a.Cin);
          uint8_t* dst = slabs + (size_t)q.slot * slab_bytes;
          for (int bk = 0; bk < nblk; bk++)
            tma_load_3d(dst + (size_t)bk * sblk, bk < nmain ? &tx_main : &tx_tail, 64 * bk, x0 - 1, r.y0 - 1 + k,
                        &full[q.slot]);
        }
      }
    }
  } else if (warp == w_mma) {
    // MMA issuer: output row i of a run accumulates 9 Cin / 16 MMAs over the
    // slabs i, i + 1, i + 2 of the run into accumulator buffer (tile count % 2)
    {   // all 32 lanes: warp-uniform descriptors, elected issue
      const uint32_t idesc = mma_idesc(kM, Nb);
      const uint32_t hi_main = desc_hi(128u), hi_tail = desc_hi(2u * (uint32_t)tail);
      const uint32_t w_lo = desc_lo(smem_u32(wsm)), s_lo = desc_lo(smem_u32(slabs));
      const uint32_t wtap16 = wtap_bytes >> 4, slab16 = slab_bytes >> 4, sblk16 = sblk >> 4, wblk16 = wblk >> 4;
      const uint32_t tail16 = (2u * (uint32_t)tail) >> 4;      // the tail's row pitch, in 16-byte units
      ok = mbar_wait_warp(&wbar, 0);
      uint32_t tc = 0;
      RingPos q{0u, 0u};    // ring position of the next slab
      TileRun r;
      for (int u = lo; ok && next_run(u, hi, a.H, r);) {
        RingPos q0 = q, q1 = q.next((uint32_t)S);    // slabs i and i + 1 of the run
        for (int i = 0; i < r.len && ok; i++, tc++) {
          const uint32_t b = tc & 1u;
          const RingPos q2 = q1.next((uint32_t)S);
          if (!(ok = mbar_wait_warp(&acc_empty[b], ((tc >> 1) & 1u) ^ 1u))) break;
          if (i == 0) ok = mbar_wait_warp(&full[q0.slot], q0.phase) && mbar_wait_warp(&full[q1.slot], q1.phase);
          if (!(ok = ok && mbar_wait_warp(&full[q2.slot], q2.phase))) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + b * ncols;
          uint32_t acc = 0;
#pragma unroll
          for (int dy = 0; dy < 3; dy++) {
            const uint32_t slot = dy == 0 ? q0.slot : dy == 1 ? q1.slot : q2.slot;
            const uint32_t xs = s_lo + slot * slab16, ws = w_lo + (uint32_t)(3 * dy) * wtap16;
            for (int bk = 0; bk < nmain; bk++) {
              const uint32_t xb = xs + (uint32_t)bk * sblk16, wb = ws + (uint32_t)bk * wblk16;
#pragma unroll
              for (int c = 0; c < 4; c++)
#pragma unroll
                for (int dx = 0; dx < 3; dx++) {
                  mma_bf16_elect(d, desc_pack(xb + 8u * dx + 2u * c, hi_main), desc_pack(wb + dx * wtap16 + 2u * c, hi_main),
                           idesc, acc);
                  acc = 1;
                }
            }
            if (tail) {
              const uint32_t xb = xs + (uint32_t)nmain * sblk16, wb = ws + (uint32_t)nmain * wblk16;
              for (uint32_t c = 0; c < tail16 / 2; c++)
#pragma unroll
                for (int dx = 0; dx < 3; dx++) {
                  mma_bf16_elect(d, desc_pack(xb + tail16 * dx + 2u * c, hi_tail), desc_pack(wb + dx * wtap16 + 2u * c, hi_tail),
                           idesc, acc);
                  acc = 1;
                }
            }
          }
          mma_commit_elect(&acc_full[b]);
          mma_commit_elect(&empty[q0.slot]);    // slab i is read by no later row
          q0 = q1;
          q1 = q2;
        }
        if (!ok) break;
        // the run's last two slabs
        mma_commit_elect(&empty[q0.slot]);
        mma_commit_elect(&empty[q1.slot]);
        q = q1.next((uint32_t)S);
      }
    }
  } else {
    // epilogue: warp w drains TMEM lanes (pixels) 32 qw .. 32 qw + 31, qw =
    // w % 4, of output channels c0 .. c0 + 15, c0 = 16 (w / 4), of each tile
    const int qw = warp & 3, c0 = 16 * (warp >> 2);
    uint32_t tc = 0;
    TileRun r;
    for (int u = lo; ok && next_run(u, hi, a.H, r);) {
      for (int i = 0; i < r.len && ok; i++, tc++) {
        const uint32_t b = tc & 1u;
        const int y = r.y0 + i, px = r.seg * kM + qw * 32 + lane;
        const bool in = px < a.W;
        const size_t o = ((size_t)y * a.W + (in ? px : 0)) * a.Cout + co0 + c0;
        // this lane's skip values, fetched while the tile's MMAs run
        uint4 sk0 = make_uint4(0, 0, 0, 0), sk1 = sk0;
        if (a.skip && in) {
          sk0 = __ldg(reinterpret_cast<const uint4*>(a.skip + o));
          sk1 = __ldg(reinterpret_cast<const uint4*>(a.skip + o) + 1);
        }
        if (!(ok = mbar_wait(&acc_full[b], (tc >> 1) & 1u, 64))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t v[16];
        tmem_ld16(tmem + b * ncols + ((uint32_t)(qw * 32) << 16) + (uint32_t)c0, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // buffer b may be overwritten by the next tile's MMAs once every
        // epilogue warp has its values
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
        if (!kPairStores && !in) continue;
        // with paired stores every lane goes on (the stores pair neighbouring
        // lanes); lanes past the row's end compute on their TMEM rows and
        // store only their partner's pixel
        const bool odd = (lane & 1) != 0;
        const bool in_partner = kPairStores ? __shfl_xor_sync(0xffffffffu, in ? 1 : 0, 1) != 0 : false;
        const ptrdiff_t po = odd ? -(ptrdiff_t)a.Cout : (ptrdiff_t)a.Cout;   // the partner pixel's offset
        // store offsets from the unclamped pixel (px - 1 <= W - 1 for the
        // partner of a lane past the row's end)
        const size_t os = ((size_t)y * a.W + px) * a.Cout + co0 + c0;
        float f[16];
#pragma unroll
        for (int e = 0; e < 16; e++) {
          const float val = __uint_as_float(v[e]) + bias_s[c0 + e];
          f[e] = a.relu ? fmaxf(val, 0.f) : val;
        }
        __align__(16) __nv_bfloat16 hb[16];
        if (a.r16) {
#pragma unroll
          for (int e = 0; e < 16; e++) hb[e] = __float2bfloat16(f[e]);
          if constexpr (kPairStores) {
            store_sector_pair(reinterpret_cast<uint4*>(a.r16 + os), reinterpret_cast<uint4*>(a.r16 + os + po),
                              reinterpret_cast<const uint4*>(hb)[0], reinterpret_cast<const uint4*>(hb)[1], odd, in,
                              in_partner);
          } else {
            reinterpret_cast<uint4*>(a.r16 + o)[0] = reinterpret_cast<const uint4*>(hb)[0];
            reinterpret_cast<uint4*>(a.r16 + o)[1] = reinterpret_cast<const uint4*>(hb)[1];
          }
        }
        if (a.skip) {
          __align__(16) __nv_bfloat16 skb[16];
          reinterpret_cast<uint4*>(skb)[0] = sk0;
          reinterpret_cast<uint4*>(skb)[1] = sk1;
#pragma unroll
          for (int e = 0; e < 16; e++) f[e] = __bfloat162float(__float2bfloat16(f[e])) + __bfloat162float(skb[e]);
        }
        if (a.y16) {
#pragma unroll
          for (int e = 0; e < 16; e++) hb[e] = __float2bfloat16(f[e]);
          if constexpr (kPairStores) {
            store_sector_pair(reinterpret_cast<uint4*>(a.y16 + os), reinterpret_cast<uint4*>(a.y16 + os + po),
                              reinterpret_cast<const uint4*>(hb)[0], reinterpret_cast<const uint4*>(hb)[1], odd, in,
                              in_partner);
          } else {
            reinterpret_cast<uint4*>(a.y16 + o)[0] = reinterpret_cast<const uint4*>(hb)[0];
            reinterpret_cast<uint4*>(a.y16 + o)[1] = reinterpret_cast<const uint4*>(hb)[1];
          }
        }
        if (a.y32 && !kPairStores) {
          float4* q4 = reinterpret_cast<float4*>(a.y32 + o);
#pragma unroll
          for (int e = 0; e < 4; e++) q4[e] = make_float4(f[4 * e], f[4 * e + 1], f[4 * e + 2], f[4 * e + 3]);
        }
        if (a.y32 && kPairStores) {   // two sectors: channels 0-7 and 8-15
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const uint4 lo = make_uint4(__float_as_uint(f[8 * h]), __float_as_uint(f[8 * h + 1]),
                                        __float_as_uint(f[8 * h + 2]), __float_as_uint(f[8 * h + 3]));
            const uint4 hi = make_uint4(__float_as_uint(f[8 * h + 4]), __float_as_uint(f[8 * h + 5]),
                                        __float_as_uint(f[8 * h + 6]), __float_as_uint(f[8 * h + 7]));
            store_sector_pair(reinterpret_cast<uint4*>(a.y32 + os + 8 * h), reinterpret_cast<uint4*>(a.y32 + os + po + 8 * h),
                              lo, hi, odd, in, in_partner);
          }
        }
      }
    }
  }
  if (!ok && (lane == 0)) atomicOr(a.status, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == w_mma) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ncols));
  }
}

// Weight gradient of a 3x3 convolution on the tensor cores:
// dW (t, co, ci) = sum over pixels p of dy (p, co) x (p + off(t), ci), as
// GEMMs with K = pixels, read straight from the pixel-major BF16 tensors
// dy (H, W, Cout) and x (H, W, Cin): both operands are MN-major (the channel
// is the contiguous dimension, a pixel is a row of the shared-memory tile).
// Substituting y' = y + dy, dW (dy, dx) = sum over (y', x) of
// dy (y' - dy, x, co) x (y', x + dx, ci): a K step is 64 pixels x .. x + 63
// of one row y'.  B is one box of x at row y', pixels x - 1 .. x + 64, read
// by three MMAs whose start rows differ by one pixel (dx = -1, 0, 1: one
// accumulator each; the swizzle follows the shared-memory address bits, so
// a start moved by whole rows reads what the TMA wrote); A the box(es) of
// dy at rows y' - dy.  Rows and pixels outside the image read zeros.
// With Cout <= 32 the three vertical taps share one MMA: A's rows 32 g + co
// hold dy at row y' - (g - 1), so one CTA computes all nine taps from one
// load of each operand per step (rows past Cout in each group are left over
// and ignored); otherwise blockIdx.y is the vertical tap and A is one or two
// boxes of 64 channels.  blockIdx.x is a band of rows y'.  Per step 4 x 3
// MMAs of 16 pixels.  The band's sums are added into dw (FP32) by the
// epilogue warps with vector atomics.  blockIdx.x takes an equal share of
// the (row, 64-pixel chunk) steps, in row order.
//
// Channel boxes: Cout (stacked) or 64 channels of dy, min(Cin, 64) channels
// of x, rows of 2 x channels bytes with the matching swizzle; a box of dy is
// 64 pixel rows, one of x 66 (72 reserved, a whole number of swizzle
// atoms); boxes along the channels lie one box apart (the MN stride of the
// descriptor), groups of 8 pixels one 8-row group apart.
constexpr int kWgMaxStages = 8;
constexpr size_t kWgA = 128 * 128;                        // A: 128 channel rows x 64 pixels
__host__ __device__ constexpr int wgrad_xbox(int cin) { return cin < 64 ? cin : 64; }
constexpr int kWgXRows = 72;                              // x box: 66 pixels, 72 rows reserved
__host__ __device__ constexpr size_t wgrad_xbox_bytes(int cin) { return (size_t)kWgXRows * 2 * wgrad_xbox(cin); }
__host__ __device__ constexpr size_t wgrad_stage_bytes(int cin) {
  return (kWgA + (size_t)((cin + 63) / 64) * wgrad_xbox_bytes(cin) + 1023) & ~size_t(1023);
}
__host__ __device__ constexpr uint32_t wgrad_acc_stride(int cin) { return cin <= 32 ? 32u : (uint32_t)cin; }
__host__ __device__ constexpr uint32_t wgrad_tmem_cols(int cin) {
  return 3 * wgrad_acc_stride(cin) <= 128 ? 128u : 3 * wgrad_acc_stride(cin) <= 256 ? 256u : 512u;
}
constexpr size_t kWgSmemCap = 200 * 1024;
constexpr size_t kWgSlack = 1024;               // alignment of the ring
__host__ __device__ constexpr int wgrad_stages(int cin) {
  return (int)(kWgSmemCap / wgrad_stage_bytes(cin)) < kWgMaxStages ? (int)(kWgSmemCap / wgrad_stage_bytes(cin))
                                                                      : kWgMaxStages;
}
struct WgradTcArgs {
  float* dw;                 // (9, Cout, Cin), accumulated into
  unsigned int* status;      // bit 0: a barrier wait gave up
  int H, W, Cin, Cout;
  int steps_per_cta;         // (row, 64-pixel chunk) steps of one CTA
  int stacked;               // Cout <= 32: the three vertical taps in one MMA
  int S;                     // stages
};
// the low descriptor word of an MN-major operand: start address and the
// stride between boxes along the channels
__device__ __forceinline__ uint32_t desc_lo_mn(uint32_t addr, uint32_t box_bytes) {
  return ((addr >> 4) & 0x3FFFu) | (((box_bytes >> 4) & 0x3FFFu) << 16);
}

__global__ void __launch_bounds__(kThreads) wgrad3x3_tc_kernel(const __grid_constant__ CUtensorMap tdy,
                                                               const __grid_constant__ CUtensorMap tx,
                                                               const WgradTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kWgMaxStages], empty[kWgMaxStages], acc_full;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = a.S;
  const uint32_t stage_bytes = (uint32_t)wgrad_stage_bytes(a.Cin), xb_bytes = (uint32_t)wgrad_xbox_bytes(a.Cin);
  const int cba = a.stacked ? a.Cout : 64, cbb = wgrad_xbox(a.Cin);     // channels per box
  const int dy_cta = a.stacked ? 0 : (int)blockIdx.y - 1;               // this CTA's vertical tap (not stacked)
  const int nseg = (a.W + 63) / 64, k0 = blockIdx.x * a.steps_per_cta;
  const int nk = max(0, min(a.H * nseg, k0 + a.steps_per_cta) - k0);
  const uint32_t stride = wgrad_acc_stride(a.Cin), ncols = wgrad_tmem_cols(a.Cin);

  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < S; s++) {
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
      const int na = a.stacked ? 3 : (a.Cout + 63) / 64, nbx = (a.Cin + 63) / 64;
      const uint32_t bytes = (uint32_t)na * 128u * (uint32_t)cba + (uint32_t)nbx * 132u * (uint32_t)cbb;
      RingPos q{0u, 0u};
      for (int k = 0; k < nk && ok; k++, q = q.next((uint32_t)S)) {
        if (!(ok = mbar_wait(&empty[q.slot], q.phase ^ 1u))) break;
        const int y = (k0 + k) / nseg, x0 = ((k0 + k) % nseg) * 64;
        uint8_t* st = ring + (size_t)q.slot * stage_bytes;
        mbar_expect_tx(&full[q.slot], bytes);
        if (a.stacked) {   // vertical tap g - 1 at A rows 32 g ..
          for (int g = 0; g < 3; g++) tma_load_3d(st + (size_t)g * 4096, &tdy, 0, x0, y - (g - 1), &full[q.slot]);
        } else {
          for (int b = 0; b < na; b++) tma_load_3d(st + (size_t)b * 8192, &tdy, 64 * b, x0, y - dy_cta, &full[q.slot]);
        }
        for (int b = 0; b < nbx; b++) tma_load_3d(st + kWgA + (size_t)b * xb_bytes, &tx, 64 * b, x0 - 1, y, &full[q.slot]);
      }
    }
  } else if (warp == 5) {
    {   // all 32 lanes: warp-uniform descriptors, elected issue
      const uint32_t idesc = mma_idesc(kM, a.Cin) | (1u << 15) | (1u << 16);   // A and B MN-major
      const uint32_t a_hi = desc_hi(2u * (uint32_t)cba), b_hi = desc_hi(2u * (uint32_t)cbb);
      const uint32_t a_lo = desc_lo_mn(smem_u32(ring), 128u * (uint32_t)cba);
      const uint32_t b_lo = desc_lo_mn(smem_u32(ring) + (uint32_t)kWgA, xb_bytes);
      // one pixel = one row of 2 x channels bytes, in 16-byte units
      const uint32_t a_row = (uint32_t)cba >> 3, b_row = (uint32_t)cbb >> 3;
      const uint32_t stage16 = stage_bytes >> 4;
      RingPos q{0u, 0u};
      for (int k = 0; k < nk && ok; k++, q = q.next((uint32_t)S)) {
        if (!(ok = mbar_wait_warp(&full[q.slot], q.phase))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
          for (int dx = 0; dx < 3; dx++)
            mma_bf16_elect(tmem + (uint32_t)dx * stride, desc_pack(a_lo + q.slot * stage16 + 16u * a_row * c, a_hi),
                     desc_pack(b_lo + q.slot * stage16 + (16u * c + (uint32_t)dx) * b_row, b_hi), idesc,
                     (k > 0 || c > 0) ? 1u : 0u);
        mma_commit_elect(&empty[q.slot]);
      }
      if (ok) mma_commit_elect(&acc_full);
    }
  } else if (nk > 0) {
    // epilogue: TMEM lane 32 w + l is A's row: (vertical tap w - 1, output
    // channel l) when stacked, else output channel 32 w + l
    const int g = a.stacked ? warp : dy_cta + 1, co = a.stacked ? lane : warp * 32 + lane;
    const bool rows_used = a.stacked ? warp < 3 : warp * 32 < a.Cout;
    if (rows_used && (ok = mbar_wait(&acc_full, 0, 64))) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int dx = 0; dx < 3; dx++) {
        float* d = a.dw + ((size_t)(3 * g + dx) * a.Cout + co) * a.Cin;
        for (int c0 = 0; c0 < a.Cin; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)dx * stride + (uint32_t)c0, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (co >= a.Cout) continue;
#pragma unroll
          for (int e = 0; e < 4; e++)
            atomicAdd(reinterpret_cast<float4*>(d + c0) + e,
                      make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]), __uint_as_float(v[4 * e + 2]),
                                  __uint_as_float(v[4 * e + 3])));
        }
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

// Launch plan of conv3x3_tc_kernel for one layer: the largest channel block
// Nb (a multiple of 16 dividing Cout) whose weights and four slabs fit in
// 220 KB of shared memory; then as many slab stages (at most kMaxStages) as
// fit in 110 KB, so that two CTAs share an SM, or else in 220 KB; and the
// CTAs that fit on one SM by shared memory and by tensor memory (512
// columns, two accumulators per CTA).
struct ConvPlan {
  int Nb, S, ctas_per_sm;
  size_t smem;
};
constexpr size_t kConvSmemCap = 220 * 1024;   // dynamic; the kernel's static shared memory comes on top
inline ConvPlan conv_plan(int cin, int cout) {
  const size_t cap = kConvSmemCap, half = kConvSmemCap / 2, slab = conv_slab_bytes(cin);
  int nb = 16;
  for (int d = 1; d <= cout / 16; d++) {
    if (cout % d || (cout / d) % 16 || cout / d > kConvMaxNb) continue;
    if (conv_smem_bytes(cin, cout / d, 4) <= cap) {
      nb = cout / d;
      break;
    }
  }
  const size_t budget = conv_smem_bytes(cin, nb, 4) <= half ? half : cap;
  int s = (int)((budget - conv_smem_bytes(cin, nb, 0)) / slab);
  s = s < kMaxStages ? s : kMaxStages;
  ConvPlan p{nb, s, 1, conv_smem_bytes(cin, nb, s)};
  const int by_tmem = 512 / (int)(2 * conv_acc_cols(nb)), by_smem = (int)((228 * 1024) / (p.smem + 2048));   // + reserved and static
  p.ctas_per_sm = by_tmem < by_smem ? by_tmem : by_smem;
  if (p.ctas_per_sm < 1) p.ctas_per_sm = 1;
  return p;
}

}  // namespace tc
}  // namespace amh
