// Host-side check of the tensor-core kernels' launch plans
// (paper_1805_07920_gb300/csrc/amh_conv_tc.cuh) for every channel pair the
// network's convolutions accept (Cin in {16, 32, 64, 96, 128}, Cout a
// multiple of 16 up to 128).  It checks the rules the kernels rely on:
// swizzled regions 1024-byte aligned, shared memory within the attribute the
// host sets, tensor-memory allocations a power of two that hold every
// accumulator, enough ring stages for the rows read at once, TMA boxes and
// the MMAs' operand reads inside their regions, descriptor fields in range.
// Prints one line per violation and exits non-zero if there is any.
#include <cstdio>

#include "../paper_1805_07920_gb300/csrc/amh_conv_tc.cuh"

using namespace amh::tc;

static int fails = 0;
#define CHECK(cond, ...)                            \
  do {                                              \
    if (!(cond)) {                                  \
      std::printf("FAIL %s: ", #cond);              \
      std::printf(__VA_ARGS__);                     \
      std::printf("\n");                            \
      fails++;                                      \
    }                                               \
  } while (0)

static bool pow2(unsigned v) { return v && !(v & (v - 1)); }

int main() {
  const int cins[] = {16, 32, 64, 96, 128};
  int n = 0;
  for (int cin : cins)
    for (int cout = 16; cout <= kMaxCout; cout += 16, n++) {
      // forward / data-gradient convolution
      const ConvPlan p = conv_plan(cin, cout);
      CHECK(p.Nb % 16 == 0 && p.Nb >= 16 && p.Nb <= kConvMaxNb && cout % p.Nb == 0, "cin %d cout %d Nb %d", cin, cout, p.Nb);
      CHECK(p.S >= 3 && p.S <= kMaxStages, "cin %d cout %d: %d slab stages (rows i .. i + 2 are read at once)", cin, cout, p.S);
      CHECK(p.smem == conv_smem_bytes(cin, p.Nb, p.S) && p.smem <= kConvSmemCap, "cin %d cout %d smem %zu", cin, cout, p.smem);
      CHECK(conv_slab_bytes(cin) % 1024 == 0 && conv_wtap_bytes(cin, p.Nb) % 1024 == 0, "cin %d: regions not 1 KB aligned", cin);
      CHECK(conv_threads(p.Nb) <= kConvMaxThreads, "cin %d cout %d threads %d", cin, cout, conv_threads(p.Nb));
      const unsigned cols = conv_acc_cols(p.Nb);
      CHECK(pow2(2 * cols) && 2 * cols >= 32 && cols >= (unsigned)p.Nb && 2 * cols * p.ctas_per_sm <= 512,
            "cin %d cout %d: tensor memory %u x 2 columns, %d CTAs per SM", cin, cout, cols, p.ctas_per_sm);
      CHECK(p.ctas_per_sm >= 1 && p.ctas_per_sm * (p.smem + 2048) <= 228 * 1024, "cin %d cout %d: %d CTAs per SM", cin, cout,
            p.ctas_per_sm);
      // the MMAs of a slab read rows dx .. dx + 127 (dx <= 2) of each block: inside the block's kHalo rows
      CHECK(2 + kM <= kHalo, "halo %d", kHalo);

      // weight gradient
      const size_t stage = wgrad_stage_bytes(cin), xb = wgrad_xbox_bytes(cin);
      const int S = wgrad_stages(cin), cbb = wgrad_xbox(cin), nbx = (cin + 63) / 64;
      const bool stacked = cout <= 32;
      const int cba = stacked ? cout : 64, na = stacked ? 3 : (cout + 63) / 64;
      CHECK(stage % 1024 == 0, "wgrad cin %d: stage %zu bytes", cin, stage);
      CHECK(S >= 2 && S <= kWgMaxStages && S * stage + kWgSlack <= kWgSmemCap + kWgSlack && kWgSmemCap + kWgSlack <= 227 * 1024,
            "wgrad cin %d: %d stages of %zu bytes", cin, S, stage);
      // A: stacked boxes of dy at 4096-byte steps (M rows 32 g + co), else 64-channel boxes 8 KB apart
      const size_t a_end = stacked ? 2 * 4096 + (size_t)128 * cba : (size_t)na * 8192;
      CHECK(a_end <= kWgA && (stacked ? 128 * cba <= 4096 : true), "wgrad cin %d cout %d: A boxes end at %zu", cin, cout, a_end);
      // B: nbx boxes of 66 loaded pixel rows in 72 reserved; the MMAs read rows dx + 16 c .. + 15 (dx <= 2, c <= 3)
      CHECK(xb % (16 * (size_t)cbb) == 0 && xb % 256 == 0, "wgrad cin %d: x box region %zu", cin, xb);
      CHECK(2 + 48 + 16 <= 66 && 66 <= kWgXRows, "wgrad: x rows");
      CHECK(kWgA + nbx * xb <= stage, "wgrad cin %d: x boxes end past the stage", cin);
      CHECK((xb >> 4) < (1u << 14) && ((128u * cba) >> 4) < (1u << 14), "wgrad cin %d: descriptor stride field", cin);
      // accumulators: three of Cin columns (the MMA's N), 16 <= N <= 256, N % 16 == 0
      const unsigned stride = wgrad_acc_stride(cin), tcols = wgrad_tmem_cols(cin);
      CHECK(cin % 16 == 0 && cin >= 16 && cin <= 256 && stride >= (unsigned)cin && 3 * stride <= tcols && pow2(tcols) &&
                tcols >= 32 && tcols <= 512,
            "wgrad cin %d: accumulators %u x 3 in %u columns", cin, stride, tcols);
    }
  std::printf("%d channel pairs checked, %d failures\n", n, fails);
  return fails ? 1 : 0;
}
