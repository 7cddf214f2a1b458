// Tensor-core (tcgen05, sm_103a) form of the travel-time MLP: forward pass and
// source Jacobian for tiles of 128 (event, station) pairs (Sec. 2.1, Sec. 3.2).
//
//   layer 1 (6 -> H)  h1 = silu(W1 [x; s] + b1): a BF16 product in both forms,
//       with operands split in BF16 pairs, v = v_hi + v_lo: the operand row
//       [x_hi, x_lo, x_hi, 0 ...] against [W_hi, W_hi, W_lo, 0 ...] (K = 32) gives
//       W1 [x; s] up to the dropped W_lo x_lo (relative 2^-16 of each term)
//   layers 2..4 (H x H, BF16 x BF16 or E4M3 x E4M3 -> FP32 in TMEM)  h_l = silu(W_l h_{l-1} + b_l)
//   output (H -> 1, FP32)  tau = w5 . h4 + b5,  T = |x - s| tau  (double-float outer product)
//   reverse sweep (H x H, BF16 -> FP32 in TMEM)
//       delta4 = w5 * silu'(z4);  delta_{l-1} = (W_l^T delta_l) * silu'(z_{l-1})
//   dtau/dx = W1[:, :3]^T delta1 (FP32),  dT/dx = tau (x - s)/r + r dtau/dx.
//
// One CTA per SM, persistent over tiles; 19 warps:
//   warps 0-15 epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (one pair per
//              lane); within every K-block of the next operand, column group
//              w / 4 takes a quarter of the K-block's columns, 16 at a time, so
//              the K-blocks of the operand complete one after the other;
//   warp 16    producer: 1-D bulk async copies (cp.async.bulk) of pre-swizzled
//              weight K-blocks (H rows x 128 bytes) into a four-stage ring;
//   warp 18    geometry: loads the (event, station) geometry of the next tile
//              into a shared-memory double buffer while the current tile runs;
//   warp 17    MMA issuer: tcgen05.mma.cta_group::1, M = 128, N = H, A = the
//              activations in TMEM, B = weights (SW128 K-major, shared memory),
//              D = FP32 accumulator in TMEM.
// TMEM (2H columns): two accumulators, [0, H) for products 0, 2, 4 and [H, 2H)
// for products -1 (the first layer), 1, 3, 5 (forward W2, W3, W4, reverse
// W4^T, W3^T, W2^T).  The epilogue of product l writes the operand of product
// l + 1 over the accumulator it is reading, each thread into its own lane and
// into columns it has already read: the values of the 16-column chunk at col
// go, packed, to the first columns of their K-step (BF16: columns [col, col + 8)
// hold K-step col / 16; E4M3: columns [32 s, 32 s + 8) hold K-step s), so
// product l + 1 reads A from one accumulator and writes D into the other.  It
// starts on K-block kb of its operand as soon as the epilogue of product l has
// written that K-block (one barrier per K-block); only its last K-block is left
// when the epilogue finishes.  The first layer's operand sits in columns
// [16, 32) of [0, H).  silu'(z1), silu'(z2), silu'(z3) (BF16) sit in three
// per-CTA slots in global memory (each thread reads back only what it wrote;
// a reverse layer's first stash loads are issued before its product completes).
// At the end of a tile the first 16 columns of [0, H) carry the column groups'
// partial sums of tau and dtau/dx to the row's first group.
// Four weight stages hold a whole layer at H = 256 (BF16), so the next layer's
// weights are resident when its operand is ready.
// Shared memory keeps W1 and the biases pre-halved (exact): the epilogue works
// with u = z/2, silu(z) = u + u tanh(u), silu'(z) = s + silu(z) (1 - s),
// s = (1 + tanh(u)) / 2.
// FP8 form (kind::f8f6f4, E4M3 operands, FP32 accumulation): the weight images
// carry one scale per output column (max |W| / 448); each activation row is
// quantised with its own scale, from a first pass over the accumulator that
// bounds the row's largest magnitude (the four threads holding a row exchange
// their bounds through a 128-arrival mbarrier); delta4 = w5 * silu'(z4)
// uses the fixed bound 1.1 max |w5|.  The accumulator of the next layer is
// rescaled by (row scale) x (column scale) before bias and activation.
// Every wait is bounded (2 s on the global timer): on timeout the kernel sets
// SPIDER_E_TIMEOUT, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "kernels.h"
#include "pairs.cuh"
#include "quant.h"
#include "spider.h"

namespace spider {
namespace {

constexpr int kRows = 128;          // pairs per tile = MMA M = TMEM lanes
constexpr int kEpiWarps = 16;
constexpr int kGroups = kEpiWarps / 4;     // column groups per TMEM lane quarter
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kCc = 16;                     // columns per epilogue chunk
constexpr int kTcThreads = kEpiThreads + 96;   // + producer, MMA issuer, geometry warps
constexpr int kStages = 4;
constexpr int kMaxKb = 4;                   // K-blocks per layer at most (H = 256, BF16)
// mbarriers: full, empty [kStages]; acc_ready, drain, red_ready; a_ready [kMaxKb];
// xbar [4]; geo_full, geo_empty [2]
constexpr int kBars = 2 * kStages + 3 + kMaxKb + 4 + 4;
constexpr uint64_t kWaitNs = 2000000000ull;

template <int H, bool F8>
struct Cfg {
  static constexpr int EB = F8 ? 1 : 2;             // bytes per operand element
  static constexpr int KB = H * EB / 128;           // K-blocks (128-byte rows) per layer
  static constexpr int kChunk = H * 128;            // bytes of one weight K-block (H rows x 128 B)
  static constexpr int kD = kRows * H * 2;          // one silu'(z) slot (BF16) in global memory
  static constexpr int kStash = 3 * kD;             // silu'(z1), silu'(z2), silu'(z3) per CTA
  static constexpr int kCols = H / kGroups;         // columns per epilogue thread
  static constexpr int kKbCols = H / KB;            // columns of one K-block of A
  static constexpr int kKstep = kKbCols / 4;        // K of one MMA instruction (16 BF16 or 32 E4M3)
  static constexpr int kCpk = kKbCols / kGroups / kCc;   // 16-column chunks per thread and K-block
  static constexpr int kChunks = kCols / kCc;       // chunks per thread and layer
  static_assert(KB <= kMaxKb && kChunks == KB * kCpk && kCpk >= 1, "tile shape");
  static constexpr int kTmemCols = 2 * H;
  static constexpr int kChunksPerTile = 1 + 6 * KB;  // the first layer's image (one K-block), then 6 layers
  // shared-memory carve-up (offsets from a 1024-aligned base)
  static constexpr int oB = 0;
  static constexpr int oPar = oB + kStages * kChunk;      // W1 (6H), b1, b2, b3, b4, w5 (5H) floats
  static constexpr int oSc = oPar + 11 * H * 4;           // FP8: column scales of the 6 images (6H floats)
  static constexpr int oXch = oSc + (F8 ? 6 * H * 4 : 0); // FP8: row-bound exchange [2][kGroups][kRows] floats
  static constexpr int oGeo = oXch + (F8 ? 2 * kGroups * kRows * 4 : 0);   // pair geometry [2][15][kRows] floats
  // silu'(z3) of the current tile (kD bytes) in shared memory when it fits
  // (read by the first reverse layer, two products after it is written);
  // otherwise it goes to the third global slot like silu'(z1), silu'(z2)
  static constexpr int oD3 = oGeo + 2 * 15 * kRows * 4;
  static constexpr bool kD3Shared = oD3 + kD + kBars * 8 + 16 + 1024 <= 232448;
  static constexpr int oBar = oD3 + (kD3Shared ? kD : 0);         // mbarriers
  static constexpr int oMisc = oBar + kBars * 8;          // tmem base, abort flag
  static constexpr int kSmem = oMisc + 16 + 1024;         // + alignment slack
  static_assert(kSmem <= 232448, "shared memory per CTA");
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// the same, letting the thread sleep (up to the hint, in ns) until the phase completes
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.  False on abort/timeout.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int32_t* gerr) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = gtime();
  for (;;) {
    if (mbar_test_sleep(b, parity)) return true;
    if (*abort_flag) return false;
    if (gtime() - t0 > kWaitNs) {
      *abort_flag = 1;
      atomicCAS(gerr, 0, SPIDER_E_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: BF16 A and B (both K-major), FP32 D, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

// Instruction descriptor, kind::f8f6f4: E4M3 A and B (both K-major), FP32 D, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_e4m3(int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

// MMA with A read from tensor memory (lane = row, K packed along columns)
template <bool F8>
__device__ __forceinline__ void umma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (F8) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3])
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld16f(uint32_t taddr, float (&v)[16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


// two FP32 lanes per instruction (f32x2): the same IEEE operations as the scalar
// forms, so results are identical to them
__device__ __forceinline__ uint64_t f2pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2unpack(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
constexpr uint64_t kHalf2 = 0x3F0000003F000000ull;    // (0.5, 0.5)
constexpr uint64_t kNegHalf2 = 0xBF000000BF000000ull;  // (-0.5, -0.5)

// silu and silu' of z = 2u on two values: t = tanh(u), h = u + u t,
// d = s + h (1 - s) with s = (1 + t) / 2 and 1 - s = (1 - t) / 2
__device__ __forceinline__ void silu_half(uint64_t u, uint64_t& h, uint64_t& d) {
  float a, b;
  f2unpack(u, a, b);
  const uint64_t t = f2pack(tanh_fast(a), tanh_fast(b));
  h = f2fma(u, t, u);
  d = f2fma(h, f2fma(t, kNegHalf2, kHalf2), f2fma(t, kHalf2, kHalf2));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }


// four FP32 values -> four E4M3 bytes (round to nearest even, saturating), first value in the low byte
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  uint16_t lo, hi;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
  return (uint32_t)lo | ((uint32_t)hi << 16);
}

// FP8: largest magnitude bound of a row over its column groups (bounded wait);
// every thread of the row takes the maximum in the same order
__device__ __forceinline__ bool group_max(float& m, float* xch, uint64_t* xbar, uint32_t& xph, int cg, int r,
                                          volatile int* abort_flag, int32_t* gerr) {
  const int slot = (int)(xph & 1);
  xch[(slot * kGroups + cg) * kRows + r] = m;
  mbar_arrive(xbar);
  const bool got = mbar_wait(xbar, xph & 1, abort_flag, gerr);
  xph ^= 1;
  if (got) {
    float a = xch[(slot * kGroups) * kRows + r];
#pragma unroll
    for (int q = 1; q < kGroups; ++q) a = fmaxf(a, xch[(slot * kGroups + q) * kRows + r]);
    m = a;
  }
  return got;
}

// silu'(z) slot: 16-byte chunk c/8 of row r at ((c/8) * 128 + r) * 16
__device__ __forceinline__ uint32_t d_off(int r, int c) { return (uint32_t)(((c >> 3) * kRows + r) * 16); }

template <int H, bool F8>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tt_mlp_tc(NetView net, PairSource src, TTOut out, const uint8_t* __restrict__ wimg, int32_t* gerr,
                uint8_t* __restrict__ stash) {
  using C = Cfg<H, F8>;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base by pointer arithmetic on the shared array itself, so
  // that every access through it compiles to a shared-memory instruction (an
  // integer round trip would leave generic addresses)
  uint8_t* sm = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  uint8_t* sB = sm + C::oB;
  // silu'(z1..3) of the current tile: this CTA's slots in global memory (each
  // thread reads back only what it wrote)
  uint8_t* sD = stash + (size_t)blockIdx.x * C::kStash;
  uint8_t* sD3 = C::kD3Shared ? sm + C::oD3 : sD + 2 * (size_t)C::kD;   // the slot of silu'(z3)
  float* pW1 = reinterpret_cast<float*>(sm + C::oPar);
  float* pb1 = pW1 + 6 * H;
  float* pb = pb1 + H;       // b2, b3, b4
  float* pw5 = pb + 3 * H;
  float* wsc = reinterpret_cast<float*>(sm + C::oSc);     // FP8 column scales [6][H]
  float* xch = reinterpret_cast<float*>(sm + C::oXch);    // FP8 row-bound exchange
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::oBar);
  uint64_t* full = bars;                     // [kStages] weight stage loaded
  uint64_t* empty = bars + kStages;          // [kStages] weight stage consumed
  uint64_t* acc_ready = bars + 2 * kStages;  // product complete (one phase per product)
  uint64_t* drain = acc_ready + 1;           // MMA drain on abort
  uint64_t* red_ready = acc_ready + 2;       // every column group of every row reduced
  uint64_t* a_ready = acc_ready + 3;         // [kMaxKb] K-block of A written by every epilogue warp
  uint64_t* xbar = a_ready + kMaxKb;         // [4] FP8 row-bound exchange within a lane quarter
  uint64_t* geo_full = xbar + 4;             // [2] geometry buffer filled
  uint64_t* geo_empty = geo_full + 2;        // [2] geometry buffer released by the epilogue
  float* geo = reinterpret_cast<float*>(sm + C::oGeo);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + C::oMisc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + C::oMisc + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(acc_ready, 1);
    for (int q = 0; q < kMaxKb; ++q) mbar_init(&a_ready[q], kEpiWarps);
    mbar_init(drain, 1);
    mbar_init(red_ready, kEpiThreads);
    for (int q = 0; q < 4; ++q) mbar_init(&xbar[q], 32 * kGroups);
    for (int q = 0; q < 2; ++q) {
      mbar_init(&geo_full[q], 32);
      mbar_init(&geo_empty[q], kEpiThreads);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // W1 / 2 transposed in shared memory (6 x H: input c, column) so that column
  // pairs are adjacent; b1 / 2 .. b4 / 2 (halving is exact)
  for (int i = threadIdx.x; i < 6 * H; i += blockDim.x) pW1[(i % 6) * H + i / 6] = 0.5f * net.W1[i];
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    pb1[i] = 0.5f * net.b1[i];
    pb[i] = 0.5f * net.bh[0][i];
    pb[H + i] = 0.5f * net.bh[1][i];
    pb[2 * H + i] = 0.5f * net.bh[2][i];
    pw5[i] = net.W5[i];
  }
  if constexpr (F8)
    for (int i = threadIdx.x; i < 6 * H; i += blockDim.x) wsc[i] = net.tc_scale[i];
  const float s4 = F8 ? net.tc_scale[6 * H] : 1.f;     // FP8 scale of delta4 = w5 * silu'(z4)
  if (warp == kEpiWarps + 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"((uint32_t)C::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t P = pair_count(src);
  const int64_t ntiles = (P + kRows - 1) / kRows;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  if (warp == kEpiWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const int64_t total = my_tiles * C::kChunksPerTile;
      int64_t n = 0;
      for (; n < total; ++n) {
        const int s = (int)(n % kStages);
        const int64_t use = n / kStages;
        if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), abort_flag, gerr)) break;
        // the images are stored in consumption order, K-block after K-block
        const int c = (int)(n % C::kChunksPerTile);
        const uint8_t* g = wimg + (size_t)c * C::kChunk;
        mbar_expect_tx(&full[s], C::kChunk);
        bulk_load(sB + s * C::kChunk, g, C::kChunk, &full[s]);
      }
      // copies still in flight must land before the CTA's shared memory goes away
      for (int64_t m = (n > kStages ? n - kStages : 0); m < n; ++m) {
        const int s = (int)(m % kStages);
        const uint64_t t0 = gtime();
        while (!mbar_test(&full[s], (uint32_t)((m / kStages) & 1)))
          if (gtime() - t0 > kWaitNs) break;
      }
    }
  } else if (warp == kEpiWarps + 2) {
    // ------------------------------------------------------------ geometry prefetch
    for (int64_t t = 0; t < my_tiles; ++t) {
      const int b = (int)(t & 1);
      if (t >= 2) {
        const bool got = mbar_wait(&geo_empty[b], (uint32_t)(((t - 2) >> 1) & 1), abort_flag, gerr);
        if (!__all_sync(0xffffffffu, got)) break;
      }
      const int64_t u0 = (blockIdx.x + t * gridDim.x) * kRows;
      float* gb = geo + b * 15 * kRows;
      for (int r = lane; r < kRows; r += 32) {
        PairGeo pg;
        load_pair(src, u0 + r < P ? u0 + r : u0, pg);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gb[(0 + c) * kRows + r] = pg.shi[c];
          gb[(3 + c) * kRows + r] = pg.slo[c];
          gb[(6 + c) * kRows + r] = pg.soff[c];
          gb[(9 + c) * kRows + r] = pg.rhi[c];
          gb[(12 + c) * kRows + r] = pg.rlo[c];
        }
      }
      mbar_arrive(&geo_full[b]);
    }
  } else if (warp == kEpiWarps + 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = F8 ? idesc_e4m3(H) : idesc_bf16(H);
      // descriptor of address a + d (d a multiple of 16, the sum below 2^18) = desc(a) + d / 16
      const uint64_t bdesc = sw128_desc(su32(sB));
      int64_t n = 0;        // weight chunks consumed
      uint32_t a_phase = 0;  // bit kb: phase of a_ready[kb]
      bool ok = true;
      int issued = 0;
      for (int64_t t = 0; t < my_tiles && ok; ++t) {
        {
          // product -1: the split first layer (BF16 in both forms), K = 32 of
          // K-block 0, into [H, 2H)
          if (!mbar_wait(&a_ready[0], a_phase & 1u, abort_flag, gerr)) { ok = false; break; }
          a_phase ^= 1u;
          const int s = (int)(n % kStages);
          if (!mbar_wait(&full[s], (uint32_t)((n / kStages) & 1), abort_flag, gerr)) { ok = false; break; }
          tc_after();
          constexpr uint32_t idesc1 = idesc_bf16(H);
          const uint64_t bd = bdesc + (uint64_t)(s * (C::kChunk / 16));
          // A: [x_hi, x_lo, x_hi, 0 ...] in columns [16, 32) of [0, H)
          umma_ta<false>(tmem + (uint32_t)H, tmem + 16u, bd, idesc1, 0u);
          umma_ta<false>(tmem + (uint32_t)H, tmem + 24u, bd + 2, idesc1, 1u);
          issued += 2;
          umma_commit(&empty[s]);
          ++n;
          umma_commit(acc_ready);
        }
        for (int layer = 0; layer < 6 && ok; ++layer) {
          const uint32_t d = tmem + (uint32_t)((layer & 1) * H);     // this product's accumulator
          // its operand: written by the previous product's epilogue over that
          // product's accumulator, K-step k (kKstep values) packed into the
          // columns [k kKstep, k kKstep + 8)
          const uint32_t a = tmem + (uint32_t)(((layer + 1) & 1) * H);
          for (int kb = 0; kb < C::KB; ++kb, ++n) {
            // K-block kb of the operand written (and the accumulator free: its last
            // reader, the epilogue two products back, finished before)
            if (!mbar_wait(&a_ready[kb], (a_phase >> kb) & 1u, abort_flag, gerr)) { ok = false; break; }
            a_phase ^= 1u << kb;
            const int s = (int)(n % kStages);
            if (!mbar_wait(&full[s], (uint32_t)((n / kStages) & 1), abort_flag, gerr)) { ok = false; break; }
            tc_after();
            const uint32_t ak = a + (uint32_t)(kb * C::kKbCols);
            const uint64_t bd = bdesc + (uint64_t)(s * (C::kChunk / 16));
#pragma unroll
            for (int k = 0; k < 4; ++k)
              umma_ta<F8>(d, ak + (uint32_t)(k * C::kKstep), bd + 2 * k, idesc, (kb | k) ? 1u : 0u);
            issued += 4;
            umma_commit(&empty[s]);
          }
          if (!ok) break;
          umma_commit(acc_ready);
        }
      }
      if (!ok && issued) {
        // let the MMAs already issued finish before TMEM is released
        umma_commit(drain);
        const uint64_t t0 = gtime();
        while (!mbar_test(drain, 0))
          if (gtime() - t0 > kWaitNs) break;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int g = warp & 3, cg = warp >> 2;
    const int r = g * 32 + lane;                       // tile row = TMEM lane
    const uint32_t lane_addr = tmem + ((uint32_t)(g * 32) << 16);
    // column of this thread's chunk j (K-block-major)
    auto ccol = [cg](int j) {
      return (j / C::kCpk) * C::kKbCols + cg * (C::kKbCols / kGroups) + (j % C::kCpk) * kCc;
    };
    // this warp's part of K-block kb of the next operand is written (and its TMEM
    // reads before it are complete)
    auto a_done = [&](int kb) {
      tmem_wait_st();
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_ready[kb]);
    };
    // the next operand's values of columns col .. col + 15, packed into this
    // row's lane of the accumulator just read (acc = its lane address): BF16
    // pairs into columns [col, col + 8) (K-step col / 16); E4M3 quadruples into
    // four of the eight columns of K-step col / 32, which starts at the first of
    // this thread's two chunks of that K-step (both columns already read)
    auto put_a = [&](uint32_t acc, int col, const float (&o)[kCc], float inv) {
      if constexpr (F8) {
        uint32_t hq[4];
#pragma unroll
        for (int i = 0; i < kCc; i += 4)
          hq[i / 4] = pack_e4m3x4(o[i] * inv, o[i + 1] * inv, o[i + 2] * inv, o[i + 3] * inv);
        tmem_st4(acc + (uint32_t)((col & ~31) + ((col & 16) >> 2)), hq);
      } else {
        uint32_t hp[8];
#pragma unroll
        for (int i = 0; i < kCc; i += 2) hp[i / 2] = pack_bf16(o[i], o[i + 1]);
        tmem_st8(acc + (uint32_t)col, hp);
      }
    };
    // silu'(z_q), q = 1, 2, 3, of columns col .. col + 15 into slot q
    auto put_d = [&](int q, int col, const uint32_t (&dp)[kCc / 2]) {
      uint8_t* b = q == 3 ? sD3 : sD + (size_t)(q - 1) * C::kD;
      *reinterpret_cast<uint4*>(b + d_off(r, col)) = make_uint4(dp[0], dp[1], dp[2], dp[3]);
      *reinterpret_cast<uint4*>(b + d_off(r, col + 8)) = make_uint4(dp[4], dp[5], dp[6], dp[7]);
    };
    uint32_t acc_phase = 0, red_phase = 0, xph = 0;
    for (int64_t t = 0; t < my_tiles; ++t) {
      const int64_t u0 = (blockIdx.x + t * gridDim.x) * kRows;
      const int64_t u = u0 + r;
      const bool valid = u < P;
      const int gbuf = (int)(t & 1);
      const float* gb = geo + gbuf * 15 * kRows;
      {
        const bool got = mbar_wait(&geo_full[gbuf], (uint32_t)((t >> 1) & 1), abort_flag, gerr);
        if (!__all_sync(0xffffffffu, got)) break;
      }
      float x[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x[c] = gb[c * kRows + r] + (gb[(3 + c) * kRows + r] + gb[(6 + c) * kRows + r]);
        x[3 + c] = gb[(9 + c) * kRows + r] + gb[(12 + c) * kRows + r];
      }
      float tpart = 0.f, gpart[3] = {0.f, 0.f, 0.f};
      bool ok = true;
      float sa = 1.f;                                  // FP8: dequantisation scale of this A row
      {
        // ---- operand of the first layer: [x_hi, x_lo, x_hi, 0 ...], this column
        // group's 8 of the row's 32 BF16 values in K-block 0 (BF16 in both forms)
        float xs[32];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const float hi = __bfloat162float(__float2bfloat16_rn(x[c]));
          xs[c] = hi;
          xs[6 + c] = __bfloat162float(__float2bfloat16_rn(x[c] - hi));
          xs[12 + c] = hi;
        }
#pragma unroll
        for (int k = 18; k < 32; ++k) xs[k] = 0.f;
        uint32_t q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float a = 0.f, b = 0.f;
#pragma unroll
          for (int gq = 0; gq < kGroups; ++gq)
            if (gq == cg) {
              a = xs[8 * gq + 2 * i];
              b = xs[8 * gq + 2 * i + 1];
            }
          q[i] = pack_bf16(a, b);
        }
        // columns [16, 32) of [0, H): free since the previous tile's last product
        tmem_st4(lane_addr + (uint32_t)(16 + 4 * cg), q);
        a_done(0);
      }
      // ---- the first layer (product -1), hidden layers and the reverse sweep
      for (int layer = -1; layer < 6; ++layer) {
        // reverse layers: this thread's silu'(z_{6 - layer}) of the first kPre
        // chunks is requested before the product completes (the slot was written
        // two to four products earlier, so the loads' latency hides behind the
        // MMA); chunk j + kPre is requested while chunk j is processed
        constexpr int kPre = C::kChunks < 2 ? C::kChunks : 2;
        const uint8_t* dsl = layer == 3 ? sD3 : sD + (size_t)(layer >= 3 ? 5 - layer : 0) * C::kD;
        uint4 dsv[2 * kPre];
        if (layer >= 3) {
#pragma unroll
          for (int j = 0; j < kPre; ++j) {
            dsv[2 * j] = *reinterpret_cast<const uint4*>(dsl + d_off(r, ccol(j)));
            dsv[2 * j + 1] = *reinterpret_cast<const uint4*>(dsl + d_off(r, ccol(j) + 8));
          }
        }
        const bool got = mbar_wait(acc_ready, acc_phase, abort_flag, gerr);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        acc_phase ^= 1;
        tc_after();
        const uint32_t acc = lane_addr + (uint32_t)((layer & 1) * H);   // this product's accumulator
        // FP8: dequantisation of the accumulator, (row scale) x (column scale); the
        // first layer's BF16 product needs none
        const float* sw = wsc + (layer > 0 ? layer : 0) * H;
        const float sa_l = layer < 0 ? 0.f : sa;
        auto dq = [&](int c) { return layer < 0 ? 1.f : sa_l * sw[c]; };
        float inv = 1.f, sa_next = sa;
        if constexpr (F8) {
          if (layer == -1 || layer == 0 || layer == 1 || layer == 3 || layer == 4) {
            // bound of the row for the next A operand (silu(z) forward, delta backward)
            const float* bias = pb + layer * H;
            float m = layer <= 1 ? 0.2785f : 1e-30f;
            for (int j = 0; j < C::kChunks; ++j) {
              const int col = ccol(j);
              float v[kCc];
              tmem_ld16f(acc + col, v);
              tmem_wait_ld();
              if (layer <= 1) {
#pragma unroll
                for (int i = 0; i < kCc; ++i) m = fmaxf(m, 2.f * fmaf(v[i] * dq(col + i), 0.5f, bias[col + i]));
              } else {
#pragma unroll
                for (int i = 0; i < kCc; ++i) m = fmaxf(m, 1.1f * fabsf(v[i] * dq(col + i)));
              }
            }
            const bool got2 = group_max(m, xch, &xbar[g], xph, cg, r, abort_flag, gerr);
            if (!__all_sync(0xffffffffu, got2)) { ok = false; break; }
            inv = 448.f / m;
            sa_next = m / 448.f;
          } else if (layer == 2) {
            inv = 1.f / s4;
            sa_next = s4;
          }
        }
        // chunk j + 1 is read from TMEM while chunk j is processed (two register
        // buffers; tcgen05.wait::ld at the end of chunk j waits for that one read)
        float vb[2][kCc];
        tmem_ld16f(acc + ccol(0), vb[0]);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < C::kChunks; ++j) {
          const int col = ccol(j);
          if (j + 1 < C::kChunks) tmem_ld16f(acc + ccol(j + 1), vb[(j + 1) & 1]);
          float* v = vb[j & 1];
          if constexpr (F8) {
#pragma unroll
            for (int i = 0; i < kCc; ++i) v[i] *= dq(col + i);
          }
          float o[kCc];                                // next A operand values (unscaled)
          if (layer < 3) {
            // forward layers 1 .. 4; pb - H is b1 / 2
            const float* bias = pb + layer * H;
            uint32_t dp[kCc / 2];
#pragma unroll
            for (int i = 0; i < kCc; i += 4) {
              const float4 b4 = *reinterpret_cast<const float4*>(bias + col + i);
              uint64_t hh[2], dd2[2];
              silu_half(f2fma(f2pack(v[i], v[i + 1]), kHalf2, f2pack(b4.x, b4.y)), hh[0], dd2[0]);
              silu_half(f2fma(f2pack(v[i + 2], v[i + 3]), kHalf2, f2pack(b4.z, b4.w)), hh[1], dd2[1]);
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int ii = i + 2 * q;
                float h0, h1;
                f2unpack(hh[q], h0, h1);
                if (layer == 2) {
                  const uint64_t w = *reinterpret_cast<const uint64_t*>(pw5 + col + ii);
                  float w0, w1;
                  f2unpack(w, w0, w1);
                  tpart = fmaf(w0, h0, fmaf(w1, h1, tpart));
                  f2unpack(f2mul(w, dd2[q]), o[ii], o[ii + 1]);          // delta4
                } else {
                  float d0, d1;
                  f2unpack(dd2[q], d0, d1);
                  o[ii] = h0;
                  o[ii + 1] = h1;
                  dp[ii / 2] = pack_bf16(d0, d1);
                }
              }
            }
            if (layer < 2) put_d(layer + 2, col, dp);  // silu'(z1), silu'(z2), silu'(z3)
          } else {
            // reverse sweep: delta_{l-1} = acc * silu'(z_{l-1})
            const int sl = j % kPre;
            const uint32_t dd[8] = {dsv[2 * sl].x, dsv[2 * sl].y, dsv[2 * sl].z, dsv[2 * sl].w,
                                    dsv[2 * sl + 1].x, dsv[2 * sl + 1].y, dsv[2 * sl + 1].z, dsv[2 * sl + 1].w};
            if (j + kPre < C::kChunks) {
              dsv[2 * sl] = *reinterpret_cast<const uint4*>(dsl + d_off(r, ccol(j + kPre)));
              dsv[2 * sl + 1] = *reinterpret_cast<const uint4*>(dsl + d_off(r, ccol(j + kPre) + 8));
            }
#pragma unroll
            for (int i = 0; i < kCc; i += 2)
              f2unpack(f2mul(f2pack(v[i], v[i + 1]), f2pack(bf16_lo(dd[i / 2]), bf16_hi(dd[i / 2]))), o[i],
                       o[i + 1]);
            if (layer == 5) {
              // dtau/dx_s: W1[:, :3]^T delta1, column pairs in two lanes
              uint64_t g2[3] = {0, 0, 0};
#pragma unroll
              for (int i = 0; i < kCc; i += 2) {
                const uint64_t e2 = f2pack(o[i], o[i + 1]);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                  g2[c] = f2fma(*reinterpret_cast<const uint64_t*>(pW1 + c * H + col + i), e2, g2[c]);
              }
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                float a, b;
                f2unpack(g2[c], a, b);
                gpart[c] += 2.f * (a + b);                 // W1 is kept halved
              }
            }
          }
          if (layer < 5) {
            put_a(acc, col, o, inv);
            if ((j + 1) % C::kCpk == 0) a_done(j / C::kCpk);
          }
          if (j + 1 < C::kChunks) tmem_wait_ld();
        }
        if (!ok) break;
        sa = sa_next;
      }
      if (!ok) break;
      // combine the column groups of each row (fixed order) and write T, dT/dx:
      // the partial sums go through accumulator columns [4 cg, 4 cg + 4) of
      // [0, H), last read by the product-4 epilogue and next written by the next
      // tile's first product (after every warp's layer-1 arrivals)
      const uint32_t red_addr = lane_addr;
      {
        const uint32_t pr[4] = {__float_as_uint(tpart), __float_as_uint(gpart[0]), __float_as_uint(gpart[1]),
                                __float_as_uint(gpart[2])};
        tmem_st4(red_addr + (uint32_t)(4 * cg), pr);
        tmem_wait_st();
      }
      tc_before();
      mbar_arrive(red_ready);
      const bool got = mbar_wait(red_ready, red_phase, abort_flag, gerr);
      red_phase ^= 1;
      if (!__all_sync(0xffffffffu, got)) break;
      tc_after();
      float part[16];
      if (cg == 0) {
        tmem_ld16f(red_addr, part);
        tmem_wait_ld();
      }
      if (cg == 0 && valid) {
        float dtau = part[0];
        float gt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) gt[c] = part[1 + c];
#pragma unroll
        for (int q = 1; q < kGroups; ++q) {
          dtau += part[4 * q];
#pragma unroll
          for (int c = 0; c < 3; ++c) gt[c] += part[4 * q + 1 + c];
        }
        PairGeo pg;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pg.shi[c] = gb[c * kRows + r];
          pg.slo[c] = gb[(3 + c) * kRows + r];
          pg.soff[c] = gb[(6 + c) * kRows + r];
          pg.rhi[c] = gb[(9 + c) * kRows + r];
          pg.rlo[c] = gb[(12 + c) * kRows + r];
        }
        df32 d[3];
        const df32 rr = geometry(pg, d);
        const df32 T = df_add_f(df_mul_f(rr, net.b5), rr.hi * dtau);
        out.T2[u] = make_float2(T.hi, T.lo);
        if (out.J) {
          const float tau = net.b5 + dtau;
          const float f = tau / rr.hi;
          out.J[u] = make_float4(f * d[0].hi + rr.hi * gt[0], f * d[1].hi + rr.hi * gt[1],
                                 f * d[2].hi + rr.hi * gt[2], 0.f);
        }
      }
      mbar_arrive(&geo_empty[gbuf]);       // this tile's geometry buffer may be refilled
    }
  }
  tc_before();
  __syncthreads();
  tc_after();
  __syncwarp();
  if (warp == kEpiWarps + 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::kTmemCols));
}

template <int H, bool F8>
cudaError_t launch_tc(const NetView& net, const PairSource& src, TTOut out, int num_sms, float* scratch,
                      cudaStream_t st) {
  using C = Cfg<H, F8>;
  cudaError_t e = cudaFuncSetAttribute(k_tt_mlp_tc<H, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  if (e != cudaSuccess) return e;
  k_tt_mlp_tc<H, F8><<<num_sms, kTcThreads, C::kSmem, st>>>(net, src, out, (const uint8_t*)net.tc, net.err,
                                                             reinterpret_cast<uint8_t*>(scratch));
  return cudaGetLastError();
}

}  // namespace

bool mlp_tc_supported(int H, int precision) {
  if (precision == SPIDER_BF16) return H == 64 || H == 128 || H == 256;
  if (precision == SPIDER_FP8) return H == 128 || H == 256;
  return false;
}

// Weight images for the B operand, in the order the MMA consumes them:
// W2, W3, W4 (forward: B[n][k] = W[n][k]) then W4^T, W3^T, W2^T (reverse:
// B[n][k] = W[k][n]); each image is K-blocks of H rows x 128 bytes (64 BF16 or
// 128 E4M3 elements) in the 128-byte-swizzled K-major layout the shared-memory
// descriptor names.  FP8: every row n of an image is divided by its scale
// max_k |B[n][k]| / 448 before rounding; `scales` receives the 6 H column
// scales followed by the scale of delta4, 1.1 max |w5| / 448.
cudaError_t mlp_tc_prepare(const float* W1_host, const float* const Wn_host[3], const float* w5_host, int H,
                           int precision, void** image, float** scales, cudaStream_t st) {
  *image = nullptr;
  *scales = nullptr;
  if (!mlp_tc_supported(H, precision)) return cudaErrorNotSupported;
  const bool f8 = precision == SPIDER_FP8;
  const int eb = f8 ? 1 : 2;
  const size_t img = (size_t)H * H * eb;
  // the first layer's split BF16 image (one K-block, H rows x 128 B) in front
  const size_t pre = (size_t)H * 128;
  std::vector<uint8_t> host(pre + 6 * img, 0);
  std::vector<float> sc(f8 ? 6 * H + 1 : 0, 1.f);
  // byte offset of (row n, k) in a K-block-major SW128 image of e-byte elements
  auto sw_off_e = [H](int n, int k, int e) {
    const int per = 128 / e, kb = k / per, j = (k % per) / (16 / e);
    return (size_t)kb * H * 128 + (size_t)(n / 8) * 1024 + (size_t)(n % 8) * 128 + (size_t)((j ^ (n % 8)) * 16) +
           (size_t)(k % (16 / e)) * e;
  };
  auto sw_off = [&](int n, int k) { return sw_off_e(n, k, eb); };
  {
    // B[n][k]: W_hi (k < 6), W_hi (6 <= k < 12), W_lo (12 <= k < 18), 0 above,
    // BF16 in both forms (2-byte elements, K-blocks of 64)
    for (int n = 0; n < H; ++n)
      for (int c = 0; c < 6; ++c) {
        const float w = W1_host[(size_t)n * 6 + c];
        const uint16_t hi = to_bf16(w);
        float whi;
        const uint32_t hb = (uint32_t)hi << 16;
        std::memcpy(&whi, &hb, 4);
        const uint16_t lo = to_bf16(w - whi);
        std::memcpy(host.data() + sw_off_e(n, c, 2), &hi, 2);
        std::memcpy(host.data() + sw_off_e(n, 6 + c, 2), &hi, 2);
        std::memcpy(host.data() + sw_off_e(n, 12 + c, 2), &lo, 2);
      }
  }
  for (int l = 0; l < 6; ++l) {
    const float* W = Wn_host[l < 3 ? l : 5 - l];
    const bool transpose = l >= 3;
    uint8_t* base = host.data() + pre + l * img;
    for (int n = 0; n < H; ++n) {
      float inv = 1.f;
      if (f8) {
        float m = 0.f;
        for (int k = 0; k < H; ++k) m = std::fmax(m, std::fabs(transpose ? W[(size_t)k * H + n] : W[(size_t)n * H + k]));
        const float scale = m > 0.f ? m / 448.f : 1.f;
        sc[(size_t)l * H + n] = scale;
        inv = 1.f / scale;
      }
      for (int k = 0; k < H; ++k) {
        const float v = transpose ? W[(size_t)k * H + n] : W[(size_t)n * H + k];
        const size_t off = sw_off(n, k);
        if (f8) {
          base[off] = to_e4m3(v * inv);
        } else {
          const uint16_t b = to_bf16(v);
          std::memcpy(base + off, &b, 2);
        }
      }
    }
  }
  if (f8) {
    float m = 0.f;
    for (int i = 0; i < H; ++i) m = std::fmax(m, std::fabs(w5_host[i]));
    sc[6 * H] = m > 0.f ? 1.1f * m / 448.f : 1.f;
  }
  void* d = nullptr;
  float* ds = nullptr;
  cudaError_t e = cudaMalloc(&d, host.size());
  if (e != cudaSuccess) return e;
  if (f8 && (e = cudaMalloc(&ds, sc.size() * sizeof(float))) != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  e = cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && f8) e = cudaMemcpyAsync(ds, sc.data(), sc.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(d);
    if (ds) cudaFree(ds);
    return e;
  }
  *image = d;
  *scales = ds;
  return cudaSuccess;
}

// scratch: num_sms x 3 x 128 x H BF16 (the silu'(z1..3) slots), see tt_scratch_floats
cudaError_t launch_mlp_tc(const NetView& net, const PairSource& src, TTOut out, int num_sms, float* scratch,
                          cudaStream_t st) {
  if (!net.tc || !net.err || !scratch) return cudaErrorNotSupported;
  if (net.precision == SPIDER_FP8) {
    if (!net.tc_scale) return cudaErrorNotSupported;
    switch (net.H) {
      case 128: return launch_tc<128, true>(net, src, out, num_sms, scratch, st);
      case 256: return launch_tc<256, true>(net, src, out, num_sms, scratch, st);
      default: return cudaErrorNotSupported;
    }
  }
  if (net.precision != SPIDER_BF16) return cudaErrorNotSupported;
  switch (net.H) {
    case 64: return launch_tc<64, false>(net, src, out, num_sms, scratch, st);
    case 128: return launch_tc<128, false>(net, src, out, num_sms, scratch, st);
    case 256: return launch_tc<256, false>(net, src, out, num_sms, scratch, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace spider
