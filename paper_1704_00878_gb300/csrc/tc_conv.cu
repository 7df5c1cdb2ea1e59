// tc_conv.cu -- the selector's 9-tap convolutions as implicit GEMMs on the
// fifth-generation tensor cores (tcgen05.mma, bf16 operands, fp32
// accumulators in tensor memory), every operand tile brought into shared
// memory by TMA.
//
// For tap t the A operand of an output tile starting at row r0 is rows
// r0 - 4 + t .. of the input, i.e. the same tile plus an 8-row halo shifted
// by t rows, so a CTA loads it once (TMA, 128-byte swizzle for 64 or 128
// channels, 64-byte swizzle for 32; rows outside the batch read as zeros)
// and points the MMA's shared-memory descriptor t rows further for each tap.
// The B operand (output channels' weights of all 9 taps) stays resident in
// shared memory for the CTA's whole life.  Warp roles:
//   warp 0   TMA producer: input tiles into two buffers,
//   warp 1   MMA issuer: 9 x (CIN / 16) MMAs per tile into one of two
//            accumulators in tensor memory, committed to mbarriers that free
//            the input buffer and hand the accumulator to the epilogue,
//   the rest epilogue: each warp reads the accumulator rows its warp may
//            address (tcgen05.ld 32x32b), hands the accumulator back, adds
//            the bias, applies the mode's activation or mask and stores
//            bf16 / fp32 rows,
// so the epilogue of tile i runs under the MMAs of tile i + 1 and the load
// of tile i + 2.
//
// k_conv_tc2 (every convolution of the network) runs this on CTA pairs with
// tcgen05.mma.cta_group::2 (M 256 per instruction, the weights split across
// the pair); k_conv_tc, the single-CTA form (M 128 x N 64), remains for the
// self-test of the bounded waits.  k_wgrad_tc computes the weight gradient.
//
// Every wait on an mbarrier gives up after a bounded number of polls, sets
// bit MSA_DERR_TIMEOUT_TC of the caller's error word and ends the role;
// tensor memory is released on every path.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "net_kernels.cuh"

namespace net {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int TBM = 128;               // output rows per tile
constexpr int TBN = 64;                // output channels per CTA
constexpr int AROWS = TBM + 2 * HALF;  // 136 staged input rows
constexpr int TC_THREADS = 192;        // producer, MMA, 4 epilogue warps
constexpr long long kSpinLimit = 1ll << 26;  // polls before a wait gives up

// Shared-memory geometry of one input width: rows of ROWB bytes (128 with
// the 128-byte swizzle for 64 / 128 channels, 64 with the 64-byte swizzle
// for 32), KB blocks of BLK channels across the reduction.
template <int CIN> struct Geo {
  static constexpr int ROWB = CIN >= 64 ? 128 : 64;
  static constexpr int BLK = ROWB / 2;
  static constexpr int KB = CIN / BLK;
  static constexpr int A_BLOCK = AROWS * ROWB;  // one block of the A tile
  static constexpr int A_BYTES = (KB * A_BLOCK + 1023) / 1024 * 1024;
};

// the single-CTA kernel's weights: TBN output channels per CTA
template <int CIN> struct SoloGeo : Geo<CIN> {
  static constexpr int B_BLOCK = TBN * Geo<CIN>::ROWB;               // one block of one tap's weights
  static constexpr int W_BYTES = TAPS * Geo<CIN>::KB * B_BLOCK;      // resident weights
  static constexpr int SMEM = W_BYTES + 2 * Geo<CIN>::A_BYTES + 1024;  // + alignment slack
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_relaxed(uint32_t bar) {
  asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// true once the phase with the given parity has completed; false after
// `spins` polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long spins) {
  for (long long i = 0; i < spins; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in a swizzled layout
// (rows of ROWB bytes, 8-row groups 8 * ROWB bytes apart).  Fields: start
// address >> 4 [0,14), leading-dimension offset >> 4 [16,30) (unused by
// these layouts, 1), stride-dimension offset >> 4 [32,46), descriptor
// version 1 [46,48), base offset [49,52) left 0, layout type [61,64) = 2
// (128-byte swizzle) or 4 (64-byte swizzle).  The swizzle phase of a row
// follows its shared-memory address (as for the TMA that wrote it), so a
// start address t rows into an aligned tile reads rows t, t+1, ... as
// written.
template <int ROWB>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3fff);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * ROWB) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(ROWB == 128 ? 2 : 4) << 61;
  return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator [4,6) = 1, A and B
// bf16 [7,10) = [10,13) = 1, both K-major (bits 15, 16 clear), N >> 3 at
// [17,23), M >> 4 at [24,29).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// arrive on the mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 32 consecutive fp32 accumulator columns of this warp's 32 rows
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive fp32 accumulator columns of this warp's 32 rows, one
// load and one wait
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}


__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// barrier slots in shared memory
enum { B_W = 0, B_AFULL = 1, B_AEMPTY = 3, B_CFULL = 5, B_CEMPTY = 7, NBARS = 9 };

// mode 0: relu(x * W + b) -> bf16; mode 1: x * W + b -> fp32; mode 2: data
// gradient (taps reversed, no bias) masked by prev > 0 -> bf16.  Rows whose
// rowseq is negative (padding between sequences) are written as zero.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_conv_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap,
          const float *__restrict__ bias, const int32_t *__restrict__ rowseq,
          const bf16 *__restrict__ prev, void *__restrict__ y, int T, unsigned *err,
          long long spins, int no_loads) {
  using Gm = SoloGeo<CIN>;
  constexpr int NH = COUT / TBN;  // output-channel slices
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) unsigned long long bars[NBARS];
  __shared__ float s_bias[TBN];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw = smem_u32(tc_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t sW = base;
  const uint32_t sA0 = base + Gm::W_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = (int)(blockIdx.x % NH);
  const int stride = (int)(gridDim.x / NH);
  const int first = (int)(blockIdx.x / NH);
  const int ntiles = (T + TBM - 1) / TBM;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  if (tid == 0) {
    mbar_init(bar(B_W), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_AFULL + b), 1);
      mbar_init(bar(B_AEMPTY + b), 1);
      mbar_init(bar(B_CFULL + b), 1);
      mbar_init(bar(B_CEMPTY + b), 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (tid < TBN) s_bias[tid] = MODE == 2 ? 0.f : bias[half * TBN + tid];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * TBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0 && first < ntiles && !no_loads) {
      mbar_expect_tx(bar(B_W), (uint32_t)Gm::W_BYTES);
      for (int t = 0; t < TAPS; ++t)
        for (int kb = 0; kb < Gm::KB; ++kb)
          tma_load_2d(sW + (uint32_t)((t * Gm::KB + kb) * Gm::B_BLOCK), &wmap, kb * Gm::BLK,
                      t * COUT + half * TBN, bar(B_W));
      int issued = 0;
      for (int it = 0, tile = first; tile < ntiles && ok; tile += stride, ++it) {
        const int b = it & 1, k = it >> 1;
        if (k > 0 && !mbar_wait(bar(B_AEMPTY + b), (uint32_t)((k - 1) & 1), spins)) { ok = false; break; }
        const uint32_t sA = sA0 + (uint32_t)(b * Gm::A_BYTES);
        mbar_expect_tx(bar(B_AFULL + b), (uint32_t)(Gm::KB * Gm::A_BLOCK));
        for (int kb = 0; kb < Gm::KB; ++kb)
          tma_load_2d(sA + (uint32_t)(kb * Gm::A_BLOCK), &xmap, kb * Gm::BLK, tile * TBM - HALF,
                      bar(B_AFULL + b));
        ++issued;
      }
      // no copy may still be landing when the CTA exits: wait (bounded) for
      // the weights and the last load into each buffer (at once if landed)
      mbar_wait(bar(B_W), 0, spins);
      for (int it = issued - 2; it < issued; ++it)
        if (it >= 0) mbar_wait(bar(B_AFULL + (it & 1)), (uint32_t)((it >> 1) & 1), spins);
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0 && first < ntiles) {
      int last = -1;
      if (!mbar_wait(bar(B_W), 0, spins)) ok = false;
      for (int it = 0, tile = first; ok && tile < ntiles; tile += stride, ++it) {
        const int b = it & 1, k = it >> 1;
        if (!mbar_wait(bar(B_AFULL + b), (uint32_t)(k & 1), spins)) { ok = false; break; }
        if (k > 0 && !mbar_wait(bar(B_CEMPTY + b), (uint32_t)((k - 1) & 1), spins)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sA = sA0 + (uint32_t)(b * Gm::A_BYTES);
        const uint32_t acc = tmem + (uint32_t)(b * TBN);
#pragma unroll 1
        for (int t = 0; t < TAPS; ++t) {
          const int wt = MODE == 2 ? TAPS - 1 - t : t;
#pragma unroll
          for (int kb = 0; kb < Gm::KB; ++kb) {
#pragma unroll
            for (int kk = 0; kk < Gm::BLK / 16; ++kk) {
              const uint64_t ad = smem_desc<Gm::ROWB>(sA + (uint32_t)(kb * Gm::A_BLOCK + t * Gm::ROWB + kk * 32));
              const uint64_t bd = smem_desc<Gm::ROWB>(sW + (uint32_t)((wt * Gm::KB + kb) * Gm::B_BLOCK + kk * 32));
              umma_bf16(acc, ad, bd, (t | kb | kk) != 0 ? 1u : 0u);
            }
          }
        }
        umma_commit(bar(B_AEMPTY + b));
        umma_commit(bar(B_CFULL + b));
        last = it;
      }
      // and no MMA may still be running: the last commit's barrier (bounded)
      if (last >= 0) mbar_wait(bar(B_AEMPTY + (last & 1)), (uint32_t)((last >> 1) & 1), spins);
    }
  } else {
    // ---- epilogue: warp w addresses accumulator rows 32 (w % 4) .. + 31
    const int q = warp & 3;
    for (int it = 0, tile = first; tile < ntiles; tile += stride, ++it) {
      const int b = it & 1, k = it >> 1;
      if (!mbar_wait(bar(B_CFULL + b), (uint32_t)(k & 1), spins)) { ok = false; break; }
      tc_fence_after();
      const int r = tile * TBM + q * 32 + lane;
      const bool inb = r < T;
      const bool valid = inb && (rowseq == nullptr || rowseq[r] >= 0);
      // the row slice into registers, then the accumulator goes back to the
      // issuer before any store
      float v[TBN / 32][32];
#pragma unroll
      for (int c = 0; c < TBN / 32; ++c)
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TBN + 32 * c), v[c]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_relaxed(bar(B_CEMPTY + b));
      if (!inb) continue;
#pragma unroll
      for (int c = 0; c < TBN / 32; ++c) {
        const int c0 = 32 * c;
        const int cb = half * TBN + c0;
        if constexpr (MODE == 1) {
          float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(y) + (size_t)r * COUT + cb);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float4 o;
            o.x = valid ? v[c][4 * j] + s_bias[c0 + 4 * j] : 0.f;
            o.y = valid ? v[c][4 * j + 1] + s_bias[c0 + 4 * j + 1] : 0.f;
            o.z = valid ? v[c][4 * j + 2] + s_bias[c0 + 4 * j + 2] : 0.f;
            o.w = valid ? v[c][4 * j + 3] + s_bias[c0 + 4 * j + 3] : 0.f;
            dst[j] = o;
          }
        } else {
          uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(y) + (size_t)r * COUT + cb);
          const uint4 *pv = MODE == 2 ? reinterpret_cast<const uint4 *>(prev + (size_t)r * COUT + cb) : nullptr;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t w[4];
            uint4 pm = make_uint4(0u, 0u, 0u, 0u);
            if constexpr (MODE == 2) pm = pv[j];
            const uint32_t pw[4] = {pm.x, pm.y, pm.z, pm.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int cc = 8 * j + 2 * h;
              float a = v[c][cc], bb = v[c][cc + 1];
              if constexpr (MODE == 0) {
                a = valid ? fmaxf(a + s_bias[c0 + cc], 0.f) : 0.f;
                bb = valid ? fmaxf(bb + s_bias[c0 + cc + 1], 0.f) : 0.f;
              } else {
                const __nv_bfloat162 p2 = *reinterpret_cast<const __nv_bfloat162 *>(&pw[h]);
                a = valid && __bfloat162float(p2.x) > 0.f ? a : 0.f;
                bb = valid && __bfloat162float(p2.y) > 0.f ? bb : 0.f;
              }
              const __nv_bfloat162 o2 = __floats2bfloat162_rn(a, bb);
              w[h] = *reinterpret_cast<const uint32_t *>(&o2);
            }
            dst[j] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
    }
  }
  if (!ok) atomicOr(err, MSA_DERR_TIMEOUT_TC);
  // every role has returned: the last MMAs and loads completed before the
  // epilogue (or timed out above); free tensor memory
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TBN));
}

// ---------------------------------------------------------------- CTA-pair convolution
// Every convolution of the network also runs on CTA pairs: a cluster of two
// CTAs on two SMs computes 256 positions x COUT (64 or 128) channels per
// tile with tcgen05.mma.cta_group::2 (M 256, N COUT, K 16).  CTA rank r
// stages rows 256 tile + 128 r - 4 .. + 135 of the input (A rows 128 r ..
// 128 r + 127 of the MMA) and the weights of output channels COUT / 2 r ..
// + COUT / 2 - 1 (its half of B), at the same shared-memory offsets in both
// CTAs; the even CTA issues every MMA, and each CTA's tensor memory
// receives the accumulator rows of its own positions for all COUT
// channels.  One instruction drives both SMs' tensor cores, and each CTA
// keeps only half the weights.
//   even CTA: warp 0 TMA of its tiles, warp 1 MMA issuer, warps 2-9 epilogue
//   odd CTA:  warp 0 TMA of its tiles, relaying each landed load to the even
//             CTA's barrier; warps 2-9 epilogue
// Epilogue warps w and w + 4 share tensor-memory lanes 32 (w % 4) .. + 31
// and take one half of the channels each.  Barriers (same offsets in both
// CTAs): W and AFULL count the even CTA's own expect_tx arrival plus the odd
// CTA's relay; AEMPTY and CFULL are signalled in both CTAs by the multicast
// commit of the MMAs; CEMPTY (even CTA) counts the sixteen epilogue warps of
// the pair.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the shared::cluster address of this CTA's shared variable at `saddr` in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// mbar_wait with cluster-scope acquire: the barriers of the pair kernel are
// also signalled from the other CTA (relayed arrivals, multicast commits)
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, long long spins) {
  for (long long i = 0; i < spins; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// no memory ordering: for handing back an accumulator whose tensor-memory
// reads have completed (tcgen05.wait::ld) and been fenced
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

// kind::f16, fp32 accumulator, bf16 A and B, K-major, N = COUT, M 256 (the pair)
template <int COUT>
__host__ __device__ constexpr uint32_t pair_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(COUT >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

template <int COUT>
__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p; }"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(pair_idesc<COUT>()), "r"(accumulate)
      : "memory");
}

// arrive once on the mbarrier at `bar` in both CTAs of the pair when every
// MMA issued before has completed
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
      ::"r"(bar), "h"((unsigned short)3)
      : "memory");
}

constexpr int PAIR_TBM = 2 * TBM;  // positions per pair tile
// the pair kernel's warps: TMA producer, MMA issuer, eight epilogue warps
// (two per 32-lane quarter of tensor memory, each taking half the channels)
constexpr int PAIR_THREADS = 320;

// Shared-memory geometry of the pair kernel: the input tile as in Geo, and
// each CTA's half of the output channels' weights (BN = COUT / 2 rows).
template <int CIN, int COUT> struct PairGeo {
  using G = Geo<CIN>;
  static constexpr int BN = COUT / 2;
  static constexpr int B_BLOCK = BN * G::ROWB;
  static constexpr int W_BYTES = TAPS * G::KB * B_BLOCK;
  static constexpr int SMEM = W_BYTES + 2 * G::A_BYTES + 1024;
  static constexpr int TMEM = 2 * COUT;  // two accumulators
};

template <int CIN, int COUT, int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PAIR_THREADS, 1)
k_conv_tc2(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap wmap,
           const float *__restrict__ bias, const int32_t *__restrict__ rowseq,
           const bf16 *__restrict__ prev, void *__restrict__ y, int T, unsigned *err,
           long long spins) {
  using Gm = Geo<CIN>;
  using Pg = PairGeo<CIN, COUT>;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) unsigned long long bars[NBARS];
  __shared__ float s_bias[COUT];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw = smem_u32(tc_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t sW = base;
  const uint32_t sA0 = base + Pg::W_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const bool even = rank == 0;
  const int first = (int)(blockIdx.x >> 1), stride = (int)(gridDim.x >> 1);
  const int ntiles = (T + PAIR_TBM - 1) / PAIR_TBM;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  if (tid == 0) {
    mbar_init(bar(B_W), even ? 2 : 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_AFULL + b), even ? 2 : 1);
      mbar_init(bar(B_AEMPTY + b), 1);
      mbar_init(bar(B_CFULL + b), 1);
      mbar_init(bar(B_CEMPTY + b), 16);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (tid < COUT) s_bias[tid] = MODE == 2 ? 0.f : bias[tid];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(Pg::TMEM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  // both CTAs' barriers are initialised before either signals the other's
  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;

  if (warp == 0) {
    // ---- TMA producer (both CTAs): own tiles into own shared memory
    if (lane == 0 && first < ntiles) {
      mbar_expect_tx(bar(B_W), (uint32_t)Pg::W_BYTES);
      for (int t = 0; t < TAPS; ++t)
        for (int kb = 0; kb < Gm::KB; ++kb)
          tma_load_2d(sW + (uint32_t)((t * Gm::KB + kb) * Pg::B_BLOCK), &wmap, kb * Gm::BLK,
                      t * COUT + (int)rank * Pg::BN, bar(B_W));
      int issued = 0;
      for (int it = 0, tile = first; tile < ntiles && ok; tile += stride, ++it) {
        const int b = it & 1, k = it >> 1;
        if (k > 0 && !mbar_wait_cl(bar(B_AEMPTY + b), (uint32_t)((k - 1) & 1), spins)) { ok = false; break; }
        const uint32_t sA = sA0 + (uint32_t)(b * Gm::A_BYTES);
        mbar_expect_tx(bar(B_AFULL + b), (uint32_t)(Gm::KB * Gm::A_BLOCK));
        for (int kb = 0; kb < Gm::KB; ++kb)
          tma_load_2d(sA + (uint32_t)(kb * Gm::A_BLOCK), &xmap, kb * Gm::BLK,
                      tile * PAIR_TBM + (int)rank * TBM - HALF, bar(B_AFULL + b));
        ++issued;
        if (!even) {
          // relay: once this CTA's weights and tile have landed, arrive on
          // the even CTA's barriers
          if (it == 0) {
            if (!mbar_wait_cl(bar(B_W), 0, spins)) { ok = false; break; }
            mbar_arrive_cluster(peer_addr(bar(B_W), 0));
          }
          if (!mbar_wait_cl(bar(B_AFULL + b), (uint32_t)(k & 1), spins)) { ok = false; break; }
          mbar_arrive_cluster(peer_addr(bar(B_AFULL + b), 0));
        }
      }
      if (even) {
        // no copy may still be landing when the CTA exits (bounded)
        mbar_wait_cl(bar(B_W), 0, spins);
        for (int it = issued - 2; it < issued; ++it)
          if (it >= 0) mbar_wait_cl(bar(B_AFULL + (it & 1)), (uint32_t)((it >> 1) & 1), spins);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer (even CTA)
    if (even && lane == 0 && first < ntiles) {
      int last = -1;
      if (!mbar_wait_cl(bar(B_W), 0, spins)) ok = false;
      for (int it = 0, tile = first; ok && tile < ntiles; tile += stride, ++it) {
        const int b = it & 1, k = it >> 1;
        if (!mbar_wait_cl(bar(B_AFULL + b), (uint32_t)(k & 1), spins)) { ok = false; break; }
        if (k > 0 && !mbar_wait_cl(bar(B_CEMPTY + b), (uint32_t)((k - 1) & 1), spins)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sA = sA0 + (uint32_t)(b * Gm::A_BYTES);
        const uint32_t acc = tmem + (uint32_t)(b * COUT);
#pragma unroll 1
        for (int t = 0; t < TAPS; ++t) {
          const int wt = MODE == 2 ? TAPS - 1 - t : t;
#pragma unroll
          for (int kb = 0; kb < Gm::KB; ++kb) {
#pragma unroll
            for (int kk = 0; kk < Gm::BLK / 16; ++kk) {
              const uint64_t ad = smem_desc<Gm::ROWB>(sA + (uint32_t)(kb * Gm::A_BLOCK + t * Gm::ROWB + kk * 32));
              const uint64_t bd = smem_desc<Gm::ROWB>(sW + (uint32_t)((wt * Gm::KB + kb) * Pg::B_BLOCK + kk * 32));
              umma_pair<COUT>(acc, ad, bd, (t | kb | kk) != 0 ? 1u : 0u);
            }
          }
        }
        umma_commit_pair(bar(B_AEMPTY + b));
        umma_commit_pair(bar(B_CFULL + b));
        last = it;
      }
      // no MMA may still be running: the last commit's barrier (bounded)
      if (last >= 0) mbar_wait_cl(bar(B_AEMPTY + (last & 1)), (uint32_t)((last >> 1) & 1), spins);
    }
  } else {
    // ---- epilogue (both CTAs): warp w reads accumulator rows 32 (w % 4) ..
    // + 31 of this CTA's tensor memory, channels hh * COUT / 2 .. + COUT / 2
    // (hh = 0 for warps 2-5, 1 for warps 6-9)
    constexpr int HC = COUT / 2;                      // channels per warp
    constexpr int OUTB = MODE == 1 ? 4 : 2;           // output bytes per channel
    constexpr int NCH = HC * OUTB / 16;               // 16-byte chunks per warp row
    const int q = warp & 3, hh = (warp - 2) >> 2;
    for (int it = 0, tile = first; tile < ntiles; tile += stride, ++it) {
      const int b = it & 1, k = it >> 1;
      if (!mbar_wait_cl(bar(B_CFULL + b), (uint32_t)(k & 1), spins)) { ok = false; break; }
      tc_fence_after();
      const int r = tile * PAIR_TBM + (int)rank * TBM + q * 32 + lane;
      const bool inb = r < T;
      const bool valid = inb && (rowseq == nullptr || rowseq[r] >= 0);
      // this warp's slice into registers (one load, one wait), then the
      // accumulator goes back to the issuer before any store
      float v[HC];
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * COUT + hh * HC);
      if constexpr (HC == 64) tmem_ld64(ta, v);
      else tmem_ld32(ta, v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster_relaxed(peer_addr(bar(B_CEMPTY + b), 0));
      if (!inb) continue;
      const int cb = hh * HC;  // first channel of this warp
      uint4 *dst = reinterpret_cast<uint4 *>(static_cast<unsigned char *>(y) + ((size_t)r * COUT + cb) * OUTB);
      const uint4 *pv = MODE == 2 ? reinterpret_cast<const uint4 *>(prev + (size_t)r * COUT + cb) : nullptr;
#pragma unroll
      for (int jc = 0; jc < NCH; ++jc) {
        if constexpr (MODE == 1) {
          const int e = 4 * jc;
          float4 o;
          o.x = valid ? v[e] + s_bias[cb + e] : 0.f;
          o.y = valid ? v[e + 1] + s_bias[cb + e + 1] : 0.f;
          o.z = valid ? v[e + 2] + s_bias[cb + e + 2] : 0.f;
          o.w = valid ? v[e + 3] + s_bias[cb + e + 3] : 0.f;
          dst[jc] = *reinterpret_cast<const uint4 *>(&o);
        } else {
          const int e = 8 * jc;
          uint4 pm = make_uint4(0u, 0u, 0u, 0u);
          if constexpr (MODE == 2) pm = pv[jc];
          [[maybe_unused]] const uint32_t pw[4] = {pm.x, pm.y, pm.z, pm.w};
          uint32_t w[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            float a = v[e + 2 * h], bb = v[e + 2 * h + 1];
            if constexpr (MODE == 0) {
              a = valid ? fmaxf(a + s_bias[cb + e + 2 * h], 0.f) : 0.f;
              bb = valid ? fmaxf(bb + s_bias[cb + e + 2 * h + 1], 0.f) : 0.f;
            } else {
              const __nv_bfloat162 p2 = *reinterpret_cast<const __nv_bfloat162 *>(&pw[h]);
              a = valid && __bfloat162float(p2.x) > 0.f ? a : 0.f;
              bb = valid && __bfloat162float(p2.y) > 0.f ? bb : 0.f;
            }
            const __nv_bfloat162 o2 = __floats2bfloat162_rn(a, bb);
            w[h] = *reinterpret_cast<const uint32_t *>(&o2);
          }
          dst[jc] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
  }
  if (!ok) atomicOr(err, MSA_DERR_TIMEOUT_TC);
  // both CTAs stay resident until every role of the pair has returned (the
  // even CTA's MMAs read the odd CTA's shared memory and write its tensor
  // memory); then the pair frees its tensor memory
  tc_fence_before();
  cluster_sync_all();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Pg::TMEM));
}

// ---------------------------------------------------------------- weight gradient
// dW[t][ci][co] += sum_r x[r + t - 4][ci] * dy[r][co] for 128 input channels.
// Per tap a GEMM with M = ci (128), N = co (COUT), K = the rows.  Both
// operands come straight from the row-major activations, so both are
// MN-major (channels contiguous, rows the reduction): TMA loads a chunk of
// 64 rows of dy and the same rows of x plus the halo of the CTA's taps, in
// the 128-byte swizzle, and tap t is again a start address t rows further.
// A CTA owns 3 taps (3 x COUT fp32 accumulator columns in TMEM) and a
// contiguous, 64-aligned range of rows, pipelined over 4 stages by a TMA
// warp and an MMA warp; at the end its four epilogue warps add the partial
// dW to global memory with fp32 atomics.
constexpr int WG_TAPS = 3;    // taps per CTA
constexpr int WG_KR = 64;     // rows per chunk
constexpr int WG_AROWS = 72;  // chunk + halo of 3 taps (66), rounded up to 8
constexpr int WG_STAGES = 4;

template <int COUT> struct WGeo {
  static constexpr int A_BLOCK = WG_AROWS * 128;  // one 64-channel block of x
  static constexpr int A_BYTES = 2 * A_BLOCK;     // 128 channels
  static constexpr int B_BLOCK = WG_KR * 128;     // one 64-channel block of dy
  static constexpr int B_BYTES = (COUT / 64) * B_BLOCK;
  static constexpr int STAGE = (A_BYTES + B_BYTES + 1023) / 1024 * 1024;
  static constexpr int SMEM = WG_STAGES * STAGE + 1024;
  static constexpr int TMEM_COLS = WG_TAPS * COUT <= 256 ? 256 : 512;
};

// MN-major operand in the 128-byte swizzle: 64-element MN blocks `lbo` bytes
// apart (leading-dimension offset), 8-row K groups 1024 bytes apart
// (stride-dimension offset), version 1, layout type 2.
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3fff);
  d |= (uint64_t)((lbo >> 4) & 0x3fff) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16, fp32 accumulator, bf16 A and B, both MN-major (bits 15, 16),
// N = COUT, M = 128
template <int COUT>
__host__ __device__ constexpr uint32_t wg_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(COUT >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

template <int COUT>
__device__ __forceinline__ void umma_wg(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(wg_idesc<COUT>()), "r"(accumulate)
      : "memory");
}

// grid: (row splits, 3 tap groups); rows [split * per, min(T, (split + 1) * per)), per % 64 == 0.
// CIN < 128 (the 32-channel one-hot input): the channels past CIN load as
// zeros (outside the tensor) and their accumulator rows are not written.
template <int CIN, int COUT>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_wgrad_tc(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dymap,
           float *__restrict__ dw, int T, int per, unsigned *err, long long spins) {
  using Gm = WGeo<COUT>;
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) unsigned long long bars[2 * WG_STAGES + 1];
  __shared__ uint32_t tmem_slot;
  const uint32_t raw = smem_u32(tc_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t0 = (int)blockIdx.y * WG_TAPS;
  const int r_begin = (int)blockIdx.x * per, r_end = min(T, r_begin + per);
  const int nchunks = r_end > r_begin ? (r_end - r_begin + WG_KR - 1) / WG_KR : 0;
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[WG_STAGES + s]); };
  const uint32_t done = smem_u32(&bars[2 * WG_STAGES]);
  if (tid == 0) {
    for (int s = 0; s < WG_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(Gm::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {
      for (int c = 0; c < nchunks && ok; ++c) {
        const int s = c % WG_STAGES, k = c / WG_STAGES;
        if (k > 0 && !mbar_wait(empty(s), (uint32_t)((k - 1) & 1), spins)) { ok = false; break; }
        const uint32_t sA = base + (uint32_t)(s * Gm::STAGE), sB = sA + Gm::A_BYTES;
        const int r0 = r_begin + c * WG_KR;
        mbar_expect_tx(full(s), (uint32_t)(Gm::A_BYTES + Gm::B_BYTES));
        for (int h = 0; h < 2; ++h)
          tma_load_2d(sA + (uint32_t)(h * Gm::A_BLOCK), &xmap, h * 64, r0 - HALF + t0, full(s));
        for (int h = 0; h < COUT / 64; ++h)
          tma_load_2d(sB + (uint32_t)(h * Gm::B_BLOCK), &dymap, h * 64, r0, full(s));
      }
      // the last loads of each stage land before the CTA may exit
      for (int c = max(0, nchunks - WG_STAGES); c < nchunks; ++c)
        mbar_wait(full(c % WG_STAGES), (uint32_t)((c / WG_STAGES) & 1), spins);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % WG_STAGES, k = c / WG_STAGES;
        if (!mbar_wait(full(s), (uint32_t)(k & 1), spins)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sA = base + (uint32_t)(s * Gm::STAGE), sB = sA + Gm::A_BYTES;
#pragma unroll
        for (int tl = 0; tl < WG_TAPS; ++tl) {
#pragma unroll
          for (int kk = 0; kk < WG_KR / 16; ++kk) {
            const uint64_t ad = mn_desc(sA + (uint32_t)((tl + 16 * kk) * 128), (uint32_t)Gm::A_BLOCK);
            const uint64_t bd = mn_desc(sB + (uint32_t)(16 * kk * 128), (uint32_t)Gm::B_BLOCK);
            umma_wg<COUT>(tmem + (uint32_t)(tl * COUT), ad, bd, (c | kk) != 0 ? 1u : 0u);
          }
        }
        umma_commit(empty(s));
      }
      if (ok && nchunks > 0) umma_commit(done);
      // no MMA may still run at exit: the last chunk's release (bounded)
      if (nchunks > 0)
        mbar_wait(empty((nchunks - 1) % WG_STAGES), (uint32_t)(((nchunks - 1) / WG_STAGES) & 1), spins);
    }
  } else if (nchunks > 0) {
    // epilogue: warp w holds ci = 32 (w % 4) + lane of every tap's accumulator
    const int q = warp & 3;
    if (!mbar_wait(done, 0, spins)) {
      ok = false;
    } else {
      tc_fence_after();
      const int ci = q * 32 + lane;
#pragma unroll 1
      for (int tl = 0; tl < WG_TAPS; ++tl) {
#pragma unroll 1
        for (int c0 = 0; c0 < COUT; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(tl * COUT + c0), v);
          if (ci >= CIN) continue;
          // 16-byte vector reductions (every dW tensor starts 16-byte aligned)
          float4 *d = reinterpret_cast<float4 *>(dw + ((size_t)(t0 + tl) * CIN + ci) * COUT + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j) atomicAdd(d + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
        }
      }
    }
  }
  if (!ok) atomicOr(err, MSA_DERR_TIMEOUT_TC);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Gm::TMEM_COLS));
}

// ---------------------------------------------------------------- host side

typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn get_encode() {
  static encode_fn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<encode_fn>(p);
  });
  return fn;
}

// 2-D bf16 tensor [rows][cols] (cols contiguous), box of box_rows x blk
// columns in the 128-byte (blk = 64) or 64-byte (blk = 32) swizzle; rows
// outside [0, rows) read as zeros
bool make_map(CUtensorMap *m, const void *ptr, uint64_t rows, uint64_t cols, uint32_t box_rows,
              uint32_t blk) {
  encode_fn enc = get_encode();
  if (!enc) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * sizeof(bf16)};
  const cuuint32_t box[2] = {blk, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE,
             blk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int CIN, int COUT, int MODE>
cudaError_t launch_tc(const bf16 *x, const bf16 *w, const float *bias, const int32_t *rowseq,
                      const bf16 *prev, void *y, int T, unsigned *err, cudaStream_t st,
                      long long spins, int no_loads) {
  using Gm = SoloGeo<CIN>;
  CUtensorMap xm, wm;
  if (!make_map(&xm, x, (uint64_t)T, CIN, AROWS, Gm::BLK) ||
      !make_map(&wm, w, (uint64_t)TAPS * COUT, CIN, TBN, Gm::BLK))
    return cudaErrorInvalidValue;
  constexpr int smem = Gm::SMEM;
  auto fn = k_conv_tc<CIN, COUT, MODE>;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  constexpr int NH = COUT / TBN;
  const int ntiles = (T + TBM - 1) / TBM;
  const int per_half = std::min(ntiles, std::max(1, sm_count() / NH));
  fn<<<per_half * NH, TC_THREADS, smem, st>>>(xm, wm, bias, rowseq, prev, y, T, err, spins, no_loads);
  return cudaGetLastError();
}

// the CTA-pair kernel: one pair per tile of 256 positions, at most as many
// pairs as can be resident at once
template <int CIN, int COUT, int MODE>
cudaError_t launch_tc2(const bf16 *x, const bf16 *w, const float *bias, const int32_t *rowseq,
                       const bf16 *prev, void *y, int T, unsigned *err, cudaStream_t st,
                       long long spins) {
  using Gm = Geo<CIN>;
  using Pg = PairGeo<CIN, COUT>;
  CUtensorMap xm, wm;
  if (!make_map(&xm, x, (uint64_t)T, CIN, AROWS, Gm::BLK) ||
      !make_map(&wm, w, (uint64_t)TAPS * COUT, CIN, Pg::BN, Gm::BLK))
    return cudaErrorInvalidValue;
  constexpr int smem = Pg::SMEM;
  auto fn = k_conv_tc2<CIN, COUT, MODE>;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // resident pairs of this instantiation per device (only the grid size
  // depends on it; devices past 63 share the last slot)
  static int mp_dev[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int &mp = mp_dev[std::min(std::max(dev, 0), 63)];
  if (mp == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (unsigned)std::max(1, sm_count() / 2));
    cfg.blockDim = dim3(PAIR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, (const void *)fn, &cfg) != cudaSuccess || clusters < 1) {
      cudaGetLastError();
      clusters = std::max(1, sm_count() / 2);
    }
    mp = clusters;
  }
  const int ntiles = (T + PAIR_TBM - 1) / PAIR_TBM;
  const int pairs = std::min(ntiles, mp);
  fn<<<2 * pairs, PAIR_THREADS, smem, st>>>(xm, wm, bias, rowseq, prev, y, T, err, spins);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_wgrad_tc(const bf16 *x, const bf16 *dy, float *dw, int T, unsigned *err,
                            cudaStream_t st, long long spins) {
  using Gm = WGeo<COUT>;
  CUtensorMap xm, dm;
  if (!make_map(&xm, x, (uint64_t)T, CIN, WG_AROWS, 64) || !make_map(&dm, dy, (uint64_t)T, COUT, WG_KR, 64))
    return cudaErrorInvalidValue;
  auto fn = k_wgrad_tc<CIN, COUT>;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM);
  if (e != cudaSuccess) return e;
  // about 8 chunks per CTA at least, one CTA per SM at most
  const int chunks = (T + WG_KR - 1) / WG_KR;
  const int groups = TAPS / WG_TAPS;
  const int splits = std::max(1, std::min(sm_count() / groups, (chunks + 7) / 8));
  const int per = (chunks + splits - 1) / splits * WG_KR;
  const dim3 grid((T + per - 1) / per, groups);
  fn<<<grid, TC_THREADS, Gm::SMEM, st>>>(xm, dm, dw, T, per, err, spins);
  return cudaGetLastError();
}

}  // namespace


cudaError_t wgrad_tc(int cin, int cout, const bf16 *x, const bf16 *dy, float *dw, int T,
                     unsigned *err, cudaStream_t st, long long spins) {
  if (T <= 0) return cudaSuccess;
  if (spins <= 0) spins = kSpinLimit;
  if (cin == 128 && cout == 128) return launch_wgrad_tc<128, 128>(x, dy, dw, T, err, st, spins);
  if (cin == 128 && cout == 64) return launch_wgrad_tc<128, 64>(x, dy, dw, T, err, st, spins);
  if (cin == 32 && cout == 128) return launch_wgrad_tc<32, 128>(x, dy, dw, T, err, st, spins);
  return cudaErrorInvalidValue;
}


cudaError_t conv_tc(int cin, int cout, int mode, const bf16 *x, const bf16 *w, const float *bias,
                    const int32_t *rowseq, const bf16 *prev, void *y, int T, unsigned *err,
                    cudaStream_t st, long long spins, bool no_loads) {
  if (T <= 0) return cudaSuccess;
  if (spins <= 0) spins = kSpinLimit;
  const int nl = no_loads ? 1 : 0;
  // every shape runs on CTA pairs (the load-free self-test keeps the
  // single-CTA kernel)
  if (!no_loads) {
#define NET_TC2(CI, CO, MD) \
    if (cin == CI && cout == CO && mode == MD) \
      return launch_tc2<CI, CO, MD>(x, w, bias, rowseq, prev, y, T, err, st, spins);
    NET_TC2(128, 128, 0)
    NET_TC2(128, 128, 2)
    NET_TC2(128, 64, 1)
    NET_TC2(64, 128, 2)
    NET_TC2(32, 128, 0)
#undef NET_TC2
    return cudaErrorInvalidValue;
  }
  // the load-free self-test: the single-CTA kernel, 128 -> 128 channels
  if (cin == 128 && cout == 128 && mode == 0)
    return launch_tc<128, 128, 0>(x, w, bias, rowseq, prev, y, T, err, st, spins, nl);
  return cudaErrorInvalidValue;
}

}  // namespace net
