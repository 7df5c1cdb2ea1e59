// dp_pass.cuh -- device pieces shared by the alignment kernels: the unrolling
// helper, profile rows, residue fetches, code-word stores and the packed
// (two subjects per int16x2 register) pass of the affine-gap fill with
// traceback codes, in the four forms the full and the traceback-light
// alignments need.  Included by one translation unit per kernel family; every
// definition has internal linkage.
#pragma once
#include "sw_kernels.cuh"
#include <type_traits>

namespace {

template <int N, int I = 0> struct Unroll {
  template <class F> __device__ __forceinline__ static void run(F &&f) {
    f(std::integral_constant<int, I>{});
    Unroll<N, I + 1>::run(f);
  }
};
template <int N> struct Unroll<N, N> {
  template <class F> __device__ __forceinline__ static void run(F &&) {}
};

__device__ __forceinline__ int dround_up(int x, int m) { return (x + m - 1) / m * m; }

// The R profile bytes of one residue row for one lane, as 32-bit words.
template <int R> struct ProfRow {
  uint32_t w[R / 4];
  __device__ __forceinline__ void load(const int8_t *p) {
    if constexpr (R % 16 == 0) {
#pragma unroll
      for (int i = 0; i < R / 16; ++i) {
        const uint4 v = reinterpret_cast<const uint4 *>(p)[i];
        w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
      }
    } else if constexpr (R % 8 == 0) {
#pragma unroll
      for (int i = 0; i < R / 8; ++i) {
        const uint2 v = reinterpret_cast<const uint2 *>(p)[i];
        w[2 * i] = v.x; w[2 * i + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < R / 4; ++i) w[i] = reinterpret_cast<const uint32_t *>(p)[i];
    }
  }
};

// Residue code of column `col` of a subject (padding code past the end).
__device__ __forceinline__ uint32_t residue_at(const uint8_t *__restrict__ r, int L, int col,
                                               uint32_t padc) {
  return col < L ? (uint32_t)__ldg(r + col) : padc;
}

// Four code words (slots k-3 .. k of a block row, 32-byte aligned) in one
// 32-byte chunk.
__device__ __forceinline__ void store_chunk(uint2 *p, uint2 w0, uint2 w1, uint2 w2, uint2 w3) {
  uint4 *q = reinterpret_cast<uint4 *>(p);
  q[0] = make_uint4(w0.x, w0.y, w1.x, w1.y);
  q[1] = make_uint4(w2.x, w2.y, w3.x, w3.y);
}

// The words of the last, partial chunk after a pass of `steps` steps (the
// newest m = steps mod 4 words sit in w[4-m..3]).
__device__ __forceinline__ void flush_chunk(uint2 *cout, bool wr, int steps, int slots, uint2 w0,
                                            uint2 w1, uint2 w2, uint2 w3) {
  const int m = steps & 3, k0 = steps - m;
  if (m == 0 || !wr || cout == nullptr || k0 >= slots) return;
  for (int s = m; s < 4; ++s) { w0 = w1; w1 = w2; w2 = w3; w3 = make_uint2(0, 0); }
  store_chunk(cout + k0, w0, w1, w2, w3);
}

// ------------------------------------------------------------ packed codes
// Two length-adjacent subjects per group, A in the low int16 lane and B in the
// high one, against the same G*16 center rows (the host takes this path only
// while every cell value fits: Lc * smax + smax + o < 2^15 and s + o >= 0).
// Every pair of values a flag compares is ordered (F* >= H_up, E* >= H_left,
// M >= P, M >= F*, a row's new best >= its old best), so each flag is one
// 32-bit subtraction, which borrows across no lane, and a per-lane min with 1:
//   F bit = min(F* - H_up, 1)          E bit = min(E* - H_left, 1)
//   a     = min(M - P, 1)              (the diagonal is not a best source)
//   x     = min(M - F*, a)             (E is the only best source)
//   src   = 1 + a + x                  (1 diagonal, 2 F, 3 E; ties in that order)
// with M = max(P, F*, E*) in one three-way DPX max.  The source is meaningful
// only where H > 0: the traceback carries the score of the cell it stands on
// along the path and stops where that score is 0, so no zero flag is stored.
// The leading 1 of every source comes from the accumulator's initial nibbles.
// The first column reaching a row's best is max(column, d * j) with
// d = min(best' - best, 1).
// per-lane unsigned min of two int16 lanes: one instruction (the library's
// three-operand form issues two)
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// a * b + c in the low 32 bits (on the multiply-add pipe, beside the integer
// pipe the DP keeps busy)
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// What one packed pass computes (Eq. 1-2 in Gotoh's form throughout):
//   kFull   every cell's 4-bit code; per row the first column reaching the
//           row's best (the full alignment to the center)
//   kScore  no codes; the same best-cell tracking (the light alignment's
//           forward pass: the best cell of each subject)
//   kCorner no codes; operands reversed from each subject's best cell, each
//           half with its own center rows; per row the LAST column reaching
//           the row's best (the reverse pass: where best-scoring alignments
//           that end at the best cell may start)
//   kBox    as kFull, each half with its own center rows and columns (the
//           codes of the box that holds the traced segment)
enum CodesMode : int { kFull = 0, kScore = 1, kCorner = 2, kBox = 3 };

// Per-half settings of the light passes: profile byte masks (kCorner: the
// rows above a reversed window's first row read as padding) and the window's
// rows (cells below them take no part in the best cell).
struct HalfRows {
  uint32_t mA[4], mB[4];
  int rowsA, rowsB;
};

template <int G, int MODE = kFull>
__device__ __forceinline__ void codes_pass2(const int8_t *__restrict__ profA,
                                            const int8_t *__restrict__ profB, int stride,
                                            const uint8_t *__restrict__ rA, int LA,
                                            const uint8_t *__restrict__ rB, int LB, int Lw, int t,
                                            int base_lane, int blk, int nblkA, int nblkB, int padc,
                                            int o, int e, const int2 *__restrict__ scr_in,
                                            int2 *__restrict__ scr_out,
                                            uint2 *__restrict__ coutA, uint2 *__restrict__ coutB,
                                            const HalfRows &hr,
                                            int (&bv)[2], int (&bi)[2], int (&bj)[2]) {
  constexpr int R = kCodesR;
  constexpr bool CODES = MODE == kFull || MODE == kBox;
  constexpr bool OWN_ROWS = MODE == kCorner || MODE == kBox;
  using C = Cell<true>;
  constexpr uint32_t ONE = 0x00010001u;
  const uint32_t negO = (uint32_t)C::splat(-o), negE = (uint32_t)C::splat(-e);
  const uint32_t pc = (uint32_t)padc;
  // kCorner reads each subject backwards from its best cell (LA, LB = the best
  // cell's column)
  auto fetch = [&](int col) -> uint32_t {
    if constexpr (MODE == kCorner)
      return (col < LA ? (uint32_t)__ldg(rA + (LA - 1 - col)) : pc) |
             ((col < LB ? (uint32_t)__ldg(rB + (LB - 1 - col)) : pc) << 8);
    else
      return residue_at(rA, LA, col, pc) | (residue_at(rB, LB, col, pc) << 8);
  };
  uint32_t H[R], E[R], rb[R], rj[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { H[r] = 0; E[r] = 0; rb[r] = 0; rj[r] = 0; }
  uint32_t hbot = 0, fbot = 0, htop_prev = 0;
  uint32_t resv = pc | (pc << 8);
  // the last four steps' code words of each subject (slot k of the block row)
  uint2 a0 = make_uint2(0, 0), a1 = a0, a2 = a0, a3 = a0, b0 = a0, b1 = a0, b2 = a0, b3 = a0;
  const int slotsA = LA + G - 1, slotsB = LB + G - 1;
  uint32_t cur = fetch(t), nxt = fetch(G + t);
  int2 sv0 = make_int2(0, 0), sv1 = make_int2(0, 0);
  if (scr_in != nullptr) {
    if (0 < Lw) sv0 = scr_in[0];
    if (1 < Lw) sv1 = scr_in[1];
  }
  const int8_t *pbA = profA + t * R;
  const int8_t *pbB = OWN_ROWS ? profB + t * R : pbA;
  const bool wr = blk < nblkA;
  const bool wrB = OWN_ROWS ? blk < nblkB : wr;
  const int steps = Lw + G - 1;
#pragma unroll 2
  for (int k = 0; k < steps; ++k) {
    const int kk = k & (G - 1);
    if (kk == 0 && k > 0) { cur = nxt; nxt = fetch(k + G + t); }
    uint32_t r0 = cur, rin = 0, hin = 0, fin = 0;
    if constexpr (G > 1) {
      r0 = __shfl_sync(MSA_FULL_MASK, cur, base_lane + kk);
      rin = __shfl_up_sync(MSA_FULL_MASK, resv, 1);
      hin = __shfl_up_sync(MSA_FULL_MASK, hbot, 1);
      fin = __shfl_up_sync(MSA_FULL_MASK, fbot, 1);
    }
    const int2 sv = sv0;
    sv0 = sv1;
    if (scr_in != nullptr && k + 2 < Lw) sv1 = scr_in[k + 2];
    if (t == 0) {
      rin = r0;
      const bool above = scr_in != nullptr && k < Lw;
      hin = above ? (uint32_t)sv.x : 0u;
      fin = above ? (uint32_t)sv.y : 0u;
    }
    resv = rin;
    ProfRow<R> pa, pq;
    pa.load(pbA + (int)(resv & 0xffu) * stride);
    pq.load(pbB + (int)(resv >> 8) * stride);
    if constexpr (MODE == kCorner) {
#pragma unroll
      for (int w = 0; w < R / 4; ++w) { pa.w[w] &= hr.mA[w]; pq.w[w] &= hr.mB[w]; }
    }
    const int j = k - t;
    const uint32_t jj = (uint32_t)j;  // see the best-column update below
    uint32_t hdiag = htop_prev;
    htop_prev = hin;
    uint32_t hup = hin, f = fin;
    uint32_t acc[4] = {0x11111111u, 0x11111111u, 0x11111111u, 0x11111111u};
    Unroll<R>::run([&](auto ic) {
      constexpr int r = decltype(ic)::value;
      const uint32_t p = hdiag + (uint32_t)C::template score<r & 3>(pa.w[r >> 2], pq.w[r >> 2]);
      f = __viaddmax_s16x2(f, negE, hup);                // F*
      if constexpr (CODES) {
        constexpr uint32_t SH = 1u << (4 * (r & 3));
        const uint32_t bF = min_u16x2(f - hup, ONE);
        const uint32_t m = __vimax3_s16x2(p, f, E[r]);    // max(P, F*, E*)
        const uint32_t hn = __viaddmax_s16x2_relu(m, negO, 0u);
        const uint32_t a = min_u16x2(m - p, ONE);
        const uint32_t x = min_u16x2(m - f, a);
        const uint32_t bE = min_u16x2(E[r] - H[r], ONE);
        const uint32_t code = mad_lo(bF, 8u, mad_lo(bE, 4u, a + x));
        acc[r >> 2] = mad_lo(code, SH, acc[r >> 2]);
        E[r] = __viaddmax_s16x2(E[r], negE, hn);         // E* of the next column
        const uint32_t rbn = __vimax_s16x2_relu(rb[r], hn);
        rj[r] = __vimax_s16x2_relu(rj[r], mad_lo(min_u16x2(rbn - rb[r], ONE), jj, 0u));
        rb[r] = rbn;
        hdiag = H[r];
        H[r] = hn;
        hup = hn;
      } else {
        const uint32_t m = __vimax3_s16x2(p, f, E[r]);
        const uint32_t hn = __viaddmax_s16x2_relu(m, negO, 0u);
        E[r] = __viaddmax_s16x2(E[r], negE, hn);
        const uint32_t rbn = __vimax_s16x2_relu(rb[r], hn);
        // first column reaching the row's best: d = min(best' - best, 1);
        // last column reaching it: d = 1 - min(best' - H, 1).  While j < 0
        // the lane sits before the matrix (H = 0): d * j is then either 0
        // or negative in both int16 lanes, and the relu max drops it.
        const uint32_t d = MODE == kCorner ? ONE - min_u16x2(rbn - hn, ONE) : min_u16x2(rbn - rb[r], ONE);
        rj[r] = __vimax_s16x2_relu(rj[r], mad_lo(d, jj, 0u));
        rb[r] = rbn;
        hdiag = H[r];
        H[r] = hn;
        hup = hn;
      }
    });
    hbot = H[R - 1];
    fbot = f;
    if constexpr (CODES) {
      a0 = a1; a1 = a2; a2 = a3;
      a3 = make_uint2(__byte_perm(acc[0], acc[1], 0x5410), __byte_perm(acc[2], acc[3], 0x5410));
      b0 = b1; b1 = b2; b2 = b3;
      b3 = make_uint2(__byte_perm(acc[0], acc[1], 0x7632), __byte_perm(acc[2], acc[3], 0x7632));
      if constexpr (OWN_ROWS) {
        if ((k & 3) == 3) {
          if (wr && coutA != nullptr && k - 3 < slotsA) store_chunk(coutA + (k - 3), a0, a1, a2, a3);
          if (wrB && coutB != nullptr && k - 3 < slotsB) store_chunk(coutB + (k - 3), b0, b1, b2, b3);
        }
      } else if ((k & 3) == 3 && wr) {
        if (coutA != nullptr && k - 3 < slotsA) store_chunk(coutA + (k - 3), a0, a1, a2, a3);
        if (coutB != nullptr && k - 3 < slotsB) store_chunk(coutB + (k - 3), b0, b1, b2, b3);
      }
    }
    if (scr_out != nullptr && t == G - 1 && j >= 0 && j < Lw) scr_out[j] = make_int2((int)hbot, (int)fbot);
  }
  if constexpr (CODES) {
    flush_chunk(coutA, wr, steps, slotsA, a0, a1, a2, a3);
    flush_chunk(coutB, wrB, steps, slotsB, b0, b1, b2, b3);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int va = C::lane0((int)rb[r]), vb = C::lane1((int)rb[r]);
    if constexpr (!OWN_ROWS) {
      if (va > bv[0]) { bv[0] = va; bi[0] = blk * R + r + 1; bj[0] = (int)(rj[r] & 0xffffu) + 1; }
      if (vb > bv[1]) { bv[1] = vb; bi[1] = blk * R + r + 1; bj[1] = (int)(rj[r] >> 16) + 1; }
      continue;
    }
    const int row = blk * R + r + 1;
    const int ja = (int)(rj[r] & 0xffffu) + 1, jb = (int)(rj[r] >> 16) + 1;
    if constexpr (MODE == kCorner) {
      // the largest value; among cells of that value the largest row and,
      // separately, the largest column (rows grow with r and with the pass)
      if (va > 0 && row <= hr.rowsA) {
        if (va > bv[0]) { bv[0] = va; bi[0] = row; bj[0] = ja; }
        else if (va == bv[0]) { bi[0] = row; bj[0] = max(bj[0], ja); }
      }
      if (vb > 0 && row <= hr.rowsB) {
        if (vb > bv[1]) { bv[1] = vb; bi[1] = row; bj[1] = jb; }
        else if (vb == bv[1]) { bi[1] = row; bj[1] = max(bj[1], jb); }
      }
    } else {  // kBox: the first best cell inside the box
      if (va > bv[0] && row <= hr.rowsA) { bv[0] = va; bi[0] = row; bj[0] = ja; }
      if (vb > bv[1] && row <= hr.rowsB) { bv[1] = vb; bi[1] = row; bj[1] = jb; }
    }
  }
}

}  // namespace
