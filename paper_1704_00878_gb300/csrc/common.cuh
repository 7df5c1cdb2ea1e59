// common.cuh -- definitions shared by the CUDA translation units of libmsa.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "msa.h"

#define MSA_FULL_MASK 0xffffffffu

// Residues of every loaded sequence sit at 16-byte aligned offsets followed by
// at least MSA_SEQ_TAIL bytes of the padding code, so 16-byte loads that start
// inside a sequence stay inside its allocation.
#define MSA_SEQ_TAIL 16

// Profile rows are padded to a multiple of this many bytes so that every
// residue row of the profile starts on the same shared-memory bank.
#define MSA_PROF_ALIGN 128

// ---------------------------------------------------------------- DPX cells
// One DP cell value is either an int32 or two int16 lanes packed in 32 bits
// (lane 0 = first subject, lane 1 = second subject).  All arithmetic goes
// through the Blackwell/Hopper DPX integer instructions.
template <bool PACK> struct Cell;

template <> struct Cell<false> {
  static __host__ __device__ __forceinline__ int splat(int x) { return x; }
  // max(a + b, c)
  static __device__ __forceinline__ int addmax(int a, int b, int c) { return __viaddmax_s32(a, b, c); }
  // max(a + b, c, 0)
  static __device__ __forceinline__ int addmax_relu(int a, int b, int c) { return __viaddmax_s32_relu(a, b, c); }
  static __device__ __forceinline__ int vmax(int a, int b) { return __vimax_s32_relu(a, b); }
  static __device__ __forceinline__ int vmax3(int a, int b, int c) { return __vimax3_s32(a, b, c); }
  // a + b (both lanes when packed)
  static __device__ __forceinline__ int add(int a, int b) { return a + b; }
  // sign-extended score of byte `sel` of (wa) -- one PRMT
  template <int B>
  static __device__ __forceinline__ int score(uint32_t wa, uint32_t /*wb*/) {
    int d;
    constexpr uint32_t sel = B | ((B | 8) << 4) | ((B | 8) << 8) | ((B | 8) << 12);
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(wa), "r"(0u), "n"(sel));
    return d;
  }
  static __device__ __forceinline__ int lane0(int v) { return v; }
  static __device__ __forceinline__ int lane1(int v) { return v; }
};

template <> struct Cell<true> {
  static __host__ __device__ __forceinline__ int splat(int x) {
    return (int)(((uint32_t)x & 0xffffu) | ((uint32_t)x << 16));
  }
  static __device__ __forceinline__ int addmax(int a, int b, int c) {
    return (int)__viaddmax_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
  }
  static __device__ __forceinline__ int addmax_relu(int a, int b, int c) {
    return (int)__viaddmax_s16x2_relu((unsigned)a, (unsigned)b, (unsigned)c);
  }
  // max(a, b, 0): the native DPX form (values fed here are never negative
  // where it matters; __vmaxs2 would be emulated with two instructions)
  static __device__ __forceinline__ int vmax(int a, int b) {
    return (int)__vimax_s16x2_relu((unsigned)a, (unsigned)b);
  }
  static __device__ __forceinline__ int vmax3(int a, int b, int c) {
    return (int)__vimax3_s16x2((unsigned)a, (unsigned)b, (unsigned)c);
  }
  static __device__ __forceinline__ int add(int a, int b) { return (int)__vadd2((unsigned)a, (unsigned)b); }
  // lane 0 <- sign-extended byte B of wa, lane 1 <- sign-extended byte B of wb
  template <int B>
  static __device__ __forceinline__ int score(uint32_t wa, uint32_t wb) {
    int d;
    constexpr uint32_t sel = B | ((B | 8) << 4) | ((B + 4) << 8) | (((B + 4) | 8) << 12);
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(wa), "r"(wb), "n"(sel));
    return d;
  }
  static __device__ __forceinline__ int lane0(int v) { return (int)(int16_t)(v & 0xffff); }
  static __device__ __forceinline__ int lane1(int v) { return (int)(int16_t)((uint32_t)v >> 16); }
};

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// Similarity of a pair for the exact center (the center is the sequence most
// similar to the others, Figure 3): the pair's local score S as a fraction of
// the larger of the two self scores, in units of 2^-16, rounded down; 2^16
// when both self scores are 0.  A row sum adds the distance 2^16 minus this.
#define MSA_SIM_ONE (1ull << 16)
__device__ __forceinline__ unsigned long long center_sim(int S, int sa, int sb) {
  const int m = sa > sb ? sa : sb;
  return m > 0 ? ((unsigned long long)(unsigned)S << 16) / (unsigned long long)(unsigned)m
               : MSA_SIM_ONE;
}

// The best cell of an alignment as one 64-bit key: a larger score first, then a
// smaller row i (center), then a smaller column j (sequence), so the maximum
// of the keys of any set of cells is the best cell under that tie rule; 0 when
// no cell is positive.  score < 2^35, i, j < 2^14.
__host__ __device__ __forceinline__ unsigned long long best_key(int v, int i, int j) {
  return v > 0 ? ((unsigned long long)v << 28) | ((unsigned long long)(16383 - i) << 14) |
                     (unsigned long long)(16383 - j)
               : 0ull;
}
__host__ __device__ __forceinline__ int best_key_score(unsigned long long k) { return (int)(k >> 28); }
__host__ __device__ __forceinline__ int best_key_row(unsigned long long k) {
  return k ? 16383 - (int)((k >> 14) & 16383u) : 0;
}
__host__ __device__ __forceinline__ int best_key_col(unsigned long long k) {
  return k ? 16383 - (int)(k & 16383u) : 0;
}

// Traceback codes of one subject of length L against a center of Lc rows,
// aligned by groups of G lanes, each lane holding one block of 16 center rows
// at a time: 8-byte words (16 rows x 4 bits), one row of S = L + G - 1
// rounded up to a multiple of 4 words per block, block b's column j in slot
// j + (b mod G) -- the wavefront step at which its lane computes it -- so
// every lane of a group fills the same 32-byte chunk of its row in the same
// four steps and writes it whole; slots outside the matrix hold no code.
__host__ __device__ __forceinline__ int code_row_words(int L, int G) { return (L + G - 1 + 3) & ~3; }
__host__ __device__ __forceinline__ size_t code_words(int L, int Lc, int G) {
  return (size_t)((Lc + 15) >> 4) * (size_t)code_row_words(L, G);
}
// word of center row i0 (0-based) and column j0 (0-based)
__host__ __device__ __forceinline__ size_t code_word(int i0, int j0, int L, int G) {
  const int b = i0 >> 4;
  return (size_t)b * (size_t)code_row_words(L, G) + (size_t)(j0 + b % G);
}

// Device-side error word bits (ctx->d_err).
#define MSA_DERR_LETTER   1u   // a letter outside the alphabet
#define MSA_DERR_TRACE    2u   // inconsistent traceback codes
#define MSA_DERR_OVERFLOW 4u   // overflow list full
#define MSA_DERR_TIMEOUT_TC 8u // a tensor-core convolution gave up waiting on an mbarrier
#define MSA_DERR_RANGE   16u   // a tree distance beyond its bound

static inline int round_up_int(int x, int m) { return (x + m - 1) / m * m; }
static inline int64_t round_up_i64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
