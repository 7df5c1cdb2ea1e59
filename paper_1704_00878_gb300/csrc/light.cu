// light.cu -- the traceback-light alignment to the center: the local
// alignment of Eq. 1-2 with its traceback (Figure 2's walk from the best cell
// back to a zero cell), computed without storing a code for every cell.
//
//   1. kScore: a forward fill over each subject's whole matrix that keeps
//      only the best cell (i2, j2), first by row, then by column, as the full
//      fill does, and its score S.
//   2. kCorner: the fill of the two prefixes ending at the best cell, both
//      read backwards.  Every cell scores at most S there (an alignment of
//      the reversed prefixes is an alignment ending inside the prefix box, and
//      none beats the best cell); a cell reaching S is the first residue pair
//      of a best-scoring alignment that ends at the best cell itself (it
//      cannot end at an earlier cell of score S: the best cell is the first).
//      The traced segment starts at one of them, so the largest reversed row
//      and the largest reversed column of such cells give a corner
//      (i2 - P, j2 - Q) above and left of the segment's start.
//   3. kBox: the codes of the box from that corner (its row rounded down to
//      16) to the best cell, a local alignment of the two slices.  The box
//      holds the traced path, so its first best cell is (i2, j2) again and
//      the walk over the box's codes retraces the same path.
//
// Packed int16x2 cells only (two subjects per register, as the full codes
// kernel): the host takes this path where every value fits.
#include "sw_kernels.cuh"
#include "dp_pass.cuh"

namespace {

template <int G, int NT, int MODE>
__global__ void __launch_bounds__(NT, 1) k_light(SeqSet ss, Scoring sc, LightJob job) {
  constexpr int R = kCodesR, NG = NT / G, GPW = 32 / G, GR = G * R;
  extern __shared__ __align__(16) int8_t smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  const int K = sc.K, padc = K;
  const int Lc = ss.len[job.center];
  const int rows = light_prof_rows(Lc, G, MODE, job.npass);
  const int stride = dround_up(rows, MSA_PROF_ALIGN);
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = sc.M[i];
  __syncthreads();
  // profile of the center (kCorner: of the center read backwards); rows past
  // Lc score -o
  const uint8_t *rc = ss.res + ss.pstart[job.center];
  for (int idx = threadIdx.x; idx < (K + 1) * rows; idx += NT) {
    const int r = idx / rows, i = idx - r * rows;
    int v = 0;
    if (r < K && i < Lc) v = sM[rc[MODE == kCorner ? Lc - 1 - i : i] * K + r] + sc.o;
    smem[r * stride + i] = (int8_t)v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, t = threadIdx.x % G, g = threadIdx.x / G;
  const int base_lane = lane - t;
  int2 *scr = job.scratch + ((size_t)blockIdx.x * NG + g) * 2 * job.scratch_cols;
  const int nitem = MODE == kScore ? (job.se - job.sb + 1) / 2 : (job.npos + 1) / 2;
  // passes past a half's own window read GR rows of padding
  const int pad_row = ((Lc + 15) & ~15) + GR;
  for (;;) {
    int x0 = 0;
    if (lane == 0) x0 = (int)atomicAdd(job.counter, (unsigned long long)GPW);
    x0 = __shfl_sync(MSA_FULL_MASK, x0, 0);
    if (x0 >= nitem) break;
    const int x = x0 + lane / G;
    const bool valid = x < nitem;
    int ka, kb, LA, LB, startA = 0, startB = 0, rowsA, rowsB, delA = 0, delB = 0;
    bool hasb;
    const uint8_t *rA, *rB;
    uint2 *cA = nullptr, *cB = nullptr;
    if constexpr (MODE == kScore) {
      ka = job.se - 1 - 2 * (valid ? x : 0);  // longest first
      kb = ka - 1;
      hasb = valid && kb >= job.sb;
      LA = valid ? ss.len[ka] : 0;
      LB = hasb ? ss.len[kb] : 0;
      rA = ss.res + ss.pstart[ka];
      rB = hasb ? ss.res + ss.pstart[kb] : rA;
      rowsA = rowsB = Lc;
    } else {
      const int pa = 2 * (valid ? x : 0), pb = pa + 1;
      hasb = valid && pb < job.npos;
      ka = job.order[pa];
      kb = hasb ? job.order[pb] : ka;
      const int4 wa = valid ? job.win[pa] : make_int4(0, 0, 0, 0);
      const int4 wb = hasb ? job.win[pb] : make_int4(0, 0, 0, 0);
      startA = wa.x; rowsA = wa.y; LA = wa.w;
      startB = wb.x; rowsB = wb.y; LB = wb.w;
      rA = ss.res + ss.pstart[ka];
      rB = ss.res + ss.pstart[kb];
      if constexpr (MODE == kBox) {
        rA += wa.z;
        rB += wb.z;
        if (valid) cA = reinterpret_cast<uint2 *>(job.codes + job.code_off[pa]);
        if (hasb) cB = reinterpret_cast<uint2 *>(job.codes + job.code_off[pb]);
      } else {
        delA = wa.z;
        delB = wb.z;
      }
    }
    const int Lw = __reduce_max_sync(MSA_FULL_MASK, max(LA, LB));
    const int npA = (rowsA + GR - 1) / GR, npB = (rowsB + GR - 1) / GR;
    const int np = MODE == kScore ? job.npass : (int)__reduce_max_sync(MSA_FULL_MASK, (unsigned)max(npA, npB));
    const int nblkA = (rowsA + R - 1) / R, nblkB = (rowsB + R - 1) / R;
    int bv[2] = {0, 0}, bi[2] = {0, 0}, bj[2] = {0, 0};
    for (int p = 0; p < np; ++p) {
      const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
      int2 *sout = p + 1 < np ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
      const int blk = p * G + t;
      const int8_t *pA = smem + (MODE == kScore ? p * GR : (p < npA ? startA + p * GR : pad_row));
      const int8_t *pB = smem + (MODE == kScore ? p * GR : (p < npB ? startB + p * GR : pad_row));
      HalfRows hr;
      hr.rowsA = rowsA;
      hr.rowsB = rowsB;
#pragma unroll
      for (int w = 0; w < R / 4; ++w) {
        // kCorner: the window's first row sits delA rows into the first
        // 16-row block; the rows above it read as padding (H stays 0 there,
        // the same state as the top of the matrix)
        uint32_t ma = 0xffffffffu, mb = 0xffffffffu;
        if (MODE == kCorner && p == 0 && t == 0) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if (4 * w + b < delA) ma &= ~(0xffu << (8 * b));
            if (4 * w + b < delB) mb &= ~(0xffu << (8 * b));
          }
        }
        hr.mA[w] = ma;
        hr.mB[w] = mb;
      }
      codes_pass2<G, MODE>(pA, pB, stride, rA, LA, rB, LB, Lw, t, base_lane, blk, nblkA, nblkB,
                           padc, sc.o, sc.e, sin, sout,
                           cA ? cA + (size_t)blk * code_row_words(LA, G) : nullptr,
                           cB ? cB + (size_t)blk * code_row_words(LB, G) : nullptr, hr, bv, bi, bj);
      __syncwarp();
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      int v = bv[s2], i2 = bi[s2], j2 = bj[s2];
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) {
        const int ov = __shfl_xor_sync(MSA_FULL_MASK, v, off);
        const int oi = __shfl_xor_sync(MSA_FULL_MASK, i2, off);
        const int oj = __shfl_xor_sync(MSA_FULL_MASK, j2, off);
        if constexpr (MODE == kCorner) {
          // largest value; on a tie the larger row and the larger column
          if (ov > v) { v = ov; i2 = oi; j2 = oj; }
          else if (ov == v) { i2 = max(i2, oi); j2 = max(j2, oj); }
        } else {
          const bool take = ov > v || (ov == v && (oi < i2 || (oi == i2 && oj < j2)));
          if (take) { v = ov; i2 = oi; j2 = oj; }
        }
      }
      const bool mine = s2 == 0 ? valid : hasb;
      if (t != 0 || !mine) continue;
      if constexpr (MODE == kScore) {
        job.best[(s2 == 0 ? ka : kb) - job.sb] = best_key(v, i2, j2);
      } else if constexpr (MODE == kCorner) {
        job.best[2 * x + s2] = best_key(v, i2 - (s2 == 0 ? delA : delB), j2);
      } else {
        job.best[2 * x + s2] = best_key(v, i2, j2);
      }
    }
  }
}

typedef void (*light_fn)(SeqSet, Scoring, LightJob);

template <int MODE>
light_fn light_kernel_of(int G) {
  switch (G) {
    case 1: return k_light<1, kLightThreads, MODE>;
    case 2: return k_light<2, kLightThreads, MODE>;
    case 4: return k_light<4, kLightThreads, MODE>;
    case 8: return k_light<8, kLightThreads, MODE>;
    case 16: return k_light<16, kLightThreads, MODE>;
    case 32: return k_light<32, kLightThreads, MODE>;
    default: return nullptr;
  }
}

light_fn light_kernel(int G, int mode) {
  switch (mode) {
    case kScore: return light_kernel_of<kScore>(G);
    case kCorner: return light_kernel_of<kCorner>(G);
    case kBox: return light_kernel_of<kBox>(G);
    default: return nullptr;
  }
}

}  // namespace

int light_smem_bytes(int K, int Lc, int G, int mode, int npass) {
  return (K + 1) * round_up_int(light_prof_rows(Lc, G, mode, npass), MSA_PROF_ALIGN);
}

cudaError_t light_allow_smem(int G, int mode, int smem) {
  light_fn fn = light_kernel(G, mode);
  if (!fn) return cudaErrorInvalidValue;
  if (smem <= 40 * 1024) return cudaSuccess;  // static shared memory counts too
  return cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

int light_grid(int G, int mode, int smem) {
  light_fn fn = light_kernel(G, mode);
  if (!fn) return 0;
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLightThreads, smem) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

cudaError_t launch_light(int G, int mode, const SeqSet &ss, const Scoring &sc, const LightJob &job,
                         int grid, int smem, cudaStream_t st) {
  light_fn fn = light_kernel(G, mode);
  if (!fn || grid < 1) return cudaErrorInvalidValue;
  fn<<<grid, kLightThreads, smem, st>>>(ss, sc, job);
  return cudaGetLastError();
}
