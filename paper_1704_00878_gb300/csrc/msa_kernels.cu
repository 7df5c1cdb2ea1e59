// msa_kernels.cu -- the non-DP steps of the center-star path: residue
// encoding, traceback walk + flank rule (the inserted-space matrix), the
// merge of inserted spaces into the "longest" center, MSA rows, the
// sum-of-pairs cost, and the distance row sums of center selection.
#include "msa_kernels.cuh"
#include <algorithm>
#include <climits>

namespace {

// ---------------------------------------------------------------- encode
// One warp per sequence (sorted order): ASCII -> alphabet index, written at
// the sequence's aligned slot and followed by padding codes.
__global__ void k_encode(const uint8_t *__restrict__ letters, const int64_t *__restrict__ src_off,
                         const int32_t *__restrict__ perm, const int64_t *__restrict__ pstart,
                         const int32_t *__restrict__ len, int n, const uint8_t *__restrict__ lut,
                         int padc, uint8_t *__restrict__ res, unsigned *err) {
  __shared__ uint8_t slut[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) slut[i] = lut[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    const int L = len[k];
    const uint8_t *src = letters + src_off[perm[k]];
    uint8_t *dst = res + pstart[k];
    const int total = ((L + 15) / 16) * 16 + MSA_SEQ_TAIL;
    for (int i = lane; i < total; i += 32) {
      uint8_t v = (uint8_t)padc;
      if (i < L) {
        v = slut[src[i]];
        if (v == 255) { bad = true; v = (uint8_t)padc; }
      }
      dst[i] = v;
    }
  }
  if (bad) atomicOr(err, MSA_DERR_LETTER);
}

// ---------------------------------------------------------------- traceback
// One thread per subject.  Walks the 4-bit codes from the best cell back to a
// zero cell (state H / F / E, as in Gotoh's traceback), then applies the flank
// rule: residues before the segment pair right-aligned with the center, after
// it left-aligned, surplus sequence residues go to slot 0 / slot Lc.
// The walk carries the score v of the cell it stands on: H = best at the best
// cell; a diagonal step from (i, j) gives H(i-1, j-1) = v - s(c_i, s_j); in a
// gap state F(i, j) = v and a step up gives F(i-1, j) = v + e (extended) or
// H(i-1, j) = v + o (opened), and likewise for E along the row.  In state H the
// walk stops where v = 0 (the paper's "cell with score of zero"), so the codes
// need a source only where H > 0.
__device__ __forceinline__ uint32_t code_at(const uint8_t *__restrict__ c, int Ls, int G, int i,
                                            int j) {
  const int r = i - 1;
  const size_t at = code_word(r, j - 1, Ls, G) * 8 + ((r & 15) >> 1);
  return (c[at] >> ((r & 1) * 4)) & 15u;
}

__global__ void k_traceback(const uint8_t *__restrict__ codes, const int64_t *__restrict__ code_off,
                            const unsigned long long *__restrict__ best, int sb, int se,
                            const int32_t *__restrict__ len, const int32_t *__restrict__ perm,
                            const uint8_t *__restrict__ res, const int64_t *__restrict__ pstart,
                            int center, const int8_t *__restrict__ M, int K, int o, int e,
                            int Lc, int G, uint16_t *__restrict__ ins, uint8_t *__restrict__ occ,
                            int32_t *__restrict__ seg, int32_t *__restrict__ score,
                            unsigned *err, const int32_t *__restrict__ list,
                            const int4 *__restrict__ box,
                            const unsigned long long *__restrict__ box_best) {
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) sM[i] = M[i];
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= se - sb) return;
  // the subject: the x-th of [sb, se), or the x-th of a list (codes and boxes
  // by list position, best cells by sorted index)
  const int k = list ? list[x] : sb + x;
  const int orig = perm[k];
  const int Ls = len[k];
  const uint8_t *c = codes + code_off[x];
  const uint8_t *rc = res + pstart[center], *rs = res + pstart[k];
  uint16_t *in = ins + (size_t)orig * (Lc + 1);
  uint8_t *oc = occ + (size_t)orig * (Lc + 1);
  const unsigned long long key = list ? best[k] : best[x];
  const int bv = best_key_score(key);
  int i2 = best_key_row(key), j2 = best_key_col(key);
  int i1 = 0, j1 = 0;
  if (bv > 0 && (i2 < 1 || i2 > Lc || j2 < 1 || j2 > Ls)) {  // a best cell outside the matrix
    atomicOr(err, MSA_DERR_TRACE);
    return;
  }
  // codes of the box rows (i0, i2] x columns (j0, j0 + cw], or of the whole
  // matrix; the box's own best cell must be the matrix's
  const int4 bx = box ? box[x] : make_int4(0, Lc, 0, Ls);
  const int i0 = bx.x, j0 = bx.z, cw = bx.w;
  if (box && bv > 0 &&
      (i0 < 0 || j0 < 0 || i0 + bx.y != i2 || j0 + cw != j2 || box_best[x] != best_key(bv, i2 - i0, j2 - j0))) {
    atomicOr(err, MSA_DERR_TRACE);
    return;
  }
  if (bv <= 0) {
    i2 = 0; j2 = 0;
  } else {
    int i = i2, j = j2, state = 0;  // 0 = H, 1 = F (center residue vs gap), 2 = E (inserted residue)
    int v = bv;
    const int limit = 2 * (i2 + j2) + 4;
    bool ok = false;
    for (int step = 0; step < limit; ++step) {
      if (i <= i0 || j <= j0) { ok = state == 0 && v == 0; break; }
      if (state == 0) {
        if (v == 0) { ok = true; break; }
        if (v < 0) break;
        const uint32_t src = code_at(c, cw, G, i - i0, j - j0) & 3u;
        if (src == 1) {
          v -= sM[rc[i - 1] * K + rs[j - 1]];
          oc[i] = 1; --i; --j;
        } else if (src == 0) {
          break;  // a positive score with no source: inconsistent codes
        } else {
          state = src == 2 ? 1 : 2;
        }
      } else if (state == 1) {
        const bool ext = (code_at(c, cw, G, i - i0, j - j0) >> 3) & 1u;
        v += ext ? e : o;
        state = ext ? 1 : 0;
        --i;
      } else {
        const bool ext = (code_at(c, cw, G, i - i0, j - j0) >> 2) & 1u;
        in[i] = (uint16_t)(in[i] + 1);
        v += ext ? e : o;
        state = ext ? 2 : 0;
        --j;
      }
    }
    if (!ok) atomicOr(err, MSA_DERR_TRACE);
    i1 = i; j1 = j;
  }
  const int kp = min(i1, j1);
  for (int t = 0; t < kp; ++t) oc[i1 - t] = 1;
  if (j1 > i1) in[0] = (uint16_t)(in[0] + (j1 - i1));
  const int a = Lc - i2, b = Ls - j2, ks = min(a, b);
  for (int t = 1; t <= ks; ++t) oc[i2 + t] = 1;
  if (b > a) in[Lc] = (uint16_t)(in[Lc] + (b - a));
  int32_t *sg = seg + (size_t)orig * 5;
  sg[0] = bv; sg[1] = i1; sg[2] = j1; sg[3] = i2; sg[4] = j2;
  score[orig] = bv;
}

// ---------------------------------------------------------------- merge
// G[j] = max over rows of ins[row][j]: threads own columns, blocks own row
// chunks; partial maxima meet with atomicMax.
__global__ void k_colmax(const uint16_t *__restrict__ ins, int n, int Lc, int rows_per_block,
                         int32_t *__restrict__ G) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > Lc) return;
  const int r0 = blockIdx.y * rows_per_block, r1 = min(n, r0 + rows_per_block);
  int m = 0;
  for (int r = r0; r < r1; ++r) m = max(m, (int)ins[(size_t)r * (Lc + 1) + j]);
  if (m) atomicMax(&G[j], m);
}

// off[j] = sum_{k<j} (G[k] + 1): the first MSA column of slot j; width W =
// Lc + sum G.  One block of 1024 threads.
__global__ void k_scan(const int32_t *__restrict__ G, int Lc, int32_t *__restrict__ off,
                       int64_t *__restrict__ width) {
  __shared__ int warp_tot[32];
  const int m = Lc + 1;
  const int per = (m + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(m, b + per);
  int local = 0;
  for (int j = b; j < e; ++j) local += G[j] + 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(MSA_FULL_MASK, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(MSA_FULL_MASK, v, d);
      if (lane >= d) v += u;
    }
    warp_tot[lane] = v;
  }
  __syncthreads();
  int run = (w > 0 ? warp_tot[w - 1] : 0) + incl - local;
  for (int j = b; j < e; ++j) { off[j] = run; run += G[j] + 1; }
  if (threadIdx.x == blockDim.x - 1) *width = (int64_t)run - 1;
}

// One warp per MSA row (input order).  Lanes own consecutive slots; a warp
// scan of (ins[j] + occ[j+1]) gives the index of the first residue each slot
// consumes.
__global__ void k_rows(const uint8_t *__restrict__ res, const int64_t *__restrict__ pstart,
                       const int32_t *__restrict__ inv, const uint16_t *__restrict__ ins,
                       const uint8_t *__restrict__ occ, const int32_t *__restrict__ G,
                       const int32_t *__restrict__ off, int n, int Lc, int64_t W,
                       const char *__restrict__ letters, uint8_t *__restrict__ out) {
  __shared__ char sl[MSA_MAX_ALPHABET + 1];
  if (threadIdx.x < MSA_MAX_ALPHABET + 1) sl[threadIdx.x] = letters[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n; t += warps) {
    const uint8_t *s = res + pstart[inv[t]];
    const uint16_t *in = ins + (size_t)t * (Lc + 1);
    const uint8_t *oc = occ + (size_t)t * (Lc + 1);
    uint8_t *row = out + (size_t)t * W;
    int carry = 0;
    for (int base = 0; base <= Lc; base += 32) {
      const int j = base + lane;
      int ni = 0, no = 0;
      if (j <= Lc) { ni = in[j]; no = j < Lc ? oc[j + 1] : 0; }
      const int cnt = ni + no;
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(MSA_FULL_MASK, incl, d);
        if (lane >= d) incl += v;
      }
      if (j <= Lc) {
        const int k0 = carry + incl - cnt;
        const int pos = off[j], g = G[j];
        for (int u = 0; u < ni; ++u) row[pos + u] = (uint8_t)sl[s[k0 + u]];
        for (int u = ni; u < g; ++u) row[pos + u] = '-';
        if (j < Lc) row[pos + g] = no ? (uint8_t)sl[s[k0 + ni]] : (uint8_t)'-';
      }
      carry += __shfl_sync(MSA_FULL_MASK, incl, 31);
    }
  }
}

// The same rows assembled in shared memory, one warp per row: the warp fills
// the row with '-' (16-byte stores), each lane writes its slots' residues
// (inserted ones left-justified, then the center column's), and the warp
// copies the row out with 16-byte stores where the row's bytes cover a whole
// aligned chunk (byte stores at the two ragged ends, which neighbour other
// rows).  `rowbytes` = W rounded up to 16, plus 16.
__global__ void k_rows_staged(const uint8_t *__restrict__ res, const int64_t *__restrict__ pstart,
                              const int32_t *__restrict__ inv, const uint16_t *__restrict__ ins,
                              const uint8_t *__restrict__ occ, const int32_t *__restrict__ off,
                              int n, int Lc, int64_t W, int rowbytes,
                              const char *__restrict__ letters, uint8_t *__restrict__ out) {
  extern __shared__ __align__(16) uint8_t srows[];
  __shared__ char sl[MSA_MAX_ALPHABET + 1];
  if (threadIdx.x < MSA_MAX_ALPHABET + 1) sl[threadIdx.x] = letters[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint8_t *buf = srows + (size_t)(threadIdx.x >> 5) * rowbytes;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const uint4 gaps = make_uint4(0x2d2d2d2du, 0x2d2d2d2du, 0x2d2d2d2du, 0x2d2d2d2du);
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n; t += warps) {
    uint8_t *row = out + (size_t)t * W;
    // the row starts a = row mod 16 bytes into the buffer, so buffer and
    // global chunks line up
    const int a = (int)((uintptr_t)row & 15);
    for (int c = lane; c < rowbytes / 16; c += 32) reinterpret_cast<uint4 *>(buf)[c] = gaps;
    __syncwarp();
    const uint8_t *s = res + pstart[inv[t]];
    const uint16_t *in = ins + (size_t)t * (Lc + 1);
    const uint8_t *oc = occ + (size_t)t * (Lc + 1);
    int carry = 0;
    for (int base = 0; base <= Lc; base += 32) {
      const int j = base + lane;
      int ni = 0, no = 0;
      if (j <= Lc) { ni = in[j]; no = j < Lc ? oc[j + 1] : 0; }
      const int cnt = ni + no;
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(MSA_FULL_MASK, incl, d);
        if (lane >= d) incl += v;
      }
      if (j <= Lc) {
        const int k0 = carry + incl - cnt;
        uint8_t *dst = buf + a + off[j];
        for (int u = 0; u < ni; ++u) dst[u] = (uint8_t)sl[s[k0 + u]];
        if (no) buf[a + off[j] + (j < Lc ? (off[j + 1] - off[j] - 1) : 0)] = (uint8_t)sl[s[k0 + ni]];
      }
      carry += __shfl_sync(MSA_FULL_MASK, incl, 31);
    }
    __syncwarp();
    // copy out: bytes [0, W) of the row sit at buf[a .. a + W)
    const int64_t first = a ? 16 - a : 0;           // bytes before the first aligned chunk
    const int64_t nfull = W > first ? (W - first) / 16 : 0;
    const int64_t tail0 = first + nfull * 16;       // first byte after the last full chunk
    for (int64_t c = lane; c < nfull; c += 32)
      reinterpret_cast<uint4 *>(row + first)[c] = reinterpret_cast<const uint4 *>(buf + a + first)[c];
    if (lane < first && lane < W) row[lane] = buf[a + lane];
    for (int64_t x = tail0 + lane; x < W; x += 32) row[x] = buf[a + x];
    __syncwarp();
  }
}

// ---------------------------------------------------------------- SP
// Per column symbol counts (letters and '-'), accumulated over row chunks.
__global__ void k_sp_count(const uint8_t *__restrict__ msa, int n, int64_t W,
                           const uint8_t *__restrict__ sym_lut, int nsym, int rows_per_block,
                           int32_t *__restrict__ counts) {
  extern __shared__ int32_t hist[];  // [nsym][blockDim.x]
  __shared__ uint8_t slut[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) slut[i] = sym_lut[i];
  for (int s = 0; s < nsym; ++s) hist[s * blockDim.x + threadIdx.x] = 0;
  __syncthreads();
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= W) return;
  const int r0 = blockIdx.y * rows_per_block, r1 = min(n, r0 + rows_per_block);
  // four rows' bytes in flight per thread; the histogram bins are private to
  // the thread, incremented by shared-memory atomics (one operation each;
  // four columns per thread from aligned word loads measured 5x slower: the
  // bins of four columns cut the resident threads by four)
  int r = r0;
  for (; r + 4 <= r1; r += 4) {
    uint8_t v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldg(msa + (size_t)(r + u) * W + x);
#pragma unroll
    for (int u = 0; u < 4; ++u) atomicAdd(&hist[slut[v[u]] * blockDim.x + threadIdx.x], 1);
  }
  for (; r < r1; ++r) atomicAdd(&hist[slut[__ldg(msa + (size_t)r * W + x)] * blockDim.x + threadIdx.x], 1);
  for (int s = 0; s < nsym; ++s) {
    const int v = hist[s * blockDim.x + threadIdx.x];
    if (v) atomicAdd(&counts[x * nsym + s], v);
  }
}

// Column cost: (R^2 - sum c_a^2)/2 differing residue pairs + 2 g R residue-gap
// pairs; the gap symbol is the last one.
__global__ void k_sp_cost(const int32_t *__restrict__ counts, int n, int64_t W, int nsym,
                          unsigned long long *total) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  long long v = 0;
  if (x < W) {
    const int32_t *c = counts + x * nsym;
    const long long g = c[nsym - 1], r = n - g;
    long long sq = 0;
    for (int s = 0; s < nsym - 1; ++s) sq += (long long)c[s] * c[s];
    v = (r * r - sq) / 2 + 2 * g * r;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(MSA_FULL_MASK, v, d);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, (unsigned long long)v);
}

// ---------------------------------------------------------------- center
// rowsum (input order) of d(i, j) = 2^16 - center_sim(S_ij, S_ii, S_jj) over
// the partners, from the similarity sums:
//   all pairs:  (n-1) 2^16 - sum_{j != i} sim(i, j)
//   refs:       nref  2^16 - sum_{r} sim(i, r)       (d(i, i) = 0 when i is a reference)
// then a per-block (min, lowest index) partial.
__global__ void k_rowsum(int mode, int n, int nref, const int32_t *__restrict__ perm,
                         const unsigned long long *__restrict__ pairsum,
                         long long *__restrict__ rowsum, long long *__restrict__ part_val,
                         long long *__restrict__ part_idx) {
  __shared__ long long sv[32], si[32];
  const long long cnt = mode == 0 ? (long long)n - 1 : (long long)nref;
  long long bv = LLONG_MAX, bi = LLONG_MAX;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const long long v = cnt * (long long)MSA_SIM_ONE - (long long)pairsum[k];
    const long long o = perm[k];
    rowsum[o] = v;
    if (v < bv || (v == bv && o < bi)) { bv = v; bi = o; }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const long long ov = __shfl_xor_sync(MSA_FULL_MASK, bv, d);
    const long long oi = __shfl_xor_sync(MSA_FULL_MASK, bi, d);
    if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sv[w] = bv; si[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int x = 1; x < (int)(blockDim.x >> 5); ++x)
      if (sv[x] < bv || (sv[x] == bv && si[x] < bi)) { bv = sv[x]; bi = si[x]; }
    part_val[blockIdx.x] = bv;
    part_idx[blockIdx.x] = bi;
  }
}

__global__ void k_argmin(int parts, const long long *__restrict__ part_val,
                         const long long *__restrict__ part_idx, long long *val, long long *idx) {
  if (threadIdx.x != 0) return;
  long long bv = LLONG_MAX, bi = LLONG_MAX;
  for (int x = 0; x < parts; ++x)
    if (part_val[x] < bv || (part_val[x] == bv && part_idx[x] < bi)) { bv = part_val[x]; bi = part_idx[x]; }
  *val = bv;
  *idx = bi;
}

// Similarities of the pairs re-run in int32 (their packed lanes may have
// overflowed), added where the center kernel would have added them.
__global__ void k_apply_overflow(int mode, const int2 *__restrict__ ovf,
                                 const int32_t *__restrict__ scores, int count,
                                 unsigned long long *pairsum, const int32_t *__restrict__ self) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= count) return;
  const int q = ovf[x].x, s = ovf[x].y;
  const unsigned long long sim = center_sim(scores[x], self[q], self[s]);
  if (mode == 0) {
    atomicAdd(&pairsum[s], sim);
    atomicAdd(&pairsum[q], sim);
  } else if (mode == 1) {
    atomicAdd(&pairsum[s], sim);
  } else {
    atomicAdd(&pairsum[q], sim);
  }
}

__global__ void k_self_pairs(int n, int2 *pairs, int32_t *dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) { pairs[k] = make_int2(k, k); dst[k] = k; }
}

__global__ void k_extract_scores(const int32_t *__restrict__ seg, int n, int32_t *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = seg[(size_t)k * 5];
}

int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b > cap ? cap : b);
}

}  // namespace

cudaError_t launch_encode(const uint8_t *letters, const int64_t *src_off, const int32_t *perm,
                          const int64_t *pstart, const int32_t *len, int n, const uint8_t *lut,
                          int padc, uint8_t *res, unsigned *err, cudaStream_t st) {
  const int threads = 256;
  const int blocks = blocks_for((int64_t)n * 32, threads, 65535);
  k_encode<<<blocks, threads, 0, st>>>(letters, src_off, perm, pstart, len, n, lut, padc, res, err);
  return cudaGetLastError();
}

cudaError_t launch_traceback(const uint8_t *codes, const int64_t *code_off,
                             const unsigned long long *best,
                             int sb, int se, const int32_t *len, const int32_t *perm,
                             const uint8_t *res, const int64_t *pstart, int center,
                             const int8_t *M, int K, int o, int e, int Lc, int G,
                             uint16_t *ins, uint8_t *occ, int32_t *seg, int32_t *score,
                             unsigned *err, cudaStream_t st, const int32_t *list, const int4 *box,
                             const unsigned long long *box_best) {
  const int cnt = se - sb;
  if (cnt <= 0) return cudaSuccess;
  const int threads = 128;
  k_traceback<<<(cnt + threads - 1) / threads, threads, 0, st>>>(codes, code_off, best, sb, se, len,
                                                                 perm, res, pstart, center, M, K, o,
                                                                 e, Lc, G, ins, occ, seg, score, err,
                                                                 list, box, box_best);
  return cudaGetLastError();
}

cudaError_t launch_colmax(const uint16_t *ins, int n, int Lc, int32_t *G, cudaStream_t st) {
  const int threads = 256;
  const int rows_per_block = 256;
  dim3 grid((Lc + 1 + threads - 1) / threads, (n + rows_per_block - 1) / rows_per_block);
  k_colmax<<<grid, threads, 0, st>>>(ins, n, Lc, rows_per_block, G);
  return cudaGetLastError();
}

cudaError_t launch_scan(const int32_t *G, int Lc, int32_t *off, int64_t *width, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(G, Lc, off, width);
  return cudaGetLastError();
}

cudaError_t launch_rows(const uint8_t *res, const int64_t *pstart, const int32_t *inv,
                        const uint16_t *ins, const uint8_t *occ, const int32_t *G,
                        const int32_t *off, int n, int Lc, int64_t W, const char *letters,
                        uint8_t *out, cudaStream_t st) {
  const int64_t rowbytes = (W + 15) / 16 * 16 + 16;
  if (rowbytes <= 96 * 1024) {  // rows staged in shared memory, 1-8 warps per CTA
    const int warps = (int)std::max<int64_t>(1, std::min<int64_t>(8, (96 * 1024) / rowbytes));
    const int smem = warps * (int)rowbytes;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute((const void *)k_rows_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int blocks = blocks_for((int64_t)n * 32, warps * 32, 8192);
    k_rows_staged<<<blocks, warps * 32, smem, st>>>(res, pstart, inv, ins, occ, off, n, Lc, W,
                                                    (int)rowbytes, letters, out);
    return cudaGetLastError();
  }
  const int threads = 256;
  const int blocks = blocks_for((int64_t)n * 32, threads, 8192);
  k_rows<<<blocks, threads, 0, st>>>(res, pstart, inv, ins, occ, G, off, n, Lc, W, letters, out);
  return cudaGetLastError();
}

cudaError_t launch_sp(const uint8_t *msa, int n, int64_t W, const uint8_t *sym_lut, int nsym,
                      int32_t *counts, unsigned long long *total, cudaStream_t st) {
  const int threads = 128, rows_per_block = 512;
  dim3 grid((unsigned)((W + threads - 1) / threads), (n + rows_per_block - 1) / rows_per_block);
  const int smem = nsym * threads * (int)sizeof(int32_t);
  k_sp_count<<<grid, threads, smem, st>>>(msa, n, W, sym_lut, nsym, rows_per_block, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sp_cost<<<(unsigned)((W + 255) / 256), 256, 0, st>>>(counts, n, W, nsym, total);
  return cudaGetLastError();
}

cudaError_t launch_center_finalize(int mode, int n, int nref, const int32_t *perm,
                                   const unsigned long long *pairsum, long long *rowsum,
                                   long long *argmin_val, long long *argmin_idx,
                                   long long *part_val, long long *part_idx, cudaStream_t st) {
  const int parts = blocks_for(n, 256, 1024);
  k_rowsum<<<parts, 256, 0, st>>>(mode, n, nref, perm, pairsum, rowsum, part_val, part_idx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_argmin<<<1, 32, 0, st>>>(parts, part_val, part_idx, argmin_val, argmin_idx);
  return cudaGetLastError();
}

cudaError_t launch_apply_overflow(int mode, const int2 *ovf, const int32_t *scores, int count,
                                  unsigned long long *pairsum, const int32_t *self, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  k_apply_overflow<<<(count + 255) / 256, 256, 0, st>>>(mode, ovf, scores, count, pairsum, self);
  return cudaGetLastError();
}

cudaError_t launch_self_pairs(int n, int2 *pairs, int32_t *dst, cudaStream_t st) {
  k_self_pairs<<<(n + 255) / 256, 256, 0, st>>>(n, pairs, dst);
  return cudaGetLastError();
}

cudaError_t launch_extract_scores(const int32_t *seg, int n, int32_t *out, cudaStream_t st) {
  k_extract_scores<<<(n + 255) / 256, 256, 0, st>>>(seg, n, out);
  return cudaGetLastError();
}
