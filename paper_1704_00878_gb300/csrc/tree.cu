// tree.cu -- the neighbour-joining tree over the MSA (the paper's section on
// NJ trees, Figure 4, citing Saitou and Nei): fixed-point p-distances between
// the merged rows, then neighbour joining on those integers.
//
// Distances: a CTA takes a 64 x 64 tile of row pairs (tiles on and above the
// diagonal), stages 256 columns of its 2 x 64 rows in shared memory and
// compares four columns per 32-bit word: x = a ^ b, a byte is nonzero iff
// ((x & 0x7f7f7f7f) + 0x7f7f7f7f | x) has its top bit set; the residue flags
// are the same test against '-' in every byte; per pair two SWAR byte
// counters (compared, mismatched) gather up to 64 words before they are
// summed into 32-bit totals.
//
// Neighbour joining: the matrix stays on the device (int32 -- every entry and
// joined distance within 2^30, else ERANGE -- positions in
// ascending slot order); every join is two launches -- the minimum of Q over
// the active pairs (warps over tiles of 8 rows x 256 columns, the last CTA to
// finish reduces the CTAs' minima) and the join itself (CTAs over the rows: branch lengths,
// the new node's row and column, the row sums updated in place; the last
// CTA to finish adds up the new node's row sum).  When a quarter of the
// positions are inactive the matrix is packed to the active ones, which keeps
// the work of a join near m^2 / 2.  No launch waits on another.
#include <algorithm>
#include <climits>
#include <vector>

#include "ctx.cuh"

namespace msa_detail {
namespace {

constexpr int kTile = 64;    // rows per side of a distance tile
constexpr int kWords = 64;   // 32-bit words (4 columns) per staged chunk
constexpr long long kDScale = 1LL << 20;
constexpr long long kDLimit = 1LL << 30;  // |distance| bound of the joins (int32 matrix)
constexpr int kArgThreads = 256;
constexpr int kRowBlk = 8;    // rows of one warp task (tile) of the Q minimum
constexpr int kColSeg = 256;  // columns of a tile: 8 per lane
constexpr int kJoinThreads = 1024;

// 0x80 in every byte of w that is nonzero
__device__ __forceinline__ uint32_t bytes_nonzero(uint32_t w) {
  return (((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;
}

// acc + (w >> 7) as one multiply-add (high half of w * 2^25) on the FMA pipe,
// beside the integer pipe the comparisons keep busy
__device__ __forceinline__ uint32_t add_top_bits(uint32_t acc, uint32_t w) {
  uint32_t d;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(1u << 25), "r"(acc));
  return d;
}

// sum of the four bytes of a SWAR counter
__device__ __forceinline__ uint32_t byte_sum(uint32_t c) {
  c = (c & 0x00ff00ffu) + ((c >> 8) & 0x00ff00ffu);
  return (c & 0xffffu) + (c >> 16);
}

// Rows of a distance tile: list A x list B (row indices of the MSA; null =
// the rows 0..nA-1 / 0..nB-1).  SYM: A and B are the same list, tiles on and
// above the diagonal, D[a][b] and D[b][a] stored (ld = nA); NEAREST: every
// tile of A x B, and per row of A the smallest (distance << 32 | position in
// B) by an atomic minimum -- the nearest row of B, ties to its first position.
struct PdistJob {
  const int32_t *ia, *ib;
  int nA, nB;
  bool sym;
  long long *D;               // SYM
  unsigned long long *near;   // NEAREST: one key per row of A
};

__global__ void __launch_bounds__(256) k_pdist(const uint8_t *__restrict__ msa, int64_t W,
                                               PdistJob job) {
  const int ta = blockIdx.y, tb = blockIdx.x;
  if (job.sym && tb < ta) return;
  __shared__ uint32_t sA[kTile][kWords + 1], sB[kTile][kWords + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int a0 = ta * kTile, b0 = tb * kTile;
  constexpr uint32_t kGap4 = 0x2d2d2d2du;  // "----"
  uint32_t comp[4][4] = {}, mism[4][4] = {};
  const int64_t nwords = (W + 3) / 4;
  for (int64_t w0 = 0; w0 < nwords; w0 += kWords) {
    __syncthreads();
    // stage 64 rows x 256 columns of each side; columns past W and rows past
    // the lists are gaps
    for (int idx = threadIdx.x; idx < kTile * kWords; idx += 256) {
      const int r = idx / kWords, w = idx - r * kWords;
      const int64_t c0 = (w0 + w) * 4;
      uint32_t va = kGap4, vb = kGap4;
      const int pa = a0 + r, pb = b0 + r;
      const int ra = pa < job.nA ? (job.ia ? job.ia[pa] : pa) : -1;
      const int rb = pb < job.nB ? (job.ib ? job.ib[pb] : pb) : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t c = c0 + u;
        if (c < W) {
          if (ra >= 0) va = (va & ~(0xffu << (8 * u))) | ((uint32_t)msa[(size_t)ra * W + c] << (8 * u));
          if (rb >= 0) vb = (vb & ~(0xffu << (8 * u))) | ((uint32_t)msa[(size_t)rb * W + c] << (8 * u));
        }
      }
      sA[r][w] = va;
      sB[r][w] = vb;
    }
    __syncthreads();
    uint32_t cc[4][4] = {}, cm[4][4] = {};  // byte counters: at most 64 per byte
#pragma unroll 4
    for (int w = 0; w < kWords; ++w) {
      uint32_t a[4], fa[4], b[4], fb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = sA[ty + 16 * i][w];
        fa[i] = bytes_nonzero(a[i] ^ kGap4);
        b[i] = sB[tx + 16 * i][w];
        fb[i] = bytes_nonzero(b[i] ^ kGap4);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t both = fa[i] & fb[j];
          cc[i][j] = add_top_bits(cc[i][j], both);
          cm[i][j] = add_top_bits(cm[i][j], bytes_nonzero(a[i] ^ b[j]) & both);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        comp[i][j] += byte_sum(cc[i][j]);
        mism[i][j] += byte_sum(cm[i][j]);
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty + 16 * i;
    if (a >= job.nA) continue;
    unsigned long long nearest = ~0ull;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx + 16 * j;
      if (b >= job.nB) continue;
      const long long d = comp[i][j] ? ((long long)mism[i][j] * kDScale) / comp[i][j] : kDScale;
      if (job.sym) {
        job.D[(size_t)a * job.nA + b] = d;
        if (ta != tb) job.D[(size_t)b * job.nA + a] = d;
      } else {
        const unsigned long long key = ((unsigned long long)d << 32) | (unsigned)b;
        nearest = key < nearest ? key : nearest;
      }
    }
    if (!job.sym && nearest != ~0ull) atomicMin(&job.near[a], nearest);
  }
}

struct Pick {
  long long q, xy;  // Q, then position pair x * 2^32 + y (x < y)
};
__device__ __forceinline__ bool pick_less(const Pick &u, const Pick &v) {
  return u.q < v.q || (u.q == v.q && u.xy < v.xy);
}
__device__ __forceinline__ Pick warp_min(Pick p) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Pick o;
    o.q = __shfl_xor_sync(MSA_FULL_MASK, p.q, off);
    o.xy = __shfl_xor_sync(MSA_FULL_MASK, p.xy, off);
    if (pick_less(o, p)) p = o;
  }
  return p;
}
__device__ __forceinline__ Pick block_min(Pick p, Pick *sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  p = warp_min(p);
  if (lane == 0) sh[w] = p;
  __syncthreads();
  if (w == 0) {
    p = lane < nw ? sh[lane] : Pick{LLONG_MAX, LLONG_MAX};
    p = warp_min(p);
  }
  return p;  // valid in warp 0
}

// The active pair of smallest Q = (m - 2) d(x, y) - r_x - r_y, ties to the
// smallest x, then y (positions ascend with the slots).  Warp tasks are tiles
// of kRowBlk rows x kColSeg columns of the upper triangle: a lane loads -r_y
// and the active flags of its kColSeg / 32 columns once per tile, then per
// row one int32 distance per column and one 64-bit multiply-add
// (m - 2) d - r_y, compared with the tile's best so far plus r_x.  Inside a
// tile a lane meets its cells in ascending (x, y), so a strict comparison
// keeps the first of equal values; tiles, lanes and CTAs then merge on
// (Q, x, y).  The last CTA to finish reduces every CTA's minimum into sel.
__global__ void __launch_bounds__(kArgThreads) k_nj_argmin(const int *__restrict__ D, int P,
                                                           const long long *__restrict__ r,
                                                           const uint8_t *__restrict__ act, int m,
                                                           const int2 *__restrict__ tasks, int ntask,
                                                           Pick *__restrict__ part,
                                                           unsigned *__restrict__ ticket,
                                                           int *__restrict__ sel) {
  constexpr int U = kColSeg / 32;
  __shared__ Pick sh[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int f = m - 2;
  Pick best{LLONG_MAX, LLONG_MAX};
  for (int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += warps) {
    const int2 tk = tasks[task];
    const int yb = tk.y + lane;
    long long nry[U];
    unsigned okm = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = yb + 32 * u;
      const bool ok = y < P && act[y];
      okm |= (ok ? 1u : 0u) << u;
      nry[u] = ok ? -r[y] : 0;
    }
    long long tq = LLONG_MAX;  // the tile's best Q for this lane, at (tx, ty)
    int tx = 0, ty = 0;
    const int xend = min(tk.x + kRowBlk, P);
    for (int x = tk.x; x < xend; ++x) {
      if (!act[x]) continue;  // the same x on every lane
      const long long rx = r[x];
      // columns y > x only: u from ceil((x + 1 - yb) / 32) on
      const int lim = x + 1 - yb;
      const int umin = lim <= 0 ? 0 : (lim + 31) >> 5;
      const unsigned rm = umin >= U ? 0u : okm & (0xffffffffu << umin);
      if (rm == 0) continue;
      const int *row = D + (size_t)x * P;
      int dv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) dv[u] = (rm >> u) & 1u ? row[yb + 32 * u] : 0;
      // q < tq  <=>  f d - r_y < tq + r_x (no overflow: |Q| < 2^63 by far)
      long long thr = tq == LLONG_MAX ? LLONG_MAX : tq + rx;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long v = (long long)f * dv[u] + nry[u];
        if (((rm >> u) & 1u) && v < thr) {
          thr = v;
          tq = v - rx;
          tx = x;
          ty = yb + 32 * u;
        }
      }
    }
    if (tq != LLONG_MAX) {
      const Pick c{tq, ((long long)tx << 32) | (long long)ty};
      if (pick_less(c, best)) best = c;
    }
  }
  best = block_min(best, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = best;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  Pick p{LLONG_MAX, LLONG_MAX};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const Pick o{__ldcg(&part[b].q), __ldcg(&part[b].xy)};  // written by other CTAs
    if (pick_less(o, p)) p = o;
  }
  __syncthreads();
  p = block_min(p, sh);
  if (threadIdx.x == 0) {
    sel[0] = (int)(p.xy >> 32);
    sel[1] = (int)(p.xy & 0xffffffffLL);
    *ticket = 0;
  }
}

// Join t of the positions sel = {x, y} (x < y): branch lengths, the new
// node n + t in position x, its distances floor((d(x,k) + d(y,k) - d(x,y)) / 2),
// the row sums, y retired.  CTAs take ranges of k; the last CTA to finish
// adds up their sums into r_x (every CTA has read r_x by then).
__global__ void __launch_bounds__(kJoinThreads) k_nj_join(int *__restrict__ D, int P,
                                                          long long *__restrict__ r,
                                                          uint8_t *__restrict__ act,
                                                          int *__restrict__ node, int m,
                                                          const int *__restrict__ sel, int t, int n,
                                                          int *__restrict__ joins,
                                                          double *__restrict__ lengths,
                                                          long long *__restrict__ part,
                                                          unsigned *__restrict__ ticket,
                                                          unsigned *__restrict__ err) {
  __shared__ long long wsum[kJoinThreads / 32];
  __shared__ bool last;
  const int x = sel[0], y = sel[1];
  const long long dxy = D[(size_t)x * P + y], rx = r[x], ry = r[y];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long f = m - 2;
    const double den = (double)(2 * f);
    lengths[2 * t] = (double)(f * dxy + rx - ry) / den;
    lengths[2 * t + 1] = (double)(f * dxy - rx + ry) / den;
    joins[2 * t] = node[x];
    joins[2 * t + 1] = node[y];
  }
  long long sum = 0;
  bool bad = false;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    if (!act[k] || k == x || k == y) continue;
    const long long dxk = D[(size_t)x * P + k], dyk = D[(size_t)y * P + k];
    const long long dn = (dxk + dyk - dxy) >> 1;
    bad |= dn > kDLimit || dn < -kDLimit;
    D[(size_t)x * P + k] = (int)dn;
    D[(size_t)k * P + x] = (int)dn;
    r[k] += dn - dxk - dyk;
    sum += dn;
  }
  if (bad) atomicOr(err, MSA_DERR_RANGE);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(MSA_FULL_MASK, sum, off);
  if (lane == 0) wsum[w] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += wsum[i];
    part[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  long long s = 0;
  for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&part[b]);
  r[x] = s;
  node[x] = n + t;
  act[y] = 0;
  *ticket = 0;
}

// Positions of the active entries, ascending (one CTA; P <= 65536).
__global__ void __launch_bounds__(1024) k_nj_index(const uint8_t *__restrict__ act, int P,
                                                   int *__restrict__ idx) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < P; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const int a = k < P && act[k] ? 1 : 0;
    int incl = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(MSA_FULL_MASK, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int v = wsum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(MSA_FULL_MASK, v, d);
        if (lane >= d) v += u;
      }
      wsum[lane] = v;
    }
    __syncthreads();
    const int before = carry + (w > 0 ? wsum[w - 1] : 0) + incl - a;
    if (a) idx[before] = k;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
}

// The matrix, row sums and node ids packed to the m active positions.
__global__ void k_nj_pack(const int *__restrict__ D, int P, const long long *__restrict__ r,
                          const int *__restrict__ node, const int *__restrict__ idx, int m,
                          int *__restrict__ D2, long long *__restrict__ r2,
                          int *__restrict__ node2, uint8_t *__restrict__ act2) {
  const int u = blockIdx.y;
  const int su = idx[u];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < m; v += gridDim.x * blockDim.x)
    D2[(size_t)u * m + v] = D[(size_t)su * P + idx[v]];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r2[u] = r[su];
    node2[u] = node[su];
    act2[u] = 1;
  }
}

// The root: the two active positions joined at the middle of their edge.
__global__ void k_nj_root(const int *__restrict__ D, int P, const uint8_t *__restrict__ act,
                          const int *__restrict__ node, int t, int *__restrict__ joins,
                          double *__restrict__ lengths) {
  if (threadIdx.x != 0) return;
  int a = -1, b = -1;
  for (int k = 0; k < P; ++k)
    if (act[k]) {
      if (a < 0) a = k;
      else { b = k; break; }
    }
  if (a < 0 || b < 0) return;
  const double half = (double)D[(size_t)a * P + b] / 2.0;
  joins[2 * t] = node[a];
  joins[2 * t + 1] = node[b];
  lengths[2 * t] = half;
  lengths[2 * t + 1] = half;
}

// The int64 matrix into the int32 one the joins work on; entries beyond the
// bound set the range error.
__global__ void k_nj_narrow(const long long *__restrict__ D64, size_t count, int *__restrict__ D,
                            unsigned *__restrict__ err) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const long long v = D64[i];
    bad |= v > kDLimit || v < -kDLimit;
    D[i] = (int)v;
  }
  if (bad) atomicOr(err, MSA_DERR_RANGE);
}

// Row sums (one warp per row), node ids, every position active.
__global__ void k_nj_init(long long *__restrict__ r, const int *__restrict__ D, int n,
                          int *__restrict__ node, uint8_t *__restrict__ act) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
    long long s = 0;
    for (int j = lane; j < n; j += 32) s += j == k ? 0 : D[(size_t)k * n + j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(MSA_FULL_MASK, s, off);
    if (lane == 0) {
      r[k] = s;
      node[k] = k;
      act[k] = 1;
    }
  }
}

// Distances among the merged rows idx[0..m) (device list, null = rows 0..m-1)
// into the m x m matrix D (device).
int list_distances(msa_ctx *ctx, const int32_t *idx, int m, long long *D) {
  const int T = (m + kTile - 1) / kTile;
  PdistJob job{idx, idx, m, m, true, D, nullptr};
  ++ctx->launches;
  k_pdist<<<dim3(T, T), 256, 0, ctx->st>>>(P<uint8_t>(ctx->msa), ctx->W, job);
  CK(cudaGetLastError());
  return MSA_OK;
}

// Per cluster c of the sample: the smallest (d(t, s) << 32 | s) over sample
// positions t in c and s outside it (the outgroup: the nearest sample row
// outside, ties to the smaller row).
__global__ void k_outgroups(const long long *__restrict__ D, int m, const int32_t *__restrict__ cl,
                            unsigned long long *__restrict__ key) {
  const int t = blockIdx.y;
  const int c = cl[t];
  unsigned long long best = ~0ull;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m; s += gridDim.x * blockDim.x)
    if (cl[s] != c) {
      const unsigned long long k = ((unsigned long long)D[(size_t)t * m + s] << 32) | (unsigned)s;
      best = k < best ? k : best;
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(MSA_FULL_MASK, best, off);
    best = o < best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&key[c], best);
}

int tree_distances(msa_ctx *ctx, DevBuf &D) {
  if (!ctx->merged) return fail(ctx, MSA_ESTATE, "merge the alignment first");
  const int n = ctx->n;
  TRY(ensure(ctx, D, sizeof(long long) * (size_t)n * n));
  return list_distances(ctx, nullptr, n, P<long long>(D));
}

// Neighbour joining of the n x n matrix in D (device, int64, left as it is).
int nj_device(msa_ctx *ctx, DevBuf &D, int n, int32_t *joins_out, double *lengths_out) {
  if (n < 2) return MSA_OK;
  DevBuf D1, D2, r, r2, node, node2, act, act2, idx, part, jpart, sel, joins, lengths, tasks;
  auto cleanup = [&]() {
    for (DevBuf *b : {&D1, &D2, &r, &r2, &node, &node2, &act, &act2, &idx, &part, &jpart, &sel, &joins,
                      &lengths, &tasks})
      release(ctx, *b);
  };
  int rc = [&]() -> int {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev);
    const int grid = std::max(1, sms) * 8;
    const int jmax = std::max(1, sms);  // CTAs of a join
    TRY(ensure(ctx, r, sizeof(long long) * n));
    TRY(ensure(ctx, node, sizeof(int) * n));
    TRY(ensure(ctx, act, (size_t)n));
    TRY(ensure(ctx, idx, sizeof(int) * n));
    TRY(ensure(ctx, part, sizeof(Pick) * grid));
    TRY(ensure(ctx, sel, sizeof(int) * 2 + 2 * sizeof(unsigned)));
    TRY(ensure(ctx, jpart, sizeof(long long) * jmax));
    TRY(ensure(ctx, joins, sizeof(int) * 2 * (size_t)(n - 1)));
    TRY(ensure(ctx, lengths, sizeof(double) * 2 * (size_t)(n - 1)));
    unsigned *ticket = reinterpret_cast<unsigned *>(P<int>(sel) + 2);
    CK(cudaMemsetAsync(ticket, 0, 2 * sizeof(unsigned), ctx->st));
    CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
    TRY(ensure(ctx, D1, sizeof(int) * (size_t)n * n));
    ctx->launches += 2;
    k_nj_narrow<<<grid, 256, 0, ctx->st>>>(P<long long>(D), (size_t)n * n, P<int>(D1), ctx->derr);
    CK(cudaGetLastError());
    k_nj_init<<<grid, 256, 0, ctx->st>>>(P<long long>(r), P<int>(D1), n, P<int>(node),
                                         P<uint8_t>(act));
    CK(cudaGetLastError());
    // the Q minimum's warp tasks for a matrix of P positions: tiles of
    // kRowBlk rows from x0, kColSeg columns from y0 > x0
    std::vector<int2> htasks;
    int ntask = 0;
    auto make_tasks = [&](int Pm) -> int {
      htasks.clear();
      for (int x0 = 0; x0 + 1 < Pm; x0 += kRowBlk)
        for (int y0 = x0 + 1; y0 < Pm; y0 += kColSeg) htasks.push_back(make_int2(x0, y0));
      ntask = (int)htasks.size();
      TRY(ensure(ctx, tasks, sizeof(int2) * std::max(ntask, 1)));
      CK(cudaMemcpyAsync(tasks.p, htasks.data(), sizeof(int2) * ntask, cudaMemcpyHostToDevice, ctx->st));
      return MSA_OK;
    };
    TRY(make_tasks(n));
    DevBuf *cD = &D1, *cR = &r, *cN = &node, *cA = &act;
    DevBuf *oD = &D2, *oR = &r2, *oN = &node2, *oA = &act2;
    int Pn = n, m = n, t = 0;
    // the Q minimum runs as many CTAs as stay resident (its warps loop over the tiles)
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nj_argmin, kArgThreads, 0);
    const int aresident = std::min(grid, std::max(1, sms) * std::max(1, per_sm));
    while (m > 2) {
      ctx->launches += 2;
      // a warp per task at least: small matrices take few CTAs
      const int agrid = std::max(1, std::min(aresident, (ntask + kArgThreads / 32 - 1) / (kArgThreads / 32)));
      k_nj_argmin<<<agrid, kArgThreads, 0, ctx->st>>>(P<int>(*cD), Pn, P<long long>(*cR),
                                                     P<uint8_t>(*cA), m, P<int2>(tasks), ntask,
                                                     P<Pick>(part), ticket, P<int>(sel));
      CK(cudaGetLastError());
      const int jgrid = std::max(1, std::min(jmax, (Pn + kJoinThreads - 1) / kJoinThreads));
      k_nj_join<<<jgrid, kJoinThreads, 0, ctx->st>>>(P<int>(*cD), Pn, P<long long>(*cR),
                                                     P<uint8_t>(*cA), P<int>(*cN), m, P<int>(sel), t,
                                                     n, P<int>(joins), P<double>(lengths),
                                                     P<long long>(jpart), ticket + 1, ctx->derr);
      CK(cudaGetLastError());
      --m;
      ++t;
      if (m > 2 && Pn >= 512 && 4 * m <= 3 * Pn) {  // pack to the active positions
        TRY(ensure(ctx, *oD, sizeof(int) * (size_t)m * m));
        TRY(ensure(ctx, *oR, sizeof(long long) * m));
        TRY(ensure(ctx, *oN, sizeof(int) * m));
        TRY(ensure(ctx, *oA, (size_t)m));
        ctx->launches += 2;
        k_nj_index<<<1, 1024, 0, ctx->st>>>(P<uint8_t>(*cA), Pn, P<int>(idx));
        CK(cudaGetLastError());
        k_nj_pack<<<dim3((m + 255) / 256, m), 256, 0, ctx->st>>>(
            P<int>(*cD), Pn, P<long long>(*cR), P<int>(*cN), P<int>(idx), m, P<int>(*oD),
            P<long long>(*oR), P<int>(*oN), P<uint8_t>(*oA));
        CK(cudaGetLastError());
        std::swap(cD, oD);
        std::swap(cR, oR);
        std::swap(cN, oN);
        std::swap(cA, oA);
        Pn = m;
        TRY(make_tasks(Pn));
      }
    }
    ++ctx->launches;
    k_nj_root<<<1, 32, 0, ctx->st>>>(P<int>(*cD), Pn, P<uint8_t>(*cA), P<int>(*cN), t,
                                      P<int>(joins), P<double>(lengths));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(joins_out, joins.p, sizeof(int) * 2 * (size_t)(n - 1), cudaMemcpyDefault,
                       ctx->st));
    CK(cudaMemcpyAsync(lengths_out, lengths.p, sizeof(double) * 2 * (size_t)(n - 1),
                       cudaMemcpyDefault, ctx->st));
    TRY(check_derr(ctx));
    return MSA_OK;
  }();
  cleanup();
  return rc;
}

// ---------------------------------------------------------------- clustered tree (host side)
// A rooted tree: kids[v] = its (child, length) pairs, none for a leaf.
using Kids = std::vector<std::vector<std::pair<int, double>>>;

// The unrooted tree of NJ joins over nleaf leaves (node nleaf + t for join t;
// the last join's two edges become one edge, its node unused).
static Kids unrooted(const std::vector<int32_t> &joins, const std::vector<double> &lengths, int nleaf) {
  const int T = nleaf - 1;
  Kids adj(2 * nleaf);
  auto link = [&](int a, int b, double l) { adj[a].push_back({b, l}); adj[b].push_back({a, l}); };
  for (int t = 0; t + 1 < T; ++t) {
    link(nleaf + t, joins[2 * t], lengths[2 * t]);
    link(nleaf + t, joins[2 * t + 1], lengths[2 * t + 1]);
  }
  link(joins[2 * (T - 1)], joins[2 * (T - 1) + 1], lengths[2 * (T - 1)] + lengths[2 * (T - 1) + 1]);
  return adj;
}

// The leaf farthest from src (distances summed along the path from src,
// ties to the smaller leaf) and each node's (parent, edge) toward src.
static int farthest(const Kids &adj, int src, int nleaf, double &dist_out,
                    std::vector<std::pair<int, double>> &par) {
  std::vector<double> dist(adj.size(), 0.0);
  std::vector<char> seen(adj.size(), 0);
  par.assign(adj.size(), {-1, 0.0});
  std::vector<int> stack = {src};
  seen[src] = 1;
  while (!stack.empty()) {
    const int v = stack.back();
    stack.pop_back();
    for (auto [w, l] : adj[v])
      if (!seen[w]) {
        seen[w] = 1;
        dist[w] = dist[v] + l;
        par[w] = {v, l};
        stack.push_back(w);
      }
  }
  int best = -1;
  for (int v = 0; v < nleaf; ++v)
    if (best < 0 || dist[v] > dist[best]) best = v;
  dist_out = dist[best];
  return best;
}

// Orient the unrooted adjacency away from `root`, skipping node `drop`.
static Kids orient(const Kids &adj, int root, int drop) {
  Kids kids(adj.size());
  std::vector<char> seen(adj.size(), 0);
  seen[root] = 1;
  if (drop >= 0) seen[drop] = 1;
  std::vector<int> stack = {root};
  while (!stack.empty()) {
    const int v = stack.back();
    stack.pop_back();
    for (auto [w, l] : adj[v])
      if (!seen[w]) {
        seen[w] = 1;
        kids[v].push_back({w, l});
        stack.push_back(w);
      }
  }
  return kids;
}

// The NJ tree rooted at the middle of its longest leaf-to-leaf path (see
// msa_nj_cluster_tree); the new root is node 2 nleaf - 2.
static Kids midpoint_rooted(const std::vector<int32_t> &joins, const std::vector<double> &lengths,
                            int nleaf, int &root) {
  Kids adj = unrooted(joins, lengths, nleaf);
  std::vector<std::pair<int, double>> par;
  double total = 0.0;
  const int a = farthest(adj, 0, nleaf, total, par);
  const int b = farthest(adj, a, nleaf, total, par);
  const double half = total / 2.0;
  int v = b;
  double walked = 0.0, l = 0.0;
  int u = -1;
  for (;;) {  // the last edge of the path at the latest (negative lengths)
    u = par[v].first;
    l = par[v].second;
    if (walked + l >= half || u == a) break;
    walked += l;
    v = u;
  }
  const double x = half - walked;
  auto drop_edge = [&](int p, int q) {
    auto &e = adj[p];
    e.erase(std::find_if(e.begin(), e.end(), [&](const std::pair<int, double> &z) { return z.first == q; }));
  };
  drop_edge(v, u);
  drop_edge(u, v);
  root = 2 * nleaf - 2;
  adj[root] = {{v, x}, {u, l - x}};
  adj[v].push_back({root, x});
  adj[u].push_back({root, l - x});
  return orient(adj, root, -1);
}

// Copy a rooted tree (leaf ids mapped to rows by name[]) into the arena.
static int graft(const Kids &kids, int root, const std::vector<int> &name, int nleaf, Kids &arena) {
  // iterative: children are copied before their parent
  std::vector<std::pair<int, int>> stack = {{root, 0}};
  std::vector<int> made(kids.size(), -1);
  while (!stack.empty()) {
    auto &[v, state] = stack.back();
    if (kids[v].empty()) {
      made[v] = name[v < nleaf ? v : 0];
      stack.pop_back();
      continue;
    }
    if (state == 0) {
      state = 1;
      const int vv = v;
      for (auto [w, l] : kids[vv]) stack.push_back({w, 0});
      continue;
    }
    const int id = (int)arena.size();
    arena.emplace_back();
    for (auto [w, l] : kids[v]) arena[id].push_back({made[w], l});
    made[v] = id;
    stack.pop_back();
  }
  return made[root];
}

int cluster_tree(msa_ctx *ctx, const std::vector<int32_t> &S, int cap, int32_t *joins_out,
                 double *lengths_out, int32_t *cluster_out) {
  const int n = ctx->n, m = (int)S.size();
  DevBuf dS, dS2, dlist, dnear, dcl, dkey;
  auto cleanup = [&]() { for (DevBuf *b : {&dS, &dS2, &dlist, &dnear, &dcl, &dkey}) release(ctx, *b); };
  int rc = [&]() -> int {
    // 1. the sample tree, midpoint-rooted
    TRY(ensure(ctx, dlist, sizeof(int32_t) * std::max(n, 1)));
    CK(cudaMemcpyAsync(dlist.p, S.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->st));
    TRY(ensure(ctx, dS, sizeof(long long) * (size_t)m * m));
    TRY(list_distances(ctx, P<int32_t>(dlist), m, P<long long>(dS)));
    std::vector<int32_t> sj(2 * std::max(m - 1, 0));
    std::vector<double> sl(2 * std::max(m - 1, 0));
    if (m > 1) TRY(nj_device(ctx, dS, m, sj.data(), sl.data()));
    CK(cudaStreamSynchronize(ctx->st));
    Kids skids;
    int sroot = 0;
    if (m > 1) skids = midpoint_rooted(sj, sl, m, sroot);
    else skids.assign(1, {});
    // leaves under every node (post-order)
    const int nn = (int)skids.size();
    std::vector<int> nleaves(nn, 0), lowleaf(nn, INT_MAX);
    {
      std::vector<std::pair<int, int>> stack = {{sroot, 0}};
      while (!stack.empty()) {
        auto &[v, st] = stack.back();
        if (skids[v].empty()) { nleaves[v] = 1; lowleaf[v] = v; stack.pop_back(); continue; }
        if (st == 0) { st = 1; const int vv = v; for (auto [w, l] : skids[vv]) stack.push_back({w, 0}); continue; }
        for (auto [w, l] : skids[v]) { nleaves[v] += nleaves[w]; lowleaf[v] = std::min(lowleaf[v], lowleaf[w]); }
        stack.pop_back();
      }
    }
    // 2. the cut: split the subtree holding the most sample rows (ties: the
    // smaller node; the root is never tied) until none holds more than cap
    std::vector<int> cuts = {sroot};
    for (;;) {
      int bi = 0;
      for (int k = 1; k < (int)cuts.size(); ++k) {
        const int v = cuts[k], w = cuts[bi];
        if (nleaves[v] > nleaves[w] || (nleaves[v] == nleaves[w] && v < w)) bi = k;
      }
      const int big = cuts[bi];
      if (nleaves[big] <= cap) break;
      cuts.erase(cuts.begin() + bi);
      for (auto [w, l] : skids[big]) cuts.push_back(w);
    }
    std::sort(cuts.begin(), cuts.end(), [&](int x, int y) { return lowleaf[x] < lowleaf[y]; });
    const int q = (int)cuts.size();
    std::vector<int32_t> leaf_cl(m, 0);
    {
      std::vector<int> is_cut(nn, -1);
      for (int c = 0; c < q; ++c) is_cut[cuts[c]] = c;
      std::vector<std::pair<int, int>> stack = {{sroot, -1}};
      while (!stack.empty()) {
        auto [v, c] = stack.back();
        stack.pop_back();
        if (is_cut[v] >= 0) c = is_cut[v];
        if (skids[v].empty()) leaf_cl[v] = c;
        for (auto [w, l] : skids[v]) stack.push_back({w, c});
      }
    }
    // 3. labels: sample rows their own cluster, others their nearest sample row's
    std::vector<int32_t> cluster(n, -1);
    {
      TRY(ensure(ctx, dnear, sizeof(unsigned long long) * n));
      CK(cudaMemsetAsync(dnear.p, 0xff, sizeof(unsigned long long) * n, ctx->st));
      const int TA = (n + kTile - 1) / kTile, TB = (m + kTile - 1) / kTile;
      PdistJob job{nullptr, P<int32_t>(dlist), n, m, false, nullptr, P<unsigned long long>(dnear)};
      ++ctx->launches;
      k_pdist<<<dim3(TB, TA), 256, 0, ctx->st>>>(P<uint8_t>(ctx->msa), ctx->W, job);
      CK(cudaGetLastError());
      std::vector<unsigned long long> near(n);
      CK(cudaMemcpyAsync(near.data(), dnear.p, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
      for (int i = 0; i < n; ++i) cluster[i] = leaf_cl[(int)(near[i] & 0xffffffffu)];
      for (int l = 0; l < m; ++l) cluster[S[l]] = leaf_cl[l];
    }
    // 4. outgroups
    std::vector<int> outgroup(q, -1);
    if (q > 1) {
      TRY(ensure(ctx, dcl, sizeof(int32_t) * m));
      TRY(ensure(ctx, dkey, sizeof(unsigned long long) * q));
      CK(cudaMemcpyAsync(dcl.p, leaf_cl.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->st));
      CK(cudaMemsetAsync(dkey.p, 0xff, sizeof(unsigned long long) * q, ctx->st));
      ++ctx->launches;
      k_outgroups<<<dim3((m + 255) / 256, m), 256, 0, ctx->st>>>(P<long long>(dS), m, P<int32_t>(dcl),
                                                                 P<unsigned long long>(dkey));
      CK(cudaGetLastError());
      std::vector<unsigned long long> key(q);
      CK(cudaMemcpyAsync(key.data(), dkey.p, sizeof(unsigned long long) * q, cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
      for (int c = 0; c < q; ++c) outgroup[c] = S[(int)(key[c] & 0xffffffffu)];
    }
    // 5. cluster trees into the arena (rows 0..n-1 are its leaves)
    Kids arena(n);
    std::vector<int> rows_of_cut(nn, -1);  // arena root of each cut's cluster tree
    std::vector<std::vector<int>> members(q);
    for (int i = 0; i < n; ++i) members[cluster[i]].push_back(i);
    for (int c = 0; c < q; ++c) {
      const std::vector<int> &R = members[c];
      if (R.size() == 1) { rows_of_cut[cuts[c]] = R[0]; continue; }
      std::vector<int> U = R;
      int opos = -1;
      if (q > 1) {
        U.push_back(outgroup[c]);
        std::sort(U.begin(), U.end());
        opos = (int)(std::lower_bound(U.begin(), U.end(), outgroup[c]) - U.begin());
      }
      const int u = (int)U.size();
      if (u > kMaxTreeRows) return fail(ctx, MSA_ERANGE, "a cluster of %d rows (at most %d)", u, kMaxTreeRows);
      std::vector<int32_t> U32(U.begin(), U.end());
      CK(cudaMemcpyAsync(dlist.p, U32.data(), sizeof(int32_t) * u, cudaMemcpyHostToDevice, ctx->st));
      TRY(ensure(ctx, dS2, sizeof(long long) * (size_t)u * u));
      TRY(list_distances(ctx, P<int32_t>(dlist), u, P<long long>(dS2)));
      std::vector<int32_t> cj(2 * (u - 1));
      std::vector<double> cl(2 * (u - 1));
      TRY(nj_device(ctx, dS2, u, cj.data(), cl.data()));
      CK(cudaStreamSynchronize(ctx->st));
      Kids ck;
      int croot;
      if (q == 1) {  // the NJ tree as it is rooted
        ck.assign(2 * u - 1, {});
        for (int t = 0; t < u - 1; ++t)
          ck[u + t] = {{cj[2 * t], cl[2 * t]}, {cj[2 * t + 1], cl[2 * t + 1]}};
        croot = 2 * u - 2;
      } else {  // rooted where the outgroup joins, the outgroup removed
        const Kids adj = unrooted(cj, cl, u);
        croot = adj[opos][0].first;
        ck = orient(adj, croot, opos);
      }
      std::vector<int> name(U.begin(), U.end());
      rows_of_cut[cuts[c]] = graft(ck, croot, name, u, arena);
    }
    // 6. the sample tree above the cuts, the cluster trees below
    int root;
    if (q == 1) {
      root = rows_of_cut[cuts[0]];
    } else {
      std::vector<int> made(nn, -1);
      std::vector<std::pair<int, int>> stack = {{sroot, 0}};
      while (!stack.empty()) {
        auto &[v, st] = stack.back();
        if (rows_of_cut[v] >= 0) { made[v] = rows_of_cut[v]; stack.pop_back(); continue; }
        if (st == 0) { st = 1; const int vv = v; for (auto [w, l] : skids[vv]) stack.push_back({w, 0}); continue; }
        const int id = (int)arena.size();
        arena.emplace_back();
        for (auto [w, l] : skids[v]) arena[id].push_back({made[w], l});
        made[v] = id;
        stack.pop_back();
      }
      root = made[sroot];
    }
    // 7. post-order, children by their smallest row, internal nodes n, n+1, ...
    if (n > 1) {
      const int na = (int)arena.size();
      std::vector<int> low(na, INT_MAX), id(na, -1);
      for (int i = 0; i < n; ++i) low[i] = i, id[i] = i;
      for (int v = n; v < na; ++v)  // arena children are always made before their parent
        for (auto [w, l] : arena[v]) low[v] = std::min(low[v], low[w]);
      for (int v = n; v < na; ++v)
        std::sort(arena[v].begin(), arena[v].end(),
                  [&](const std::pair<int, double> &x, const std::pair<int, double> &y) {
                    return low[x.first] < low[y.first];
                  });
      int t = 0;
      std::vector<std::pair<int, int>> stack = {{root, 0}};
      while (!stack.empty()) {
        auto &top = stack.back();
        const int v = top.first;
        if (v < n) { stack.pop_back(); continue; }
        if (top.second == 0) {
          top.second = 1;
          const int c0 = arena[v][0].first, c1 = arena[v][1].first;
          stack.push_back({c1, 0});  // the first child is finished first
          stack.push_back({c0, 0});
          continue;
        }
        id[v] = n + t;
        joins_out[2 * t] = id[arena[v][0].first];
        joins_out[2 * t + 1] = id[arena[v][1].first];
        lengths_out[2 * t] = arena[v][0].second;
        lengths_out[2 * t + 1] = arena[v][1].second;
        ++t;
        stack.pop_back();
      }
    }
    if (cluster_out) std::copy(cluster.begin(), cluster.end(), cluster_out);
    return MSA_OK;
  }();
  cleanup();
  return rc;
}

}  // namespace
}  // namespace msa_detail

using namespace msa_detail;

int msa_tree_distances(msa_ctx *ctx, int64_t *dist_out) {
  if (!ctx || !dist_out) return MSA_EINVAL;
  TRY(set_device(ctx));
  DevBuf D;
  int rc = [&]() -> int {
    stage_begin(ctx, ST_TREE);
    TRY(tree_distances(ctx, D));
    stage_end(ctx, ST_TREE);
    const size_t n = ctx->n;
    CK(cudaMemcpyAsync(dist_out, D.p, sizeof(long long) * n * n, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_TREE);
    return MSA_OK;
  }();
  release(ctx, D);
  return rc;
}

int msa_nj(msa_ctx *ctx, const int64_t *dist, int64_t n, int32_t *joins_out, double *lengths_out) {
  if (!ctx || !dist || n < 1 || n > kMaxTreeRows || ((!joins_out || !lengths_out) && n > 1))
    return MSA_EINVAL;
  TRY(set_device(ctx));
  DevBuf D;
  int rc = [&]() -> int {
    TRY(ensure(ctx, D, sizeof(long long) * (size_t)n * n));
    CK(cudaMemcpyAsync(D.p, dist, sizeof(long long) * (size_t)n * n, cudaMemcpyDefault, ctx->st));
    stage_begin(ctx, ST_TREE);
    TRY(nj_device(ctx, D, (int)n, joins_out, lengths_out));
    stage_end(ctx, ST_TREE);
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_TREE);
    return MSA_OK;
  }();
  release(ctx, D);
  return rc;
}

int msa_nj_tree(msa_ctx *ctx, int32_t *joins_out, double *lengths_out) {
  if (!ctx) return MSA_EINVAL;
  if (ctx->n > 1 && (!joins_out || !lengths_out)) return MSA_EINVAL;
  if (ctx->n > kMaxTreeRows) return fail(ctx, MSA_ERANGE, "more than %d sequences", kMaxTreeRows);
  TRY(set_device(ctx));
  DevBuf D;
  int rc = [&]() -> int {
    stage_begin(ctx, ST_TREE);
    TRY(tree_distances(ctx, D));
    TRY(nj_device(ctx, D, ctx->n, joins_out, lengths_out));
    stage_end(ctx, ST_TREE);
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_TREE);
    return MSA_OK;
  }();
  release(ctx, D);
  return rc;
}

int msa_nj_cluster_tree(msa_ctx *ctx, const int64_t *sample, int64_t nsample, int32_t cap,
                        int32_t *joins_out, double *lengths_out, int32_t *cluster_out) {
  if (!ctx || !sample || nsample < 1 || cap < 1) return MSA_EINVAL;
  if (ctx->n > 1 && (!joins_out || !lengths_out)) return MSA_EINVAL;
  if (!ctx->merged) return fail(ctx, MSA_ESTATE, "merge the alignment first");
  std::vector<int32_t> S;
  S.reserve(nsample);
  for (int64_t k = 0; k < nsample; ++k) {
    if (sample[k] < 0 || sample[k] >= ctx->n) return fail(ctx, MSA_EINVAL, "sample row out of range");
    S.push_back((int32_t)sample[k]);
  }
  std::sort(S.begin(), S.end());
  S.erase(std::unique(S.begin(), S.end()), S.end());
  if ((int64_t)S.size() > kMaxTreeRows) return fail(ctx, MSA_ERANGE, "a sample of more than %d rows", kMaxTreeRows);
  TRY(set_device(ctx));
  std::vector<int32_t> joins(2 * (size_t)std::max(ctx->n - 1, 0));
  std::vector<double> lengths(joins.size());
  std::vector<int32_t> cluster(ctx->n);
  stage_begin(ctx, ST_TREE);
  TRY(cluster_tree(ctx, S, cap, joins.data(), lengths.data(), cluster.data()));
  stage_end(ctx, ST_TREE);
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_TREE);
  if (!joins.empty()) {
    CK(cudaMemcpyAsync(joins_out, joins.data(), sizeof(int32_t) * joins.size(), cudaMemcpyDefault, ctx->st));
    CK(cudaMemcpyAsync(lengths_out, lengths.data(), sizeof(double) * lengths.size(), cudaMemcpyDefault, ctx->st));
  }
  if (cluster_out)
    CK(cudaMemcpyAsync(cluster_out, cluster.data(), sizeof(int32_t) * cluster.size(), cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}
