// anchored.cu -- alignment of similar sequences to the center by anchors (the
// paper's trie path for similar nucleotides: the center's segments are
// indexed, matched segments of the other sequence are skipped and only the
// unmatched stretches are aligned).
//
// The center is cut into non-overlapping segments of k residues; their keys
// (k residues of ceil(log2 K) bits each) are sorted on the host and held in
// shared memory.  One warp per subject: the lanes roll the keys of the
// subject's k-mers over contiguous chunks and binary-search them, collecting
// every (segment, position) match; the warp sorts the matches and runs the
// longest-chain recurrence (a match's predecessor is the first compatible
// match of the longest chains before it: increasing segment, sequence
// positions at least k apart); the lanes mark the anchors, then the warp
// aligns the stretches between consecutive anchors one after another,
// globally (Gotoh, W = open + (n-1) extend; lanes over the stretch's center
// rows in an anti-diagonal wavefront, codes in shared memory, traceback from
// the end: diagonal, then F, then E; a gap extends only when strictly better)
// and writes the inserted-space row.  The
// flanks follow the local path's rule.  A subject with no match, more
// matches than the warp holds (the smallest power of two >= max(64, 2S)), or
// a stretch longer than kBoxSide on either side goes to the Smith-Waterman
// kernels instead.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "sw_kernels.cuh"

namespace msa_detail {
namespace {

constexpr int kAnchThreads = 256, kAnchWarps = kAnchThreads / 32;
constexpr int kBoxSide = 80;                         // longest stretch side a lane aligns
constexpr int kNeg = -(1 << 29);                      // stands for minus infinity
constexpr int kPosBits = 13;                          // match = segment << 13 | position

struct AnchJob {
  int center;                          // sorted index
  int nseg, k, bits;
  const unsigned long long *seg_key;   // sorted segment keys
  const int32_t *seg_id;               // the segment of each sorted key
  int cap;                             // matches a warp holds (power of two)
  uint16_t *ins;
  uint8_t *occ;
  int32_t *seg;
  int32_t *score;
  int32_t *fallback;                   // subjects (sorted index) left to the local path
  unsigned *nfallback;
  unsigned long long *counter;
};

// Per-warp workspace of the stretch aligner: one code byte per cell and two
// ping-pong rows (H and F of a pass's bottom row) for stretches of more than
// 32 center residues.
constexpr int kRowInts = 2 * (kBoxSide + 1);
constexpr int kStretchBytes = kBoxSide * kBoxSide + 2 * kRowInts * 4;

__device__ __forceinline__ int gap_cost(int len, int o, int e) { return -(o + (len - 1) * e); }

// Global affine alignment of the stretch c[0..lc) x x[0..lx) by the whole
// warp (center residue cb + i + 1 is c[i]); writes its columns to the row and
// returns its score (the same value in every lane).  Lanes hold center rows
// (32 per pass) and sweep the columns as an anti-diagonal wavefront: the cell
// above comes from the lane above by shuffle, the row above a pass from the
// workspace.  Gotoh with W_k = o + (k - 1) e, the edges charged from the
// stretch's corner; the codes (source 1 diagonal / 2 F / 3 E, ties in that
// order; E and F extend only when strictly better) go to shared memory and
// lane 0 walks them back from the end.
__device__ int stretch_align_warp(const uint8_t *__restrict__ c, int lc, const uint8_t *__restrict__ x,
                                  int lx, const int8_t *__restrict__ sM, int K, int o, int e, int cb,
                                  uint16_t *__restrict__ in, uint8_t *__restrict__ oc,
                                  uint8_t *__restrict__ work, int lane) {
  if (lc == 0 && lx == 0) return 0;
  if (lc == 0) {  // residues inserted before center residue cb + 1
    if (lane == 0) in[cb] = (uint16_t)(in[cb] + lx);
    return gap_cost(lx, o, e);
  }
  if (lx == 0) return gap_cost(lc, o, e);  // center residues against gaps
  uint8_t *codes = work;
  int *rows = reinterpret_cast<int *>(work + kBoxSide * kBoxSide);
  int hlast = 0;
  const int npass = (lc + 31) / 32;
  for (int p = 0; p < npass; ++p) {
    const int i0 = 32 * p, R = min(32, lc - i0);
    const int *rin = rows + ((p + 1) & 1) * kRowInts;  // H, F of row i0 (pass p > 0)
    int *rout = rows + (p & 1) * kRowInts;
    const int i = i0 + lane + 1;  // this lane's row (1-based)
    const bool row_ok = lane < R;
    const int8_t *srow = sM + (row_ok ? c[i - 1] : 0) * K;
    int hs = 0, fs = kNeg, hl = 0, el = kNeg, hup_prev = 0;
    const int steps = lx + R - 1;
    for (int k = 0; k < steps; ++k) {
      int hup = __shfl_up_sync(MSA_FULL_MASK, hs, 1), fup = __shfl_up_sync(MSA_FULL_MASK, fs, 1);
      const int j = k - lane + 1;
      if (lane == 0 && j <= lx) {
        hup = p == 0 ? gap_cost(j, o, e) : rin[j];
        fup = p == 0 ? kNeg : rin[kBoxSide + 1 + j];
      }
      if (row_ok && j >= 1 && j <= lx) {
        int hdiag = hup_prev;
        if (j == 1) {
          hl = gap_cost(i, o, e);                         // H(i, 0)
          el = kNeg;
          hdiag = i == 1 ? 0 : gap_cost(i - 1, o, e);     // H(i - 1, 0)
        }
        const int eo = hl - o, ee = el - e, E = max(eo, ee);
        const int fo = hup - o, fe = fup - e, F = max(fo, fe);
        const int d = hdiag + srow[x[j - 1]];
        const int h = max(d, max(E, F));
        const int src = h == d ? 1 : (h == F ? 2 : 3);
        codes[(i - 1) * lx + (j - 1)] = (uint8_t)(src | ((ee > eo) << 2) | ((fe > fo) << 3));
        hs = h; fs = F; hl = h; el = E;
        if (lane == R - 1 && p + 1 < npass) { rout[j] = h; rout[kBoxSide + 1 + j] = F; }
        if (i == lc && j == lx) hlast = h;
      }
      hup_prev = hup;
    }
    __syncwarp();
  }
  const int score = __shfl_sync(MSA_FULL_MASK, hlast, (lc - 1) & 31);
  if (lane == 0) {
    int i = lc, j = lx, state = 0;  // 0 = H, 1 = F (center residue vs gap), 2 = E (inserted residue)
    while (i > 0 || j > 0) {
      if (state == 0) {
        if (i == 0) state = 2;
        else if (j == 0) state = 1;
        else {
          const int src = codes[(i - 1) * lx + (j - 1)] & 3;
          if (src == 1) { oc[cb + i] = 1; --i; --j; continue; }
          state = src == 2 ? 1 : 2;
        }
      }
      if (state == 1) {
        const bool ext = j == 0 ? i > 1 : ((codes[(i - 1) * lx + (j - 1)] >> 3) & 1);
        --i;
        state = ext ? 1 : 0;
      } else {
        const bool ext = i == 0 ? j > 1 : ((codes[(i - 1) * lx + (j - 1)] >> 2) & 1);
        in[cb + i] = (uint16_t)(in[cb + i] + 1);
        --j;
        state = ext ? 2 : 0;
      }
    }
  }
  __syncwarp();
  return score;
}

__global__ void __launch_bounds__(kAnchThreads) k_anchored(SeqSet ss, Scoring sc, AnchJob job,
                                                            const int32_t *__restrict__ perm) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  __shared__ int s_nm[kAnchWarps], s_subj[kAnchWarps];
  const int K = sc.K, kk = job.k, S = job.nseg;
  unsigned long long *skey = reinterpret_cast<unsigned long long *>(smem);
  int32_t *sid = reinterpret_cast<int32_t *>(skey + S);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *mbuf = reinterpret_cast<uint32_t *>(sid + S + (S & 1)) + (size_t)w * job.cap * 2;
  int16_t *mlen = reinterpret_cast<int16_t *>(mbuf + job.cap);
  int16_t *mpred = mlen + job.cap;
  uint8_t *work = reinterpret_cast<uint8_t *>(reinterpret_cast<uint32_t *>(sid + S + (S & 1)) +
                                              (size_t)kAnchWarps * job.cap * 2) +
                  (size_t)w * kStretchBytes;
  for (int i = threadIdx.x; i < K * K; i += kAnchThreads) sM[i] = sc.M[i];
  for (int i = threadIdx.x; i < S; i += kAnchThreads) { skey[i] = job.seg_key[i]; sid[i] = job.seg_id[i]; }
  __syncthreads();
  const unsigned long long mask =
      job.bits * kk >= 64 ? ~0ull : ((1ull << (job.bits * kk)) - 1ull);
  const int Lc = ss.len[job.center];
  const uint8_t *rc = ss.res + ss.pstart[job.center];
  for (;;) {
    __syncwarp();  // every lane is done with the last subject's shared state
    if (lane == 0) {
      s_subj[w] = (int)atomicAdd(job.counter, 1ull);
      s_nm[w] = 0;
    }
    __syncwarp();
    const int kx = s_subj[w];
    if (kx >= ss.n) break;
    const int Ls = ss.len[kx];
    const uint8_t *x = ss.res + ss.pstart[kx];
    // (a) every match of a center segment, lanes over contiguous chunks
    const int npos = Ls - kk + 1;
    if (npos > 0) {
      const int chunk = (npos + 31) / 32;
      const int p0 = lane * chunk, p1 = min(npos, p0 + chunk);
      unsigned long long key = 0ull;
      if (p0 < p1)
        for (int u = 0; u < kk - 1; ++u) key = (key << job.bits) | x[p0 + u];
      for (int p = p0; p < p1; ++p) {
        key = ((key << job.bits) | x[p + kk - 1]) & mask;
        int lo = 0, hi = S;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (skey[mid] < key) lo = mid + 1; else hi = mid;
        }
        for (int q = lo; q < S && skey[q] == key; ++q) {
          const int slot = atomicAdd(&s_nm[w], 1);
          if (slot < job.cap) mbuf[slot] = ((uint32_t)sid[q] << kPosBits) | (uint32_t)p;
        }
      }
    }
    __syncwarp();
    const int M = s_nm[w];
    if (M == 0 || M > job.cap) {  // no anchor, or more matches than the warp holds
      if (lane == 0) {
        const unsigned slot = atomicAdd(job.nfallback, 1u);
        job.fallback[slot] = kx;
      }
      continue;
    }
    // (b) sort the matches by (segment, position): bitonic over a power of two
    int P = 1;
    while (P < M) P <<= 1;
    for (int i = M + lane; i < P; i += 32) mbuf[i] = 0xffffffffu;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int jx = i ^ stride;
          if (jx > i) {
            const uint32_t a = mbuf[i], b = mbuf[jx];
            const bool up = (i & size) == 0;
            if ((a > b) == up) { mbuf[i] = b; mbuf[jx] = a; }
          }
        }
        __syncwarp();
      }
    // (c) longest chain: len[m] = 1 + the longest compatible chain before it
    // (its first match on ties), the chain ending at the first longest
    int best_len = 0, best_m = 0;
    for (int m = 0; m < M; ++m) {
      const int sm = (int)(mbuf[m] >> kPosBits), pm = (int)(mbuf[m] & ((1u << kPosBits) - 1));
      int bl = 0, bq = INT_MAX;
      for (int q = lane; q < m; q += 32) {
        const int sq = (int)(mbuf[q] >> kPosBits), pq = (int)(mbuf[q] & ((1u << kPosBits) - 1));
        if (sq < sm && pq + kk <= pm && mlen[q] > bl) { bl = mlen[q]; bq = q; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const int ol = __shfl_xor_sync(MSA_FULL_MASK, bl, off);
        const int oq = __shfl_xor_sync(MSA_FULL_MASK, bq, off);
        if (ol > bl || (ol == bl && oq < bq)) { bl = ol; bq = oq; }
      }
      if (lane == 0) {
        mlen[m] = (int16_t)(bl + 1);
        mpred[m] = (int16_t)(bl > 0 ? bq : -1);
      }
      if (bl + 1 > best_len) { best_len = bl + 1; best_m = m; }
      __syncwarp();
    }
    // the chain (match indices, in order) into mlen[0..T)
    const int T = best_len;
    if (lane == 0) {
      int m = best_m;
      for (int t = T - 1; t >= 0; --t) { const int pm = mpred[m]; mlen[t] = (int16_t)m; m = pm; }
    }
    __syncwarp();
    auto anchor_s = [&](int t) { return (int)(mbuf[mlen[t]] >> kPosBits); };
    auto anchor_p = [&](int t) { return (int)(mbuf[mlen[t]] & ((1u << kPosBits) - 1)); };
    // (d) stretches a lane cannot hold send the subject to the local path
    bool big = false;
    for (int t = lane; t + 1 < T; t += 32) {
      const int lc = anchor_s(t + 1) * kk - (anchor_s(t) * kk + kk);
      const int lx = anchor_p(t + 1) - (anchor_p(t) + kk);
      big |= lc > kBoxSide || lx > kBoxSide;
    }
    if (__any_sync(MSA_FULL_MASK, big)) {
      if (lane == 0) {
        const unsigned slot = atomicAdd(job.nfallback, 1u);
        job.fallback[slot] = kx;
      }
      continue;
    }
    // (e) anchors, stretches, flanks: the row of this subject
    const int orig = perm[kx];
    uint16_t *in = job.ins + (size_t)orig * (Lc + 1);
    uint8_t *oc = job.occ + (size_t)orig * (Lc + 1);
    int score = 0;
    for (int t = lane; t < T; t += 32) {
      const int ca = anchor_s(t) * kk, xa = anchor_p(t);
      for (int u = 0; u < kk; ++u) {
        oc[ca + u + 1] = 1;
        score += sM[rc[ca + u] * K + x[xa + u]];
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) score += __shfl_xor_sync(MSA_FULL_MASK, score, off);
    for (int t = 0; t + 1 < T; ++t) {
      const int cb = anchor_s(t) * kk + kk, xb = anchor_p(t) + kk;
      score += stretch_align_warp(rc + cb, anchor_s(t + 1) * kk - cb, x + xb, anchor_p(t + 1) - xb,
                                  sM, K, sc.o, sc.e, cb, in, oc, work, lane);
    }
    if (lane == 0) {
      const int i1 = anchor_s(0) * kk, j1 = anchor_p(0);
      const int i2 = anchor_s(T - 1) * kk + kk, j2 = anchor_p(T - 1) + kk;
      const int kp = min(i1, j1);
      for (int t = 0; t < kp; ++t) oc[i1 - t] = 1;
      if (j1 > i1) in[0] = (uint16_t)(in[0] + (j1 - i1));
      const int a = Lc - i2, b = Ls - j2, ks = min(a, b);
      for (int t = 1; t <= ks; ++t) oc[i2 + t] = 1;
      if (b > a) in[Lc] = (uint16_t)(in[Lc] + (b - a));
      int32_t *sg = job.seg + (size_t)orig * 5;
      sg[0] = score; sg[1] = i1; sg[2] = j1; sg[3] = i2; sg[4] = j2;
      job.score[orig] = score;
    }
    __syncwarp();
  }
}

int anchored_smem(int nseg, int cap) {
  return nseg * 12 + (nseg & 1) * 4 + kAnchWarps * cap * 8 + kAnchWarps * kStretchBytes;
}

// The local path (Smith-Waterman fill with codes, traceback) for a list of
// subjects (sorted indices, ascending length) over a view of the set whose
// last entry is the center; rows land at their input indices.
int align_subset_local(msa_ctx *ctx, int kc, const std::vector<int32_t> &subj, float &ms) {
  const int nv = (int)subj.size() + 1;
  std::vector<int64_t> vstart(nv);
  std::vector<int32_t> vlen(nv), vperm(nv);
  for (int v = 0; v + 1 < nv; ++v) {
    vstart[v] = ctx->pstart[subj[v]];
    vlen[v] = ctx->len_sorted[subj[v]];
    vperm[v] = ctx->perm[subj[v]];
  }
  vstart[nv - 1] = ctx->pstart[kc];
  vlen[nv - 1] = ctx->len_sorted[kc];
  vperm[nv - 1] = ctx->perm[kc];
  const int Lc = vlen[nv - 1];
  const bool packed = align_packed(ctx, Lc);
  const int R = kCodesR, G = align_lanes(ctx, Lc, packed);
  const int npass = (Lc + G * R - 1) / (G * R);
  std::vector<int64_t> offs(nv, 0);
  int64_t acc = 0;
  for (int v = 0; v + 1 < nv; ++v) { offs[v] = acc; acc += (int64_t)code_words(vlen[v], Lc, G) * 8; }
  DevBuf vs, vl, vp, vo;
  auto cleanup = [&]() { for (DevBuf *b : {&vs, &vl, &vp, &vo}) release(ctx, *b); };
  int rc = [&]() -> int {
    TRY(ensure(ctx, vs, sizeof(int64_t) * nv));
    TRY(ensure(ctx, vl, sizeof(int32_t) * nv));
    TRY(ensure(ctx, vp, sizeof(int32_t) * nv));
    TRY(ensure(ctx, vo, sizeof(int64_t) * nv));
    TRY(ensure(ctx, ctx->codes, (size_t)std::max<int64_t>(acc, 8)));
    TRY(ensure(ctx, ctx->best, sizeof(unsigned long long) * nv));
    CK(cudaMemcpyAsync(vs.p, vstart.data(), sizeof(int64_t) * nv, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(vl.p, vlen.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(vp.p, vperm.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(vo.p, offs.data(), sizeof(int64_t) * nv, cudaMemcpyHostToDevice, ctx->st));
    const SeqSet vss{P<uint8_t>(ctx->res), P<int64_t>(vs), P<int32_t>(vl), nv};
    const Scoring sc = scoring(ctx);
    const int smem = codes_smem_bytes(ctx->K, npass * G * R);
    const int cta = align_cta(ctx, G, packed);
    const int grid = codes_grid(G, packed, smem, cta);
    if (npass > 1)
      TRY(ensure(ctx, ctx->scratch, (size_t)grid * (codes_threads(packed, cta) / G) * 2 * ctx->maxlen * sizeof(int2)));
    CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
    CodesJob job;
    job.center = nv - 1;
    job.sb = 0;
    job.se = nv - 1;
    job.code_off = P<int64_t>(vo);
    job.codes = P<uint8_t>(ctx->codes);
    job.best = P<unsigned long long>(ctx->best);
    job.npass = npass;
    job.counter = ctx->dcounter;
    job.scratch = P<int2>(ctx->scratch);
    job.scratch_cols = ctx->maxlen;
    cudaEvent_t e0 = ctx->ev[2 * ST_TRACE], e1 = ctx->ev[2 * ST_TRACE + 1];
    CK(cudaEventRecord(e0, ctx->st));
    CK((++ctx->launches, launch_codes)(G, packed, vss, sc, job, grid, ctx->st, true, cta));
    CK((++ctx->launches, launch_traceback)(P<uint8_t>(ctx->codes), P<int64_t>(vo),
                                           P<unsigned long long>(ctx->best), 0, nv - 1,
                                           P<int32_t>(vl), P<int32_t>(vp), vss.res, vss.pstart,
                                           nv - 1, sc.M, sc.K, sc.o, sc.e, Lc, G,
                                           P<uint16_t>(ctx->ins), P<uint8_t>(ctx->occ),
                                           P<int32_t>(ctx->seg), P<int32_t>(ctx->score),
                                           ctx->derr, ctx->st, nullptr, nullptr, nullptr));
    CK(cudaEventRecord(e1, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms += t;
    return MSA_OK;
  }();
  cleanup();
  return rc;
}

}  // namespace
}  // namespace msa_detail

using namespace msa_detail;

extern "C" int msa_align_anchored(msa_ctx *ctx, int64_t center, int32_t k, int32_t *scores_out,
                                  int64_t *fallback_out) {
  if (!ctx) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (center < 0 || center >= ctx->n) return fail(ctx, MSA_EINVAL, "center index out of range");
  int bits = 1;
  while ((1 << bits) < ctx->K) ++bits;
  if (k < 1 || k * bits > 64) return fail(ctx, MSA_EINVAL, "segment length %d outside 1..%d", k, 64 / bits);
  TRY(set_device(ctx));
  const int n = ctx->n;
  const int kc = ctx->inv[center];
  const int Lc = ctx->len_sorted[kc];
  if (Lc >= (1 << 13) || ctx->maxlen >= (1 << 13))
    return fail(ctx, MSA_ERANGE, "anchored path holds sequences below 8192 residues");
  ctx->aligned = ctx->merged = false;
  ctx->center = center;
  ctx->Lc = Lc;
  // the center's segment keys, sorted (host: one pass over Lc residues)
  const int S = Lc / k;
  std::vector<uint8_t> cres(Lc);
  CK(cudaMemcpyAsync(cres.data(), P<uint8_t>(ctx->res) + ctx->pstart[kc], Lc, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  std::vector<std::pair<unsigned long long, int32_t>> segs(S);
  for (int s = 0; s < S; ++s) {
    unsigned long long key = 0ull;
    for (int u = 0; u < k; ++u) key = (key << bits) | cres[(size_t)s * k + u];
    segs[s] = {key, s};
  }
  std::sort(segs.begin(), segs.end());
  std::vector<unsigned long long> keys(S);
  std::vector<int32_t> ids(S);
  for (int s = 0; s < S; ++s) { keys[s] = segs[s].first; ids[s] = segs[s].second; }
  // matches a warp holds: the smallest power of two >= max(64, 2 S) (more
  // send the sequence to the local path); it must fit shared memory
  int cap = 64;
  while (cap < 2 * S) cap <<= 1;
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->dev);
  const int smem = anchored_smem(S, cap);
  if (smem + 2048 > dev_smem)
    return fail(ctx, MSA_ERANGE, "%d center segments of k = %d need more shared memory", S, k);
  const size_t row = (size_t)Lc + 1;
  TRY(ensure(ctx, ctx->ins, sizeof(uint16_t) * row * n));
  TRY(ensure(ctx, ctx->occ, row * n));
  TRY(ensure(ctx, ctx->seg, sizeof(int32_t) * 5 * n));
  TRY(ensure(ctx, ctx->score, sizeof(int32_t) * n));
  DevBuf dk, di, df, dn;
  auto cleanup = [&]() { for (DevBuf *b : {&dk, &di, &df, &dn}) release(ctx, *b); };
  int rc = [&]() -> int {
    TRY(ensure(ctx, dk, sizeof(unsigned long long) * std::max(S, 1)));
    TRY(ensure(ctx, di, sizeof(int32_t) * std::max(S, 1)));
    TRY(ensure(ctx, df, sizeof(int32_t) * n));
    TRY(ensure(ctx, dn, sizeof(unsigned)));
    if (S > 0) {
      CK(cudaMemcpyAsync(dk.p, keys.data(), sizeof(unsigned long long) * S, cudaMemcpyHostToDevice, ctx->st));
      CK(cudaMemcpyAsync(di.p, ids.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, ctx->st));
    }
    CK(cudaMemsetAsync(ctx->ins.p, 0, sizeof(uint16_t) * row * n, ctx->st));
    CK(cudaMemsetAsync(ctx->occ.p, 0, row * n, ctx->st));
    CK(cudaMemsetAsync(dn.p, 0, sizeof(unsigned), ctx->st));
    CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
    CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
    AnchJob job;
    job.center = kc;
    job.nseg = S;
    job.k = k;
    job.bits = bits;
    job.seg_key = P<unsigned long long>(dk);
    job.seg_id = P<int32_t>(di);
    job.cap = cap;
    job.ins = P<uint16_t>(ctx->ins);
    job.occ = P<uint8_t>(ctx->occ);
    job.seg = P<int32_t>(ctx->seg);
    job.score = P<int32_t>(ctx->score);
    job.fallback = P<int32_t>(df);
    job.nfallback = P<unsigned>(dn);
    job.counter = ctx->dcounter;
    if (smem > 48 * 1024)
      CK(cudaFuncSetAttribute((const void *)k_anchored, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0, sms = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_anchored, kAnchThreads, smem));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev);
    const int grid = std::max(1, per_sm) * std::max(1, sms);
    stage_begin(ctx, ST_ALIGN);
    ++ctx->launches;
    k_anchored<<<grid, kAnchThreads, smem, ctx->st>>>(seqset(ctx), scoring(ctx), job,
                                                      P<int32_t>(ctx->d_perm));
    CK(cudaGetLastError());
    stage_end(ctx, ST_ALIGN);
    unsigned nf = 0;
    CK(cudaMemcpyAsync(&nf, dn.p, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_ALIGN);
    float ms_local = 0.f;
    if (nf > 0) {
      std::vector<int32_t> fb(nf);
      CK(cudaMemcpyAsync(fb.data(), df.p, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
      std::sort(fb.begin(), fb.end());  // sorted positions ascend in length
      // chunks whose codes fit the budget
      const int G = align_lanes(ctx, Lc, align_packed(ctx, Lc));
      size_t budget = std::max<size_t>(ctx->codes_budget, code_words(ctx->maxlen, Lc, G) * 8);
      size_t acc = 0;
      std::vector<int32_t> part;
      for (size_t x = 0; x <= fb.size(); ++x) {
        const size_t sz = x < fb.size() ? code_words(ctx->len_sorted[fb[x]], Lc, G) * 8 : 0;
        if (x == fb.size() || (acc + sz > budget && !part.empty())) {
          if (!part.empty()) TRY(align_subset_local(ctx, kc, part, ms_local));
          part.clear();
          acc = 0;
          if (x == fb.size()) break;
        }
        part.push_back(fb[x]);
        acc += sz;
      }
    }
    ctx->stage_ms[ST_ALIGN_K] = ctx->stage_ms[ST_ALIGN];
    ctx->stage_ms[ST_TRACE] = ms_local;
    int64_t cells = 0;  // the local path's cells only (the anchored ones are not a full DP)
    if (fallback_out) *fallback_out = (int64_t)nf;
    ctx->cells[1] = cells;
    TRY(check_derr(ctx));
    if (scores_out) {
      CK(cudaMemcpyAsync(scores_out, ctx->score.p, sizeof(int32_t) * n, cudaMemcpyDefault, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
    ctx->aligned = true;
    return MSA_OK;
  }();
  cleanup();
  return rc;
}
