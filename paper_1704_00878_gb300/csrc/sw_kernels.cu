// sw_kernels.cu -- affine-gap Smith-Waterman fills (HAlign-II Eq. 1-2 in
// Gotoh's form) as anti-diagonal wavefronts over groups of G threads.
//
// A group of G lanes owns one pass of G*R query rows: lane t holds rows
// [t*R, t*R+R) in registers and, at step k, fills column j = k - t of the
// subject.  The bottom row of lane t (H and F) reaches lane t+1 through a warp
// shuffle one step later, so the whole pass advances one anti-diagonal per
// step without shared-memory traffic.  Queries longer than G*R rows take
// several passes; the bottom row of one pass (H and F per column) is kept in a
// small per-group global buffer for the next.
//
// Scores come from a query profile in shared memory, biased by the gap-open
// penalty: prof[r*stride + i] = s(query_i, r) + o, every residue row starting
// on the same bank so the lanes of one load phase never conflict.
//
// Per cell (all DPX instructions but the first add), with E* = E + o and
// F* = F + o:
//   P = Hdiag + (s + o);  F* = max(F*_up - e, H_up);  M = max(P, E*, F*);
//   H = max(M - o, 0);    E*' = max(E* - e, H);       best = max(best, H)
// Packed mode keeps two subjects in the int16 halves of each register.
#include "sw_kernels.cuh"
#include "dp_pass.cuh"
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

namespace {

// One pass of G*R rows, score only.  prof points at the pass's row 0 and
// holds s(query_i, r) + o (>= 0; padding rows hold 0, i.e. a score of -o).
// The cell update works with E* = E + o and F* = F + o:
//   P  = Hdiag + (s + o)          one 32-bit add: never carries across the
//                                 int16 lanes because every lane stays >= 0
//   F* = max(F*_up - e, H_up)     M = max(P, E*, F*)     H = max(M - o, 0)
//   E*' = max(E* - e, H)          best = max(best, H)
// i.e. 4.5 DPX instructions per register of cells, the lane-local add aside.
// scr_in: H,F* of the row above the pass per column (nullptr: the top row of
// the matrix, H = 0, F* = 0 (F = -o)).  scr_out: where the last lane stores
// its bottom row (nullptr for the last pass).  Returns the lane's best H.
template <int G, int R, bool PACK>
__device__ __forceinline__ int wave_pass(const int8_t *__restrict__ prof, int stride,
                                         const uint8_t *__restrict__ rA, int LA,
                                         const uint8_t *__restrict__ rB, int LB, int Lw, int t,
                                         int base_lane, int padc, int o, int e,
                                         const int2 *__restrict__ scr_in,
                                         int2 *__restrict__ scr_out) {
  using C = Cell<PACK>;
  const int negO = C::splat(-o), negE = C::splat(-e);
  const uint32_t pc = (uint32_t)padc;
  auto fetch = [&](int col) -> uint32_t {
    uint32_t v = residue_at(rA, LA, col, pc);
    if constexpr (PACK) v |= residue_at(rB, LB, col, pc) << 8;
    return v;
  };

  int H[R], E[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { H[r] = 0; E[r] = 0; }
  int hbot = 0, fbot = 0, htop_prev = 0, best = 0;
  uint32_t resv = pc | (pc << 8);
  uint32_t cur = fetch(t), nxt = fetch(G + t);
  // the row above the pass, prefetched two columns ahead
  int2 sv0 = make_int2(0, 0), sv1 = make_int2(0, 0);
  if (scr_in != nullptr) {
    if (0 < Lw) sv0 = scr_in[0];
    if (1 < Lw) sv1 = scr_in[1];
  }
  const int8_t *pb = prof + t * R;
  const int steps = Lw + G - 1;

#pragma unroll 4
  for (int k = 0; k < steps; ++k) {
    const int kk = k & (G - 1);
    if (kk == 0 && k > 0) { cur = nxt; nxt = fetch(k + G + t); }
    const uint32_t r0 = __shfl_sync(MSA_FULL_MASK, cur, base_lane + kk);
    uint32_t rin = __shfl_up_sync(MSA_FULL_MASK, resv, 1);
    int hin = __shfl_up_sync(MSA_FULL_MASK, hbot, 1);
    int fin = __shfl_up_sync(MSA_FULL_MASK, fbot, 1);
    const int2 sv = sv0;
    sv0 = sv1;
    if (scr_in != nullptr && k + 2 < Lw) sv1 = scr_in[k + 2];
    if (t == 0) {
      rin = r0;
      const bool above = scr_in != nullptr && k < Lw;
      hin = above ? sv.x : 0;
      fin = above ? sv.y : 0;
    }
    resv = rin;
    ProfRow<R> pa, pq;
    pa.load(pb + (int)(resv & 0xffu) * stride);
    if constexpr (PACK) pq.load(pb + (int)(resv >> 8) * stride);

    int hdiag = htop_prev;
    htop_prev = hin;
    int hup = hin;
    int f = fin;
    Unroll<R>::run([&](auto ic) {
      constexpr int r = decltype(ic)::value;
      int s;
      if constexpr (PACK) s = C::template score<r & 3>(pa.w[r >> 2], pq.w[r >> 2]);
      else s = C::template score<r & 3>(pa.w[r >> 2], 0u);
      const int pdiag = hdiag + s;              // lanes stay in [0, 32767]: no carry
      f = C::addmax(f, negE, hup);              // F*
      const int m = C::vmax3(pdiag, E[r], f);   // max(P, E*, F*)
      const int hn = C::addmax_relu(m, negO, 0);
      E[r] = C::addmax(E[r], negE, hn);         // E* of the next column
      hdiag = H[r];
      H[r] = hn;
      hup = hn;
      if constexpr ((r & 1) == 1) best = C::vmax3(best, H[r - 1], hn);
    });
    hbot = H[R - 1];
    fbot = f;
    if (scr_out != nullptr && t == G - 1) {
      const int j = k - (G - 1);
      if (j >= 0 && j < Lw) scr_out[j] = make_int2(hbot, fbot);
    }
  }
  return best;
}

// ------------------------------------------------------------ center scores
// Work item = (query q, block of SPI consecutive subjects).  The CTA builds q's
// profile, each group aligns LANES subjects against it; results go straight
// into the per-sequence sums of center_sim used by the distance row sums.
template <int G, int R, bool PACK>
__global__ void __launch_bounds__(kCenterThreads)
k_center(SeqSet ss, Scoring sc, CenterJob job) {
  extern __shared__ __align__(16) int8_t smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  __shared__ long long s_item;
  __shared__ unsigned long long s_qsum;
  constexpr int NT = kCenterThreads, NG = NT / G, LANES = PACK ? 2 : 1, SPI = NG * LANES;
  const int K = sc.K, padc = K;
  const int stride = dround_up(job.npass * G * R, MSA_PROF_ALIGN);
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = sc.M[i];
  const int g = threadIdx.x / G, t = threadIdx.x % G;
  const int base_lane = (threadIdx.x & 31) - t;
  int2 *scr = job.scratch + ((size_t)blockIdx.x * NG + g) * 2 * job.scratch_cols;

  for (;;) {
    if (threadIdx.x == 0) {
      s_item = (long long)atomicAdd(job.counter, 1ull);
      s_qsum = 0ull;
    }
    __syncthreads();
    long long item = s_item;
    if (item >= job.n_items) break;
    item = job.n_items - 1 - item;  // longest queries first
    int lo = 0, hi = job.qe - job.qb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (job.prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int q = job.mode == 0 ? job.qb + lo : job.qlist[job.qb + lo];
    const int s0 = (job.mode == 0 ? q : job.sub_off) + (int)(item - job.prefix[lo]) * SPI;
    const int send = job.mode == 0 ? ss.n : job.sub_off + job.sub_n;
    const int Lq = ss.len[q];
    const uint8_t *rq = ss.res + ss.pstart[q];
    const int np = (Lq + G * R - 1) / (G * R);
    const int prow = np * G * R;
    for (int idx = threadIdx.x; idx < (K + 1) * prow; idx += NT) {
      const int r = idx / prow, i = idx - r * prow;
      int v = 0;  // padding: score -o
      if (r < K && i < Lq) v = sM[rq[i] * K + r] + sc.o;
      smem[r * stride + i] = (int8_t)v;
    }
    __syncthreads();

    const int sA = s0 + g * LANES, sB = sA + 1;
    const bool vA = sA < send, vB = PACK && sB < send;
    const int LA = vA ? ss.len[sA] : 0, LB = vB ? ss.len[sB] : 0;
    const uint8_t *rA = ss.res + (vA ? ss.pstart[sA] : 0);
    const uint8_t *rB = ss.res + (vB ? ss.pstart[sB] : 0);
    const int Lw = __reduce_max_sync(MSA_FULL_MASK, max(LA, LB));
    int best = 0;
    if (Lw > 0) {
      for (int p = 0; p < np; ++p) {
        const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
        int2 *sout = p + 1 < np ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
        const int b = wave_pass<G, R, PACK>(smem + p * G * R, stride, rA, LA, rB, LB, Lw, t,
                                            base_lane, padc, sc.o, sc.e, sin, sout);
        best = Cell<PACK>::vmax(best, b);
        __syncwarp();
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
      best = Cell<PACK>::vmax(best, __shfl_xor_sync(MSA_FULL_MASK, best, off));
    if (t == 0) {
      unsigned long long qadd = 0;
#pragma unroll
      for (int l = 0; l < LANES; ++l) {
        const int s = l ? sB : sA;
        if (!(l ? vB : vA)) continue;
        if (job.mode == 0 && s == q) continue;  // d(q, q) = 0
        const int S = l ? Cell<PACK>::lane1(best) : Cell<PACK>::lane0(best);
        if (PACK && S > job.sat_thresh) {
          const unsigned slot = atomicAdd(job.ovf_count, 1u);
          if (slot < (unsigned)job.ovf_cap) job.ovf[slot] = make_int2(q, s);
          else atomicOr(job.err, MSA_DERR_OVERFLOW);
          continue;
        }
        const unsigned long long sim = center_sim(S, job.self[q], job.self[s]);
        if (job.mode == 0) {
          atomicAdd(&job.pairsum[s], sim);
          qadd += sim;
        } else if (job.mode == 1) {
          atomicAdd(&job.pairsum[s], sim);
        } else {
          qadd += sim;
        }
      }
      if (qadd) atomicAdd(&s_qsum, qadd);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_qsum) atomicAdd(&job.pairsum[q], s_qsum);
  }
}

// ------------------------------------------------------------ paired queries
// The int16 lanes hold two queries (adjacent in length order) against ONE
// subject, so the profile can be stored pre-packed: prof[r*stride + i] =
// (s(qA_i, r) + o) | (s(qB_i, r) + o) << 16, and P = Hdiag + prof is a single
// add with no unpacking.  Lane t reads R words (R/4 16-byte loads) at word
// offset t*R; with R/4 odd the eight lanes of a load phase hit eight
// different 16-byte bank groups whatever residues they read.
// IN / OUT: the pass reads the row above from scr_in / writes its bottom row
// to scr_out (compile-time, so a single-pass query carries no test for them).
template <int G, int R, bool IN, bool OUT>
__device__ __forceinline__ int wave_pass_pp(const uint32_t *__restrict__ prof, int stride,
                                            const uint8_t *__restrict__ rs, int Ls, int Lw, int t,
                                            int base_lane, int padc, int o, int e, bool top,
                                            const int2 *__restrict__ scr_in,
                                            int2 *__restrict__ scr_out) {
  using C = Cell<true>;
  static_assert(R % 4 == 0 && (R / 4) % 2 == 1, "R/4 must be odd");
  const int negO = C::splat(-o), negE = C::splat(-e);
  const uint32_t pc = (uint32_t)padc;
  int H[R], E[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { H[r] = 0; E[r] = 0; }
  int hbot = 0, fbot = 0, htop_prev = 0, best = 0;
  uint32_t resv = pc;
  uint32_t cur = residue_at(rs, Ls, t, pc), nxt = residue_at(rs, Ls, G + t, pc);
  int2 sv0 = make_int2(0, 0), sv1 = make_int2(0, 0);
  if (IN) {
    if (0 < Lw) sv0 = scr_in[0];
    if (1 < Lw) sv1 = scr_in[1];
  }
  const uint32_t *pb = prof + t * R;
  const int steps = Lw + G - 1;
#pragma unroll 4
  for (int k = 0; k < steps; ++k) {
    const int kk = k & (G - 1);
    if (kk == 0 && k > 0) { cur = nxt; nxt = residue_at(rs, Ls, k + G + t, pc); }
    const uint32_t r0 = __shfl_sync(MSA_FULL_MASK, cur, base_lane + kk);
    uint32_t rin = __shfl_up_sync(MSA_FULL_MASK, resv, 1);
    int hin = __shfl_up_sync(MSA_FULL_MASK, hbot, 1);
    int fin = __shfl_up_sync(MSA_FULL_MASK, fbot, 1);
    const int2 sv = sv0;
    if (IN) {
      sv0 = sv1;
      if (k + 2 < Lw) sv1 = scr_in[k + 2];
    }
    if (t == 0) {
      rin = r0;
      const bool above = IN && k < Lw;
      hin = above ? sv.x : 0;
      fin = above ? sv.y : 0;
    }
    if (top) {  // the lane's first row starts a query (pair): the matrix top
      hin = 0;
      fin = 0;
    }
    resv = rin;
    const uint4 *pr = reinterpret_cast<const uint4 *>(pb + resv * stride);
    uint32_t w[R];
#pragma unroll
    for (int c = 0; c < R / 4; ++c) {
      const uint4 v = pr[c];
      w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
    }
    int hdiag = htop_prev;
    htop_prev = hin;
    int hup = hin;
    int f = fin;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int pdiag = hdiag + (int)w[r];       // both lanes stay in [0, 32767]
      f = C::addmax(f, negE, hup);
      const int m = C::vmax3(pdiag, E[r], f);
      const int hn = C::addmax_relu(m, negO, 0);
      E[r] = C::addmax(E[r], negE, hn);
      hdiag = H[r];
      H[r] = hn;
      hup = hn;
      if ((r & 1) == 1) best = C::vmax3(best, H[r - 1], hn);
    }
    hbot = H[R - 1];
    fbot = f;
    if (OUT && t == G - 1) {
      const int j = k - (G - 1);
      if (j >= 0 && j < Lw) scr_out[j] = make_int2(hbot, fbot);
    }
  }
  return best;
}

// Work item = (query pair p, block of NG consecutive subjects, one per group).
// three CTAs per SM for the 12-row variants (their registers fit 85 per
// thread without spilling); two otherwise
template <int G, int R>
__global__ void __launch_bounds__(kCenterThreads, R <= 12 ? 3 : 2)
k_center2(SeqSet ss, Scoring sc, CenterJob job) {
  extern __shared__ __align__(16) uint32_t smem32[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  __shared__ long long s_item;
  __shared__ int s_q[kMaxSeg][2], s_len[kMaxSeg][2], s_start[kMaxSeg + 1];
  __shared__ const uint8_t *s_res[kMaxSeg][2];
  __shared__ unsigned long long s_qsum[kMaxSeg][2];
  constexpr int NT = kCenterThreads, NG = NT / G;
  const int K = sc.K, padc = K, o = sc.o;
  const int stride = dround_up(job.npass * G * R, 32);
  // after the profile: the segment of every R-row block, then the best score
  // of every segment per group (two int16 lanes kept as two ints)
  int *s_blk = reinterpret_cast<int *>(smem32 + (K + 1) * stride);
  int *s_best = s_blk + ((stride / R + 1 + 3) & ~3);
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = sc.M[i];
  const int g = threadIdx.x / G, t = threadIdx.x % G;
  const int base_lane = (threadIdx.x & 31) - t;
  int2 *scr = job.scratch + ((size_t)blockIdx.x * NG + g) * 2 * job.scratch_cols;
  int *gbest = s_best + g * kMaxSeg * 2;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(job.counter, 1ull);
    __syncthreads();
    long long item = s_item;
    if (item >= job.n_items) break;
    item = job.n_items - 1 - item;  // longest queries first
    int lo = 0, hi = job.qe - job.qb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (job.prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int2 st = job.streams[job.qb + lo];  // pairs [st.x, st.x + st.y)
    const int m = st.y;
    if (m == 1) {
      // a single pair: its rows start at the first pass, so the lanes keep
      // their best in registers and no segment table is needed
      const int xa = 2 * st.x, xb = xa + 1;
      const int qA = job.mode == 0 ? xa : job.qlist[xa];
      const int qB = xb < job.nq ? (job.mode == 0 ? xb : job.qlist[xb]) : -1;
      const int LqA = ss.len[qA], LqB = qB >= 0 ? ss.len[qB] : 0;
      const uint8_t *ra = ss.res + ss.pstart[qA];
      const uint8_t *rb = ss.res + ss.pstart[qB >= 0 ? qB : qA];
      const int np = (max(LqA, LqB) + G * R - 1) / (G * R);
      const int prow = np * G * R;
      if (threadIdx.x < 2) s_qsum[0][threadIdx.x] = 0ull;
      for (int idx = threadIdx.x; idx < (K + 1) * prow; idx += NT) {
        const int r = idx / prow, i = idx - r * prow;
        uint32_t a = 0, b = 0;  // padding: score -o
        if (r < K) {
          if (i < LqA) a = (uint32_t)(sM[ra[i] * K + r] + o);
          if (i < LqB) b = (uint32_t)(sM[rb[i] * K + r] + o);
        }
        smem32[r * stride + i] = a | (b << 16);
      }
      __syncthreads();
      const int s0 = (job.mode == 0 ? xa : job.sub_off) + (int)(item - job.prefix[lo]) * NG;
      const int send = job.mode == 0 ? ss.n : job.sub_off + job.sub_n;
      const int s = s0 + g;
      const bool valid = s < send;
      const int Ls = valid ? ss.len[s] : 0;
      const uint8_t *rs = ss.res + (valid ? ss.pstart[s] : 0);
      const int Lw = __reduce_max_sync(MSA_FULL_MASK, Ls);
      int best = 0;
      if (Lw > 0) {
        for (int p = 0; p < np; ++p) {
          const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
          int2 *sout = p + 1 < np ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
          const uint32_t *pp = smem32 + p * G * R;
          int b;
          if (np == 1)
            b = wave_pass_pp<G, R, false, false>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, false, sin, sout);
          else if (p == 0)
            b = wave_pass_pp<G, R, false, true>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, false, sin, sout);
          else if (p + 1 == np)
            b = wave_pass_pp<G, R, true, false>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, false, sin, sout);
          else
            b = wave_pass_pp<G, R, true, true>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, false, sin, sout);
          best = Cell<true>::vmax(best, b);
          __syncwarp();
        }
      }
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1)
        best = Cell<true>::vmax(best, __shfl_xor_sync(MSA_FULL_MASK, best, off));
      if (t == 0 && valid) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int q = l ? qB : qA;
          if (q < 0) continue;
          // (s, q) with s < q is counted by the earlier query; d(q, q) = 0
          if (job.mode == 0 && s <= q) continue;
          const int S = l ? Cell<true>::lane1(best) : Cell<true>::lane0(best);
          if (S > job.sat_thresh) {
            const unsigned slot = atomicAdd(job.ovf_count, 1u);
            if (slot < (unsigned)job.ovf_cap) job.ovf[slot] = make_int2(q, s);
            else atomicOr(job.err, MSA_DERR_OVERFLOW);
            continue;
          }
          const unsigned long long sim = center_sim(S, job.self[q], job.self[s]);
          if (job.mode == 0) {
            atomicAdd(&job.pairsum[s], sim);
            atomicAdd(&s_qsum[0][l], sim);
          } else if (job.mode == 1) {
            atomicAdd(&job.pairsum[s], sim);
          } else {
            atomicAdd(&s_qsum[0][l], sim);
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && job.mode != 1) {
        if (s_qsum[0][0]) atomicAdd(&job.pairsum[qA], s_qsum[0][0]);
        if (qB >= 0 && s_qsum[0][1]) atomicAdd(&job.pairsum[qB], s_qsum[0][1]);
      }
      continue;
    }
    // segment k = pair st.x + k: queries of the two lanes, lengths, first row
    if (threadIdx.x < m) {
      const int k = threadIdx.x, xa = 2 * (st.x + k), xb = xa + 1;
      const int qa = job.mode == 0 ? xa : job.qlist[xa];
      const int qb = xb < job.nq ? (job.mode == 0 ? xb : job.qlist[xb]) : -1;
      s_q[k][0] = qa;
      s_q[k][1] = qb;
      s_len[k][0] = ss.len[qa];
      s_len[k][1] = qb >= 0 ? ss.len[qb] : 0;
      s_res[k][0] = ss.res + ss.pstart[qa];
      s_res[k][1] = ss.res + ss.pstart[qb >= 0 ? qb : qa];
      s_qsum[k][0] = s_qsum[k][1] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int r = 0;
      for (int k = 0; k < m; ++k) {
        s_start[k] = r;
        r += dround_up(max(s_len[k][0], s_len[k][1]), R);
      }
      s_start[m] = r;
    }
    __syncthreads();
    const int rows = s_start[m];
    const int np = (rows + G * R - 1) / (G * R);
    const int prow = np * G * R;
    for (int b = threadIdx.x; b < prow / R; b += NT) {
      int k = -1;
      if (b * R < rows)
        for (k = m - 1; s_start[k] > b * R; --k) {}
      s_blk[b] = k;
    }
    for (int i = threadIdx.x; i < NG * kMaxSeg * 2; i += NT) s_best[i] = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < (K + 1) * prow; idx += NT) {
      const int r = idx / prow, i = idx - r * prow;
      uint32_t a = 0, b = 0;  // padding: score -o
      const int k = s_blk[i / R];
      if (r < K && k >= 0) {
        const int li = i - s_start[k];
        if (li < s_len[k][0]) a = (uint32_t)(sM[s_res[k][0][li] * K + r] + o);
        if (li < s_len[k][1]) b = (uint32_t)(sM[s_res[k][1][li] * K + r] + o);
      }
      smem32[r * stride + i] = a | (b << 16);
    }
    __syncthreads();

    const int xf = 2 * st.x;  // mode 0: the stream's subjects start at its first query
    const int s0 = (job.mode == 0 ? xf : job.sub_off) + (int)(item - job.prefix[lo]) * NG;
    const int send = job.mode == 0 ? ss.n : job.sub_off + job.sub_n;
    const int s = s0 + g;
    const bool valid = s < send;
    const int Ls = valid ? ss.len[s] : 0;
    const uint8_t *rs = ss.res + (valid ? ss.pstart[s] : 0);
    const int Lw = __reduce_max_sync(MSA_FULL_MASK, Ls);
    if (Lw > 0) {
      for (int p = 0; p < np; ++p) {
        const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
        int2 *sout = p + 1 < np ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
        const uint32_t *pp = smem32 + p * G * R;
        const int blk = p * G + t, kseg = s_blk[blk];
        const bool top = kseg >= 0 && blk * R == s_start[kseg];
        int b;
        if (np == 1)
          b = wave_pass_pp<G, R, false, false>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, top, sin, sout);
        else if (p == 0)
          b = wave_pass_pp<G, R, false, true>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, top, sin, sout);
        else if (p + 1 == np)
          b = wave_pass_pp<G, R, true, false>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, top, sin, sout);
        else
          b = wave_pass_pp<G, R, true, true>(pp, stride, rs, Ls, Lw, t, base_lane, padc, o, sc.e, top, sin, sout);
        if (kseg >= 0) {
          atomicMax(&gbest[2 * kseg], Cell<true>::lane0(b));
          atomicMax(&gbest[2 * kseg + 1], Cell<true>::lane1(b));
        }
        __syncwarp();
      }
    }
    __syncwarp();
    // every query of the stream against this group's subject
    if (valid) {
      unsigned long long sub = 0ull;
      for (int k = t; k < m; k += G) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int q = s_q[k][l];
          if (q < 0) continue;
          // (s, q) with s < q is counted by the earlier query; d(q, q) = 0
          if (job.mode == 0 && s <= q) continue;
          const int S = gbest[2 * k + l];
          if (S > job.sat_thresh) {
            const unsigned slot = atomicAdd(job.ovf_count, 1u);
            if (slot < (unsigned)job.ovf_cap) job.ovf[slot] = make_int2(q, s);
            else atomicOr(job.err, MSA_DERR_OVERFLOW);
            continue;
          }
          const unsigned long long sim = center_sim(S, job.self[q], job.self[s]);
          if (job.mode == 0) {
            sub += sim;
            atomicAdd(&s_qsum[k][l], sim);
          } else if (job.mode == 1) {
            sub += sim;
          } else {
            atomicAdd(&s_qsum[k][l], sim);
          }
        }
      }
      if (sub) atomicAdd(&job.pairsum[s], sub);
    }
    __syncthreads();
    if (job.mode != 1 && threadIdx.x < 2 * m) {
      const int k = threadIdx.x >> 1, l = threadIdx.x & 1;
      if (s_q[k][l] >= 0 && s_qsum[k][l]) atomicAdd(&job.pairsum[s_q[k][l]], s_qsum[k][l]);
    }
  }
}

// ------------------------------------------------------------ pair list
// Each group takes one pair at a time; its own profile holds the current
// pass's G*R query rows.
template <int G>
__global__ void __launch_bounds__(256) k_pairs(SeqSet ss, Scoring sc, PairJob job) {
  constexpr int R = kPairsR, NT = 256, NG = NT / G, SR = G * R, GPW = 32 / G;
  extern __shared__ __align__(16) int8_t smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  const int K = sc.K, padc = K;
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = sc.M[i];
  __syncthreads();
  const int g = threadIdx.x / G, t = threadIdx.x % G, lane = threadIdx.x & 31;
  const int base_lane = lane - t;
  int8_t *prof = smem + (size_t)g * (K + 1) * SR;
  int2 *scr = job.scratch + ((size_t)blockIdx.x * NG + g) * 2 * job.scratch_cols;

  for (;;) {
    int base = 0;
    if (lane == 0) base = (int)atomicAdd(job.counter, (unsigned long long)GPW);
    base = __shfl_sync(MSA_FULL_MASK, base, 0);
    if (base >= job.npairs) break;
    const int pi = base + lane / G;
    const bool valid = pi < job.npairs;
    int a = 0, b = 0;
    if (valid) { const int2 pr = job.pairs[pi]; a = pr.x; b = pr.y; }
    const int La = valid ? ss.len[a] : 0, Lb = valid ? ss.len[b] : 0;
    const uint8_t *ra = ss.res + ss.pstart[a], *rb = ss.res + ss.pstart[b];
    const int Lw = __reduce_max_sync(MSA_FULL_MASK, Lb);
    const int np = __reduce_max_sync(MSA_FULL_MASK, (La + SR - 1) / SR);
    int best = 0;
    for (int p = 0; p < np; ++p) {
      __syncwarp();
      for (int idx = t; idx < (K + 1) * SR; idx += G) {
        const int r = idx / SR, i = idx - r * SR, qi = p * SR + i;
        int v = 0;  // padding: score -o
        if (r < K && qi < La) v = sM[ra[qi] * K + r] + sc.o;
        prof[idx] = (int8_t)v;
      }
      __syncwarp();
      if (Lw > 0) {
        const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
        int2 *sout = p + 1 < np ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
        best = max(best, wave_pass<G, R, false>(prof, SR, rb, Lb, nullptr, 0, Lw, t, base_lane,
                                                padc, sc.o, sc.e, sin, sout));
      }
      __syncwarp();
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
      best = max(best, __shfl_xor_sync(MSA_FULL_MASK, best, off));
    if (valid && t == 0) job.out[job.dst[pi]] = best;
  }
}

// ------------------------------------------------------------ codes
// One pass of G*16 center rows against one subject, int32 cells, writing
// the 4-bit traceback code of every cell: bits 0-1 the source of H (0 zero,
// 1 diagonal, 2 F, 3 E; ties in that order), bit 2 "E extended", bit 3 "F
// extended" (extension only when strictly better than opening).  Each lane
// also keeps, per row, the first column reaching the row's maximum.
//
// Same biased form as the score kernels (profile s + o, E* = E + o,
// F* = F + o).  Every comparison the codes need is the "a >= b" flag of a max
// (__vibmax_s32 returns max(a, b) and whether a >= b):
//   F* = vibmax(H_up, F*_up - e)   -> F extended   = !(H_up >= F*_up - e)
//   T  = vibmax(P, F*)             -> P >= F*
//   M  = vibmax(T, E*)             -> T >= E*   (source 1 / 2 / 3, in priority)
//   H  = vibmax(0, M - o)          -> H == 0    (source 0, the stop)
//   E*'= vibmax(H, E* - e)         -> E extended for the next column
//   best row value = vibmax(best, H) -> a strictly larger H moves the column
template <int G>
__device__ __forceinline__ void codes_pass(const int8_t *__restrict__ prof, int stride,
                                           const uint8_t *__restrict__ rs, int Ls, int Lw, int t,
                                           int base_lane, int blk, int nblk, int padc, int o, int e,
                                           const int2 *__restrict__ scr_in,
                                           int2 *__restrict__ scr_out, uint2 *__restrict__ cout,
                                           int &bv, int &bi, int &bj) {
  constexpr int R = kCodesR;
  int H[R], E[R], rb[R], rj[R];
  uint32_t emask = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) { H[r] = 0; E[r] = 0; rb[r] = 0; rj[r] = 0; }
  int hbot = 0, fbot = 0, htop_prev = 0;
  const uint32_t pc = (uint32_t)padc;
  uint32_t resv = pc;
  // the last four steps' code words (column k - t at slot k of the block row)
  uint2 q0 = make_uint2(0, 0), q1 = q0, q2 = q0, q3 = q0;
  const int slots = Ls + G - 1;
  uint32_t cur = residue_at(rs, Ls, t, pc), nxt = residue_at(rs, Ls, G + t, pc);
  const int8_t *pb = prof + t * R;
  const bool wr = blk < nblk;
  const int steps = Lw + G - 1;  // warp-uniform; columns past Ls are padding
  for (int k = 0; k < steps; ++k) {
    const int kk = k & (G - 1);
    if (kk == 0 && k > 0) { cur = nxt; nxt = residue_at(rs, Ls, k + G + t, pc); }
    // one lane per subject (G = 1) has no neighbour: it reads its own column
    // and the boundary row of its previous pass
    uint32_t r0 = cur, rin = 0;
    int hin = 0, fin = 0;
    if constexpr (G > 1) {
      r0 = __shfl_sync(MSA_FULL_MASK, cur, base_lane + kk);
      rin = __shfl_up_sync(MSA_FULL_MASK, resv, 1);
      hin = __shfl_up_sync(MSA_FULL_MASK, hbot, 1);
      fin = __shfl_up_sync(MSA_FULL_MASK, fbot, 1);
    }
    if (t == 0) {
      rin = r0;
      if (scr_in != nullptr && k < Ls) {
        const int2 v = scr_in[k];
        hin = v.x; fin = v.y;
      } else {
        hin = 0; fin = 0;
      }
    }
    resv = rin;
    ProfRow<R> pa;
    pa.load(pb + (int)resv * stride);
    const int j = k - t;
    int hdiag = htop_prev;
    htop_prev = hin;
    int hup = hin;
    int f = fin;
    uint32_t lo = 0, hi = 0;
    uint32_t enew = 0;
    Unroll<R>::run([&](auto ic) {
      constexpr int r = decltype(ic)::value;
      const int sp = Cell<false>::template score<r & 3>(pa.w[r >> 2], 0u);
      bool pf, p1, p2, pz, pe, pk;
      f = __vibmax_s32(hup, f - e, &pf);
      const int tv = __vibmax_s32(hdiag + sp, f, &p1);
      const int m = __vibmax_s32(tv, E[r], &p2);
      const int hv = __vibmax_s32(0, m - o, &pz);
      uint32_t src = p2 ? (p1 ? 1u : 2u) : 3u;
      src = pz ? 0u : src;
      const uint32_t code = src | (((emask >> r) & 1u) << 2) | ((pf ? 0u : 1u) << 3);
      if constexpr (r < 8) lo |= code << (4 * r);
      else hi |= code << (4 * (r - 8));
      E[r] = __vibmax_s32(hv, E[r] - e, &pe);
      enew |= (pe ? 0u : 1u) << r;
      rb[r] = __vibmax_s32(rb[r], hv, &pk);
      rj[r] = pk ? rj[r] : j;
      hdiag = H[r];
      H[r] = hv;
      hup = hv;
    });
    emask = enew;
    hbot = H[R - 1];
    fbot = f;
    q0 = q1; q1 = q2; q2 = q3; q3 = make_uint2(lo, hi);
    if ((k & 3) == 3 && wr && cout != nullptr && k - 3 < slots) store_chunk(cout + (k - 3), q0, q1, q2, q3);
    if (scr_out != nullptr && t == G - 1 && j >= 0 && j < Ls) scr_out[j] = make_int2(hbot, fbot);
  }
  flush_chunk(cout, wr, steps, slots, q0, q1, q2, q3);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (rb[r] > bv) { bv = rb[r]; bi = blk * R + r + 1; bj = rj[r] + 1; }
  }
}

// Groups of G lanes (G in {1, 2, 4, 8, 16, 32}; one lane per subject at G = 1), each
// aligning one subject at a time; the groups of a warp fetch their subjects
// together and run the warp's longest subject's number of columns.
template <int G>
__global__ void __launch_bounds__(256) k_codes(SeqSet ss, Scoring sc, CodesJob job) {
  constexpr int R = kCodesR, NT = 256, NG = NT / G, GPW = 32 / G;
  extern __shared__ __align__(16) int8_t smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  const int K = sc.K, padc = K;
  const int rows = job.npass * G * R;
  const int stride = dround_up(rows, MSA_PROF_ALIGN);
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = sc.M[i];
  __syncthreads();
  const int Lc = ss.len[job.center];
  const uint8_t *rc = ss.res + ss.pstart[job.center];
  for (int idx = threadIdx.x; idx < (K + 1) * rows; idx += NT) {
    const int r = idx / rows, i = idx - r * rows;
    int v = 0;  // padding: score -o
    if (r < K && i < Lc) v = sM[rc[i] * K + r] + sc.o;
    smem[r * stride + i] = (int8_t)v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, t = threadIdx.x % G, g = threadIdx.x / G;
  const int base_lane = lane - t;
  const int nblk = (Lc + R - 1) / R;
  int2 *scr = job.scratch + ((size_t)blockIdx.x * NG + g) * 2 * job.scratch_cols;
  const int nsub = job.se - job.sb;
  for (;;) {
    int x0 = 0;
    if (lane == 0) x0 = (int)atomicAdd(job.counter, (unsigned long long)GPW);
    x0 = __shfl_sync(MSA_FULL_MASK, x0, 0);
    if (x0 >= nsub) break;
    const int x = x0 + lane / G;
    const bool valid = x < nsub;
    const int k = job.se - 1 - (valid ? x : 0);  // longest first
    const int Ls = valid ? ss.len[k] : 0;
    const uint8_t *rs = ss.res + ss.pstart[k];
    uint2 *cbase = valid ? reinterpret_cast<uint2 *>(job.codes + job.code_off[k - job.sb]) : nullptr;
    const int Lw = __reduce_max_sync(MSA_FULL_MASK, Ls);
    int bv = 0, bi = 0, bj = 0;
    for (int p = 0; p < job.npass; ++p) {
      const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
      int2 *sout = p + 1 < job.npass ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
      const int blk = p * G + t;
      codes_pass<G>(smem + p * G * R, stride, rs, Ls, Lw, t, base_lane, blk, nblk, padc, sc.o, sc.e,
                    sin, sout, valid ? cbase + (size_t)blk * code_row_words(Ls, G) : nullptr, bv, bi, bj);
      __syncwarp();
    }
    // best cell over the group: largest H, then smallest row, then smallest column
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      const int ov = __shfl_xor_sync(MSA_FULL_MASK, bv, off);
      const int oi = __shfl_xor_sync(MSA_FULL_MASK, bi, off);
      const int oj = __shfl_xor_sync(MSA_FULL_MASK, bj, off);
      const bool take = ov > bv || (ov == bv && (oi < bi || (oi == bi && oj < bj)));
      if (take) { bv = ov; bi = oi; bj = oj; }
    }
    if (t == 0 && valid) job.best[k - job.sb] = best_key(bv, bi, bj);
  }
}

// NT threads per CTA, one CTA per SM: 256 (8 warps, ~210 registers) or 384
// (12 warps, registers capped near 160 without spills; faster on many short
// subjects, slower where few long ones leave the last warps' work unbalanced
// -- the alignment tuner times both).  Running several subject pairs back to
// back along one group's columns to share the wavefront ramp measured slower:
// the lanes leave a pair at different steps, so the per-pair bookkeeping runs
// once per lane.
template <int G, int NT>
__global__ void __launch_bounds__(NT, 1) k_codes2(SeqSet ss, Scoring sc, CodesJob job) {
  constexpr int R = kCodesR, NG = NT / G, GPW = 32 / G;
  extern __shared__ __align__(16) int8_t smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  const int K = sc.K, padc = K;
  const int rows = job.npass * G * R;
  const int stride = dround_up(rows, MSA_PROF_ALIGN);
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = sc.M[i];
  __syncthreads();
  const int Lc = ss.len[job.center];
  const uint8_t *rc = ss.res + ss.pstart[job.center];
  for (int idx = threadIdx.x; idx < (K + 1) * rows; idx += NT) {
    const int r = idx / rows, i = idx - r * rows;
    int v = 0;  // padding: score -o
    if (r < K && i < Lc) v = sM[rc[i] * K + r] + sc.o;
    smem[r * stride + i] = (int8_t)v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, t = threadIdx.x % G, g = threadIdx.x / G;
  const int base_lane = lane - t;
  const int nblk = (Lc + R - 1) / R;
  int2 *scr = job.scratch + ((size_t)blockIdx.x * NG + g) * 2 * job.scratch_cols;
  const int nsub = job.se - job.sb, nitem = (nsub + 1) / 2;
  for (;;) {
    int x0 = 0;
    if (lane == 0) x0 = (int)atomicAdd(job.counter, (unsigned long long)GPW);
    x0 = __shfl_sync(MSA_FULL_MASK, x0, 0);
    if (x0 >= nitem) break;
    const int x = x0 + lane / G;
    const bool valid = x < nitem;
    const int ka = job.se - 1 - 2 * (valid ? x : 0);  // longest first
    const int kb = ka - 1;
    const bool hasb = valid && kb >= job.sb;
    const int LA = valid ? ss.len[ka] : 0, LB = hasb ? ss.len[kb] : 0;
    const uint8_t *rA = ss.res + ss.pstart[ka];
    const uint8_t *rB = hasb ? ss.res + ss.pstart[kb] : rA;
    uint2 *cA = valid ? reinterpret_cast<uint2 *>(job.codes + job.code_off[ka - job.sb]) : nullptr;
    uint2 *cB = hasb ? reinterpret_cast<uint2 *>(job.codes + job.code_off[kb - job.sb]) : nullptr;
    const int Lw = __reduce_max_sync(MSA_FULL_MASK, max(LA, LB));
    int bv[2] = {0, 0}, bi[2] = {0, 0}, bj[2] = {0, 0};
    for (int p = 0; p < job.npass; ++p) {
      const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * job.scratch_cols : nullptr;
      int2 *sout = p + 1 < job.npass ? scr + (size_t)(p & 1) * job.scratch_cols : nullptr;
      const int blk = p * G + t;
      codes_pass2<G, kFull>(smem + p * G * R, smem + p * G * R, stride, rA, LA, rB, LB, Lw, t,
                            base_lane, blk, nblk, nblk, padc, sc.o, sc.e, sin, sout,
                            cA ? cA + (size_t)blk * code_row_words(LA, G) : nullptr,
                            cB ? cB + (size_t)blk * code_row_words(LB, G) : nullptr, HalfRows{}, bv,
                            bi, bj);
      __syncwarp();
    }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      int v = bv[s2], bi2 = bi[s2], bj2 = bj[s2];
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) {
        const int ov = __shfl_xor_sync(MSA_FULL_MASK, v, off);
        const int oi = __shfl_xor_sync(MSA_FULL_MASK, bi2, off);
        const int oj = __shfl_xor_sync(MSA_FULL_MASK, bj2, off);
        const bool take = ov > v || (ov == v && (oi < bi2 || (oi == bi2 && oj < bj2)));
        if (take) { v = ov; bi2 = oi; bj2 = oj; }
      }
      const int ks = s2 == 0 ? ka : kb;
      if (t == 0 && (s2 == 0 ? valid : hasb)) job.best[ks - job.sb] = best_key(v, bi2, bj2);
    }
  }
}

}  // namespace

// ------------------------------------------------------------ host side

// Kernel variants of center selection.  Paired-query variants (k_center2)
// carry two queries in the int16 lanes; single-query variants (k_center) carry
// two subjects (packed) or one (int32).  Every shape keeps the profile loads
// free of shared-memory bank conflicts.
const CenterVariant kCenterVariants[] = {
    {1, 8, 12, true},  {1, 8, 20, true},  {1, 8, 28, true},  {1, 16, 12, true},
    {1, 16, 20, true}, {1, 16, 28, true}, {1, 32, 12, true}, {1, 32, 20, true},
    {1, 32, 28, true}, {0, 32, 16, true}, {0, 32, 24, true}, {0, 8, 16, false},
    {0, 16, 16, false}, {0, 32, 16, false}};
const int kNumCenterVariants = sizeof(kCenterVariants) / sizeof(kCenterVariants[0]);

int center_profile_bytes(int variant, int K, int rows_alloc) {
  const CenterVariant &v = kCenterVariants[variant];
  if (v.paired) return (K + 1) * round_up_int(rows_alloc, 32) * 4;
  return (K + 1) * round_up_int(rows_alloc, MSA_PROF_ALIGN);
}

// paired: the profile, then the segment of every R-row block and the
// per-group best scores of every segment
int center_smem_bytes(int variant, int K, int rows_alloc) {
  const CenterVariant &v = kCenterVariants[variant];
  int b = center_profile_bytes(variant, K, rows_alloc);
  if (v.paired)
    b += round_up_int(round_up_int(rows_alloc, 32) / v.R + 1, 4) * 4 +
         (kCenterThreads / v.G) * kMaxSeg * 8;
  return b;
}

typedef void (*center_fn)(SeqSet, Scoring, CenterJob);

static center_fn center_kernel(int variant) {
  switch (variant) {
    case 0: return k_center2<8, 12>;
    case 1: return k_center2<8, 20>;
    case 2: return k_center2<8, 28>;
    case 3: return k_center2<16, 12>;
    case 4: return k_center2<16, 20>;
    case 5: return k_center2<16, 28>;
    case 6: return k_center2<32, 12>;
    case 7: return k_center2<32, 20>;
    case 8: return k_center2<32, 28>;
    case 9: return k_center<32, 16, true>;
    case 10: return k_center<32, 24, true>;
    case 11: return k_center<8, 16, false>;
    case 12: return k_center<16, 16, false>;
    case 13: return k_center<32, 16, false>;
    default: return nullptr;
  }
}

static int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

static int occupancy_grid(const void *fn, int threads, int smem) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sm_count();
}

int center_grid(int variant, int smem) {
  center_fn fn = center_kernel(variant);
  if (!fn) return 0;
  return occupancy_grid((const void *)fn, kCenterThreads, smem);
}

// (static shared memory counts against the 48 KB default too, so the limit
// is raised whatever the dynamic size)
cudaError_t center_allow_smem(int variant, int smem) {
  center_fn fn = center_kernel(variant);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_center(int variant, const SeqSet &ss, const Scoring &sc, const CenterJob &job,
                          int grid, cudaStream_t st, bool set_smem) {
  center_fn fn = center_kernel(variant);
  if (!fn) return cudaErrorInvalidValue;
  const CenterVariant &v = kCenterVariants[variant];
  const int smem = center_smem_bytes(variant, sc.K, job.npass * v.G * v.R);
  if (set_smem) {
    const cudaError_t e = center_allow_smem(variant, smem);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, kCenterThreads, smem, st>>>(ss, sc, job);
  return cudaGetLastError();
}

typedef void (*pairs_fn)(SeqSet, Scoring, PairJob);
static pairs_fn pairs_kernel(int G) {
  return G == 8 ? k_pairs<8> : (G == 32 ? k_pairs<32> : nullptr);
}
int pairs_rows(int G) { return G * kPairsR; }
static int pairs_smem(int G, int K) { return (256 / G) * (K + 1) * G * kPairsR; }

int pairs_grid(int G) {
  pairs_fn fn = pairs_kernel(G);
  if (!fn) return 0;
  return occupancy_grid((const void *)fn, 256, pairs_smem(G, MSA_MAX_ALPHABET));
}

cudaError_t launch_pairs(int G, const SeqSet &ss, const Scoring &sc, const PairJob &job,
                         int grid, cudaStream_t st) {
  pairs_fn fn = pairs_kernel(G);
  if (!fn) return cudaErrorInvalidValue;
  const int smem = pairs_smem(G, sc.K);
  if (smem > 40 * 1024)  // static shared memory counts too
    cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  fn<<<grid, 256, smem, st>>>(ss, sc, job);
  return cudaGetLastError();
}

int codes_smem_bytes(int K, int rows_alloc) {
  return (K + 1) * round_up_int(rows_alloc, MSA_PROF_ALIGN);
}

typedef void (*codes_fn)(SeqSet, Scoring, CodesJob);
static codes_fn codes_kernel(int G, bool packed, int threads) {
  if (packed && threads == kCodes2WideThreads) {
    switch (G) {
      case 8: return k_codes2<8, kCodes2WideThreads>;
      case 16: return k_codes2<16, kCodes2WideThreads>;
      case 32: return k_codes2<32, kCodes2WideThreads>;
      default: return nullptr;
    }
  }
  if (threads != kCodes2Threads) return nullptr;
  switch (G) {
    case 1: return packed ? k_codes2<1, kCodes2Threads> : k_codes<1>;
    case 2: return packed ? k_codes2<2, kCodes2Threads> : k_codes<2>;
    case 4: return packed ? k_codes2<4, kCodes2Threads> : k_codes<4>;
    case 8: return packed ? k_codes2<8, kCodes2Threads> : k_codes<8>;
    case 16: return packed ? k_codes2<16, kCodes2Threads> : k_codes<16>;
    case 32: return packed ? k_codes2<32, kCodes2Threads> : k_codes<32>;
    default: return nullptr;
  }
}

int codes_threads(bool packed, int threads) { return packed ? threads : 256; }

int codes_grid(int G, bool packed, int smem, int threads) {
  codes_fn fn = codes_kernel(G, packed, threads);
  return fn ? occupancy_grid((const void *)fn, codes_threads(packed, threads), smem) : 0;
}

// Group size for a center of length Lc.  A group of G lanes spends
// npass * (L + G - 1) steps on a subject of length L (npass = ceil(Lc / 16G)),
// and the groups share the resident warps, so the estimate is the larger of
// the total steps spread over the warps and the longest subject's own steps.
int codes_group(int Lc, bool packed, int K, int64_t n, double mean_len, int max_len) {
  int best_g = 32;
  double best = 0.0;
  for (int G : {32, 16, 8}) {
    const int npass = (Lc + G * kCodesR - 1) / (G * kCodesR);
    const int grid = codes_grid(G, packed, codes_smem_bytes(K, npass * G * kCodesR));
    const double warps = (double)grid * (codes_threads(packed) / 32);
    const double units = packed ? (double)((n + 1) / 2) : (double)n;
    const double tasks = std::ceil(units / (32 / G));
    const double mean_steps = npass * (mean_len + G - 1), max_steps = npass * (max_len + G - 1.0);
    // a step costs more the narrower the group (measured on one GB300: 1.5 kb
    // DNA against a 1.5 kb center at G = 8 / 16 / 32 took 1.17 / 1.04 / 1 x
    // the time for the same number of steps): 1 + 1.8 / G
    const double est = std::max(tasks * mean_steps / warps, max_steps) * (1.0 + 1.8 / G);
    if (G == 32 || est < best) { best = est; best_g = G; }
  }
  return best_g;
}

cudaError_t codes_allow_smem(int G, bool packed, int smem, int threads) {
  codes_fn fn = codes_kernel(G, packed, threads);
  if (!fn) return cudaErrorInvalidValue;
  if (smem <= 40 * 1024) return cudaSuccess;  // static shared memory counts too
  return cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_codes(int G, bool packed, const SeqSet &ss, const Scoring &sc, const CodesJob &job,
                         int grid, cudaStream_t st, bool set_smem, int threads) {
  codes_fn fn = codes_kernel(G, packed, threads);
  if (!fn) return cudaErrorInvalidValue;
  const int smem = codes_smem_bytes(sc.K, job.npass * G * kCodesR);
  if (set_smem) {
    const cudaError_t e = codes_allow_smem(G, packed, smem, threads);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, codes_threads(packed, threads), smem, st>>>(ss, sc, job);
  return cudaGetLastError();
}

// ===================================================================
// Allocation-free pair scores (msa_pair_scores_noalloc in include/msa.h).
//
// Some callers cannot allocate device memory: plug-ins hosted by an
// application whose allocator owns all of the GPU's memory, processes whose
// device memory is handed out by another framework's pool, or
// latency-critical services that forbid driver allocations after start-up.
// This entry point serves them: the caller passes every input and output
// buffer, and the only working memory is the fixed array below, which each
// GPU that loads the library holds until the process exits.  Every call on a
// device shares it, so calls that overlap on the GPU race; issue them one
// after another (for example on one stream).  Before it returns, the call
// copies the array's error word to the host and waits for its stream.
namespace {

constexpr size_t kNoallocControlBytes = 256;               // counter + error word
constexpr size_t kNoallocRowBytes = (size_t)32 << 20;      // boundary rows: 32 MiB
constexpr size_t kNoallocScratchBytes = kNoallocControlBytes + kNoallocRowBytes;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// error word bits
constexpr unsigned kNoallocBadIndex = 1u;    // a pair index or a length out of range
constexpr unsigned kNoallocBadResidue = 2u;  // a residue code >= alphabet

constexpr int kNoallocG = 32;  // one group per warp, 512 query rows per pass

struct NoallocArgs {
  int8_t M[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  int K, o, e, max_len;
  const uint8_t *res;        // alphabet indices, sequence i at offsets[i] .. offsets[i+1]
  const int64_t *offsets;    // n + 1 entries
  int64_t n;
  const int64_t *pairs;      // npairs x 2
  int64_t npairs;
  int32_t *out;
  unsigned char *scratch;    // device address of g_noalloc_scratch
  int scratch_cols;          // columns of each group's boundary rows (= max_len)
};

// The pair-list kernel with its inputs read straight from caller buffers and
// its counter, error word and boundary rows in the fixed array.
__global__ void __launch_bounds__(256) k_pairs_noalloc(NoallocArgs a) {
  constexpr int G = kNoallocG, R = kPairsR, NT = 256, NG = NT / G, SR = G * R;
  extern __shared__ __align__(16) int8_t smem[];
  __shared__ int8_t sM[MSA_MAX_ALPHABET * MSA_MAX_ALPHABET];
  const int K = a.K, padc = K;
  for (int i = threadIdx.x; i < K * K; i += NT) sM[i] = a.M[i];
  __syncthreads();
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(a.scratch);
  unsigned *err = reinterpret_cast<unsigned *>(a.scratch + 8);
  int2 *rows = reinterpret_cast<int2 *>(a.scratch + kNoallocControlBytes);
  const int g = threadIdx.x / G, t = threadIdx.x % G;
  int8_t *prof = smem + (size_t)g * (K + 1) * SR;
  int2 *scr = rows + ((size_t)blockIdx.x * NG + g) * 2 * a.scratch_cols;
  for (;;) {
    long long pi = 0;
    if (t == 0) pi = (long long)atomicAdd(counter, 1ull);
    pi = __shfl_sync(MSA_FULL_MASK, pi, 0);
    if (pi >= a.npairs) break;
    const int64_t ia = a.pairs[2 * pi], ib = a.pairs[2 * pi + 1];
    bool ok = ia >= 0 && ia < a.n && ib >= 0 && ib < a.n;
    int La = 0, Lb = 0;
    const uint8_t *ra = a.res, *rb = a.res;
    if (ok) {
      const int64_t la = a.offsets[ia + 1] - a.offsets[ia], lb = a.offsets[ib + 1] - a.offsets[ib];
      ok = la >= 1 && la <= a.max_len && lb >= 1 && lb <= a.max_len;
      if (ok) {
        La = (int)la; Lb = (int)lb;
        ra = a.res + a.offsets[ia];
        rb = a.res + a.offsets[ib];
      }
    }
    if (!ok) {  // the whole warp takes this branch together
      if (t == 0) { a.out[pi] = -1; atomicOr(err, kNoallocBadIndex); }
      continue;
    }
    // every residue code must index a profile row (0..K-1) before any is used
    bool bad = false;
    for (int i = t; i < La; i += G) bad |= ra[i] >= K;
    for (int i = t; i < Lb; i += G) bad |= rb[i] >= K;
    if (__any_sync(MSA_FULL_MASK, bad)) {
      if (t == 0) { a.out[pi] = -1; atomicOr(err, kNoallocBadResidue); }
      continue;
    }
    const int np = (La + SR - 1) / SR;
    int best = 0;
    for (int p = 0; p < np; ++p) {
      __syncwarp();
      for (int idx = t; idx < (K + 1) * SR; idx += G) {
        const int r = idx / SR, i = idx - r * SR, qi = p * SR + i;
        int v = 0;
        if (r < K && qi < La) v = sM[ra[qi] * K + r] + a.o;
        prof[idx] = (int8_t)v;
      }
      __syncwarp();
      const int2 *sin = p > 0 ? scr + (size_t)((p - 1) & 1) * a.scratch_cols : nullptr;
      int2 *sout = p + 1 < np ? scr + (size_t)(p & 1) * a.scratch_cols : nullptr;
      best = max(best, wave_pass<G, R, false>(prof, SR, rb, Lb, nullptr, 0, Lb, t, 0, padc, a.o,
                                              a.e, sin, sout));
      __syncwarp();
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
      best = max(best, __shfl_xor_sync(MSA_FULL_MASK, best, off));
    if (t == 0) a.out[pi] = best;
  }
}

// Device address of g_noalloc_scratch per device, looked up once (with that
// device current) by the first call made on it.
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[64] = {};

}  // namespace

extern "C" int msa_pair_scores_noalloc(const uint8_t *residues, const int64_t *offsets, int64_t n,
                                       const int64_t *pairs, int64_t npairs, int32_t max_len,
                                       const int8_t *matrix, int32_t alphabet, int32_t gap_open,
                                       int32_t gap_extend, int32_t *scores_out,
                                       void *cuda_stream) {
  if (npairs == 0) return MSA_OK;
  if (!residues || !offsets || !pairs || !scores_out || !matrix || n < 1 || npairs < 0)
    return MSA_EINVAL;
  if (alphabet < 1 || alphabet > MSA_MAX_ALPHABET) return MSA_EINVAL;
  if (gap_extend < 1 || gap_open < gap_extend) return MSA_EINVAL;
  if (max_len < 1 || max_len > MSA_MAX_LEN) return MSA_ERANGE;
  NoallocArgs a;
  memset(&a, 0, sizeof a);
  for (int i = 0; i < alphabet * alphabet; ++i) {
    const int v = matrix[i] + gap_open;
    if (v > 127 || v < -128) return MSA_EINVAL;
    a.M[i] = matrix[i];
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MSA_ECUDA;
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return MSA_ECUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  constexpr int NG = 256 / kNoallocG;
  const int np_max = (max_len + kNoallocG * kPairsR - 1) / (kNoallocG * kPairsR);
  const size_t per_cta = np_max > 1 ? (size_t)NG * 2 * max_len * sizeof(int2) : 0;
  const int smem = NG * (alphabet + 1) * kNoallocG * kPairsR;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute((const void *)k_pairs_noalloc,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return MSA_ECUDA;
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_noalloc, 256, smem);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (long long)std::max(per_sm, 1) * std::max(sms, 1);
  if (per_cta > 0) grid = std::min<long long>(grid, (long long)(kNoallocRowBytes / per_cta));
  if (grid < 1) return MSA_ERANGE;
  a.K = alphabet; a.o = gap_open; a.e = gap_extend; a.max_len = max_len;
  a.res = residues; a.offsets = offsets; a.n = n; a.pairs = pairs; a.npairs = npairs;
  a.out = scores_out;
  a.scratch = static_cast<unsigned char *>(base);
  a.scratch_cols = max_len;
  // the work counter and the error word must start at zero on every call
  if (cudaMemsetAsync(base, 0, kNoallocControlBytes, st) != cudaSuccess) return MSA_ECUDA;
  k_pairs_noalloc<<<(unsigned)grid, 256, smem, st>>>(a);
  if (cudaGetLastError() != cudaSuccess) return MSA_ECUDA;
  unsigned herr = 0;
  if (cudaMemcpyAsync(&herr, static_cast<unsigned char *>(base) + 8, sizeof herr,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MSA_ECUDA;
  if (herr & kNoallocBadResidue) return MSA_EINVAL;
  return herr ? MSA_ERANGE : MSA_OK;
}
