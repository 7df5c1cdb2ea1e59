// msa_api.cu -- the C ABI (include/msa.h) and its host-side planner:
// length sorting, work-item classes for the center kernels, batching of the
// traceback codes, and the stage timers.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "msa.h"
#include "msa_kernels.cuh"
#include "sw_kernels.cuh"

#include "ctx.cuh"

namespace msa_detail {

int fail(msa_ctx *c, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int ensure(msa_ctx *ctx, DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return MSA_OK;
  if (b.p) {
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaFree(b.p));
    ctx->dev_bytes -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  bytes = (bytes + 255) / 256 * 256;
  if (ctx->dev_limit && ctx->dev_bytes + bytes > ctx->dev_limit)
    return fail(ctx, MSA_ENOMEM, "device memory limit: %zu bytes held, %zu more wanted, limit %zu",
                ctx->dev_bytes, bytes, ctx->dev_limit);
  CK(cudaMalloc(&b.p, bytes));
  b.cap = bytes;
  ctx->dev_bytes += bytes;
  ctx->dev_peak = std::max(ctx->dev_peak, ctx->dev_bytes);
  return MSA_OK;
}

void release(msa_ctx *ctx, DevBuf &b) {
  if (!b.p) return;
  cudaFree(b.p);
  ctx->dev_bytes -= b.cap;
  b.p = nullptr;
  b.cap = 0;
}


bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int set_device(msa_ctx *ctx) {
  CK(cudaSetDevice(ctx->dev));
  return MSA_OK;
}

void stage_begin(msa_ctx *ctx, int s) { cudaEventRecord(ctx->ev[2 * s], ctx->st); }
void stage_end(msa_ctx *ctx, int s) { cudaEventRecord(ctx->ev[2 * s + 1], ctx->st); }
void stage_collect(msa_ctx *ctx, int s) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, ctx->ev[2 * s], ctx->ev[2 * s + 1]) == cudaSuccess)
    ctx->stage_ms[s] = ms;
  else
    cudaGetLastError();
}

int check_derr(msa_ctx *ctx) {
  unsigned h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, ctx->derr, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (h[0] & MSA_DERR_LETTER) return fail(ctx, MSA_EINVAL, "letter outside the alphabet");
  if (h[0] & MSA_DERR_TRACE) return fail(ctx, MSA_ECUDA, "inconsistent traceback codes");
  if (h[0] & MSA_DERR_OVERFLOW) return fail(ctx, MSA_ENOMEM, "int16 overflow list full");
  if (h[0] & MSA_DERR_TIMEOUT_TC) return fail(ctx, MSA_ETIMEOUT, "tensor-core convolution timed out");
  if (h[0] & MSA_DERR_RANGE) return fail(ctx, MSA_ERANGE, "a tree distance beyond 2^30");
  return MSA_OK;
}

SeqSet seqset(msa_ctx *ctx) {
  return SeqSet{P<uint8_t>(ctx->res), P<int64_t>(ctx->d_pstart), P<int32_t>(ctx->d_len), ctx->n};
}
Scoring scoring(msa_ctx *ctx) { return Scoring{ctx->dM, ctx->K, ctx->o, ctx->e}; }

// ------------------------------------------------------------ pair scores
// Scores of (a, b) pairs given in sorted indices, int32 cells.  dst[x] is the
// output slot of pair x.  Pairs are grouped by the query's pass height and
// ordered by subject length so the groups of a warp stay in step.
int run_pairs(msa_ctx *ctx, const std::vector<int2> &pairs_in, const std::vector<int32_t> &dst_in,
              int32_t *d_out) {
  const int np = (int)pairs_in.size();
  if (np == 0) return MSA_OK;
  std::vector<int32_t> order(np);
  std::iota(order.begin(), order.end(), 0);
  const int short_rows = pairs_rows(8);
  auto before = [&](int x, int y) {
    const int ax = ctx->len_sorted[pairs_in[x].x] > short_rows;
    const int ay = ctx->len_sorted[pairs_in[y].x] > short_rows;
    if (ax != ay) return ax < ay;
    const int lx = ctx->len_sorted[pairs_in[x].y], ly = ctx->len_sorted[pairs_in[y].y];
    return lx < ly;
  };
  // (self pairs of the sorted set arrive in order already)
  if (!std::is_sorted(order.begin(), order.end(), before))
    std::stable_sort(order.begin(), order.end(), before);
  std::vector<int2> pr(np);
  std::vector<int32_t> dst(np);
  int n_short = 0;
  for (int x = 0; x < np; ++x) {
    pr[x] = pairs_in[order[x]];
    dst[x] = dst_in[order[x]];
    if (ctx->len_sorted[pr[x].x] <= short_rows) ++n_short;
  }
  TRY(ensure(ctx, ctx->pairs, sizeof(int2) * np));
  TRY(ensure(ctx, ctx->pair_dst, sizeof(int32_t) * np));
  CK(cudaMemcpyAsync(ctx->pairs.p, pr.data(), sizeof(int2) * np, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->pair_dst.p, dst.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice,
                     ctx->st));
  const SeqSet ss = seqset(ctx);
  const Scoring sc = scoring(ctx);
  for (int part = 0; part < 2; ++part) {
    const int G = part == 0 ? 8 : 32;
    const int b = part == 0 ? 0 : n_short, e = part == 0 ? n_short : np;
    if (e <= b) continue;
    const int grid = pairs_grid(G);
    const size_t scr = (size_t)grid * (256 / G) * 2 * ctx->maxlen * sizeof(int2);
    TRY(ensure(ctx, ctx->scratch, scr));
    CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
    PairJob job;
    job.pairs = P<int2>(ctx->pairs) + b;
    job.dst = P<int32_t>(ctx->pair_dst) + b;
    job.out = d_out;
    job.npairs = e - b;
    job.counter = ctx->dcounter;
    job.scratch = P<int2>(ctx->scratch);
    job.scratch_cols = ctx->maxlen;
    CK((++ctx->launches, launch_pairs)(G, ss, sc, job, grid, ctx->st));
  }
  return MSA_OK;
}

// ------------------------------------------------------------ center planning
// Largest pre-packed profile (bytes) a paired-query launch may hold in shared
// memory; longer queries use the single-query kernel with an int8 profile.
constexpr int kMaxPairedProfile = 110 * 1024;

// Modelled cost of one query against subjects of length ~Ls_est with a
// variant: rows x (columns + ramp), a charge per extra pass (scratch traffic,
// a second sweep of the subject), the per-column overhead of small R, and the
// byte unpacking of the single-query packed kernel.
double variant_cost(int v, int Lq, int Ls_est) {
  const CenterVariant &cv = kCenterVariants[v];
  const int rows = cv.G * cv.R;
  const int np = (Lq + rows - 1) / rows;
  double c = (double)np * rows * (Ls_est + cv.G - 1 + (np > 1 ? 48 : 0)) * (1.0 + 3.0 / cv.R);
  if (!cv.paired && cv.packed) c *= 1.2;
  return c;
}

bool variant_fits(msa_ctx *ctx, int v, int Lq) {
  const CenterVariant &cv = kCenterVariants[v];
  const int rows = cv.G * cv.R;
  const int np = (Lq + rows - 1) / rows;
  const int smem = center_smem_bytes(v, ctx->K, np * rows);
  return !(cv.paired && center_profile_bytes(v, ctx->K, np * rows) > kMaxPairedProfile) &&
         smem <= 200 * 1024;
}

int choose_variant(msa_ctx *ctx, int Lq, int Ls_est, bool packed) {
  // msa_autotune's correction of the model for this length bucket, if any
  const std::vector<double> *corr = nullptr;
  if (packed && !ctx->tune_corr.empty())
    for (size_t b = 0; b + 1 < ctx->tune_edges.size(); ++b)
      if (Lq >= ctx->tune_edges[b] && Lq < ctx->tune_edges[b + 1]) corr = &ctx->tune_corr[b];
  int best = -1;
  double best_cost = 1e300;
  for (int v = 0; v < kNumCenterVariants; ++v) {
    const CenterVariant &cv = kCenterVariants[v];
    if (cv.packed != packed) continue;
    const int rows = cv.G * cv.R;
    const int np = (Lq + rows - 1) / rows;
    const int smem = center_smem_bytes(v, ctx->K, np * rows);
    if (cv.paired && center_profile_bytes(v, ctx->K, np * rows) > kMaxPairedProfile) continue;
    if (smem > 200 * 1024) continue;
    double c = variant_cost(v, Lq, Ls_est);
    if (corr && (*corr)[v] > 0) c /= (*corr)[v];
    if (c < best_cost) { best_cost = c; best = v; }
  }
  return best;
}

// int16 lanes need every biased score s + o >= 0 (the lane-local add) and,
// under MSA_AUTO, an a-priori bound on any local score of a sequence of
// length Lq that stays below the overflow guard.
int sat_thresh(msa_ctx *ctx) { return ctx->sat_limit - ctx->smax - ctx->o; }

// int16 lanes hold every value of the alignment to a center of length Lc:
// H <= Lc * smax, and the biased P = H + s + o never passes Lc * smax + smax + o.
static bool codes_packed(msa_ctx *ctx, int Lc) {
  if (ctx->precision == MSA_INT32 || ctx->align_int32 || ctx->smin + ctx->o < 0) return false;
  const long long top = (long long)Lc * std::max(ctx->smax, 0) + std::max(ctx->smax, 0) + ctx->o;
  return top <= std::min(ctx->sat_limit, 32767);
}

// group size of the alignment kernel for this set and a center of length Lc
static int align_group(msa_ctx *ctx, int Lc, bool packed) {
  if (ctx->align_group > 0) return ctx->align_group;
  double total = 0.0;
  for (int L : ctx->len_sorted) total += L;
  return codes_group(Lc, packed, ctx->K, ctx->n, ctx->n ? total / ctx->n : 0.0, ctx->maxlen);
}

bool align_packed(msa_ctx *ctx, int Lc) { return codes_packed(ctx, Lc); }
int align_cta(msa_ctx *ctx, int G, bool packed) {
  return packed && G >= 8 && ctx->align_threads == kCodes2WideThreads ? kCodes2WideThreads
                                                                      : kCodes2Threads;
}
int align_lanes(msa_ctx *ctx, int Lc, bool packed) { return align_group(ctx, Lc, packed); }

bool use_packed(msa_ctx *ctx, int Lq) {
  if (ctx->precision == MSA_INT32 || ctx->smin + ctx->o < 0) return false;
  if (ctx->precision == MSA_INT16) return true;
  const long long bound = (long long)Lq * std::max(ctx->smax, 0);
  return bound <= (long long)sat_thresh(ctx);
}

struct CenterClass {
  int variant, ub, ue;  // item units [ub, ue): query pairs (paired) or queries
};

// A class launch planned on the host: its slice of the item prefix, its
// pass count, shared memory and grid.
struct ClassPlan {
  CenterClass cc;
  int nq_list, npass, smem, grid;
  size_t prefix_off;  // into the concatenated prefix of all planned classes
  int64_t n_items;
};

// rows of query pair p in a stream of R-row blocks: the longer of its two
// queries, rounded up to R
static int pair_rows(const std::vector<int> &qlen, int nq_list, int p, int R) {
  const int xa = 2 * p, xb = std::min(2 * p + 1, nq_list - 1);
  return round_up_int(std::max(qlen[xa], qlen[xb]), R);
}

ClassPlan plan_class(msa_ctx *ctx, int mode, int nq_list, const CenterClass &cc,
                     const std::vector<int> &qlen, int sub_n, std::vector<int64_t> &prefix_all,
                     const std::vector<int2> &streams) {
  const CenterVariant &cv = kCenterVariants[cc.variant];
  const int NG = kCenterThreads / cv.G;
  const int n = mode == 0 ? ctx->n : sub_n;
  ClassPlan pl;
  pl.cc = cc;
  pl.nq_list = nq_list;
  pl.prefix_off = prefix_all.size();
  prefix_all.push_back(0);
  int maxrows = 0;
  for (int u = cc.ub; u < cc.ue; ++u) {
    int64_t items;
    if (cv.paired) {
      // unit = stream u of consecutive pairs, subjects from its first query on
      const int2 st = streams[u];
      int rows = 0;
      for (int q = st.x; q < st.x + st.y; ++q) rows += pair_rows(qlen, nq_list, q, cv.R);
      maxrows = std::max(maxrows, rows);
      const int xa = 2 * st.x;
      items = mode == 0 ? (n - xa + NG - 1) / NG : (n + NG - 1) / NG;
    } else {
      const int spi = NG * (cv.packed ? 2 : 1);
      maxrows = std::max(maxrows, qlen[u]);
      items = mode == 0 ? (n - u + spi - 1) / spi : (n + spi - 1) / spi;
    }
    prefix_all.push_back(prefix_all.back() + items);
  }
  pl.n_items = prefix_all.back();
  const int rows = cv.G * cv.R;
  pl.npass = (maxrows + rows - 1) / rows;
  pl.smem = center_smem_bytes(cc.variant, ctx->K, pl.npass * rows);
  pl.grid = center_grid(cc.variant, pl.smem);
  return pl;
}

CenterJob class_job(msa_ctx *ctx, int mode, const ClassPlan &pl, int sub_off, int sub_n,
                    unsigned long long *counter, const int32_t *self) {
  CenterJob job;
  job.mode = mode;
  job.qlist = P<int32_t>(ctx->qlist);
  job.nq = pl.nq_list;
  job.sub_off = sub_off;
  job.sub_n = sub_n;
  job.qb = pl.cc.ub;
  job.qe = pl.cc.ue;
  job.prefix = P<int64_t>(ctx->prefix) + pl.prefix_off;
  job.n_items = pl.n_items;
  job.npass = pl.npass;
  job.counter = counter;
  job.pairsum = P<unsigned long long>(ctx->pairsum);
  job.self = self;
  job.sat_thresh = sat_thresh(ctx);
  job.ovf = P<int2>(ctx->ovf);
  job.ovf_count = ctx->derr + 1;
  job.ovf_cap = (int)(ctx->ovf.cap / sizeof(int2));
  job.err = ctx->derr;
  job.scratch = P<int2>(ctx->scratch);
  job.scratch_cols = ctx->maxlen;
  job.streams = P<int2>(ctx->streams);
  return job;
}

// Upload the plans' prefixes and size the scratch rows of multi-pass
// classes (all classes run in stream order, so they share one scratch).
int stage_plans(msa_ctx *ctx, const std::vector<ClassPlan> &plans,
                const std::vector<int64_t> &prefix_all, const std::vector<int2> &streams) {
  TRY(ensure(ctx, ctx->streams, sizeof(int2) * std::max<size_t>(streams.size(), 1)));
  if (!streams.empty())
    CK(cudaMemcpyAsync(ctx->streams.p, streams.data(), sizeof(int2) * streams.size(),
                       cudaMemcpyHostToDevice, ctx->st));
  size_t scratch = 0;
  for (const ClassPlan &pl : plans)
    if (pl.npass > 1)
      scratch = std::max(scratch, (size_t)pl.grid * (kCenterThreads / kCenterVariants[pl.cc.variant].G) *
                                      2 * ctx->maxlen * sizeof(int2));
  // the graph runs its classes on two streams: one boundary-row area each
  if (scratch) TRY(ensure(ctx, ctx->scratch, 2 * scratch));
  ctx->scratch_half = scratch / sizeof(int2);
  TRY(ensure(ctx, ctx->prefix, sizeof(int64_t) * prefix_all.size()));
  TRY(ensure(ctx, ctx->counters, sizeof(unsigned long long) * std::max<size_t>(plans.size(), 1)));
  CK(cudaMemcpyAsync(ctx->prefix.p, prefix_all.data(), sizeof(int64_t) * prefix_all.size(),
                     cudaMemcpyHostToDevice, ctx->st));
  return MSA_OK;
}

// One class, timed on its own (the autotuner's measurement).
int launch_class(msa_ctx *ctx, int mode, int nq_list, const CenterClass &cc,
                 const std::vector<int> &qlen, float &center_ms, int sub_off = 0, int sub_n = -1) {
  if (sub_n < 0) sub_n = ctx->n;
  std::vector<int64_t> prefix_all;
  std::vector<int2> streams;  // paired: one pair per stream
  if (kCenterVariants[cc.variant].paired)
    for (int u = 0; u < cc.ue; ++u) streams.push_back(make_int2(u, 1));
  const ClassPlan pl = plan_class(ctx, mode, nq_list, cc, qlen, sub_n, prefix_all, streams);
  TRY(stage_plans(ctx, {pl}, prefix_all, streams));
  CK(cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long), ctx->st));
  // (the autotuner's sums are never read, so the self scores need not be current)
  const CenterJob job = class_job(ctx, mode, pl, sub_off, sub_n, P<unsigned long long>(ctx->counters),
                                  P<int32_t>(ctx->self));
  stage_begin(ctx, ST_CENTER_K);
  ++ctx->launches;
  CK(launch_center(cc.variant, seqset(ctx), scoring(ctx), job, pl.grid, ctx->st, true));
  stage_end(ctx, ST_CENTER_K);
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_CENTER_K);
  center_ms += ctx->stage_ms[ST_CENTER_K];
  return MSA_OK;
}

// All classes of a center selection as one CUDA graph: the per-class
// counters are cleared by the graph's first node and the class kernels
// follow one another in stream order, so the whole length-bucketed set is a
// single submission with no host round trip between buckets.  The graph is
// captured on the context's private capture stream and launched on its
// stream (which may be the legacy default stream).
int launch_plans(msa_ctx *ctx, int mode, const std::vector<ClassPlan> &plans, int sub_off,
                 int sub_n, const SeqSet &ss, const int32_t *self) {
  const Scoring sc = scoring(ctx);
  std::vector<int> top(kNumCenterVariants, 0);
  for (const ClassPlan &pl : plans) top[pl.cc.variant] = std::max(top[pl.cc.variant], pl.smem);
  for (int v = 0; v < kNumCenterVariants; ++v)
    if (top[v] > 0) CK(center_allow_smem(v, top[v]));
  unsigned long long *cnt = P<unsigned long long>(ctx->counters);
  // Everything the graph bakes in; a selection with the same key (the same
  // set and buffers, e.g. a repeated step) relaunches the cached graph.
  // The classes run longest queries first, alternating between two streams
  // (a fork and a join in the graph), so a class's tail of long items
  // overlaps the next class instead of idling the GPU; each stream has its
  // own boundary-row area.
  std::vector<CenterJob> jobs;
  std::vector<int64_t> key = {mode, sub_off, sub_n, (int64_t)ss.res, (int64_t)ss.pstart,
                              (int64_t)ss.len, ss.n, (int64_t)sc.M, sc.K, sc.o, sc.e,
                              (int64_t)cnt, (int64_t)plans.size()};
  for (size_t c = 0; c < plans.size(); ++c) {
    CenterJob job = class_job(ctx, mode, plans[c], sub_off, sub_n, cnt + c, self);
    const size_t order = plans.size() - 1 - c;  // launch position
    if (order & 1) job.scratch += ctx->scratch_half;
    jobs.push_back(job);
    const int64_t f[] = {plans[c].cc.variant, plans[c].grid, plans[c].smem, job.mode,
                         (int64_t)job.qlist, job.nq, job.qb, job.qe, job.sub_off, job.sub_n,
                         (int64_t)job.prefix, job.n_items, job.npass, (int64_t)job.counter,
                         (int64_t)job.pairsum, (int64_t)job.self, job.sat_thresh,
                         (int64_t)job.ovf, (int64_t)job.ovf_count, job.ovf_cap, (int64_t)job.err,
                         (int64_t)job.scratch, job.scratch_cols, (int64_t)job.streams};
    key.insert(key.end(), f, f + sizeof(f) / sizeof(f[0]));
  }
  if (!ctx->center_exec || key != ctx->center_key) {
    if (ctx->center_exec) {
      CK(cudaStreamSynchronize(ctx->st));
      cudaGraphExecDestroy(ctx->center_exec);
      ctx->center_exec = nullptr;
      ctx->center_key.clear();
    }
    CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * plans.size(), ctx->cap_st);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->cap_fork, ctx->cap_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap_st2, ctx->cap_fork, 0);
    int failed = -1;
    for (size_t k = 0; k < plans.size() && e == cudaSuccess; ++k) {
      const size_t c = plans.size() - 1 - k;
      e = launch_center(plans[c].cc.variant, ss, sc, jobs[c], plans[c].grid,
                        (k & 1) ? ctx->cap_st2 : ctx->cap_st, false);
      if (e != cudaSuccess) failed = (int)c;
    }
    {
      const cudaError_t e2 = cudaEventRecord(ctx->cap_join, ctx->cap_st2);
      const cudaError_t e3 = cudaStreamWaitEvent(ctx->cap_st, ctx->cap_join, 0);
      if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(ctx->cap_st, &graph);
    if (failed >= 0) {
      if (graph) cudaGraphDestroy(graph);
      const ClassPlan &pl = plans[failed];
      return fail(ctx, MSA_ECUDA, "center kernel variant %d (grid %d, %d B shared, %d passes): %s",
                  pl.cc.variant, pl.grid, pl.smem, pl.npass, cudaGetErrorString(e));
    }
    if (e == cudaSuccess) e = e_end;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    CK(e);
    ctx->center_exec = exec;
    ctx->center_key = key;
  }
  ctx->launches += (int64_t)plans.size();
  stage_begin(ctx, ST_CENTER_K);
  CK(cudaGraphLaunch(ctx->center_exec, ctx->st));
  stage_end(ctx, ST_CENTER_K);
  return MSA_OK;
}

int run_center(msa_ctx *ctx, int mode, const std::vector<int32_t> &qsorted, const SetView *view,
               int q_begin, int q_end) {
  // qsorted: ascending sorted indices of the queries (modes 1, 2); mode 0 uses all.
  // With a view, indices are the view's and its first n_sub entries are the subjects.
  // The self scores (ctx->self, or the view's) must be current: the kernels
  // add center_sim of every pair, which needs both sequences' self scores.
  if (view && mode == 0) return fail(ctx, MSA_EINVAL, "all-pairs selection over a view");
  const std::vector<int32_t> &lens = view ? view->len : ctx->len_sorted;
  const int n = view ? view->n_sub : ctx->n;
  if (n < 1) return fail(ctx, MSA_EINVAL, "no subjects");
  const SeqSet ss = view ? view->ss : seqset(ctx);
  std::vector<int> qlen;
  if (mode == 0) qlen.assign(lens.begin(), lens.end());
  else for (int q : qsorted) qlen.push_back(lens[q]);
  const int nq = (int)qlen.size();
  double mean = 0;
  for (int k = 0; k < n; ++k) mean += lens[k];
  mean /= n;
  std::vector<int64_t> suffix(n + 1, 0);
  for (int k = n - 1; k >= 0; --k) suffix[k] = suffix[k + 1] + lens[k];
  if (mode != 0) {
    TRY(ensure(ctx, ctx->qlist, sizeof(int32_t) * qsorted.size()));
    CK(cudaMemcpyAsync(ctx->qlist.p, qsorted.data(), sizeof(int32_t) * qsorted.size(),
                       cudaMemcpyHostToDevice, ctx->st));
  }
  // Queries ascend in length: a packed prefix [0, x1), an int32 rest.  The
  // local score of any pair is at most min(Lq, Ls) * smax <= Lq * smax.
  int x1 = 0;
  while (x1 < nq && use_packed(ctx, qlen[x1])) ++x1;
  // partner length: all-pairs queries meet the (longer) sequences after them
  auto est_at = [&](int x) {
    return mode == 0 ? (int)(suffix[x] / std::max(1, n - x)) : (int)mean;
  };

  std::vector<CenterClass> classes;
  std::vector<int2> streams;
  // Packed part: query pairs [0, ceil(x1/2)).  Consecutive pairs are stacked
  // into streams (each pair's rows rounded up to R, not to a whole pass) when
  // that lowers the modelled cost per real cell; mode 0 streams see the
  // subjects from their first query on.
  const int npairs = (x1 + 1) / 2;
  // mode 0 may run a share of the queries only, [q_begin, q_end) with even
  // bounds (a shard of the all-pairs triangle); packed pairs [p_begin, p_end)
  if (q_end < 0 || q_end > nq) q_end = nq;
  if (mode != 0) { q_begin = 0; q_end = nq; }
  if (q_begin < 0 || (q_begin & 1) || (q_end < nq && (q_end & 1)) || q_begin > q_end)
    return fail(ctx, MSA_EINVAL, "bad query range");
  const int p_begin = q_begin >= x1 ? npairs : q_begin / 2;
  const int p_end = q_end >= x1 ? npairs : q_end / 2;
  const double total_len = (double)suffix[0];
  auto partner_cells = [&](int x) { return mode == 0 ? (double)suffix[x] : total_len; };
  auto partners = [&](int x) { return mode == 0 ? (double)(n - x) : (double)n; };
  auto add_class = [&](int v, int ub, int ue) {
    if (!classes.empty() && classes.back().variant == v && classes.back().ue == ub) classes.back().ue = ue;
    else classes.push_back({v, ub, ue});
  };
  // Stacking shortens the item list by the stack height; it is only worth
  // it while the queries' own items fill the GPU many times over, in the
  // all-pairs and reference modes (not for a short candidate list), and
  // within one pass (a stack over several passes pays boundary rows the
  // model does not see).
  int64_t items_single = 0;
  for (int p = p_begin; p < p_end; ++p) items_single += (int64_t)(mode == 0 ? n - 2 * p : n) / 8;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev);
  const bool stack = mode != 2 && items_single >= 16 * 2 * 3 * (int64_t)std::max(sms, 1);
  for (int p = p_begin; p < p_end;) {
    int bv = -1, bm = 0;
    double bcost = 1e300;
    for (int v = 0; v < kNumCenterVariants; ++v) {
      const CenterVariant &cv = kCenterVariants[v];
      if (!cv.paired || !cv.packed) continue;
      const int GR = cv.G * cv.R;
      double corr = 1.0;
      if (!ctx->tune_corr.empty())
        for (size_t b = 0; b + 1 < ctx->tune_edges.size(); ++b)
          if (qlen[2 * p] >= ctx->tune_edges[b] && qlen[2 * p] < ctx->tune_edges[b + 1] &&
              ctx->tune_corr[b][v] > 0)
            corr = ctx->tune_corr[b][v];
      int rows = 0;
      double real = 0;
      for (int q = p; q < p_end && q - p < (stack ? kMaxSeg : 1); ++q) {
        const int rq = pair_rows(qlen, x1, q, cv.R);
        if (q > p && rows + rq > GR) break;  // stacks stay within one pass
        if (center_profile_bytes(v, ctx->K, round_up_int(rows + rq, GR)) > kMaxPairedProfile) break;
        rows += rq;
        const int xa = 2 * q, xb = 2 * q + 1;
        real += (double)qlen[xa] * partner_cells(xa) + (xb < x1 ? (double)qlen[xb] * partner_cells(xb) : 0.0);
        const int np = (rows + GR - 1) / GR;
        const double cost = (double)np * GR * (1.0 + 3.0 / cv.R) *
                            (partner_cells(2 * p) + partners(2 * p) * (cv.G - 1 + (np > 1 ? 48 : 0))) / corr;
        if (cost / real < bcost) { bcost = cost / real; bv = v; bm = q - p + 1; }
      }
    }
    if (bv < 0) {
      // no paired profile fits: the single-query packed kernels
      const int xq = std::min(2 * p + 1, x1 - 1);
      const int v = choose_variant(ctx, qlen[xq], est_at(xq), true);
      if (v < 0) return fail(ctx, MSA_ERANGE, "no center kernel fits a query of length %d", qlen[xq]);
      if (kCenterVariants[v].paired) {
        streams.push_back(make_int2(p, 1));
        add_class(v, (int)streams.size() - 1, (int)streams.size());
      } else {
        add_class(v, 2 * p, std::min(2 * p + 2, x1));
      }
      p += 1;
      continue;
    }
    streams.push_back(make_int2(p, bm));
    add_class(bv, (int)streams.size() - 1, (int)streams.size());
    p += bm;
  }
  // int32 part: single queries [x1, nq)
  for (int x = std::max(x1, q_begin); x < q_end;) {
    const int v = choose_variant(ctx, qlen[x], est_at(x), false);
    if (v < 0) return fail(ctx, MSA_ERANGE, "no center kernel fits a query of length %d", qlen[x]);
    int xe = x + 1;
    while (xe < q_end && choose_variant(ctx, qlen[xe], est_at(xe), false) == v) ++xe;
    classes.push_back({v, x, xe});
    x = xe;
  }
  if (classes.empty()) {  // an empty share
    ctx->cells[0] = 0;
    return MSA_OK;
  }
  std::vector<ClassPlan> plans;
  std::vector<int64_t> prefix_all;
  for (const CenterClass &cc : classes) {
    // a paired class may not pair across the packed / int32 boundary
    const int nq_list = kCenterVariants[cc.variant].paired ? x1 : nq;
    plans.push_back(plan_class(ctx, mode, nq_list, cc, qlen, n, prefix_all, streams));
  }
  TRY(stage_plans(ctx, plans, prefix_all, streams));
  const int32_t *self = view ? view->self : P<int32_t>(ctx->self);
  TRY(launch_plans(ctx, mode, plans, 0, n, ss, self));
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_CENTER_K);
  const float center_ms = ctx->stage_ms[ST_CENTER_K];
  int64_t cells = 0;
  if (mode == 0) {  // pairs q < s (the self scores are counted by their own pass)
    for (int x = q_begin; x < q_end; ++x) cells += (int64_t)lens[x] * suffix[x + 1];
  } else {
    for (int q : qsorted) cells += (int64_t)lens[q] * suffix[0];
  }
  ctx->cells[0] = cells;
  ctx->stage_ms[ST_CENTER_K] = center_ms;

  // pairs whose packed lanes may have overflowed: recompute in int32
  unsigned h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, ctx->derr, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (h[0] & MSA_DERR_OVERFLOW) return fail(ctx, MSA_ENOMEM, "int16 overflow list full");
  if (h[1] > 0) {
    const int cnt = (int)h[1];
    std::vector<int2> ov(cnt);
    CK(cudaMemcpyAsync(ov.data(), ctx->ovf.p, sizeof(int2) * cnt, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int32_t> dst(cnt);
    std::iota(dst.begin(), dst.end(), 0);
    TRY(ensure(ctx, ctx->ovf_scores, sizeof(int32_t) * cnt));
    std::vector<int2> ov_set(ov);  // the re-run takes loaded-set indices
    if (view)
      for (int2 &p : ov_set) p = make_int2(view->idx[p.x], view->idx[p.y]);
    TRY(run_pairs(ctx, ov_set, dst, P<int32_t>(ctx->ovf_scores)));
    CK((++ctx->launches, launch_apply_overflow)(mode, P<int2>(ctx->ovf),
                                                P<int32_t>(ctx->ovf_scores), cnt,
                                                P<unsigned long long>(ctx->pairsum), self,
                                                ctx->st));
  }
  return MSA_OK;
}

// Time every packed variant on each query-length bucket: up to 128 queries
// of the bucket, evenly spaced, against their real partners (every sequence
// from the bucket on, as in the all-pairs selection; query-side sums, which
// the selection never reads), keeping the second of two runs.
int autotune(msa_ctx *ctx) {
  static const int edges[] = {1, 48, 80, 112, 144, 176, 208, 256, 320, 384, 448, 512, 640,
                              768, 896, 1024, 1280, 1536, 2048, 3072, 4096, MSA_MAX_LEN + 1};
  const int nb = (int)(sizeof(edges) / sizeof(edges[0])) - 1;
  const int n = ctx->n;
  std::vector<std::vector<double>> rate(nb, std::vector<double>(kNumCenterVariants, 0.0));
  std::vector<std::vector<double>> corr(nb, std::vector<double>(kNumCenterVariants, 0.0));
  TRY(ensure(ctx, ctx->pairsum, sizeof(unsigned long long) * n));
  for (int b = 0; b < nb; ++b) {
    const int lo = edges[b], hi = edges[b + 1];
    const int xb = (int)(std::lower_bound(ctx->len_sorted.begin(), ctx->len_sorted.end(), lo) - ctx->len_sorted.begin());
    const int xe = (int)(std::lower_bound(ctx->len_sorted.begin(), ctx->len_sorted.end(), hi) - ctx->len_sorted.begin());
    if (xe <= xb) continue;
    std::vector<int32_t> qs;
    const int want = std::min(128, xe - xb);
    for (int i = 0; i < want; ++i) qs.push_back(xb + (int)((int64_t)i * (xe - xb) / want));
    std::vector<int> qlen;
    double qcells = 0;
    for (int q : qs) { qlen.push_back(ctx->len_sorted[q]); qcells += ctx->len_sorted[q]; }
    const int sub_off = xb, sub_n = n - xb;
    double scells = 0;
    for (int s = sub_off; s < n; ++s) scells += ctx->len_sorted[s];
    TRY(ensure(ctx, ctx->qlist, sizeof(int32_t) * qs.size()));
    CK(cudaMemcpyAsync(ctx->qlist.p, qs.data(), sizeof(int32_t) * qs.size(), cudaMemcpyHostToDevice, ctx->st));
    for (int v = 0; v < kNumCenterVariants; ++v) {
      const CenterVariant &cv = kCenterVariants[v];
      if (!cv.packed || !variant_fits(ctx, v, hi - 1)) continue;
      const int units = cv.paired ? ((int)qs.size() + 1) / 2 : (int)qs.size();
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        ms = 0.f;
        TRY(launch_class(ctx, 2, (int)qs.size(), CenterClass{v, 0, units}, qlen, ms, sub_off, sub_n));
      }
      if (ms > 0) rate[b][v] = qcells * scells / (ms * 1e-3);
    }
    // correction = measured / modelled rate, the model's rate being the
    // sample's cells over its modelled cost (the same constant for all
    // variants of the bucket)
    const int ls = (int)(scells / sub_n);
    for (int v = 0; v < kNumCenterVariants; ++v) {
      if (rate[b][v] <= 0) continue;
      double model = 0;
      for (int L : qlen) model += variant_cost(v, L, ls);
      corr[b][v] = rate[b][v] * model / (qcells * ls * (double)sub_n);
    }
  }
  ctx->tune_edges.assign(edges, edges + nb + 1);
  ctx->tune_rate = rate;
  ctx->tune_corr = corr;
  return MSA_OK;
}

// A reference list (input indices, distinct) -> ascending sorted positions.
int reference_positions(msa_ctx *ctx, const int64_t *refs, int64_t nref, std::vector<int32_t> &out) {
  const int n = ctx->n;
  if (!refs || nref < 1 || nref > n) return fail(ctx, MSA_EINVAL, "bad reference list");
  std::vector<char> seen(n, 0);
  out.clear();
  for (int64_t r = 0; r < nref; ++r) {
    if (refs[r] < 0 || refs[r] >= n) return fail(ctx, MSA_EINVAL, "reference index out of range");
    if (seen[refs[r]]) return fail(ctx, MSA_EINVAL, "duplicate reference index");
    seen[refs[r]] = 1;
    out.push_back(ctx->inv[refs[r]]);
  }
  std::sort(out.begin(), out.end());
  return MSA_OK;
}

// ------------------------------------------------------------ traceback-light alignment
// The passes of MSA_ALIGN_BOX (light.cu has the reasoning): every subject's
// best cell, then where best-scoring alignments ending there may start, then
// codes only inside the box between and the traceback over them.  The host
// reads the best cells and the corners back between the passes to order the
// subjects by their windows (pass count, then columns), so the groups of a
// warp stay in step.

// positions of items sorted by (passes of GR rows, columns), both descending
static void order_by_window(const std::vector<int4> &w, const std::vector<int32_t> &items, int GR,
                            int max_cols, int32_t *pos_of) {
  int max_np = 1;
  for (int k : items) max_np = std::max(max_np, (w[k].y + GR - 1) / GR);
  const size_t nb = (size_t)max_np * (max_cols + 1);
  std::vector<int32_t> start(nb + 1, 0);
  auto key = [&](int k) {
    const int np = std::max(1, (w[k].y + GR - 1) / GR);
    return (size_t)(np - 1) * (max_cols + 1) + (size_t)std::min(w[k].w, max_cols);
  };
  for (int k : items) ++start[key(k)];
  int acc = 0;
  for (size_t b = nb; b-- > 0;) {
    const int c = start[b];
    start[b] = acc;
    acc += c;
  }
  for (int k : items) pos_of[start[key(k)]++] = k;
}

// Pinned host staging of the light passes' round trips, per subject: its
// window (16 bytes), best-cell key, corner key, codes offset (8 bytes each)
// and position order (4 bytes).
struct LightStage {
  int4 *wpos;
  unsigned long long *keys, *keys2;
  int64_t *offs;
  int32_t *order;
};
static int light_staging(msa_ctx *ctx, int n, LightStage *ls) {
  const size_t need = (size_t)n * 44 + 64;
  if (need > ctx->pinned_cap) {
    if (ctx->pinned) {
      CK(cudaStreamSynchronize(ctx->st));
      CK(cudaFreeHost(ctx->pinned));
      ctx->pinned = nullptr;
      ctx->pinned_cap = 0;
    }
    CK(cudaHostAlloc(&ctx->pinned, need, cudaHostAllocDefault));
    ctx->pinned_cap = need;
  }
  char *p = static_cast<char *>(ctx->pinned);
  ls->wpos = reinterpret_cast<int4 *>(p);
  ls->keys = reinterpret_cast<unsigned long long *>(p + (size_t)16 * n);
  ls->keys2 = reinterpret_cast<unsigned long long *>(p + (size_t)24 * n);
  ls->offs = reinterpret_cast<int64_t *>(p + (size_t)32 * n);
  ls->order = reinterpret_cast<int32_t *>(p + (size_t)40 * n);
  return MSA_OK;
}

// Lanes per group of the box pass: the codes kernel's cost model with the
// boxes' mean height as the center length and their mean and largest widths
// as the subject lengths.  (On the 200,000 peptides and the 10k proteins it
// measured faster than a rule that fits 90% of the boxes into one pass.)
static int box_group(msa_ctx *ctx, const std::vector<int4> &box, int n) {
  double hs = 0.0, ws = 0.0;
  int wmax = 1, cnt = 0;
  for (int k = 0; k < n; ++k) {
    if (box[k].y <= 0) continue;
    hs += box[k].y;
    ws += box[k].w;
    wmax = std::max(wmax, box[k].w);
    ++cnt;
  }
  if (cnt == 0) return 32;
  return codes_group((int)std::ceil(hs / cnt), true, ctx->K, cnt, ws / cnt, wmax);
}

static int align_light(msa_ctx *ctx, int kc, int Lc) {
  const int n = ctx->n, R = kCodesR;
  const SeqSet ss = seqset(ctx);
  const Scoring sc = scoring(ctx);
  const int G = align_group(ctx, Lc, true), GR = G * R;
  const int npass = (Lc + GR - 1) / GR;
  const int smem1 = light_smem_bytes(ctx->K, Lc, G, 1, npass);
  CK(light_allow_smem(G, 1, smem1));
  const int grid1 = light_grid(G, 1, smem1);
  if (grid1 < 1)
    return fail(ctx, MSA_ERANGE, "a center of %d residues leaves no shared memory for the light passes", Lc);
  TRY(ensure(ctx, ctx->best, sizeof(unsigned long long) * n));
  TRY(ensure(ctx, ctx->light_order, sizeof(int32_t) * n));
  TRY(ensure(ctx, ctx->light_win, sizeof(int4) * n));
  TRY(ensure(ctx, ctx->light_keys, sizeof(unsigned long long) * n));
  TRY(ensure(ctx, ctx->code_off, sizeof(int64_t) * n));
  LightJob job{};
  job.center = kc;
  job.counter = ctx->dcounter;
  job.scratch_cols = ctx->maxlen;

  // 1. the best cell of every subject
  TRY(ensure(ctx, ctx->scratch, (size_t)grid1 * (kLightThreads / G) * 2 * ctx->maxlen * sizeof(int2)));
  job.scratch = P<int2>(ctx->scratch);
  job.sb = 0;
  job.se = n;
  job.npass = npass;
  job.best = P<unsigned long long>(ctx->best);
  CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
  stage_begin(ctx, ST_LIGHT_SCORE);
  CK((++ctx->launches, launch_light)(G, 1, ss, sc, job, grid1, smem1, ctx->st));
  stage_end(ctx, ST_LIGHT_SCORE);
  LightStage ls;
  TRY(light_staging(ctx, n, &ls));
  unsigned long long *keys = ls.keys, *keys2 = ls.keys2;
  int32_t *order = ls.order;
  int4 *wpos = ls.wpos;
  CK(cudaMemcpyAsync(keys, ctx->best.p, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_LIGHT_SCORE);

  // 2. the reversed prefixes of the subjects with a positive cell: rows
  // (i2 - p of the center, read from the reversed profile at Lc - i2, its
  // start rounded down to 16 with the rows above masked) and columns j2 - q
  std::vector<int4> &win = ctx->h_win;
  win.assign(n, make_int4(0, 0, 0, 0));
  std::vector<int32_t> &items = ctx->h_items;
  items.clear();
  for (int k = 0; k < n; ++k) {
    if (best_key_score(keys[k]) <= 0) continue;
    const int i2 = best_key_row(keys[k]), j2 = best_key_col(keys[k]);
    const int top = Lc - i2;
    win[k] = make_int4(top & ~15, (top & 15) + i2, top & 15, j2);
    items.push_back(k);
  }
  const int npos = (int)items.size();
  order_by_window(win, items, GR, ctx->maxlen, order);
  // the reversed windows span up to the whole center: the full pass's lanes
  const int G2 = G;
  const int smem2 = light_smem_bytes(ctx->K, Lc, G2, 2, 0);
  CK(light_allow_smem(G2, 2, smem2));
  const int grid2 = light_grid(G2, 2, smem2);
  if (grid2 < 1)
    return fail(ctx, MSA_ERANGE, "a center of %d residues leaves no shared memory for the light passes", Lc);
  TRY(ensure(ctx, ctx->scratch, (size_t)grid2 * (kLightThreads / G2) * 2 * ctx->maxlen * sizeof(int2)));
  job.scratch = P<int2>(ctx->scratch);
  for (int x = 0; x < npos; ++x) wpos[x] = win[order[x]];
  ctx->stage_ms[ST_LIGHT_CORNER] = 0.f;
  if (npos > 0) {
    CK(cudaMemcpyAsync(ctx->light_order.p, order, sizeof(int32_t) * npos, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->light_win.p, wpos, sizeof(int4) * npos, cudaMemcpyHostToDevice, ctx->st));
    job.npos = npos;
    job.order = P<int32_t>(ctx->light_order);
    job.win = P<int4>(ctx->light_win);
    job.best = P<unsigned long long>(ctx->light_keys);
    CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
    stage_begin(ctx, ST_LIGHT_CORNER);
    CK((++ctx->launches, launch_light)(G2, 2, ss, sc, job, grid2, smem2, ctx->st));
    stage_end(ctx, ST_LIGHT_CORNER);
    CK(cudaMemcpyAsync(keys2, ctx->light_keys.p, sizeof(unsigned long long) * npos, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_LIGHT_CORNER);
  }

  // 3. boxes: rows (i0, i2] with i0 = i2 - P rounded down to 16, columns
  // (j2 - Q, j2]; every subject takes part (no positive cell: an empty box,
  // the traceback writes its flanks)
  std::vector<int4> &box = ctx->h_box;
  box.assign(n, make_int4(0, 0, 0, 0));
  for (int x = 0; x < npos; ++x) {
    const int k = order[x];
    const int S = best_key_score(keys[k]), i2 = best_key_row(keys[k]), j2 = best_key_col(keys[k]);
    const int V = best_key_score(keys2[x]), Pr = best_key_row(keys2[x]), Qc = best_key_col(keys2[x]);
    if (V != S || Pr < 1 || Pr > i2 || Qc < 1 || Qc > j2)
      return fail(ctx, MSA_ECUDA, "light alignment: the reverse pass of sequence %d found %d at (%d, %d), "
                  "its best score is %d", ctx->perm[k], V, Pr, Qc, S);
    const int i0 = (i2 - Pr) & ~15;
    box[k] = make_int4(i0, i2 - i0, j2 - Qc, Qc);
  }
  // lanes per group of the box pass (or the context's fixed choice)
  std::vector<int32_t> &all = ctx->h_all;
  if ((int)all.size() != n) {
    all.resize(n);
    std::iota(all.begin(), all.end(), 0);
  }
  const int G3 = ctx->align_group_fixed ? ctx->align_group : box_group(ctx, box, n);
  const int smem3 = light_smem_bytes(ctx->K, Lc, G3, 3, 0);
  CK(light_allow_smem(G3, 3, smem3));
  const int grid3 = light_grid(G3, 3, smem3);
  if (grid3 < 1)
    return fail(ctx, MSA_ERANGE, "a center of %d residues leaves no shared memory for the light passes", Lc);
  TRY(ensure(ctx, ctx->scratch, (size_t)grid3 * (kLightThreads / G3) * 2 * ctx->maxlen * sizeof(int2)));
  job.scratch = P<int2>(ctx->scratch);
  order_by_window(box, all, G3 * R, ctx->maxlen, order);
  for (int x = 0; x < n; ++x) wpos[x] = box[order[x]];
  auto box_bytes = [&](const int4 &b) -> size_t { return b.y > 0 ? code_words(b.w, b.y, G3) * 8 : 0; };
  size_t all_codes = 0, max_one = 8;
  for (int x = 0; x < n; ++x) {
    all_codes += box_bytes(wpos[x]);
    max_one = std::max(max_one, box_bytes(wpos[x]));
  }
  size_t budget = all_codes;
  if (all_codes > ctx->codes.cap || all_codes > ctx->codes_budget) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    budget = std::min(ctx->codes_budget, free_b / 2);
    if (ctx->dev_limit) budget = std::min(budget, ctx->dev_limit > ctx->dev_bytes ? (ctx->dev_limit - ctx->dev_bytes) / 2 : 0);
  }
  if (budget < max_one) budget = max_one;
  std::vector<std::pair<int, int>> batches;
  int64_t *offs = ls.offs;
  size_t biggest = 8;
  {
    int b = 0;
    size_t acc = 0;
    for (int x = 0; x < n; ++x) {
      const size_t sz = box_bytes(wpos[x]);
      if (acc + sz > budget && x > b) {
        batches.push_back({b, x});
        biggest = std::max(biggest, acc);
        b = x;
        acc = 0;
      }
      offs[x] = (int64_t)acc;
      acc += sz;
    }
    batches.push_back({b, n});
    biggest = std::max(biggest, acc);
  }
  TRY(ensure(ctx, ctx->codes, biggest));
  CK(cudaMemcpyAsync(ctx->light_order.p, order, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->light_win.p, wpos, sizeof(int4) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->code_off.p, offs, sizeof(int64_t) * n, cudaMemcpyHostToDevice, ctx->st));
  const int nb = (int)batches.size();
  while ((int)ctx->align_ev.size() < 3 * nb) {
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreate(&ev));
    ctx->align_ev.push_back(ev);
  }
  for (int bi = 0; bi < nb; ++bi) {
    const int pb = batches[bi].first, pe = batches[bi].second;
    job.npos = pe - pb;
    job.order = P<int32_t>(ctx->light_order) + pb;
    job.win = P<int4>(ctx->light_win) + pb;
    job.code_off = P<int64_t>(ctx->code_off) + pb;
    job.codes = P<uint8_t>(ctx->codes);
    job.best = P<unsigned long long>(ctx->light_keys) + pb;
    CK(cudaEventRecord(ctx->align_ev[3 * bi], ctx->st));
    CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
    CK((++ctx->launches, launch_light)(G3, 3, ss, sc, job, grid3, smem3, ctx->st));
    CK(cudaEventRecord(ctx->align_ev[3 * bi + 1], ctx->st));
    CK((++ctx->launches, launch_traceback)(
        P<uint8_t>(ctx->codes), P<int64_t>(ctx->code_off) + pb, P<unsigned long long>(ctx->best), 0,
        pe - pb, P<int32_t>(ctx->d_len), P<int32_t>(ctx->d_perm), ss.res, ss.pstart, kc, sc.M, sc.K,
        sc.o, sc.e, Lc, G3, P<uint16_t>(ctx->ins), P<uint8_t>(ctx->occ), P<int32_t>(ctx->seg),
        P<int32_t>(ctx->score), ctx->derr, ctx->st, P<int32_t>(ctx->light_order) + pb,
        P<int4>(ctx->light_win) + pb, P<unsigned long long>(ctx->light_keys) + pb));
    CK(cudaEventRecord(ctx->align_ev[3 * bi + 2], ctx->st));
  }
  CK(cudaStreamSynchronize(ctx->st));
  float ms_box = 0.f, ms_tb = 0.f;
  for (int bi = 0; bi < nb; ++bi) {
    float a = 0.f, t = 0.f;
    CK(cudaEventElapsedTime(&a, ctx->align_ev[3 * bi], ctx->align_ev[3 * bi + 1]));
    CK(cudaEventElapsedTime(&t, ctx->align_ev[3 * bi + 1], ctx->align_ev[3 * bi + 2]));
    ms_box += a;
    ms_tb += t;
  }
  ctx->stage_ms[ST_LIGHT_BOX] = ms_box;
  ctx->stage_ms[ST_TRACE] = ms_tb;
  ctx->stage_ms[ST_ALIGN_K] = ctx->stage_ms[ST_LIGHT_SCORE] + ctx->stage_ms[ST_LIGHT_CORNER] + ms_box;
  ctx->stage_ms[ST_ALIGN] = ctx->stage_ms[ST_ALIGN_K];
  std::vector<int32_t> &hb = ctx->h_boxes;
  hb.assign((size_t)4 * n, 0);
  for (int k = 0; k < n; ++k) {
    if (box[k].y <= 0) continue;
    int32_t *b = &hb[(size_t)4 * ctx->perm[k]];
    b[0] = box[k].x;
    b[1] = box[k].z;
    b[2] = box[k].x + box[k].y;
    b[3] = box[k].z + box[k].w;
  }
  return MSA_OK;
}

}  // namespace msa_detail

using namespace msa_detail;

// ================================================================== C ABI

extern "C" {

int msa_create(msa_ctx **out, const msa_params *p, void *cuda_stream) {
  msa_ctx *ctx = nullptr;
  if (!out || !p) return MSA_EINVAL;
  *out = nullptr;
  if (p->alphabet < 1 || p->alphabet > MSA_MAX_ALPHABET || !p->matrix || !p->letters)
    return MSA_EINVAL;
  if (p->gap_extend < 1 || p->gap_open < p->gap_extend || p->gap_open > 1000) return MSA_EINVAL;
  if (p->precision < MSA_AUTO || p->precision > MSA_INT32) return MSA_EINVAL;
  if ((int)strlen(p->letters) != p->alphabet) return MSA_EINVAL;
  for (int a = 0; a < p->alphabet; ++a) {
    if (p->letters[a] == '-') return MSA_EINVAL;
    for (int b = 0; b < p->alphabet; ++b) {
      if (p->matrix[a * p->alphabet + b] != p->matrix[b * p->alphabet + a]) return MSA_EINVAL;
    }
    for (int b = 0; b < a; ++b)
      if (p->letters[a] == p->letters[b]) return MSA_EINVAL;
  }
  ctx = new (std::nothrow) msa_ctx;
  if (!ctx) return MSA_ENOMEM;
  ctx->K = p->alphabet;
  ctx->o = p->gap_open;
  ctx->e = p->gap_extend;
  ctx->precision = p->precision;
  ctx->sat_limit = p->sat_limit > 0 ? std::min(p->sat_limit, 32767) : 32767;
  ctx->hM.assign(p->matrix, p->matrix + ctx->K * ctx->K);
  ctx->letters.assign(p->letters, p->letters + ctx->K);
  ctx->smax = -128;
  ctx->smin = 127;
  for (int8_t v : ctx->hM) {
    ctx->smax = std::max<int>(ctx->smax, v);
    ctx->smin = std::min<int>(ctx->smin, v);
  }
  // the profiles hold s + o as int8
  if (ctx->smax + ctx->o > 127 || ctx->smin + ctx->o < -128) {
    delete ctx;
    return MSA_EINVAL;
  }
  memset(ctx->hlut, 255, sizeof ctx->hlut);
  for (int a = 0; a < ctx->K; ++a) ctx->hlut[(uint8_t)ctx->letters[a]] = (uint8_t)a;
  ctx->st = (cudaStream_t)cuda_stream;

  auto init = [&]() -> int {
    CK(cudaGetDevice(&ctx->dev));
    CK(cudaMalloc(&ctx->dM, MSA_MAX_ALPHABET * MSA_MAX_ALPHABET));
    CK(cudaMemcpy(ctx->dM, ctx->hM.data(), ctx->hM.size(), cudaMemcpyHostToDevice));
    char lt[MSA_MAX_ALPHABET + 1] = {0};
    memcpy(lt, ctx->letters.data(), ctx->K);
    lt[ctx->K] = '-';
    CK(cudaMalloc(&ctx->dLetters, sizeof lt));
    CK(cudaMemcpy(ctx->dLetters, lt, sizeof lt, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->dLut, 256));
    CK(cudaMemcpy(ctx->dLut, ctx->hlut, 256, cudaMemcpyHostToDevice));
    // SP symbols: letters 0..K-1, any other byte K, the gap '-' last (K+1)
    uint8_t sym[256];
    memset(sym, ctx->K, sizeof sym);
    for (int a = 0; a < ctx->K; ++a) sym[(uint8_t)ctx->letters[a]] = (uint8_t)a;
    sym[(uint8_t)'-'] = (uint8_t)(ctx->K + 1);
    CK(cudaMalloc(&ctx->dSymLut, 256));
    CK(cudaMemcpy(ctx->dSymLut, sym, 256, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->dcounter, sizeof(unsigned long long)));
    CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->cap_st2, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->cap_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->cap_join, cudaEventDisableTiming));
    CK(cudaMalloc(&ctx->derr, 2 * sizeof(unsigned)));
    CK(cudaMemset(ctx->derr, 0, 2 * sizeof(unsigned)));
    CK(cudaMalloc(&ctx->dsmall, 8 * sizeof(long long)));
    for (auto &ev : ctx->ev) CK(cudaEventCreate(&ev));
    TRY(ensure(ctx, ctx->ovf, sizeof(int2) * (1 << 20)));
    return MSA_OK;
  };
  int rc = init();
  if (rc != MSA_OK) {
    msa_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return MSA_OK;
}

void msa_destroy(msa_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->st);
  selector_free(ctx, ctx->sel);
  ctx->sel = nullptr;
  DevBuf *bufs[] = {&ctx->res, &ctx->d_pstart, &ctx->d_len, &ctx->d_perm, &ctx->d_inv,
                    &ctx->d_srcoff, &ctx->staging, &ctx->pairsum, &ctx->self, &ctx->rowsum,
                    &ctx->prefix, &ctx->qlist, &ctx->ovf, &ctx->ovf_scores, &ctx->ovf_dst,
                    &ctx->part_val, &ctx->part_idx, &ctx->pairs, &ctx->pair_dst,
                    &ctx->pair_out, &ctx->ins, &ctx->occ, &ctx->seg, &ctx->score,
                    &ctx->codes, &ctx->code_off, &ctx->best, &ctx->G, &ctx->off, &ctx->msa,
                    &ctx->counts, &ctx->scratch, &ctx->counters, &ctx->streams,
                    &ctx->light_order, &ctx->light_win, &ctx->light_keys};
  for (DevBuf *b : bufs)
    if (b->p) cudaFree(b->p);
  cudaFree(ctx->dM);
  cudaFree(ctx->dLetters);
  cudaFree(ctx->dLut);
  cudaFree(ctx->dSymLut);
  cudaFree(ctx->dcounter);
  if (ctx->center_exec) cudaGraphExecDestroy(ctx->center_exec);
  if (ctx->align_exec) cudaGraphExecDestroy(ctx->align_exec);
  for (cudaEvent_t ev : ctx->align_ev) cudaEventDestroy(ev);
  if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
  if (ctx->cap_st2) cudaStreamDestroy(ctx->cap_st2);
  if (ctx->cap_fork) cudaEventDestroy(ctx->cap_fork);
  if (ctx->cap_join) cudaEventDestroy(ctx->cap_join);
  cudaFree(ctx->derr);
  cudaFree(ctx->dsmall);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (auto &ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  delete ctx;
}

const char *msa_last_error(const msa_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int msa_load(msa_ctx *ctx, const uint8_t *letters, const int64_t *offsets, int64_t n) {
  if (!ctx) return MSA_EINVAL;
  if (!letters || !offsets || n < 1) return fail(ctx, MSA_EINVAL, "empty input");
  if (n > (int64_t)INT32_MAX / 2) return fail(ctx, MSA_ERANGE, "too many sequences");
  if (offsets[0] != 0) return fail(ctx, MSA_EINVAL, "offsets[0] must be 0");
  TRY(set_device(ctx));
  std::vector<int32_t> &lens = ctx->h_lens;
  lens.resize(n);
  int maxlen = 0;
  for (int64_t t = 0; t < n; ++t) {
    const int64_t L = offsets[t + 1] - offsets[t];
    if (L <= 0) return fail(ctx, MSA_EINVAL, "sequence %lld is empty", (long long)t);
    if (L > MSA_MAX_LEN) return fail(ctx, MSA_ERANGE, "sequence %lld longer than %d", (long long)t, MSA_MAX_LEN);
    lens[t] = (int32_t)L;
    maxlen = std::max(maxlen, (int)L);
  }
  ctx->aligned = ctx->merged = ctx->have_rowsum = false;
  ctx->n = (int)n;
  ctx->maxlen = maxlen;
  // stable sort by length: a counting sort (lengths are at most MSA_MAX_LEN);
  // the inverse permutation is written in input order during the scatter and
  // the sorted lengths from the bucket counts, so no pass gathers at random
  ctx->perm.resize(n);
  ctx->inv.resize(n);
  ctx->len_sorted.resize(n);
  ctx->pstart.resize(n);
  {
    std::vector<int64_t> first(maxlen + 2, 0);
    for (int64_t t = 0; t < n; ++t) ++first[lens[t] + 1];
    for (int L = 1; L <= maxlen + 1; ++L) first[L] += first[L - 1];
    for (int L = 1; L <= maxlen; ++L)
      std::fill(ctx->len_sorted.begin() + first[L], ctx->len_sorted.begin() + first[L + 1], L);
    for (int64_t t = 0; t < n; ++t) {
      const int64_t k = first[lens[t]]++;
      ctx->perm[k] = (int32_t)t;
      ctx->inv[t] = (int32_t)k;
    }
  }
  int64_t pos = 0;
  for (int64_t k = 0; k < n; ++k) {
    ctx->pstart[k] = pos;
    pos += round_up_i64(ctx->len_sorted[k], 16) + MSA_SEQ_TAIL;
  }
  const int64_t total = offsets[n];
  TRY(ensure(ctx, ctx->res, pos));
  TRY(ensure(ctx, ctx->d_pstart, sizeof(int64_t) * n));
  TRY(ensure(ctx, ctx->d_len, sizeof(int32_t) * n));
  TRY(ensure(ctx, ctx->d_perm, sizeof(int32_t) * n));
  TRY(ensure(ctx, ctx->d_inv, sizeof(int32_t) * n));
  TRY(ensure(ctx, ctx->d_srcoff, sizeof(int64_t) * (n + 1)));
  TRY(ensure(ctx, ctx->pairsum, sizeof(unsigned long long) * n));
  TRY(ensure(ctx, ctx->self, sizeof(int32_t) * n));
  TRY(ensure(ctx, ctx->rowsum, sizeof(long long) * n));
  TRY(ensure(ctx, ctx->part_val, sizeof(long long) * 1024));
  TRY(ensure(ctx, ctx->part_idx, sizeof(long long) * 1024));
  stage_begin(ctx, ST_ENCODE);
  const uint8_t *src = letters;
  if (!is_device_ptr(letters)) {
    TRY(ensure(ctx, ctx->staging, total));
    CK(cudaMemcpyAsync(ctx->staging.p, letters, total, cudaMemcpyHostToDevice, ctx->st));
    src = P<uint8_t>(ctx->staging);
  }
  CK(cudaMemcpyAsync(ctx->d_pstart.p, ctx->pstart.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_len.p, ctx->len_sorted.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_perm.p, ctx->perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_inv.p, ctx->inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->d_srcoff.p, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
  CK((++ctx->launches, launch_encode)(src, P<int64_t>(ctx->d_srcoff), P<int32_t>(ctx->d_perm), P<int64_t>(ctx->d_pstart),
                   P<int32_t>(ctx->d_len), ctx->n, ctx->dLut, ctx->K, P<uint8_t>(ctx->res), ctx->derr,
                   ctx->st));
  stage_end(ctx, ST_ENCODE);
  int rc = check_derr(ctx);
  stage_collect(ctx, ST_ENCODE);
  if (rc != MSA_OK) {
    ctx->n = 0;
    return rc;
  }
  return MSA_OK;
}

int msa_pair_scores(msa_ctx *ctx, const int64_t *pairs, int64_t npairs, int32_t *scores_out) {
  if (!ctx) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (npairs < 0 || (npairs > 0 && (!pairs || !scores_out))) return fail(ctx, MSA_EINVAL, "bad pair list");
  if (npairs == 0) return MSA_OK;
  if (npairs > INT32_MAX / 2) return fail(ctx, MSA_ERANGE, "too many pairs");
  TRY(set_device(ctx));
  std::vector<int2> pr(npairs);
  std::vector<int32_t> dst(npairs);
  for (int64_t x = 0; x < npairs; ++x) {
    const int64_t a = pairs[2 * x], b = pairs[2 * x + 1];
    if (a < 0 || b < 0 || a >= ctx->n || b >= ctx->n) return fail(ctx, MSA_EINVAL, "pair index out of range");
    pr[x] = make_int2(ctx->inv[a], ctx->inv[b]);
    dst[x] = (int32_t)x;
  }
  TRY(ensure(ctx, ctx->pair_out, sizeof(int32_t) * npairs));
  TRY(run_pairs(ctx, pr, dst, P<int32_t>(ctx->pair_out)));
  CK(cudaMemcpyAsync(scores_out, ctx->pair_out.p, sizeof(int32_t) * npairs, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_select_center_refined(msa_ctx *ctx, int32_t candidates, const int64_t *refs, int64_t nref,
                              int64_t *center_out, int64_t *sum_dist_out) {
  if (!ctx) return MSA_EINVAL;
  if (!center_out) return fail(ctx, MSA_EINVAL, "center_out is NULL");
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (candidates < 0) return fail(ctx, MSA_EINVAL, "negative candidate count");
  TRY(set_device(ctx));
  if (sum_dist_out) *sum_dist_out = 0;
  std::vector<int32_t> rs;
  if (refs && nref > 0) TRY(reference_positions(ctx, refs, nref, rs));
  return selector_center_refined(ctx, candidates > 0 ? std::min(candidates, ctx->n) : 32, rs,
                                 center_out, sum_dist_out);
}

int msa_select_center(msa_ctx *ctx, int mode, const int64_t *refs, int64_t nref,
                      int64_t *center_out, int64_t *sum_dist_out) {
  if (!ctx) return MSA_EINVAL;
  if (!center_out) return fail(ctx, MSA_EINVAL, "center_out is NULL");
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  TRY(set_device(ctx));
  if (sum_dist_out) *sum_dist_out = 0;
  if (mode == MSA_CENTER_FIRST) {
    *center_out = 0;
    return MSA_OK;
  }
  if (mode == MSA_CENTER_LEARNED) return selector_center(ctx, center_out);
  if (mode == MSA_CENTER_LEARNED_REFINED)
    return selector_center_refined(ctx, nref > 0 ? (int)std::min<int64_t>(nref, ctx->n) : 32,
                                   {}, center_out, sum_dist_out);
  if (mode != MSA_CENTER_EXACT && mode != MSA_CENTER_EXACT_SAMPLED)
    return fail(ctx, MSA_EINVAL, "unknown center mode %d", mode);
  const int n = ctx->n;
  std::vector<int32_t> qs;
  if (mode == MSA_CENTER_EXACT_SAMPLED) TRY(reference_positions(ctx, refs, nref, qs));
  stage_begin(ctx, ST_CENTER);
  CK(cudaMemsetAsync(ctx->pairsum.p, 0, sizeof(unsigned long long) * n, ctx->st));
  CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
  // self scores of every sequence first: every pair's similarity needs both
  {
    std::vector<int2> sp(n);
    std::vector<int32_t> dst(n);
    for (int k = 0; k < n; ++k) { sp[k] = make_int2(k, k); dst[k] = k; }
    TRY(run_pairs(ctx, sp, dst, P<int32_t>(ctx->self)));
  }
  TRY(run_center(ctx, mode == MSA_CENTER_EXACT ? 0 : 1, qs));
  {
    double sumsq = 0;
    for (int k = 0; k < n; ++k) sumsq += (double)ctx->len_sorted[k] * ctx->len_sorted[k];
    ctx->cells[0] += (int64_t)sumsq;
  }
  CK((++ctx->launches, launch_center_finalize)(mode == MSA_CENTER_EXACT ? 0 : 1, n, (int)qs.size(),
                            P<int32_t>(ctx->d_perm), P<unsigned long long>(ctx->pairsum),
                            P<long long>(ctx->rowsum), ctx->dsmall + 1, ctx->dsmall + 2,
                            P<long long>(ctx->part_val), P<long long>(ctx->part_idx), ctx->st));
  stage_end(ctx, ST_CENTER);
  long long h[3];
  CK(cudaMemcpyAsync(h, ctx->dsmall, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  TRY(check_derr(ctx));
  stage_collect(ctx, ST_CENTER);
  *center_out = h[2];
  if (sum_dist_out) *sum_dist_out = h[1];
  ctx->have_rowsum = true;
  return MSA_OK;
}

int msa_center_rowsums(msa_ctx *ctx, int64_t *rowsum_out) {
  if (!ctx || !rowsum_out) return MSA_EINVAL;
  if (!ctx->have_rowsum) return fail(ctx, MSA_ESTATE, "no exact center selection yet");
  TRY(set_device(ctx));
  CK(cudaMemcpyAsync(rowsum_out, ctx->rowsum.p, sizeof(int64_t) * ctx->n, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_center_partial(msa_ctx *ctx, const int64_t *refs, int64_t nref, int32_t shard,
                       int32_t nshards, uint64_t *sums_out) {
  if (!ctx) return MSA_EINVAL;
  if (!sums_out) return fail(ctx, MSA_EINVAL, "sums_out is NULL");
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (nshards < 1 || shard < 0 || shard >= nshards) return fail(ctx, MSA_EINVAL, "bad shard");
  TRY(set_device(ctx));
  const int n = ctx->n;
  const bool sampled = refs && nref > 0;
  std::vector<int32_t> qs;
  if (sampled) TRY(reference_positions(ctx, refs, nref, qs));
  CK(cudaMemsetAsync(ctx->pairsum.p, 0, sizeof(unsigned long long) * n, ctx->st));
  CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
  {  // every pair's similarity needs both self scores
    std::vector<int2> sp(n);
    std::vector<int32_t> dst(n);
    for (int k = 0; k < n; ++k) { sp[k] = make_int2(k, k); dst[k] = k; }
    TRY(run_pairs(ctx, sp, dst, P<int32_t>(ctx->self)));
  }
  if (sampled) {
    // the references (queries) in contiguous chunks of about equal length sum
    std::vector<int32_t> mine;
    int64_t total = 0, acc = 0;
    for (int q : qs) total += ctx->len_sorted[q];
    for (int q : qs) {
      const int64_t mid2 = 2 * acc + ctx->len_sorted[q];  // twice the query's midpoint
      const int owner = (int)std::min<int64_t>(nshards - 1, mid2 * nshards / std::max<int64_t>(2 * total, 1));
      if (owner == shard) mine.push_back(q);
      acc += ctx->len_sorted[q];
    }
    if (!mine.empty()) TRY(run_center(ctx, 1, mine));
  } else {
    // the all-pairs triangle: query x meets the sequences after it, work
    // len[x] * (sum of the later lengths); contiguous even-aligned ranges of
    // about equal work
    std::vector<int64_t> suffix(n + 1, 0);
    for (int k = n - 1; k >= 0; --k) suffix[k] = suffix[k + 1] + ctx->len_sorted[k];
    std::vector<double> work(n + 1, 0.0);
    for (int k = 0; k < n; ++k) work[k + 1] = work[k] + (double)ctx->len_sorted[k] * suffix[k + 1];
    auto cut = [&](int r) {
      if (r <= 0) return 0;
      if (r >= nshards) return n;
      const double target = work[n] * r / nshards;
      int x = (int)(std::lower_bound(work.begin(), work.end(), target) - work.begin());
      x = std::min(n, std::max(0, x & ~1));
      return x;
    };
    const int qa = cut(shard), qe = shard + 1 == nshards ? n : cut(shard + 1);
    if (qe > qa) TRY(run_center(ctx, 0, {}, nullptr, qa, qe));
  }
  std::vector<unsigned long long> sorted(n), out(n);
  CK(cudaMemcpyAsync(sorted.data(), ctx->pairsum.p, sizeof(unsigned long long) * n,
                     cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  TRY(check_derr(ctx));
  for (int k = 0; k < n; ++k) out[ctx->perm[k]] = sorted[k];
  CK(cudaMemcpyAsync(sums_out, out.data(), sizeof(uint64_t) * n, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_center_combine(msa_ctx *ctx, const uint64_t *sums, int64_t nref, int64_t *center_out,
                       int64_t *sum_dist_out) {
  if (!ctx) return MSA_EINVAL;
  if (!sums || !center_out) return fail(ctx, MSA_EINVAL, "NULL argument");
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (nref < 0 || nref > ctx->n) return fail(ctx, MSA_EINVAL, "bad reference count");
  TRY(set_device(ctx));
  const int n = ctx->n;
  std::vector<unsigned long long> in(n), sorted(n);
  CK(cudaMemcpyAsync(in.data(), sums, sizeof(uint64_t) * n, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int k = 0; k < n; ++k) sorted[k] = in[ctx->perm[k]];
  CK(cudaMemcpyAsync(ctx->pairsum.p, sorted.data(), sizeof(unsigned long long) * n,
                     cudaMemcpyHostToDevice, ctx->st));
  CK((++ctx->launches, launch_center_finalize)(nref > 0 ? 1 : 0, n, (int)nref,
                            P<int32_t>(ctx->d_perm), P<unsigned long long>(ctx->pairsum),
                            P<long long>(ctx->rowsum), ctx->dsmall + 1, ctx->dsmall + 2,
                            P<long long>(ctx->part_val), P<long long>(ctx->part_idx), ctx->st));
  long long h[3];
  CK(cudaMemcpyAsync(h, ctx->dsmall, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *center_out = h[2];
  if (sum_dist_out) *sum_dist_out = h[1];
  ctx->have_rowsum = true;
  return MSA_OK;
}

int msa_align_to_center(msa_ctx *ctx, int64_t center, int32_t *scores_out) {
  if (!ctx) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (center < 0 || center >= ctx->n) return fail(ctx, MSA_EINVAL, "center index out of range");
  TRY(set_device(ctx));
  const int n = ctx->n;
  const int kc = ctx->inv[center];
  const int Lc = ctx->len_sorted[kc];
  ctx->aligned = ctx->merged = false;
  ctx->center = center;
  ctx->Lc = Lc;
  const bool packed = codes_packed(ctx, Lc);
  const int R = kCodesR, G = align_group(ctx, Lc, packed);
  const int npass = (Lc + G * R - 1) / (G * R);
  const size_t row = (size_t)Lc + 1;
  TRY(ensure(ctx, ctx->ins, sizeof(uint16_t) * row * n));
  TRY(ensure(ctx, ctx->occ, row * n));
  TRY(ensure(ctx, ctx->seg, sizeof(int32_t) * 5 * n));
  TRY(ensure(ctx, ctx->score, sizeof(int32_t) * n));
  CK(cudaMemsetAsync(ctx->ins.p, 0, sizeof(uint16_t) * row * n, ctx->st));
  CK(cudaMemsetAsync(ctx->occ.p, 0, row * n, ctx->st));
  CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
  ctx->light_used = false;
  if (ctx->align_mode == MSA_ALIGN_BOX && packed) {
    int64_t matrix_cells = 0;
    for (int k = 0; k < n; ++k) matrix_cells += (int64_t)Lc * ctx->len_sorted[k];
    TRY(align_light(ctx, kc, Lc));
    ctx->cells[1] = matrix_cells;
    TRY(check_derr(ctx));
    if (scores_out) {
      CK(cudaMemcpyAsync(scores_out, ctx->score.p, sizeof(int32_t) * n, cudaMemcpyDefault, ctx->st));
      CK(cudaStreamSynchronize(ctx->st));
    }
    ctx->light_used = true;
    ctx->aligned = true;
    return MSA_OK;
  }

  // batches of subjects (sorted order) whose codes fit the budget; when all
  // of them fit the codes buffer the context already holds (and the budget),
  // one batch, without asking the driver for the free memory
  size_t all_codes = 0;
  int64_t cells = 0;
  for (int k = 0; k < n; ++k) {
    all_codes += code_words(ctx->len_sorted[k], Lc, G) * 8;
    cells += (int64_t)Lc * ctx->len_sorted[k];
  }
  size_t budget = all_codes;
  if (all_codes > ctx->codes.cap || all_codes > ctx->codes_budget ||
      (ctx->dev_limit && all_codes > ctx->codes.cap)) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    budget = std::min(ctx->codes_budget, free_b / 2);
    if (ctx->dev_limit) budget = std::min(budget, ctx->dev_limit > ctx->dev_bytes ? (ctx->dev_limit - ctx->dev_bytes) / 2 : 0);
  }
  size_t max_one = code_words(ctx->maxlen, Lc, G) * 8;
  if (budget < max_one) budget = max_one;
  std::vector<std::pair<int, int>> batches;
  std::vector<int64_t> &offs = ctx->h_offs;
  offs.resize(n);
  size_t biggest = 0;
  {
    int b = 0;
    size_t acc = 0;
    for (int k = 0; k < n; ++k) {
      const size_t sz = code_words(ctx->len_sorted[k], Lc, G) * 8;
      if (acc + sz > budget && k > b) {
        batches.push_back({b, k});
        biggest = std::max(biggest, acc);
        b = k;
        acc = 0;
      }
      offs[k] = (int64_t)acc;
      acc += sz;
    }
    batches.push_back({b, n});
    biggest = std::max(biggest, acc);
  }
  TRY(ensure(ctx, ctx->codes, biggest));
  TRY(ensure(ctx, ctx->code_off, sizeof(int64_t) * n));
  TRY(ensure(ctx, ctx->best, sizeof(unsigned long long) * n));
  CK(cudaMemcpyAsync(ctx->code_off.p, offs.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, ctx->st));
  const SeqSet ss = seqset(ctx);
  const Scoring sc = scoring(ctx);
  const int smem = codes_smem_bytes(ctx->K, npass * G * R);
  const int cta = align_cta(ctx, G, packed);
  const int grid = codes_grid(G, packed, smem, cta);
  if (npass > 1)
    TRY(ensure(ctx, ctx->scratch, (size_t)grid * (codes_threads(packed, cta) / G) * 2 * ctx->maxlen * sizeof(int2)));
  float ms_dp = 0.f, ms_tb = 0.f;
  // All batches as one CUDA graph (captured on the context's private stream,
  // launched on its stream, cached while the key holds): per batch the fill
  // and the traceback, with timing events, and no host round trip between
  // batches (the codes buffer is reused in stream order).
  const int nb = (int)batches.size();
  while ((int)ctx->align_ev.size() < 3 * nb) {
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreate(&ev));
    ctx->align_ev.push_back(ev);
  }
  std::vector<int64_t> key = {kc, Lc, packed, G, cta, npass, grid, smem, n, (int64_t)ss.res,
                              (int64_t)ss.pstart, (int64_t)ss.len, (int64_t)sc.M, sc.K, sc.o, sc.e,
                              (int64_t)ctx->codes.p, (int64_t)ctx->code_off.p, (int64_t)ctx->best.p,
                              (int64_t)ctx->ins.p, (int64_t)ctx->occ.p, (int64_t)ctx->seg.p,
                              (int64_t)ctx->score.p, (int64_t)ctx->scratch.p, (int64_t)ctx->derr,
                              (int64_t)ctx->dcounter, (int64_t)ctx->d_perm.p, ctx->maxlen};
  for (auto [sb, se] : batches) { key.push_back(sb); key.push_back(se); }
  CK(codes_allow_smem(G, packed, smem, cta));
  if (!ctx->align_exec || key != ctx->align_key) {
    if (ctx->align_exec) {
      CK(cudaStreamSynchronize(ctx->st));
      cudaGraphExecDestroy(ctx->align_exec);
      ctx->align_exec = nullptr;
      ctx->align_key.clear();
    }
    CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int bi = 0; bi < nb && e == cudaSuccess; ++bi) {
      const int sb = batches[bi].first, se = batches[bi].second;
      CodesJob job;
      job.center = kc;
      job.sb = sb;
      job.se = se;
      job.code_off = P<int64_t>(ctx->code_off) + sb;
      job.codes = P<uint8_t>(ctx->codes);
      job.best = P<unsigned long long>(ctx->best) + sb;
      job.npass = npass;
      job.counter = ctx->dcounter;
      job.scratch = P<int2>(ctx->scratch);
      job.scratch_cols = ctx->maxlen;
      e = cudaEventRecordWithFlags(ctx->align_ev[3 * bi], ctx->cap_st, cudaEventRecordExternal);
      if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->cap_st);
      // offsets inside the batch are relative to the batch start
      if (e == cudaSuccess) e = launch_codes(G, packed, ss, sc, job, grid, ctx->cap_st, false, cta);
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(ctx->align_ev[3 * bi + 1], ctx->cap_st, cudaEventRecordExternal);
      if (e == cudaSuccess)
        e = launch_traceback(P<uint8_t>(ctx->codes), P<int64_t>(ctx->code_off) + sb,
                             P<unsigned long long>(ctx->best) + sb, sb, se, P<int32_t>(ctx->d_len),
                             P<int32_t>(ctx->d_perm), ss.res, ss.pstart, kc, sc.M, sc.K, sc.o, sc.e,
                             Lc, G, P<uint16_t>(ctx->ins), P<uint8_t>(ctx->occ), P<int32_t>(ctx->seg),
                             P<int32_t>(ctx->score), ctx->derr, ctx->cap_st);
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(ctx->align_ev[3 * bi + 2], ctx->cap_st, cudaEventRecordExternal);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(ctx->cap_st, &graph);
    if (e == cudaSuccess) e = e_end;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    CK(e);
    ctx->align_exec = exec;
    ctx->align_key = key;
  }
  ctx->launches += 2 * nb;
  stage_begin(ctx, ST_ALIGN);
  CK(cudaGraphLaunch(ctx->align_exec, ctx->st));
  stage_end(ctx, ST_ALIGN);
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_ALIGN);
  bool split = true;
  for (int bi = 0; bi < nb && split; ++bi) {
    float a = 0.f, t = 0.f;
    if (cudaEventElapsedTime(&a, ctx->align_ev[3 * bi], ctx->align_ev[3 * bi + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&t, ctx->align_ev[3 * bi + 1], ctx->align_ev[3 * bi + 2]) == cudaSuccess) {
      ms_dp += a;
      ms_tb += t;
    } else {
      cudaGetLastError();
      split = false;
    }
  }
  if (!split) {  // no per-batch split: the whole graph counts as the fill
    ms_dp = ctx->stage_ms[ST_ALIGN];
    ms_tb = 0.f;
  }
  ctx->stage_ms[ST_ALIGN] = ms_dp;
  ctx->stage_ms[ST_ALIGN_K] = ms_dp;
  ctx->stage_ms[ST_TRACE] = ms_tb;
  ctx->cells[1] = cells;
  TRY(check_derr(ctx));
  if (scores_out) {
    CK(cudaMemcpyAsync(scores_out, ctx->score.p, sizeof(int32_t) * n, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  ctx->aligned = true;
  return MSA_OK;
}

int msa_alignment_info(msa_ctx *ctx, int32_t *seg_out, uint16_t *ins_out, uint8_t *occ_out) {
  if (!ctx) return MSA_EINVAL;
  if (!ctx->aligned) return fail(ctx, MSA_ESTATE, "no alignment yet");
  TRY(set_device(ctx));
  const size_t n = ctx->n, row = (size_t)ctx->Lc + 1;
  if (seg_out) CK(cudaMemcpyAsync(seg_out, ctx->seg.p, sizeof(int32_t) * 5 * n, cudaMemcpyDefault, ctx->st));
  if (ins_out) CK(cudaMemcpyAsync(ins_out, ctx->ins.p, sizeof(uint16_t) * row * n, cudaMemcpyDefault, ctx->st));
  if (occ_out) CK(cudaMemcpyAsync(occ_out, ctx->occ.p, row * n, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_debug_codes(msa_ctx *ctx, int64_t seq, uint8_t *codes_out) {
  if (!ctx || !codes_out) return MSA_EINVAL;
  if (!ctx->aligned) return fail(ctx, MSA_ESTATE, "no alignment yet");
  if (seq < 0 || seq >= ctx->n) return fail(ctx, MSA_EINVAL, "sequence index out of range");
  TRY(set_device(ctx));
  // Recompute the codes of this one subject into a private buffer.  On the
  // packed path a subject at an odd sorted position is recomputed in the
  // high lane, beside the next one, so both lanes are open to inspection.
  const int ks = ctx->inv[seq], kc = ctx->inv[ctx->center];
  const int Lc = ctx->Lc, Ls = ctx->len_sorted[ks];
  const bool packed = codes_packed(ctx, Lc);
  const int R = kCodesR, G = align_group(ctx, Lc, packed);
  const int npass = (Lc + G * R - 1) / (G * R);
  const bool high = packed && (ks & 1) && ks + 1 < ctx->n;
  const int se = high ? ks + 2 : ks + 1;
  const size_t bytes = code_words(Ls, Lc, G) * 8;
  const size_t bytes_all = high ? bytes + code_words(ctx->len_sorted[ks + 1], Lc, G) * 8 : bytes;
  DevBuf cb, ob, bb;
  auto cleanup = [&]() { for (DevBuf *b : {&cb, &ob, &bb}) release(ctx, *b); };
  int rc = [&]() -> int {
    TRY(ensure(ctx, cb, bytes_all));
    TRY(ensure(ctx, ob, 2 * sizeof(int64_t)));
    TRY(ensure(ctx, bb, sizeof(unsigned long long) * 2));
    const int64_t offs[2] = {0, (int64_t)bytes};
    CK(cudaMemcpyAsync(ob.p, offs, sizeof(offs), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(ctx->dcounter, 0, sizeof(unsigned long long), ctx->st));
    const int smem = codes_smem_bytes(ctx->K, npass * G * R);
    const int grid = 1;
    const int cta = align_cta(ctx, G, packed);
    if (npass > 1)
      TRY(ensure(ctx, ctx->scratch, (size_t)codes_grid(G, packed, smem, cta) * (codes_threads(packed, cta) / G) *
                                        2 * ctx->maxlen * sizeof(int2)));
    CodesJob job;
    job.center = kc;
    job.sb = ks;
    job.se = se;
    job.code_off = P<int64_t>(ob);
    job.codes = P<uint8_t>(cb);
    job.best = P<unsigned long long>(bb);
    job.npass = npass;
    job.counter = ctx->dcounter;
    job.scratch = P<int2>(ctx->scratch);
    job.scratch_cols = ctx->maxlen;
    CK((++ctx->launches, launch_codes)(G, packed, seqset(ctx), scoring(ctx), job, grid, ctx->st, true, cta));
    std::vector<uint8_t> raw(bytes), out((size_t)Lc * Ls);
    CK(cudaMemcpyAsync(raw.data(), cb.p, bytes, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int i = 0; i < Lc; ++i)
      for (int j = 0; j < Ls; ++j) {
        const size_t at = code_word(i, j, Ls, G) * 8 + ((i & 15) >> 1);
        out[(size_t)i * Ls + j] = (raw[at] >> ((i & 1) * 4)) & 15;
      }
    CK(cudaMemcpyAsync(codes_out, out.data(), out.size(), cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MSA_OK;
  }();
  cleanup();
  return rc;
}

int msa_merge_gaps(msa_ctx *ctx, uint8_t *msa_out, int64_t *width_out) {
  if (!ctx || !width_out) return MSA_EINVAL;
  if (!ctx->aligned) return fail(ctx, MSA_ESTATE, "align to a center first");
  TRY(set_device(ctx));
  const int n = ctx->n, Lc = ctx->Lc;
  if (!ctx->merged) {
    TRY(ensure(ctx, ctx->G, sizeof(int32_t) * (Lc + 1)));
    TRY(ensure(ctx, ctx->off, sizeof(int32_t) * (Lc + 1)));
    stage_begin(ctx, ST_MERGE);
    CK(cudaMemsetAsync(ctx->G.p, 0, sizeof(int32_t) * (Lc + 1), ctx->st));
    CK((++ctx->launches, launch_colmax)(P<uint16_t>(ctx->ins), n, Lc, P<int32_t>(ctx->G), ctx->st));
    CK((++ctx->launches, launch_scan)(P<int32_t>(ctx->G), Lc, P<int32_t>(ctx->off), (int64_t *)(ctx->dsmall + 3), ctx->st));
    stage_end(ctx, ST_MERGE);
    long long W = 0;
    CK(cudaMemcpyAsync(&W, ctx->dsmall + 3, sizeof W, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_MERGE);
    ctx->W = W;
    TRY(ensure(ctx, ctx->msa, (size_t)n * (size_t)W));
    stage_begin(ctx, ST_ROWS);
    CK((++ctx->launches, launch_rows)(P<uint8_t>(ctx->res), P<int64_t>(ctx->d_pstart), P<int32_t>(ctx->d_inv),
                   P<uint16_t>(ctx->ins), P<uint8_t>(ctx->occ), P<int32_t>(ctx->G),
                   P<int32_t>(ctx->off), n, Lc, W, ctx->dLetters, P<uint8_t>(ctx->msa), ctx->st));
    stage_end(ctx, ST_ROWS);
    CK(cudaStreamSynchronize(ctx->st));
    stage_collect(ctx, ST_ROWS);
    ctx->merged = true;
  }
  *width_out = ctx->W;
  if (msa_out) {
    CK(cudaMemcpyAsync(msa_out, ctx->msa.p, (size_t)n * (size_t)ctx->W, cudaMemcpyDefault, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  return MSA_OK;
}

int msa_insert_maxima(msa_ctx *ctx, int32_t *G_out) {
  if (!ctx || !G_out) return MSA_EINVAL;
  if (!ctx->aligned) return fail(ctx, MSA_ESTATE, "align to a center first");
  TRY(set_device(ctx));
  const int Lc = ctx->Lc;
  TRY(ensure(ctx, ctx->G, sizeof(int32_t) * (Lc + 1)));
  CK(cudaMemsetAsync(ctx->G.p, 0, sizeof(int32_t) * (Lc + 1), ctx->st));
  CK((++ctx->launches, launch_colmax)(P<uint16_t>(ctx->ins), ctx->n, Lc, P<int32_t>(ctx->G), ctx->st));
  CK(cudaMemcpyAsync(G_out, ctx->G.p, sizeof(int32_t) * (Lc + 1), cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->merged = false;
  return MSA_OK;
}

int msa_merge_gaps_with(msa_ctx *ctx, const int32_t *G, uint8_t *msa_out, int64_t *width_out) {
  if (!ctx || !G || !width_out) return MSA_EINVAL;
  if (!ctx->aligned) return fail(ctx, MSA_ESTATE, "align to a center first");
  TRY(set_device(ctx));
  const int n = ctx->n, Lc = ctx->Lc;
  std::vector<int32_t> hg(Lc + 1), local(Lc + 1);
  CK(cudaMemcpyAsync(hg.data(), G, sizeof(int32_t) * (Lc + 1), cudaMemcpyDefault, ctx->st));
  TRY(ensure(ctx, ctx->G, sizeof(int32_t) * (Lc + 1)));
  TRY(ensure(ctx, ctx->off, sizeof(int32_t) * (Lc + 1)));
  CK(cudaMemsetAsync(ctx->G.p, 0, sizeof(int32_t) * (Lc + 1), ctx->st));
  CK((++ctx->launches, launch_colmax)(P<uint16_t>(ctx->ins), n, Lc, P<int32_t>(ctx->G), ctx->st));
  CK(cudaMemcpyAsync(local.data(), ctx->G.p, sizeof(int32_t) * (Lc + 1), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int j = 0; j <= Lc; ++j)
    if (hg[j] < local[j]) return fail(ctx, MSA_EINVAL, "G[%d] = %d is below this set's %d", j, hg[j], local[j]);
  CK(cudaMemcpyAsync(ctx->G.p, hg.data(), sizeof(int32_t) * (Lc + 1), cudaMemcpyHostToDevice, ctx->st));
  stage_begin(ctx, ST_MERGE);
  CK((++ctx->launches, launch_scan)(P<int32_t>(ctx->G), Lc, P<int32_t>(ctx->off), (int64_t *)(ctx->dsmall + 3), ctx->st));
  stage_end(ctx, ST_MERGE);
  long long W = 0;
  CK(cudaMemcpyAsync(&W, ctx->dsmall + 3, sizeof W, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->W = W;
  TRY(ensure(ctx, ctx->msa, (size_t)n * (size_t)W));
  CK((++ctx->launches, launch_rows)(P<uint8_t>(ctx->res), P<int64_t>(ctx->d_pstart), P<int32_t>(ctx->d_inv),
                                    P<uint16_t>(ctx->ins), P<uint8_t>(ctx->occ), P<int32_t>(ctx->G),
                                    P<int32_t>(ctx->off), n, Lc, W, ctx->dLetters, P<uint8_t>(ctx->msa), ctx->st));
  ctx->merged = true;
  *width_out = W;
  if (msa_out) CK(cudaMemcpyAsync(msa_out, ctx->msa.p, (size_t)n * (size_t)W, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_sp_score(msa_ctx *ctx, int64_t *sp_cost_out) {
  if (!ctx || !sp_cost_out) return MSA_EINVAL;
  if (!ctx->merged) return fail(ctx, MSA_ESTATE, "merge first");
  TRY(set_device(ctx));
  const int nsym = ctx->K + 2;
  TRY(ensure(ctx, ctx->counts, sizeof(int32_t) * nsym * (size_t)ctx->W));
  stage_begin(ctx, ST_SP);
  CK(cudaMemsetAsync(ctx->counts.p, 0, sizeof(int32_t) * nsym * (size_t)ctx->W, ctx->st));
  CK(cudaMemsetAsync(ctx->dsmall + 4, 0, sizeof(long long), ctx->st));
  CK((++ctx->launches, launch_sp)(P<uint8_t>(ctx->msa), ctx->n, ctx->W, ctx->dSymLut, nsym, P<int32_t>(ctx->counts),
               (unsigned long long *)(ctx->dsmall + 4), ctx->st));
  stage_end(ctx, ST_SP);
  long long v = 0;
  CK(cudaMemcpyAsync(&v, ctx->dsmall + 4, sizeof v, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_SP);
  *sp_cost_out = v;
  return MSA_OK;
}

int msa_autotune(msa_ctx *ctx, double *rates_out, int32_t *dims_out) {
  if (!ctx) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  TRY(set_device(ctx));
  if (ctx->smin + ctx->o < 0 || ctx->precision == MSA_INT32) {
    ctx->tune_rate.clear();  // no packed variants to time
  } else {
    TRY(autotune(ctx));
  }
  const int nb = ctx->tune_rate.empty() ? 0 : (int)ctx->tune_rate.size();
  if (dims_out) { dims_out[0] = nb; dims_out[1] = kNumCenterVariants; }
  if (rates_out)
    for (int b = 0; b < nb; ++b)
      for (int v = 0; v < kNumCenterVariants; ++v) rates_out[b * kNumCenterVariants + v] = ctx->tune_rate[b][v];
  return MSA_OK;
}

int msa_dims(msa_ctx *ctx, int64_t *dims_out) {
  if (!ctx || !dims_out) return MSA_EINVAL;
  dims_out[0] = ctx->n;
  dims_out[1] = ctx->aligned ? ctx->center : -1;
  dims_out[2] = ctx->aligned ? ctx->Lc : 0;
  dims_out[3] = ctx->merged ? ctx->W : 0;
  return MSA_OK;
}

int msa_stage_times(msa_ctx *ctx, float *ms_out, int32_t n, int64_t *counters_out) {
  if (!ctx) return MSA_EINVAL;
  for (int i = 0; i < n && i < ST_N; ++i) ms_out[i] = ctx->stage_ms[i];
  if (counters_out) {
    counters_out[0] = ctx->cells[0];
    counters_out[1] = ctx->cells[1];
    counters_out[2] = ctx->launches;
  }
  return MSA_OK;
}

int msa_memory(msa_ctx *ctx, int64_t *bytes_out, int64_t *peak_out) {
  if (!ctx) return MSA_EINVAL;
  if (bytes_out) *bytes_out = (int64_t)ctx->dev_bytes;
  if (peak_out) *peak_out = (int64_t)ctx->dev_peak;
  return MSA_OK;
}

int msa_set_memory_limit(msa_ctx *ctx, int64_t limit_bytes) {
  if (!ctx || limit_bytes < 0) return MSA_EINVAL;
  ctx->dev_limit = (size_t)limit_bytes;
  return MSA_OK;
}

int msa_align_autotune(msa_ctx *ctx, int64_t center, double *rates_out, int32_t *choice_out) {
  if (!ctx) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (center < 0 || center >= ctx->n) return fail(ctx, MSA_EINVAL, "center index out of range");
  TRY(set_device(ctx));
  const int Lc = ctx->len_sorted[ctx->inv[center]];
  ctx->align_int32 = 0;
  const bool can_pack = codes_packed(ctx, Lc);
  // the shapes are those of the full alignment
  struct ModeGuard {
    msa_ctx *c;
    int saved;
    ~ModeGuard() { c->align_mode = saved; }
  } guard{ctx, ctx->align_mode};
  ctx->align_mode = MSA_ALIGN_FULL;
  // rows: packed cells in 256-thread CTAs, int32 cells, packed cells in
  // 384-thread CTAs (groups of 8 lanes and more)
  double rates[3][kAlignWidths] = {};
  double best = -1.0;
  int best_g = 32, best_i32 = 0, best_cta = 0;
  for (int row = 0; row < 3; ++row) {
    const int i32 = row == 1 ? 1 : 0;
    if (i32 == 0 && !can_pack) continue;
    for (int gi = 0; gi < kAlignWidths; ++gi) {
      const int G = 1 << gi;
      if (row == 2 && G < 8) continue;
      ctx->align_int32 = i32;
      ctx->align_group = G;
      ctx->align_threads = row == 2 ? kCodes2WideThreads : 0;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the second run is timed
        TRY(msa_align_to_center(ctx, center, nullptr));
        ms = ctx->stage_ms[ST_ALIGN_K] + ctx->stage_ms[ST_TRACE];
      }
      const double r = ms > 0.f ? (double)ctx->cells[1] / (ms * 1e-3) : 0.0;
      rates[row][gi] = r;
      if (r > best) { best = r; best_g = G; best_i32 = i32; best_cta = ctx->align_threads; }
    }
  }
  ctx->align_group = best_g;
  ctx->align_int32 = best_i32;
  ctx->align_threads = best_cta;
  ctx->aligned = false;
  if (rates_out) memcpy(rates_out, rates, sizeof rates);
  if (choice_out) {
    choice_out[0] = best_g;
    choice_out[1] = best_i32 ? 0 : 1;
    choice_out[2] = align_cta(ctx, best_g, !best_i32);
  }
  return MSA_OK;
}

int msa_set_align_threads(msa_ctx *ctx, int32_t threads) {
  if (!ctx || (threads != 0 && threads != kCodes2Threads && threads != kCodes2WideThreads))
    return MSA_EINVAL;
  ctx->align_threads = threads == kCodes2Threads ? 0 : threads;
  return MSA_OK;
}

int msa_set_align_group(msa_ctx *ctx, int32_t lanes) {
  if (!ctx || lanes < 0 || lanes > 32 || (lanes & (lanes - 1)) != 0) return MSA_EINVAL;
  ctx->align_group = lanes;
  ctx->align_group_fixed = lanes > 0;
  return MSA_OK;
}

int msa_set_align_mode(msa_ctx *ctx, int32_t mode) {
  if (!ctx || (mode != MSA_ALIGN_FULL && mode != MSA_ALIGN_BOX)) return MSA_EINVAL;
  ctx->align_mode = mode;
  return MSA_OK;
}

int msa_align_boxes(msa_ctx *ctx, int32_t *box_out) {
  if (!ctx || !box_out) return MSA_EINVAL;
  if (!ctx->aligned || !ctx->light_used) return fail(ctx, MSA_ESTATE, "no alignment in MSA_ALIGN_BOX mode");
  TRY(set_device(ctx));
  CK(cudaMemcpyAsync(box_out, ctx->h_boxes.data(), sizeof(int32_t) * ctx->h_boxes.size(), cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_set_codes_budget(msa_ctx *ctx, int64_t bytes) {
  if (!ctx || bytes < 1) return MSA_EINVAL;
  ctx->codes_budget = (size_t)bytes;
  return MSA_OK;
}

}  // extern "C"
