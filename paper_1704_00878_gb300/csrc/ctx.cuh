// ctx.cuh -- the context behind the C ABI and the host helpers shared by
// its translation units (msa_api.cu, selector.cu).  Private to the library.
#pragma once
#include <string>
#include <vector>

#include "msa.h"
#include "msa_kernels.cuh"
#include "sw_kernels.cuh"

namespace msa_detail {

struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};

enum Stage {
  ST_ENCODE = 0, ST_CENTER, ST_ALIGN, ST_TRACE, ST_MERGE, ST_ROWS, ST_SP, ST_CENTER_K, ST_ALIGN_K,
  ST_SELECTOR, ST_TREE, ST_LIGHT_SCORE, ST_LIGHT_CORNER, ST_LIGHT_BOX, ST_N
};

struct Selector;  // the learned center selector (selector.cu)
constexpr int kMaxTreeRows = 65536;  // rows of a neighbour-joining tree
void selector_free(msa_ctx *ctx, Selector *s);

}  // namespace msa_detail

struct msa_ctx {
  using DevBuf = msa_detail::DevBuf;
  int dev = 0;
  cudaStream_t st = nullptr;
  int K = 0, o = 0, e = 0, precision = MSA_AUTO, sat_limit = 32767, smax = 0, smin = 0;
  std::vector<int8_t> hM;
  std::string letters;
  uint8_t hlut[256];
  std::string err;

  // scoring tables on the device
  int8_t *dM = nullptr;
  char *dLetters = nullptr;
  uint8_t *dLut = nullptr, *dSymLut = nullptr;

  // the loaded set (sorted by length, ascending, stable)
  int n = 0, maxlen = 0;
  std::vector<int32_t> len_sorted, perm, inv;
  std::vector<int64_t> pstart;
  // host scratch kept between calls (a fresh multi-megabyte vector per call
  // pays its page faults every time)
  std::vector<int32_t> h_lens;
  std::vector<int64_t> h_offs;
  DevBuf res, d_pstart, d_len, d_perm, d_inv, d_srcoff, staging;

  // center selection
  DevBuf pairsum, self, rowsum, prefix, qlist, ovf, ovf_scores, ovf_dst, part_val, part_idx,
      pairs, pair_dst, pair_out, counters, streams;
  cudaStream_t cap_st = nullptr;  // private streams the center graph is captured on
  cudaStream_t cap_st2 = nullptr;
  cudaEvent_t cap_fork = nullptr, cap_join = nullptr;
  cudaGraphExec_t center_exec = nullptr;  // the last center graph and what it bakes in
  std::vector<int64_t> center_key;
  cudaGraphExec_t align_exec = nullptr;   // the last alignment graph and what it bakes in
  std::vector<int64_t> align_key;
  std::vector<cudaEvent_t> align_ev;      // per code batch: fill start/end, traceback end
  bool have_rowsum = false;

  // alignment
  int64_t center = -1;
  int Lc = 0;
  DevBuf ins, occ, seg, score, codes, code_off, best;
  bool aligned = false;

  // merge
  DevBuf G, off, msa, counts;
  int64_t W = 0;
  bool merged = false;

  // small device scalars
  unsigned long long *dcounter = nullptr;
  unsigned *derr = nullptr;     // derr[0] error bits, derr[1] overflow count
  long long *dsmall = nullptr;  // [0] total, [1] argmin val, [2] argmin idx, [3] width, [4] sp
  DevBuf scratch;
  size_t scratch_half = 0;  // int2 offset of the second stream's boundary rows (center graph)

  cudaEvent_t ev[2 * msa_detail::ST_N] = {};
  float stage_ms[msa_detail::ST_N] = {};
  int64_t cells[2] = {0, 0};
  int64_t launches = 0;
  // device memory held through ensure(): current, peak, optional cap (0 = none)
  size_t dev_bytes = 0, dev_peak = 0, dev_limit = 0;
  // traceback codes held at once (0.5 B per cell): the alignment runs in
  // batches of subjects whose codes fit; a batch should fill the GPU many
  // times over, and the traceback of each batch waits for its fill
  size_t codes_budget = (size_t)32 << 30;
  int align_group = 0;  // lanes per subject group of the codes kernels, 0 = modelled choice
  bool align_group_fixed = false;  // set by msa_set_align_group: every light pass uses it too
  int align_int32 = 0;  // 1: the alignment uses int32 cells even where packed ones fit
  int align_threads = 0;  // CTA size of the packed codes kernel, 0 = kCodes2Threads
  // traceback-light alignment (MSA_ALIGN_BOX): per position of its passes the
  // subject, its window and the pass's best-cell keys; per sequence (input
  // order) the box of its last light alignment
  int align_mode = MSA_ALIGN_FULL;
  bool light_used = false;
  DevBuf light_order, light_win, light_keys;
  void *pinned = nullptr;  // pinned host staging of the light passes' round trips
  size_t pinned_cap = 0;
  std::vector<int4> h_win, h_box;
  std::vector<int32_t> h_boxes, h_items, h_all;

  msa_detail::Selector *sel = nullptr;

  // autotuner: measured cells/s of each center variant per query-length bucket
  std::vector<int> tune_edges;                 // bucket b = [edges[b], edges[b+1])
  std::vector<std::vector<double>> tune_rate;  // [bucket][variant], 0 = not measured
  std::vector<std::vector<double>> tune_corr;  // [bucket][variant]: measured / modelled rate
};

namespace msa_detail {

int fail(msa_ctx *c, int code, const char *fmt, ...);
int ensure(msa_ctx *ctx, DevBuf &b, size_t bytes);
void release(msa_ctx *ctx, DevBuf &b);  // frees a buffer taken with ensure()
template <class T> T *P(DevBuf &b) { return reinterpret_cast<T *>(b.p); }
bool is_device_ptr(const void *p);
int set_device(msa_ctx *ctx);
void stage_begin(msa_ctx *ctx, int s);
void stage_end(msa_ctx *ctx, int s);
void stage_collect(msa_ctx *ctx, int s);
SeqSet seqset(msa_ctx *ctx);
Scoring scoring(msa_ctx *ctx);
int run_pairs(msa_ctx *ctx, const std::vector<int2> &pairs_in, const std::vector<int32_t> &dst_in,
              int32_t *d_out);
int selector_center(msa_ctx *ctx, int64_t *center_out);
// refs: ascending sorted positions of a reference sample, empty = every sequence
int selector_center_refined(msa_ctx *ctx, int k, const std::vector<int32_t> &refs,
                            int64_t *center_out, int64_t *sum_out);
// A subset of the loaded set with indices of its own: entry v is the loaded
// sequence at sorted position idx[v] (device starts and lengths in ss); the
// center planner and kernels see only the view, its first n_sub entries being
// the subjects.  Entries ascend in length within the subjects and within the
// queries.
struct SetView {
  SeqSet ss;
  std::vector<int32_t> idx, len;
  int n_sub = 0;
  const int32_t *self = nullptr;  // device: S(v, v) of every view entry
};
int run_center(msa_ctx *ctx, int mode, const std::vector<int32_t> &qsorted,
               const SetView *view = nullptr, int q_begin = 0, int q_end = -1);
// the device error word -> an MSA_E* code (synchronises the stream)
int check_derr(msa_ctx *ctx);
// cell precision and lanes per group of the alignment to a center of length Lc
bool align_packed(msa_ctx *ctx, int Lc);
int align_lanes(msa_ctx *ctx, int Lc, bool packed);
// CTA size of the codes kernel for this group width and precision
int align_cta(msa_ctx *ctx, int G, bool packed);
SeqSet seqset(msa_ctx *ctx);
Scoring scoring(msa_ctx *ctx);

}  // namespace msa_detail

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return msa_detail::fail(ctx, e_ == cudaErrorMemoryAllocation ? MSA_ENOMEM : MSA_ECUDA, \
                              "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)                \
  do {                           \
    int r_ = (expr);             \
    if (r_ != MSA_OK) return r_; \
  } while (0)
