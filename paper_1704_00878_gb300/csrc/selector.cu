// selector.cu -- the learned center selector behind the C ABI: a 1-D conv
// embedding network whose squared embedding distances are trained on scaled
// exact-center distances d(A,B) = 2^16 - floor(2^16 S(A,B) / max(S(A,A),
// S(B,B))) from the scores the exact Smith-Waterman kernel produces, then used
// to pick the center in O(n):
// argmin of ||e_i - mean(e)||^2, which equals argmin of sum_j ||e_i - e_j||^2,
// the embedding stand-in for the exact center's argmin of sum_j d(i,j).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "ctx.cuh"
#include "net_kernels.cuh"

namespace msa_detail {

typedef __nv_bfloat16 bf16;

struct Selector {
  DevBuf params, grads, m, v;                      // fp32, net::N_PARAMS each
  DevBuf w1t, w2t, w2n, w3t, w3n, w4t, w4n;        // bf16 weight copies
  int step = 0;
  // batch buffers
  DevBuf seq, base, len, rowseq, x0, a1, a2, a3, pw, yw, emb, demb, dy4, dz3, dz2, dz1;
  DevBuf bpairs, btargets, loss, small, allemb, dist;
  DevBuf vstart, vlen, vself;  // a reference/candidate view of the loaded set
};

namespace {


// splitmix64 (Steele, Lea & Flood 2014) as a counter-based generator.
uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}
double unit(uint64_t seed, uint64_t i) {
  return (double)(splitmix64(seed * 0x9e3779b97f4a7c15ull + i) >> 11) * (1.0 / 9007199254740992.0);
}

// He-uniform weights (bound sqrt(6 / fan_in)) for the ReLU layers, bound
// sqrt(3 / fan_in) for the linear last layer, zero biases; the one-hot
// channels beyond the alphabet stay zero.
std::vector<float> default_params(uint64_t seed, int K) {
  std::vector<float> p(net::N_PARAMS, 0.f);
  uint64_t c = 0;
  auto fill = [&](size_t off, int cin, int cout, int fan_in, double gain) {
    const double a = std::sqrt(gain / fan_in);
    for (int t = 0; t < net::TAPS; ++t)
      for (int ci = 0; ci < cin; ++ci)
        for (int co = 0; co < cout; ++co) {
          const size_t at = off + ((size_t)t * cin + ci) * cout + co;
          const double u = unit(seed, c++);
          p[at] = (cin == net::KP && ci >= K) ? 0.f : (float)((2.0 * u - 1.0) * a);
        }
  };
  fill(net::W1_OFF, net::KP, net::WD, net::TAPS * K, 6.0);
  fill(net::W2_OFF, net::WD, net::WD, net::TAPS * net::WD, 6.0);
  fill(net::W3_OFF, net::WD, net::WD, net::TAPS * net::WD, 6.0);
  fill(net::W4_OFF, net::WD, net::DIM, net::TAPS * net::WD, 3.0);
  return p;
}

int sel_get(msa_ctx *ctx, Selector **out) {
  if (!ctx->sel) {
    ctx->sel = new (std::nothrow) Selector;
    if (!ctx->sel) return fail(ctx, MSA_ENOMEM, "selector allocation failed");
  }
  *out = ctx->sel;
  return MSA_OK;
}

int refresh_all(msa_ctx *ctx, Selector *s) {
  float *p = P<float>(s->params);
  CK((++ctx->launches, net::refresh)(p + net::W1_OFF, net::KP, net::WD, P<bf16>(s->w1t), nullptr, ctx->st));
  CK((++ctx->launches, net::refresh)(p + net::W2_OFF, net::WD, net::WD, P<bf16>(s->w2t), P<bf16>(s->w2n), ctx->st));
  CK((++ctx->launches, net::refresh)(p + net::W3_OFF, net::WD, net::WD, P<bf16>(s->w3t), P<bf16>(s->w3n), ctx->st));
  CK((++ctx->launches, net::refresh)(p + net::W4_OFF, net::WD, net::DIM, P<bf16>(s->w4t), P<bf16>(s->w4n), ctx->st));
  return MSA_OK;
}

int set_params(msa_ctx *ctx, Selector *s, const float *host) {
  const size_t bytes = sizeof(float) * net::N_PARAMS;
  TRY(ensure(ctx, s->params, bytes));
  TRY(ensure(ctx, s->grads, bytes));
  TRY(ensure(ctx, s->m, bytes));
  TRY(ensure(ctx, s->v, bytes));
  TRY(ensure(ctx, s->w1t, sizeof(bf16) * net::W1_N));
  TRY(ensure(ctx, s->w2t, sizeof(bf16) * net::W2_N));
  TRY(ensure(ctx, s->w2n, sizeof(bf16) * net::W2_N));
  TRY(ensure(ctx, s->w3t, sizeof(bf16) * net::W3_N));
  TRY(ensure(ctx, s->w3n, sizeof(bf16) * net::W3_N));
  TRY(ensure(ctx, s->w4t, sizeof(bf16) * net::W4_N));
  TRY(ensure(ctx, s->w4n, sizeof(bf16) * net::W4_N));
  TRY(ensure(ctx, s->small, 1024));
  TRY(ensure(ctx, s->loss, sizeof(float)));
  CK(cudaMemcpyAsync(s->params.p, host, bytes, cudaMemcpyDefault, ctx->st));
  CK(cudaMemsetAsync(s->m.p, 0, bytes, ctx->st));
  CK(cudaMemsetAsync(s->v.p, 0, bytes, ctx->st));
  s->step = 0;
  return refresh_all(ctx, s);
}

// Lay out the listed sequences (sorted indices) as one flat batch and build
// its one-hot input.
int build_batch(msa_ctx *ctx, Selector *s, const std::vector<int32_t> &seqs, net::Batch &b) {
  const int ns = (int)seqs.size();
  std::vector<int32_t> base(ns), len(ns);
  int64_t row = net::HALF;
  for (int i = 0; i < ns; ++i) {
    base[i] = (int32_t)row;
    len[i] = ctx->len_sorted[seqs[i]];
    row += len[i] + net::HALF;
  }
  if (row > INT32_MAX / 2) return fail(ctx, MSA_ERANGE, "selector batch too large");
  const int T = (int)row;
  TRY(ensure(ctx, s->seq, sizeof(int32_t) * ns));
  TRY(ensure(ctx, s->base, sizeof(int32_t) * ns));
  TRY(ensure(ctx, s->len, sizeof(int32_t) * ns));
  TRY(ensure(ctx, s->rowseq, sizeof(int32_t) * T));
  TRY(ensure(ctx, s->x0, sizeof(bf16) * (size_t)T * net::KP));
  TRY(ensure(ctx, s->a1, sizeof(bf16) * (size_t)T * net::WD));
  TRY(ensure(ctx, s->a2, sizeof(bf16) * (size_t)T * net::WD));
  TRY(ensure(ctx, s->a3, sizeof(bf16) * (size_t)T * net::WD));
  TRY(ensure(ctx, s->pw, sizeof(bf16) * (size_t)net::TAPS * ns * net::WD));
  TRY(ensure(ctx, s->yw, sizeof(float) * (size_t)net::TAPS * ns * net::DIM));
  TRY(ensure(ctx, s->emb, sizeof(float) * (size_t)ns * net::DIM));
  CK(cudaMemcpyAsync(s->seq.p, seqs.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(s->base.p, base.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(s->len.p, len.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, ctx->st));
  b.nseq = ns;
  b.T = T;
  b.seq = P<int32_t>(s->seq);
  b.base = P<int32_t>(s->base);
  b.len = P<int32_t>(s->len);
  b.rowseq = P<int32_t>(s->rowseq);
  CK((++ctx->launches, net::fill_rows)(b, ctx->st));
  CK((++ctx->launches, net::onehot)(b, P<uint8_t>(ctx->res), P<int64_t>(ctx->d_pstart), P<bf16>(s->x0), ctx->st));
  // the stream orders the small host arrays' copies before their use; keep
  // them alive until then
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

// One weight gradient / convolution on the tensor cores (every shape of the
// network has its tcgen05 kernel).
cudaError_t wgrad(msa_ctx *ctx, int cin, int cout, const bf16 *x, const bf16 *dy, float *dw, int T) {
  ++ctx->launches;
  return net::wgrad_tc(cin, cout, x, dy, dw, T, ctx->derr, ctx->st);
}

cudaError_t conv(msa_ctx *ctx, int cin, int cout, int mode, const bf16 *x, const bf16 *w,
                 const float *bias, const int32_t *rowseq, const bf16 *prev, void *y, int T) {
  ++ctx->launches;
  return net::conv_tc(cin, cout, mode, x, w, bias, rowseq, prev, y, T, ctx->derr, ctx->st);
}

int forward(msa_ctx *ctx, Selector *s, const net::Batch &b) {
  const float *p = P<float>(s->params);
  const int T = b.T;
  CK(conv(ctx, net::KP, net::WD, 0, P<bf16>(s->x0), P<bf16>(s->w1t), p + net::B1_OFF, b.rowseq, nullptr, s->a1.p, T));
  CK(conv(ctx, net::WD, net::WD, 0, P<bf16>(s->a1), P<bf16>(s->w2t), p + net::B2_OFF, b.rowseq, nullptr, s->a2.p, T));
  CK(conv(ctx, net::WD, net::WD, 0, P<bf16>(s->a2), P<bf16>(s->w3t), p + net::B3_OFF, b.rowseq, nullptr, s->a3.p, T));
  // output layer and pooling: the output convolution runs on the nine
  // window sums of each sequence instead of on every row
  CK((++ctx->launches, net::window_sums)(b, P<bf16>(s->a3), P<bf16>(s->pw), ctx->st));
  CK(conv(ctx, net::WD, net::DIM, 1, P<bf16>(s->pw), P<bf16>(s->w4t), p + net::B4_OFF, nullptr, nullptr,
          s->yw.p, net::TAPS * b.nseq));
  CK((++ctx->launches, net::emb_from_windows)(b, P<float>(s->yw), p + net::B4_OFF, P<float>(s->emb), ctx->st));
  return MSA_OK;
}

// Loss of the listed (batch-local) pairs and the gradient of every parameter.
int forward_backward(msa_ctx *ctx, Selector *s, const net::Batch &b, int npairs) {
  const int T = b.T;
  TRY(ensure(ctx, s->demb, sizeof(float) * (size_t)b.nseq * net::DIM));
  TRY(ensure(ctx, s->dy4, sizeof(bf16) * (size_t)T * net::DIM));
  TRY(ensure(ctx, s->dz3, sizeof(bf16) * (size_t)T * net::WD));
  TRY(ensure(ctx, s->dz2, sizeof(bf16) * (size_t)T * net::WD));
  TRY(ensure(ctx, s->dz1, sizeof(bf16) * (size_t)T * net::WD));
  TRY(forward(ctx, s, b));
  float *g = P<float>(s->grads);
  CK(cudaMemsetAsync(g, 0, sizeof(float) * net::N_PARAMS, ctx->st));
  CK(cudaMemsetAsync(s->demb.p, 0, sizeof(float) * (size_t)b.nseq * net::DIM, ctx->st));
  CK(cudaMemsetAsync(s->loss.p, 0, sizeof(float), ctx->st));
  CK((++ctx->launches, net::pair_loss)(P<int2>(s->bpairs), P<float>(s->btargets), npairs, P<float>(s->emb), P<float>(s->demb), P<float>(s->loss), ctx->st));
  CK((++ctx->launches, net::pool_backward)(b, P<float>(s->demb), P<bf16>(s->dy4), ctx->st));
  // layer 4 (linear)
  CK(wgrad(ctx, net::WD, net::DIM, P<bf16>(s->a3), P<bf16>(s->dy4), g + net::W4_OFF, T));
  CK((++ctx->launches, net::colsum)(net::DIM, P<bf16>(s->dy4), g + net::B4_OFF, T, ctx->st));
  CK(conv(ctx, net::DIM, net::WD, 2, P<bf16>(s->dy4), P<bf16>(s->w4n), nullptr, b.rowseq, P<bf16>(s->a3), s->dz3.p, T));
  // layer 3
  CK(wgrad(ctx, net::WD, net::WD, P<bf16>(s->a2), P<bf16>(s->dz3), g + net::W3_OFF, T));
  CK((++ctx->launches, net::colsum)(net::WD, P<bf16>(s->dz3), g + net::B3_OFF, T, ctx->st));
  CK(conv(ctx, net::WD, net::WD, 2, P<bf16>(s->dz3), P<bf16>(s->w3n), nullptr, b.rowseq, P<bf16>(s->a2), s->dz2.p, T));
  // layer 2
  CK(wgrad(ctx, net::WD, net::WD, P<bf16>(s->a1), P<bf16>(s->dz2), g + net::W2_OFF, T));
  CK((++ctx->launches, net::colsum)(net::WD, P<bf16>(s->dz2), g + net::B2_OFF, T, ctx->st));
  CK(conv(ctx, net::WD, net::WD, 2, P<bf16>(s->dz2), P<bf16>(s->w2n), nullptr, b.rowseq, P<bf16>(s->a1), s->dz1.p, T));
  // layer 1 (one-hot input: no data gradient)
  CK(wgrad(ctx, net::KP, net::WD, P<bf16>(s->x0), P<bf16>(s->dz1), g + net::W1_OFF, T));
  CK((++ctx->launches, net::colsum)(net::WD, P<bf16>(s->dz1), g + net::B1_OFF, T, ctx->st));
  return MSA_OK;
}

// Batch of pairs (input indices) -> unique batch sequences and local pairs.
int stage_pairs(msa_ctx *ctx, Selector *s, const int64_t *pairs, const float *targets, int64_t np,
                net::Batch &b) {
  std::unordered_map<int32_t, int32_t> local;
  std::vector<int32_t> seqs;
  std::vector<int2> lp(np);
  for (int64_t x = 0; x < np; ++x) {
    int32_t ids[2];
    for (int h = 0; h < 2; ++h) {
      const int64_t t = pairs[2 * x + h];
      if (t < 0 || t >= ctx->n) return fail(ctx, MSA_EINVAL, "pair index out of range");
      const int32_t k = ctx->inv[t];
      auto it = local.find(k);
      if (it == local.end()) {
        it = local.emplace(k, (int32_t)seqs.size()).first;
        seqs.push_back(k);
      }
      ids[h] = it->second;
    }
    lp[x] = make_int2(ids[0], ids[1]);
  }
  TRY(ensure(ctx, s->bpairs, sizeof(int2) * np));
  TRY(ensure(ctx, s->btargets, sizeof(float) * np));
  CK(cudaMemcpyAsync(s->bpairs.p, lp.data(), sizeof(int2) * np, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(s->btargets.p, targets, sizeof(float) * np, cudaMemcpyHostToDevice, ctx->st));
  return build_batch(ctx, s, seqs, b);  // synchronises before the host vectors go away
}

// The exact center's distance of a pair in units of 2^-16 (the kernels' sums
// add 2^16 - center_sim of the same scores).
long long center_distance(int sab, int saa, int sbb) {
  const long long m = std::max(saa, sbb);
  return m > 0 ? 65536 - ((long long)sab * 65536) / m : 0;
}

// Scaled exact distances t = scale * d(a, b).
int exact_targets(msa_ctx *ctx, const int64_t *pairs, int64_t np, float scale,
                  std::vector<float> &t) {
  std::vector<int2> pr;
  std::vector<int32_t> dst;
  std::unordered_map<int32_t, int32_t> selfslot;
  pr.reserve(np + 2 * np);
  for (int64_t x = 0; x < np; ++x) {
    const int64_t a = pairs[2 * x], b = pairs[2 * x + 1];
    if (a < 0 || b < 0 || a >= ctx->n || b >= ctx->n) return fail(ctx, MSA_EINVAL, "pair index out of range");
    pr.push_back(make_int2(ctx->inv[a], ctx->inv[b]));
    dst.push_back((int32_t)x);
  }
  for (int64_t x = 0; x < np; ++x)
    for (int h = 0; h < 2; ++h) {
      const int32_t k = ctx->inv[pairs[2 * x + h]];
      if (selfslot.count(k)) continue;
      selfslot[k] = (int32_t)(np + selfslot.size());
      pr.push_back(make_int2(k, k));
      dst.push_back(selfslot[k]);
    }
  const size_t total = pr.size();
  TRY(ensure(ctx, ctx->pair_out, sizeof(int32_t) * total));
  TRY(run_pairs(ctx, pr, dst, P<int32_t>(ctx->pair_out)));
  std::vector<int32_t> S(total);
  CK(cudaMemcpyAsync(S.data(), ctx->pair_out.p, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  t.resize(np);
  for (int64_t x = 0; x < np; ++x) {
    const int saa = S[selfslot[ctx->inv[pairs[2 * x]]]];
    const int sbb = S[selfslot[ctx->inv[pairs[2 * x + 1]]]];
    t[x] = (float)(scale * (double)center_distance(S[x], saa, sbb));
  }
  return MSA_OK;
}

// Embeddings of every loaded sequence, in sorted order, into s->allemb.
int embed_all(msa_ctx *ctx, Selector *s) {
  const int n = ctx->n;
  TRY(ensure(ctx, s->allemb, sizeof(float) * (size_t)n * net::DIM));
  const int64_t max_rows = (int64_t)1 << 23;  // ~1.1 KB of activations per row
  int k = 0;
  while (k < n) {
    std::vector<int32_t> seqs;
    int64_t rows = net::HALF;
    while (k < n && (seqs.empty() || rows + ctx->len_sorted[k] + net::HALF <= max_rows)) {
      rows += ctx->len_sorted[k] + net::HALF;
      seqs.push_back(k++);
    }
    net::Batch b;
    TRY(build_batch(ctx, s, seqs, b));
    TRY(forward(ctx, s, b));
    CK(cudaMemcpyAsync(P<float>(s->allemb) + (size_t)seqs.front() * net::DIM, s->emb.p,
                       sizeof(float) * seqs.size() * net::DIM, cudaMemcpyDeviceToDevice, ctx->st));
  }
  return MSA_OK;
}

}  // namespace

void selector_free(msa_ctx *ctx, Selector *s) {
  if (!s) return;
  DevBuf *bufs[] = {&s->params, &s->grads, &s->m, &s->v, &s->w1t, &s->w2t, &s->w2n, &s->w3t,
                    &s->w3n, &s->w4t, &s->w4n, &s->seq, &s->base, &s->len, &s->rowseq, &s->x0,
                    &s->a1, &s->a2, &s->a3, &s->pw, &s->yw, &s->emb, &s->demb, &s->dy4, &s->dz3,
                    &s->dz2, &s->dz1, &s->bpairs, &s->btargets, &s->loss, &s->small, &s->allemb,
                    &s->dist, &s->vstart, &s->vlen, &s->vself};
  for (DevBuf *b : bufs) release(ctx, *b);
  delete s;
}

// LEARNED center: argmin over the embeddings of ||e_i - mean(e)||^2.
int selector_center(msa_ctx *ctx, int64_t *center_out) {
  Selector *s = ctx->sel;
  if (!s || !s->params.p) return fail(ctx, MSA_ESTATE, "no trained selector loaded");
  stage_begin(ctx, ST_SELECTOR);
  TRY(embed_all(ctx, s));
  CK((++ctx->launches, net::emb_center)(P<float>(s->allemb), ctx->n, P<float>(s->small),
                                        reinterpret_cast<long long *>(P<char>(s->small) + 768), ctx->st));
  stage_end(ctx, ST_SELECTOR);
  long long k = 0;
  CK(cudaMemcpyAsync(&k, P<char>(s->small) + 768, sizeof k, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_SELECTOR);
  TRY(check_derr(ctx));
  if (k < 0 || k >= ctx->n) return fail(ctx, MSA_ECUDA, "selector center out of range");
  *center_out = ctx->perm[k];
  return MSA_OK;
}

// LEARNED_REFINED: the k candidates with the smallest ||e_i - mean(e)||^2,
// then their exact row sums sum_j d(i, j) and the argmin among them (lowest
// input index on ties).  refs (ascending sorted positions) empty: j runs over
// every sequence (k x n alignments with the center kernels, summed on the
// query side); else j runs over refs, the EXACT_SAMPLED row sum, computed as
// k x |refs| alignments over a view whose subjects are the references and
// whose queries are the candidates.
int selector_center_refined(msa_ctx *ctx, int k, const std::vector<int32_t> &refs,
                            int64_t *center_out, int64_t *sum_out) {
  Selector *s = ctx->sel;
  if (!s || !s->params.p) return fail(ctx, MSA_ESTATE, "no trained selector loaded");
  const int n = ctx->n;
  k = std::max(1, std::min(k, n));
  stage_begin(ctx, ST_SELECTOR);
  TRY(embed_all(ctx, s));
  TRY(ensure(ctx, s->dist, sizeof(float) * n));
  CK((++ctx->launches, net::emb_dist)(P<float>(s->allemb), n, P<float>(s->small), P<float>(s->dist), ctx->st));
  stage_end(ctx, ST_SELECTOR);
  std::vector<float> dist(n);
  CK(cudaMemcpyAsync(dist.data(), s->dist.p, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_SELECTOR);
  TRY(check_derr(ctx));
  // the k smallest distances (a total order: ties by input index), as a set
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  if (k < n)
    std::nth_element(idx.begin(), idx.begin() + (k - 1), idx.end(), [&](int32_t a, int32_t b) {
      return dist[a] < dist[b] || (dist[a] == dist[b] && ctx->perm[a] < ctx->perm[b]);
    });
  std::vector<int32_t> qs(idx.begin(), idx.begin() + k);
  std::sort(qs.begin(), qs.end());
  stage_begin(ctx, ST_CENTER);
  CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
  std::vector<unsigned long long> ps(k);  // sum_j center_sim(q, j) per candidate
  if (refs.empty()) {
    // self scores of every sequence (every candidate meets every sequence)
    std::vector<int2> sp(n);
    std::vector<int32_t> dst(n);
    for (int x = 0; x < n; ++x) { sp[x] = make_int2(x, x); dst[x] = x; }
    TRY(run_pairs(ctx, sp, dst, P<int32_t>(ctx->self)));
    CK(cudaMemsetAsync(ctx->pairsum.p, 0, sizeof(unsigned long long) * n, ctx->st));
    TRY(run_center(ctx, 2, qs));
    stage_end(ctx, ST_CENTER);
    std::vector<unsigned long long> all(n);
    CK(cudaMemcpyAsync(all.data(), ctx->pairsum.p, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int c = 0; c < k; ++c) ps[c] = all[qs[c]];
  } else {
    const int R = (int)refs.size();
    SetView view;
    view.idx = refs;
    view.idx.insert(view.idx.end(), qs.begin(), qs.end());
    view.n_sub = R;
    const int nv = (int)view.idx.size();
    std::vector<int64_t> vstart(nv);
    view.len.resize(nv);
    for (int v = 0; v < nv; ++v) {
      vstart[v] = ctx->pstart[view.idx[v]];
      view.len[v] = ctx->len_sorted[view.idx[v]];
    }
    TRY(ensure(ctx, s->vstart, sizeof(int64_t) * nv));
    TRY(ensure(ctx, s->vlen, sizeof(int32_t) * nv));
    TRY(ensure(ctx, s->vself, sizeof(int32_t) * nv));
    TRY(ensure(ctx, ctx->pairsum, sizeof(unsigned long long) * std::max(n, nv)));
    CK(cudaMemcpyAsync(s->vstart.p, vstart.data(), sizeof(int64_t) * nv, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(s->vlen.p, view.len.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, ctx->st));
    // self scores of the view's entries (references, then candidates)
    std::vector<int2> sp(nv);
    std::vector<int32_t> dst(nv);
    for (int v = 0; v < nv; ++v) { sp[v] = make_int2(view.idx[v], view.idx[v]); dst[v] = v; }
    TRY(run_pairs(ctx, sp, dst, P<int32_t>(s->vself)));
    CK(cudaMemsetAsync(ctx->pairsum.p, 0, sizeof(unsigned long long) * nv, ctx->st));
    view.ss = SeqSet{P<uint8_t>(ctx->res), P<int64_t>(s->vstart), P<int32_t>(s->vlen), nv};
    view.self = P<int32_t>(s->vself);
    std::vector<int32_t> vq(k);
    std::iota(vq.begin(), vq.end(), R);
    TRY(run_center(ctx, 2, vq, &view));
    stage_end(ctx, ST_CENTER);
    CK(cudaMemcpyAsync(ps.data(), P<unsigned long long>(ctx->pairsum) + R,
                       sizeof(unsigned long long) * k, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  stage_collect(ctx, ST_CENTER);
  // sum_j d(q, j) = |J| 2^16 - sum_j center_sim(q, j) (the candidate meets itself
  // among the j when it is one of them: similarity 2^16, distance 0)
  const long long nj = refs.empty() ? n : (long long)refs.size();
  long long best = 0;
  int bestq = -1;
  for (int c = 0; c < k; ++c) {
    const int q = qs[c];
    const long long v = nj * 65536 - (long long)ps[c];
    if (bestq < 0 || v < best || (v == best && ctx->perm[q] < ctx->perm[bestq])) { best = v; bestq = q; }
  }
  *center_out = ctx->perm[bestq];
  if (sum_out) *sum_out = best;
  return check_derr(ctx);
}

}  // namespace msa_detail

using namespace msa_detail;

extern "C" {

int msa_selector_init(msa_ctx *ctx, uint64_t seed, const float *params, int64_t count) {
  if (!ctx) return MSA_EINVAL;
  if (params && count != (int64_t)net::N_PARAMS)
    return fail(ctx, MSA_EINVAL, "expected %lld parameters", (long long)net::N_PARAMS);
  TRY(set_device(ctx));
  Selector *s = nullptr;
  TRY(sel_get(ctx, &s));
  std::vector<float> host;
  if (!params) {
    host = default_params(seed, ctx->K);
    params = host.data();
  }
  TRY(set_params(ctx, s, params));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_selector_params(msa_ctx *ctx, float *params_out, int64_t *count_out) {
  if (!ctx) return MSA_EINVAL;
  if (count_out) *count_out = (int64_t)net::N_PARAMS;
  if (!params_out) return MSA_OK;
  if (!ctx->sel || !ctx->sel->params.p) return fail(ctx, MSA_ESTATE, "no selector");
  TRY(set_device(ctx));
  CK(cudaMemcpyAsync(params_out, ctx->sel->params.p, sizeof(float) * net::N_PARAMS, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_selector_targets(msa_ctx *ctx, const int64_t *pairs, int64_t npairs, float scale,
                         float *targets_out) {
  if (!ctx || (npairs > 0 && (!pairs || !targets_out)) || npairs < 0) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (npairs == 0) return MSA_OK;
  TRY(set_device(ctx));
  std::vector<float> t;
  TRY(exact_targets(ctx, pairs, npairs, scale, t));
  CK(cudaMemcpyAsync(targets_out, t.data(), sizeof(float) * npairs, cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return MSA_OK;
}

int msa_selector_grad(msa_ctx *ctx, const int64_t *pairs, const float *targets, int64_t npairs,
                      float *grad_out, float *loss_out) {
  if (!ctx || !pairs || !targets || npairs < 1) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (!ctx->sel || !ctx->sel->params.p) return fail(ctx, MSA_ESTATE, "no selector");
  TRY(set_device(ctx));
  Selector *s = ctx->sel;
  net::Batch b;
  TRY(stage_pairs(ctx, s, pairs, targets, npairs, b));
  TRY(forward_backward(ctx, s, b, (int)npairs));
  if (grad_out)
    CK(cudaMemcpyAsync(grad_out, s->grads.p, sizeof(float) * net::N_PARAMS, cudaMemcpyDefault, ctx->st));
  if (loss_out) CK(cudaMemcpyAsync(loss_out, s->loss.p, sizeof(float), cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return check_derr(ctx);
}

int msa_selector_train(msa_ctx *ctx, const int64_t *pairs, const float *targets, int64_t npairs,
                       const msa_train_cfg *cfg, float *losses_out) {
  if (!ctx || !pairs || !cfg || npairs < 1 || cfg->steps < 0 || cfg->batch_pairs < 1) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  TRY(set_device(ctx));
  Selector *s = nullptr;
  TRY(sel_get(ctx, &s));
  if (!s->params.p) {
    std::vector<float> host = default_params(cfg->seed, ctx->K);
    TRY(set_params(ctx, s, host.data()));
  }
  std::vector<float> tv;
  if (!targets) {
    // scale <= 0: put the mean target at 50, where the embedding's squared
    // distances sit at a natural scale for the initialisation and Adam steps
    TRY(exact_targets(ctx, pairs, npairs, cfg->target_scale > 0 ? cfg->target_scale : 1.f, tv));
    if (cfg->target_scale <= 0) {
      double mean = 0;
      for (float v : tv) mean += v;
      mean /= (double)npairs;
      const float k = mean > 0 ? (float)(50.0 / mean) : 1.f;
      for (float &v : tv) v *= k;
    }
    targets = tv.data();
  }
  // one shuffled pass over the pairs per epoch (splitmix64 Fisher-Yates)
  std::vector<int64_t> order(npairs);
  std::iota(order.begin(), order.end(), 0);
  int64_t at = npairs;
  uint64_t epoch = 0;
  const int bp = (int)std::min<int64_t>(cfg->batch_pairs, npairs);
  std::vector<int64_t> bpairs(2 * (size_t)bp);
  std::vector<float> bt(bp);
  stage_begin(ctx, ST_SELECTOR);
  for (int step = 0; step < cfg->steps; ++step) {
    if (at + bp > npairs) {
      for (int64_t i = npairs - 1; i > 0; --i) {
        const int64_t j = (int64_t)(splitmix64(cfg->seed ^ (epoch * 0x9e3779b97f4a7c15ull) ^ (uint64_t)i) % (uint64_t)(i + 1));
        std::swap(order[i], order[j]);
      }
      ++epoch;
      at = 0;
    }
    for (int x = 0; x < bp; ++x) {
      const int64_t q = order[at + x];
      bpairs[2 * x] = pairs[2 * q];
      bpairs[2 * x + 1] = pairs[2 * q + 1];
      bt[x] = targets[q];
    }
    at += bp;
    net::Batch b;
    TRY(stage_pairs(ctx, s, bpairs.data(), bt.data(), bp, b));
    TRY(forward_backward(ctx, s, b, bp));
    s->step += 1;
    // cosine decay of the learning rate from lr to lr / 10 over the steps
    const double frac = cfg->steps > 1 ? (double)step / (cfg->steps - 1) : 0.0;
    const float lr = (float)(cfg->lr * (0.1 + 0.45 * (1.0 + std::cos(3.141592653589793 * frac))));
    CK((++ctx->launches, net::adam)(P<float>(s->params), P<float>(s->grads), P<float>(s->m), P<float>(s->v),
                                    net::N_PARAMS, lr, cfg->beta1, cfg->beta2, cfg->eps, s->step, ctx->st));
    TRY(refresh_all(ctx, s));
    if (losses_out)
      CK(cudaMemcpyAsync(losses_out + step, s->loss.p, sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
  }
  stage_end(ctx, ST_SELECTOR);
  CK(cudaStreamSynchronize(ctx->st));
  stage_collect(ctx, ST_SELECTOR);
  return check_derr(ctx);
}

int msa_selector_embed(msa_ctx *ctx, float *emb_out) {
  if (!ctx || !emb_out) return MSA_EINVAL;
  if (ctx->n == 0) return fail(ctx, MSA_ESTATE, "no sequences loaded");
  if (!ctx->sel || !ctx->sel->params.p) return fail(ctx, MSA_ESTATE, "no selector");
  TRY(set_device(ctx));
  Selector *s = ctx->sel;
  TRY(embed_all(ctx, s));
  std::vector<float> h((size_t)ctx->n * net::DIM), o((size_t)ctx->n * net::DIM);
  CK(cudaMemcpyAsync(h.data(), s->allemb.p, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int k = 0; k < ctx->n; ++k)
    memcpy(&o[(size_t)ctx->perm[k] * net::DIM], &h[(size_t)k * net::DIM], sizeof(float) * net::DIM);
  CK(cudaMemcpyAsync(emb_out, o.data(), sizeof(float) * o.size(), cudaMemcpyDefault, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return check_derr(ctx);
}

int msa_save_selector(msa_ctx *ctx, const char *path) {
  if (!ctx || !path) return MSA_EINVAL;
  std::vector<float> p(net::N_PARAMS);
  TRY(msa_selector_params(ctx, p.data(), nullptr));
  FILE *f = fopen(path, "wb");
  if (!f) return fail(ctx, MSA_EINVAL, "cannot open %s", path);
  const char magic[8] = {'M', 'S', 'A', 'S', 'E', 'L', '1', 0};
  const int64_t count = (int64_t)net::N_PARAMS;
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&count, sizeof count, 1, f) == 1 &&
            fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? MSA_OK : fail(ctx, MSA_EINVAL, "write to %s failed", path);
}

int msa_load_selector(msa_ctx *ctx, const char *path) {
  if (!ctx || !path) return MSA_EINVAL;
  FILE *f = fopen(path, "rb");
  if (!f) return fail(ctx, MSA_EINVAL, "cannot open %s", path);
  char magic[8];
  int64_t count = 0;
  std::vector<float> p(net::N_PARAMS);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "MSASEL1", 8) == 0 &&
            fread(&count, sizeof count, 1, f) == 1 && count == (int64_t)net::N_PARAMS &&
            fread(p.data(), sizeof(float), p.size(), f) == p.size();
  fclose(f);
  if (!ok) return fail(ctx, MSA_EINVAL, "%s is not a selector file", path);
  return msa_selector_init(ctx, 0, p.data(), count);
}

// One 128-row (128 -> 128 channel) convolution with its loads suppressed and
// a poll limit of 4,096: every wait runs out and the kernel reports it.
int msa_debug_wait_timeout(msa_ctx *ctx, int32_t *timed_out) {
  if (!ctx || !timed_out) return MSA_EINVAL;
  TRY(set_device(ctx));
  *timed_out = 0;
  const int T = 128, C = net::WD;
  DevBuf x, w, bias, rows, y;
  auto cleanup = [&]() { for (DevBuf *b : {&x, &w, &bias, &rows, &y}) release(ctx, *b); };
  int rc = [&]() -> int {
    TRY(ensure(ctx, x, sizeof(bf16) * T * C));
    TRY(ensure(ctx, w, sizeof(bf16) * net::TAPS * C * C));
    TRY(ensure(ctx, bias, sizeof(float) * C));
    TRY(ensure(ctx, rows, sizeof(int32_t) * T));
    TRY(ensure(ctx, y, sizeof(bf16) * T * C));
    CK(cudaMemsetAsync(x.p, 0, x.cap, ctx->st));
    CK(cudaMemsetAsync(w.p, 0, w.cap, ctx->st));
    CK(cudaMemsetAsync(bias.p, 0, bias.cap, ctx->st));
    CK(cudaMemsetAsync(rows.p, 0, rows.cap, ctx->st));
    CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
    ++ctx->launches;
    CK(net::conv_tc(C, C, 0, P<bf16>(x), P<bf16>(w), P<float>(bias), P<int32_t>(rows), nullptr, y.p, T,
                    ctx->derr, ctx->st, 4096, true));
    unsigned h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, ctx->derr, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *timed_out = (h[0] & MSA_DERR_TIMEOUT_TC) ? 1 : 0;
    CK(cudaMemsetAsync(ctx->derr, 0, 2 * sizeof(unsigned), ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MSA_OK;
  }();
  cleanup();
  return rc;
}

}  // extern "C"
