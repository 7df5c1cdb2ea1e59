// net_kernels.cuh -- kernels of the learned center selector (a 1-D conv
// embedding network, bf16 tensor-core GEMMs with fp32 accumulation).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace net {

constexpr int KP = 32;     // one-hot input channels (alphabet padded)
constexpr int WD = 128;    // conv width
constexpr int DIM = 64;    // embedding size
constexpr int TAPS = 9;    // kernel taps
constexpr int HALF = 4;    // zero rows on each side of a sequence

// Parameter block (fp32, flat): W1 [9][32][128] b1 [128] W2 [9][128][128] b2
// W3 [9][128][128] b3 W4 [9][128][64] b4 [64].
constexpr size_t W1_OFF = 0, W1_N = (size_t)TAPS * KP * WD;
constexpr size_t B1_OFF = W1_OFF + W1_N;
constexpr size_t W2_OFF = B1_OFF + WD, W2_N = (size_t)TAPS * WD * WD;
constexpr size_t B2_OFF = W2_OFF + W2_N;
constexpr size_t W3_OFF = B2_OFF + WD, W3_N = W2_N;
constexpr size_t B3_OFF = W3_OFF + W3_N;
constexpr size_t W4_OFF = B3_OFF + WD, W4_N = (size_t)TAPS * WD * DIM;
constexpr size_t B4_OFF = W4_OFF + W4_N;
constexpr size_t N_PARAMS = B4_OFF + DIM;

// Batch layout: sequence s occupies rows [base[s], base[s] + len[s]) of a flat
// activation array; HALF zero rows separate consecutive sequences and pad the
// ends, so a 9-tap window never mixes two sequences.
struct Batch {
  int nseq, T;
  const int32_t *seq;   // sorted index of each batch sequence
  const int32_t *base;  // first row of each batch sequence
  const int32_t *len;
  int32_t *rowseq;      // batch sequence of each row, -1 on padding rows
};

cudaError_t fill_rows(const Batch &b, cudaStream_t st);
cudaError_t onehot(const Batch &b, const uint8_t *res, const int64_t *pstart, __nv_bfloat16 *x0,
                   cudaStream_t st);

// The 9-tap convolutions on the tcgen05 tensor cores (tc_conv.cu): (cin,
// cout) = (32, 128) and (128, 128) mode 0, (128, 128) and (64, 128) mode 2,
// (128, 64) mode 1.  mode 0: relu(x * W + b) -> bf16; mode 1: x * W + b ->
// fp32; mode 2 (data gradient): (dy * W^T, taps reversed) masked by prev >
// 0 -> bf16.  Padding rows (rowseq < 0) are written as zero; rowseq may be
// null (every row valid).  w: bf16 [9][cout][cin]
// ([tap][n][k]).  err: device error word (MSA_DERR_TIMEOUT_TC).  spins: polls
// before an mbarrier wait gives up (<= 0: the default, seconds); no_loads:
// the TMA warp issues nothing, so every wait runs out (the self-test of the
// bounded waits).
cudaError_t conv_tc(int cin, int cout, int mode, const __nv_bfloat16 *x, const __nv_bfloat16 *w,
                    const float *bias, const int32_t *rowseq, const __nv_bfloat16 *prev, void *y,
                    int T, unsigned *err, cudaStream_t st, long long spins = 0,
                    bool no_loads = false);
// dW[tap][ci][co] += sum_r x[r + tap - 4][ci] * dy[r][co] on the tcgen05
// tensor cores (tc_conv.cu): 128 input channels with 128 or 64 output
// channels, and 32 with 128 (fp32 atomics into dw).
cudaError_t wgrad_tc(int cin, int cout, const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *dw,
                     int T, unsigned *err, cudaStream_t st, long long spins = 0);
// db[c] += sum_r dy[r][c]
cudaError_t colsum(int cout, const __nv_bfloat16 *dy, float *db, int T, cudaStream_t st);

// Pooled output layer: the nine window sums of the last hidden layer per
// sequence (pw: bf16 [9 nseq][128], rows 9 s + t), then, after the output
// convolution over them (mode 1, 9 nseq rows), the embedding
// emb[s] = (yw[9 s + 4] + (len - 1) b4) / sqrt(len) of the length-scaled sum
// of the output layer over the sequence's rows.
cudaError_t window_sums(const Batch &b, const __nv_bfloat16 *a3, __nv_bfloat16 *pw, cudaStream_t st);
cudaError_t emb_from_windows(const Batch &b, const float *yw, const float *b4, float *emb,
                             cudaStream_t st);
cudaError_t pair_loss(const int2 *pairs, const float *targets, int npairs, const float *emb,
                      float *demb, float *loss, cudaStream_t st);
cudaError_t pool_backward(const Batch &b, const float *demb, __nv_bfloat16 *dy4, cudaStream_t st);

cudaError_t adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1,
                 float b2, float eps, int step, cudaStream_t st);
// bf16 copies of the conv weights: wt [9][cout][cin] (forward) and wn
// [9][cin][cout] (data gradient; may be null)
cudaError_t refresh(const float *w, int cin, int cout, __nv_bfloat16 *wt, __nv_bfloat16 *wn,
                    cudaStream_t st);
// argmin_i ||e_i - mean(e)||^2 over n embeddings (lowest index on ties)
cudaError_t emb_center(const float *emb, int n, float *mean_scratch, long long *out_idx,
                       cudaStream_t st);

// dist[i] = ||e_i - mean(e)||^2
cudaError_t emb_dist(const float *emb, int n, float *mean_scratch, float *dist, cudaStream_t st);

}  // namespace net
