// net_kernels.cu -- the selector's small kernels: batch layout, one-hot
// input, bias gradients, pooling, the pair loss, Adam, weight refresh and the
// embedding-space center.  The convolutions and weight gradients run on the
// tensor cores in tc_conv.cu.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "net_kernels.cuh"

namespace net {
namespace {

typedef __nv_bfloat16 bf16;

__global__ void k_colsum(int cout, const bf16 *__restrict__ dy, float *__restrict__ db, int T,
                         int chunk) {
  const int c = threadIdx.x;
  if (c >= cout) return;
  const int r0 = blockIdx.x * chunk, r1 = min(T, r0 + chunk);
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s += __bfloat162float(dy[(size_t)r * cout + c]);
  if (s != 0.f) atomicAdd(db + c, s);
}

__global__ void k_fill_rows(Batch b) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < b.nseq; s += warps)
    for (int i = lane; i < b.len[s]; i += 32) b.rowseq[b.base[s] + i] = s;
}

__global__ void k_onehot(Batch b, const uint8_t *__restrict__ res, const int64_t *__restrict__ pstart,
                         bf16 *__restrict__ x0) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= b.T) return;
  const int s = b.rowseq[r];
  int ch = -1;
  if (s >= 0) ch = res[pstart[b.seq[s]] + (r - b.base[s])];
  uint4 *out = reinterpret_cast<uint4 *>(x0 + (size_t)r * KP);
#pragma unroll
  for (int q = 0; q < KP / 8; ++q) {
    uint32_t wv[4] = {0u, 0u, 0u, 0u};
    if (ch >= q * 8 && ch < q * 8 + 8) {
      const int e = ch - q * 8;  // bf16 1.0 = 0x3f80
      wv[e >> 1] = (e & 1) ? 0x3f800000u : 0x00003f80u;
    }
    out[q] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
}

// Pooling commutes with the linear output convolution: summed over the rows
// r of sequence s, y4[r] = sum_t a3[r + t - 4] W4_t + b4 gives
// sum_t P_t W4_t + len b4 with the window sums P_t = sum_r a3[r + t - 4]
// (rows outside the sequence are zero).  P_0 covers rows base - 4 ..
// base + len - 5 and P_{t+1} = P_t - a3[base - 4 + t] + a3[base + len - 4 + t].
// One 128-thread block per sequence: each warp sums every fourth row of P_0
// (four channels per lane), warp 0 adds the partial sums and slides the
// window; the nine sums are written as rows 9 s .. 9 s + 8 of pw (bf16),
// the input of the output convolution.
__device__ __forceinline__ void load4(const bf16 *p, float (&v)[4]) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
  v[0] = __low2float(lo);
  v[1] = __high2float(lo);
  v[2] = __low2float(hi);
  v[3] = __high2float(hi);
}

__global__ void k_window_sums(Batch b, const bf16 *__restrict__ a3, bf16 *__restrict__ pw) {
  __shared__ float part[4][WD];
  const int s = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (s >= b.nseq) return;
  const int base = b.base[s], L = b.len[s];
  const bf16 *row0 = a3 + (size_t)(base - HALF) * WD + 4 * lane;  // row base - 4
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int i = warp; i < L; i += 4) {
    float v[4];
    load4(row0 + (size_t)i * WD, v);
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += v[c];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) part[warp][4 * lane + c] = acc[c];
  __syncthreads();
  if (warp != 0) return;
  float p[4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    p[c] = part[0][4 * lane + c] + part[1][4 * lane + c] + part[2][4 * lane + c] + part[3][4 * lane + c];
  for (int t = 0; t < TAPS; ++t) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(p[0], p[1]), hi = __floats2bfloat162_rn(p[2], p[3]);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t *>(&lo);
    u.y = *reinterpret_cast<const uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(pw + ((size_t)TAPS * s + t) * WD + 4 * lane) = u;
    if (t + 1 < TAPS) {
      float out[4], in[4];
      load4(row0 + (size_t)t * WD, out);
      load4(row0 + (size_t)(L + t) * WD, in);
#pragma unroll
      for (int c = 0; c < 4; ++c) p[c] += in[c] - out[c];
    }
  }
}

// emb[s] = (row 9 s + 4 of the output convolution over the window sums,
// which holds sum_t P_t W4_t + b4, plus (len - 1) b4) / sqrt(len)
__global__ void k_emb_from_windows(Batch b, const float *__restrict__ yw, const float *__restrict__ b4,
                                   float *__restrict__ emb) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)b.nseq * DIM) return;
  const int s = (int)(idx / DIM), c = (int)(idx - (size_t)s * DIM);
  const int L = b.len[s];
  emb[idx] = (yw[((size_t)TAPS * s + HALF) * DIM + c] + (float)(L - 1) * b4[c]) * rsqrtf((float)L);
}

// One warp per pair: r = ||e_a - e_b||^2 - t; loss += r^2 / m;
// d e_a += 4 r (e_a - e_b) / m; d e_b -= the same.
__global__ void k_pair_loss(const int2 *__restrict__ pairs, const float *__restrict__ targets,
                            int npairs, const float *__restrict__ emb, float *__restrict__ demb,
                            float *loss) {
  const int pw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (pw >= npairs) return;
  const int a = pairs[pw].x, b = pairs[pw].y;
  const float d0 = emb[(size_t)a * DIM + lane] - emb[(size_t)b * DIM + lane];
  const float d1 = emb[(size_t)a * DIM + lane + 32] - emb[(size_t)b * DIM + lane + 32];
  float q = d0 * d0 + d1 * d1;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(MSA_FULL_MASK, q, off);
  const float m = (float)npairs;
  const float r = q - targets[pw];
  if (lane == 0) atomicAdd(loss, r * r / m);
  const float g = 4.f * r / m;
  atomicAdd(demb + (size_t)a * DIM + lane, g * d0);
  atomicAdd(demb + (size_t)a * DIM + lane + 32, g * d1);
  atomicAdd(demb + (size_t)b * DIM + lane, -g * d0);
  atomicAdd(demb + (size_t)b * DIM + lane + 32, -g * d1);
}

__global__ void k_pool_backward(Batch b, const float *__restrict__ demb, bf16 *__restrict__ dy4) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)b.T * DIM) return;
  const int r = (int)(idx / DIM), c = (int)(idx - (size_t)r * DIM);
  const int s = b.rowseq[r];
  float v = 0.f;
  if (s >= 0) v = demb[(size_t)s * DIM + c] * rsqrtf((float)b.len[s]);
  dy4[idx] = __float2bfloat16(v);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_refresh(const float *__restrict__ w, int cin, int cout, bf16 *__restrict__ wt,
                          bf16 *__restrict__ wn) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)TAPS * cin * cout;
  if (idx >= total) return;
  const int co = (int)(idx % cout);
  const int ci = (int)((idx / cout) % cin);
  const int tap = (int)(idx / ((size_t)cout * cin));
  const bf16 h = __float2bfloat16(w[idx]);
  wt[((size_t)tap * cout + co) * cin + ci] = h;
  if (wn) wn[idx] = h;
}

__global__ void k_emb_mean(const float *__restrict__ emb, int n, double *__restrict__ mean) {
  __shared__ double part[DIM];
  if (threadIdx.x < DIM) part[threadIdx.x] = 0.0;
  __syncthreads();
  const int c = threadIdx.x % DIM, rstep = blockDim.x / DIM;
  double acc = 0.0;
  for (int r = blockIdx.x * rstep + threadIdx.x / DIM; r < n; r += gridDim.x * rstep)
    acc += emb[(size_t)r * DIM + c];
  atomicAdd(&part[c], acc);
  __syncthreads();
  if (threadIdx.x < DIM) atomicAdd(&mean[threadIdx.x], part[threadIdx.x]);
}

// key = (float bits of the distance) << 32 | index: the smallest key is the
// smallest distance with the lowest index (distances are >= 0).
__global__ void k_emb_argmin(const float *__restrict__ emb, int n, const double *__restrict__ mean,
                             unsigned long long *key) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long best = ULLONG_MAX;
  if (r < n) {
    float d = 0.f;
    for (int c = 0; c < DIM; ++c) {
      const float x = emb[(size_t)r * DIM + c] - (float)(mean[c] / n);
      d += x * x;
    }
    best = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)r;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(MSA_FULL_MASK, best, off);
    best = o < best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best != ULLONG_MAX) atomicMin(key, best);
}

__global__ void k_emb_dist(const float *__restrict__ emb, int n, const double *__restrict__ mean,
                           float *__restrict__ dist) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float d = 0.f;
  for (int c = 0; c < DIM; ++c) {
    const float x = emb[(size_t)r * DIM + c] - (float)(mean[c] / n);
    d += x * x;
  }
  dist[r] = d;
}

__global__ void k_key_to_idx(const unsigned long long *key, long long *out) {
  *out = (long long)(*key & 0xffffffffull);
}

}  // namespace

cudaError_t fill_rows(const Batch &b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b.rowseq, 0xff, sizeof(int32_t) * (size_t)b.T, st);
  if (e != cudaSuccess) return e;
  const int blocks = std::max(1, std::min(4096, (b.nseq * 32 + 255) / 256));
  k_fill_rows<<<blocks, 256, 0, st>>>(b);
  return cudaGetLastError();
}

cudaError_t onehot(const Batch &b, const uint8_t *res, const int64_t *pstart, bf16 *x0,
                   cudaStream_t st) {
  k_onehot<<<(b.T + 255) / 256, 256, 0, st>>>(b, res, pstart, x0);
  return cudaGetLastError();
}

cudaError_t colsum(int cout, const bf16 *dy, float *db, int T, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  const int chunk = 128;  // short serial sums, many CTAs
  k_colsum<<<(T + chunk - 1) / chunk, cout, 0, st>>>(cout, dy, db, T, chunk);
  return cudaGetLastError();
}

cudaError_t window_sums(const Batch &b, const bf16 *a3, bf16 *pw, cudaStream_t st) {
  if (b.nseq <= 0) return cudaSuccess;
  k_window_sums<<<b.nseq, 128, 0, st>>>(b, a3, pw);
  return cudaGetLastError();
}

cudaError_t emb_from_windows(const Batch &b, const float *yw, const float *b4, float *emb,
                             cudaStream_t st) {
  const size_t total = (size_t)b.nseq * DIM;
  if (total == 0) return cudaSuccess;
  k_emb_from_windows<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(b, yw, b4, emb);
  return cudaGetLastError();
}

cudaError_t pair_loss(const int2 *pairs, const float *targets, int npairs, const float *emb,
                      float *demb, float *loss, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  k_pair_loss<<<(npairs * 32 + 255) / 256, 256, 0, st>>>(pairs, targets, npairs, emb, demb, loss);
  return cudaGetLastError();
}

cudaError_t pool_backward(const Batch &b, const float *demb, bf16 *dy4, cudaStream_t st) {
  const size_t total = (size_t)b.T * DIM;
  k_pool_backward<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(b, demb, dy4);
  return cudaGetLastError();
}

cudaError_t adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1,
                 float b2, float eps, int step, cudaStream_t st) {
  const float c1 = 1.f / (1.f - powf(b1, (float)step));
  const float c2 = 1.f / (1.f - powf(b2, (float)step));
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t refresh(const float *w, int cin, int cout, bf16 *wt, bf16 *wn, cudaStream_t st) {
  const size_t total = (size_t)TAPS * cin * cout;
  k_refresh<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(w, cin, cout, wt, wn);
  return cudaGetLastError();
}

cudaError_t emb_center(const float *emb, int n, float *mean_scratch, long long *out_idx,
                       cudaStream_t st) {
  double *mean = reinterpret_cast<double *>(mean_scratch);  // DIM doubles
  unsigned long long *key = reinterpret_cast<unsigned long long *>(mean + DIM);
  cudaError_t e = cudaMemsetAsync(mean, 0, sizeof(double) * DIM, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(key, 0xff, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int blocks = std::max(1, std::min(1024, (n + 3) / 4));
  k_emb_mean<<<blocks, 256, 0, st>>>(emb, n, mean);
  k_emb_argmin<<<(n + 255) / 256, 256, 0, st>>>(emb, n, mean, key);
  k_key_to_idx<<<1, 1, 0, st>>>(key, out_idx);
  return cudaGetLastError();
}

cudaError_t emb_dist(const float *emb, int n, float *mean_scratch, float *dist, cudaStream_t st) {
  double *mean = reinterpret_cast<double *>(mean_scratch);
  cudaError_t e = cudaMemsetAsync(mean, 0, sizeof(double) * DIM, st);
  if (e != cudaSuccess) return e;
  const int blocks = std::max(1, std::min(1024, (n + 3) / 4));
  k_emb_mean<<<blocks, 256, 0, st>>>(emb, n, mean);
  k_emb_dist<<<(n + 255) / 256, 256, 0, st>>>(emb, n, mean, dist);
  return cudaGetLastError();
}

}  // namespace net
