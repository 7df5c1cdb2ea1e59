// net_kernels.cu -- kernels of the learned center selector.
//
// The 9-tap 1-D convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, bf16 operands, fp32 accumulation): rows = positions of
// the flat batch, reduction = taps x input channels.  A CTA stages 128 output
// rows plus the 8 halo rows of its input tile once, then streams one tap of
// weights at a time; each of its 8 warps owns 16 rows and every output
// channel.  The weight gradient is the same contraction with the positions as
// the reduction (both operands read transposed with ldmatrix.trans).
#include <algorithm>
#include <cfloat>
#include <climits>

#include "net_kernels.cuh"

namespace net {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// d += a (16x16, row) * b (16x8, col)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int BM = 128;  // output rows per CTA

template <int CIN, int COUT>
constexpr int conv_smem() { return ((BM + 2 * HALF) * (CIN + 8) + COUT * (CIN + 8)) * 2; }

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(256) k_conv(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                                              const float *__restrict__ bias,
                                              const int32_t *__restrict__ rowseq,
                                              const bf16 *__restrict__ prev, void *__restrict__ y,
                                              int T) {
  constexpr int SA = CIN + 8, SB = CIN + 8, CH = CIN / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  bf16 *sA = reinterpret_cast<bf16 *>(smraw);
  bf16 *sB = sA + (BM + 2 * HALF) * SA;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int r0 = blockIdx.x * BM;
  for (int idx = tid; idx < (BM + 2 * HALF) * CH; idx += 256) {
    const int i = idx / CH, c = idx - i * CH;
    const int r = r0 - HALF + i;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r >= 0 && r < T) v = *reinterpret_cast<const uint4 *>(x + (size_t)r * CIN + c * 8);
    *reinterpret_cast<uint4 *>(sA + i * SA + c * 8) = v;
  }
  float acc[COUT / 8][4];
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

  for (int tap = 0; tap < TAPS; ++tap) {
    const int wt = MODE == 2 ? TAPS - 1 - tap : tap;
    __syncthreads();
    for (int idx = tid; idx < COUT * CH; idx += 256) {
      const int n = idx / CH, c = idx - n * CH;
      *reinterpret_cast<uint4 *>(sB + n * SB + c * 8) =
          *reinterpret_cast<const uint4 *>(w + ((size_t)wt * COUT + n) * CIN + c * 8);
    }
    __syncthreads();
#pragma unroll
    for (int kc = 0; kc < CIN / 16; ++kc) {
      uint32_t a[4];
      ldsm_x4(a, sA + (wp * 16 + tap + (lane & 15)) * SA + kc * 16 + (lane >> 4) * 8);
#pragma unroll
      for (int j = 0; j < COUT / 16; ++j) {
        uint32_t b[4];
        ldsm_x4(b, sB + ((2 * j + (lane >> 4)) * 8 + (lane & 7)) * SB + kc * 16 + ((lane >> 3) & 1) * 8);
        mma16816(acc[2 * j], a, b[0], b[1]);
        mma16816(acc[2 * j + 1], a, b[2], b[3]);
      }
    }
  }
  const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = r0 + wp * 16 + gid + 8 * h;
    if (r >= T) continue;
    const bool valid = rowseq[r] >= 0;
#pragma unroll
    for (int nt = 0; nt < COUT / 8; ++nt) {
      const int c = nt * 8 + tig * 2;
      float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
      if constexpr (MODE == 0) {
        v0 = valid ? fmaxf(v0 + bias[c], 0.f) : 0.f;
        v1 = valid ? fmaxf(v1 + bias[c + 1], 0.f) : 0.f;
        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(y) + (size_t)r * COUT + c) =
            __floats2bfloat162_rn(v0, v1);
      } else if constexpr (MODE == 1) {
        v0 = valid ? v0 + bias[c] : 0.f;
        v1 = valid ? v1 + bias[c + 1] : 0.f;
        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(y) + (size_t)r * COUT + c) =
            make_float2(v0, v1);
      } else {
        const __nv_bfloat162 pv =
            *reinterpret_cast<const __nv_bfloat162 *>(prev + (size_t)r * COUT + c);
        v0 = valid && __bfloat162float(pv.x) > 0.f ? v0 : 0.f;
        v1 = valid && __bfloat162float(pv.y) > 0.f ? v1 : 0.f;
        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(y) + (size_t)r * COUT + c) =
            __floats2bfloat162_rn(v0, v1);
      }
    }
  }
}

// dW[tap][ci][co] += sum over rows r of x[r + tap - 4][ci] * dy[r][co].
// CTA = (chunk of rows, tap); warps tile ci x co; partials meet in fp32
// atomics.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(const bf16 *__restrict__ x, const bf16 *__restrict__ dy,
                                               float *__restrict__ dw, int T, int chunk) {
  constexpr int KS = 64, SX = CIN + 8, SD = COUT + 8;
  constexpr int WM = CIN / 16, WN = 8 / WM, NT = COUT / (8 * WN);
  static_assert(WM * WN == 8 && NT % 2 == 0, "warp tiling");
  __shared__ __align__(16) bf16 sX[KS * SX];
  __shared__ __align__(16) bf16 sD[KS * SD];
  const int tap = blockIdx.y;
  const int c0 = blockIdx.x * chunk, c1 = min(T, c0 + chunk);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int wm = wp % WM, wn = wp / WM;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int p0 = c0; p0 < c1; p0 += KS) {
    __syncthreads();
    for (int idx = tid; idx < KS * (CIN / 8); idx += 256) {
      const int i = idx / (CIN / 8), c = idx - i * (CIN / 8);
      const int r = p0 + i + tap - HALF;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r >= 0 && r < T) v = *reinterpret_cast<const uint4 *>(x + (size_t)r * CIN + c * 8);
      *reinterpret_cast<uint4 *>(sX + i * SX + c * 8) = v;
    }
    for (int idx = tid; idx < KS * (COUT / 8); idx += 256) {
      const int i = idx / (COUT / 8), c = idx - i * (COUT / 8);
      const int r = p0 + i;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r < c1) v = *reinterpret_cast<const uint4 *>(dy + (size_t)r * COUT + c * 8);
      *reinterpret_cast<uint4 *>(sD + i * SD + c * 8) = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KS / 16; ++kk) {
      uint32_t a[4];
      ldsm_x4_t(a, sX + (kk * 16 + (lane >> 4) * 8 + (lane & 7)) * SX + wm * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int j = 0; j < NT / 2; ++j) {
        uint32_t b[4];
        ldsm_x4_t(b, sD + (kk * 16 + ((lane >> 3) & 1) * 8 + (lane & 7)) * SD +
                         (wn * NT + 2 * j + (lane >> 4)) * 8);
        mma16816(acc[2 * j], a, b[0], b[1]);
        mma16816(acc[2 * j + 1], a, b[2], b[3]);
      }
    }
  }
  const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ci = wm * 16 + gid + 8 * h;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int co = (wn * NT + nt) * 8 + tig * 2;
      float *d = dw + ((size_t)tap * CIN + ci) * COUT + co;
      atomicAdd(d, acc[nt][2 * h]);
      atomicAdd(d + 1, acc[nt][2 * h + 1]);
    }
  }
}

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

__global__ void k_pool(Batch b, const float *__restrict__ y4, float *__restrict__ emb) {
  const int s = blockIdx.x, c = threadIdx.x;
  if (s >= b.nseq || c >= DIM) return;
  float acc = 0.f;
  const int base = b.base[s], L = b.len[s];
  for (int i = 0; i < L; ++i) acc += y4[(size_t)(base + i) * DIM + c];
  emb[(size_t)s * DIM + c] = acc * rsqrtf((float)L);
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

template <int CIN, int COUT, int MODE>
cudaError_t launch_conv(const bf16 *x, const bf16 *w, const float *bias, const int32_t *rowseq,
                        const bf16 *prev, void *y, int T, cudaStream_t st) {
  constexpr int smem = conv_smem<CIN, COUT>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_conv<CIN, COUT, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  k_conv<CIN, COUT, MODE><<<(T + BM - 1) / BM, 256, smem, st>>>(x, w, bias, rowseq, prev, y, T);
  return cudaGetLastError();
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

cudaError_t conv(int cin, int cout, int mode, const bf16 *x, const bf16 *w, const float *bias,
                 const int32_t *rowseq, const bf16 *prev, void *y, int T, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
#define NET_CONV(CI, CO, MD) \
  if (cin == CI && cout == CO && mode == MD) return launch_conv<CI, CO, MD>(x, w, bias, rowseq, prev, y, T, st);
  NET_CONV(32, 128, 0)
  NET_CONV(128, 128, 0)
  NET_CONV(128, 64, 1)
  NET_CONV(64, 128, 2)
  NET_CONV(128, 128, 2)
#undef NET_CONV
  return cudaErrorInvalidValue;
}

cudaError_t wgrad(int cin, int cout, const bf16 *x, const bf16 *dy, float *dw, int T,
                  cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  const int chunk = 2048;
  dim3 grid((T + chunk - 1) / chunk, TAPS);
  if (cin == 32 && cout == 128) k_wgrad<32, 128><<<grid, 256, 0, st>>>(x, dy, dw, T, chunk);
  else if (cin == 128 && cout == 128) k_wgrad<128, 128><<<grid, 256, 0, st>>>(x, dy, dw, T, chunk);
  else if (cin == 128 && cout == 64) k_wgrad<128, 64><<<grid, 256, 0, st>>>(x, dy, dw, T, chunk);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t colsum(int cout, const bf16 *dy, float *db, int T, cudaStream_t st) {
  if (T <= 0) return cudaSuccess;
  const int chunk = 128;  // short serial sums, many CTAs
  k_colsum<<<(T + chunk - 1) / chunk, cout, 0, st>>>(cout, dy, db, T, chunk);
  return cudaGetLastError();
}

cudaError_t pool(const Batch &b, const float *y4, float *emb, cudaStream_t st) {
  if (b.nseq <= 0) return cudaSuccess;
  k_pool<<<b.nseq, DIM, 0, st>>>(b, y4, emb);
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
