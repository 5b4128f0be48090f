// Learned coarse correction (an extra stage of the flexible GMRES; the paper
// has no learned component): a 6-layer 3x3 convolutional network on an
// Nc x Nc coarse grid, BF16 activations and weights with FP32 accumulation.
//
// k_conv_tc: one 3x3 convolution (zero padding) as an implicit GEMM on the
//   5th-generation tensor cores. A CTA of 128 threads takes 128 consecutive
//   pixels: D[128 x CO] = A[128 x 9CI] B[9CI x CO] with A the im2col rows of
//   those pixels (K index = tap * CI + ci) and B the weights. A and B are
//   staged in shared memory in the no-swizzle K-major core-matrix layout
//   (8 rows x 16 bytes per core matrix; core matrices adjacent in K are
//   LBO bytes apart, adjacent 8-row groups SBO bytes apart), one thread
//   issues the K/16 tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator in
//   TMEM), tcgen05.commit signals an mbarrier, and each warp reads its 32
//   accumulator rows back with tcgen05.ld for the epilogue (bias, ReLU or a
//   ReLU mask, BF16 and/or FP32 store). The same kernel runs the backward
//   data gradient with the transposed, tap-flipped weights.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace rp {

namespace {

constexpr int kConvPix = 128;     // pixels per CTA (the MMA's M)
constexpr int kTmemCols = 32;     // accumulator columns allocated (CO <= 32)

template <int CI, int CO>
struct ConvSmem {
  static constexpr int K = 9 * CI;
  static constexpr int A_BYTES = kConvPix * K * 2;
  static constexpr int B_BYTES = CO * K * 2;
  static constexpr int BYTES = A_BYTES + B_BYTES + 64;
};

}  // namespace

// in: NHWC BF16 [H*X][CI]; wt: B in core-matrix order ([K/8][CO/8][8][8]
// BF16); bias: CO floats or null; mask: NHWC BF16 [H*X][CO] or null (output
// multiplied by (mask > 0)); relu: apply max(., 0); outputs NHWC (BF16
// and/or FP32, [H*X][CO]). blockIdx.y selects the image of a batch: every
// pointer is offset by blockIdx.y times its per-image size.
template <int CI, int CO>
__global__ void __launch_bounds__(128)
    k_conv_tc(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ wt,
              const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask, int relu, int H, int X,
              __nv_bfloat16* __restrict__ out_bf, float* __restrict__ out_f, DevStatus* status) {
  using SM = ConvSmem<CI, CO>;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* A = sm;
  unsigned char* B = sm + SM::A_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SM::A_BYTES + SM::B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long npix = (long long)H * X;
  const long long img = blockIdx.y;
  in += img * npix * CI;
  if (mask) mask += img * npix * CO;
  if (out_bf) out_bf += img * npix * CO;
  if (out_f) out_f += img * npix * CO;
  const long long p0 = (long long)blockIdx.x * kConvPix;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  // B: the weights are stored in core-matrix order already
  {
    const uint4* src = reinterpret_cast<const uint4*>(wt);
    uint4* dst = reinterpret_cast<uint4*>(B);
    for (int i = tid; i < SM::B_BYTES / 16; i += 128) dst[i] = src[i];
  }
  // A: im2col of pixel p0 + tid, one 16-byte chunk (8 channels) at a time
  {
    const int m = tid;
    const long long p = p0 + m;
    const int y = (int)(p / X), x = (int)(p % X);
    const bool live = p < npix;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int sy = y + tap / 3 - 1, sx = x + tap % 3 - 1;
      const bool ok = live && sy >= 0 && sy < H && sx >= 0 && sx < X;
      const uint4* src = reinterpret_cast<const uint4*>(in + ((long long)sy * X + sx) * CI);
#pragma unroll
      for (int q = 0; q < CI / 8; ++q) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (ok) v = src[q];
        const int c = tap * (CI / 8) + q;   // K chunk
        *reinterpret_cast<uint4*>(A + ((c * (kConvPix / 8) + (m >> 3)) * 128 + (m & 7) * 16)) = v;
      }
    }
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    constexpr uint32_t lbo_a = (kConvPix / 8) * 128, lbo_b = (CO / 8) * 128;
    constexpr uint32_t idesc = idesc_bf16(kConvPix, CO);
#pragma unroll 1
    for (int s = 0; s < SM::K / 16; ++s) {
      const uint64_t ad = smem_desc(a0 + 2 * s * lbo_a, lbo_a, 128);
      const uint64_t bd = smem_desc(b0 + 2 * s * lbo_b, lbo_b, 128);
      tc_mma(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
    }
    tc_commit(bar);
  }
  __syncwarp();
  bool ok = mbar_wait_bounded(bar, 0);
  if (!ok) {
    // record the time-out; wait once more (bounded) for the MMAs in flight
    if (tid == 0) atomicExch(&status->timeout, 1);
    ok = mbar_wait_bounded(bar, 0);
  }
  tc_fence_after();
  if (ok) {
    const int m = warp * 32 + lane;
    const long long p = p0 + m;
#pragma unroll
    for (int h = 0; h < CO / 16; ++h) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 16), v);
      if (p < npix) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int co = h * 16 + i;
          float t = v[i] + (bias ? bias[co] : 0.f);
          if (relu) t = fmaxf(t, 0.f);
          if (mask && !(__bfloat162float(mask[p * CO + co]) > 0.f)) t = 0.f;
          v[i] = t;
        }
        if (out_f) {
          float4* o = reinterpret_cast<float4*>(out_f + p * CO + h * 16);
#pragma unroll
          for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
        if (out_bf) {
          __nv_bfloat162 pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) pk[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
          uint4* o = reinterpret_cast<uint4*>(out_bf + p * CO + h * 16);
          o[0] = *reinterpret_cast<uint4*>(&pk[0]);
          o[1] = *reinterpret_cast<uint4*>(&pk[4]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

namespace {

// ---------------------------------------------------------------------------
// Layout helpers
// ---------------------------------------------------------------------------
// Master parameters (FP32), layer by layer: W[co][ci][3][3] then b[co], the
// real channel counts (2, 32, 32, 32, 32, 32, 2).
constexpr int kLayers = 6;
__host__ __device__ constexpr int ch_real(int i) { return (i == 0 || i == kLayers) ? 2 : 32; }
__host__ __device__ constexpr int ch_pad(int i) { return (i == 0 || i == kLayers) ? 16 : 32; }

// B tile (core-matrix order) of layer l, forward: n = co, k = tap*CI + ci.
// Transposed (data gradient): n = ci, k = tap'*CO + co with tap' = 8 - tap.
__global__ void k_prep_weights(const float* __restrict__ W, int cir, int cor, int cip, int cop, int transposed,
                               __nv_bfloat16* __restrict__ tile) {
  const int N = transposed ? cip : cop, CIk = transposed ? cop : cip, K = 9 * CIk;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * K) return;
  // element e of the tile: chunk c, n-group g, row r, column q
  const int q = e & 7, r = (e >> 3) & 7, rest = e >> 6;
  const int g = rest % (N / 8), c = rest / (N / 8);
  const int n = g * 8 + r, k = c * 8 + q;
  const int tap = k / CIk, kc = k % CIk;
  float v = 0.f;
  if (!transposed) {
    const int co = n, ci = kc;
    if (co < cor && ci < cir) v = W[(co * cir + ci) * 9 + tap];
  } else {
    const int ci = n, co = kc;
    if (co < cor && ci < cir) v = W[(co * cir + ci) * 9 + (8 - tap)];
  }
  tile[e] = __float2bfloat16_rn(v);
}

__global__ void k_pad_bias(const float* __restrict__ b, int cor, int cop, float* __restrict__ bp) {
  const int i = threadIdx.x;
  if (i < cop) bp[i] = i < cor ? b[i] : 0.f;
}

// NCHW FP32 (2 channels) -> NHWC BF16 with 16 channels (zeros beyond 2)
__global__ void k_to_nhwc16(const float* __restrict__ x, long long npix, __nv_bfloat16* __restrict__ a) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long img = blockIdx.y;
  if (p >= npix) return;
  __nv_bfloat16* o = a + (img * npix + p) * 16;
  const float* xi = x + img * 2 * npix;
  o[0] = __float2bfloat16_rn(xi[p]);
  o[1] = __float2bfloat16_rn(xi[npix + p]);
#pragma unroll
  for (int c = 2; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
}

// NHWC FP32 (16 channels, first 2 used) -> NCHW FP32 (2 channels)
__global__ void k_from_nhwc16(const float* __restrict__ y, long long npix, float* __restrict__ x) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long img = blockIdx.y;
  if (p >= npix) return;
  x[img * 2 * npix + p] = y[(img * npix + p) * 16];
  x[img * 2 * npix + npix + p] = y[(img * npix + p) * 16 + 1];
}

template <int CI, int CO>
cudaError_t conv_t(const __nv_bfloat16* in, const __nv_bfloat16* wt, const float* bias, const __nv_bfloat16* mask,
                   int relu, int H, int X, int nimg, __nv_bfloat16* out_bf, float* out_f, DevStatus* status,
                   cudaStream_t st) {
  using SM = ConvSmem<CI, CO>;
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::BYTES);
  if (e != cudaSuccess) return e;
  const long long npix = (long long)H * X;
  dim3 grid((unsigned)((npix + kConvPix - 1) / kConvPix), (unsigned)nimg);
  k_conv_tc<CI, CO><<<grid, 128, SM::BYTES, st>>>(in, wt, bias, mask, relu, H, X, out_bf, out_f, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv(int ci, int co, const void* in, const void* wt, const float* bias, const void* mask, int relu,
                        int H, int X, int nimg, void* out_bf, float* out_f, DevStatus* status, cudaStream_t st) {
  using bf = __nv_bfloat16;
  if (ci == 16 && co == 32)
    return conv_t<16, 32>((const bf*)in, (const bf*)wt, bias, (const bf*)mask, relu, H, X, nimg, (bf*)out_bf, out_f,
                          status, st);
  if (ci == 32 && co == 32)
    return conv_t<32, 32>((const bf*)in, (const bf*)wt, bias, (const bf*)mask, relu, H, X, nimg, (bf*)out_bf, out_f,
                          status, st);
  if (ci == 32 && co == 16)
    return conv_t<32, 16>((const bf*)in, (const bf*)wt, bias, (const bf*)mask, relu, H, X, nimg, (bf*)out_bf, out_f,
                          status, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_prep_weights(const float* W, int l, int transposed, void* tile, cudaStream_t st) {
  const int cip = ch_pad(l), cop = ch_pad(l + 1);
  const int n = 9 * cip * cop;
  k_prep_weights<<<(n + 255) / 256, 256, 0, st>>>(W, ch_real(l), ch_real(l + 1), cip, cop, transposed,
                                                 (__nv_bfloat16*)tile);
  return cudaGetLastError();
}

cudaError_t launch_pad_bias(const float* b, int l, float* bp, cudaStream_t st) {
  k_pad_bias<<<1, 32, 0, st>>>(b, ch_real(l + 1), ch_pad(l + 1), bp);
  return cudaGetLastError();
}

cudaError_t launch_to_nhwc16(const float* x, long long npix, int nimg, void* a, cudaStream_t st) {
  dim3 grid((unsigned)((npix + 255) / 256), (unsigned)nimg);
  k_to_nhwc16<<<grid, 256, 0, st>>>(x, npix, (__nv_bfloat16*)a);
  return cudaGetLastError();
}

cudaError_t launch_from_nhwc16(const float* y, long long npix, int nimg, float* x, cudaStream_t st) {
  dim3 grid((unsigned)((npix + 255) / 256), (unsigned)nimg);
  k_from_nhwc16<<<grid, 256, 0, st>>>(y, npix, x);
  return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------------------
// Backward pieces
// ---------------------------------------------------------------------------
// Loss L = (1/nimg) sum_images mean_{pixel, channel<2} (out - t)^2 / 2 and its
// gradient g = (out - t) / (2 npix nimg) on the first two of 16 channels
// (BF16 NHWC); per-block partial sums of L in lossp.
__global__ void k_loss_grad(const float* __restrict__ out, const float* __restrict__ t, long long npix, int nimg,
                            __nv_bfloat16* __restrict__ g, double* __restrict__ lossp) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long img = blockIdx.y;
  const double inv = 1.0 / (2.0 * (double)npix * nimg);
  double l = 0.0;
  if (p < npix) {
    const float* o = out + (img * npix + p) * 16;
    const float* ti = t + img * 2 * npix;
    const float d0 = o[0] - ti[p], d1 = o[1] - ti[npix + p];
    l = 0.5 * ((double)d0 * d0 + (double)d1 * d1) * inv;
    __nv_bfloat16* go = g + (img * npix + p) * 16;
    go[0] = __float2bfloat16_rn((float)(d0 * inv));
    go[1] = __float2bfloat16_rn((float)(d1 * inv));
#pragma unroll
    for (int c = 2; c < 16; ++c) go[c] = __float2bfloat16_rn(0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    lossp[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

constexpr int kWgRows = 8;   // image rows per weight-gradient block

// Partial weight and bias gradients of one layer over kWgRows image rows:
// dW[co][ci][tap] = sum_p g[p][co] a[p + tap - 4][ci], db[co] = sum_p g[p][co],
// FP32. Thread (ci, group of four co) keeps 4 x 9 sums; the three input
// rows around the current one and the gradient row are staged in shared
// memory. Only the real channels are written, in the master layout.
template <int CI, int CO>
__global__ void __launch_bounds__(256)
    k_wgrad(const __nv_bfloat16* __restrict__ a, const __nv_bfloat16* __restrict__ g, int H, int X, int cir,
            int cor, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smw[];
  __nv_bfloat16* as = reinterpret_cast<__nv_bfloat16*>(smw);   // [3][X + 2][CI]
  __nv_bfloat16* gs = as + 3 * (X + 2) * CI;                    // [X][CO]
  const int tid = threadIdx.x;
  const int ci = tid % CI, cg = tid / CI;
  const bool act = cg < CO / 4;
  const long long npix = (long long)H * X;
  const long long img = blockIdx.y;
  a += img * npix * CI;
  g += img * npix * CO;
  float acc[4][9], bacc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    bacc[u] = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[u][t] = 0.f;
  }
  const int y0 = blockIdx.x * kWgRows;
  for (int y = y0; y < y0 + kWgRows && y < H; ++y) {
    __syncthreads();
    for (int e = tid; e < 3 * (X + 2) * CI; e += blockDim.x) {
      const int c = e % CI, xx = (e / CI) % (X + 2) - 1, dy = e / (CI * (X + 2));
      const int sy = y + dy - 1;
      __nv_bfloat16 v = __float2bfloat16_rn(0.f);
      if (sy >= 0 && sy < H && xx >= 0 && xx < X) v = a[((long long)sy * X + xx) * CI + c];
      as[e] = v;
    }
    for (int e = tid; e < X * CO; e += blockDim.x) gs[e] = g[(long long)y * X * CO + e];
    __syncthreads();
    if (act) {
      for (int x = 0; x < X; ++x) {
        float gv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) gv[u] = __bfloat162float(gs[x * CO + cg * 4 + u]);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const float av = __bfloat162float(as[(dy * (X + 2) + x + dx) * CI + ci]);
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u][dy * 3 + dx] = fmaf(gv[u], av, acc[u][dy * 3 + dx]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) bacc[u] += gv[u];
      }
    }
  }
  const int nw = cor * cir * 9;
  float* out = part + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * (nw + cor);
  if (act) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int co = cg * 4 + u;
      if (co < cor && ci < cir) {
#pragma unroll
        for (int t = 0; t < 9; ++t) out[(co * cir + ci) * 9 + t] = acc[u][t];
      }
      if (co < cor && ci == 0) out[nw + co] = bacc[u];
    }
  }
}

// grad[i] = sum over blocks of part[b][i], i < count
__global__ void k_sum_parts(const float* __restrict__ part, int nblocks, int count, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.f;
  for (int b = 0; b < nblocks; ++b) s += part[(long long)b * count + i];
  grad[i] = s;
}

// Adam (bias-corrected moments) on the FP32 master parameters
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <int CI, int CO>
cudaError_t wgrad_t(const void* a, const void* g, int H, int X, int nimg, int cir, int cor, float* part,
                    cudaStream_t st) {
  const size_t smem = (size_t)(3 * (X + 2) * CI + X * CO) * sizeof(__nv_bfloat16);
  cudaError_t e = cudaFuncSetAttribute(k_wgrad<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((H + kWgRows - 1) / kWgRows), (unsigned)nimg);
  k_wgrad<CI, CO><<<grid, 256, smem, st>>>((const __nv_bfloat16*)a, (const __nv_bfloat16*)g, H, X, cir, cor, part);
  return cudaGetLastError();
}

}  // namespace

int wgrad_blocks(int H, int nimg) { return ((H + kWgRows - 1) / kWgRows) * nimg; }

cudaError_t launch_loss_grad(const float* out, const float* t, long long npix, int nimg, void* g, double* lossp,
                             int* nparts, cudaStream_t st) {
  dim3 grid((unsigned)((npix + 255) / 256), (unsigned)nimg);
  *nparts = (int)(grid.x * grid.y);
  k_loss_grad<<<grid, 256, 0, st>>>(out, t, npix, nimg, (__nv_bfloat16*)g, lossp);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(int l, const void* a, const void* g, int H, int X, int nimg, float* part, float* grad,
                         cudaStream_t st) {
  const int cir = ch_real(l), cor = ch_real(l + 1);
  cudaError_t e;
  if (l == 0)
    e = wgrad_t<16, 32>(a, g, H, X, nimg, cir, cor, part, st);
  else if (l == kLayers - 1)
    e = wgrad_t<32, 16>(a, g, H, X, nimg, cir, cor, part, st);
  else
    e = wgrad_t<32, 32>(a, g, H, X, nimg, cir, cor, part, st);
  if (e != cudaSuccess) return e;
  const int count = cor * cir * 9 + cor;
  k_sum_parts<<<(count + 255) / 256, 256, 0, st>>>(part, wgrad_blocks(H, nimg), count, grad);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, long long t, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, c1, c2, 1e-8f);
  return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------------------
// Coarse grid transfers (fine unknowns nx x ny, x fastest; pixel (I, J) owns
// the nodes with floor(i Nc / nx) = I, floor(j Nc / ny) = J)
// ---------------------------------------------------------------------------
constexpr int kRT = 256;

__global__ void k_restrict(const c128* __restrict__ r, int nx, int ny, int Nc, float* __restrict__ out,
                           double* __restrict__ partial, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  const int pix = blockIdx.x * kRT + threadIdx.x;
  const int npix = Nc * Nc;
  double ss = 0.0;
  if (pix < npix) {
    const int I = pix % Nc, J = pix / Nc;
    const int i0 = (int)(((long long)I * nx + Nc - 1) / Nc), i1 = (int)(((long long)(I + 1) * nx + Nc - 1) / Nc);
    const int j0 = (int)(((long long)J * ny + Nc - 1) / Nc), j1 = (int)(((long long)(J + 1) * ny + Nc - 1) / Nc);
    double re = 0.0, im = 0.0;
    for (int j = j0; j < j1; ++j)
      for (int i = i0; i < i1; ++i) {
        const c128 v = r[(long long)j * nx + i];
        re += v.re;
        im += v.im;
      }
    const double inv = 1.0 / ((double)(i1 - i0) * (j1 - j0));
    re *= inv;
    im *= inv;
    out[pix] = (float)re;
    out[npix + pix] = (float)im;
    ss = re * re + im * im;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __shared__ double red[kRT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRT / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_normalise(float* __restrict__ out, int Nc, const double* __restrict__ partial, int nparts,
                            double* __restrict__ s_dev, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  __shared__ double sh;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += partial[b];
    sh = sqrt(t);
    if (blockIdx.x == 0) *s_dev = sh;
  }
  __syncthreads();
  const double s = sh;
  const float f = s > 0.0 ? (float)((double)Nc / s) : 0.f;
  const int n = 2 * Nc * Nc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] *= f;
}

__device__ __forceinline__ void bilin_1d(int i, int n, int Nc, int& i0, float& w) {
  float u = ((float)i + 0.5f) * (float)Nc / (float)n - 0.5f;
  u = fminf(fmaxf(u, 0.f), (float)(Nc - 1));
  i0 = min((int)floorf(u), Nc - 2);
  w = u - (float)i0;
}

__global__ void k_prolong_add(const float* __restrict__ out16, int Nc, int nx, int ny, const double* __restrict__ s_dev,
                              double gamma, c128* __restrict__ z, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= (long long)nx * ny) return;
  const double s = *s_dev;
  if (!(s > 0.0)) return;
  const int j = (int)r / nx, i = (int)r - j * nx;   // n < 2^31
  int I0, J0;
  float wx, wy;
  bilin_1d(i, nx, Nc, I0, wx);
  bilin_1d(j, ny, Nc, J0, wy);
  const float* a = out16 + ((long long)J0 * Nc + I0) * 16;
  const float* b = a + 16;
  const float* c = a + (long long)Nc * 16;
  const float* d = c + 16;
  const float v0 = (1.f - wy) * ((1.f - wx) * a[0] + wx * b[0]) + wy * ((1.f - wx) * c[0] + wx * d[0]);
  const float v1 = (1.f - wy) * ((1.f - wx) * a[1] + wx * b[1]) + wy * ((1.f - wx) * c[1] + wx * d[1]);
  const double f = gamma * s / Nc;
  z[r] = z[r] + mk(f * v0, f * v1);
}

__global__ void k_scale_f32(float* __restrict__ v, long long n, float f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) v[i] *= f;
}

__global__ void k_csub(const c128* __restrict__ a, const c128* __restrict__ b, c128* __restrict__ o, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] - b[i];
}

}  // namespace

int restrict_blocks(int Nc) { return (Nc * Nc + kRT - 1) / kRT; }

cudaError_t launch_restrict(const c128* r, int nx, int ny, int Nc, float* out, double* partial, const KState* kst,
                            cudaStream_t st) {
  k_restrict<<<restrict_blocks(Nc), kRT, 0, st>>>(r, nx, ny, Nc, out, partial, kst);
  return cudaGetLastError();
}

cudaError_t launch_normalise(float* out, int Nc, const double* partial, double* s_dev, const KState* kst,
                             cudaStream_t st) {
  k_normalise<<<64, 256, 0, st>>>(out, Nc, partial, restrict_blocks(Nc), s_dev, kst);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(const float* out16, int Nc, int nx, int ny, const double* s_dev, double gamma, c128* z,
                               const KState* kst, cudaStream_t st) {
  const long long n = (long long)nx * ny;
  k_prolong_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out16, Nc, nx, ny, s_dev, gamma, z, kst);
  return cudaGetLastError();
}

cudaError_t launch_scale_f32(float* v, long long n, float f, cudaStream_t st) {
  k_scale_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, n, f);
  return cudaGetLastError();
}

cudaError_t launch_csub(const c128* a, const c128* b, c128* out, long long n, cudaStream_t st) {
  k_csub<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, out, n);
  return cudaGetLastError();
}

}  // namespace rp
