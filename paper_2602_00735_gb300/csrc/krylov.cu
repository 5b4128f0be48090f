// Global SpMV and the device-side flexible GMRES kernels (Section 4.1: GMRES
// with B^-1 as preconditioner), all in complex128.
//
// The global matrix is stored as four arrays over unknowns: D (diagonal) and
// the couplings of each node to its W, S and SW neighbours; the E, N and NE
// couplings are the W, S, SW couplings of those neighbours (symmetry).
//
// Reductions are deterministic: fixed per-block trees, then a fixed-order
// sum over blocks. Every kernel launched inside an Arnoldi cycle first reads
// the cycle's stop flag and returns at once when it is set, so the host can
// enqueue several iterations ahead and synchronise rarely.
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

constexpr int kThreads = 256;
int g_num_sms = 0;

// Kernels of a cycle return at once after the stop flag is set; gated ones
// (the second Gram-Schmidt pass) also when no reorthogonalisation is due.
__device__ __forceinline__ bool skip(const KState* kst, int gate) {
  return kst != nullptr && (kst->stop || (gate && !kst->reorth));
}

__device__ __forceinline__ c128 warp_sum(c128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}

__device__ __forceinline__ c128 block_sum(c128 v) {
  __shared__ c128 red[kThreads / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  c128 t = mk(0.0, 0.0);
  if (threadIdx.x < 32) {
    t = (l < kThreads / 32) ? red[l] : mk(0.0, 0.0);
    t = warp_sum(t);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// y = A x, or y = bsub - A x (bsub complex128 (bdf 0), double-float (1) or
// complex64 (2))
__global__ void k_spmv(long long n, int nx, const c128* __restrict__ D, const c128* __restrict__ CW,
                       const c128* __restrict__ CS, const c128* __restrict__ CSW, const c128* __restrict__ x,
                       const c128* __restrict__ bsub, int bdf, c128* __restrict__ y, const KState* __restrict__ kst,
                       int xdf) {
  if (kst != nullptr && kst->stop) return;
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  // x in complex128, or in double-float form (xdf: the FGMRES directions z_j)
  auto X = [&](long long q) -> c128 {
    if (!xdf) return x[q];
    const dfc v = reinterpret_cast<const dfc*>(x)[q];
    return mk(df_to_d(v.rh, v.rl), df_to_d(v.ih, v.il));
  };
  c128 a0 = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
  a0 = fmac(a0, D[r], X(r));
  if (r >= 1) a1 = fmac(a1, CW[r], X(r - 1));
  if (r + 1 < n) a0 = fmac(a0, CW[r + 1], X(r + 1));
  if (r >= nx) a1 = fmac(a1, CS[r], X(r - nx));
  if (r + nx < n) a0 = fmac(a0, CS[r + nx], X(r + nx));
  if (r >= nx + 1) a1 = fmac(a1, CSW[r], X(r - nx - 1));
  if (r + nx + 1 < n) a0 = fmac(a0, CSW[r + nx + 1], X(r + nx + 1));
  const c128 acc = a0 + a1;
  if (bsub) {
    c128 bv;
    if (bdf == 1) {
      const dfc d = reinterpret_cast<const dfc*>(bsub)[r];
      bv = mk(df_to_d(d.rh, d.rl), df_to_d(d.ih, d.il));
    } else if (bdf == 2) {
      bv = cvt<double>(reinterpret_cast<const c64*>(bsub)[r]);
    } else {
      bv = bsub[r];
    }
    y[r] = bv - acc;
  } else {
    y[r] = acc;
  }
}

// y = A x with the coefficients in double-float form (split once at set-up)
// and the products and sums in double-float arithmetic on the FP32 pipe
// (about 46 bits): the Arnoldi products w = A z_j. The true residual keeps
// the FP64 k_spmv.
__device__ __forceinline__ void cmac_df(float& rh, float& rl, float& ih, float& il, const dfc& a, const dfc& x) {
  const dfl ar = dfl_of(a.rh, a.rl), ai = dfl_of(a.ih, a.il);
  const dfl xr = dfl_of(x.rh, x.rl), xi = dfl_of(x.ih, x.il);
  float p, t;
  // a x = (ar xr - ai xi) + i (ar xi + ai xr)
  df_prod(ar, xr, p, t);
  df_acc(rh, rl, p, t);
  df_prod(ai, xi, p, t);
  df_acc(rh, rl, -p, -t);
  df_prod(ar, xi, p, t);
  df_acc(ih, il, p, t);
  df_prod(ai, xr, p, t);
  df_acc(ih, il, p, t);
}

// y = A x in double-float arithmetic on split coefficients, tiled: a CTA
// takes kSpTX x kSpTY grid points, splits the x values of the tile and its
// one-point halo into shared memory once (1.3 splits per row instead of 7),
// and each thread sums its row's seven products in the fixed order D, W, E,
// S, N, SW, NE. Couplings to points outside the grid are zero in the stored
// coefficients and are skipped.
constexpr int kSpTX = 32, kSpTY = 8;

__global__ void __launch_bounds__(kSpTX * kSpTY)
    k_spmv_df(int nx, int ny, const dfc* __restrict__ D, const dfc* __restrict__ CW, const dfc* __restrict__ CS,
              const dfc* __restrict__ CSW, const c128* __restrict__ x, c128* __restrict__ y, int out_df,
              int in_df, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  __shared__ dfc xs[kSpTY + 2][kSpTX + 2];
  const int i0 = blockIdx.x * kSpTX, j0 = blockIdx.y * kSpTY;
  for (int e = threadIdx.x; e < (kSpTX + 2) * (kSpTY + 2); e += kSpTX * kSpTY) {
    const int li = e % (kSpTX + 2), lj = e / (kSpTX + 2);
    const int gi = i0 + li - 1, gj = j0 + lj - 1;
    dfc v = {0.f, 0.f, 0.f, 0.f};
    if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
      const long long idx = (long long)gj * nx + gi;
      v = in_df ? reinterpret_cast<const dfc*>(x)[idx] : split_c(x[idx]);
    }
    xs[lj][li] = v;
  }
  __syncthreads();
  const int ti = threadIdx.x % kSpTX, tj = threadIdx.x / kSpTX;
  const int i = i0 + ti, j = j0 + tj;
  if (i >= nx || j >= ny) return;
  const long long r = (long long)j * nx + i;
  const bool e_ok = i + 1 < nx, n_ok = j + 1 < ny;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  cmac_df(rh, rl, ih, il, D[r], xs[tj + 1][ti + 1]);
  if (i >= 1) cmac_df(rh, rl, ih, il, CW[r], xs[tj + 1][ti]);
  if (e_ok) cmac_df(rh, rl, ih, il, CW[r + 1], xs[tj + 1][ti + 2]);
  if (j >= 1) cmac_df(rh, rl, ih, il, CS[r], xs[tj][ti + 1]);
  if (n_ok) cmac_df(rh, rl, ih, il, CS[r + nx], xs[tj + 2][ti + 1]);
  if (i >= 1 && j >= 1) cmac_df(rh, rl, ih, il, CSW[r], xs[tj][ti]);
  if (e_ok && n_ok) cmac_df(rh, rl, ih, il, CSW[r + nx + 1], xs[tj + 2][ti + 2]);
  if (out_df) {
    df_norm(rh, rl);
    df_norm(ih, il);
    dfc o;
    o.rh = rh;
    o.rl = rl;
    o.ih = ih;
    o.il = il;
    reinterpret_cast<dfc*>(y)[r] = o;
  } else {
    y[r] = mk(df_to_d(rh, rl), df_to_d(ih, il));
  }
}

// partial[c * gridDim.x + blk] = sum over the block's rows of conj(V_c) w
__global__ void __launch_bounds__(kThreads)
    k_dots(const c128* __restrict__ V, long long ldv, const c128* __restrict__ w, long long n,
           c128* __restrict__ partial, const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  const int c = blockIdx.y;
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per;
  const long long r1 = min(n, r0 + per);
  const c128* v = V + c * ldv;
  c128 a0 = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
  long long r = r0 + threadIdx.x;
  for (; r + kThreads < r1; r += 2 * kThreads) {
    a0 = fcma(a0, v[r], w[r]);
    a1 = fcma(a1, v[r + kThreads], w[r + kThreads]);
  }
  if (r < r1) a0 = fcma(a0, v[r], w[r]);
  c128 s = block_sum(a0 + a1);
  if (threadIdx.x == 0) partial[(long long)c * gridDim.x + blockIdx.x] = s;
}

// out[c] (+)= sum_blk partial[c][blk], one warp per column
__global__ void k_dots_finish(const c128* __restrict__ partial, int G, int ncols, c128* __restrict__ out,
                              int accumulate, const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int l = threadIdx.x & 31;
  if (c >= ncols) return;
  c128 s = mk(0.0, 0.0);
  for (int b = l; b < G; b += 32) s = s + partial[(long long)c * G + b];
  s = warp_sum(s);
  if (l == 0) out[c] = accumulate ? out[c] + s : s;
}

// w += sign * sum_c V_c h_c
__global__ void __launch_bounds__(kThreads)
    k_axpys(const c128* __restrict__ V, long long ldv, int ncols, const c128* __restrict__ h, double sign,
            c128* __restrict__ w, long long n, const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  extern __shared__ c128 hs[];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = sign * h[c];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    c128 a0 = w[r], a1 = mk(0.0, 0.0);
    int c = 0;
    for (; c + 1 < ncols; c += 2) {
      const c128 v0 = V[c * ldv + r], v1 = V[(c + 1) * ldv + r];
      a0 = fmac(a0, v0, hs[c]);
      a1 = fmac(a1, v1, hs[c + 1]);
    }
    if (c < ncols) a0 = fmac(a0, V[c * ldv + r], hs[c]);
    w[r] = a0 + a1;
  }
}

// ---------------------------------------------------------------------------
// Gram-Schmidt in double-float arithmetic on the FP32 pipe (ortho = 3). The
// Krylov basis V is stored in double-float form (dfc, split once when a
// vector is normalised) and w is split once per projection, so the
// projection and the update read pre-split operands. Products use the exact
// FMA residual, sums the TwoSum transformation: about 46 correct bits.
// ---------------------------------------------------------------------------
// wdf = split(w)
__global__ void k_split(const c128* __restrict__ w, dfc* __restrict__ wdf, long long n,
                        const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) wdf[r] = split_c(w[r]);
}

// v (in place) = split(w / nrm): the new basis vector in double-float form
__global__ void k_scale_to_df(c128* __restrict__ v, long long n, const double* __restrict__ nrm,
                              const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  const double d = *nrm;
  if (!(d > 0.0)) return;
  const double s = 1.0 / d;
  dfc* out = reinterpret_cast<dfc*>(v);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    const c128 x = v[r];
    out[r] = split_c(mk(s * x.re, s * x.im));
  }
}

// Four columns per block: partial[c * gridDim.x + blk] = sum over the
// block's rows of conj(V_c) w for c = 4*blockIdx.y + 0..3 (< ncols); w is
// read once for the four.
constexpr int kDfCols = 4;

__global__ void __launch_bounds__(kThreads)
    k_dots_df(const dfc* __restrict__ V, long long ldv, int ncols, const dfc* __restrict__ w, long long n,
              c128* __restrict__ partial, const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  const int c0 = blockIdx.y * kDfCols;
  const int nc = min(kDfCols, ncols - c0);
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per;
  const long long r1 = min(n, r0 + per);
  float rh[kDfCols], rl[kDfCols], ih[kDfCols], il[kDfCols];
#pragma unroll
  for (int q = 0; q < kDfCols; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.f;
  for (long long r = r0 + threadIdx.x; r < r1; r += kThreads) {
    const dfc b = w[r];
    const dfl br = dfl_of(b.rh, b.rl), bi = dfl_of(b.ih, b.il);
    dfc a[kDfCols];
#pragma unroll
    for (int q = 0; q < kDfCols; ++q)
      if (q < nc) a[q] = V[(long long)(c0 + q) * ldv + r];
#pragma unroll
    for (int q = 0; q < kDfCols; ++q) {
      if (q >= nc) continue;
      const dfl ar = dfl_of(a[q].rh, a[q].rl), ai = dfl_of(a[q].ih, a[q].il);
      float p, t;
      // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
      df_prod(ar, br, p, t);
      df_acc(rh[q], rl[q], p, t);
      df_prod(ai, bi, p, t);
      df_acc(rh[q], rl[q], p, t);
      df_prod(ar, bi, p, t);
      df_acc(ih[q], il[q], p, t);
      df_prod(ai, br, p, t);
      df_acc(ih[q], il[q], -p, -t);
    }
  }
#pragma unroll
  for (int q = 0; q < kDfCols; ++q) {
    if (q >= nc) break;
    c128 s = block_sum(mk(df_to_d(rh[q], rl[q]), df_to_d(ih[q], il[q])));
    if (threadIdx.x == 0) partial[(long long)(c0 + q) * gridDim.x + blockIdx.x] = s;
  }
}

// w += sign * sum_c V_c h_c with double-float accumulation
__global__ void __launch_bounds__(kThreads)
    k_axpys_df(const dfc* __restrict__ V, long long ldv, int ncols, const c128* __restrict__ h, double sign,
               c128* __restrict__ w, long long n, const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  extern __shared__ dfc hsd[];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) hsd[c] = split_c(mk(sign * h[c].re, sign * h[c].im));
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    const dfc w0 = split_c(w[r]);
    float rh = w0.rh, rl = w0.rl, ih = w0.ih, il = w0.il;
    for (int c0 = 0; c0 < ncols; c0 += kDfCols) {
      dfc a[kDfCols];
#pragma unroll
      for (int q = 0; q < kDfCols; ++q)
        if (c0 + q < ncols) a[q] = V[(long long)(c0 + q) * ldv + r];   // loads first
#pragma unroll
      for (int q = 0; q < kDfCols; ++q) {
        if (c0 + q >= ncols) continue;
        const dfc hc = hsd[c0 + q];
        const dfl ar = dfl_of(a[q].rh, a[q].rl), ai = dfl_of(a[q].ih, a[q].il);
        const dfl hr = dfl_of(hc.rh, hc.rl), hi_ = dfl_of(hc.ih, hc.il);
        float p, t;
        // a h = (ar hr - ai hi) + i (ar hi + ai hr)
        df_prod(ar, hr, p, t);
        df_acc(rh, rl, p, t);
        df_prod(ai, hi_, p, t);
        df_acc(rh, rl, -p, -t);
        df_prod(ar, hi_, p, t);
        df_acc(ih, il, p, t);
        df_prod(ai, hr, p, t);
        df_acc(ih, il, p, t);
      }
    }
    w[r] = mk(df_to_d(rh, rl), df_to_d(ih, il));
  }
}

// ---------------------------------------------------------------------------
// Complex64 Krylov basis (ortho = 4). The basis vectors are the complex64
// roundings of the normalised w; the projection and the update use those
// values exactly (products of a float by a double-float as FMA residual
// pairs, double-float sums), so V takes 8 bytes per entry.
// ---------------------------------------------------------------------------
// a * b for a float a and a double-float b, as p + t
__device__ __forceinline__ void fdf_prod(float a, const dfl& b, float& p, float& t) {
  p = a * b.hi;
  const float e = fmaf(a, b.hi, -p);
  t = fmaf(a, b.lo, e);
}

__global__ void k_scale_to_c64(const c128* __restrict__ w, c64* __restrict__ v, long long n,
                               const double* __restrict__ nrm, const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  const double d = *nrm;
  if (!(d > 0.0)) return;
  const double s = 1.0 / d;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    const c128 x = w[r];
    v[r] = mk((float)(s * x.re), (float)(s * x.im));
  }
}

// Basis entries of the two stored forms: complex64 roundings (ortho = 4) or
// double-float pairs (ortho = 3). bprod_* gives the real or imaginary part of
// the entry times a double-float b as p + t (exact FMA residual of the
// leading product).
__device__ __forceinline__ void bprod_re(const c64& a, const dfl& b, float& p, float& t) { fdf_prod(a.re, b, p, t); }
__device__ __forceinline__ void bprod_im(const c64& a, const dfl& b, float& p, float& t) { fdf_prod(a.im, b, p, t); }
__device__ __forceinline__ void bprod_re(const dfc& a, const dfl& b, float& p, float& t) {
  df_prod(dfl_of(a.rh, a.rl), b, p, t);
}
__device__ __forceinline__ void bprod_im(const dfc& a, const dfl& b, float& p, float& t) {
  df_prod(dfl_of(a.ih, a.il), b, p, t);
}
template <typename B>
__device__ __forceinline__ B bzero();
template <>
__device__ __forceinline__ c64 bzero<c64>() { return mk(0.f, 0.f); }
template <>
__device__ __forceinline__ dfc bzero<dfc>() { return dfc{0.f, 0.f, 0.f, 0.f}; }

// partial[c * nrb + rb] = sum over row block rb's rows of conj(V_c) w, four
// columns per block, w read and split once per row of the block (eight
// columns were measured on the complex64 basis: 105 registers per thread,
// slower on c2 and c4). The blocks of one row block (its column groups) are
// consecutive in the grid, so they run together and their reads of the same
// rows of w after the first come from L2.
constexpr int kC64Cols = 4;

template <typename B>
__global__ void __launch_bounds__(kThreads)
    k_dots_b(const B* __restrict__ V, long long ldv, int ncols, const c128* __restrict__ w, int wdf, long long n,
             c128* __restrict__ partial, const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  constexpr int kDfCols = kC64Cols;
  const int ncg = (ncols + kDfCols - 1) / kDfCols;   // column groups
  const int cg = blockIdx.x % ncg, rb = blockIdx.x / ncg, nrb = gridDim.x / ncg;
  const int c0 = cg * kDfCols;
  const int nc = min(kDfCols, ncols - c0);
  const long long per = (n + nrb - 1) / nrb;
  const long long r0 = rb * per;
  const long long r1 = min(n, r0 + per);
  float rh[kDfCols], rl[kDfCols], ih[kDfCols], il[kDfCols];
#pragma unroll
  for (int q = 0; q < kDfCols; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.f;
  // two rows per iteration, all loads issued before the arithmetic
  for (long long r = r0 + threadIdx.x; r < r1; r += 2 * kThreads) {
    const bool two = r + kThreads < r1;
    c128 wv[2];
    B a[2][kDfCols];
    wv[0] = w[r];
    wv[1] = two ? w[r + kThreads] : mk(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int q = 0; q < kDfCols; ++q)
        a[u][q] = (q < nc && (u == 0 || two)) ? V[(long long)(c0 + q) * ldv + r + u * kThreads] : bzero<B>();
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // w held in double-float form already (wdf), or complex128 split here
      const dfc b = wdf ? *reinterpret_cast<const dfc*>(&wv[u]) : split_c(wv[u]);
      const dfl br = dfl_of(b.rh, b.rl), bi = dfl_of(b.ih, b.il);
#pragma unroll
      for (int q = 0; q < kDfCols; ++q) {
        if (q >= nc) continue;
        float p, t;
        // conj(a) w = (ar wr + ai wi) + i (ar wi - ai wr)
        bprod_re(a[u][q], br, p, t);
        df_acc(rh[q], rl[q], p, t);
        bprod_im(a[u][q], bi, p, t);
        df_acc(rh[q], rl[q], p, t);
        bprod_re(a[u][q], bi, p, t);
        df_acc(ih[q], il[q], p, t);
        bprod_im(a[u][q], br, p, t);
        df_acc(ih[q], il[q], -p, -t);
      }
    }
  }
  // the kDfCols sums of the block in one pass, in double-float on the FP32
  // pipe (FP64 runs at a small fraction of it here: summing in FP64 per
  // thread cost as much as the main loop): shuffles within each warp, one
  // barrier, the first warp adds the warps' values, one conversion per column
  __shared__ float4 red[kThreads / 32][kDfCols];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kDfCols; ++q) {
    float a = rh[q], b = rl[q], c = ih[q], d = il[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a2 = __shfl_xor_sync(0xffffffffu, a, o), b2 = __shfl_xor_sync(0xffffffffu, b, o);
      const float c2 = __shfl_xor_sync(0xffffffffu, c, o), d2 = __shfl_xor_sync(0xffffffffu, d, o);
      df_acc(a, b, a2, b2);
      df_acc(c, d, c2, d2);
    }
    if (lane == 0) red[wid][q] = make_float4(a, b, c, d);
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    float4 t = red[0][threadIdx.x];
#pragma unroll
    for (int u = 1; u < kThreads / 32; ++u) {
      const float4 v = red[u][threadIdx.x];
      df_acc(t.x, t.y, v.x, v.y);
      df_acc(t.z, t.w, v.z, v.w);
    }
    partial[(long long)(c0 + threadIdx.x) * nrb + rb] = mk(df_to_d(t.x, t.y), df_to_d(t.z, t.w));
  }
}

// w += sign * sum_c V_c h_c, double-float accumulation. With wdf, w is held
// in double-float form (read and written as dfc); with pnorm, the block's
// sum of |w|^2 (double-float, FP64 at the end) goes to pnorm[blockIdx.x].re.
template <typename B>
__global__ void __launch_bounds__(kThreads)
    k_axpys_b(const B* __restrict__ V, long long ldv, int ncols, const c128* __restrict__ h, double sign,
              c128* __restrict__ w, int wdf, c128* __restrict__ pnorm, long long n, const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  extern __shared__ dfc hsc[];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) hsc[c] = split_c(mk(sign * h[c].re, sign * h[c].im));
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  float nh = 0.f, nl = 0.f;   // sum of |w|^2 of this thread's rows
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    const dfc w0 = wdf ? reinterpret_cast<const dfc*>(w)[r] : split_c(w[r]);
    // two accumulator sets (even and odd columns) for two independent
    // dependency chains per part; added together at the end
    float rh[2] = {w0.rh, 0.f}, rl[2] = {w0.rl, 0.f}, ih[2] = {w0.ih, 0.f}, il[2] = {w0.il, 0.f};
    constexpr int kU = 2 * kC64Cols;   // basis entries loaded ahead of the arithmetic
    for (int c0 = 0; c0 < ncols; c0 += kU) {
      B a[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q)
        if (c0 + q < ncols) a[q] = V[(long long)(c0 + q) * ldv + r];   // loads first
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        if (c0 + q >= ncols) continue;
        const int u = q & 1;
        const dfc hc = hsc[c0 + q];
        const dfl hr = dfl_of(hc.rh, hc.rl), hi_ = dfl_of(hc.ih, hc.il);
        float p, t;
        // a h = (ar hr - ai hi) + i (ar hi + ai hr)
        bprod_re(a[q], hr, p, t);
        df_acc(rh[u], rl[u], p, t);
        bprod_im(a[q], hi_, p, t);
        df_acc(rh[u], rl[u], -p, -t);
        bprod_re(a[q], hi_, p, t);
        df_acc(ih[u], il[u], p, t);
        bprod_im(a[q], hr, p, t);
        df_acc(ih[u], il[u], p, t);
      }
    }
    df_acc(rh[0], rl[0], rh[1], rl[1]);
    df_acc(ih[0], il[0], ih[1], il[1]);
    df_norm(rh[0], rl[0]);
    df_norm(ih[0], il[0]);
    if (wdf) {
      dfc o;
      o.rh = rh[0];
      o.rl = rl[0];
      o.ih = ih[0];
      o.il = il[0];
      reinterpret_cast<dfc*>(w)[r] = o;
    } else {
      w[r] = mk(df_to_d(rh[0], rl[0]), df_to_d(ih[0], il[0]));
    }
    if (pnorm != nullptr) {
      // |w|^2 = rh^2 + 2 rh rl + ih^2 + 2 ih il (+ terms below 2^-46 relative)
      float p = rh[0] * rh[0];
      float t = fmaf(rh[0], rh[0], -p) + 2.f * rh[0] * rl[0];
      df_acc(nh, nl, p, t);
      p = ih[0] * ih[0];
      t = fmaf(ih[0], ih[0], -p) + 2.f * ih[0] * il[0];
      df_acc(nh, nl, p, t);
    }
  }
  if (pnorm != nullptr) {
    __shared__ float2 red[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a2 = __shfl_xor_sync(0xffffffffu, nh, o), b2 = __shfl_xor_sync(0xffffffffu, nl, o);
      df_acc(nh, nl, a2, b2);
    }
    if (lane == 0) red[wid] = make_float2(nh, nl);
    __syncthreads();
    if (threadIdx.x == 0) {
      float a = red[0].x, b = red[0].y;
      for (int u = 1; u < kThreads / 32; ++u) df_acc(a, b, red[u].x, red[u].y);
      pnorm[blockIdx.x] = mk(df_to_d(a, b), 0.0);
    }
  }
}

// v = w / nrm in double-float form, both in double-float form (in place
// allowed): 1/nrm as a double-float pair from an FP32 reciprocal and one
// Newton step, products as FMA residual pairs, each part renormalised
// (|lo| <= ulp(hi)/2) so that the stored basis is a valid split
__global__ void k_scale_df_to_df(const dfc* w, dfc* v, long long n, const double* __restrict__ nrm,
                                 const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  const double d = *nrm;
  if (!(d > 0.0)) return;
  const dfl dd = split_d(d);
  const float s0 = 1.f / dd.hi;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (!(dd.hi > 0.f) || !(s0 < 3e38f)) {
    // nrm outside the FP32 range: FP64 (never on a regular step)
    const double sd = 1.0 / d;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
      const dfc x = w[r];
      v[r] = split_c(mk(sd * ((double)x.rh + (double)x.rl), sd * ((double)x.ih + (double)x.il)));
    }
    return;
  }
  const float r0 = fmaf(-dd.hi, s0, 1.f) - dd.lo * s0;
  const dfl s = dfl_of(s0, s0 * r0);
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    const dfc x = w[r];
    float p, t;
    dfc o;
    df_prod(dfl_of(x.rh, x.rl), s, p, t);
    o.rh = p + t;
    o.rl = t - (o.rh - p);
    df_prod(dfl_of(x.ih, x.il), s, p, t);
    o.ih = p + t;
    o.il = t - (o.ih - p);
    v[r] = o;
  }
}

// v = fl32(w / nrm) for w in double-float form: 1/nrm as a double-float
// pair from an FP32 reciprocal and one Newton step, products as FMA
// residual pairs (FP32 pipe only)
__global__ void k_scale_df_to_c64(const dfc* __restrict__ w, c64* __restrict__ v, long long n,
                                  const double* __restrict__ nrm, const KState* __restrict__ kst) {
  if (skip(kst, 0)) return;
  const double d = *nrm;
  if (!(d > 0.0)) return;
  const dfl dd = split_d(d);
  const float s0 = 1.f / dd.hi;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (!(dd.hi > 0.f) || !(s0 < 3e38f)) {
    // nrm outside the FP32 range: FP64 (never on a regular step)
    const double sd = 1.0 / d;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
      const dfc x = w[r];
      v[r] = mk((float)(sd * ((double)x.rh + (double)x.rl)), (float)(sd * ((double)x.ih + (double)x.il)));
    }
    return;
  }
  // 1 - d s0 in double-float, then s = s0 + s0 (1 - d s0)
  const float r0 = fmaf(-dd.hi, s0, 1.f) - dd.lo * s0;
  const float sh = s0, sl = s0 * r0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    const dfc x = w[r];
    float p = x.rh * sh;
    const float vr = p + (fmaf(x.rh, sh, -p) + fmaf(x.rh, sl, x.rl * sh));
    p = x.ih * sh;
    const float vi = p + (fmaf(x.ih, sh, -p) + fmaf(x.ih, sl, x.il * sh));
    v[r] = mk(vr, vi);
  }
}

__global__ void k_add(c128* __restrict__ dst, const c128* __restrict__ src, int cnt,
                      const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) dst[i] = dst[i] + src[i];
}

// ||w|| from the partial sums of conj(w) w
__global__ void k_norm_finish(const c128* __restrict__ partial, int G, double* out, c128* hslot,
                              const KState* __restrict__ kst, int gate) {
  if (skip(kst, gate)) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < G; b += 32) s += partial[b].re;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    double nv = sqrt(s);
    *out = nv;
    if (hslot) *hslot = mk(nv, 0.0);
  }
}

__global__ void k_scale_inv(c128* __restrict__ v, long long n, const double* __restrict__ nrm,
                            const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  const double d = *nrm;
  if (!(d > 0.0)) return;
  const double s = 1.0 / d;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) v[r] = s * v[r];
}

// DGKS test after one classical Gram-Schmidt pass: hcol[j+1] holds ||w||^2
// from before the projection, kst->hnorm = ||w'|| after it. A second pass is
// due when ||w'|| < ||w|| / sqrt(2); otherwise ||w'|| is the new subdiagonal.
// eta2 = 0 disables the second pass (classical Gram-Schmidt once).
__global__ void k_reorth_decide(KState* kst, c128* hcol, int j, double eta2) {
  if (threadIdx.x != 0 || kst->stop) return;
  const double w2 = hcol[j + 1].re;
  const double nu = kst->hnorm;
  const int need = (nu * nu < eta2 * w2) ? 1 : 0;
  kst->reorth = need;
  kst->reorths += need;
  if (!need) hcol[j + 1] = mk(nu, 0.0);
}

// Start of an Arnoldi cycle: beta = ||r0|| (in kst->hnorm), g = beta e_1.
__global__ void k_cycle_init(KState* kst, c128* gvec, int m, double rtol, double* hist) {
  const double beta = kst->hnorm;
  for (int i = threadIdx.x; i <= m; i += blockDim.x) gvec[i] = mk(i == 0 ? beta : 0.0, 0.0);
  if (threadIdx.x == 0) {
    kst->jdone = 0;
    kst->stop = 0;
    kst->conv = 0;
    kst->breakdown = 0;
    kst->beta0 = beta;
    const double est = beta / kst->bnorm;
    kst->est = est;
    if (hist) hist[kst->total] = est;
    if (!isfinite(est)) {
      kst->nan = 1;
      kst->stop = 1;
    } else if (est <= rtol || beta == 0.0) {
      kst->conv = 1;
      kst->stop = 1;
    }
  }
}

// Givens step j of the cycle (one thread): rotate the new Hessenberg column,
// build the new rotation, update g and the residual estimate, decide stop.
// One warp applies the previous rotations to column j of H (givens_prev_warp)
// and lane 0 forms the new rotation.
__global__ void k_givens(KState* kst, c128* H, int ldh, double* cs, c128* sn, c128* gvec, int j, double rtol,
                         int mcycle, int maxit, double* hist, double cfloor) {
  if (kst->stop) return;
  const int lane = threadIdx.x;
  c128* col = H + (long long)j * ldh;
  const c128 cj = givens_prev_warp(col, cs, sn, j, lane);
  if (lane != 0) return;
  col[j] = cj;
  c128 a = col[j], b = col[j + 1];
  double aa = sqrt(abs2(a)), bb = sqrt(abs2(b));
  double c;
  c128 s, r;
  if (bb == 0.0) {
    c = 1.0; s = mk(0.0, 0.0); r = a;
  } else if (aa == 0.0) {
    c = 0.0; s = mk(1.0, 0.0); r = b;
  } else {
    double nrm = hypot(aa, bb);
    c128 ph = (1.0 / aa) * a;
    c = aa / nrm;
    s = (1.0 / nrm) * (ph * conj(b));
    r = nrm * ph;
  }
  col[j] = r;
  col[j + 1] = mk(0.0, 0.0);
  cs[j] = c;
  sn[j] = s;
  c128 gj = gvec[j];
  gvec[j + 1] = mk(0.0, 0.0) - conj(s) * gj;
  gvec[j] = c * gj;
  kst->total += 1;
  kst->jdone = j + 1;
  const double est = sqrt(abs2(gvec[j + 1])) / kst->bnorm;
  kst->est = est;
  if (hist) hist[kst->total] = est;
  if (!isfinite(est)) { kst->nan = 1; kst->stop = 1; }
  if (est <= rtol) { kst->conv = 1; kst->stop = 1; }
  if (kst->hnorm == 0.0) { kst->breakdown = 1; kst->stop = 1; }
  if (j + 1 >= mcycle || kst->total >= maxit) kst->stop = 1;
  // the attainable reduction of one cycle (complex64 basis): restart from the
  // true residual instead of iterating on a stagnating estimate
  if (sqrt(abs2(gvec[j + 1])) <= cfloor * kst->beta0) kst->stop = 1;
}

// y = H(0:m,0:m)^-1 g for the upper-triangular Hessenberg after rotations,
// m = kst->jdone; one warp.
__global__ void k_backsolve(const c128* __restrict__ H, int ldh, const c128* __restrict__ gvec,
                            const KState* __restrict__ kst, c128* __restrict__ y) {
  const int m = kst->jdone;
  const int l = threadIdx.x;
  for (int i = m - 1; i >= 0; --i) {
    c128 s = mk(0.0, 0.0);
    for (int c = i + 1 + l; c < m; c += 32) s = s + H[(long long)c * ldh + i] * y[c];
    s = warp_sum(s);
    if (l == 0) y[i] = cdiv(gvec[i] - s, H[(long long)i * ldh + i]);
    __syncwarp();
    __threadfence_block();
  }
}

__global__ void k_axpy(c128* __restrict__ x, const c128* __restrict__ v, long long n, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) x[r] = x[r] + v[r];
}

// z += alpha c with alpha = hv[0] / hv[1] (the minimal-residual step of a
// correction c: hv[0] = <A c, r1>, hv[1] = <A c, A c>); nothing when hv[1] = 0
// z += alpha c, alpha = <Ac, r1> / ||Ac||^2 (hv[0], hv[1]; hv[2] = ||r1||^2):
// the minimal-residual step of the learned stage. Block 0 also records the
// fraction of ||r1||^2 the step removes, |<Ac, r1>|^2 / (||Ac||^2 ||r1||^2),
// as the stage's gain (largest over the solve, KState::lgain). z in
// complex128, or in double-float form (zdf).
__global__ void k_mr_axpy(c128* __restrict__ z, const c128* __restrict__ c, const c128* __restrict__ hv,
                          long long n, KState* __restrict__ kst, int zdf) {
  if (kst != nullptr && kst->stop) return;
  const double d = hv[1].re;
  if (!(d > 0.0)) return;
  const c128 a = mk(hv[0].re / d, hv[0].im / d);
  if (kst != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    const double rr = hv[2].re;
    const double gain = rr > 0.0 ? abs2(hv[0]) / (d * rr) : 0.0;
    kst->lgain = fmax(kst->lgain, gain);
    kst->ldirs += 1;
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += stride) {
    if (zdf) {
      dfc* zd = reinterpret_cast<dfc*>(z);
      const dfc v = zd[r];
      zd[r] = split_c(fmac(mk(df_to_d(v.rh, v.rl), df_to_d(v.ih, v.il)), a, c[r]));
    } else {
      z[r] = fmac(z[r], a, c[r]);
    }
  }
}

unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)(g_num_sms > 0 ? g_num_sms : 152) * 16;
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

int dot_blocks() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 152;
  }
  return kDotBlocksPerSM * g_num_sms;
}

cudaError_t launch_spmv(long long n, int nx, const c128* D, const c128* CW, const c128* CS, const c128* CSW,
                        const c128* x, const c128* bsub, c128* y, const KState* kst, cudaStream_t st, int bsub_kind,
                        int xdf) {
  unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
  k_spmv<<<blocks, kThreads, 0, st>>>(n, nx, D, CW, CS, CSW, x, bsub, bsub_kind, y, kst, xdf);
  return cudaGetLastError();
}

cudaError_t launch_spmv_df(long long n, int nx, const void* D, const void* CW, const void* CS, const void* CSW,
                           const c128* x, c128* y, const KState* kst, cudaStream_t st, int out_df, int in_df) {
  const int ny = (int)(n / nx);
  dim3 grid((nx + kSpTX - 1) / kSpTX, (ny + kSpTY - 1) / kSpTY);
  k_spmv_df<<<grid, kSpTX * kSpTY, 0, st>>>(nx, ny, (const dfc*)D, (const dfc*)CW, (const dfc*)CS, (const dfc*)CSW,
                                            x, y, out_df, in_df, kst);
  return cudaGetLastError();
}

cudaError_t launch_dots(const c128* V, long long ldv, int ncols, const c128* w, long long n, c128* partial,
                        const KState* kst, int gate, cudaStream_t st) {
  dim3 grid(dot_blocks(), ncols);
  k_dots<<<grid, kThreads, 0, st>>>(V, ldv, w, n, partial, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_dots_finish(const c128* partial, int ncols, c128* out, int accumulate, const KState* kst,
                               int gate, cudaStream_t st) {
  int per = kThreads / 32;
  k_dots_finish<<<(ncols + per - 1) / per, kThreads, 0, st>>>(partial, dot_blocks(), ncols, out, accumulate,
                                                              kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_axpys(const c128* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                         long long n, const KState* kst, int gate, cudaStream_t st) {
  dot_blocks();
  size_t smem = (size_t)ncols * sizeof(c128);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axpys, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_axpys<<<grid_for(n, kThreads), kThreads, smem, st>>>(V, ldv, ncols, h, sign, w, n, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_split(const c128* w, void* wdf, long long n, const KState* kst, cudaStream_t st) {
  dot_blocks();
  k_split<<<grid_for(n, kThreads), kThreads, 0, st>>>(w, (dfc*)wdf, n, kst);
  return cudaGetLastError();
}

cudaError_t launch_scale_to_df(c128* v, long long n, const double* nrm, const KState* kst, cudaStream_t st) {
  dot_blocks();
  k_scale_to_df<<<grid_for(n, kThreads), kThreads, 0, st>>>(v, n, nrm, kst);
  return cudaGetLastError();
}

cudaError_t launch_dots_df(const void* V, long long ldv, int ncols, const void* wdf, long long n, c128* partial,
                           const KState* kst, int gate, cudaStream_t st) {
  dim3 grid(dot_blocks(), (ncols + kDfCols - 1) / kDfCols);
  k_dots_df<<<grid, kThreads, 0, st>>>((const dfc*)V, ldv, ncols, (const dfc*)wdf, n, partial, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_axpys_df(const void* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                            long long n, const KState* kst, int gate, cudaStream_t st) {
  dot_blocks();
  size_t smem = (size_t)ncols * sizeof(dfc);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axpys_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_axpys_df<<<grid_for(n, kThreads), kThreads, smem, st>>>((const dfc*)V, ldv, ncols, h, sign, w, n, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_add(c128* dst, const c128* src, int cnt, const KState* kst, int gate, cudaStream_t st) {
  k_add<<<(cnt + 127) / 128, 128, 0, st>>>(dst, src, cnt, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_norm_finish(const c128* partial, double* out, c128* hslot, const KState* kst, int gate,
                               cudaStream_t st, int nparts) {
  k_norm_finish<<<1, 32, 0, st>>>(partial, nparts > 0 ? nparts : dot_blocks(), out, hslot, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_scale_df_to_c64(const void* w, void* v, long long n, const double* nrm, const KState* kst,
                                   cudaStream_t st) {
  dot_blocks();
  k_scale_df_to_c64<<<grid_for(n, kThreads), kThreads, 0, st>>>((const dfc*)w, (c64*)v, n, nrm, kst);
  return cudaGetLastError();
}

cudaError_t launch_scale_inv(c128* v, long long n, const double* nrm, const KState* kst, cudaStream_t st) {
  dot_blocks();
  k_scale_inv<<<grid_for(n, kThreads), kThreads, 0, st>>>(v, n, nrm, kst);
  return cudaGetLastError();
}

cudaError_t launch_cycle_init(KState* kst, c128* gvec, int m, double rtol, double* hist, cudaStream_t st) {
  k_cycle_init<<<1, 128, 0, st>>>(kst, gvec, m, rtol, hist);
  return cudaGetLastError();
}

cudaError_t launch_givens(KState* kst, c128* H, int ldh, double* cs, c128* sn, c128* gvec, int j, double rtol,
                          int mcycle, int maxit, double* hist, cudaStream_t st, double cfloor) {
  k_givens<<<1, 32, 0, st>>>(kst, H, ldh, cs, sn, gvec, j, rtol, mcycle, maxit, hist, cfloor);
  return cudaGetLastError();
}

cudaError_t launch_reorth_decide(KState* kst, c128* hcol, int j, double eta2, cudaStream_t st) {
  k_reorth_decide<<<1, 32, 0, st>>>(kst, hcol, j, eta2);
  return cudaGetLastError();
}

cudaError_t launch_backsolve(const c128* H, int ldh, const c128* gvec, const KState* kst, c128* y,
                             cudaStream_t st) {
  k_backsolve<<<1, 32, 0, st>>>(H, ldh, gvec, kst, y);
  return cudaGetLastError();
}

cudaError_t launch_scale_to_c64(const c128* w, void* v, long long n, const double* nrm, const KState* kst,
                                cudaStream_t st) {
  dot_blocks();
  k_scale_to_c64<<<grid_for(n, kThreads), kThreads, 0, st>>>(w, (c64*)v, n, nrm, kst);
  return cudaGetLastError();
}

template <typename B>
cudaError_t launch_dots_bt(const void* V, long long ldv, int ncols, const c128* w, long long n, c128* partial,
                           const KState* kst, cudaStream_t st, int wdf) {
  // row blocks x column groups, the column group varying fastest
  const unsigned grid = (unsigned)dot_blocks() * (unsigned)((ncols + kC64Cols - 1) / kC64Cols);
  k_dots_b<B><<<grid, kThreads, 0, st>>>((const B*)V, ldv, ncols, w, wdf, n, partial, kst);
  return cudaGetLastError();
}

template <typename B>
cudaError_t launch_axpys_bt(const void* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                            long long n, const KState* kst, cudaStream_t st, int wdf, c128* pnorm, int* nblocks) {
  dot_blocks();
  const size_t smem = (size_t)ncols * sizeof(dfc);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axpys_b<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned g = grid_for(n, kThreads);
  if (nblocks) *nblocks = (int)g;
  k_axpys_b<B><<<g, kThreads, smem, st>>>((const B*)V, ldv, ncols, h, sign, w, wdf, pnorm, n, kst);
  return cudaGetLastError();
}

cudaError_t launch_dots_c64b(const void* V, long long ldv, int ncols, const c128* w, long long n, c128* partial,
                             const KState* kst, cudaStream_t st, int wdf) {
  return launch_dots_bt<c64>(V, ldv, ncols, w, n, partial, kst, st, wdf);
}

cudaError_t launch_axpys_c64b(const void* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                              long long n, const KState* kst, cudaStream_t st, int wdf, c128* pnorm,
                              int* nblocks) {
  return launch_axpys_bt<c64>(V, ldv, ncols, h, sign, w, n, kst, st, wdf, pnorm, nblocks);
}

cudaError_t launch_dots_dfb(const void* V, long long ldv, int ncols, const void* wdf, long long n, c128* partial,
                            const KState* kst, cudaStream_t st) {
  return launch_dots_bt<dfc>(V, ldv, ncols, (const c128*)wdf, n, partial, kst, st, 1);
}

cudaError_t launch_axpys_dfb(const void* V, long long ldv, int ncols, const c128* h, double sign, void* wdf,
                             long long n, const KState* kst, cudaStream_t st, c128* pnorm, int* nblocks) {
  return launch_axpys_bt<dfc>(V, ldv, ncols, h, sign, (c128*)wdf, n, kst, st, 1, pnorm, nblocks);
}

cudaError_t launch_scale_df_to_df(const void* w, void* v, long long n, const double* nrm, const KState* kst,
                                  cudaStream_t st) {
  dot_blocks();
  k_scale_df_to_df<<<grid_for(n, kThreads), kThreads, 0, st>>>((const dfc*)w, (dfc*)v, n, nrm, kst);
  return cudaGetLastError();
}

cudaError_t launch_mr_axpy(c128* z, const c128* c, const c128* hv, long long n, KState* kst, cudaStream_t st,
                           int zdf) {
  dot_blocks();
  k_mr_axpy<<<grid_for(n, kThreads), kThreads, 0, st>>>(z, c, hv, n, kst, zdf);
  return cudaGetLastError();
}

// The residual check of a sweep of Algorithm 1: rel = ||r|| / ||b|| from
// kst->hnorm and kst->bnorm, into hist[it]; the stop flag once rel <= rtol,
// it reaches maxit, or rel is not finite (every later kernel of the loop
// returns at once).
__global__ void k_rich_check(KState* kst, double rtol, int maxit, int it, double* hist) {
  if (kst->stop) return;
  const double rel = kst->bnorm > 0.0 ? kst->hnorm / kst->bnorm : 0.0;
  hist[it] = rel;
  kst->est = rel;
  kst->total = it;
  if (!isfinite(rel)) {
    kst->nan = 1;
    kst->stop = 1;
  } else if (rel <= rtol) {
    kst->conv = 1;
    kst->stop = 1;
  } else if (it >= maxit) {
    kst->stop = 1;
  }
}

cudaError_t launch_rich_check(KState* kst, double rtol, int maxit, int it, double* hist, cudaStream_t st) {
  k_rich_check<<<1, 1, 0, st>>>(kst, rtol, maxit, it, hist);
  return cudaGetLastError();
}

cudaError_t launch_axpy_state(c128* x, const c128* v, long long n, cudaStream_t st, const KState* kst) {
  dot_blocks();
  k_axpy<<<grid_for(n, kThreads), kThreads, 0, st>>>(x, v, n, kst);
  return cudaGetLastError();
}

}  // namespace rp
