// Kernels of the batched form: many independent problems whose vectors are
// concatenated, problem q at [goff_q, goff_q + n_q) with goff_q a multiple of
// the 2048-row tile, so that every tile belongs to one problem
// (tile_prob[t]). Each kernel below handles whole tiles and skips the tiles
// of problems that its gate excludes:
//   gate 0: every problem; gate 1: problems whose cycle is running
//   (kst[q].stop == 0); gate 2: problems still being solved (kst[q].live).
// The FGMRES of Section 4.1 runs in lockstep over the problems: step j of
// every running problem in the same launches. The kernels of one Arnoldi
// step read j from device memory (ctl->j), so the step can be captured once
// as a CUDA graph and replayed; k_bnext advances j at the end of the step.
// Rows between problems (the tile padding) are written as zero.
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

constexpr int kBT = 256;                   // threads per tile block
constexpr double kBasisFloor = 1e-6;       // per-cycle reduction trusted on a complex64 basis
constexpr int kRows = kBatchTile / kBT;    // rows per thread

__device__ __forceinline__ bool gated(const KState* kst, int q, int gate) {
  if (gate == 1) return kst[q].stop != 0;
  if (gate == 2) return kst[q].live == 0;
  return false;
}

__device__ __forceinline__ c128 warp_sum(c128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the block of v (valid in thread 0)
__device__ __forceinline__ double block_sumd(double v) {
  __shared__ double red[kBT / 32];
  v = warp_sumd(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < kBT / 32 ? red[threadIdx.x] : 0.0;
    s = warp_sumd(s);
  }
  return s;
}

// ---------------------------------------------------------------------------
// Prolongation: z_q = sum_j R_j^T (chi_j .* x_j) for every problem, one tile
// per block; the (at most four) covering subdomains of a node are summed in a
// fixed order. sub_index maps a problem's natural subdomain index
// (sub0 + qy*px + qx) to its position in the launch order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBT)
    k_bprolong(const int* __restrict__ tile_prob, const Geo* __restrict__ geos, const SubDesc* __restrict__ subs,
               const int* __restrict__ sub_index, const cx<R>* __restrict__ Y, c128* __restrict__ zbase,
               long long ldz, const int* __restrict__ jptr, const KState* __restrict__ kst, int gate, int zdf) {
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (gated(kst, q, gate)) return;
  const Geo& g = geos[q];
  const int nx = g.nx, n = g.n, o = g.ovlp, Mx = g.Mx, My = g.My, px = g.px, py = g.py, sub0 = g.sub0;
  const long long goff = g.goff;
  c128* z = zbase + (jptr ? (long long)(*jptr) * ldz : 0);
  const Boxes bxs = boxes_of(Mx, px), bys = boxes_of(My, py);
#pragma unroll 1
  for (int s = 0; s < kRows; ++s) {
    const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
    const int lr = (int)(r - goff);   // < 2^31 within a problem
    if (lr >= n) {
      z[r] = mk(0.0, 0.0);
      continue;
    }
    const int j = lr / nx + 1, i = lr - (j - 1) * nx + 1;
    const int2 cxr = cover_range(bxs, i, o), cyr = cover_range(bys, j, o);
    const int qx0 = cxr.x, qx1 = cxr.y, qy0 = cyr.x, qy1 = cyr.y;
    if constexpr (sizeof(R) == sizeof(float)) {
      if (zdf) {
        // complex64 local values summed in double-float into the dfc form
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
        for (int qy = qy0; qy <= qy1; ++qy) {
          for (int qx = qx0; qx <= qx1; ++qx) {
            const SubDesc& sd = subs[sub_index[sub0 + qy * px + qx]];
            const int li = i - sd.ix0, lj = j - sd.iy0;
            if (li < 0 || li >= sd.nlx || lj < 0 || lj >= sd.nly) continue;
            const cx<R> v = Y[sd.v_off + (long long)lj * sd.nlx + li];
            df_acc(rh, rl, v.re, 0.f);
            df_acc(ih, il, v.im, 0.f);
          }
        }
        df_norm(rh, rl);
        df_norm(ih, il);
        dfc o;
        o.rh = rh;
        o.rl = rl;
        o.ih = ih;
        o.il = il;
        reinterpret_cast<dfc*>(z)[r] = o;
        continue;
      }
    }
    double re = 0.0, im = 0.0;
    for (int qy = qy0; qy <= qy1; ++qy) {
      for (int qx = qx0; qx <= qx1; ++qx) {
        const SubDesc& sd = subs[sub_index[sub0 + qy * px + qx]];
        const int li = i - sd.ix0, lj = j - sd.iy0;
        if (li < 0 || li >= sd.nlx || lj < 0 || lj >= sd.nly) continue;
        const cx<R> v = Y[sd.v_off + (long long)lj * sd.nlx + li];
        re += (double)v.re;
        im += (double)v.im;
      }
    }
    z[r] = mk(re, im);
  }
}

// ---------------------------------------------------------------------------
// y = A x (bsub == nullptr) or y = bsub - A x with each problem's 7-point
// stencil; x = xbase + (*jptr) * ldx when jptr is set. With pnorm set, the
// block also writes sum |y|^2 over its tile to pnorm[t].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBT)
    k_bspmv(const int* __restrict__ tile_prob, const Geo* __restrict__ geos, const c128* __restrict__ D,
            const c128* __restrict__ CW, const c128* __restrict__ CS, const c128* __restrict__ CSW,
            const c128* __restrict__ xbase, long long ldx, const int* __restrict__ jptr,
            const c128* __restrict__ bsub, c128* __restrict__ y, double* __restrict__ pnorm,
            const KState* __restrict__ kst, int gate) {
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (gated(kst, q, gate)) return;
  const long long goff = geos[q].goff;
  const int nx = geos[q].nx, n = geos[q].n;
  const c128* x = xbase + (jptr ? (long long)(*jptr) * ldx : 0);
  double nrm = 0.0;
#pragma unroll 2
  for (int s = 0; s < kRows; ++s) {
    const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
    const int lr = (int)(r - goff);
    if (lr >= n) {
      y[r] = mk(0.0, 0.0);
      continue;
    }
    c128 a0 = mk(0.0, 0.0), a1 = mk(0.0, 0.0);
    a0 = fmac(a0, D[r], x[r]);
    if (lr >= 1) a1 = fmac(a1, CW[r], x[r - 1]);
    if (lr + 1 < n) a0 = fmac(a0, CW[r + 1], x[r + 1]);
    if (lr >= nx) a1 = fmac(a1, CS[r], x[r - nx]);
    if (lr + nx < n) a0 = fmac(a0, CS[r + nx], x[r + nx]);
    if (lr >= nx + 1) a1 = fmac(a1, CSW[r], x[r - nx - 1]);
    if (lr + nx + 1 < n) a0 = fmac(a0, CSW[r + nx + 1], x[r + nx + 1]);
    c128 v = a0 + a1;
    if (bsub) v = bsub[r] - v;
    y[r] = v;
    nrm = fma(v.re, v.re, fma(v.im, v.im, nrm));
  }
  if (pnorm) {
    const double s = block_sumd(nrm);
    if (threadIdx.x == 0) pnorm[t] = s;
  }
}

// The Arnoldi product w = A z_j of step j with the coefficients in
// double-float form (split once at set-up) and double-float products and
// sums; the cycle-start residual b - A x keeps the FP64 k_bspmv.
__device__ __forceinline__ void bcmac_df(float& rh, float& rl, float& ih, float& il, const dfc& a, const dfc& x) {
  const dfl ar = dfl_of(a.rh, a.rl), ai = dfl_of(a.ih, a.il);
  const dfl xr = dfl_of(x.rh, x.rl), xi = dfl_of(x.ih, x.il);
  float p, t;
  df_prod(ar, xr, p, t);
  df_acc(rh, rl, p, t);
  df_prod(ai, xi, p, t);
  df_acc(rh, rl, -p, -t);
  df_prod(ar, xi, p, t);
  df_acc(ih, il, p, t);
  df_prod(ai, xr, p, t);
  df_acc(ih, il, p, t);
}

__global__ void __launch_bounds__(kBT)
    k_bspmv_df(const int* __restrict__ tile_prob, const Geo* __restrict__ geos, const dfc* __restrict__ D,
               const dfc* __restrict__ CW, const dfc* __restrict__ CS, const dfc* __restrict__ CSW,
               const c128* __restrict__ xbase, long long ldx, const int* __restrict__ jptr, c128* __restrict__ y,
               int xdf, const KState* __restrict__ kst) {
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (kst[q].stop) return;
  const long long goff = geos[q].goff;
  const int nx = geos[q].nx, n = geos[q].n;
  const c128* x = xbase + (long long)(*jptr) * ldx;
  // x in double-float form (xdf) or complex128 split here; y written as dfc
  auto X = [&](long long k) -> dfc { return xdf ? reinterpret_cast<const dfc*>(x)[k] : split_c(x[k]); };
  dfc* yd = reinterpret_cast<dfc*>(y);
#pragma unroll 2
  for (int s = 0; s < kRows; ++s) {
    const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
    const int lr = (int)(r - goff);
    dfc o = {0.f, 0.f, 0.f, 0.f};
    if (lr >= n) {
      yd[r] = o;
      continue;
    }
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    bcmac_df(rh, rl, ih, il, D[r], X(r));
    if (lr >= 1) bcmac_df(rh, rl, ih, il, CW[r], X(r - 1));
    if (lr + 1 < n) bcmac_df(rh, rl, ih, il, CW[r + 1], X(r + 1));
    if (lr >= nx) bcmac_df(rh, rl, ih, il, CS[r], X(r - nx));
    if (lr + nx < n) bcmac_df(rh, rl, ih, il, CS[r + nx], X(r + nx));
    if (lr >= nx + 1) bcmac_df(rh, rl, ih, il, CSW[r], X(r - nx - 1));
    if (lr + nx + 1 < n) bcmac_df(rh, rl, ih, il, CSW[r + nx + 1], X(r + nx + 1));
    df_norm(rh, rl);
    df_norm(ih, il);
    o.rh = rh;
    o.rl = rl;
    o.ih = ih;
    o.il = il;
    yd[r] = o;
  }
}

// ---------------------------------------------------------------------------
// Gram-Schmidt of step j in double-float arithmetic on a complex64 basis
// (the basis vectors are the complex64 roundings of w/||w||, used exactly as
// stored; products of a float by the double-float split of w or h are FMA
// residual pairs, sums are double-float):
// k_bdots_df: partial[c * ntiles + t] = sum over tile t of conj(V_c) w,
//   c = 0..j; the tile's rows of w are split once and held in registers,
//   the columns are read four at a time; per-warp sums are kept in shared
//   memory and reduced across the warps once at the end.
// ---------------------------------------------------------------------------
constexpr int kBCols = 4;

// a * b for a float a and a double-float b, as p + t
__device__ __forceinline__ void fdf_mul(float a, const dfl& b, float& p, float& t) {
  p = a * b.hi;
  const float e = fmaf(a, b.hi, -p);
  t = fmaf(a, b.lo, e);
}

__global__ void __launch_bounds__(kBT)
    k_bdots_df(const int* __restrict__ tile_prob, const c64* __restrict__ V, long long ldv,
               const c128* __restrict__ w, const int* __restrict__ jptr, c128* __restrict__ partial, int ntiles,
               const KState* __restrict__ kst) {
  extern __shared__ float4 wsum[];   // [ncols][kBT / 32] double-float sums (rh, rl, ih, il)
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (kst[q].stop) return;
  const int ncols = *jptr + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long r0 = (long long)t * kBatchTile + threadIdx.x;
  dfl wr[kRows], wi[kRows];
#pragma unroll
  for (int s = 0; s < kRows; ++s) {
    const dfc b = reinterpret_cast<const dfc*>(w)[r0 + s * kBT];   // w in double-float form
    wr[s] = dfl_of(b.rh, b.rl);
    wi[s] = dfl_of(b.ih, b.il);
  }
  for (int c0 = 0; c0 < ncols; c0 += kBCols) {
    float rh[kBCols], rl[kBCols], ih[kBCols], il[kBCols];
#pragma unroll
    for (int u = 0; u < kBCols; ++u) rh[u] = rl[u] = ih[u] = il[u] = 0.f;
#pragma unroll
    for (int s = 0; s < kRows; ++s) {
      c64 a[kBCols];
#pragma unroll
      for (int u = 0; u < kBCols; ++u)
        if (c0 + u < ncols) a[u] = V[(long long)(c0 + u) * ldv + r0 + s * kBT];
#pragma unroll
      for (int u = 0; u < kBCols; ++u) {
        if (c0 + u >= ncols) continue;
        float p, e;
        // conj(a) w = (ar wr + ai wi) + i (ar wi - ai wr)
        fdf_mul(a[u].re, wr[s], p, e);
        df_acc(rh[u], rl[u], p, e);
        fdf_mul(a[u].im, wi[s], p, e);
        df_acc(rh[u], rl[u], p, e);
        fdf_mul(a[u].re, wi[s], p, e);
        df_acc(ih[u], il[u], p, e);
        fdf_mul(a[u].im, wr[s], p, e);
        df_acc(ih[u], il[u], -p, -e);
      }
    }
    // warp sums in double-float on the FP32 pipe (an FP64 sum per thread
    // and column cost more than the products here)
#pragma unroll
    for (int u = 0; u < kBCols; ++u) {
      if (c0 + u >= ncols) break;
      float a = rh[u], b = rl[u], c = ih[u], d = il[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float a2 = __shfl_xor_sync(0xffffffffu, a, o), b2 = __shfl_xor_sync(0xffffffffu, b, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, o), d2 = __shfl_xor_sync(0xffffffffu, d, o);
        df_acc(a, b, a2, b2);
        df_acc(c, d, c2, d2);
      }
      if (lane == 0) wsum[(c0 + u) * (kBT / 32) + wid] = make_float4(a, b, c, d);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += kBT) {
    float4 s4 = wsum[c * (kBT / 32)];
#pragma unroll
    for (int u = 1; u < kBT / 32; ++u) {
      const float4 v = wsum[c * (kBT / 32) + u];
      df_acc(s4.x, s4.y, v.x, v.y);
      df_acc(s4.z, s4.w, v.z, v.w);
    }
    partial[(long long)c * ntiles + t] = mk(df_to_d(s4.x, s4.y), df_to_d(s4.z, s4.w));
  }
}

// H_q(c, j) = sum over problem q's tiles of partial[c][t], c = 0..j; one
// block per problem, one warp per column.
__global__ void __launch_bounds__(kBT)
    k_bdots_finish(const int* __restrict__ tile0, const int* __restrict__ tile1, const c128* __restrict__ partial,
                   int ntiles, const int* __restrict__ jptr, c128* __restrict__ H, int ldh, long long hstride,
                   const KState* __restrict__ kst) {
  const int q = blockIdx.x;
  if (kst[q].stop) return;
  const int j = *jptr;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int a = tile0[q], b = tile1[q];
  c128* col = H + q * hstride + (long long)j * ldh;
  for (int c = wid; c <= j; c += kBT / 32) {
    c128 s = mk(0.0, 0.0);
    for (int u = a + lane; u < b; u += 32) s = s + partial[(long long)c * ntiles + u];
    s = warp_sum(s);
    if (lane == 0) col[c] = s;
  }
}

// w -= sum_{c<=j} V_c H_q(c, j) with double-float accumulation; then
// pnorm[t] = sum over the tile of |w|^2 (FP64).
__global__ void __launch_bounds__(kBT)
    k_baxpys_df(const int* __restrict__ tile_prob, const c64* __restrict__ V, long long ldv,
                const c128* __restrict__ H, int ldh, long long hstride, const int* __restrict__ jptr,
                c128* __restrict__ w, double* __restrict__ pnorm, const KState* __restrict__ kst) {
  extern __shared__ dfc hsd[];
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (kst[q].stop) return;
  const int j = *jptr, ncols = j + 1;
  const c128* col = H + q * hstride + (long long)j * ldh;
  for (int c = threadIdx.x; c < ncols; c += kBT) hsd[c] = split_c(mk(-col[c].re, -col[c].im));
  __syncthreads();
  const long long r0 = (long long)t * kBatchTile + threadIdx.x;
  dfc* wd = reinterpret_cast<dfc*>(w);   // w in double-float form
  float nh = 0.f, nl = 0.f;               // this thread's sum of |w|^2, double-float
#pragma unroll 1
  for (int s = 0; s < kRows; ++s) {
    const long long r = r0 + s * kBT;
    const dfc w0 = wd[r];
    float rh = w0.rh, rl = w0.rl, ih = w0.ih, il = w0.il;
    for (int c0 = 0; c0 < ncols; c0 += 2 * kBCols) {
      c64 a[2 * kBCols];
#pragma unroll
      for (int u = 0; u < 2 * kBCols; ++u)
        if (c0 + u < ncols) a[u] = V[(long long)(c0 + u) * ldv + r];   // loads first
#pragma unroll
      for (int u = 0; u < 2 * kBCols; ++u) {
        if (c0 + u >= ncols) continue;
        const dfc hc = hsd[c0 + u];
        const dfl hr = dfl_of(hc.rh, hc.rl), hi_ = dfl_of(hc.ih, hc.il);
        float p, e;
        // a h = (ar hr - ai hi) + i (ar hi + ai hr)
        fdf_mul(a[u].re, hr, p, e);
        df_acc(rh, rl, p, e);
        fdf_mul(a[u].im, hi_, p, e);
        df_acc(rh, rl, -p, -e);
        fdf_mul(a[u].re, hi_, p, e);
        df_acc(ih, il, p, e);
        fdf_mul(a[u].im, hr, p, e);
        df_acc(ih, il, p, e);
      }
    }
    df_norm(rh, rl);
    df_norm(ih, il);
    dfc o;
    o.rh = rh;
    o.rl = rl;
    o.ih = ih;
    o.il = il;
    wd[r] = o;
    // |w|^2 = rh^2 + 2 rh rl + ih^2 + 2 ih il (+ terms below 2^-46 relative)
    float p = rh * rh;
    float e = fmaf(rh, rh, -p) + 2.f * rh * rl;
    df_acc(nh, nl, p, e);
    p = ih * ih;
    e = fmaf(ih, ih, -p) + 2.f * ih * il;
    df_acc(nh, nl, p, e);
  }
  // block sum in double-float, one conversion
  __shared__ float2 red[kBT / 32];
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
    for (int u = 1; u < kBT / 32; ++u) df_acc(a, b, red[u].x, red[u].y);
    pnorm[t] = df_to_d(a, b);
  }
}

// Step j, one warp per problem: h_{j+1,j} = ||w|| from the tile partials,
// the complex Givens rotation of Section 4.1's least-squares problem, the
// residual estimate |g_{j+1}| / ||b||, and the stop decision of the cycle
// (estimate <= rtol, cycle length m, maxit directions, breakdown, NaN).
__global__ void k_bnorm_givens(const int* __restrict__ tile0, const int* __restrict__ tile1,
                               const double* __restrict__ pnorm, const int* __restrict__ jptr, BCtl* ctl,
                               c128* __restrict__ H, int ldh, long long hstride, double* __restrict__ cs,
                               c128* __restrict__ sn, c128* __restrict__ gvec, int m, double rtol, int maxit,
                               KState* __restrict__ kst) {
  const int q = blockIdx.x;
  KState& k = kst[q];
  if (k.stop) return;
  const int j = *jptr;
  double s = 0.0;
  for (int u = tile0[q] + threadIdx.x; u < tile1[q]; u += 32) s += pnorm[u];
  s = warp_sumd(s);   // in every lane
  const double hn = sqrt(s);
  c128* col = H + q * hstride + (long long)j * ldh;
  double* csq = cs + (long long)q * m;
  c128* snq = sn + (long long)q * m;
  c128* gq = gvec + (long long)q * (m + 1);
  // the previous rotations on column j (one warp), then lane 0 continues
  const c128 cj = givens_prev_warp(col, csq, snq, j, threadIdx.x);
  if (threadIdx.x != 0) return;
  k.hnorm = hn;
  col[j] = cj;
  col[j + 1] = mk(hn, 0.0);
  const c128 a = col[j], b = col[j + 1];
  const double aa = sqrt(abs2(a)), bb = sqrt(abs2(b));
  double c;
  c128 sv, r;
  if (bb == 0.0) {
    c = 1.0; sv = mk(0.0, 0.0); r = a;
  } else if (aa == 0.0) {
    c = 0.0; sv = mk(1.0, 0.0); r = b;
  } else {
    const double nrm = hypot(aa, bb);
    const c128 ph = (1.0 / aa) * a;
    c = aa / nrm;
    sv = (1.0 / nrm) * (ph * conj(b));
    r = nrm * ph;
  }
  col[j] = r;
  col[j + 1] = mk(0.0, 0.0);
  csq[j] = c;
  snq[j] = sv;
  const c128 gj = gq[j];
  gq[j + 1] = mk(0.0, 0.0) - conj(sv) * gj;
  gq[j] = c * gj;
  k.total += 1;
  k.jdone = j + 1;
  const double est = sqrt(abs2(gq[j + 1])) / k.bnorm;
  k.est = est;
  int stop = 0;
  if (!isfinite(est)) { k.nan = 1; stop = 1; }
  if (est <= rtol) { k.conv = 1; stop = 1; }
  if (hn == 0.0) { k.breakdown = 1; stop = 1; }
  if (j + 1 >= m || k.total >= maxit) stop = 1;
  // one cycle on the complex64 basis is trusted down to 1e-6 of its start;
  // below that the next cycle starts from the true residual
  if (sqrt(abs2(gq[j + 1])) <= kBasisFloor * k.beta0) stop = 1;
  if (stop) {
    k.stop = 1;
    atomicSub(&ctl->active, 1);
  }
}

// v_{j+1} = fl32(w / h_{j+1,j}) for problems whose cycle continues, w in
// double-float form, 1/h as a double-float pair from an FP32 reciprocal and
// one Newton step (FP32 pipe only); with jptr == nullptr, v_0 = fl32(w / beta)
// at a cycle start (w complex128, beta in hnorm, FP64).
__global__ void __launch_bounds__(kBT)
    k_bscale_df(const int* __restrict__ tile_prob, const c128* __restrict__ w, c64* __restrict__ V, long long ldv,
                const int* __restrict__ jptr, const KState* __restrict__ kst) {
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (kst[q].stop) return;
  const double d = kst[q].hnorm;
  if (!(d > 0.0)) return;
  c64* v = V + (jptr ? (long long)(*jptr + 1) * ldv : 0);
  const dfl dd = split_d(d);
  const float s0 = 1.f / dd.hi;
  if (jptr == nullptr || !(dd.hi > 0.f) || !(s0 < 3e38f)) {
    const double sc = 1.0 / d;
#pragma unroll 2
    for (int s = 0; s < kRows; ++s) {
      const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
      if (jptr == nullptr) {
        const c128 x = w[r];
        v[r] = mk((float)(sc * x.re), (float)(sc * x.im));
      } else {
        const dfc x = reinterpret_cast<const dfc*>(w)[r];
        v[r] = mk((float)(sc * ((double)x.rh + (double)x.rl)), (float)(sc * ((double)x.ih + (double)x.il)));
      }
    }
    return;
  }
  const float r0 = fmaf(-dd.hi, s0, 1.f) - dd.lo * s0;
  const float sh = s0, sl = s0 * r0;
#pragma unroll 2
  for (int s = 0; s < kRows; ++s) {
    const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
    const dfc x = reinterpret_cast<const dfc*>(w)[r];
    float p = x.rh * sh;
    const float vr = p + (fmaf(x.rh, sh, -p) + fmaf(x.rh, sl, x.rl * sh));
    p = x.ih * sh;
    const float vi = p + (fmaf(x.ih, sh, -p) + fmaf(x.ih, sl, x.il * sh));
    v[r] = mk(vr, vi);
  }
}

__global__ void k_bnext(BCtl* ctl) { ctl->j += 1; }

// Cycle start, one warp per problem still being solved: beta = ||b - A x||
// from the tile partials. The first cycle takes ||b|| = beta. A problem
// finishes when beta/||b|| <= rtol, when it is non-finite, or when maxit
// directions are spent; otherwise its cycle starts with g = beta e_1.
__global__ void k_bcycle_init(const int* __restrict__ tile0, const int* __restrict__ tile1,
                              const double* __restrict__ pnorm, BCtl* ctl, c128* __restrict__ gvec, int m,
                              double rtol, int maxit, int first, KState* __restrict__ kst) {
  const int q = blockIdx.x;
  KState& k = kst[q];
  if (!k.live) return;
  double s = 0.0;
  for (int u = tile0[q] + threadIdx.x; u < tile1[q]; u += 32) s += pnorm[u];
  s = warp_sumd(s);
  c128* gq = gvec + (long long)q * (m + 1);
  for (int i = threadIdx.x; i <= m; i += 32) gq[i] = mk(0.0, 0.0);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(s);
  if (first) k.bnorm = beta;
  const double rel = k.bnorm > 0.0 ? beta / k.bnorm : (beta == 0.0 ? 0.0 : beta);
  k.relres = rel;
  k.jdone = 0;
  k.hnorm = beta;
  k.beta0 = beta;
  if (!isfinite(beta) || !isfinite(rel)) {
    k.nan = 1;
    k.live = 0;
  } else if (rel <= rtol || beta == 0.0) {
    k.conv = 1;
    k.live = 0;
  } else if (k.total >= maxit) {
    k.live = 0;
  } else {
    k.conv = 0;
    k.stop = 0;
    gq[0] = mk(beta, 0.0);
    atomicAdd(&ctl->active, 1);
  }
}

// y_q = R_q^-1 g_q for the jdone_q x jdone_q upper triangle left by the
// rotations; one warp per problem still being solved.
__global__ void k_bbacksolve(const c128* __restrict__ H, int ldh, long long hstride, const c128* __restrict__ gvec,
                             int m, const KState* __restrict__ kst, c128* __restrict__ y) {
  const int q = blockIdx.x;
  if (!kst[q].live) return;
  const int nj = kst[q].jdone;
  const c128* Hq = H + q * hstride;
  const c128* gq = gvec + (long long)q * (m + 1);
  c128* yq = y + (long long)q * m;
  const int l = threadIdx.x;
  for (int i = nj - 1; i >= 0; --i) {
    c128 s = mk(0.0, 0.0);
    for (int c = i + 1 + l; c < nj; c += 32) s = s + Hq[(long long)c * ldh + i] * yq[c];
    s = warp_sum(s);
    if (l == 0) yq[i] = cdiv(gq[i] - s, Hq[(long long)i * ldh + i]);
    __syncwarp();
    __threadfence_block();
  }
}

// x += sum_{c < jdone_q} Z_c y_q[c] for problems still being solved: in
// FP64 for complex128 columns of Z, in double-float on the FP32 pipe (y split
// once per column, x once per row) when Z holds double-float pairs (zdf).
__global__ void __launch_bounds__(kBT)
    k_bupdate(const int* __restrict__ tile_prob, const c128* __restrict__ Z, long long ldz,
              const c128* __restrict__ y, int m, const KState* __restrict__ kst, c128* __restrict__ x, int zdf) {
  extern __shared__ c128 ys[];
  const int t = blockIdx.x;
  const int q = tile_prob[t];
  if (!kst[q].live) return;
  const int nj = kst[q].jdone;
  for (int c = threadIdx.x; c < nj; c += kBT) {
    const c128 yc = y[(long long)q * m + c];
    if (zdf) reinterpret_cast<dfc*>(ys)[c] = split_c(yc);
    else ys[c] = yc;
  }
  __syncthreads();
  if (zdf) {
    const dfc* Zd = reinterpret_cast<const dfc*>(Z);
    const dfc* yd = reinterpret_cast<const dfc*>(ys);
#pragma unroll 1
    for (int s = 0; s < kRows; ++s) {
      const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
      const dfc x0 = split_c(x[r]);
      float rh = x0.rh, rl = x0.rl, ih = x0.ih, il = x0.il;
      for (int c = 0; c < nj; ++c) {
        const dfc a = Zd[(long long)c * ldz + r], h = yd[c];
        const dfl ar = dfl_of(a.rh, a.rl), ai = dfl_of(a.ih, a.il);
        const dfl hr = dfl_of(h.rh, h.rl), hi_ = dfl_of(h.ih, h.il);
        float p, e;
        // a h = (ar hr - ai hi) + i (ar hi + ai hr)
        df_prod(ar, hr, p, e);
        df_acc(rh, rl, p, e);
        df_prod(ai, hi_, p, e);
        df_acc(rh, rl, -p, -e);
        df_prod(ar, hi_, p, e);
        df_acc(ih, il, p, e);
        df_prod(ai, hr, p, e);
        df_acc(ih, il, p, e);
      }
      x[r] = mk(df_to_d(rh, rl), df_to_d(ih, il));
    }
    return;
  }
#pragma unroll 1
  for (int s = 0; s < kRows; ++s) {
    const long long r = (long long)t * kBatchTile + s * kBT + threadIdx.x;
    c128 a0 = x[r], a1 = mk(0.0, 0.0);
    int c = 0;
    for (; c + 1 < nj; c += 2) {
      a0 = fmac(a0, Z[(long long)c * ldz + r], ys[c]);
      a1 = fmac(a1, Z[(long long)(c + 1) * ldz + r], ys[c + 1]);
    }
    if (c < nj) a0 = fmac(a0, Z[(long long)c * ldz + r], ys[c]);
    x[r] = a0 + a1;
  }
}

}  // namespace

cudaError_t launch_bprolong(int prec, int ntiles, const int* tile_prob, const Geo* geos, const SubDesc* subs,
                            const int* sub_index, const void* Y, c128* z, long long ldz, const int* jptr,
                            const KState* kst, int gate, cudaStream_t st, int zdf) {
  if (prec == 0)
    k_bprolong<double><<<ntiles, kBT, 0, st>>>(tile_prob, geos, subs, sub_index, (const c128*)Y, z, ldz, jptr, kst,
                                               gate, 0);
  else
    k_bprolong<float><<<ntiles, kBT, 0, st>>>(tile_prob, geos, subs, sub_index, (const c64*)Y, z, ldz, jptr, kst,
                                              gate, zdf);
  return cudaGetLastError();
}

cudaError_t launch_bspmv(int ntiles, const int* tile_prob, const Geo* geos, const c128* D, const c128* CW,
                         const c128* CS, const c128* CSW, const c128* x, long long ldx, const int* jptr,
                         const c128* bsub, c128* y, double* pnorm, const KState* kst, int gate, cudaStream_t st) {
  k_bspmv<<<ntiles, kBT, 0, st>>>(tile_prob, geos, D, CW, CS, CSW, x, ldx, jptr, bsub, y, pnorm, kst, gate);
  return cudaGetLastError();
}

cudaError_t launch_bstep(const BStep& a, cudaStream_t st) {
  const int* jp = &a.ctl->j;
  cudaError_t e = cudaSuccess;
  const size_t dsm = (size_t)(a.m + 1) * (kBT / 32) * sizeof(c128);
  const size_t hsm = (size_t)(a.m + 1) * sizeof(dfc);   // h column split, double-float
  if (dsm > 48 * 1024) {
    e = cudaFuncSetAttribute(k_bdots_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (e != cudaSuccess) return e;
  }
  if (hsm > 48 * 1024) {
    e = cudaFuncSetAttribute(k_baxpys_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
    if (e != cudaSuccess) return e;
  }
  e = launch_local_solves(a.prec, a.cols, a.geos, a.subs, a.nsub, a.max_b, a.max_bp, a.L, a.Lrev, a.dinv,
                          (const c128*)a.V, a.ld, jp, a.Y, a.kst, a.status, st, RK_C64, a.as);
  if (e != cudaSuccess) return e;
  // z_j in double-float form with complex64 local values; w always in that form
  const int zdf = a.prec >= 1 ? 1 : 0;
  e = launch_bprolong(a.prec, a.ntiles, a.tile_prob, a.geos, a.subs, a.sub_index, a.Y, a.Z, a.ld, jp, a.kst, 1, st,
                      zdf);
  if (e != cudaSuccess) return e;
  k_bspmv_df<<<a.ntiles, kBT, 0, st>>>(a.tile_prob, a.geos, (const dfc*)a.Ddf, (const dfc*)a.CWdf,
                                       (const dfc*)a.CSdf, (const dfc*)a.CSWdf, a.Z, a.ld, jp, a.w, zdf, a.kst);
  k_bdots_df<<<a.ntiles, kBT, dsm, st>>>(a.tile_prob, (const c64*)a.V, a.ld, a.w, jp, a.partial, a.ntiles, a.kst);
  k_bdots_finish<<<a.nprob, kBT, 0, st>>>(a.tile0, a.tile1, a.partial, a.ntiles, jp, a.H, a.m + 1, a.hstride,
                                          a.kst);
  k_baxpys_df<<<a.ntiles, kBT, hsm, st>>>(a.tile_prob, (const c64*)a.V, a.ld, a.H, a.m + 1, a.hstride, jp, a.w,
                                          a.pnorm, a.kst);
  k_bnorm_givens<<<a.nprob, 32, 0, st>>>(a.tile0, a.tile1, a.pnorm, jp, a.ctl, a.H, a.m + 1, a.hstride, a.cs, a.sn,
                                         a.gvec, a.m, a.rtol, a.maxit, a.kst);
  k_bscale_df<<<a.ntiles, kBT, 0, st>>>(a.tile_prob, a.w, (c64*)a.V, a.ld, jp, a.kst);
  k_bnext<<<1, 1, 0, st>>>(a.ctl);
  return cudaGetLastError();
}

cudaError_t launch_bcycle_start(const BStep& a, const c128* b, const c128* x, int first, cudaStream_t st) {
  cudaError_t e = launch_bspmv(a.ntiles, a.tile_prob, a.geos, a.D, a.CW, a.CS, a.CSW, x, 0, nullptr, b, a.w,
                               a.pnorm, a.kst, 2, st);
  if (e != cudaSuccess) return e;
  k_bcycle_init<<<a.nprob, 32, 0, st>>>(a.tile0, a.tile1, a.pnorm, a.ctl, a.gvec, a.m, a.rtol, a.maxit, first, a.kst);
  k_bscale_df<<<a.ntiles, kBT, 0, st>>>(a.tile_prob, a.w, (c64*)a.V, a.ld, nullptr, a.kst);
  return cudaGetLastError();
}

cudaError_t launch_bcycle_end(const BStep& a, c128* x, cudaStream_t st) {
  k_bbacksolve<<<a.nprob, 32, 0, st>>>(a.H, a.m + 1, a.hstride, a.gvec, a.m, a.kst, a.yv);
  const size_t ysm = (size_t)a.m * sizeof(c128);
  if (ysm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bupdate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm);
    if (e != cudaSuccess) return e;
  }
  k_bupdate<<<a.ntiles, kBT, ysm, st>>>(a.tile_prob, a.Z, a.ld, a.yv, a.m, a.kst, x, a.prec >= 1 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rp
