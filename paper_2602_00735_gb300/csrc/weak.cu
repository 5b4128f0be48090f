// Kernels of form 1, the paper's eq. weak as printed (Section 1): its matrix
// is not symmetric (the beta term), so the global product reads seven
// coupling arrays and the local operators A_j are factored as A_j = L D U
// (L unit lower, U unit upper band, no pivoting) instead of L D L^T.
//
// k_spmv7: y = A x (or y = b - A x), one thread per row, couplings summed in
//   the fixed order D, W, E, S, N, SW, NE in FP64.
// k_factor_lu: one CTA per subdomain, right-looking. The active window
//   (rows and columns k..k+b) is a (b+1) x (b+1) square in shared memory,
//   circular in both indices: entry (r, c) at slot ((r mod (b+1)), (c mod
//   (b+1))). Step k
//     1. reads the pivot column c_t = W(k+t, k) and row r_t = W(k, k+t),
//        d = c_0, writes L(k+t, k) = c_t / d, U(k, k+t) = u_t = r_t / d and
//        D^-1(k) = 1/d;
//     2. applies W(k+i, k+j) -= c_i u_j, 1 <= i, j <= b (a thread keeps one
//        column j and steps through rows i with a fixed stride, so the
//        circular slots advance by additions), and at the same time
//        moves row k+b+1 and column k+b+1 of A_j into the slots of row k and
//        column k (disjoint from the update's slots; neither has been touched
//        by an earlier pivot, since they lie outside its band).
//   Output layout (the apply's, unchanged): L column k at l_off + k*bp,
//   rows k+1..k+b; the backward factor stored as a unit lower band in
//   reversed order: column k' = npad-1-i holds U(i-1, i), U(i-2, i), ...,
//   i.e. U(k, k+t) at l_off + (npad-1-(k+t))*bp + t-1. With U = L^T this is
//   exactly the reversed row copy of L that the L D L^T factor writes, so the
//   apply's two sweeps solve L y = r, then U x = D^-1 y. The caller
//   zero-fills that copy first.
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

__global__ void k_spmv7(long long n, int nx, Stencil7 A, const c128* __restrict__ x, const c128* __restrict__ bsub,
                        int bdf, c128* __restrict__ y, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= n) return;
  c128 acc = A.D[r] * x[r];
  if (r >= 1) acc = fmac(acc, A.W[r], x[r - 1]);
  if (r + 1 < n) acc = fmac(acc, A.E[r], x[r + 1]);
  if (r >= nx) acc = fmac(acc, A.S[r], x[r - nx]);
  if (r + nx < n) acc = fmac(acc, A.N[r], x[r + nx]);
  if (r >= nx + 1) acc = fmac(acc, A.SW[r], x[r - nx - 1]);
  if (r + nx + 1 < n) acc = fmac(acc, A.NE[r], x[r + nx + 1]);
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

// Entry (r, c) of A_j from the seven stored couplings of row r (offsets 0,
// -1, +1, -(b-1), +(b-1), -b, +b); identity beyond the n local unknowns.
template <typename R>
__device__ __forceinline__ cx<R> aw_entry(const c128* __restrict__ Aw, const SubDesc& sd, int r, int c) {
  if (r >= sd.n || c >= sd.n) return mk((R)(r == c ? 1 : 0), (R)0);
  const int d = c - r, b = sd.b;
  const c128* a = Aw + 7 * (sd.v_off + r);
  c128 v = mk(0.0, 0.0);
  if (d == 0) v = v + a[0];
  if (d == -1) v = v + a[1];
  if (d == 1) v = v + a[2];
  if (d == 1 - b) v = v + a[3];
  if (d == b - 1) v = v + a[4];
  if (d == -b) v = v + a[5];
  if (d == b) v = v + a[6];
  return cvt<R>(v);
}

constexpr int kLuThreads = 256;

template <typename R, typename S>
__global__ void __launch_bounds__(kLuThreads)
    k_factor_lu(const SubDesc* __restrict__ subs, const c128* __restrict__ Aw, S* __restrict__ Lall,
                S* __restrict__ Urev_all, cx<R>* __restrict__ dinv_all, double* __restrict__ pivstats,
                DevStatus* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
  const int tid = threadIdx.x;
  const int b = sd.b, bp = sd.bp, Wc = b + 1, npad = sd.npad;
  cx<R>* W = reinterpret_cast<cx<R>*>(sm);     // Wc x Wc, row slot major
  cx<R>* cbuf = W + Wc * Wc;                   // pivot column c_t
  cx<R>* ubuf = cbuf + Wc;                     // u_t = W(k, k+t) / d
  S* L = Lall + sd.l_off;
  S* Ur = Urev_all + sd.l_off;
  cx<R>* dv = dinv_all + sd.v_off;

  // rows and columns 0..b of A_j
  for (int e = tid; e < Wc * Wc; e += kLuThreads) W[e] = aw_entry<R>(Aw, sd, e / Wc, e % Wc);
  __syncthreads();

  R dmin2 = (R)3e38, dmax2 = (R)0;
  bool bad = false;
  int ks = 0;   // k mod Wc
  // update mapping: G = NT / b row groups; thread tid < G*b owns column
  // j = 1 + tid mod b and rows i = 1 + tid / b, 1 + tid / b + G, ...
  const int G = kLuThreads / b;
  const int uj = 1 + tid % b, ui0 = 1 + tid / b;
  const bool upd = tid < G * b;
  for (int k = 0; k < npad; ++k) {
    // 1. pivot column and row
    if (tid <= b) {
      int st = ks + tid;
      if (st >= Wc) st -= Wc;
      const cx<R> d = W[ks * Wc + ks];
      const cx<R> di = crecip(d);
      const cx<R> c = W[st * Wc + ks];
      const cx<R> u = W[ks * Wc + st] * di;
      cbuf[tid] = c;
      ubuf[tid] = u;
      if (tid == 0) {
        const R ad2 = abs2(d);
        if (!(ad2 > (R)0) || !isfinite(ad2) || !isfinite(di.re) || !isfinite(di.im)) bad = true;
        dmin2 = fmin(dmin2, ad2);
        dmax2 = fmax(dmax2, ad2);
        dv[k] = di;
        if (bp > b) L[(long long)k * bp + b] = st_entry<S, R>(mk((R)0, (R)0));
      } else {
        L[(long long)k * bp + (tid - 1)] = st_entry<S, R>(c * di);
        if (k + tid < npad) Ur[(long long)(npad - 1 - (k + tid)) * bp + (tid - 1)] = st_entry<S, R>(u);
      }
    }
    __syncthreads();
    // 2. update of rows and columns k+1..k+b; row and column k+b+1 enter the
    //    slots of row k and column k
    if (upd) {
      int cj = ks + uj, ri = ks + ui0;
      if (cj >= Wc) cj -= Wc;
      if (ri >= Wc) ri -= Wc;
      const cx<R> u = ubuf[uj];
      for (int i = ui0; i <= b; i += G) {   // i + G <= b implies ri + G < 2 Wc
        cx<R>* w = &W[ri * Wc + cj];
        *w = fms(*w, cbuf[i], u);
        ri += G;
        if (ri >= Wc) ri -= Wc;
      }
    }
    if (tid <= b) {
      const int rn = k + b + 1;
      int st = ks + 1 + tid;   // slot of index k+1+tid
      if (st >= Wc) st -= Wc;
      W[ks * Wc + st] = aw_entry<R>(Aw, sd, rn, k + 1 + tid);           // row k+b+1, columns k+1..k+b+1
      if (tid < b) W[st * Wc + ks] = aw_entry<R>(Aw, sd, k + 1 + tid, rn);   // column k+b+1, rows k+1..k+b
    }
    __syncthreads();
    if (++ks == Wc) ks = 0;
  }
  if (tid == 0) {
    pivstats[2 * blockIdx.x] = sqrt((double)dmin2);
    pivstats[2 * blockIdx.x + 1] = sqrt((double)dmax2);
    if (bad) atomicCAS(&status->pivot_bad_sub, -1, (int)blockIdx.x);
  }
}

template <typename R, typename S>
cudaError_t launch_lu_t(const SubDesc* subs, int nsub, int max_b, const c128* Aw, void* L, void* Urev, void* dinv,
                        double* pivstats, DevStatus* status, cudaStream_t st) {
  const size_t smem = factor_lu_smem_bytes(max_b, sizeof(cx<R>) == sizeof(c128) ? 0 : 1);
  cudaError_t e = cudaFuncSetAttribute(k_factor_lu<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor_lu<R, S><<<nsub, kLuThreads, smem, st>>>(subs, Aw, (S*)L, (S*)Urev, (cx<R>*)dinv, pivstats, status);
  return cudaGetLastError();
}

}  // namespace

int max_band_lu(int prec) { return prec == 0 ? kMaxBandLuC128 : kMaxBandLuC64; }

size_t factor_lu_smem_bytes(int b, int prec) {
  const size_t es = prec == 0 ? sizeof(c128) : sizeof(c64);
  const size_t wc = (size_t)b + 1;
  return (wc * wc + 2 * wc) * es;
}

cudaError_t launch_spmv7(long long n, int nx, const Stencil7& A, const c128* x, const c128* bsub, c128* y,
                         const KState* kst, cudaStream_t st, int bsub_kind) {
  const int threads = 256;
  k_spmv7<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(n, nx, A, x, bsub, bsub_kind, y, kst);
  return cudaGetLastError();
}

cudaError_t launch_factor_lu(int prec, const SubDesc* subs, int nsub, int max_b, const c128* Aw, void* L, void* Urev,
                             void* dinv, double* pivstats, DevStatus* status, cudaStream_t st) {
  if (max_b < 1 || max_b > max_band_lu(prec)) return cudaErrorInvalidValue;
  if (prec == 0) return launch_lu_t<double, c128>(subs, nsub, max_b, Aw, L, Urev, dinv, pivstats, status, st);
  if (prec == 1) return launch_lu_t<float, c64>(subs, nsub, max_b, Aw, L, Urev, dinv, pivstats, status, st);
  return launch_lu_t<float, h2c>(subs, nsub, max_b, Aw, L, Urev, dinv, pivstats, status, st);
}

}  // namespace rp
