// Batched band LDL^T factorisation of the local operators A_j (the local
// solves A_j^-1 of the preconditioner, Section 2). A_j is complex symmetric
// (the gamma_1 gamma_2 form), so A_j = L_j D_j L_j^T without pivoting; with
// the x-fastest local numbering its half-bandwidth is b = nlx + 1.
//
// One CTA factors one subdomain, right-looking, holding the active
// (b+1) x (b+1) window of the matrix in shared memory as a circular buffer:
// row/column index i lives in slot i mod (b+1). Step k
//   1. reads the pivot column c_i = W(k+i, k), d = c_0, l_i = c_i / d,
//      and writes L(:, k) = l and D^-1(k) = 1/d to global memory;
//   2. applies the rank-1 update W(k+i, k+j) -= c_i l_j, 1 <= j <= i <= b;
//   3. moves row k+b+1 of A_j into the slot freed by row k; those rows are
//      staged in shared memory 32 steps ahead, so no global load sits on a
//      step's critical path.
// Output layout: L_j column k at l_off + k*bp (bp >= b, entries b..bp-1 are
// zero), rows k+1..k+b; D^-1 at v_off + k. Rows n..npad-1 are identity
// padding, so their L columns are zero. A second copy holds the rows of L_j
// in reversed order: row i of L, read leftwards (L(i,i-1), L(i,i-2), ...),
// at l_off + (npad-1-i)*bp; this is the column band of L^T in reversed
// index order, which the backward sweep of the apply streams. The caller
// zero-fills that copy first (entries left of column 0 stay zero).
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

constexpr int kFactorThreads = 256;

template <typename R>
__device__ __forceinline__ cx<R> aloc_val(const c128* __restrict__ A, const SubDesc& sd, int row, int t) {
  // entry (row, row - t) of A_j, t in [0, b]; rows >= n are identity
  if (row >= sd.n) return (t == 0) ? mk((R)1, (R)0) : mk((R)0, (R)0);
  const c128* a = A + 4 * (sd.v_off + row);
  c128 v = mk(0.0, 0.0);
  if (t == 0) v = a[0];
  if (t == 1) v = v + a[1];
  if (t == sd.b - 1) v = v + a[2];
  if (t == sd.b) v = v + a[3];
  return cvt<R>(v);
}

// The four stored entries of row `row` of A_j (D, W, S, SW couplings);
// identity for padding rows.
template <typename R>
__device__ __forceinline__ void aloc_row(const c128* __restrict__ A, const SubDesc& sd, int row, cx<R> (&v)[4]) {
  if (row >= sd.n) {
    v[0] = mk((R)1, (R)0);
    v[1] = v[2] = v[3] = mk((R)0, (R)0);
    return;
  }
  const c128* a = A + 4 * (sd.v_off + row);
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = cvt<R>(a[i]);
}

// Entry (row, row - t) from a row's four stored entries.
template <typename R>
__device__ __forceinline__ cx<R> row_entry(const cx<R> (&v)[4], int t, int b) {
  cx<R> r = mk((R)0, (R)0);
  if (t == 0) r = v[0];
  if (t == 1) r = r + v[1];
  if (t == b - 1) r = r + v[2];
  if (t == b) r = r + v[3];
  return r;
}

// R: arithmetic; S: storage of the L entries (cx<R>, or h2c halves).
template <typename R, typename S>
__global__ void __launch_bounds__(kFactorThreads)
    k_factor_ldlt(const SubDesc* __restrict__ subs, const c128* __restrict__ Aloc, S* __restrict__ Lall,
                  S* __restrict__ Lrev_all, cx<R>* __restrict__ dinv_all, double* __restrict__ pivstats,
                  DevStatus* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
  const int tid = threadIdx.x;
  const int b = sd.b, Wc = b + 1, bp = sd.bp;
  const int npairs = b * (b + 1) / 2;
  cx<R>* W = reinterpret_cast<cx<R>*>(sm);          // W[colslot * Wc + rowslot]
  cx<R>* cbuf = W + Wc * Wc;
  cx<R>* lbuf = cbuf + Wc;
  uint16_t* pairs = reinterpret_cast<uint16_t*>(lbuf + Wc);
  S* L = Lall + sd.l_off;
  S* Lr = Lrev_all + sd.l_off;
  cx<R>* dv = dinv_all + sd.v_off;

  // (i', j') with 1 <= j' <= i' <= b, column by column
  for (int e = tid; e < npairs; e += blockDim.x) {
    int j = 1, start = 0;
    while (start + (b - j + 1) <= e) {
      start += b - j + 1;
      ++j;
    }
    int i = j + (e - start);
    pairs[e] = (uint16_t)((i << 8) | j);
  }
  for (int e = tid; e < Wc * Wc; e += blockDim.x) W[e] = mk((R)0, (R)0);
  __syncthreads();
  // rows 0..b of A_j: row r at slot r
  if (tid <= b) {
    const int r = tid;
    for (int t = 0; t <= b && t <= r; ++t) {
      cx<R> v = aloc_val<R>(Aloc, sd, r, t);
      if (v.re != (R)0 || v.im != (R)0) W[(r - t) * Wc + r] = v;
    }
  }
  __syncthreads();

  R dmin2 = (R)3e38, dmax2 = (R)0;
  bool bad = false;
  int pk = 0;  // slot of row k
  __shared__ cx<R> rows[2][32][4];   // rows entering at the next steps, double-buffered
  if (tid < 128) {
    const int s = tid >> 2, e = tid & 3;
    cx<R> v[4];
    aloc_row<R>(Aloc, sd, b + 1 + s, v);
    rows[0][s][e] = v[e];
  }
  __syncthreads();
  for (int k = 0; k < sd.npad; ++k) {
    if ((k & 31) == 0 && tid < 128) {
      // rows entering at steps k+32..k+63; that buffer's last reader was
      // step k-1, which ended at the barrier before this point
      const int s = tid >> 2, e = tid & 3;
      cx<R> v[4];
      aloc_row<R>(Aloc, sd, k + 32 + b + 1 + s, v);
      rows[((k >> 5) + 1) & 1][s][e] = v[e];
    }
    // 1. pivot column
    if (tid <= b) {
      int s = pk + tid;
      if (s >= Wc) s -= Wc;
      cx<R> c = W[pk * Wc + s];
      cx<R> d = W[pk * Wc + pk];
      cx<R> di = crecip(d);
      cbuf[tid] = c;
      if (tid == 0) {
        const R ad2 = abs2(d);
        if (!(ad2 > (R)0) || !isfinite(ad2) || !isfinite(di.re) || !isfinite(di.im)) bad = true;
        dmin2 = fmin(dmin2, ad2);
        dmax2 = fmax(dmax2, ad2);
        dv[k] = di;
        if (bp > b) L[(long long)k * bp + b] = st_entry<S, R>(mk((R)0, (R)0));
      } else {
        cx<R> l = c * di;
        lbuf[tid] = l;
        const S ls = st_entry<S, R>(l);
        L[(long long)k * bp + (tid - 1)] = ls;
        if (k + tid < sd.npad) Lr[(long long)(sd.npad - 1 - (k + tid)) * bp + (tid - 1)] = ls;
      }
    }
    __syncthreads();
    // 2. rank-1 update of the trailing window
    for (int e = tid; e < npairs; e += blockDim.x) {
      const int pr = pairs[e];
      const int i = pr >> 8, j = pr & 255;
      int si = pk + i;
      if (si >= Wc) si -= Wc;
      int sj = pk + j;
      if (sj >= Wc) sj -= Wc;
      cx<R>* w = &W[sj * Wc + si];
      *w = fms(*w, cbuf[i], lbuf[j]);
    }
    // 3. row k+b+1 enters slot pk (disjoint from the slots updated above)
    if (tid <= b) {
      const int t = tid;
      int sc = pk + (b + 1 - t);  // slot of column k+b+1-t
      if (sc >= Wc) sc -= Wc;
      cx<R> v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = rows[(k >> 5) & 1][k & 31][i];
      W[sc * Wc + pk] = row_entry<R>(v, t, b);
    }
    __syncthreads();
    pk = (pk + 1 == Wc) ? 0 : pk + 1;
  }
  if (tid == 0) {
    pivstats[2 * blockIdx.x] = sqrt((double)dmin2);
    pivstats[2 * blockIdx.x + 1] = sqrt((double)dmax2);
    if (bad) atomicCAS(&status->pivot_bad_sub, -1, (int)blockIdx.x);
  }
}

}  // namespace

size_t factor_smem_bytes(int b, int prec) {
  size_t es = prec == 0 ? sizeof(c128) : sizeof(c64);   // window in the arithmetic type
  size_t wc = (size_t)b + 1;
  return wc * wc * es + 2 * wc * es + (size_t)b * (b + 1) / 2 * sizeof(uint16_t);
}

cudaError_t launch_factor(int prec, const SubDesc* subs, int nsub, int max_b, const c128* Aloc, void* L,
                          void* Lrev, void* dinv, double* pivstats, DevStatus* status, cudaStream_t st) {
  size_t smem = factor_smem_bytes(max_b, prec);
  cudaError_t e;
  if (prec == 0) {
    e = cudaFuncSetAttribute(k_factor_ldlt<double, c128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt<double, c128><<<nsub, kFactorThreads, smem, st>>>(subs, Aloc, (c128*)L, (c128*)Lrev,
                                                                     (c128*)dinv, pivstats, status);
  } else if (prec == 1) {
    e = cudaFuncSetAttribute(k_factor_ldlt<float, c64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt<float, c64><<<nsub, kFactorThreads, smem, st>>>(subs, Aloc, (c64*)L, (c64*)Lrev, (c64*)dinv,
                                                                   pivstats, status);
  } else {
    e = cudaFuncSetAttribute(k_factor_ldlt<float, h2c>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt<float, h2c><<<nsub, kFactorThreads, smem, st>>>(subs, Aloc, (h2c*)L, (h2c*)Lrev, (c64*)dinv,
                                                                   pivstats, status);
  }
  return cudaGetLastError();
}

}  // namespace rp
