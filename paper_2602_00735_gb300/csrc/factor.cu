// Batched band LDL^T factorisation of the local operators A_j (the local
// solves A_j^-1 of the preconditioner, Section 2). A_j is complex symmetric
// (the gamma_1 gamma_2 form), so A_j = L_j D_j L_j^T without pivoting; with
// the x-fastest local numbering its half-bandwidth is b = nlx + 1.
//
// One CTA factors one subdomain, right-looking, holding the active
// window of the matrix (rows and columns k..k+b, lower triangle) in shared
// memory. The window is stored by diagonals: entry (c+t, c), 0 <= t <= b,
// lives on diagonal t, a circular buffer of m_t = b+1-t slots at offset
// off_t = t(b+1) - t(t-1)/2, column c in slot c mod m_t. At step k diagonal
// t holds columns k..k+b-t (exactly m_t of them), so the window needs
// (b+1)(b+2)/2 entries, half of a square window, and the row entering at
// step k meets diagonal t at column k+b+1-t = k (mod m_t): it takes the slot
// that the pivot column frees. Step k
//   1. reads the pivot column c_t = W(k+t, k), d = c_0, l_t = c_t / d,
//      and writes L(:, k) = l and D^-1(k) = 1/d to global memory;
//   2. applies the rank-1 update W(k+i, k+j) -= c_i l_j, 1 <= j <= i <= b;
//      diagonals t and b-1-t are paired (b+1 entries per pair), so the
//      flattened work is spread evenly over the block and consecutive
//      threads touch consecutive slots of one diagonal;
//   3. moves row k+b+1 of A_j into the freed slots; those rows are staged in
//      shared memory 32 steps ahead, so no global load sits on a step's
//      critical path.
// Output layout: L_j column k at l_off + k*bp (bp >= b, entries b..bp-1 are
// zero), rows k+1..k+b; D^-1 at v_off + k. Rows n..npad-1 are identity
// padding, so their L columns are zero. A second copy holds the rows of L_j
// in reversed order: row i of L, read leftwards (L(i,i-1), L(i,i-2), ...),
// at l_off + (npad-1-i)*bp; this is the column band of L^T in reversed
// index order, which the backward sweep of the apply streams. The caller
// zero-fills that copy first (entries left of column 0 stay zero).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace rp {

namespace {

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

// R: arithmetic; S: storage of the L entries (cx<R>, or h2c halves);
// NT: threads per CTA (128, 256 or 512, a tuned tile shape).
template <typename R, typename S, int NT>
__global__ void __launch_bounds__(NT)
    k_factor_ldlt(const SubDesc* __restrict__ subs, const c128* __restrict__ Aloc, S* __restrict__ Lall,
                  S* __restrict__ Lrev_all, cx<R>* __restrict__ dinv_all, double* __restrict__ pivstats,
                  DevStatus* status, int bcap) {
  extern __shared__ __align__(16) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
  if (sd.b > bcap) return;   // wider than this launch's window: the wide kernel takes it
  const int tid = threadIdx.x;
  const int b = sd.b, bp = sd.bp, Wc = b + 1;
  const int nwin = Wc * (b + 2) / 2;
  const int npairs = b * (b + 1) / 2;
  cx<R>* W = reinterpret_cast<cx<R>*>(sm);
  cx<R>* cbuf = W + nwin;
  cx<R>* lbuf = cbuf + Wc;
  // pos[2][Wc]: {slot of column k on diagonal t, end of diagonal t}, one
  // copy read during step k, the other written for step k+1
  int2* pos = reinterpret_cast<int2*>(lbuf + Wc);
  S* L = Lall + sd.l_off;
  S* Lr = Lrev_all + sd.l_off;
  cx<R>* dv = dinv_all + sd.v_off;

  for (int e = tid; e < nwin; e += blockDim.x) W[e] = mk((R)0, (R)0);
  if (tid <= b) {
    const int t = tid, off = t * Wc - t * (t - 1) / 2;
    pos[t] = make_int2(off, off + Wc - t);
  }
  __syncthreads();
  // rows 0..b of A_j: entry (r, r-t) on diagonal t, column r-t < m_t
  if (tid <= b) {
    const int r = tid;
    cx<R> v[4];
    aloc_row<R>(Aloc, sd, r, v);
    const int ts[4] = {0, 1, b - 1, b};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = ts[q];
      if (t <= r) W[t * Wc - t * (t - 1) / 2 + (r - t)] = row_entry<R>(v, t, b);
    }
  }

  // this thread's first update entry e = tid: pair p = e / Wc, offset q = e % Wc;
  // e advances by the block size, (p, q) by (dp, dq) with one carry
  const int dp = NT / Wc, dq = NT % Wc;
  const int p0 = tid / Wc, q0 = tid % Wc;

  R dmin2 = (R)3e38, dmax2 = (R)0;
  bool bad = false;
  __shared__ cx<R> rows[2][32][4];   // rows entering at the next steps, double-buffered
  if (tid < 128) {
    const int s = tid >> 2, e = tid & 3;
    cx<R> v[4];
    aloc_row<R>(Aloc, sd, b + 1 + s, v);
    rows[0][s][e] = v[e];
  }
  __syncthreads();
  for (int k = 0; k < sd.npad; ++k) {
    const int2* pc = pos + (k & 1) * Wc;
    int2* pn = pos + ((k + 1) & 1) * Wc;
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
      cx<R> c = W[pc[tid].x];
      cx<R> d = W[pc[0].x];
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
    // 2. rank-1 update: pair p covers diagonal p (entries j = 1..b-p) then
    //    diagonal b-1-p (j = 1..p+1); for odd b the last pair is the middle
    //    diagonal alone, and e < npairs ends it there
    {
      int p = p0, q = q0;
      for (int e = tid; e < npairs; e += NT) {
        const int l1 = b - p;
        int t, j;
        if (q < l1) { t = p; j = q + 1; } else { t = b - 1 - p; j = q - l1 + 1; }
        const int2 ps = pc[t];
        int a = ps.x + j;
        if (a >= ps.y) a -= Wc - t;
        cx<R>* w = &W[a];
        *w = fms(*w, cbuf[j + t], lbuf[j]);
        p += dp;
        q += dq;
        if (q >= Wc) { q -= Wc; ++p; }
      }
    }
    // 3. row k+b+1 enters the slots of column k (untouched by the update above)
    if (tid <= b) {
      const int t = tid;
      cx<R> v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = rows[(k >> 5) & 1][k & 31][i];
      const int2 ps = pc[t];
      W[ps.x] = row_entry<R>(v, t, b);
      pn[t] = make_int2(ps.x + 1 == ps.y ? ps.y - (Wc - t) : ps.x + 1, ps.y);
    }
    __syncthreads();
  }
  if (tid == 0) {
    pivstats[2 * blockIdx.x] = sqrt((double)dmin2);
    pivstats[2 * blockIdx.x + 1] = sqrt((double)dmax2);
    if (bad) atomicCAS(&status->pivot_bad_sub, -1, (int)blockIdx.x);
  }
}

// Two pivots per pass (rank-2 update), same window storage. Pass k (k even):
//   A. thread t reads c_t = W(k+t, k) and forms column k+1 after step k,
//      e_t = W(k+1+t, k+1) - c_{t+1} l_1 (e_b from the entering row k+b+1),
//      then l_t = c_t / c_0 and l2_t = e_t / e_0, and writes both L columns;
//      it stores c_i, e_{i-1} and l_j, l2_{j-1} side by side for phase B;
//   B. W(k+i, k+j) -= c_i l_j + e_{i-1} l2_{j-1}, 2 <= j <= i <= b+1, where
//      row k+b+1 (i = b+1, c_{b+1} = 0) is taken from the staged rows and
//      lands in the slots of column k;
//   C. row k+b+2 enters the slots of column k+1.
// Each window entry is read and written once per two pivots, and a pass has
// two barriers instead of four.
template <typename R>
struct __align__(4 * sizeof(R)) cx2 {
  cx<R> a, b;
};

template <typename R, typename S, int NT>
__global__ void __launch_bounds__(NT)
    k_factor_ldlt2(const SubDesc* __restrict__ subs, const c128* __restrict__ Aloc, S* __restrict__ Lall,
                   S* __restrict__ Lrev_all, cx<R>* __restrict__ dinv_all, double* __restrict__ pivstats,
                   DevStatus* status, int bcap) {
  extern __shared__ __align__(16) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
  if (sd.b > bcap) return;   // wider than this launch's window: the wide kernel takes it
  const int tid = threadIdx.x;
  const int b = sd.b, bp = sd.bp, Wc = b + 1, npad = sd.npad;
  const int nwin = Wc * (b + 2) / 2;
  const int npairs = b * (b + 1) / 2;
  cx<R>* W = reinterpret_cast<cx<R>*>(sm);
  cx2<R>* CE = reinterpret_cast<cx2<R>*>(W + nwin + (nwin & 1));   // [Wc + 1], 2x aligned
  cx2<R>* LL = CE + Wc + 1;
  int2* pos = reinterpret_cast<int2*>(LL + Wc + 1);
  S* L = Lall + sd.l_off;
  S* Lr = Lrev_all + sd.l_off;
  cx<R>* dv = dinv_all + sd.v_off;
  const cx<R> zero = mk((R)0, (R)0);

  for (int e = tid; e < nwin; e += NT) W[e] = zero;
  if (tid <= b) {
    const int t = tid, off = t * Wc - t * (t - 1) / 2;
    pos[t] = make_int2(off, off + Wc - t);
  }
  __syncthreads();
  if (tid <= b) {
    const int r = tid;
    cx<R> v[4];
    aloc_row<R>(Aloc, sd, r, v);
    const int ts[4] = {0, 1, b - 1, b};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = ts[q];
      if (t <= r) W[t * Wc - t * (t - 1) / 2 + (r - t)] = row_entry<R>(v, t, b);
    }
  }
  const int dp = NT / Wc, dq = NT % Wc;
  const int p0 = tid / Wc, q0 = tid % Wc;

  R dmin2 = (R)3e38, dmax2 = (R)0;
  bool bad = false;
  __shared__ cx<R> rows[2][32][4];   // rows k+b+1.. entering in the next steps, double-buffered
  if (tid < 128) {
    const int s = tid >> 2, e = tid & 3;
    cx<R> v[4];
    aloc_row<R>(Aloc, sd, b + 1 + s, v);
    rows[0][s][e] = v[e];
  }
  __syncthreads();
  for (int k = 0; k < npad; k += 2) {
    const int2* pc = pos + ((k >> 1) & 1) * Wc;
    int2* pn = pos + (((k >> 1) + 1) & 1) * Wc;
    if ((k & 31) == 0 && tid < 128) {
      // rows entering at steps k+32..k+63; that buffer's last readers were
      // the passes before, which ended at the barrier before this point
      const int s = tid >> 2, e = tid & 3;
      cx<R> v[4];
      aloc_row<R>(Aloc, sd, k + 32 + b + 1 + s, v);
      rows[((k >> 5) + 1) & 1][s][e] = v[e];
    }
    const cx<R>(&raw1)[4] = rows[(k >> 5) & 1][k & 31];         // row k+b+1
    const cx<R>(&raw2)[4] = rows[(k >> 5) & 1][(k & 31) + 1];   // row k+b+2
    // A. both pivot columns
    if (tid <= b) {
      const int t = tid;
      auto slot1 = [&](int tt) {   // slot of column k+1 on diagonal tt
        const int2 ps = pc[tt];
        return ps.x + 1 >= ps.y ? ps.x + 1 - (Wc - tt) : ps.x + 1;
      };
      const cx<R> d1 = W[pc[0].x];
      const cx<R> c1 = W[pc[1].x];
      const cx<R> di1 = crecip(d1);
      const cx<R> l1 = c1 * di1;
      const cx<R> d2 = fms(W[slot1(0)], c1, l1);
      const cx<R> di2 = crecip(d2);
      const cx<R> ct = W[pc[t].x];
      cx<R> et;
      if (t < b) {
        et = fms(W[slot1(t)], W[pc[t + 1].x], l1);
      } else {
        cx<R> v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = raw1[i];
        et = row_entry<R>(v, b, b);
      }
      if (t == 0) {
        const R a1 = abs2(d1), a2 = abs2(d2);
        if (!(a1 > (R)0) || !isfinite(a1) || !isfinite(di1.re) || !isfinite(di1.im)) bad = true;
        if (!(a2 > (R)0) || !isfinite(a2) || !isfinite(di2.re) || !isfinite(di2.im)) bad = true;
        dmin2 = fmin(dmin2, fmin(a1, a2));
        dmax2 = fmax(dmax2, fmax(a1, a2));
        dv[k] = di1;
        dv[k + 1] = di2;
        if (bp > b) {
          L[(long long)k * bp + b] = st_entry<S, R>(zero);
          L[(long long)(k + 1) * bp + b] = st_entry<S, R>(zero);
        }
      } else {
        const cx<R> lt = ct * di1, l2t = et * di2;
        const S ls = st_entry<S, R>(lt), l2s = st_entry<S, R>(l2t);
        L[(long long)k * bp + (t - 1)] = ls;
        if (k + t < npad) Lr[(long long)(npad - 1 - (k + t)) * bp + (t - 1)] = ls;
        L[(long long)(k + 1) * bp + (t - 1)] = l2s;
        if (k + 1 + t < npad) Lr[(long long)(npad - 2 - (k + t)) * bp + (t - 1)] = l2s;
        if (t >= 2) {
          CE[t].a = ct;
          LL[t].a = lt;
        }
        CE[t + 1].b = et;
        LL[t + 1].b = l2t;
      }
      if (t == b) {
        CE[b + 1].a = zero;
        LL[b + 1].a = zero;
      }
    }
    __syncthreads();
    // B. rank-2 update; pair p covers diagonal p (j' = 1..b-p) then diagonal
    //    b-1-p (j' = 1..p+1), column offset j = j' + 1
    {
      int p = p0, q = q0;
      for (int e = tid; e < npairs; e += NT) {
        const int l1n = b - p;
        int t, j;
        if (q < l1n) { t = p; j = q + 2; } else { t = b - 1 - p; j = q - l1n + 2; }
        const int i = j + t;
        const int2 ps = pc[t];
        int a = ps.x + j;
        if (a >= ps.y) a -= Wc - t;
        cx<R> w;
        if (i <= b) {
          w = W[a];
        } else {
          cx<R> v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = raw1[u];
          w = row_entry<R>(v, b + 1 - j, b);
        }
        const cx2<R> ce = CE[i], ll = LL[j];
        w = fms(w, ce.a, ll.a);
        w = fms(w, ce.b, ll.b);
        W[a] = w;
        p += dp;
        q += dq;
        if (q >= Wc) { q -= Wc; ++p; }
      }
    }
    // C. row k+b+2 enters the slots of column k+1 (untouched by B)
    if (tid <= b) {
      const int t = tid;
      const int2 ps = pc[t];
      const int m = Wc - t;
      const int a = ps.x + 1 >= ps.y ? ps.x + 1 - m : ps.x + 1;
      cx<R> v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = raw2[u];
      W[a] = row_entry<R>(v, t, b);
      int x = ps.x + 2;
      while (x >= ps.y) x -= m;
      pn[t] = make_int2(x, ps.y);
    }
    __syncthreads();
  }
  if (tid == 0) {
    pivstats[2 * blockIdx.x] = sqrt((double)dmin2);
    pivstats[2 * blockIdx.x + 1] = sqrt((double)dmax2);
    if (bad) atomicCAS(&status->pivot_bad_sub, -1, (int)blockIdx.x);
  }
}


// ---------------------------------------------------------------------------
// Blocked form on the tensor cores (complex64 arithmetic, b <= 127), the
// same factorisation with NB = 8 or 16 pivots per panel (a tuned shape: the
// narrower panel needs less shared memory, so that two subdomains share an
// SM and hide each other's latencies). One CTA of 128 threads
// per subdomain. Rows k..k+NB+b-1 live in a ring of R = NB + b row slots
// (row i in slot i mod R), each holding the band part of the row, columns
// i-b..i, at position c - i + b. Panel k (columns k..k+NB-1):
//   1. warp 0 factors the NB x NB diagonal block in registers (lane a holds
//      row k+a; pivot j broadcasts d_j and the multipliers by shuffles) and
//      writes L11 and 1/d to shared memory;
//   2. thread t < b takes row i = k+NB+t and eliminates its panel part with
//      the diagonal block: c_ij = A(i, k+j) as pivot j reaches it and
//      l_ij = c_ij / d_j;
//   3. the trailing update A(i, c) -= sum_j c_ij l_cj, k+NB <= c <= i <
//      k+NB+b, is the product P Q^T of P = (c_ij) and Q = (l_cj), both
//      b x NB. It runs as tcgen05.mma kind::tf32 (M = 128 rows, N = b
//      rounded up to 16, FP32 accumulators in TMEM): complex products as
//      real ones (Re = Pr Qr^T - Pi Qi^T through the instruction
//      descriptor's negate-A bit, Im = Pr Qi^T + Pi Qr^T) and every
//      FP32 operand as a TF32 head plus tail (x = xh + xl, xh = x with the 13
//      low mantissa bits cleared, exact in TF32), of which the three products
//      xh yh + xh yl + xl yh are kept: about 2^-21 relative rounding per
//      product, next to FP32's 2^-24;
//   4. while one thread issues the MMAs, warps 1-3 write the NB rows entering
//      the window (read from global memory a panel ahead) into the slots of
//      rows k..k+NB-1;
//   5. each warp reads its 32 accumulator rows back (tcgen05.ld) and
//      subtracts them from the ring; warp 0 then factors the next diagonal
//      block (its rows are the first NB of this trailing block), while the
//      other warps finish their rows.
// Output layout and pivot statistics as k_factor_ldlt.
// ---------------------------------------------------------------------------
constexpr int kTcM = 128;
__host__ __device__ constexpr uint32_t tc_ab(int NB) { return kTcM * NB * 4; }   // bytes of one A operand array

__host__ __device__ inline int tc_ldw(int b) { return (b & 1) ? b + 1 : b + 2; }   // even: conflict-free columns
__host__ __device__ inline int tc_n(int b) { return (b + 15) & ~15; }

// Fills positions sub, sub+step, ... of ring slot `slot` with row r of A_j,
// whose four stored entries are v (position p holds column r - b + p).
__device__ __forceinline__ void tc_fill_row(c64* ring, int LDW, int slot, int r, int b, const c64 (&v)[4],
                                            int sub, int step) {
  for (int p = sub; p < LDW; p += step) {
    c64 x = mk(0.f, 0.f);
    if (p <= b && r - (b - p) >= 0) x = row_entry<float>(v, b - p, b);
    ring[slot * LDW + p] = x;
  }
}

// 1. the NB x NB diagonal block of the panel at k (one warp; lane a < NB
// holds row k+a, the other lanes mirror lanes 0..NB-1 without writing).
// Pivot j broadcasts d_j and the multipliers by shuffles (a shared-memory
// broadcast with a warp barrier per pivot measured twice as slow); the
// multipliers also go to L11[j*NB + a] = L(k+a, k+j) for step 2. Lane a
// keeps its own pivot and takes its statistics after the loop, so the loop
// has no divergent branch. The block's global outputs are written
// afterwards by the whole CTA (tc_diag_out).
template <int NB>
__device__ __forceinline__ void tc_diag_block(int k, int lane, const c64* ring, int R, int LDW, int b, c64* L11,
                                              c64* dis, float& dmin2, float& dmax2, bool& bad) {
  const c64 zero = mk(0.f, 0.f);
  const int a = lane & (NB - 1);
  const c64* row = ring + ((k + a) % R) * LDW;
  c64 x[NB];
#pragma unroll
  for (int jj = 0; jj < NB; ++jj) {
    const int p = jj - a + b;
    x[jj] = (jj <= a && p >= 0) ? row[p] : zero;
  }
  c64 mydi = zero;
  float myd2 = 0.f;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const c64 d = shfl(x[j], j);
    const float ad2 = abs2(d);
    const float inv = __frcp_rn(ad2);
    const c64 di = mk(d.re * inv, -d.im * inv);
    const c64 l = x[j] * di;
    if (a == j) {
      mydi = di;
      myd2 = ad2;
    }
    // entries jj > a are never read back: updated without a predicate
#pragma unroll
    for (int jj = j + 1; jj < NB; ++jj) x[jj] = fms(x[jj], x[j], shfl(l, jj));
    if (lane < NB) L11[j * NB + a] = l;   // entries a <= j are never read
  }
  if (lane < NB) {
    dis[a] = mydi;
    if (!(myd2 > 0.f) || !isfinite(myd2) || !isfinite(mydi.re) || !isfinite(mydi.im)) bad = true;
    dmin2 = fminf(dmin2, myd2);
    dmax2 = fmaxf(dmax2, myd2);
  }
}

// Global outputs of the diagonal block at k: 1/d, the zero entry b of each
// column (bp > b), and L(k+a, k+j) for j < a in both copies of L.
template <typename S, int NB>
__device__ __forceinline__ void tc_diag_out(int k, int tid, int b, int bp, int npad, const c64* L11,
                                            const c64* dis, c64* dv, S* L, S* Lr) {
  if (tid < NB) {
    dv[k + tid] = dis[tid];
    if (bp > b) L[(long long)(k + tid) * bp + b] = st_entry<S, float>(mk(0.f, 0.f));
  }
  for (int e = tid; e < NB * NB; e += kTcM) {
    const int j = e / NB, a = e % NB;
    if (a > j && a - j <= b) {
      const S ls = st_entry<S, float>(L11[j * NB + a]);
      L[(long long)(k + j) * bp + (a - j - 1)] = ls;
      Lr[(long long)(npad - 1 - (k + a)) * bp + (a - j - 1)] = ls;
    }
  }
}

template <typename S, int NB>
__global__ void __launch_bounds__(kTcM)
    k_factor_tc(const SubDesc* __restrict__ subs, const c128* __restrict__ Aloc, S* __restrict__ Lall,
                S* __restrict__ Lrev_all, c64* __restrict__ dinv_all, double* __restrict__ pivstats,
                DevStatus* status, int Nmax, int ring_elems, int tcols, int sub_base, int bcap) {
  extern __shared__ __align__(1024) unsigned char smt[];
  unsigned char* sm = smt;
  const int sub = sub_base + (int)blockIdx.x;   // launch position of this subdomain
  const SubDesc sd = subs[sub];
  if (sd.b > bcap) return;   // wider than this launch's ring (before any TMEM allocation)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = sd.b, bp = sd.bp, npad = sd.npad;
  const int R = NB + b, LDW = tc_ldw(b), N = tc_n(b);
  constexpr uint32_t AB = tc_ab(NB);              // bytes of one A operand array
  const uint32_t BB = (uint32_t)Nmax * NB * 4;   // bytes of one B operand array
  unsigned char* Aop = sm;                          // Prh, Prl, Pih, Pil
  unsigned char* Bop = sm + 4 * AB;              // Qrh, Qrl, Qih, Qil
  c64* ring = reinterpret_cast<c64*>(Bop + 4 * BB);
  c64* L11 = ring + ring_elems;                     // L11[j*16 + a] = L(k+a, k+j)
  c64* dis = L11 + NB * NB;                   // 1/d_{k+j}
  uint64_t* bar = reinterpret_cast<uint64_t*>(dis + NB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  S* L = Lall + sd.l_off;
  S* Lr = Lrev_all + sd.l_off;
  c64* dv = dinv_all + sd.v_off;
  const c64 zero = mk(0.f, 0.f);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  // rows 0..R-1, eight threads per row
  for (int r0 = 0; r0 < R; r0 += kTcM / 8) {
    const int r = r0 + (tid >> 3);
    if (r < R) {
      c64 v[4];
      aloc_row<float>(Aloc, sd, r, v);
      tc_fill_row(ring, LDW, r, r, b, v, tid & 7, 8);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  float dmin2 = 3e38f, dmax2 = 0.f;   // lane j of warp 0: pivots k+j
  bool bad = false;
  if (warp == 0) tc_diag_block<NB>(0, lane, ring, R, LDW, b, L11, dis, dmin2, dmax2, bad);
  __syncthreads();
  const uint32_t lba = kTcM * 16, lbb = (uint32_t)N * 16;
  const uint64_t adesc0 = smem_desc(smem_u32(Aop), lba, 128), bdesc0 = smem_desc(smem_u32(Bop), lbb, 128);
  const uint32_t id = idesc_tf32(kTcM, N), idn = id | (1u << 13);   // bit 13: negate A

  bool failed = false;
  uint32_t phase = 0;
  const int t = tid;
  // step 4's rows, read one panel ahead (warps 1-3, 96/NB threads per row)
  constexpr int TPR = 96 / NB;
  const int fq = (tid - 32) / TPR, fsub = (tid - 32) - TPR * ((tid - 32) / TPR);
  c64 vnext[4];
  if (warp > 0) aloc_row<float>(Aloc, sd, NB + b + fq, vnext);
  for (int k = 0; k < npad; k += NB) {
    const bool more = k + NB < npad;
    const int i = k + NB + t;   // this thread's trailing row
    c64 vcur[4];
    if (warp > 0) {
#pragma unroll
      for (int e = 0; e < 4; ++e) vcur[e] = vnext[e];
      if (k + 2 * NB < npad) aloc_row<float>(Aloc, sd, k + 2 * NB + b + fq, vnext);
    }
    tc_diag_out<S, NB>(k, tid, b, bp, npad, L11, dis, dv, L, Lr);
    // 2. the panel part of the trailing rows
    c64 cv[NB], lv[NB];
    if (t < b) {
      const c64* row = ring + (i % R) * LDW;
      c64 y[NB];
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        const int p = jj - NB - t + b;
        y[jj] = p >= 0 ? row[p] : zero;
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        cv[j] = y[j];
        lv[j] = y[j] * dis[j];
#pragma unroll
        for (int jj = j + 1; jj < NB; ++jj) y[jj] = fms(y[jj], cv[j], L11[j * NB + jj]);
      }
      // L(i, k+j) at entry o-1 of column k+j and of reversed row i, o = i-(k+j)
      S* Lc = L + (long long)k * bp + (NB - 1 + t);
      S* Lrr = Lr + (long long)(npad - 1 - i) * bp + (NB - 1 + t);
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (NB + t - j <= b) {
          const S ls = st_entry<S, float>(lv[j]);
          Lc[j * (bp - 1)] = ls;
          if (i < npad) Lrr[-j] = ls;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < NB; ++j) cv[j] = lv[j] = zero;
    }
    if (more) {
      tc_put_split<NB>(Aop, AB, kTcM, t, cv);
      if (t < N) tc_put_split<NB>(Bop, BB, N, t, lv);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (!more) break;
    tc_fence_after();
    // 3. trailing update on the tensor cores (descriptors: the start address
    //    field, bits 0-13 in 16-byte units, advances with the operand offset)
    if (tid == 0) {
      // (A array, B array, negate): Re += Prh Qrh + Prh Qrl + Prl Qrh - (Pih Qih + Pih Qil + Pil Qih)
      //                             Im += Prh Qih + Prh Qil + Prl Qih + Pih Qrh + Pih Qrl + Pil Qrh
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const uint32_t ta = (0x322100u >> (4 * u)) & 0xFu;    // 0, 0, 1, 2, 2, 3
        const uint32_t tre = (0x232010u >> (4 * u)) & 0xFu;   // 0, 1, 0, 2, 3, 2
        const uint32_t tim = (0x010232u >> (4 * u)) & 0xFu;   // 2, 3, 2, 0, 1, 0
#pragma unroll
        for (int s = 0; s < NB / 8; ++s) {
          const uint64_t ad = adesc0 + ((ta * AB + 2 * s * lba) >> 4);
          tc_mma_tf32(tmem, ad, bdesc0 + ((tre * BB + 2 * s * lbb) >> 4), u >= 3 ? idn : id, (u | s) ? 1u : 0u);
          tc_mma_tf32(tmem + (uint32_t)N, ad, bdesc0 + ((tim * BB + 2 * s * lbb) >> 4), id, (u | s) ? 1u : 0u);
        }
      }
      tc_commit(bar);
    }
    // 4. entering rows k+NB+b.. into the slots of rows k..k+NB-1 (warps 1-3,
    //    while warp 0 issues the MMAs)
    if (warp > 0) {
      const int r = k + NB + b + fq;
      tc_fill_row(ring, LDW, r % R, r, b, vcur, fsub, TPR);
    }
    // 5. accumulators back into the ring
    const bool ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      // a bounded wait gave up: record it, wait once more (bounded) for the MMAs in flight, leave
      if (tid == 0) atomicExch(&status->timeout, 1);
      mbar_wait_bounded(bar, phase ^ 1u);
      failed = true;
      break;
    }
    tc_fence_after();
    {
      const int nch = min(N / 16, 2 * warp + 2);
      c64* row = ring + (i % R) * LDW;
      for (int h = 0; h < nch; ++h) {
        float re[16], im[16];
        const uint32_t ta0 = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * h);
        tc_ld16x2(ta0, ta0 + (uint32_t)N, re, im);
        if (t < b) {
          // all loads first, then the stores (entries c <= t of row i)
          c64* w = row + (16 * h - t + b);
          c64 cur[16];
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (16 * h + u <= t) cur[u] = w[u];
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (16 * h + u <= t) w[u] = mk(cur[u].re - re[u], cur[u].im - im[u]);
        }
      }
    }
    tc_fence_before();
    if (warp == 0) {
      __syncwarp();
      tc_diag_block<NB>(k + NB, lane, ring, R, LDW, b, L11, dis, dmin2, dmax2, bad);
    }
    __syncthreads();
  }
  (void)failed;
  if (warp == 0) {
    // pivot statistics of the lanes that held pivots
    float mn = lane < NB ? dmin2 : 3e38f, mx = lane < NB ? dmax2 : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const bool anybad = __any_sync(0xffffffffu, lane < NB && bad);
    if (lane == 0) {
      pivstats[2 * sub] = sqrt((double)mn);
      pivstats[2 * sub + 1] = sqrt((double)mx);
      if (anybad) atomicCAS(&status->pivot_bad_sub, -1, sub);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

}  // namespace

int max_band(int prec) { return prec == 0 ? kMaxBandC128 : kMaxBandC64; }

size_t factor_smem_bytes(int b, int prec, int rank) {
  const size_t es = prec == 0 ? sizeof(c128) : sizeof(c64);   // window in the arithmetic type
  const size_t wc = (size_t)b + 1, nwin = wc * (wc + 1) / 2;
  if (rank == 2) return (nwin + (nwin & 1) + 4 * (wc + 1)) * es + 2 * wc * sizeof(int2);
  return (nwin + 2 * wc) * es + 2 * wc * sizeof(int2);
}

namespace {

template <typename R, typename S, int NT>
cudaError_t launch_factor_t(int rank, size_t smem, const SubDesc* subs, int nsub, const c128* Aloc, void* L,
                            void* Lrev, void* dinv, double* pivstats, DevStatus* status, cudaStream_t st, int bcap) {
  cudaError_t e;
  if (NT == 1024 || rank == 2) {
    e = cudaFuncSetAttribute(k_factor_ldlt2<R, S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt2<R, S, NT><<<nsub, NT, smem, st>>>(subs, Aloc, (S*)L, (S*)Lrev, (cx<R>*)dinv, pivstats, status,
                                                     bcap);
  } else if constexpr (NT < 1024) {
    e = cudaFuncSetAttribute(k_factor_ldlt<R, S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt<R, S, NT><<<nsub, NT, smem, st>>>(subs, Aloc, (S*)L, (S*)Lrev, (cx<R>*)dinv, pivstats, status,
                                                    bcap);
  }
  return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_factor_s(int threads, int rank, size_t smem, const SubDesc* subs, int nsub, const c128* Aloc,
                            void* L, void* Lrev, void* dinv, double* pivstats, DevStatus* status, cudaStream_t st,
                            int bcap) {
  switch (threads) {
    case 128: return launch_factor_t<R, S, 128>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st, bcap);
    case 256: return launch_factor_t<R, S, 256>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st, bcap);
    case 512: return launch_factor_t<R, S, 512>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st, bcap);
    case 1024:
      if (rank == 2)
        return launch_factor_t<R, S, 1024>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st, bcap);
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool factor_tc_ok(int prec, int max_b) { return prec >= 1 && max_b >= 1 && max_b <= kMaxBandTc; }

// max_b: the widest subdomain the shared-memory kernels take. Their steps give
// one thread to each of the b + 1 window diagonals (and the entering row), so
// a CUDA-core shape needs at least b + 2 threads.
bool factor_shape_valid(int prec, int max_b, int threads, int rank, BandSplit split) {
  if (rank == kRankTcBlocked)
    return prec >= 1 && split.nwide >= 0 && threads == kTcM && (split.max_b_tc == 0 || factor_tc_ok(prec, split.max_b_tc));
  if (is_tc_rank(rank)) {
    if (threads == kTcM) return factor_tc_ok(prec, max_b);
    return prec >= 1 && split.nwide >= 0 && (threads == 256 || threads == 512 || threads == 1024) &&
           threads >= max_b + 2;
  }
  return (((threads == 128 || threads == 256 || threads == 512) && (rank == 1 || rank == 2)) ||
          (threads == 1024 && rank == 2)) &&
         threads >= max_b + 2;
}

int narrow_band(int prec, int max_b, BandSplit split) {
  return max_b > max_band(prec) ? split.max_b_narrow : max_b;
}

namespace {

// shared memory of k_factor_tc<., NB> for half-bandwidths up to max_b, and
// its TMEM columns (a power of two >= 2N); the request is raised where
// needed so that the CTAs resident on one SM never ask for more than its 512
// columns
void tc_sizes(int max_b, int NB, size_t* smem, int* nmax, int* ring_elems, int* tcols) {
  *nmax = tc_n(max_b);
  *ring_elems = (NB + max_b) * (max_b + 2);
  int tc = 32;
  while (tc < 2 * *nmax) tc *= 2;
  *tcols = tc;
  size_t s = 4 * (size_t)tc_ab(NB) + 4 * (size_t)(*nmax) * NB * 4 + (size_t)(*ring_elems) * sizeof(c64) +
             (size_t)(NB * NB + NB) * sizeof(c64) + 16;
  const size_t per_sm = 228 * 1024, per_cta_reserved = 1024;
  while (per_sm / (s + per_cta_reserved) > (size_t)(512 / tc)) s += 1024;
  *smem = s;
}

template <typename S, int NB>
cudaError_t launch_factor_tc(const SubDesc* subs, int nsub, int max_b, const c128* Aloc, void* L, void* Lrev,
                             void* dinv, double* pivstats, DevStatus* status, cudaStream_t st, int sub_base) {
  size_t smem;
  int nmax, ring_elems, tcols;
  tc_sizes(max_b, NB, &smem, &nmax, &ring_elems, &tcols);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e =
      cudaFuncSetAttribute(k_factor_tc<S, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor_tc<S, NB><<<nsub, kTcM, smem, st>>>(subs, Aloc, (S*)L, (S*)Lrev, (c64*)dinv, pivstats, status, nmax,
                                               ring_elems, tcols, sub_base, max_b);
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch_factor_tc_nb(int rank, const SubDesc* subs, int nsub, int max_b, const c128* Aloc, void* L,
                                void* Lrev, void* dinv, double* pivstats, DevStatus* status, cudaStream_t st,
                                int sub_base = 0) {
  if (rank == 8) return launch_factor_tc<S, 8>(subs, nsub, max_b, Aloc, L, Lrev, dinv, pivstats, status, st, sub_base);
  return launch_factor_tc<S, 16>(subs, nsub, max_b, Aloc, L, Lrev, dinv, pivstats, status, st, sub_base);
}

// mixed shape: the wide subdomains (launch positions 0..nwide-1) on the CUDA
// cores with two pivots per pass (on st_cuda), the others on the tensor cores
// (on st)
template <typename S>
cudaError_t launch_factor_mixed(int threads, int rank, const SubDesc* subs, int nsub, int max_b, BandSplit sp,
                                const c128* Aloc, void* L, void* Lrev, void* dinv, double* pivstats,
                                DevStatus* status, cudaStream_t st, cudaStream_t st_cuda) {
  cudaError_t e = cudaSuccess;
  const int nw = sp.nwide < nsub ? sp.nwide : nsub;
  if (nw > 0)
    e = launch_factor_s<float, S>(threads, 2, factor_smem_bytes(max_b, 1, 2), subs, nw, Aloc, L, Lrev, dinv, pivstats,
                                  status, st_cuda, max_b);
  if (e == cudaSuccess && nsub > nw) {
    const int mb = nw > 0 ? sp.max_b_tc : max_b;
    if (!factor_tc_ok(1, mb)) return cudaErrorInvalidValue;
    e = launch_factor_tc_nb<S>(rank, subs, nsub - nw, mb, Aloc, L, Lrev, dinv, pivstats, status, st, nw);
  }
  return e;
}

}  // namespace

cudaError_t launch_factor(int prec, int threads, int rank, const SubDesc* subs, int nsub, int max_b,
                          const c128* Aloc, void* L, void* Lrev, void* dinv, double* pivstats, DevStatus* status,
                          cudaStream_t st, BandSplit split, void* wscratch, bool skip_wide, int wide_cluster,
                          const ApplyStreams* as) {
  if (rank == kRankTcBlocked) {
    // launch positions 0..nw-1 hold the subdomains with b > kMaxBandTc: the
    // blocked tensor-core kernel takes them up to max_band(prec) (all of
    // them when the wide-band shape is the tensor-core form too: one launch),
    // the wide-band shape those above; the rest go to the tensor-core kernel
    if (!factor_shape_valid(prec, max_b, threads, rank, split)) return cudaErrorInvalidValue;
    const int nw = std::min(split.nwide, nsub);
    const bool has_wide = max_b > max_band(prec) && !skip_wide;
    const int cl = wide_cluster > 0 ? wide_cluster : wide_cluster_auto(split.nblocked);
    const bool merged = has_wide && cl == kWideTensorCores;
    const bool conc = as != nullptr && as->side[0] != nullptr && as->side[1] != nullptr;
    cudaError_t e = cudaSuccess;
    if (conc) {
      e = cudaEventRecord(as->fork, st);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(as->side[i], as->fork, 0);
    }
    cudaStream_t s_wide = conc ? as->side[0] : st, s_mid = conc ? as->side[1] : st;
    if (e == cudaSuccess && has_wide && !merged)
      e = launch_factor_wide(prec, subs, nw, max_b, Aloc, L, Lrev, dinv, pivstats, status, wscratch, s_wide, cl);
    if (e == cudaSuccess && nw > 0)
      e = launch_factor_wide(prec, subs, nw, max_b, Aloc, L, Lrev, dinv, pivstats, status, wscratch,
                             merged ? s_wide : s_mid, kWideTensorCores, kMaxBandTc,
                             merged ? kMaxBandWide : max_band(prec));
    if (e == cudaSuccess && nsub > nw)
      e = prec == 1 ? launch_factor_tc_nb<c64>(16, subs, nsub - nw, split.max_b_tc, Aloc, L, Lrev, dinv, pivstats,
                                              status, st, nw)
                    : launch_factor_tc_nb<h2c>(16, subs, nsub - nw, split.max_b_tc, Aloc, L, Lrev, dinv, pivstats,
                                              status, st, nw);
    if (conc) {
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(as->join[i], as->side[i]);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, as->join[i], 0);
    }
    return e;
  }
  if (max_b > max_band(prec)) {
    // the subdomains wider than the shared-memory window first (blocked
    // kernel, window in scratch), then the others with the chosen shape,
    // sized for the widest of them; each launch skips the other kind
    const int cl = wide_cluster > 0 ? wide_cluster : wide_cluster_auto(split.nblocked);
    const bool conc = as != nullptr && as->side[0] != nullptr && as->side[1] != nullptr && !skip_wide &&
                      split.max_b_narrow > 0 && factor_shape_valid(prec, split.max_b_narrow, threads, rank, split);
    cudaError_t e = cudaSuccess;
    if (conc) {
      e = cudaEventRecord(as->fork, st);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(as->side[i], as->fork, 0);
    }
    if (e == cudaSuccess && !skip_wide)
      e = launch_factor_wide(prec, subs, nsub, max_b, Aloc, L, Lrev, dinv, pivstats, status, wscratch,
                             conc ? as->side[0] : st, cl);
    if (e != cudaSuccess || split.max_b_narrow <= 0) return e;
    if (conc) {
      const int mn = split.max_b_narrow;
      if (is_tc_rank(rank) && threads != kTcM)
        e = prec == 1 ? launch_factor_mixed<c64>(threads, rank, subs, nsub, mn, split, Aloc, L, Lrev, dinv, pivstats,
                                                 status, st, as->side[1])
                      : launch_factor_mixed<h2c>(threads, rank, subs, nsub, mn, split, Aloc, L, Lrev, dinv, pivstats,
                                                 status, st, as->side[1]);
      else
        e = launch_factor(prec, threads, rank, subs, nsub, mn, Aloc, L, Lrev, dinv, pivstats, status, as->side[1],
                          split, nullptr, true, 0, nullptr);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(as->join[i], as->side[i]);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, as->join[i], 0);
      return e;
    }
    max_b = split.max_b_narrow;
  }
  if (!factor_shape_valid(prec, max_b, threads, rank, split)) return cudaErrorInvalidValue;
  if (is_tc_rank(rank) && threads != kTcM) {
    if (prec == 1)
      return launch_factor_mixed<c64>(threads, rank, subs, nsub, max_b, split, Aloc, L, Lrev, dinv, pivstats, status, st,
                                      st);
    return launch_factor_mixed<h2c>(threads, rank, subs, nsub, max_b, split, Aloc, L, Lrev, dinv, pivstats, status, st,
                                    st);
  }
  if (is_tc_rank(rank)) {
    if (prec == 1) return launch_factor_tc_nb<c64>(rank, subs, nsub, max_b, Aloc, L, Lrev, dinv, pivstats, status, st);
    return launch_factor_tc_nb<h2c>(rank, subs, nsub, max_b, Aloc, L, Lrev, dinv, pivstats, status, st);
  }
  const size_t smem = factor_smem_bytes(max_b, prec, rank);
  if (prec == 0)
    return launch_factor_s<double, c128>(threads, rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st,
                                         max_b);
  if (prec == 1)
    return launch_factor_s<float, c64>(threads, rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st,
                                       max_b);
  return launch_factor_s<float, h2c>(threads, rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st,
                                     max_b);
}

}  // namespace rp
