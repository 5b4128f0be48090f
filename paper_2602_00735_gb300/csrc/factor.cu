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
#include "common.cuh"
#include "kernels.h"

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
                  DevStatus* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
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
                   DevStatus* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
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
                            void* Lrev, void* dinv, double* pivstats, DevStatus* status, cudaStream_t st) {
  cudaError_t e;
  if (NT == 1024 || rank == 2) {
    e = cudaFuncSetAttribute(k_factor_ldlt2<R, S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt2<R, S, NT><<<nsub, NT, smem, st>>>(subs, Aloc, (S*)L, (S*)Lrev, (cx<R>*)dinv, pivstats, status);
  } else if constexpr (NT < 1024) {
    e = cudaFuncSetAttribute(k_factor_ldlt<R, S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_factor_ldlt<R, S, NT><<<nsub, NT, smem, st>>>(subs, Aloc, (S*)L, (S*)Lrev, (cx<R>*)dinv, pivstats, status);
  }
  return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_factor_s(int threads, int rank, size_t smem, const SubDesc* subs, int nsub, const c128* Aloc,
                            void* L, void* Lrev, void* dinv, double* pivstats, DevStatus* status, cudaStream_t st) {
  switch (threads) {
    case 128: return launch_factor_t<R, S, 128>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
    case 256: return launch_factor_t<R, S, 256>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
    case 512: return launch_factor_t<R, S, 512>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
    case 1024:
      if (rank == 2)
        return launch_factor_t<R, S, 1024>(rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool factor_shape_valid(int threads, int rank) {
  return ((threads == 128 || threads == 256 || threads == 512) && (rank == 1 || rank == 2)) ||
         (threads == 1024 && rank == 2);
}

cudaError_t launch_factor(int prec, int threads, int rank, const SubDesc* subs, int nsub, int max_b,
                          const c128* Aloc, void* L, void* Lrev, void* dinv, double* pivstats, DevStatus* status,
                          cudaStream_t st) {
  if (!factor_shape_valid(threads, rank)) return cudaErrorInvalidValue;
  const size_t smem = factor_smem_bytes(max_b, prec, rank);
  if (prec == 0)
    return launch_factor_s<double, c128>(threads, rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
  if (prec == 1)
    return launch_factor_s<float, c64>(threads, rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
  return launch_factor_s<float, h2c>(threads, rank, smem, subs, nsub, Aloc, L, Lrev, dinv, pivstats, status, st);
}

}  // namespace rp
