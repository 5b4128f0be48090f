// The RAS-PML apply z = B^-1 r = sum_j R_j^T (chi_j .* A_j^-1 R_j r)
// (Section 2, the equation defining B^-1; restriction as in
// eq. local-ras-discrete, weighted prolongation as in eq. update1).
//
// k_apply: one warp per subdomain computes R_j r (a gather of the global
//   residual), y = L^-1 R_j r, z = D^-1 y, x = L^-T z, and writes chi_j .* x
//   to the subdomain's slice of Y. Both triangular solves run as the same
//   column sweep on a unit lower band matrix stored by columns: the forward
//   sweep reads L by columns, the backward sweep reads the row-band copy of
//   L stored in reversed row order (column k' of that copy is row npad-1-k'
//   of L read leftwards), so that L^T x = z becomes a forward sweep on
//   reversed vectors.
//   Sweep: the rows k..k+32S-1 of the right-hand side live in a register
//   window, row r in lane r mod 32, slot (r/32) mod S, S = ceil((b+1)/32).
//   Step k broadcasts the finished row k from its lane, subtracts
//   column k times y_k from the rows below (one complex FMA per slot and
//   lane), and refills row k's slot with row k+32S.
//   The band columns stream from HBM through a 4-stage shared-memory ring of
//   8-column chunks filled by the bulk-copy (TMA) engine; both sweeps use one
//   continuous chunk sequence.
// k_prolong: one thread per global unknown sums the (at most four) weighted
//   local values that cover it, in a fixed order (bit-reproducible).
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

constexpr int kCol = 8;       // columns per bulk copy
// ring depth: 4 stages of 8 columns (a deeper ring for half-pair entries was
// measured: no gain on c2, slower on c4)
template <typename ST>
constexpr int stages_for() { return 4; }

// R_j r at local row `row`: r is complex128, or double-float (dfc) when rdf
template <typename R>
__device__ __forceinline__ cx<R> gather_row(const SubDesc& sd, const Geo& g, const c128* __restrict__ r, int rdf,
                                            int row) {
  if (row >= sd.n) return mk((R)0, (R)0);
  int i = sd.ix0 + row % sd.nlx, j = sd.iy0 + row / sd.nlx;
  const long long idx = (long long)(j - 1) * g.nx + (i - 1);
  if (rdf) {
    const dfc v = reinterpret_cast<const dfc*>(r)[idx];
    return mk((R)((R)v.rh + (R)v.rl), (R)((R)v.ih + (R)v.il));
  }
  return cvt<R>(r[idx]);
}

template <typename S>
struct Pipe {
  uint64_t* bar;
  S* stg;
  const S* src0;       // forward band (columns of L)
  const S* src1;       // reversed row band of L
  int stage_elems, Q, bp;
  uint32_t bytes;
  __device__ void issue(int s) const {
    const S* src = s < Q ? src0 + (long long)s * kCol * bp : src1 + (long long)(s - Q) * kCol * bp;
    const int st = s % stages_for<S>();
    mbar_arrive_expect_tx(&bar[st], bytes);
    bulk_g2s(stg + st * stage_elems, src, bytes, &bar[st]);
  }
  __device__ const S* wait(int s, bool& ok) const {
    const int st = s % stages_for<S>();
    ok = mbar_wait_bounded(&bar[st], (uint32_t)((s / stages_for<S>()) & 1));
    return stg + st * stage_elems;
  }
};

// The 32 steps of one row group with window phase PH (= group mod S);
// ST is the storage type of the factor entries.
template <typename R, typename ST, int S, int PH>
__device__ __forceinline__ bool group_steps(const Pipe<ST>& pp, int s0, int b, int lane, cx<R> (&win)[S],
                                            const cx<R>& nxt, cx<R>& outv) {
  const int bp = pp.bp;
#pragma unroll 1
  for (int c4 = 0; c4 < 32 / kCol; ++c4) {
    const int s = s0 + c4;
    bool ok;
    const ST* Lc = pp.wait(s, ok);
    if (!__all_sync(0xffffffffu, ok)) return false;
#pragma unroll 2
    for (int ii = 0; ii < kCol; ++ii) {
      const int i = c4 * kCol + ii;
      const ST* col = Lc + ii * bp;
      const cx<R> y = shfl(win[PH], i);
      if (lane == i) {
        outv = y;
        win[PH] = nxt;
      }
      const int base = lane - i - 1;
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        const int t = (sl == PH) ? ((lane > i) ? base : base + 32 * S) : base + 32 * ((sl - PH + S) % S);
        if (t < b) win[sl] = fms(win[sl], ld_entry(col[t]), y);
      }
    }
    __syncwarp();
    if (lane == 0 && s + stages_for<ST>() < 2 * pp.Q) {
      fence_proxy_async_smem();
      pp.issue(s + stages_for<ST>());
    }
  }
  return true;
}

template <typename R, typename ST, int S>
__device__ __forceinline__ bool group_dispatch(int ph, const Pipe<ST>& pp, int s0, int b, int lane, cx<R> (&win)[S],
                                               const cx<R>& nxt, cx<R>& outv) {
  switch (ph) {
    case 0: return group_steps<R, ST, S, 0>(pp, s0, b, lane, win, nxt, outv);
    case 1: if constexpr (S > 1) return group_steps<R, ST, S, 1>(pp, s0, b, lane, win, nxt, outv); break;
    case 2: if constexpr (S > 2) return group_steps<R, ST, S, 2>(pp, s0, b, lane, win, nxt, outv); break;
    case 3: if constexpr (S > 3) return group_steps<R, ST, S, 3>(pp, s0, b, lane, win, nxt, outv); break;
    case 4: if constexpr (S > 4) return group_steps<R, ST, S, 4>(pp, s0, b, lane, win, nxt, outv); break;
    case 5: if constexpr (S > 5) return group_steps<R, ST, S, 5>(pp, s0, b, lane, win, nxt, outv); break;
    case 6: if constexpr (S > 6) return group_steps<R, ST, S, 6>(pp, s0, b, lane, win, nxt, outv); break;
    case 7: if constexpr (S > 7) return group_steps<R, ST, S, 7>(pp, s0, b, lane, win, nxt, outv); break;
  }
  return false;
}

template <typename R, typename ST, int S>
__global__ void __launch_bounds__(32)
    k_apply(Geo g, const SubDesc* __restrict__ subs, const ST* __restrict__ Lf, const ST* __restrict__ Lb,
            const cx<R>* __restrict__ dinv_all, const c128* __restrict__ rglob, int rdf, cx<R>* __restrict__ Y,
            int stage_elems, const KState* __restrict__ kst, DevStatus* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  if (kst != nullptr && kst->stop) return;
  const SubDesc sd = subs[blockIdx.x];
  const int lane = threadIdx.x;
  const int b = sd.b, npad = sd.npad, G = npad / 32;
  Pipe<ST> pp;
  pp.bar = reinterpret_cast<uint64_t*>(sm);
  pp.stg = reinterpret_cast<ST*>(sm + 128);
  pp.src0 = Lf + sd.l_off;
  pp.src1 = Lb + sd.l_off;
  pp.stage_elems = stage_elems;
  pp.Q = npad / kCol;
  pp.bp = sd.bp;
  pp.bytes = (uint32_t)(kCol * sd.bp * sizeof(ST));
  const cx<R>* dv = dinv_all + sd.v_off;
  cx<R>* Yj = Y + sd.v_off;
  const int nseq = 2 * pp.Q;
  constexpr int NST = stages_for<ST>();
  if (lane == 0) {
    for (int t = 0; t < NST; ++t) mbar_init(&pp.bar[t], 1);
    mbar_fence_init();
    for (int t = 0; t < NST && t < nseq; ++t) pp.issue(t);
  }
  __syncwarp();
  auto fail = [&](int s) {
    // a bounded wait gave up: record it, drain this warp's copies in flight, leave
    if (lane == 0) {
      atomicExch(&status->timeout, 1);
      for (int t = s; t < s + NST && t < nseq; ++t) mbar_wait_bounded(&pp.bar[t % NST], (t / NST) & 1);
    }
    __syncwarp();
  };

  // ---------------- forward: L y = R_j r, z = D^-1 y ----------------
  cx<R> win[S];
#pragma unroll
  for (int sl = 0; sl < S; ++sl) win[sl] = gather_row<R>(sd, g, rglob, rdf, 32 * sl + lane);
  cx<R> nxt = gather_row<R>(sd, g, rglob, rdf, 32 * S + lane);
  for (int gi = 0; gi < G; ++gi) {
    const cx<R> nxt2 = gather_row<R>(sd, g, rglob, rdf, 32 * (gi + S + 1) + lane);
    const cx<R> d = dv[32 * gi + lane];
    cx<R> outv;
    if (!group_dispatch<R, ST, S>(gi % S, pp, 4 * gi, b, lane, win, nxt, outv)) { fail(4 * gi); return; }
    Yj[32 * gi + lane] = outv * d;
    nxt = nxt2;
  }
  __threadfence_block();
  __syncwarp();

  // ---------------- backward: L^T x = z on reversed rows ----------------
  auto zrow = [&](int q) -> cx<R> { return q < npad ? Yj[npad - 1 - q] : mk((R)0, (R)0); };
#pragma unroll
  for (int sl = 0; sl < S; ++sl) win[sl] = zrow(32 * sl + lane);
  nxt = zrow(32 * S + lane);
  const int o = g.ovlp;
  for (int gi = 0; gi < G; ++gi) {
    const cx<R> nxt2 = zrow(32 * (gi + S + 1) + lane);
    cx<R> outv;
    if (!group_dispatch<R, ST, S>(gi % S, pp, pp.Q + 4 * gi, b, lane, win, nxt, outv)) {
      fail(pp.Q + 4 * gi);
      return;
    }
    const int row = npad - 1 - (32 * gi + lane);
    cx<R> v = mk((R)0, (R)0);
    if (row < sd.n) {
      const int i = sd.ix0 + row % sd.nlx, j = sd.iy0 + row / sd.nlx;
      v = (R)pou_weight(sd, i, j, o) * outv;
    }
    Yj[row] = v;
    nxt = nxt2;
  }
}

template <typename R>
__global__ void k_prolong(Geo g, const SubDesc* __restrict__ subs, const cx<R>* __restrict__ Y,
                          c128* __restrict__ z, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = (long long)g.nx * g.ny;
  if (r >= n) return;
  const int i = (int)(r % g.nx) + 1, j = (int)(r / g.nx) + 1;
  const int o = g.ovlp;
  int bx = box_of_node(i, g.Mx, g.px), by = box_of_node(j, g.My, g.py);
  int qx0 = bx, qx1 = bx, qy0 = by, qy1 = by;
  if (bx > 0 && i < box_start(bx, g.Mx, g.px) + o) qx0 = bx - 1;
  if (bx + 1 < g.px && i > box_start(bx + 1, g.Mx, g.px) - o) qx1 = bx + 1;
  if (by > 0 && j < box_start(by, g.My, g.py) + o) qy0 = by - 1;
  if (by + 1 < g.py && j > box_start(by + 1, g.My, g.py) - o) qy1 = by + 1;
  double re = 0.0, im = 0.0;
  for (int qy = qy0; qy <= qy1; ++qy) {
    for (int qx = qx0; qx <= qx1; ++qx) {
      const SubDesc& sd = subs[qy * g.px + qx];
      const int li = i - sd.ix0, lj = j - sd.iy0;
      if (li < 0 || li >= sd.nlx || lj < 0 || lj >= sd.nly) continue;
      const cx<R> v = Y[sd.v_off + (long long)lj * sd.nlx + li];
      re += (double)v.re;
      im += (double)v.im;
    }
  }
  z[r] = mk(re, im);
}

template <typename R, typename ST, int S>
cudaError_t launch_apply_t(const Geo& g, const SubDesc* subs, int nsub, int max_bp, const void* Lf, const void* Lb,
                           const void* dinv, const c128* r, int rdf, void* Y, const KState* kst, DevStatus* status,
                           cudaStream_t st) {
  const int stage_elems = kCol * max_bp;
  const size_t smem = 128 + (size_t)stages_for<ST>() * kCol * max_bp * sizeof(ST);
  cudaError_t e = cudaFuncSetAttribute(k_apply<R, ST, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_apply<R, ST, S><<<nsub, 32, smem, st>>>(g, subs, (const ST*)Lf, (const ST*)Lb, (const cx<R>*)dinv, r, rdf,
                                            (cx<R>*)Y, stage_elems, kst, status);
  return cudaGetLastError();
}

template <typename R, typename ST>
cudaError_t launch_apply_s(int S, const Geo& g, const SubDesc* subs, int nsub, int max_bp, const void* Lf,
                           const void* Lb, const void* dinv, const c128* r, int rdf, void* Y, const KState* kst,
                           DevStatus* status, cudaStream_t st) {
  switch (S) {
    case 1: return launch_apply_t<R, ST, 1>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
    case 2: return launch_apply_t<R, ST, 2>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
    case 3: return launch_apply_t<R, ST, 3>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
    case 4: return launch_apply_t<R, ST, 4>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
    case 5: return launch_apply_t<R, ST, 5>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
    case 6: return launch_apply_t<R, ST, 6>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
  }
  if constexpr (sizeof(R) == 4) {
    // complex64 factors allow bands up to 232 (b + 1 <= 256)
    if (S == 7) return launch_apply_t<R, ST, 7>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
    if (S == 8) return launch_apply_t<R, ST, 8>(g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

size_t apply_smem_bytes(int max_bp, int prec) {
  if (prec == 0) return 128 + (size_t)stages_for<c128>() * kCol * max_bp * sizeof(c128);
  if (prec == 1) return 128 + (size_t)stages_for<c64>() * kCol * max_bp * sizeof(c64);
  return 128 + (size_t)stages_for<h2c>() * kCol * max_bp * sizeof(h2c);
}

cudaError_t launch_apply(int prec, const Geo& g, const SubDesc* subs, int nsub, int max_b, int max_bp,
                         const void* Lf, const void* Lb, const void* dinv, const c128* r, void* Y, c128* z,
                         const KState* kst, DevStatus* status, cudaStream_t st, bool r_is_df) {
  const int rdf = r_is_df ? 1 : 0;
  const int S = (max_b + 1 + 31) / 32;
  cudaError_t e;
  if (prec == 0)
    e = launch_apply_s<double, c128>(S, g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
  else if (prec == 1)
    e = launch_apply_s<float, c64>(S, g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
  else
    e = launch_apply_s<float, h2c>(S, g, subs, nsub, max_bp, Lf, Lb, dinv, r, rdf, Y, kst, status, st);
  if (e != cudaSuccess) return e;
  long long n = (long long)g.nx * g.ny;
  int threads = 256;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (prec == 0)
    k_prolong<double><<<blocks, threads, 0, st>>>(g, subs, (const c128*)Y, z, kst);
  else
    k_prolong<float><<<blocks, threads, 0, st>>>(g, subs, (const c64*)Y, z, kst);
  return cudaGetLastError();
}

}  // namespace rp
