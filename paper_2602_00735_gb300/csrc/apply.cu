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
//   KC-column chunks (KC = 4, 8 or 16, a tuned tile shape) filled by the
//   bulk-copy (TMA) engine; both sweeps use one continuous chunk sequence.
//   Subdomains may belong to different problems of a batch: each reads its
//   problem's geometry (geos[prob]) and skips when that problem has stopped.
// k_apply_mw: the same sweeps for the wide band classes (more register slots
//   than one warp's phase-dispatched window holds) on several warps per
//   subdomain, each holding the row group being finished and a share of the
//   slots below it; every row takes its updates in the order of a one-warp
//   sweep (two warps measured bit for bit equal to one).
// k_prolong: one thread per global unknown sums the (at most four) weighted
//   local values that cover it, in a fixed order (bit-reproducible): in FP64
//   into complex128 (or split into the double-float form), or, for complex64
//   local values, in double-float on the FP32 pipe into the double-float form
//   (dfc) the Arnoldi SpMV reads.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

// Limit of the waits for the ring's bulk copies, in SM clock cycles: the
// default bound (about a second), or a smaller one set from the host to
// inject a time-out (ras_pml_set_copy_wait_limit). The drain after a time-out
// always waits with the default bound.
__device__ long long g_copy_wait_limit = kWaitLimitCycles;

// ring depth: 4 stages of 8 columns (a deeper ring for half-pair entries was
// measured: no gain on c2, slower on c4)
template <typename ST>
constexpr int stages_for() { return 4; }

// R_j r at local row `row`: r is complex128 (rdf 0), double-float dfc
// (rdf 1) or complex64 (rdf 2)
template <typename R>
__device__ __forceinline__ cx<R> gather_row(const SubDesc& sd, int nx, long long goff, const c128* __restrict__ r,
                                            int rdf, int row) {
  if (row >= sd.n) return mk((R)0, (R)0);
  int i = sd.ix0 + row % sd.nlx, j = sd.iy0 + row / sd.nlx;
  const long long idx = goff + (long long)(j - 1) * nx + (i - 1);
  if (rdf == 1) {
    const dfc v = reinterpret_cast<const dfc*>(r)[idx];
    return mk((R)((R)v.rh + (R)v.rl), (R)((R)v.ih + (R)v.il));
  }
  if (rdf == 2) return cvt<R>(reinterpret_cast<const c64*>(r)[idx]);
  return cvt<R>(r[idx]);
}

template <typename S, int KC>
struct Pipe {
  uint64_t* bar;
  S* stg;
  const S* src0;       // forward band (columns of L)
  const S* src1;       // reversed row band of L
  int stage_elems, Q, bp;
  uint32_t bytes;
  long long limit;     // wait limit of the copies (g_copy_wait_limit)
  __device__ void issue(int s) const {
    const S* src = s < Q ? src0 + (long long)s * KC * bp : src1 + (long long)(s - Q) * KC * bp;
    const int st = s % stages_for<S>();
    mbar_arrive_expect_tx(&bar[st], bytes);
    bulk_g2s(stg + st * stage_elems, src, bytes, &bar[st]);
  }
  __device__ const S* wait(int s, bool& ok) const {
    const int st = s % stages_for<S>();
    // limit 1: every wait gives up at once (the deterministic form of the
    // failure injection); otherwise a bounded wait
    ok = limit > 1 && mbar_wait_limited(&bar[st], (uint32_t)((s / stages_for<S>()) & 1), limit);
    return stg + st * stage_elems;
  }
};

// The 32 steps of one row group with window phase PH (= group mod S);
// ST is the storage type of the factor entries.
template <typename R, typename ST, int S, int KC, int PH>
__device__ __forceinline__ bool group_steps(const Pipe<ST, KC>& pp, int s0, int b, int lane, cx<R> (&win)[S],
                                            const cx<R>& nxt, cx<R>& outv) {
  const int bp = pp.bp;
#pragma unroll 1
  for (int c4 = 0; c4 < 32 / KC; ++c4) {
    const int s = s0 + c4;
    bool ok;
    const ST* Lc = pp.wait(s, ok);
    if (!__all_sync(0xffffffffu, ok)) return false;
#pragma unroll 2
    for (int ii = 0; ii < KC; ++ii) {
      const int i = c4 * KC + ii;
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

template <typename R, typename ST, int S, int KC>
__device__ __forceinline__ bool group_dispatch(int ph, const Pipe<ST, KC>& pp, int s0, int b, int lane,
                                               cx<R> (&win)[S], const cx<R>& nxt, cx<R>& outv) {
  switch (ph) {
    case 0: return group_steps<R, ST, S, KC, 0>(pp, s0, b, lane, win, nxt, outv);
    case 1: if constexpr (S > 1) return group_steps<R, ST, S, KC, 1>(pp, s0, b, lane, win, nxt, outv); break;
    case 2: if constexpr (S > 2) return group_steps<R, ST, S, KC, 2>(pp, s0, b, lane, win, nxt, outv); break;
    case 3: if constexpr (S > 3) return group_steps<R, ST, S, KC, 3>(pp, s0, b, lane, win, nxt, outv); break;
    case 4: if constexpr (S > 4) return group_steps<R, ST, S, KC, 4>(pp, s0, b, lane, win, nxt, outv); break;
    case 5: if constexpr (S > 5) return group_steps<R, ST, S, KC, 5>(pp, s0, b, lane, win, nxt, outv); break;
    case 6: if constexpr (S > 6) return group_steps<R, ST, S, KC, 6>(pp, s0, b, lane, win, nxt, outv); break;
    case 7: if constexpr (S > 7) return group_steps<R, ST, S, KC, 7>(pp, s0, b, lane, win, nxt, outv); break;
  }
  return false;
}

// The two sweeps of one subdomain with an S-slot register window (S >= the
// subdomain's ceil((b+1)/32)); the bulk-copy ring is already started.
template <typename R, typename ST, int S, int KC>
__device__ __forceinline__ void sweeps(const SubDesc& sd, const Pipe<ST, KC>& pp, int nx, long long goff, int o,
                                       const c128* __restrict__ rglob, int rdf, const cx<R>* __restrict__ dv,
                                       cx<R>* __restrict__ Yj, DevStatus* status) {
  const int lane = threadIdx.x;
  const int b = sd.b, npad = sd.npad, G = npad / 32;
  const int nseq = 2 * pp.Q;
  constexpr int NST = stages_for<ST>();
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
  for (int sl = 0; sl < S; ++sl) win[sl] = gather_row<R>(sd, nx, goff, rglob, rdf, 32 * sl + lane);
  cx<R> nxt = gather_row<R>(sd, nx, goff, rglob, rdf, 32 * S + lane);
  for (int gi = 0; gi < G; ++gi) {
    const cx<R> nxt2 = gather_row<R>(sd, nx, goff, rglob, rdf, 32 * (gi + S + 1) + lane);
    const cx<R> d = dv[32 * gi + lane];
    cx<R> outv;
    const bool ok = group_dispatch<R, ST, S, KC>(gi % S, pp, (32 / KC) * gi, b, lane, win, nxt, outv);
    if (!ok) {
      fail((32 / KC) * gi);
      return;
    }
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
  for (int gi = 0; gi < G; ++gi) {
    const cx<R> nxt2 = zrow(32 * (gi + S + 1) + lane);
    cx<R> outv;
    const bool ok = group_dispatch<R, ST, S, KC>(gi % S, pp, pp.Q + (32 / KC) * gi, b, lane, win, nxt, outv);
    if (!ok) {
      fail(pp.Q + (32 / KC) * gi);
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

// One warp per subdomain; the register window is sized per subdomain
// (S = ceil((b+1)/32)), so subdomains of different bands share one launch
// without the small ones paying for the largest window: the subdomains with
// smin <= S <= smax (<= SMAX, the phase-dispatched window). Each launch
// returns at once for the subdomains outside its band class, before it issues
// any copy. rbase + (*jptr) * r_ld is the input vector when jptr is set (a
// step of a captured Arnoldi graph reads its column index from device memory).
template <typename R, typename ST, int SMAX, int KC>
__global__ void __launch_bounds__(32)
    k_apply(const Geo* __restrict__ geos, const SubDesc* __restrict__ subs, const ST* __restrict__ Lf,
            const ST* __restrict__ Lb, const cx<R>* __restrict__ dinv_all, const c128* __restrict__ rbase,
            long long r_ld, const int* __restrict__ jptr, int rdf, cx<R>* __restrict__ Y, int stage_elems,
            const KState* __restrict__ kst, DevStatus* status, int smin, int smax) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
  const int S = (sd.b + 32) / 32;
  // this launch's band class (smin..smax register slots, smax <= SMAX)
  if (S < smin || S > smax) return;
  if (kst != nullptr && kst[sd.prob].stop) return;
  const int nx = geos[sd.prob].nx, o = geos[sd.prob].ovlp;
  const long long goff = geos[sd.prob].goff;
  const c128* rglob = rbase;
  if (jptr != nullptr)
    rglob = rdf == 2 ? (const c128*)((const c64*)rbase + (long long)(*jptr) * r_ld)
                     : (const c128*)((const dfc*)rbase + (long long)(*jptr) * r_ld);
  const int lane = threadIdx.x;
  Pipe<ST, KC> pp;
  pp.bar = reinterpret_cast<uint64_t*>(sm);
  pp.stg = reinterpret_cast<ST*>(sm + 128);
  pp.src0 = Lf + sd.l_off;
  pp.src1 = Lb + sd.l_off;
  pp.stage_elems = stage_elems;
  pp.Q = sd.npad / KC;
  pp.bp = sd.bp;
  pp.bytes = (uint32_t)(KC * sd.bp * sizeof(ST));
  pp.limit = g_copy_wait_limit;
  const int nseq = 2 * pp.Q;
  constexpr int NST = stages_for<ST>();
  if (lane == 0) {
    for (int t = 0; t < NST; ++t) mbar_init(&pp.bar[t], 1);
    mbar_fence_init();
    for (int t = 0; t < NST && t < nseq; ++t) pp.issue(t);
  }
  __syncwarp();
  const cx<R>* dv = dinv_all + sd.v_off;
  cx<R>* Yj = Y + sd.v_off;
#define RP_CASE(S_) \
  case S_:          \
    if constexpr (S_ <= SMAX) sweeps<R, ST, S_, KC>(sd, pp, nx, goff, o, rglob, rdf, dv, Yj, status); \
    break;
  switch (S) { RP_CASE(1) RP_CASE(2) RP_CASE(3) RP_CASE(4) RP_CASE(5) RP_CASE(6) RP_CASE(7) RP_CASE(8) }
  static_assert(SMAX <= 8, "the case list covers S = 1..SMAX");
#undef RP_CASE
}

// The wide class on W warps per subdomain (a CTA of 32 W threads). Every
// warp keeps the row group being finished (slot 0) and performs its 32 steps
// itself, so the multiplier y_k of each step comes from a shuffle inside the
// warp, the same in every warp (explicit FMAs); the other S - 1 slots are shared
// out, warp w holding slots 1 + w SPW .. (SPW = ceil((S - 1) / W)). After
// each group the window moves up one slot: warp 0's first slot becomes every
// warp's slot 0, warp w's first slot becomes warp w-1's last, and the rows
// entering at the bottom (collected in slot 0, whose lanes take them as they
// finish their rows) go to the warp holding slot S - 1; one block barrier and
// 32 W entries through shared memory per group. The copy ring is shared: one
// block barrier per stage combines the warps' wait results and frees the
// previous stage, whose refill thread 0 then issues. Two warps measured
// fastest on a batch of 64 problems with 208 wide subdomains (b up to 408;
// four warps: more barriers per slot).
// The KC steps of one ring stage for warp WI: slot 0 and the warp's SPW
// slots. Slots 1..S-2 lie inside the band for every lane and step (their
// entry t = lane - i - 1 + 32 g is at most 32 S - 34 < b, since S =
// floor((b + 32) / 32)); only slot 0 (rows entering at the bottom) and slot
// S - 1 are checked against b. WI is a template argument so that each slot's
// offset in the column is an immediate.
template <typename R, typename ST, int S, int KC, int W, int WI>
__device__ __forceinline__ void stage_steps_mw(const ST* __restrict__ Lc, int bp, int c4, int b, int lane,
                                               cx<R>& win0, cx<R> (&own)[(S - 1 + W - 1) / W], const cx<R>& nxt,
                                               cx<R>& outv) {
  constexpr int SPW = (S - 1 + W - 1) / W;
  constexpr int G0 = 1 + WI * SPW;
#pragma unroll 4
  for (int ii = 0; ii < KC; ++ii) {
    const int i = c4 * KC + ii;
    const int base = lane - i - 1;
    const ST* col = Lc + ii * bp + base;   // entry t of the column at col[t - base]
    const cx<R> y = shfl(win0, i);
    if (lane == i) {
      outv = y;
      win0 = nxt;
    }
    {
      const int off = (lane > i) ? 0 : 32 * S;
      if (base + off < b) win0 = fms(win0, ld_entry(col[off]), y);
    }
#pragma unroll
    for (int m = 0; m < SPW; ++m) {
      if (G0 + m < S - 1) {
        own[m] = fms(own[m], ld_entry(col[32 * (G0 + m)]), y);
      } else if (G0 + m == S - 1) {
        if (base + 32 * (S - 1) < b) own[m] = fms(own[m], ld_entry(col[32 * (S - 1)]), y);
      }
    }
  }
}

template <typename R, typename ST, int S, int KC, int W, int WI>
__device__ __forceinline__ void stage_dispatch_mw(int w, const ST* Lc, int bp, int c4, int b, int lane, cx<R>& win0,
                                                  cx<R> (&own)[(S - 1 + W - 1) / W], const cx<R>& nxt,
                                                  cx<R>& outv) {
  if constexpr (WI < W) {
    if (w == WI) {
      stage_steps_mw<R, ST, S, KC, W, WI>(Lc, bp, c4, b, lane, win0, own, nxt, outv);
      return;
    }
    stage_dispatch_mw<R, ST, S, KC, W, WI + 1>(w, Lc, bp, c4, b, lane, win0, own, nxt, outv);
  }
}

template <typename R, typename ST, int S, int KC, int W>
__device__ __forceinline__ bool group_steps_mw(const Pipe<ST, KC>& pp, int s0, int b, int lane, int w,
                                               cx<R>& win0, cx<R> (&own)[(S - 1 + W - 1) / W], const cx<R>& nxt,
                                               cx<R>& outv, cx<R>* xch, int& sfail) {
  constexpr int SPW = (S - 1 + W - 1) / W;
  constexpr int NST = stages_for<ST>();
  const int g0 = 1 + w * SPW;
#pragma unroll 1
  for (int c4 = 0; c4 < 32 / KC; ++c4) {
    const int s = s0 + c4;
    bool ok;
    const ST* Lc = pp.wait(s, ok);
    if (!__syncthreads_and(ok)) {
      sfail = s;
      return false;
    }
    // every warp is past stage s - 1: its buffer takes stage s - 1 + NST
    if (threadIdx.x == 0 && s > 0 && s - 1 + NST < 2 * pp.Q) {
      fence_proxy_async_smem();
      pp.issue(s - 1 + NST);
    }
    // the steps themselves have no barrier: the warps take their own code
    stage_dispatch_mw<R, ST, S, KC, W, 0>(w, Lc, pp.bp, c4, b, lane, win0, own, nxt, outv);
  }
  // move the window up one slot
  xch[w * 32 + lane] = own[0];
  __syncthreads();
  const cx<R> f = win0;   // the rows entering at the bottom: slot S - 1
  win0 = xch[lane];
#pragma unroll
  for (int m = 0; m + 1 < SPW; ++m) own[m] = own[m + 1];
  if (w + 1 < W) own[SPW - 1] = xch[(w + 1) * 32 + lane];
  if (S - 1 >= g0 && S - 1 < g0 + SPW) {
#pragma unroll
    for (int m = 0; m < SPW; ++m)
      if (g0 + m == S - 1) own[m] = f;
  }
  return true;
}

template <typename R, typename ST, int S, int KC, int W>
__device__ __forceinline__ void sweeps_mw(const SubDesc& sd, const Pipe<ST, KC>& pp, int nx, long long goff, int o,
                                          const c128* __restrict__ rglob, int rdf, const cx<R>* __restrict__ dv,
                                          cx<R>* __restrict__ Yj, cx<R>* xch, DevStatus* status) {
  constexpr int SPW = (S - 1 + W - 1) / W;
  constexpr int NST = stages_for<ST>();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = sd.b, npad = sd.npad, G = npad / 32;
  const int nseq = 2 * pp.Q, g0 = 1 + w * SPW;
  const cx<R> zero = mk((R)0, (R)0);
  auto fail = [&](int s) {
    // a bounded wait gave up: record it, drain the copies in flight (stages
    // s .. s + NST - 1 issued before the first stage's barrier, s .. s + NST - 2
    // after it), leave
    if (threadIdx.x == 0) {
      atomicExch(&status->timeout, 1);
      const int hi = s + (s == 0 ? NST : NST - 1);
      for (int t = s; t < hi && t < nseq; ++t) mbar_wait_bounded(&pp.bar[t % NST], (t / NST) & 1);
    }
  };
  int sfail = 0;

  // ---------------- forward: L y = R_j r, z = D^-1 y ----------------
  cx<R> win0 = gather_row<R>(sd, nx, goff, rglob, rdf, lane);
  cx<R> own[SPW];
#pragma unroll
  for (int m = 0; m < SPW; ++m)
    own[m] = g0 + m < S ? gather_row<R>(sd, nx, goff, rglob, rdf, 32 * (g0 + m) + lane) : zero;
  cx<R> nxt = gather_row<R>(sd, nx, goff, rglob, rdf, 32 * S + lane);
  for (int gi = 0; gi < G; ++gi) {
    const cx<R> nxt2 = gather_row<R>(sd, nx, goff, rglob, rdf, 32 * (gi + S + 1) + lane);
    const cx<R> d = dv[32 * gi + lane];
    cx<R> outv;
    if (!group_steps_mw<R, ST, S, KC, W>(pp, (32 / KC) * gi, b, lane, w, win0, own, nxt, outv, xch, sfail)) {
      fail(sfail);
      return;
    }
    if (w == 0) Yj[32 * gi + lane] = outv * d;
    nxt = nxt2;
  }
  __syncthreads();   // warp 0's z visible to every warp

  // ---------------- backward: L^T x = z on reversed rows ----------------
  auto zrow = [&](int q) -> cx<R> { return q < npad ? Yj[npad - 1 - q] : zero; };
  win0 = zrow(lane);
#pragma unroll
  for (int m = 0; m < SPW; ++m) own[m] = g0 + m < S ? zrow(32 * (g0 + m) + lane) : zero;
  nxt = zrow(32 * S + lane);
  for (int gi = 0; gi < G; ++gi) {
    const cx<R> nxt2 = zrow(32 * (gi + S + 1) + lane);
    cx<R> outv;
    if (!group_steps_mw<R, ST, S, KC, W>(pp, pp.Q + (32 / KC) * gi, b, lane, w, win0, own, nxt, outv, xch,
                                         sfail)) {
      fail(sfail);
      return;
    }
    if (w == 0) {
      const int row = npad - 1 - (32 * gi + lane);
      cx<R> v = zero;
      if (row < sd.n) {
        const int i = sd.ix0 + row % sd.nlx, j = sd.iy0 + row / sd.nlx;
        v = (R)pou_weight(sd, i, j, o) * outv;
      }
      Yj[row] = v;
    }
    nxt = nxt2;
  }
}

// The wide class (SMAX < S <= kApplyWideSlots) on kApplyWideWarps warps per
// subdomain; arguments and band-class skipping as k_apply.
template <typename R, typename ST, int SMAX, int KC, int W>
__global__ void __launch_bounds__(32 * W, 1)
    k_apply_mw(const Geo* __restrict__ geos, const SubDesc* __restrict__ subs, const ST* __restrict__ Lf,
               const ST* __restrict__ Lb, const cx<R>* __restrict__ dinv_all, const c128* __restrict__ rbase,
               long long r_ld, const int* __restrict__ jptr, int rdf, cx<R>* __restrict__ Y, int stage_elems,
               const KState* __restrict__ kst, DevStatus* status, int smin, int smax) {
  extern __shared__ __align__(128) unsigned char sm[];
  const SubDesc sd = subs[blockIdx.x];
  const int S = (sd.b + 32) / 32;
  if (S < smin || S > smax) return;
  if (kst != nullptr && kst[sd.prob].stop) return;
  const int nx = geos[sd.prob].nx, o = geos[sd.prob].ovlp;
  const long long goff = geos[sd.prob].goff;
  const c128* rglob = rbase;
  if (jptr != nullptr)
    rglob = rdf == 2 ? (const c128*)((const c64*)rbase + (long long)(*jptr) * r_ld)
                     : (const c128*)((const dfc*)rbase + (long long)(*jptr) * r_ld);
  constexpr int NST = stages_for<ST>();
  Pipe<ST, KC> pp;
  pp.bar = reinterpret_cast<uint64_t*>(sm);
  pp.stg = reinterpret_cast<ST*>(sm + 128);
  pp.src0 = Lf + sd.l_off;
  pp.src1 = Lb + sd.l_off;
  pp.stage_elems = stage_elems;
  pp.Q = sd.npad / KC;
  pp.bp = sd.bp;
  pp.bytes = (uint32_t)(KC * sd.bp * sizeof(ST));
  pp.limit = g_copy_wait_limit;
  cx<R>* xch = reinterpret_cast<cx<R>*>(sm + 128 + (size_t)NST * stage_elems * sizeof(ST));
  const int nseq = 2 * pp.Q;
  if (threadIdx.x == 0) {
    for (int t = 0; t < NST; ++t) mbar_init(&pp.bar[t], 1);
    mbar_fence_init();
    for (int t = 0; t < NST && t < nseq; ++t) pp.issue(t);
  }
  __syncthreads();
  const cx<R>* dv = dinv_all + sd.v_off;
  cx<R>* Yj = Y + sd.v_off;
#define RP_CASE(S_) \
  case S_:          \
    if constexpr (S_ > SMAX) sweeps_mw<R, ST, S_, KC, W>(sd, pp, nx, goff, o, rglob, rdf, dv, Yj, xch, status); \
    break;
  switch (S) {
    RP_CASE(5) RP_CASE(6) RP_CASE(7) RP_CASE(8)
    RP_CASE(9) RP_CASE(10) RP_CASE(11) RP_CASE(12) RP_CASE(13) RP_CASE(14) RP_CASE(15) RP_CASE(16)
    RP_CASE(17) RP_CASE(18) RP_CASE(19) RP_CASE(20) RP_CASE(21) RP_CASE(22) RP_CASE(23) RP_CASE(24)
    RP_CASE(25) RP_CASE(26) RP_CASE(27) RP_CASE(28) RP_CASE(29)
  }
  static_assert(kApplyWideSlots == 29, "the case list covers S = 1..29");
#undef RP_CASE
}

template <typename R>
__global__ void k_prolong(Geo g, const SubDesc* __restrict__ subs, const cx<R>* __restrict__ Y,
                          c128* __restrict__ z, int out_df, const KState* __restrict__ kst) {
  if (kst != nullptr && kst->stop) return;
  // n < 2^31 (checked at set-up): 32-bit index arithmetic
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= g.nx * g.ny) return;
  const int j = r / g.nx + 1, i = r - (j - 1) * g.nx + 1;
  const int2 cxr = cover_range(boxes_of(g.Mx, g.px), i, g.ovlp), cyr = cover_range(boxes_of(g.My, g.py), j, g.ovlp);
  const int qx0 = cxr.x, qx1 = cxr.y, qy0 = cyr.x, qy1 = cyr.y;
  if constexpr (sizeof(R) == sizeof(float)) {
    if (out_df) {
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      for (int qy = qy0; qy <= qy1; ++qy) {
        for (int qx = qx0; qx <= qx1; ++qx) {
          const SubDesc& sd = subs[qy * g.px + qx];
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
      return;
    }
  }
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
  if (out_df)
    reinterpret_cast<dfc*>(z)[r] = split_c(mk(re, im));
  else
    z[r] = mk(re, im);
}

// SMAX: the narrow kernel's window, 6 slots for complex128, 8 for complex64
// storage. The subdomains are launched in band classes by register slots
// S = (b + 32) / 32: 1..4 and 5..SMAX on the narrow kernel, SMAX+1..29 on
// k_apply_mw; each launch covers all subdomains, skips those of the other
// classes, and sizes its ring for its own class, so that a few wide
// subdomains do not shrink every warp's share of shared memory. The wide
// class copies the most columns per bulk copy (16, 8 or 4) for which two of
// its CTAs share an SM, else the most for which its ring fits. With side
// streams the classes run concurrently (the widest first, on the side
// streams), else one after the other.
template <typename R>
constexpr int smax_for() { return sizeof(R) == 8 ? 6 : 8; }

template <typename R, typename ST, int KC>
cudaError_t launch_apply_k(int bp_max, int smin, int smax, const Geo* geos, const SubDesc* subs, int nsub,
                           const void* Lf, const void* Lb, const void* dinv, const c128* r, long long r_ld,
                           const int* jptr, int rdf, void* Y, const KState* kst, DevStatus* status,
                           cudaStream_t st) {
  const int stage_elems = KC * bp_max;
  const size_t smem = 128 + (size_t)stages_for<ST>() * KC * bp_max * sizeof(ST);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_apply<R, ST, smax_for<R>(), KC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_apply<R, ST, smax_for<R>(), KC><<<nsub, 32, smem, st>>>(geos, subs, (const ST*)Lf, (const ST*)Lb,
                                                            (const cx<R>*)dinv, r, r_ld, jptr, rdf, (cx<R>*)Y,
                                                            stage_elems, kst, status, smin, smax);
  return cudaGetLastError();
}

template <typename R, typename ST, int KC>
cudaError_t launch_apply_mw(int bp_max, int smin, int smax, const Geo* geos, const SubDesc* subs, int nsub,
                            const void* Lf, const void* Lb, const void* dinv, const c128* r, long long r_ld,
                            const int* jptr, int rdf, void* Y, const KState* kst, DevStatus* status,
                            cudaStream_t st) {
  constexpr int W = kApplyWideWarps;
  const int stage_elems = KC * bp_max;
  const size_t smem = 128 + (size_t)stages_for<ST>() * KC * bp_max * sizeof(ST) + (size_t)W * 32 * sizeof(cx<R>);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = k_apply_mw<R, ST, smax_for<R>(), KC, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nsub, 32 * W, smem, st>>>(geos, subs, (const ST*)Lf, (const ST*)Lb, (const cx<R>*)dinv, r, r_ld, jptr, rdf,
                                   (cx<R>*)Y, stage_elems, kst, status, smin, smax);
  return cudaGetLastError();
}

// the wide class: the widest chunk (columns per copy) whose ring lets two
// CTAs share an SM, else the widest whose ring fits
template <typename R, typename ST>
cudaError_t launch_apply_wide(int bp_max, int smin, int smax, const Geo* geos, const SubDesc* subs, int nsub,
                              const void* Lf, const void* Lb, const void* dinv, const c128* r, long long r_ld,
                              const int* jptr, int rdf, void* Y, const KState* kst, DevStatus* status,
                              cudaStream_t st) {
  auto bytes = [&](int kc) {
    return 128 + (size_t)stages_for<ST>() * kc * bp_max * sizeof(ST) + (size_t)kApplyWideWarps * 32 * sizeof(cx<R>);
  };
  auto fits = [&](int kc, int per_sm) { return per_sm * (bytes(kc) + 1024) <= 228 * 1024; };
#define RP_WIDE_ARGS bp_max, smin, smax, geos, subs, nsub, Lf, Lb, dinv, r, r_ld, jptr, rdf, Y, kst, status, st
  for (int per_sm : {2, 1}) {
    if constexpr (sizeof(ST) < 16) {
      if (fits(16, per_sm)) return launch_apply_mw<R, ST, 16>(RP_WIDE_ARGS);
    }
    if (fits(8, per_sm)) return launch_apply_mw<R, ST, 8>(RP_WIDE_ARGS);
    if (fits(4, per_sm)) return launch_apply_mw<R, ST, 4>(RP_WIDE_ARGS);
  }
  return cudaErrorInvalidValue;
#undef RP_WIDE_ARGS
}

template <typename R, typename ST, int KC>
cudaError_t launch_apply_t(int max_b, const Geo* geos, const SubDesc* subs, int nsub, int max_bp, const void* Lf,
                           const void* Lb, const void* dinv, const c128* r, long long r_ld, const int* jptr, int rdf,
                           void* Y, const KState* kst, DevStatus* status, cudaStream_t st,
                           const ApplyStreams* as) {
  constexpr int SMAX = smax_for<R>();
  if (max_b > kMaxBandWide) return cudaErrorInvalidValue;
  const int stop = (max_b + 32) / 32;   // the most slots any subdomain needs
  // classes, widest first: {smin, smax}
  int cls[3][2] = {{SMAX + 1, kApplyWideSlots}, {5, SMAX}, {1, 4}};
  int use[3], nuse = 0;
  for (int c = 0; c < 3; ++c) {
    const int lo = cls[c][0], hi = std::min(cls[c][1], stop);
    if (lo > hi) continue;
    if (as != nullptr && as->slot_mask != 0) {
      const uint32_t bits = ((1u << hi) - 1u) & ~((1u << (lo - 1)) - 1u);
      if ((as->slot_mask & bits) == 0) continue;   // no subdomain in this class
    }
    cls[c][1] = hi;
    use[nuse++] = c;
  }
  auto launch = [&](int c, cudaStream_t s) {
    const int bp = std::min(max_bp, 32 * cls[c][1]);
    if (c == 0)
      return launch_apply_wide<R, ST>(bp, cls[c][0], cls[c][1], geos, subs, nsub, Lf, Lb, dinv, r, r_ld, jptr, rdf, Y,
                                      kst, status, s);
    return launch_apply_k<R, ST, KC>(bp, cls[c][0], cls[c][1], geos, subs, nsub, Lf, Lb, dinv, r, r_ld, jptr,
                                           rdf, Y, kst, status, s);
  };
  cudaError_t e = cudaSuccess;
  const bool concurrent = as != nullptr && as->side[0] != nullptr && as->side[1] != nullptr && nuse > 1;
  if (!concurrent) {
    for (int i = 0; i < nuse && e == cudaSuccess; ++i) e = launch(use[i], st);
    return e;
  }
  // fork: the wider classes on the side streams, the narrowest on st; join
  e = cudaEventRecord(as->fork, st);
  for (int i = 0; i + 1 < nuse && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(as->side[i], as->fork, 0);
    if (e == cudaSuccess) e = launch(use[i], as->side[i]);
    if (e == cudaSuccess) e = cudaEventRecord(as->join[i], as->side[i]);
  }
  if (e == cudaSuccess) e = launch(use[nuse - 1], st);
  for (int i = 0; i + 1 < nuse && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st, as->join[i], 0);
  return e;
}

}  // namespace

cudaError_t set_copy_wait_limit(long long cycles) {
  const long long v = cycles > 0 ? cycles : kWaitLimitCycles;
  return cudaMemcpyToSymbol(g_copy_wait_limit, &v, sizeof(v));
}

uint32_t apply_slot_mask(const SubDesc* subs_host, int nsub) {
  uint32_t m = 0;
  for (int j = 0; j < nsub; ++j) {
    const int S = (subs_host[j].b + 32) / 32;
    if (S >= 1 && S <= 32) m |= 1u << (S - 1);
  }
  return m;
}

bool apply_cols_valid(int prec, int cols) { return cols == 8 || (prec == 1 && (cols == 4 || cols == 16)); }

size_t apply_smem_bytes(int max_bp, int prec, int cols) {
  const size_t es = prec == 0 ? sizeof(c128) : prec == 1 ? sizeof(c64) : sizeof(h2c);
  const int narrow_bp = std::min(max_bp, 32 * (prec == 0 ? 6 : 8));   // the wide launch has its own ring
  return 128 + (size_t)4 * cols * narrow_bp * es;
}

cudaError_t launch_local_solves(int prec, int cols, const Geo* geos, const SubDesc* subs, int nsub, int max_b,
                                int max_bp, const void* Lf, const void* Lb, const void* dinv, const c128* r,
                                long long r_ld, const int* jptr, void* Y, const KState* kst, DevStatus* status,
                                cudaStream_t st, int rkind, const ApplyStreams* as) {
  const int rdf = rkind;
  if (!apply_cols_valid(prec, cols)) return cudaErrorInvalidValue;
#define RP_APPLY_ARGS max_b, geos, subs, nsub, max_bp, Lf, Lb, dinv, r, r_ld, jptr, rdf, Y, kst, status, st, as
  if (prec == 0) return launch_apply_t<double, c128, 8>(RP_APPLY_ARGS);
  if (prec == 2) return launch_apply_t<float, h2c, 8>(RP_APPLY_ARGS);
  if (cols == 4) return launch_apply_t<float, c64, 4>(RP_APPLY_ARGS);
  if (cols == 16) return launch_apply_t<float, c64, 16>(RP_APPLY_ARGS);
  return launch_apply_t<float, c64, 8>(RP_APPLY_ARGS);
}
#undef RP_APPLY_ARGS

cudaError_t launch_prolong(int prec, const Geo& g, const SubDesc* subs, const void* Y, c128* z, const KState* kst,
                           cudaStream_t st, int out_df) {
  long long n = (long long)g.nx * g.ny;
  int threads = 256;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (prec == 0) {
    k_prolong<double><<<blocks, threads, 0, st>>>(g, subs, (const c128*)Y, z, out_df, kst);
  } else {
    k_prolong<float><<<blocks, threads, 0, st>>>(g, subs, (const c64*)Y, z, out_df, kst);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(int prec, int cols, const Geo& g, const Geo* geos, const SubDesc* subs, int nsub, int max_b,
                         int max_bp, const void* Lf, const void* Lb, const void* dinv, const c128* r, void* Y,
                         c128* z, const KState* kst, DevStatus* status, cudaStream_t st, int rkind, int out_df,
                         const ApplyStreams* as) {
  cudaError_t e = launch_local_solves(prec, cols, geos, subs, nsub, max_b, max_bp, Lf, Lb, dinv, r, 0, nullptr, Y,
                                      kst, status, st, rkind, as);
  if (e != cudaSuccess) return e;
  return launch_prolong(prec, g, subs, Y, z, kst, st, out_df);
}

}  // namespace rp
