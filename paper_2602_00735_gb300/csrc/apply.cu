// The RAS-PML apply z = B^-1 r = sum_j R_j^T (chi_j .* A_j^-1 R_j r)
// (Section 2, the equation defining B^-1; restriction as in
// eq. local-ras-discrete, weighted prolongation as in eq. update1).
//
// k_apply: one warp per subdomain runs the restriction R_j r (a gather of the
//   global residual), the forward solve L y = R_j r, z = D^-1 y, the backward
//   solve L^T x = z, and writes chi_j .* x to the subdomain's slice of Y.
//   The factor L_j is streamed from HBM in chunks of 32 columns by the bulk
//   copy (TMA) engine into a two-stage shared-memory ring, first in
//   ascending then in descending chunk order. Both sweeps work in blocks of
//   32 rows: a 32x32 triangular solve carried by warp shuffles, and a
//   band-panel update (rows below the block in the forward sweep, rows
//   below the block as known values in the backward sweep).
// k_prolong: one thread per global unknown sums the (at most four) weighted
//   local values that cover it, in a fixed order (bit-reproducible).
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

constexpr int kRing = 256;   // backward-sweep ring of solved values (>= b + 32)

template <typename R>
__device__ __forceinline__ cx<R> gather_row(const SubDesc& sd, const Geo& g, const c128* __restrict__ r, int row) {
  if (row >= sd.n) return mk((R)0, (R)0);
  int i = sd.ix0 + row % sd.nlx, j = sd.iy0 + row / sd.nlx;
  c128 v = r[(long long)(j - 1) * g.nx + (i - 1)];
  return cvt<R>(v);
}

template <typename R, int NS>
__global__ void __launch_bounds__(32)
    k_apply(Geo g, const SubDesc* __restrict__ subs, const cx<R>* __restrict__ Lall,
            const cx<R>* __restrict__ dinv_all, const c128* __restrict__ rglob, cx<R>* __restrict__ Y,
            int stage_elems, const KState* __restrict__ kst, DevStatus* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  if (kst != nullptr && kst->stop) return;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  cx<R>* xr = reinterpret_cast<cx<R>*>(sm + 128);
  cx<R>* stg = xr + kRing;
  const SubDesc sd = subs[blockIdx.x];
  const int lane = threadIdx.x;
  const int b = sd.b, bp = sd.bp, Q = sd.npad / 32, S = 2 * Q;
  const cx<R>* L = Lall + sd.l_off;
  const cx<R>* dv = dinv_all + sd.v_off;
  cx<R>* Yj = Y + sd.v_off;
  const uint32_t chunk_bytes = 32u * (uint32_t)bp * (uint32_t)sizeof(cx<R>);

  // load sequence s = 0..2Q-1: chunks 0..Q-1, then Q-1..0
  auto issue = [&](int s) {
    const int q = s < Q ? s : S - 1 - s;
    mbar_arrive_expect_tx(&bar[s & 1], chunk_bytes);
    bulk_g2s(stg + (s & 1) * stage_elems, L + (long long)q * 32 * bp, chunk_bytes, &bar[s & 1]);
  };
  auto fail = [&](int s) {
    // a wait gave up: record it, drain the copies still in flight, leave
    if (lane == 0) {
      atomicExch(&status->timeout, 1);
      for (int t = s; t < s + 2 && t < S; ++t) mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1);
    }
    __syncwarp();
  };
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    issue(0);
    if (S > 1) issue(1);
  }
  __syncwarp();

  // ---------------- forward sweep: L y = R_j r, z = D^-1 y ----------------
  cx<R> acc = gather_row<R>(sd, g, rglob, lane);
  cx<R> win[NS];
#pragma unroll
  for (int m = 0; m < NS; ++m) win[m] = gather_row<R>(sd, g, rglob, 32 * (m + 1) + lane);

  for (int s = 0; s < Q; ++s) {
    const int k0 = 32 * s;
    const bool ok = mbar_wait_bounded(&bar[s & 1], (s >> 1) & 1);
    if (!__all_sync(0xffffffffu, ok)) { fail(s); return; }
    const cx<R>* Lc = stg + (s & 1) * stage_elems;
    // 32x32 unit lower triangle of the block
#pragma unroll 4
    for (int i = 0; i < 31; ++i) {
      cx<R> yi = shfl(acc, i);
      if (lane > i && lane - i - 1 < b) acc = fms(acc, Lc[i * bp + (lane - i - 1)], yi);
    }
    const cx<R> y = acc;
    Yj[k0 + lane] = y * dv[k0 + lane];
    // band-panel update of the next b rows
#pragma unroll 2
    for (int i = 0; i < 32; ++i) {
      cx<R> yi = shfl(y, i);
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        const int t = 32 * m + lane + 31 - i;
        if (t < b) win[m] = fms(win[m], Lc[i * bp + t], yi);
      }
    }
    acc = win[0];
#pragma unroll
    for (int m = 0; m + 1 < NS; ++m) win[m] = win[m + 1];
    win[NS - 1] = gather_row<R>(sd, g, rglob, k0 + 32 * (NS + 1) + lane);
    __syncwarp();
    if (lane == 0 && s + 2 < S) {
      fence_proxy_async_smem();
      issue(s + 2);
    }
  }

  // ---------------- backward sweep: L^T x = z ----------------
  for (int t = lane; t < kRing; t += 32) xr[t] = mk((R)0, (R)0);
  __syncwarp();
  const double o = g.ovlp;
  for (int s = Q; s < S; ++s) {
    const int k0 = 32 * (S - 1 - s);
    const bool ok = mbar_wait_bounded(&bar[s & 1], (s >> 1) & 1);
    if (!__all_sync(0xffffffffu, ok)) { fail(s); return; }
    const cx<R>* Lc = stg + (s & 1) * stage_elems;
    cx<R> a0 = Yj[k0 + lane], a1 = mk((R)0, (R)0);
    // known values below the block: rows k0+32+u, coefficient L(k0+32+u, k0+lane)
    const cx<R>* col = Lc + lane * bp + 31 - lane;
    int u = 0;
    for (; u + 1 < b; u += 2) {
      const cx<R> x0 = xr[(k0 + 32 + u) & (kRing - 1)];
      const cx<R> x1 = xr[(k0 + 33 + u) & (kRing - 1)];
      if (31 + u - lane < b) a0 = fms(a0, col[u], x0);
      if (32 + u - lane < b) a1 = fms(a1, col[u + 1], x1);
    }
    if (u < b) {
      const cx<R> x0 = xr[(k0 + 32 + u) & (kRing - 1)];
      if (31 + u - lane < b) a0 = fms(a0, col[u], x0);
    }
    cx<R> acc2 = a0 + a1;
    // 32x32 unit upper triangle (L^T) of the block, bottom-up
#pragma unroll 4
    for (int r = 31; r > 0; --r) {
      cx<R> xv = shfl(acc2, r);
      if (lane < r && r - lane - 1 < b) acc2 = fms(acc2, Lc[lane * bp + (r - lane - 1)], xv);
    }
    xr[(k0 + lane) & (kRing - 1)] = acc2;
    const int row = k0 + lane;
    cx<R> outv = mk((R)0, (R)0);
    if (row < sd.n) {
      const int i = sd.ix0 + row % sd.nlx, j = sd.iy0 + row / sd.nlx;
      const R chi = (R)pou_weight(sd, i, j, (int)o);
      outv = chi * acc2;
    }
    Yj[row] = outv;
    __syncwarp();
    if (lane == 0 && s + 2 < S) {
      fence_proxy_async_smem();
      issue(s + 2);
    }
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

template <typename R, int NS>
cudaError_t launch_apply_t(const Geo& g, const SubDesc* subs, int nsub, int max_bp, const void* L,
                           const void* dinv, const c128* r, void* Y, const KState* kst, DevStatus* status,
                           cudaStream_t st) {
  const int stage_elems = 32 * max_bp;
  const size_t smem = apply_smem_bytes(max_bp, sizeof(R) == 8 ? 0 : 1);
  cudaError_t e = cudaFuncSetAttribute(k_apply<R, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_apply<R, NS><<<nsub, 32, smem, st>>>(g, subs, (const cx<R>*)L, (const cx<R>*)dinv, r, (cx<R>*)Y,
                                         stage_elems, kst, status);
  return cudaGetLastError();
}

}  // namespace

size_t apply_smem_bytes(int max_bp, int prec) {
  size_t es = prec == 0 ? sizeof(c128) : sizeof(c64);
  return 128 + kRing * es + 2 * (size_t)32 * max_bp * es;
}

cudaError_t launch_apply(int prec, const Geo& g, const SubDesc* subs, int nsub, int max_b, int max_bp,
                         const void* L, const void* dinv, const c128* r, void* Y, c128* z, const KState* kst,
                         DevStatus* status, cudaStream_t st) {
  const int ns = (max_b + 31) / 32;
  cudaError_t e;
  if (prec == 0) {
    switch (ns) {
      case 1: e = launch_apply_t<double, 1>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
      case 2: e = launch_apply_t<double, 2>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
      case 3: e = launch_apply_t<double, 3>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
      default: e = launch_apply_t<double, 4>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
    }
  } else {
    switch (ns) {
      case 1: e = launch_apply_t<float, 1>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
      case 2: e = launch_apply_t<float, 2>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
      case 3: e = launch_apply_t<float, 3>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
      default: e = launch_apply_t<float, 4>(g, subs, nsub, max_bp, L, dinv, r, Y, kst, status, st); break;
    }
  }
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
