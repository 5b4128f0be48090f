// Band LDL^T of the subdomains whose window does not fit in shared memory
// (Section 2: the local solves A_j^-1 of B^-1), kMaxBandC64 / kMaxBandC128 <
// b <= kMaxBandWide: A_j = L_j D_j L_j^T without pivoting, blocked.
//
// A thread-block cluster of CL CTAs (1, 2 or 4) of kWideThreads threads per
// subdomain, right-looking, panels of NB pivots. The active rows
// k..k+NB+b-1 of the lower band live in a window in device scratch (one slot
// per wide subdomain, SubDesc::wslot, set aside by the caller), shared by the
// cluster: row r in row slot r mod (NB+b), its entries A(r, r-b..r) at
// positions 0..b (position q holds column r-b+q), in the arithmetic type.
// Panel at k:
//   1. every CTA copies the panel's NB columns, rows k..k+NB+b-1, to its
//      shared memory, column-major (Pn[j][i] = W(k+i, k+j)); cluster barrier;
//   2. every CTA factors them pivot by pivot (the same arithmetic in each, so
//      the copies agree bit for bit): the multipliers of the pivot column,
//      then c_i l_j' subtracted from the later panel columns (two block
//      barriers per pivot), and the pivot column scaled to L;
//   3. CTA 0 writes L(k+i, k+j) to both output copies and 1/d to D^-1 (the
//      layout of factor.cu); the rows k+NB+b..k+2NB+b-1 of A_j enter the
//      slots of the finished rows k..k+NB-1 (zero except their four stored
//      couplings), rows shared out over the cluster;
//   4. the trailing window, rows and columns k+NB..k+NB+b-1, takes the rank-NB
//      update W(r, c) -= sum_j (L(r, k+j) d_j) L(c, k+j) for c <= r: groups
//      of 8 rows go round-robin to the warps of the cluster, a warp takes
//      them in tiles of 8 rows x 64 columns, each thread 4 rows x 4 columns
//      (16 apart) kept in registers over the NB terms, the panel read from
//      shared memory; the window is read and written once per panel;
//      cluster barrier.
// Rows n..npad-1 are identity padding. Zero or non-finite pivots are reported
// like the narrow kernels do (status->pivot_bad_sub). The only waits are the
// block and cluster barriers, which every CTA of a cluster reaches the same
// number of times (one subdomain, one loop).
//
// k_factor_wide_tc (below) is the same factorisation in complex64 with the
// trailing update on the tensor cores, one CTA per subdomain; it also takes
// the bands from kMaxBandTc up to the shared-memory window's limit (factor
// shape kRankTcBlocked of the batched form). Every launch addresses the
// scratch slots with one stride, factor_wide_slot_bytes(prec, max_b), so
// launches that run concurrently never share memory.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace rp {

namespace {

namespace cg = cooperative_groups;

constexpr int kWideThreads = 512;
constexpr int kWideWarps = kWideThreads / 32;
constexpr int kWideOverhang = 64;   // zero rows after the panel: the tile overhang of step 4

// window entry at position q of row r (column r - b + q): the stored
// couplings D, W, S, SW of row r sit at distances 0, 1, b-1 and b below the
// diagonal, every other entry of the band is zero, and padding rows are
// identity; only the coupling an entry needs is read
template <typename R>
__device__ __forceinline__ cx<R> band_entry(const c128* __restrict__ A, const SubDesc& sd, int r, int q, int b) {
  const int t = b - q;   // distance below the diagonal
  cx<R> x = mk((R)0, (R)0);
  if (q > b || r - t < 0 || (t != 0 && t != 1 && t != b - 1 && t != b)) return x;
  if (r >= sd.n) return t == 0 ? mk((R)1, (R)0) : x;
  const c128* a = A + 4 * (sd.v_off + r);
  if (t == 0) x = cvt<R>(a[0]);
  if (t == 1) x = x + cvt<R>(a[1]);
  if (t == b - 1) x = x + cvt<R>(a[2]);
  if (t == b) x = x + cvt<R>(a[3]);
  return x;
}

// rows r0 <= r < r1 (and < npad) of A_j into their window slots; the
// entries are shared out over the `parts` CTAs of the cluster (this one: part)
template <typename R>
__device__ __forceinline__ void fill_rows(cx<R>* Wn, const c128* __restrict__ Aloc, const SubDesc& sd, int r0,
                                          int r1, int RS, int LDW, int part, int parts) {
  const int b = sd.b;
  r1 = min(r1, sd.npad);
  const long long cnt = (long long)max(0, r1 - r0) * LDW;
  for (long long e = (long long)part * blockDim.x + threadIdx.x; e < cnt; e += (long long)parts * blockDim.x) {
    const int r = r0 + (int)(e / LDW), q = (int)(e % LDW);
    Wn[(long long)(r % RS) * LDW + q] = band_entry<R>(Aloc, sd, r, q, b);
  }
}

template <typename R, typename S, int NB>
__global__ void __launch_bounds__(kWideThreads)
    k_factor_wide(const SubDesc* __restrict__ subs, const c128* __restrict__ Aloc, S* __restrict__ Lall,
                  S* __restrict__ Lrev_all, cx<R>* __restrict__ dinv_all, double* __restrict__ pivstats,
                  DevStatus* status, cx<R>* __restrict__ scratch, long long slot_elems, int bmin, int pld) {
  extern __shared__ __align__(16) unsigned char smw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int sub = blockIdx.x / CL, crank = (int)cluster.block_rank();   // the cluster's CTAs are consecutive
  const SubDesc sd = subs[sub];
  if (sd.b <= bmin || sd.wslot < 0) return;   // the whole cluster: the shared-memory kernels take it
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = sd.b, bp = sd.bp, npad = sd.npad;
  const int RS = NB + b, LDW = b + 1;
  cx<R>* Wn = scratch + (long long)sd.wslot * slot_elems;
  cx<R>* Pn = reinterpret_cast<cx<R>*>(smw);   // Pn[j * pld + i], i < NB + b + kWideOverhang
  cx<R>* dsh = Pn + (long long)NB * pld;        // 1/d of the panel's pivots
  cx<R>* dpv = dsh + NB;                        // the pivots d
  cx<R>* lb = dpv + NB;                         // multipliers of the panel rows
  S* L = Lall + sd.l_off;
  S* Lr = Lrev_all + sd.l_off;
  cx<R>* dv = dinv_all + sd.v_off;
  const cx<R> zero = mk((R)0, (R)0);

  fill_rows<R>(Wn, Aloc, sd, 0, RS, RS, LDW, crank, CL);
  for (int e = tid; e < NB * pld; e += kWideThreads) Pn[e] = zero;
  R dmin2 = (R)3e38, dmax2 = (R)0;
  bool bad = false;
  __threadfence();
  cluster.sync();

  for (int k = 0; k < npad; k += NB) {
    const int nbk = min(NB, npad - k);           // pivots in this panel
    const int rows = min(NB + b, npad - k);      // panel rows present
    // 1. panel columns into shared memory (rows of the window read along q)
    for (int e = tid; e < rows * NB; e += kWideThreads) {
      const int i = e / NB, j = e % NB;
      const int q = j - i + b;
      cx<R> x = zero;
      if (j < nbk && q >= 0 && q <= b) x = Wn[(long long)((k + i) % RS) * LDW + q];
      Pn[j * pld + i] = x;
    }
    for (int e = tid; e < NB * (NB + b - rows); e += kWideThreads) {
      const int j = e / (NB + b - rows), i = rows + e % (NB + b - rows);
      Pn[j * pld + i] = zero;
    }
    // every CTA has read the panel rows before any refills their slots (step 3)
    cluster.sync();
    // 2. factor the panel
    for (int j = 0; j < nbk; ++j) {
      const cx<R> d = Pn[j * pld + j];
      const R ad2 = abs2(d);
      const cx<R> di = crecip(d);
      if (tid == 0) {
        dsh[j] = di;
        dpv[j] = d;
        if (!(ad2 > (R)0) || !isfinite(ad2) || !isfinite(di.re) || !isfinite(di.im)) bad = true;
        dmin2 = fmin(dmin2, ad2);
        dmax2 = fmax(dmax2, ad2);
      }
      for (int i = j + 1 + tid; i < NB; i += kWideThreads) lb[i] = Pn[j * pld + i] * di;
      __syncthreads();
      for (int i = j + 1 + tid; i < rows; i += kWideThreads) {
        const cx<R> c = Pn[j * pld + i];
        const int jmax = min(NB - 1, i);
        for (int jj = j + 1; jj <= jmax; ++jj) Pn[jj * pld + i] = fms(Pn[jj * pld + i], c, lb[jj]);
        Pn[j * pld + i] = c * di;
      }
      __syncthreads();
    }
    // 3. outputs (CTA 0) and the rows entering the window
    if (crank == 0) {
      for (int e = tid; e < nbk; e += kWideThreads) dv[k + e] = dsh[e];
      for (int e = tid; e < nbk * bp; e += kWideThreads) {
        const int j = e / bp, t = e % bp;   // L column k+j, entry t: row k+j+1+t
        const int i = j + 1 + t;
        L[(long long)(k + j) * bp + t] = st_entry<S, R>((t < b && i < rows) ? Pn[j * pld + i] : zero);
      }
      for (int e = tid; e < (rows - 1) * NB; e += kWideThreads) {
        const int i = 1 + e / NB, j = e % NB;   // reversed row k+i, entry i-j-1
        if (j < i && j < nbk && i - j <= b)
          Lr[(long long)(npad - 1 - (k + i)) * bp + (i - j - 1)] = st_entry<S, R>(Pn[j * pld + i]);
      }
    }
    fill_rows<R>(Wn, Aloc, sd, k + RS, k + RS + NB, RS, LDW, crank, CL);
    __syncthreads();
    // 4. trailing update of rows and columns k+NB..k+NB+b-1
    if (k + NB < npad) {
      const int nt = rows - NB;                 // trailing rows present
      const int ng = (nt + 7) / 8;              // row groups of 8
      // rows ii0..ii0+3, columns jj0 + 16 v: a half-warp reads 16 consecutive
      // panel entries per load (four consecutive columns per thread read
      // them 32 bytes apart, a 4-way bank conflict)
      const int ur = 4 * (lane >> 4), uc = lane & 15;
      for (int g = crank * kWideWarps + warp; g < ng; g += CL * kWideWarps) {
        const int ii0 = 8 * g + ur;             // this thread's first trailing row
        const int nct = (8 * g + 7) / 64 + 1;   // column tiles reaching the diagonal
        for (int ct = 0; ct < nct; ++ct) {
          const int jj0 = 64 * ct + uc;
          if (jj0 > ii0 + 3) continue;          // this thread's part lies above the diagonal
          cx<R> acc[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int ii = ii0 + u;
            const int r = k + NB + ii;
            cx<R>* wr = Wn + (long long)(r % RS) * LDW + (b - ii);   // position of column k+NB
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int jj = jj0 + 16 * v;
              acc[u][v] = (ii < nt && jj <= ii) ? wr[jj] : zero;
            }
          }
#pragma unroll 2
          for (int j = 0; j < nbk; ++j) {
            const cx<R>* pj = Pn + j * pld + NB;
            const cx<R> d = dpv[j];
            cx<R> a[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              a[u] = pj[ii0 + u] * d;         // L(r, k+j) d_j
              q[u] = pj[jj0 + 16 * u];        // L(c, k+j)
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fms(acc[u][v], a[u], q[v]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int ii = ii0 + u;
            if (ii >= nt) continue;
            const int r = k + NB + ii;
            cx<R>* wr = Wn + (long long)(r % RS) * LDW + (b - ii);
#pragma unroll
            for (int v = 0; v < 4; ++v)
              if (jj0 + 16 * v <= ii) wr[jj0 + 16 * v] = acc[u][v];
          }
        }
      }
    }
    __threadfence();
    cluster.sync();   // the window is complete for the next panel
  }
  if (crank == 0 && tid == 0) {
    pivstats[2 * sub] = sqrt((double)dmin2);
    pivstats[2 * sub + 1] = sqrt((double)dmax2);
    if (bad) atomicCAS(&status->pivot_bad_sub, -1, sub);
  }
}

// ---------------------------------------------------------------------------
// The same factorisation with the trailing update on the tensor cores
// (complex64 arithmetic; the tuner's wide shape 16). One CTA of
// kWideTcThreads threads per subdomain, panels of kWideTcNB pivots; steps 1-3
// as above (one CTA, block barriers). Step 4: the trailing window is cut into
// 128 x 128 tiles (row block I, column block J <= I), and tile (I, J) takes
// D = (L D)_I L_J^T from tcgen05.mma kind::tf32 (M = N = 128, K = 8, two K
// steps): complex products as four real ones (the negate-A bit of the
// instruction descriptor for -Li Li^T), each FP32 operand as a TF32 head
// plus tail with the three products head head, head tail, tail head kept
// (about 2^-21 relative rounding per product), the scheme of k_factor_tc.
// The accumulators (Re and Im, 256 TMEM columns) are read back by sixteen
// warps (32 rows and 32 columns each), transposed through shared memory in
// 8-column slices, and subtracted from the window's entries with c <= r along
// rows. A_I is staged in shared memory once per row block, B_J once per
// tile, both in the no-swizzle K-major core-matrix layout. The one wait, for
// the MMAs' completion, is bounded: on time-out the kernel records it, waits
// once more (bounded), frees its TMEM and returns.
constexpr int kWideTcThreads = 512;
constexpr int kWideTcNB = 16;
constexpr int kWideTcTile = 128;
constexpr uint32_t kWideTcArr = kWideTcTile * kWideTcNB * 4;   // bytes of one operand array
constexpr uint32_t kWideTcCols = 2 * kWideTcTile;              // TMEM columns: Re and Im

template <typename S>
__global__ void __launch_bounds__(kWideTcThreads)
    k_factor_wide_tc(const SubDesc* __restrict__ subs, const c128* __restrict__ Aloc, S* __restrict__ Lall,
                     S* __restrict__ Lrev_all, c64* __restrict__ dinv_all, double* __restrict__ pivstats,
                     DevStatus* status, c64* __restrict__ scratch, long long slot_elems, int bmin, int bmax,
                     int pld) {
  constexpr int NB = kWideTcNB, T = kWideTcTile;
  constexpr uint32_t AB = kWideTcArr;
  extern __shared__ __align__(1024) unsigned char smt[];
  const int sub = blockIdx.x;
  const SubDesc sd = subs[sub];
  if (sd.b <= bmin || sd.b > bmax || sd.wslot < 0) return;   // before any TMEM allocation
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = sd.b, bp = sd.bp, npad = sd.npad;
  const int RS = NB + b, LDW = b + 1;
  c64* Wn = scratch + (long long)sd.wslot * slot_elems;
  unsigned char* Aop = smt;            // (L D)_I: Re head, Re tail, Im head, Im tail
  unsigned char* Bop = smt + 4 * AB;   // L_J, the same four arrays
  c64* Pn = reinterpret_cast<c64*>(smt + 8 * AB);   // Pn[j * pld + i]
  c64* dsh = Pn + (long long)NB * pld;              // 1/d of the panel's pivots
  c64* dpv = dsh + NB;                              // the pivots d
  uint64_t* bar = reinterpret_cast<uint64_t*>(dpv + NB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  S* L = Lall + sd.l_off;
  S* Lr = Lrev_all + sd.l_off;
  c64* dv = dinv_all + sd.v_off;
  const c64 zero = mk(0.f, 0.f);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kWideTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  fill_rows<float>(Wn, Aloc, sd, 0, RS, RS, LDW, 0, 1);
  for (int e = tid; e < NB * pld; e += kWideTcThreads) Pn[e] = zero;
  float dmin2 = 3e38f, dmax2 = 0.f;
  bool bad = false, failed = false;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t lbo = T * 16;   // both operands have T rows
  const uint64_t adesc0 = smem_desc(smem_u32(Aop), lbo, 128), bdesc0 = smem_desc(smem_u32(Bop), lbo, 128);
  const uint32_t id = idesc_tf32(T, T), idn = id | (1u << 13);   // bit 13: negate A
  uint32_t phase = 0;

  for (int k = 0; k < npad && !failed; k += NB) {
    const int rows = min(NB + b, npad - k);   // panel rows present (npad is a multiple of 32)
    // 1. panel columns into shared memory
#pragma unroll 4
    for (int e = tid; e < rows * NB; e += kWideTcThreads) {
      const int i = e / NB, j = e % NB;
      const int q = j - i + b;
      Pn[j * pld + i] = (q >= 0 && q <= b) ? Wn[(long long)((k + i) % RS) * LDW + q] : zero;
    }
    for (int e = tid; e < NB * (NB + b - rows); e += kWideTcThreads) {
      const int j = e / (NB + b - rows), i = rows + e % (NB + b - rows);
      Pn[j * pld + i] = zero;
    }
    __syncthreads();
    // 2. factor the panel: its NB x NB diagonal block on warp 0 (row a in
    //    lane a, multipliers passed by shuffles; L(k+a, k+j) into Pn[j][a]),
    //    then every trailing row forward-substituted against it in registers
    if (warp == 0) {
      const int a = lane & (NB - 1);
      c64 x[NB];
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) x[jj] = jj <= a ? Pn[jj * pld + a] : zero;
      c64 myd = zero, mydi = zero;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const c64 d = shfl(x[j], j);
        const c64 di = crecip(d);
        const c64 l = x[j] * di;
        if (a == j) {
          myd = d;
          mydi = di;
        }
        // entries jj > a of a row are never read back: updated without a predicate
#pragma unroll
        for (int jj = j + 1; jj < NB; ++jj) x[jj] = fms(x[jj], x[j], shfl(l, jj));
        if (lane < NB && a > j) Pn[j * pld + a] = l;
      }
      if (lane < NB) {
        const float ad2 = abs2(myd);
        dsh[a] = mydi;
        dpv[a] = myd;
        if (!(ad2 > 0.f) || !isfinite(ad2) || !isfinite(mydi.re) || !isfinite(mydi.im)) bad = true;
        dmin2 = fminf(dmin2, ad2);
        dmax2 = fmaxf(dmax2, ad2);
      }
    }
    __syncthreads();
    for (int i = NB + tid; i < rows; i += kWideTcThreads) {
      c64 y[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) y[j] = Pn[j * pld + i];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const c64 c = y[j];
#pragma unroll
        for (int jj = j + 1; jj < NB; ++jj) y[jj] = fms(y[jj], c, Pn[j * pld + jj]);
        y[j] = c * dsh[j];
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) Pn[j * pld + i] = y[j];
    }
    __syncthreads();
    // 3. outputs and the rows entering the window
    for (int e = tid; e < NB; e += kWideTcThreads) dv[k + e] = dsh[e];
    for (int e = tid; e < NB * bp; e += kWideTcThreads) {
      const int j = e / bp, t = e % bp;   // L column k+j, entry t: row k+j+1+t
      const int i = j + 1 + t;
      L[(long long)(k + j) * bp + t] = st_entry<S, float>((t < b && i < rows) ? Pn[j * pld + i] : zero);
    }
    for (int e = tid; e < (rows - 1) * NB; e += kWideTcThreads) {
      const int i = 1 + e / NB, j = e % NB;   // reversed row k+i, entry i-j-1
      if (j < i && i - j <= b)
        Lr[(long long)(npad - 1 - (k + i)) * bp + (i - j - 1)] = st_entry<S, float>(Pn[j * pld + i]);
    }
    fill_rows<float>(Wn, Aloc, sd, k + RS, k + RS + NB, RS, LDW, 0, 1);
    __syncthreads();
    // 4. trailing update of rows and columns k+NB..k+NB+b-1, tile by tile
    if (k + NB >= npad) continue;
    const int nt = rows - NB;               // trailing rows present
    const int nbl = (nt + T - 1) / T;       // row blocks
    for (int I = 0; I < nbl && !failed; ++I) {
      for (int J = 0; J <= I && !failed; ++J) {
        // operands: A_I (rows T I.., L d) when a row block starts, B_J (L);
        // four threads per row, each with four of the NB columns (one 16-byte
        // core-matrix row of each split array), a warp on 32 consecutive rows
        for (int e = tid; e < (J == 0 ? 2 : 1) * 4 * T; e += kWideTcThreads) {
          const bool isa = J == 0 && e < 4 * T;
          const int ee = isa ? e : e - (J == 0 ? 4 * T : 0);
          const int qq = (ee >> 5) & 3, rr = (ee & 31) + 32 * (ee >> 7);
          const int t = T * (isa ? I : J) + rr;
          c64 z[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const c64 l = t < nt ? Pn[(4 * qq + j) * pld + NB + t] : zero;
            z[j] = isa ? l * dpv[4 * qq + j] : l;
          }
          tc_put_split_quad(isa ? Aop : Bop, AB, T, rr, qq, z);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
          // (A array, B array, negate): Re += Arh Brh + Arh Brl + Arl Brh - (Aih Bih + Aih Bil + Ail Bih)
          //                             Im += Arh Bih + Arh Bil + Arl Bih + Aih Brh + Aih Brl + Ail Brh
#pragma unroll
          for (int u = 0; u < 6; ++u) {
            const uint32_t ta = (0x322100u >> (4 * u)) & 0xFu;    // 0, 0, 1, 2, 2, 3
            const uint32_t tre = (0x232010u >> (4 * u)) & 0xFu;   // 0, 1, 0, 2, 3, 2
            const uint32_t tim = (0x010232u >> (4 * u)) & 0xFu;   // 2, 3, 2, 0, 1, 0
#pragma unroll
            for (int s = 0; s < NB / 8; ++s) {
              const uint64_t ad = adesc0 + ((ta * AB + 2 * s * lbo) >> 4);
              tc_mma_tf32(tmem, ad, bdesc0 + ((tre * AB + 2 * s * lbo) >> 4), u >= 3 ? idn : id, (u | s) ? 1u : 0u);
              tc_mma_tf32(tmem + (uint32_t)T, ad, bdesc0 + ((tim * AB + 2 * s * lbo) >> 4), id, (u | s) ? 1u : 0u);
            }
          }
          tc_commit(bar);
        }
        // read back: warp w holds tile rows 32 (w mod 4).. (one per lane, as
        // TMEM gives them) and columns 32 (w div 4)..; each 8-column slice
        // (chunk q = 0..3) goes through the warp's 2 KB of the B operand area
        // (free once the MMAs have completed) so that the window's
        // read-modify-write runs along rows, eight lanes per row. The lane's
        // window entries (rows row0 + 4 it + lane/8, column col0 + 8 q) are
        // loaded two chunks ahead, the first two while the MMAs run.
        const int row0 = T * I + 32 * (warp & 3);
        const int col0 = T * J + 32 * (warp >> 2) + (lane & 7);
        int off[8];   // window offset of column 0 in each of the lane's rows
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int t = row0 + 4 * it + (lane >> 3);
          off[it] = ((k + NB + t) % RS) * LDW + (b - t);
        }
        auto load_chunk = [&](int q, c64 (&v)[8]) {
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int t = row0 + 4 * it + (lane >> 3), col = col0 + 8 * q;
            v[it] = (t < nt && col <= t) ? Wn[off[it] + col] : zero;
          }
        };
        c64 w0[8], w1[8], w2[8];
        load_chunk(0, w0);
        load_chunk(1, w1);
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
          // 32 rows x 8 columns; column XOR (row/2) mod 8 keeps both the
          // row-wise writes and the column-wise reads free of bank conflicts
          c64* sc = reinterpret_cast<c64*>(Bop) + warp * 256;
          float re[16], im[16];
          auto slice = [&](int q, const c64 (&v)[8]) {
            const int half = q & 1;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 8; ++u) sc[lane * 8 + (u ^ ((lane >> 1) & 7))] = mk(re[8 * half + u], im[8 * half + u]);
            __syncwarp();
            const int u = lane & 7, col = col0 + 8 * q;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
              const int rho = 4 * it + (lane >> 3), t = row0 + rho;
              if (t < nt && col <= t) {
                const c64 d = sc[rho * 8 + (u ^ ((rho >> 1) & 7))];
                Wn[off[it] + col] = mk(v[it].re - d.re, v[it].im - d.im);
              }
            }
          };
          const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
          tc_ld16x2(ta, ta + (uint32_t)T, re, im);
          load_chunk(2, w2);
          slice(0, w0);
          load_chunk(3, w0);
          slice(1, w1);
          tc_ld16x2(ta + 16u, ta + (uint32_t)T + 16u, re, im);
          slice(2, w2);
          slice(3, w0);
        }
        tc_fence_before();
        __syncthreads();
      }
    }
  }
  if (warp == 0) {
    // pivot statistics of the lanes that held pivots
    float mn = dmin2, mx = dmax2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const bool anybad = __any_sync(0xffffffffu, bad);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWideTcCols)
                 : "memory");
  }
}

// entries between the panel's columns in shared memory: odd, so that the 16
// or 32 columns of one row fall in different banks (the panel copy and the
// reversed-row outputs walk a row across the columns)
inline int wide_pld(int nb, int max_b) { return (nb + max_b + kWideOverhang) | 1; }

// the panel width for bands up to max_b: the largest NB whose panel fits in
// shared memory; 0 when none does
template <typename R>
int wide_nb(int max_b) {
  for (int nb : {32, 16, 8}) {
    const size_t bytes = ((size_t)nb * wide_pld(nb, max_b) + 3 * nb) * sizeof(cx<R>);
    if (bytes <= 220 * 1024) return nb;
  }
  return 0;
}

template <typename R, typename S, int NB>
cudaError_t launch_wide_t(const SubDesc* subs, int nsub, int bmin, int max_b, int cl, const c128* Aloc, void* L,
                          void* Lrev, void* dinv, double* pivstats, DevStatus* status, void* scratch,
                          cudaStream_t st) {
  const int pld = wide_pld(NB, max_b);
  const size_t smem = ((size_t)NB * pld + 3 * NB) * sizeof(cx<R>);
  auto kern = k_factor_wide<R, S, NB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long slot = (long long)(NB + max_b) * (max_b + 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nsub * cl);
  cfg.blockDim = dim3(kWideThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, subs, Aloc, (S*)L, (S*)Lrev, (cx<R>*)dinv, pivstats, status, (cx<R>*)scratch,
                         slot, bmin, pld);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R, typename S>
cudaError_t launch_wide_s(const SubDesc* subs, int nsub, int bmin, int max_b, int cl, const c128* Aloc, void* L,
                          void* Lrev, void* dinv, double* pivstats, DevStatus* status, void* scratch,
                          cudaStream_t st) {
  switch (wide_nb<R>(max_b)) {
    case 32: return launch_wide_t<R, S, 32>(subs, nsub, bmin, max_b, cl, Aloc, L, Lrev, dinv, pivstats, status, scratch, st);
    case 16: return launch_wide_t<R, S, 16>(subs, nsub, bmin, max_b, cl, Aloc, L, Lrev, dinv, pivstats, status, scratch, st);
    case 8: return launch_wide_t<R, S, 8>(subs, nsub, bmin, max_b, cl, Aloc, L, Lrev, dinv, pivstats, status, scratch, st);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
cudaError_t launch_wide_tc(const SubDesc* subs, int nsub, int bmin, int bmax, int max_b, long long slot,
                           const c128* Aloc, void* L, void* Lrev, void* dinv, double* pivstats, DevStatus* status,
                           void* scratch, cudaStream_t st) {
  constexpr int NB = kWideTcNB;
  const int bl = std::min(max_b, bmax);   // the widest band this launch factors
  const int pld = wide_pld(NB, bl);
  const size_t smem = 8 * (size_t)kWideTcArr + ((size_t)NB * pld + 2 * NB) * sizeof(c64) + 16;
  if (smem > 227 * 1024 || (long long)(NB + bl) * (bl + 1) > slot) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_factor_wide_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor_wide_tc<S><<<nsub, kWideTcThreads, smem, st>>>(subs, Aloc, (S*)L, (S*)Lrev, (c64*)dinv, pivstats, status,
                                                          (c64*)scratch, slot, bmin, bmax, pld);
  return cudaGetLastError();
}

}  // namespace

// one slot: the window of the widest CUDA-core panel for max_b, or, below
// the shared-memory window's limit (where only the tensor-core form runs,
// complex64), of its 16-pivot panel
size_t factor_wide_slot_bytes(int prec, int max_b) {
  if (max_b > kMaxBandWide) return 0;
  if (max_b <= max_band(prec)) {
    if (prec == 0 || max_b <= kMaxBandTc) return 0;
    return (size_t)(kWideTcNB + max_b) * (max_b + 1) * sizeof(c64);
  }
  const size_t es = prec == 0 ? sizeof(c128) : sizeof(c64);
  const int nb = prec == 0 ? wide_nb<double>(max_b) : wide_nb<float>(max_b);
  return (size_t)(nb + max_b) * (max_b + 1) * es;
}

int wide_cluster_auto(int nblocked) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  for (int cl : {4, 2})
    if ((long long)nblocked * cl <= sms) return cl;
  return 1;
}

cudaError_t launch_factor_wide(int prec, const SubDesc* subs, int nsub, int max_b, const c128* Aloc, void* L,
                               void* Lrev, void* dinv, double* pivstats, DevStatus* status, void* scratch,
                               cudaStream_t st, int cl, int bmin, int bmax) {
  if (bmin < 0) bmin = max_band(prec);
  if (max_b <= bmin || bmax <= bmin) return cudaSuccess;
  if (max_b > kMaxBandWide || scratch == nullptr) return cudaErrorInvalidValue;
  if (cl == kWideTensorCores) {
    // the tensor-core form: complex64 arithmetic; its panel (16 pivots) is
    // never wider than the CUDA-core form's, so the slot of max_b holds it
    if (bmin < kMaxBandTc) return cudaErrorInvalidValue;
    const long long slot = (long long)(factor_wide_slot_bytes(prec, max_b) / sizeof(c64));
    if (prec == 1)
      return launch_wide_tc<c64>(subs, nsub, bmin, bmax, max_b, slot, Aloc, L, Lrev, dinv, pivstats, status, scratch,
                                 st);
    if (prec == 2)
      return launch_wide_tc<h2c>(subs, nsub, bmin, bmax, max_b, slot, Aloc, L, Lrev, dinv, pivstats, status, scratch,
                                 st);
    return cudaErrorInvalidValue;
  }
  if (!(cl == 1 || cl == 2 || cl == 4) || bmin != max_band(prec) || bmax < max_b) return cudaErrorInvalidValue;
  if (prec == 0)
    return launch_wide_s<double, c128>(subs, nsub, bmin, max_b, cl, Aloc, L, Lrev, dinv, pivstats, status, scratch, st);
  if (prec == 1)
    return launch_wide_s<float, c64>(subs, nsub, bmin, max_b, cl, Aloc, L, Lrev, dinv, pivstats, status, scratch, st);
  return launch_wide_s<float, h2c>(subs, nsub, bmin, max_b, cl, Aloc, L, Lrev, dinv, pivstats, status, scratch, st);
}

}  // namespace rp
