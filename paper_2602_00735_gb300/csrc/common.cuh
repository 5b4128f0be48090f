// Shared device-side definitions of libraspml: complex arithmetic, the mesh
// geometry, per-subdomain descriptors, the PML stretching and the PTX helpers
// for bulk (TMA) copies with mbarrier completion.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rp {

// ---------------------------------------------------------------------------
// Complex numbers in interleaved (re, im) layout, float or double.
// ---------------------------------------------------------------------------
template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};
using c64 = cx<float>;
using c128 = cx<double>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <typename R>
__host__ __device__ __forceinline__ R abs2(cx<R> a) { return a.re * a.re + a.im * a.im; }
// acc - a*b with fused multiply-adds
template <typename R>
__device__ __forceinline__ cx<R> fms(cx<R> acc, cx<R> a, cx<R> b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
// acc + a*b with fused multiply-adds
template <typename R>
__device__ __forceinline__ cx<R> fmac(cx<R> acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a)*b
template <typename R>
__device__ __forceinline__ cx<R> fcma(cx<R> acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cdiv(cx<R> a, cx<R> b) {
  R d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> crecip(cx<R> b) {
  R d = b.re * b.re + b.im * b.im;
  return {b.re / d, -b.im / d};
}
template <typename To, typename From>
__host__ __device__ __forceinline__ cx<To> cvt(cx<From> a) { return {(To)a.re, (To)a.im}; }

// Storage of factor entries: the arithmetic type itself, or (for complex64
// arithmetic) a pair of IEEE halves, 4 bytes per complex entry.
struct __align__(4) h2c {
  __half re, im;
};
template <typename R>
__device__ __forceinline__ cx<R> ld_entry(const cx<R>& v) { return v; }
__device__ __forceinline__ c64 ld_entry(const h2c& v) { return {__half2float(v.re), __half2float(v.im)}; }
template <typename S, typename R>
__device__ __forceinline__ S st_entry(cx<R> v);
template <>
__device__ __forceinline__ c64 st_entry<c64, float>(c64 v) { return v; }
template <>
__device__ __forceinline__ c128 st_entry<c128, double>(c128 v) { return v; }
template <>
__device__ __forceinline__ h2c st_entry<h2c, float>(c64 v) { return {__float2half_rn(v.re), __float2half_rn(v.im)}; }

template <typename R>
__device__ __forceinline__ cx<R> shfl(cx<R> v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

// ---------------------------------------------------------------------------
// Geometry: Omega = [X0, X0 + Mx h] x [Y0, Y0 + My h]; positions in half-cell
// index units s (x = X0 + s*hh, hh = h/2). Coordinates are formed with
// explicitly rounded multiply and add (no contraction), so that a position
// equals the one a plain two-step evaluation gives.
// ---------------------------------------------------------------------------
struct Geo {
  double X0, Y0, h, hh;
  double x0, x1, y0, y1;    // Omega_int
  double k, g_amp, g_ramp;
  int Mx, My, nx, ny;       // nx = Mx - 1 unknowns per grid row
  int px, py, ovlp, pml;
  int local_bc;
  int g_profile;            // 0 smoothstep ramp, 1 g(d) = g_amp d^3
  long long goff;           // first element of this problem in a concatenated vector
  int sub0;                 // index of its first subdomain (natural order)
  int n;                    // nx * ny
};

enum : int { LO_X = 1, HI_X = 2, LO_Y = 4, HI_Y = 8 };

// One subdomain of the covering (Section 2). Cell ranges are half-open
// [lo, hi) in cells, i.e. node ranges [lo, hi].
struct SubDesc {
  int ext_lo_x, ext_hi_x, ext_lo_y, ext_hi_y;   // Omega_j
  int int_lo_x, int_hi_x, int_lo_y, int_hi_y;   // Omega_j,int
  int box_lo_x, box_hi_x, box_lo_y, box_hi_y;   // non-overlapping box
  int flags;                                    // LO_X|HI_X|LO_Y|HI_Y: interior sides
  int ix0, iy0, nlx, nly;                       // local unknown nodes
  int n;                                        // nlx*nly
  int npad;                                     // n rounded up to 32
  int b;                                        // half-bandwidth nlx + 1
  int bp;                                       // L column stride (b rounded up to even)
  long long l_off;                              // element offset of L_j
  long long v_off;                              // element offset of per-row arrays
  int prob;                                     // problem of a batch (0 for one problem)
  int wslot;                                    // scratch slot of the wide-band factor, -1: none
};

__device__ __forceinline__ double xpos(const Geo& g, double s) {
  return __dadd_rn(g.X0, __dmul_rn(s, g.hh));
}
__device__ __forceinline__ double ypos(const Geo& g, double s) {
  return __dadd_rn(g.Y0, __dmul_rn(s, g.hh));
}

// g'(d), zero for d <= 0. profile 0: amp (3t^2 - 2t^3), t = min(d/ramp, 1);
// profile 1: 3 amp d^2 (g(d) = amp d^3).
__device__ __forceinline__ double gprime(double d, double amp, double ramp, int profile) {
  if (!(d > 0.0)) return 0.0;
  if (profile == 1) return 3.0 * amp * d * d;
  double t = fmin(d / ramp, 1.0);
  return amp * t * t * (3.0 - 2.0 * t);
}

// Global stretching gamma_1(x) = 1 + i g'(distance of x beyond (x0, x1)).
__device__ __forceinline__ c128 gam_global_x(const Geo& g, double s) {
  double x = xpos(g, s);
  double d = fmax(fmax(g.x0 - x, x - g.x1), 0.0);
  return mk(1.0, gprime(d, g.g_amp, g.g_ramp, g.g_profile));
}
__device__ __forceinline__ c128 gam_global_y(const Geo& g, double s) {
  double y = ypos(g, s);
  double d = fmax(fmax(g.y0 - y, y - g.y1), 0.0);
  return mk(1.0, gprime(d, g.g_amp, g.g_ramp, g.g_profile));
}

// Local stretching g_j (Section 2): restarts beyond an interior side of
// Omega_j,int; the global stretching elsewhere.
__device__ __forceinline__ c128 gam_local_x(const Geo& g, const SubDesc& sd, double s) {
  if ((sd.flags & HI_X) && s >= 2.0 * sd.int_hi_x)
    return mk(1.0, gprime((s - 2.0 * sd.int_hi_x) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
  if ((sd.flags & LO_X) && s <= 2.0 * sd.int_lo_x)
    return mk(1.0, gprime((2.0 * sd.int_lo_x - s) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
  return gam_global_x(g, s);
}
__device__ __forceinline__ c128 gam_local_y(const Geo& g, const SubDesc& sd, double s) {
  if ((sd.flags & HI_Y) && s >= 2.0 * sd.int_hi_y)
    return mk(1.0, gprime((s - 2.0 * sd.int_hi_y) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
  if ((sd.flags & LO_Y) && s <= 2.0 * sd.int_lo_y)
    return mk(1.0, gprime((2.0 * sd.int_lo_y - s) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
  return gam_global_y(g, s);
}

// Partition-of-unity weight chi_j at node (i, j) (Section 2, linear ramps
// across the 2*ovlp-cell overlap strips, Section 4).
__device__ __forceinline__ double pou_weight(const SubDesc& sd, int i, int j, int o) {
  double inv = 1.0 / (2.0 * o);
  double wx = 1.0, wy = 1.0;
  if ((sd.flags & LO_X) && i < sd.box_lo_x + o) wx = (double)(i - (sd.box_lo_x - o)) * inv;
  if ((sd.flags & HI_X) && i > sd.box_hi_x - o) wx = (double)((sd.box_hi_x + o) - i) * inv;
  if ((sd.flags & LO_Y) && j < sd.box_lo_y + o) wy = (double)(j - (sd.box_lo_y - o)) * inv;
  if ((sd.flags & HI_Y) && j > sd.box_hi_y - o) wy = (double)((sd.box_hi_y + o) - j) * inv;
  wx = fmin(fmax(wx, 0.0), 1.0);
  wy = fmin(fmax(wy, 0.0), 1.0);
  return wx * wy;
}

// Box index of node i for M cells split into P boxes (first M mod P boxes
// one cell wider); a node on a box edge belongs to the upper box.
__host__ __device__ __forceinline__ int box_of_node(int i, int M, int P) {
  int base = M / P, extra = M % P;
  int split = extra * (base + 1);
  int p = (i < split) ? i / (base + 1) : extra + (i - split) / base;
  return p < P ? p : P - 1;
}
__host__ __device__ __forceinline__ int box_start(int p, int M, int P) {
  int base = M / P, extra = M % P;
  return p * base + (p < extra ? p : extra);
}

// The same box arithmetic with the divisions by P done once (per thread,
// not per query): cover_range gives the boxes whose subdomains hold node i,
// its own box and the neighbours whose overlap of o cells reaches it.
struct Boxes {
  int base, extra, split, P;
};
__device__ __forceinline__ Boxes boxes_of(int M, int P) {
  Boxes b;
  b.base = M / P;
  b.extra = M % P;
  b.split = b.extra * (b.base + 1);
  b.P = P;
  return b;
}
__device__ __forceinline__ int box_first(const Boxes& b, int p) { return p * b.base + (p < b.extra ? p : b.extra); }
__device__ __forceinline__ int2 cover_range(const Boxes& b, int i, int o) {
  int p = (i < b.split) ? i / (b.base + 1) : b.extra + (i - b.split) / b.base;
  p = p < b.P ? p : b.P - 1;
  int q0 = p, q1 = p;
  if (p > 0 && i < box_first(b, p) + o) q0 = p - 1;
  if (p + 1 < b.P && i > box_first(b, p + 1) - o) q1 = p + 1;
  return make_int2(q0, q1);
}

// ---------------------------------------------------------------------------
// Double-float numbers: a double x held as floats hi + lo, split with integer
// operations and one exact float subtraction. hi keeps the sign, exponent and
// top 23 mantissa bits; lo the next 23 bits, so |x - hi - lo| < 2^-46 |x|.
// Magnitudes below 2^-103 keep hi only, below 2^-126 become 0; magnitudes
// beyond the float range become NaN (there is no such value in a normalised
// Krylov basis; a NaN is caught by the residual checks).
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};
// a complex128 value in double-float form (16 bytes, like the double pair)
struct __align__(16) dfc {
  float rh, rl, ih, il;
};

__device__ __forceinline__ dfl split_d(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(u >> 32), lw = (unsigned int)u;
  const unsigned int sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const int ef = e - 896;                              // biased float exponent of hi
  dfl r;
  if (ef <= 0) {
    r.hi = 0.f;
    r.lo = 0.f;
    return r;
  }
  if (ef >= 255) {
    r.hi = __int_as_float(0x7fc00000);
    r.lo = 0.f;
    return r;
  }
  const unsigned int mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  r.hi = __uint_as_float(sign | ((unsigned int)ef << 23) | mh);
  // the 29 remaining bits rem weigh 2^(e-1075); with E = ef - 23,
  // (1 + (rem>>6)/2^23) 2^(E-127) - 2^(E-127) = (rem>>6) 2^(e-1069), exactly
  float lo = 0.f;
  const int E = ef - 23;
  if (E > 0) {
    const unsigned int base = (unsigned int)E << 23;
    lo = __uint_as_float(base | ((lw & 0x1FFFFFFFu) >> 6)) - __uint_as_float(base);
  }
  r.lo = __uint_as_float(__float_as_uint(lo) | sign);
  return r;
}

__device__ __forceinline__ dfc split_c(c128 v) {
  const dfl a = split_d(v.re), b = split_d(v.im);
  dfc r;
  r.rh = a.hi;
  r.rl = a.lo;
  r.ih = b.hi;
  r.il = b.lo;
  return r;
}

// Double-float arithmetic on the FP32 pipe: a*b as p + t with p = fl(a_hi*b_hi)
// and t the remaining terms (exact FMA residual of the leading product)
__device__ __forceinline__ void df_prod(const dfl& a, const dfl& b, float& p, float& t) {
  p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
}

// (hi, lo) += p + t, TwoSum on the leading part
__device__ __forceinline__ void df_acc(float& hi, float& lo, float p, float t) {
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err + t;
}

__device__ __forceinline__ double df_to_d(float hi, float lo) { return (double)hi + (double)lo; }

// Renormalise a double-float pair in place (TwoSum of its two parts):
// afterwards |lo| <= ulp(hi)/2 and hi + lo is unchanged. Sums kept in
// double-float form (df_acc) leave lo as a running total of rounding errors,
// which after cancellation in hi can be as large as hi itself; a product of
// two double-float values (df_prod) drops the lo * lo term, so every pair that
// later enters such a product is renormalised where it is produced.
__device__ __forceinline__ void df_norm(float& hi, float& lo) {
  const float s = hi + lo;
  const float bb = s - hi;
  lo = (hi - (s - bb)) + (lo - bb);
  hi = s;
}

__device__ __forceinline__ dfl dfl_of(float hi, float lo) {
  dfl r;
  r.hi = hi;
  r.lo = lo;
  return r;
}


// Complex Givens rotations (Section 4.1's least-squares update): applies the
// previous rotations i = 0..j-1 (cosine cs[i], sine sn[i]) to column j of the
// Hessenberg matrix, one warp, all lanes calling. The sweep is the recurrence
// carry_0 = col[0]; col'[i] = c_i carry_i + s_i col[i+1], carry_{i+1} =
// -conj(s_i) carry_i + c_i col[i+1]; each lane takes a chunk of consecutive
// i, composes its chunk's affine maps carry -> A carry + B, a warp scan
// composes the chunks (log2(32) + 2 j/32 dependent steps instead of j), and
// each lane replays its chunk from its incoming carry, writing col'[0..j-1].
// Returns carry_j (the new col[j]) in every lane; col[j] is not written.
__device__ __forceinline__ c128 shfl_c128(c128 v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}
__device__ __forceinline__ c128 shfl_up_c128(c128 v, int d) {
  return {__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d)};
}
__device__ __forceinline__ c128 givens_prev_warp(c128* col, const double* cs, const c128* sn, int j, int lane) {
  const int K = (j + 31) / 32;
  const int i0 = min(lane * K, j), i1 = min(i0 + K, j);
  const c128 one = {1.0, 0.0}, zero = {0.0, 0.0};
  c128 A = one, B = zero;
  for (int i = i0; i < i1; ++i) {
    const c128 ai = {-sn[i].re, sn[i].im};   // -conj(s_i)
    const c128 bi = cs[i] * col[i + 1];
    A = ai * A;
    B = ai * B + bi;
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const c128 Ap = shfl_up_c128(A, d), Bp = shfl_up_c128(B, d);
    if (lane >= d) {
      B = A * Bp + B;
      A = A * Ap;
    }
  }
  const c128 c0 = col[0];
  const c128 Ae = shfl_up_c128(A, 1), Be = shfl_up_c128(B, 1);
  c128 carry = lane == 0 ? c0 : Ae * c0 + Be;
  // col[i1] is the next lane's first output: read it before any lane writes
  const c128 bnd = i1 > i0 ? col[i1] : zero;
  __syncwarp();
  for (int i = i0; i < i1; ++i) {
    const c128 b = i + 1 == i1 ? bnd : col[i + 1];
    const c128 t = cs[i] * carry + sn[i] * b;
    carry = cs[i] * b - conj(sn[i]) * carry;
    col[i] = t;
  }
  const int last = j > 0 ? (j - 1) / K : 0;
  const c128 cj = shfl_c128(carry, last);
  __syncwarp();
  return cj;
}

// Device status words shared by the kernels of one handle.
struct DevStatus {
  int pivot_bad_sub;    // first subdomain with a zero / non-finite pivot, else -1
  int timeout;          // a bounded wait gave up
  int nan;              // non-finite value seen
  int pad;
};

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and one-dimensional bulk copies (TMA engine).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` SM clock cycles; returns false on
// time-out.
__device__ __forceinline__ bool mbar_wait_limited(uint64_t* bar, uint32_t parity, long long limit) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
constexpr long long kWaitLimitCycles = 1ll << 31;   // about a second at the GB300 clock
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  return mbar_wait_limited(bar, parity, kWaitLimitCycles);
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace rp
