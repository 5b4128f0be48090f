// Assembly kernels (paper Section 1, eq. weak; Section 2, local forms a_j;
// Section 3 (ii), impedance closure).
//
// The bilinear form is eq. weak multiplied by gamma_1 gamma_2 (complex
// symmetric, same solution):
//   a(u,v) = int (g2/g1) u_x v_x + (g1/g2) u_y v_y - k^2 g1 g2 u v
// on P1 triangles (cells split along the (i,j)-(i+1,j+1) diagonal), every
// element integral by the edge-midpoint rule. Rows are built node by node
// from the four cells around the node, so every kernel writes its own
// output with no atomics. Only the diagonal and the couplings to the W, S and
// SW neighbours are produced; symmetry gives the rest.
#include "common.cuh"
#include "kernels.h"

namespace rp {

namespace {

// Element quantities of the two triangles of one cell, from the stretching
// at the cell's edge midpoints. K* are (1/h^2) int_T of the stiffness
// coefficients, mu* = (h^2/6) g1 g2 at a midpoint (the midpoint-rule weight
// of the mass term).
template <typename T>
struct CellTerms {
  cx<T> KxL, KyL, KxU, KyU;
  cx<T> m01, m12, m02, m23, m03;
};

template <typename T, class S>
__device__ CellTerms<T> cell_terms(const Geo& g, const S& st, int ci, int cj) {
  // x positions: 2ci (left edge), 2ci+1 (middle), 2ci+2 (right edge)
  cx<T> xa = st.gx(2.0 * ci + 1.0), xb = st.gx(2.0 * ci + 2.0), xc = st.gx(2.0 * ci);
  cx<T> ya = st.gy(2.0 * cj), yb = st.gy(2.0 * cj + 1.0), yc = st.gy(2.0 * cj + 2.0);
  const T sixth = (T)(1.0 / 6.0);
  const T w = (T)(g.h * g.h * (1.0 / 6.0));
  CellTerms<T> t;
  // lower triangle: m01 = (xa, ya), m12 = (xb, yb), m02 = (xa, yb)
  t.KxL = sixth * (cdiv(ya, xa) + cdiv(yb, xb) + cdiv(yb, xa));
  t.KyL = sixth * (cdiv(xa, ya) + cdiv(xb, yb) + cdiv(xa, yb));
  // upper triangle: m02 = (xa, yb), m23 = (xa, yc), m03 = (xc, yb)
  t.KxU = sixth * (cdiv(yb, xa) + cdiv(yc, xa) + cdiv(yb, xc));
  t.KyU = sixth * (cdiv(xa, yb) + cdiv(xa, yc) + cdiv(xc, yb));
  t.m01 = w * (xa * ya);
  t.m12 = w * (xb * yb);
  t.m02 = w * (xa * yb);
  t.m23 = w * (xa * yc);
  t.m03 = w * (xc * yb);
  return t;
}

// g'(d) in arithmetic type T; for T = double it is gprime() of common.cuh.
template <typename T>
__device__ __forceinline__ T gprime_t(double d, double amp, double ramp, int profile) {
  if (!(d > 0.0)) return (T)0;
  if (profile == 1) return (T)3 * (T)amp * (T)d * (T)d;
  const T t = fmin((T)d / (T)ramp, (T)1);
  return (T)amp * t * t * ((T)3 - (T)2 * t);
}

// Local stretching g_j (Section 2) evaluated in arithmetic type T. Positions
// and branch decisions are in double (half-index units), as for the global one.
template <typename T>
struct LocalStretch {
  Geo g;
  SubDesc sd;
  __device__ cx<T> gam(double s, double x0, double x1, int lo, int hi, int flo, int fhi, double X0) const {
    if ((sd.flags & fhi) && s >= 2.0 * hi) return mk((T)1, gprime_t<T>((s - 2.0 * hi) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
    if ((sd.flags & flo) && s <= 2.0 * lo) return mk((T)1, gprime_t<T>((2.0 * lo - s) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
    const double x = __dadd_rn(X0, __dmul_rn(s, g.hh));
    const double d = fmax(fmax(x0 - x, x - x1), 0.0);
    return mk((T)1, gprime_t<T>(d, g.g_amp, g.g_ramp, g.g_profile));
  }
  __device__ cx<T> gx(double s) const { return gam(s, g.x0, g.x1, sd.int_lo_x, sd.int_hi_x, LO_X, HI_X, g.X0); }
  __device__ cx<T> gy(double s) const { return gam(s, g.y0, g.y1, sd.int_lo_y, sd.int_hi_y, LO_Y, HI_Y, g.Y0); }
  __device__ bool cell_ok(int ci, int cj) const {
    return ci >= sd.ext_lo_x && ci < sd.ext_hi_x && cj >= sd.ext_lo_y && cj < sd.ext_hi_y;
  }
};

template <typename T, class S>
__device__ __forceinline__ CellTerms<T> cell_of(const Geo& g, const S& st, int ci, int cj) {
  return cell_terms<T>(g, st, ci, cj);
}

// Diagonal and lower couplings of node (i, j) from the cells around it.
template <typename T, class S>
__device__ void node_row(const Geo& g, const S& st, int i, int j, cx<T>& D, cx<T>& W, cx<T>& Sx, cx<T>& SW) {
  const T q = (T)(0.25 * g.k * g.k);  // k^2 * (hat product 1/2 * 1/2)
  D = W = Sx = SW = mk((T)0, (T)0);
  if (st.cell_ok(i, j)) {
    CellTerms<T> t = cell_of<T>(g, st, i, j);
    D = D + t.KxL - q * (t.m01 + t.m02) + t.KyU - q * (t.m02 + t.m03);
  }
  if (st.cell_ok(i - 1, j)) {
    CellTerms<T> t = cell_of<T>(g, st, i - 1, j);
    D = D + t.KxL + t.KyL - q * (t.m01 + t.m12);
    W = W - t.KxL - q * t.m01;
  }
  if (st.cell_ok(i, j - 1)) {
    CellTerms<T> t = cell_of<T>(g, st, i, j - 1);
    D = D + t.KxU + t.KyU - q * (t.m23 + t.m03);
    Sx = Sx - t.KyU - q * t.m03;
  }
  if (st.cell_ok(i - 1, j - 1)) {
    CellTerms<T> t = cell_of<T>(g, st, i - 1, j - 1);
    D = D + t.KyL - q * (t.m12 + t.m02) + t.KxU - q * (t.m02 + t.m23);
    W = W - t.KxU - q * t.m23;
    Sx = Sx - t.KyL - q * t.m12;
    SW = SW - q * (t.m02 + t.m02);
  }
}

// Impedance closure (Section 3 (ii)): -i k int gamma_t phi_a phi_b ds on the
// edges of the artificial boundary of Omega_j, 2-point Gauss per edge.
template <typename T>
__device__ void impedance_terms(const Geo& g, const SubDesc& sd, const LocalStretch<T>& st, int i, int j,
                                cx<T>& D, cx<T>& W, cx<T>& Sx) {
  const double q1d = 0.5 - 0.5 / sqrt(3.0), q2d = 0.5 + 0.5 / sqrt(3.0);
  const T q1 = (T)q1d, q2 = (T)q2d, one = (T)1;
  const cx<T> mik = mk((T)0, (T)(-g.k * 0.5 * g.h));  // -i k * (h/2): Gauss weight h/2
  // vertical sides x = const: tangential stretch gamma_2
  bool left = sd.ext_lo_x > 0 && i == sd.ext_lo_x;
  bool right = sd.ext_hi_x < g.Mx && i == sd.ext_hi_x;
  if (left || right) {
    if (j - 1 >= sd.ext_lo_y) {  // edge (i,j-1)-(i,j): node is its upper end
      int jc = j - 1;
      cx<T> a = st.gy(2.0 * (jc + q1d)), b = st.gy(2.0 * (jc + q2d));
      D = D + mik * (q1 * q1 * a + q2 * q2 * b);
      Sx = Sx + mik * ((q1 * (one - q1)) * a + (q2 * (one - q2)) * b);
    }
    if (j < sd.ext_hi_y) {       // edge (i,j)-(i,j+1): node is its lower end
      cx<T> a = st.gy(2.0 * (j + q1d)), b = st.gy(2.0 * (j + q2d));
      D = D + mik * ((one - q1) * (one - q1) * a + (one - q2) * (one - q2) * b);
    }
  }
  // horizontal sides y = const: tangential stretch gamma_1
  bool bottom = sd.ext_lo_y > 0 && j == sd.ext_lo_y;
  bool top = sd.ext_hi_y < g.My && j == sd.ext_hi_y;
  if (bottom || top) {
    if (i - 1 >= sd.ext_lo_x) {
      int ic = i - 1;
      cx<T> a = st.gx(2.0 * (ic + q1d)), b = st.gx(2.0 * (ic + q2d));
      D = D + mik * (q1 * q1 * a + q2 * q2 * b);
      W = W + mik * ((q1 * (one - q1)) * a + (q2 * (one - q2)) * b);
    }
    if (i < sd.ext_hi_x) {
      cx<T> a = st.gx(2.0 * (i + q1d)), b = st.gx(2.0 * (i + q2d));
      D = D + mik * ((one - q1) * (one - q1) * a + (one - q2) * (one - q2) * b);
    }
  }
}

// The global stretching is Cartesian: gamma_1 depends on x alone, gamma_2
// on y alone. tab holds, at every half-index position s, gamma_1(s) and
// 1/gamma_1(s) (first 2Mx+1 pairs), then gamma_2 and 1/gamma_2 (2My+1 pairs).
__global__ void k_stretch_tables(Geo g, c128* __restrict__ tab) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nxs = 2 * g.Mx + 1, nys = 2 * g.My + 1;
  if (e >= nxs + nys) return;
  const c128 v = e < nxs ? gam_global_x(g, (double)e) : gam_global_y(g, (double)(e - nxs));
  tab[2 * e] = v;
  tab[2 * e + 1] = crecip(v);
}

// Global stretching read from the tables; quotients become products with
// the tabulated reciprocals.
struct TabStretch {
  const c128* tx;   // (gamma_1, 1/gamma_1) at half-index s
  const c128* ty;
  __device__ c128 gx(double s) const { return tx[2 * (int)s]; }
  __device__ c128 gy(double s) const { return ty[2 * (int)s]; }
  __device__ c128 rgx(double s) const { return tx[2 * (int)s + 1]; }
  __device__ c128 rgy(double s) const { return ty[2 * (int)s + 1]; }
};

__device__ CellTerms<double> cell_terms_tab(const Geo& g, const TabStretch& st, int ci, int cj) {
  const double sa = 2.0 * ci + 1.0, sb = 2.0 * ci + 2.0, sc = 2.0 * ci;
  const double ta = 2.0 * cj, tb = 2.0 * cj + 1.0, tc = 2.0 * cj + 2.0;
  const c128 xa = st.gx(sa), xb = st.gx(sb), xc = st.gx(sc);
  const c128 ya = st.gy(ta), yb = st.gy(tb), yc = st.gy(tc);
  const c128 ixa = st.rgx(sa), ixb = st.rgx(sb), ixc = st.rgx(sc);
  const c128 iya = st.rgy(ta), iyb = st.rgy(tb), iyc = st.rgy(tc);
  const double sixth = 1.0 / 6.0;
  const double w = g.h * g.h * (1.0 / 6.0);
  CellTerms<double> t;
  t.KxL = sixth * (ya * ixa + yb * ixb + yb * ixa);
  t.KyL = sixth * (xa * iya + xb * iyb + xa * iyb);
  t.KxU = sixth * (yb * ixa + yc * ixa + yb * ixc);
  t.KyU = sixth * (xa * iyb + xa * iyc + xc * iyb);
  t.m01 = w * (xa * ya);
  t.m12 = w * (xb * yb);
  t.m02 = w * (xa * yb);
  t.m23 = w * (xa * yc);
  t.m03 = w * (xc * yb);
  return t;
}

struct TabCells {
  Geo g;
  TabStretch st;
  __device__ bool cell_ok(int ci, int cj) const { return ci >= 0 && ci < g.Mx && cj >= 0 && cj < g.My; }
  __device__ CellTerms<double> cell(int ci, int cj) const { return cell_terms_tab(g, st, ci, cj); }
};

template <typename T>
__device__ __forceinline__ CellTerms<T> cell_of(const Geo& g, const TabCells& st, int ci, int cj) {
  return st.cell(ci, cj);
}

__global__ void k_global_stencil(Geo g, const c128* __restrict__ tab, c128* __restrict__ D, c128* __restrict__ CW,
                                 c128* __restrict__ CS, c128* __restrict__ CSW) {
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = (long long)g.nx * g.ny;
  if (r >= n) return;
  const int jq = (int)r / g.nx, i = (int)r - jq * g.nx + 1, j = jq + 1;   // n < 2^31
  TabCells st{g, TabStretch{tab, tab + 2 * (2 * g.Mx + 1)}};
  c128 d, w, s, sw;
  node_row<double>(g, st, i, j, d, w, s, sw);
  const c128 z = mk(0.0, 0.0);
  D[r] = d;
  CW[r] = (i > 1) ? w : z;            // couplings to outer-boundary nodes drop out
  CS[r] = (j > 1) ? s : z;
  CSW[r] = (i > 1 && j > 1) ? sw : z;
}

// Local stretching read from per-CTA tables: gamma_1 and 1/gamma_1 at the
// half-indices sx0..sx0+nxs-1 of the subdomain's x range, gamma_2 and
// 1/gamma_2 at sy0..sy0+nys-1 (the rows one CTA covers); quotients become
// products with the tabulated reciprocals.
template <typename T>
struct LocalTab {
  const cx<T>* tx;   // (gamma_1, 1/gamma_1) pairs
  const cx<T>* ty;
  int sx0, sy0;
  SubDesc sd;
  __device__ bool cell_ok(int ci, int cj) const {
    return ci >= sd.ext_lo_x && ci < sd.ext_hi_x && cj >= sd.ext_lo_y && cj < sd.ext_hi_y;
  }
};

template <typename T>
__device__ __forceinline__ CellTerms<T> cell_of(const Geo& g, const LocalTab<T>& st, int ci, int cj) {
  const int sa = 2 * ci + 1 - st.sx0, sb = sa + 1, sc = sa - 1;
  const int ta = 2 * cj - st.sy0, tb = ta + 1, tc = ta + 2;
  const cx<T> xa = st.tx[2 * sa], xb = st.tx[2 * sb], xc = st.tx[2 * sc];
  const cx<T> ixa = st.tx[2 * sa + 1], ixb = st.tx[2 * sb + 1], ixc = st.tx[2 * sc + 1];
  const cx<T> ya = st.ty[2 * ta], yb = st.ty[2 * tb], yc = st.ty[2 * tc];
  const cx<T> iya = st.ty[2 * ta + 1], iyb = st.ty[2 * tb + 1], iyc = st.ty[2 * tc + 1];
  const T sixth = (T)(1.0 / 6.0);
  const T w = (T)(g.h * g.h * (1.0 / 6.0));
  CellTerms<T> t;
  t.KxL = sixth * (ya * ixa + yb * ixb + yb * ixa);
  t.KyL = sixth * (xa * iya + xb * iyb + xa * iyb);
  t.KxU = sixth * (yb * ixa + yc * ixa + yb * ixc);
  t.KyU = sixth * (xa * iyb + xa * iyc + xc * iyb);
  t.m01 = w * (xa * ya);
  t.m12 = w * (xb * yb);
  t.m02 = w * (xa * yb);
  t.m23 = w * (xa * yc);
  t.m03 = w * (xc * yb);
  return t;
}

// table sizes of k_local_rows: the x half-indices of a subdomain (2 nlx + 3
// of them, nlx = b - 1) in dynamic shared memory sized per launch by the
// widest band, tab_x(max_b) entries; the y half-indices of the lines of 128
// rows in a fixed array
constexpr int kLrThreads = 128;
constexpr int kLrTabY = 2 * (kLrThreads + 1) + 4;
inline int lr_tab_x(int max_b) { return 2 * max_b + 4; }

// kLrThreads local rows per CTA; blockIdx.y = subdomain. Output
// Aloc[v_off + r] = {D, W, S, SW}; padding rows (r >= n) are identity rows.
// T is the arithmetic type: double for complex128 factors, float for
// complex64 ones (those entries are rounded to complex64 before the
// factorisation anyway). The stretching of the CTA's cells is tabulated
// first (one evaluation per half-index instead of six per cell).
template <typename T>
__global__ void __launch_bounds__(kLrThreads)
    k_local_rows(const Geo* __restrict__ geos, const SubDesc* __restrict__ subs, c128* __restrict__ Aloc,
                 int tab_x) {
  extern __shared__ __align__(16) unsigned char lr_sm[];
  cx<T>* tabx = reinterpret_cast<cx<T>*>(lr_sm);   // 2 tab_x values
  __shared__ cx<T> taby[2 * kLrTabY];
  const SubDesc sd = subs[blockIdx.y];
  const int r0 = blockIdx.x * kLrThreads;
  if (r0 >= sd.npad) return;   // whole CTA
  if (2 * sd.nlx + 3 > tab_x) return;   // never: the launch sizes the table by the widest band
  const int r = r0 + threadIdx.x;
  const Geo g = geos[sd.prob];
  const LocalStretch<T> ls{g, sd};
  // half-indices: x from 2(ix0-1) to 2(ix0+nlx); y over the lines of rows r0..r0+127
  const int sx0 = 2 * (sd.ix0 - 1), nxs = 2 * sd.nlx + 3;
  const int jlo = sd.iy0 + min(r0, sd.n - 1) / sd.nlx, jhi = sd.iy0 + min(r0 + kLrThreads - 1, sd.n - 1) / sd.nlx;
  const int sy0 = 2 * (jlo - 1), nys = 2 * (jhi - jlo) + 5;
  for (int e = threadIdx.x; e < nxs + nys; e += kLrThreads) {
    const cx<T> v = e < nxs ? ls.gx((double)(sx0 + e)) : ls.gy((double)(sy0 + e - nxs));
    cx<T>* d = e < nxs ? tabx + 2 * e : taby + 2 * (e - nxs);
    d[0] = v;
    d[1] = crecip(v);
  }
  __syncthreads();
  if (r >= sd.npad) return;
  c128* out = Aloc + 4 * (sd.v_off + r);
  const c128 z = mk(0.0, 0.0);
  if (r >= sd.n) {
    out[0] = mk(1.0, 0.0);
    out[1] = out[2] = out[3] = z;
    return;
  }
  int i = sd.ix0 + r % sd.nlx, j = sd.iy0 + r / sd.nlx;
  const LocalTab<T> st{tabx, taby, sx0, sy0, sd};
  cx<T> d, w, s, sw;
  node_row<T>(g, st, i, j, d, w, s, sw);
  if (g.local_bc == 0) impedance_terms<T>(g, sd, ls, i, j, d, w, s);
  out[0] = cvt<double>(d);
  out[1] = (i > sd.ix0) ? cvt<double>(w) : z;
  out[2] = (j > sd.iy0) ? cvt<double>(s) : z;
  out[3] = (i > sd.ix0 && j > sd.iy0) ? cvt<double>(sw) : z;
}

// f at half-index (sx, sy): sum of Gaussians, cut to the closed Omega_int.
// Terms with exponent e >= 700 (below 1e-304) are skipped. With a source
// width above 5e-6 the decision is screened in FP32 first (centres cf, the
// first kRhsScreen sources): the FP32 exponent is within 3% of e for
// positions of magnitude below 4, so a term it puts at or above 720 has
// e > 700 and is skipped either way; the others take the FP64 test and
// value, so the result is the same bits as without the screen.
constexpr int kRhsScreen = 64;

__device__ double source_at(const Geo& g, const double* __restrict__ cen, const double* __restrict__ amp, int ns,
                            const float2* cf, double inv_w2, double sx, double sy) {
  double x = xpos(g, sx), y = ypos(g, sy);
  if (!(x >= g.x0 && x <= g.x1 && y >= g.y0 && y <= g.y1)) return 0.0;
  const bool screen = inv_w2 < 4e10 && fabs(x) < 4.0 && fabs(y) < 4.0;
  const float xf = (float)x, yf = (float)y, iwf = (float)inv_w2;
  double f = 0.0;
  for (int s = 0; s < ns; ++s) {
    if (screen && s < kRhsScreen) {
      const float dxf = xf - cf[s].x, dyf = yf - cf[s].y;
      if ((dxf * dxf + dyf * dyf) * iwf >= 720.f) continue;
    }
    const double dx = x - cen[2 * s], dy = y - cen[2 * s + 1];
    const double e = (dx * dx + dy * dy) * inv_w2;
    if (e < 700.0) f += amp[s] * exp(-e);
  }
  return f;
}

// F_i = int f phi_i: each of the node's six edges has its midpoint in two
// triangles with phi_i = 1/2 there, so F_i = (h^2/6) sum_edges f(midpoint).
__global__ void k_rhs(Geo g, const double* __restrict__ cen, const double* __restrict__ amp, int ns, double width,
                      c128* __restrict__ b) {
  __shared__ float2 cf[kRhsScreen];
  for (int s = threadIdx.x; s < min(ns, kRhsScreen); s += blockDim.x)
    cf[s] = make_float2((float)cen[2 * s], (float)cen[2 * s + 1]);
  __syncthreads();
  long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long n = (long long)g.nx * g.ny;
  if (r >= n) return;
  const int jq = (int)r / g.nx, i = (int)r - jq * g.nx + 1, j = jq + 1;   // n < 2^31
  double iw2 = 1.0 / (width * width);
  double si = 2.0 * i, sj = 2.0 * j;
  double f = source_at(g, cen, amp, ns, cf, iw2, si + 1, sj) + source_at(g, cen, amp, ns, cf, iw2, si - 1, sj) +
             source_at(g, cen, amp, ns, cf, iw2, si, sj + 1) + source_at(g, cen, amp, ns, cf, iw2, si, sj - 1) +
             source_at(g, cen, amp, ns, cf, iw2, si + 1, sj + 1) + source_at(g, cen, amp, ns, cf, iw2, si - 1, sj - 1);
  b[r] = mk(f * (g.h * g.h / 6.0), 0.0);
}

// ---------------------------------------------------------------------------
// Form 1: eq. weak as printed (Section 1),
//   a(u,v) = int (D grad u).grad v - (beta.grad u) v - k^2 u v,
//   D = diag(gamma_1^-2, gamma_2^-2), beta_i = gamma_i' / gamma_i^3,
// which is not symmetric, so every row keeps all seven couplings
// {D, W, E, S, N, SW, NE}. Each node's row is summed from the element
// matrices of the (up to six) triangles around it, in a fixed order, every
// integral by the edge-midpoint rule (weight h^2/6 per midpoint).
// ---------------------------------------------------------------------------

// g''(d) in arithmetic type T (zero for d <= 0; continuous).
template <typename T>
__device__ __forceinline__ T gsecond_t(double d, double amp, double ramp, int profile) {
  if (!(d > 0.0)) return (T)0;
  if (profile == 1) return (T)6 * (T)amp * (T)d;
  const T t = fmin((T)d / (T)ramp, (T)1);
  return (T)6 * (T)amp * t * ((T)1 - t) / (T)ramp;
}

// The two triangles of cell (ci, cj): vertex offsets, hat gradients (units
// 1/h), edge-midpoint half-index offsets from (2ci, 2cj) and the hat values
// there (phi[t][m][a]: hat of vertex a at midpoint m).
struct TriTab {
  int vx[2][3], vy[2][3];
  double gx[2][3], gy[2][3];
  int mx[2][3], my[2][3];
  double phi[2][3][3];
};
__constant__ TriTab kTri = {
    {{0, 1, 1}, {0, 1, 0}},
    {{0, 0, 1}, {0, 1, 1}},
    {{-1.0, 1.0, 0.0}, {0.0, 1.0, -1.0}},
    {{0.0, -1.0, 1.0}, {-1.0, 0.0, 1.0}},
    {{1, 2, 1}, {1, 1, 0}},
    {{0, 1, 1}, {1, 2, 1}},
    {{{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}}, {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}}}};

// coupling slot of a neighbour offset: D, W, E, S, N, SW, NE
__device__ __forceinline__ int slot7(int dx, int dy) {
  return dy == 0 ? (dx == 0 ? 0 : dx < 0 ? 1 : 2) : (dx == 0 ? (dy < 0 ? 3 : 4) : (dy < 0 ? 5 : 6));
}

// Global stretching and its derivative: gamma_1' = i (g''(x - x1) - g''(x0 - x)).
struct GlobalStretchW {
  Geo g;
  __device__ c128 gx(double s) const { return gam_global_x(g, s); }
  __device__ c128 gy(double s) const { return gam_global_y(g, s); }
  __device__ c128 dgx(double s) const {
    const double x = xpos(g, s);
    return mk(0.0, gsecond_t<double>(x - g.x1, g.g_amp, g.g_ramp, g.g_profile) -
                       gsecond_t<double>(g.x0 - x, g.g_amp, g.g_ramp, g.g_profile));
  }
  __device__ c128 dgy(double s) const {
    const double y = ypos(g, s);
    return mk(0.0, gsecond_t<double>(y - g.y1, g.g_amp, g.g_ramp, g.g_profile) -
                       gsecond_t<double>(g.y0 - y, g.g_amp, g.g_ramp, g.g_profile));
  }
  __device__ bool cell_ok(int ci, int cj) const { return ci >= 0 && ci < g.Mx && cj >= 0 && cj < g.My; }
};

// Local stretching g_j (Section 2) and its derivative: beyond an interior
// side hi of Omega_j,int gamma' = i g''(x - hi), below an interior side lo
// gamma' = -i g''(lo - x), the global derivative elsewhere.
template <typename T>
struct LocalStretchW {
  LocalStretch<T> ls;
  __device__ cx<T> dg(double s, double c0, double c1, int lo, int hi, int flo, int fhi, double X0) const {
    const Geo& g = ls.g;
    if ((ls.sd.flags & fhi) && s >= 2.0 * hi)
      return mk((T)0, gsecond_t<T>((s - 2.0 * hi) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
    if ((ls.sd.flags & flo) && s <= 2.0 * lo)
      return mk((T)0, -gsecond_t<T>((2.0 * lo - s) * g.hh, g.g_amp, g.g_ramp, g.g_profile));
    const double x = __dadd_rn(X0, __dmul_rn(s, g.hh));
    return mk((T)0, gsecond_t<T>(x - c1, g.g_amp, g.g_ramp, g.g_profile) -
                        gsecond_t<T>(c0 - x, g.g_amp, g.g_ramp, g.g_profile));
  }
  __device__ cx<T> gx(double s) const { return ls.gx(s); }
  __device__ cx<T> gy(double s) const { return ls.gy(s); }
  __device__ cx<T> dgx(double s) const {
    return dg(s, ls.g.x0, ls.g.x1, ls.sd.int_lo_x, ls.sd.int_hi_x, LO_X, HI_X, ls.g.X0);
  }
  __device__ cx<T> dgy(double s) const {
    return dg(s, ls.g.y0, ls.g.y1, ls.sd.int_lo_y, ls.sd.int_hi_y, LO_Y, HI_Y, ls.g.Y0);
  }
  __device__ bool cell_ok(int ci, int cj) const { return ls.cell_ok(ci, cj); }
};

// Row of node (i, j): c[slot7(dx, dy)] += a(phi_(i+dx, j+dy), phi_(i,j)) over
// the cells around the node that S admits.
template <typename T, class S>
__device__ void node_row_w(const Geo& g, const S& st, int i, int j, cx<T> (&c)[7]) {
  const T sixth = (T)(1.0 / 6.0), hs = (T)(g.h / 6.0), k2m = (T)(g.k * g.k * g.h * g.h / 6.0);
#pragma unroll
  for (int q = 0; q < 7; ++q) c[q] = mk((T)0, (T)0);
  for (int q = 0; q < 4; ++q) {
    const int ci = i - 1 + (q & 1), cj = j - 1 + (q >> 1);
    if (!st.cell_ok(ci, cj)) continue;
    for (int t = 0; t < 2; ++t) {
      int a = -1;
      for (int v = 0; v < 3; ++v)
        if (ci + kTri.vx[t][v] == i && cj + kTri.vy[t][v] == j) a = v;
      if (a < 0) continue;
      cx<T> d1 = mk((T)0, (T)0), d2 = d1, b1[3], b2[3];
      for (int m = 0; m < 3; ++m) {
        const double sx = 2.0 * ci + kTri.mx[t][m], sy = 2.0 * cj + kTri.my[t][m];
        const cx<T> r1 = crecip(st.gx(sx)), r2 = crecip(st.gy(sy));
        const cx<T> r1s = r1 * r1, r2s = r2 * r2;
        d1 = d1 + r1s;
        d2 = d2 + r2s;
        b1[m] = st.dgx(sx) * (r1s * r1);
        b2[m] = st.dgy(sy) * (r2s * r2);
      }
      d1 = sixth * d1;
      d2 = sixth * d2;
      const T gax = (T)kTri.gx[t][a], gay = (T)kTri.gy[t][a];
      for (int b = 0; b < 3; ++b) {
        const T gbx = (T)kTri.gx[t][b], gby = (T)kTri.gy[t][b];
        cx<T> adv = mk((T)0, (T)0);
        T mass = (T)0;
        for (int m = 0; m < 3; ++m) {
          const T pa = (T)kTri.phi[t][m][a];
          adv = adv + pa * (gbx * b1[m] + gby * b2[m]);
          mass += pa * (T)kTri.phi[t][m][b];
        }
        const cx<T> v = (gbx * gax) * d1 + (gby * gay) * d2 - hs * adv - mk(k2m * mass, (T)0);
        const int sl = slot7(ci + kTri.vx[t][b] - i, cj + kTri.vy[t][b] - j);
        c[sl] = c[sl] + v;
      }
    }
  }
}

// Impedance closure of form 1 (Section 3 (ii), read in the stretched normal
// coordinate): -i k int gamma_n^-1 phi_a phi_b ds on the edges of the
// artificial boundary of Omega_j; gamma_n is constant along a side, so an
// edge of length h contributes h/3 on the diagonal and h/6 to the coupling.
template <typename T>
__device__ void impedance_terms_w(const Geo& g, const SubDesc& sd, const LocalStretch<T>& st, int i, int j,
                                  cx<T> (&c)[7]) {
  const cx<T> mik = mk((T)0, (T)(-g.k * g.h));
  const T third = (T)(1.0 / 3.0), sixth = (T)(1.0 / 6.0);
  const bool left = sd.ext_lo_x > 0 && i == sd.ext_lo_x;
  const bool right = sd.ext_hi_x < g.Mx && i == sd.ext_hi_x;
  if (left || right) {
    const cx<T> w = mik * crecip(st.gx(2.0 * i));
    if (j - 1 >= sd.ext_lo_y) { c[0] = c[0] + third * w; c[3] = c[3] + sixth * w; }
    if (j < sd.ext_hi_y) { c[0] = c[0] + third * w; c[4] = c[4] + sixth * w; }
  }
  const bool bottom = sd.ext_lo_y > 0 && j == sd.ext_lo_y;
  const bool top = sd.ext_hi_y < g.My && j == sd.ext_hi_y;
  if (bottom || top) {
    const cx<T> w = mik * crecip(st.gy(2.0 * j));
    if (i - 1 >= sd.ext_lo_x) { c[0] = c[0] + third * w; c[1] = c[1] + sixth * w; }
    if (i < sd.ext_hi_x) { c[0] = c[0] + third * w; c[2] = c[2] + sixth * w; }
  }
}

// one thread per global row; couplings to outer-boundary nodes are zero
__global__ void k_global_stencil_w(Geo g, Stencil7W A) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)g.nx * g.ny;
  if (r >= n) return;
  const int jq = (int)r / g.nx, i = (int)r - jq * g.nx + 1, j = jq + 1;   // n < 2^31
  c128 c[7];
  node_row_w<double>(g, GlobalStretchW{g}, i, j, c);
  const c128 z = mk(0.0, 0.0);
  A.D[r] = c[0];
  A.W[r] = i > 1 ? c[1] : z;
  A.E[r] = i < g.nx ? c[2] : z;
  A.S[r] = j > 1 ? c[3] : z;
  A.N[r] = j < g.ny ? c[4] : z;
  A.SW[r] = (i > 1 && j > 1) ? c[5] : z;
  A.NE[r] = (i < g.nx && j < g.ny) ? c[6] : z;
}

// one thread per local row: Aw[7 (v_off + r) + q] = coupling q of row r of
// A_j; couplings to nodes that are not local unknowns are zero; padding
// rows (r >= n) are identity rows
template <typename T>
__global__ void __launch_bounds__(kLrThreads)
    k_local_rows_w(const Geo* __restrict__ geos, const SubDesc* __restrict__ subs, c128* __restrict__ Aw) {
  const SubDesc sd = subs[blockIdx.y];
  const int r = blockIdx.x * kLrThreads + threadIdx.x;
  if (r >= sd.npad) return;
  c128* out = Aw + 7 * (sd.v_off + r);
  const c128 z = mk(0.0, 0.0);
  if (r >= sd.n) {
    out[0] = mk(1.0, 0.0);
    for (int q = 1; q < 7; ++q) out[q] = z;
    return;
  }
  const Geo g = geos[sd.prob];
  const LocalStretch<T> ls{g, sd};
  const int i = sd.ix0 + r % sd.nlx, j = sd.iy0 + r / sd.nlx;
  cx<T> c[7];
  node_row_w<T>(g, LocalStretchW<T>{ls}, i, j, c);
  if (g.local_bc == 0) impedance_terms_w<T>(g, sd, ls, i, j, c);
  const bool w = i > sd.ix0, e = i < sd.ix0 + sd.nlx - 1, s = j > sd.iy0, nn = j < sd.iy0 + sd.nly - 1;
  out[0] = cvt<double>(c[0]);
  out[1] = w ? cvt<double>(c[1]) : z;
  out[2] = e ? cvt<double>(c[2]) : z;
  out[3] = s ? cvt<double>(c[3]) : z;
  out[4] = nn ? cvt<double>(c[4]) : z;
  out[5] = (w && s) ? cvt<double>(c[5]) : z;
  out[6] = (e && nn) ? cvt<double>(c[6]) : z;
}

}  // namespace

size_t stretch_table_elems(const Geo& g) { return (size_t)2 * (2 * g.Mx + 1 + 2 * g.My + 1); }

cudaError_t launch_global_stencil(const Geo& g, c128* tab, c128* D, c128* CW, c128* CS, c128* CSW, cudaStream_t st) {
  const int ne = 2 * g.Mx + 1 + 2 * g.My + 1;
  k_stretch_tables<<<(ne + 255) / 256, 256, 0, st>>>(g, tab);
  long long n = (long long)g.nx * g.ny;
  int threads = 256;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  k_global_stencil<<<blocks, threads, 0, st>>>(g, tab, D, CW, CS, CSW);
  return cudaGetLastError();
}

cudaError_t launch_local_rows(int prec, const Geo* geos, const SubDesc* subs, int nsub, int max_npad, int max_b,
                              c128* Aloc, cudaStream_t st) {
  const int threads = kLrThreads;
  dim3 grid((max_npad + threads - 1) / threads, nsub);
  const int tx = lr_tab_x(max_b);
  cudaError_t e;
  if (prec == 0) {
    const size_t smem = (size_t)2 * tx * sizeof(c128);
    e = cudaFuncSetAttribute(k_local_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_local_rows<double><<<grid, threads, smem, st>>>(geos, subs, Aloc, tx);
  } else {
    const size_t smem = (size_t)2 * tx * sizeof(c64);
    e = cudaFuncSetAttribute(k_local_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_local_rows<float><<<grid, threads, smem, st>>>(geos, subs, Aloc, tx);
  }
  return cudaGetLastError();
}

cudaError_t launch_rhs(const Geo& g, const double* cen, const double* amp, int ns, double width, c128* b,
                       cudaStream_t st) {
  long long n = (long long)g.nx * g.ny;
  int threads = 256;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  k_rhs<<<blocks, threads, 0, st>>>(g, cen, amp, ns, width, b);
  return cudaGetLastError();
}

cudaError_t launch_global_stencil_w(const Geo& g, const Stencil7W& A, cudaStream_t st) {
  const long long n = (long long)g.nx * g.ny;
  const int threads = 256;
  k_global_stencil_w<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(g, A);
  return cudaGetLastError();
}

cudaError_t launch_local_rows_w(int prec, const Geo* geos, const SubDesc* subs, int nsub, int max_npad, c128* Aw,
                                cudaStream_t st) {
  dim3 grid((max_npad + kLrThreads - 1) / kLrThreads, nsub);
  if (prec == 0)
    k_local_rows_w<double><<<grid, kLrThreads, 0, st>>>(geos, subs, Aw);
  else
    k_local_rows_w<float><<<grid, kLrThreads, 0, st>>>(geos, subs, Aw);
  return cudaGetLastError();
}

}  // namespace rp
