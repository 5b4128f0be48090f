// Host side of libraspml: parameter validation, the Cartesian covering of
// Section 2, device memory, and the flexible GMRES driver of Section 4.1.
// Every arithmetic step runs in the kernels of assembly.cu, factor.cu,
// apply.cu and krylov.cu; this file only sizes, launches and synchronises.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "net_internal.h"

using rp::c128;
using rp::c64;
using rp::KState;
using rp::SubDesc;

struct ras_pml_handle {
  ras_pml_params p{};
  cudaStream_t st = nullptr;
  int dev = 0;
  rp::Geo geo{};
  rp::Geo* geo_d = nullptr;      // the same geometry in device memory
  rp::Tune tune{};               // tile shapes of the factor and apply launches
  ras_pml_net* net = nullptr;    // learned coarse-correction stage (optional)
  c128 *lc = nullptr, *lac = nullptr, *lhv = nullptr;   // its correction, A times it, two inner products
  std::vector<SubDesc> subs_h;
  SubDesc* subs_d = nullptr;
  int nsub = 0, max_b = 0, max_bp = 0, max_npad = 0, max_n = 0;
  int nwslot = 0;                // subdomains of the wide-band factor (b > max_band)
  rp::BandSplit split{};         // the widest of the other subdomains (no band order here)
  rp::ApplyStreams as{};         // band classes of the local solves, run concurrently
  long long n = 0, sum_npad = 0, sum_l = 0, sum_n = 0, sum_bn = 0;
  c128 *D = nullptr, *CW = nullptr, *CS = nullptr, *CSW = nullptr;
  c128 *CE = nullptr, *CN = nullptr, *CNE = nullptr;   // form 1: the couplings symmetry no longer gives
  c128 *Ddf = nullptr, *CWdf = nullptr, *CSdf = nullptr, *CSWdf = nullptr;   // the same, split (ortho >= 3)
  void *L = nullptr, *Lrev = nullptr, *dinv = nullptr, *Y = nullptr;
  double* pivstats = nullptr;
  rp::DevStatus* status = nullptr;
  bool factored = false;
  double min_pivot_ratio = 0.0;
  int bad_sub = -1;
  // Krylov workspace (capacity kcap directions)
  int kcap = 0;
  c128 *V = nullptr, *Z = nullptr, *H = nullptr, *sn = nullptr, *gvec = nullptr, *yv = nullptr;
  c128 *partial = nullptr, *hbuf = nullptr;
  c128* wdf = nullptr;   // w split into double-float form (ortho = 3)
  double *cs = nullptr, *hist = nullptr, *scal = nullptr;
  int hist_cap = 0;
  KState* kst = nullptr;
  KState* kst_host = nullptr;   // pinned
  c128 *tmp_b = nullptr, *tmp_x = nullptr, *tmp_r = nullptr;
  int last_iters = 0;
  std::vector<double> hist_host;
  // event timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;     // per-direction events (2 batch slots), solve and batch marks
  ras_pml_timing_t tm{};
};

namespace {

using rp::dalloc;
using rp::dfree;
using rp::ev_ms;

// Reduction of the residual estimate after which a cycle on a complex64
// Krylov basis ends and restarts from the true residual: the basis
// rounding (2^-24) bounds what one cycle's estimate can be trusted to.
constexpr double kC64BasisFloor = 1e-6;

#define RP_ALLOC(ptr, cnt)            \
  do {                                \
    int s_ = dalloc(&(ptr), (cnt));   \
    if (s_ != RASPML_OK) return s_;   \
  } while (0)

// y = A x, or y = bsub - A x: the four-array product of the symmetric form
// (form 0) or the seven-array one of eq. weak as printed (form 1)
// y = A x or bsub - A x in FP64; x in double-float form with xdf (form 0)
cudaError_t spmv_A(const ras_pml_handle* h, const c128* x, const c128* bsub, c128* y, const rp::KState* kst,
                   cudaStream_t st, int bkind = rp::RK_C128, int xdf = 0) {
  if (h->p.form == 1) {
    if (xdf) return cudaErrorInvalidValue;
    return rp::launch_spmv7(h->n, h->geo.nx, rp::Stencil7{h->D, h->CW, h->CE, h->CS, h->CN, h->CSW, h->CNE}, x,
                            bsub, y, kst, st, bkind);
  }
  return rp::launch_spmv(h->n, h->geo.nx, h->D, h->CW, h->CS, h->CSW, x, bsub, y, kst, st, bkind, xdf);
}

int ensure_events(ras_pml_handle* h, int count) {
  while ((int)h->ev.size() < count) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return RASPML_ECUDA;
    h->ev.push_back(e);
  }
  return RASPML_OK;
}

int law_cells(double k, double h) {
  if (!(k > 1.0)) return 1;
  int c = (int)std::floor(0.5 * std::log(k) / k / h + 0.5);
  return c < 1 ? 1 : c;
}

struct Range {
  int box_lo, box_hi, int_lo, int_hi, ext_lo, ext_hi;
  bool lo_in, hi_in;
};

std::vector<Range> ranges(int M, int P, int o, int pml, bool* ok) {
  std::vector<Range> out;
  *ok = true;
  for (int q = 0; q < P; ++q) {
    Range r;
    r.box_lo = rp::box_start(q, M, P);
    r.box_hi = rp::box_start(q + 1, M, P);
    if (q + 1 == P) r.box_hi = M;
    r.lo_in = q > 0;
    r.hi_in = q < P - 1;
    if (r.box_hi - r.box_lo < 2 * o) *ok = false;
    r.int_lo = r.box_lo - (r.lo_in ? o : 0);
    r.int_hi = r.box_hi + (r.hi_in ? o : 0);
    r.ext_lo = std::max(0, r.int_lo - (r.lo_in ? pml : 0));
    r.ext_hi = std::min(M, r.int_hi + (r.hi_in ? pml : 0));
    out.push_back(r);
  }
  return out;
}

int ensure_krylov(ras_pml_handle* h, int m, int maxit) {
  if (h->kcap < m) {
    dfree(h->V); dfree(h->Z); dfree(h->H); dfree(h->sn); dfree(h->gvec); dfree(h->yv);
    dfree(h->partial); dfree(h->hbuf); dfree(h->cs); dfree(h->wdf);
    h->kcap = 0;
    RP_ALLOC(h->wdf, (size_t)h->n);
    RP_ALLOC(h->V, (size_t)(m + 1) * h->n);
    RP_ALLOC(h->Z, (size_t)m * h->n);
    RP_ALLOC(h->H, (size_t)(m + 1) * m);
    RP_ALLOC(h->sn, (size_t)m);
    RP_ALLOC(h->gvec, (size_t)m + 1);
    RP_ALLOC(h->yv, (size_t)m);
    RP_ALLOC(h->hbuf, (size_t)m + 1);
    RP_ALLOC(h->cs, (size_t)m);
    // projections: (m + 1) x dot_blocks(); norms from the update: up to 16 per SM
    RP_ALLOC(h->partial, (size_t)std::max(m + 1, 8) * rp::dot_blocks());
    h->kcap = m;
  }
  if (h->hist_cap < maxit + 1) {
    dfree(h->hist);
    RP_ALLOC(h->hist, (size_t)maxit + 1);
    h->hist_cap = maxit + 1;
  }
  // each one on its own, so a failed allocation leaves none of them half-set
  if (!h->kst) RP_ALLOC(h->kst, 1);
  if (!h->scal) RP_ALLOC(h->scal, 4);
  if (!h->kst_host && cudaMallocHost((void**)&h->kst_host, 2 * sizeof(KState)) != cudaSuccess) {
    h->kst_host = nullptr;
    cudaGetLastError();
    return RASPML_ENOMEM;
  }
  return RASPML_OK;
}

// *out = ||v||_2 (device double), through the deterministic dot kernels
int dev_norm(ras_pml_handle* h, const c128* v, double* out, c128* hslot, const KState* kst, int gate = 0) {
  RP_CUDA(rp::launch_dots(v, h->n, 1, v, h->n, h->partial, kst, gate, h->st));
  RP_CUDA(rp::launch_norm_finish(h->partial, out, hslot, kst, gate, h->st));
  return RASPML_OK;
}

int check_status(ras_pml_handle* h) {
  rp::DevStatus s;
  RP_CUDA(cudaMemcpyAsync(&s, h->status, sizeof(s), cudaMemcpyDeviceToHost, h->st));
  RP_CUDA(cudaStreamSynchronize(h->st));
  if (s.timeout) return RASPML_ETIMEOUT;
  return RASPML_OK;
}

}  // namespace

namespace rp {

int build_problem(const ras_pml_params& p, int prob, Geo& g, std::vector<SubDesc>& subs) {
  if (!(p.k >= 0.0) || !(p.h > 0.0) || !(p.kappa_g >= 0.0) || !(p.x1 > p.x0) || !(p.y1 > p.y0) || p.px < 1 ||
      p.py < 1 || !(p.g_ramp > 0.0) || !(p.g_amp >= 0.0) || (p.local_bc != 0 && p.local_bc != 1) ||
      (p.factor_prec < 0 || p.factor_prec > 2) || (p.ortho < 0 || p.ortho > 4) || (p.g_profile != 0 && p.g_profile != 1) ||
      (p.form != 0 && p.form != 1) || (p.form == 1 && p.ortho > 2))
    return RASPML_EBADARG;
  // form 0: shared-memory window up to max_band, blocked wide kernel beyond
  const int band_limit = p.form == 1 ? max_band_lu(p.factor_prec) : kMaxBandWide;
  const double lx = p.x1 - p.x0 + 2 * p.kappa_g, ly = p.y1 - p.y0 + 2 * p.kappa_g;
  const long long Mx = std::llround(lx / p.h), My = std::llround(ly / p.h);
  if (Mx < 2 || My < 2 || std::fabs(Mx * p.h - lx) > 1e-9 * lx || std::fabs(My * p.h - ly) > 1e-9 * ly ||
      Mx > (1 << 20) || My > (1 << 20))
    return RASPML_EBADARG;
  const int o = p.ovlp_cells < 0 ? law_cells(p.k, p.h) : p.ovlp_cells;
  const int pml = p.pml_cells < 0 ? law_cells(p.k, p.h) : p.pml_cells;
  if (o < 1 || pml < 0 || p.px > Mx || p.py > My) return RASPML_EBADARG;
  bool okx, oky;
  auto rx = ranges((int)Mx, p.px, o, pml, &okx);
  auto ry = ranges((int)My, p.py, o, pml, &oky);
  if (!okx || !oky) return RASPML_EBADARG;

  g = Geo{};
  g.X0 = p.x0 - p.kappa_g;
  g.Y0 = p.y0 - p.kappa_g;
  g.h = p.h;
  g.hh = 0.5 * p.h;
  g.x0 = p.x0; g.x1 = p.x1; g.y0 = p.y0; g.y1 = p.y1;
  g.k = p.k; g.g_amp = p.g_amp; g.g_ramp = p.g_ramp;
  g.Mx = (int)Mx; g.My = (int)My; g.nx = (int)Mx - 1; g.ny = (int)My - 1;
  g.px = p.px; g.py = p.py; g.ovlp = o; g.pml = pml; g.local_bc = p.local_bc;
  g.g_profile = p.g_profile;
  g.n = g.nx * g.ny;
  if ((long long)g.nx * g.ny > (1ll << 31) - 1) return RASPML_EBADARG;

  const bool imp = p.local_bc == 0;
  const size_t first = subs.size();
  for (int qy = 0; qy < p.py; ++qy) {
    for (int qx = 0; qx < p.px; ++qx) {
      const Range& X = rx[qx];
      const Range& Yr = ry[qy];
      SubDesc d{};
      d.ext_lo_x = X.ext_lo; d.ext_hi_x = X.ext_hi; d.ext_lo_y = Yr.ext_lo; d.ext_hi_y = Yr.ext_hi;
      d.int_lo_x = X.int_lo; d.int_hi_x = X.int_hi; d.int_lo_y = Yr.int_lo; d.int_hi_y = Yr.int_hi;
      d.box_lo_x = X.box_lo; d.box_hi_x = X.box_hi; d.box_lo_y = Yr.box_lo; d.box_hi_y = Yr.box_hi;
      d.flags = (X.lo_in ? LO_X : 0) | (X.hi_in ? HI_X : 0) | (Yr.lo_in ? LO_Y : 0) | (Yr.hi_in ? HI_Y : 0);
      int ix0 = imp ? X.ext_lo : X.ext_lo + 1, ix1 = imp ? X.ext_hi : X.ext_hi - 1;
      int iy0 = imp ? Yr.ext_lo : Yr.ext_lo + 1, iy1 = imp ? Yr.ext_hi : Yr.ext_hi - 1;
      ix0 = std::max(ix0, 1); iy0 = std::max(iy0, 1);
      ix1 = std::min(ix1, g.Mx - 1); iy1 = std::min(iy1, g.My - 1);
      if (ix1 < ix0 || iy1 < iy0 || (d.b = ix1 - ix0 + 2) > band_limit) {
        subs.resize(first);
        return RASPML_EBADARG;
      }
      d.ix0 = ix0; d.iy0 = iy0; d.nlx = ix1 - ix0 + 1; d.nly = iy1 - iy0 + 1;
      d.n = d.nlx * d.nly;
      d.npad = (d.n + 31) / 32 * 32;
      d.b = d.nlx + 1;
      d.bp = d.b + (d.b & 1);
      d.prob = prob;
      subs.push_back(d);
    }
  }
  return RASPML_OK;
}

}  // namespace rp

extern "C" {

const char* ras_pml_error_string(int s) {
  switch (s) {
    case RASPML_OK: return "success";
    case RASPML_NOT_CONVERGED: return "not converged within maxit";
    case RASPML_EBADARG: return "invalid argument";
    case RASPML_ENOMEM: return "device out of memory";
    case RASPML_ECUDA: return "CUDA runtime error";
    case RASPML_EPIVOT: return "zero or non-finite pivot in a local factor";
    case RASPML_ENAN: return "NaN or Inf in the residual";
    case RASPML_ETIMEOUT: return "a bounded device-side wait timed out";
    case RASPML_ESTATE: return "call out of order (not factored)";
    default: return "unknown status";
  }
}

void ras_pml_destroy(ras_pml_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->st) cudaStreamSynchronize(h->st);
  dfree(h->Ddf); dfree(h->CWdf); dfree(h->CSdf); dfree(h->CSWdf);
  dfree(h->subs_d); dfree(h->geo_d); dfree(h->D); dfree(h->CW); dfree(h->CS); dfree(h->CSW);
  dfree(h->CE); dfree(h->CN); dfree(h->CNE);
  dfree(h->L); dfree(h->Lrev); dfree(h->dinv); dfree(h->Y); dfree(h->pivstats); dfree(h->status);
  dfree(h->V); dfree(h->Z); dfree(h->H); dfree(h->sn); dfree(h->gvec); dfree(h->yv);
  dfree(h->partial); dfree(h->hbuf); dfree(h->cs); dfree(h->hist); dfree(h->scal); dfree(h->kst);
  dfree(h->wdf);
  dfree(h->tmp_b); dfree(h->tmp_x); dfree(h->tmp_r);
  dfree(h->lc); dfree(h->lac); dfree(h->lhv);
  if (h->kst_host) cudaFreeHost(h->kst_host);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  rp::destroy_apply_streams(&h->as);
  delete h;
}

int ras_pml_setup(const ras_pml_params* pp, void* stream, ras_pml_handle** out) {
  if (!pp || !out) return RASPML_EBADARG;
  *out = nullptr;
  ras_pml_handle* h = new ras_pml_handle();
  const int bs = rp::build_problem(*pp, 0, h->geo, h->subs_h);
  if (bs != RASPML_OK) { delete h; return bs; }
  rp::Geo& g = h->geo;
  h->p = *pp;
  h->p.ovlp_cells = g.ovlp;
  h->p.pml_cells = g.pml;
  h->st = (cudaStream_t)stream;
  cudaGetDevice(&h->dev);
  h->n = (long long)g.nx * g.ny;
  long long l_off = 0, v_off = 0;
  for (SubDesc& d : h->subs_h) {
    d.l_off = l_off;
    d.v_off = v_off;
    l_off += rp::sub_l_entries(d);
    v_off += d.npad;
    h->max_b = std::max(h->max_b, d.b);
    h->max_bp = std::max(h->max_bp, d.bp);
    h->max_npad = std::max(h->max_npad, d.npad);
    h->max_n = std::max(h->max_n, d.n);
    h->sum_n += d.n;
    h->sum_bn += (long long)d.b * d.n;
  }
  h->nsub = (int)h->subs_h.size();
  h->sum_npad = v_off;
  h->sum_l = l_off;
  h->nwslot = rp::assign_wide_slots(h->subs_h, h->p.factor_prec, &h->split.max_b_narrow, &h->split.nblocked);
  if (const int sa = rp::make_apply_streams(&h->as, h->subs_h, h->p.factor_prec); sa != RASPML_OK) {
    ras_pml_destroy(h);
    return sa;
  }

  int s;
#define SETUP_ALLOC(ptr, cnt) \
  if ((s = dalloc(&(ptr), (cnt))) != RASPML_OK) { ras_pml_destroy(h); return s; }
  cudaSetDevice(h->dev);
  SETUP_ALLOC(h->subs_d, (size_t)h->nsub);
  SETUP_ALLOC(h->geo_d, (size_t)1);
  SETUP_ALLOC(h->D, (size_t)h->n);
  SETUP_ALLOC(h->CW, (size_t)h->n);
  SETUP_ALLOC(h->CS, (size_t)h->n);
  SETUP_ALLOC(h->CSW, (size_t)h->n);
  if (h->p.form == 1) {
    SETUP_ALLOC(h->CE, (size_t)h->n);
    SETUP_ALLOC(h->CN, (size_t)h->n);
    SETUP_ALLOC(h->CNE, (size_t)h->n);
  }
  SETUP_ALLOC(h->pivstats, (size_t)2 * h->nsub);
  SETUP_ALLOC(h->status, (size_t)1);
  cudaError_t e = cudaMemcpyAsync(h->subs_d, h->subs_h.data(), sizeof(SubDesc) * h->nsub, cudaMemcpyHostToDevice,
                                  h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->geo_d, &h->geo, sizeof(rp::Geo), cudaMemcpyHostToDevice, h->st);
  rp::DevStatus s0{-1, 0, 0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->status, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->st);
  c128* tab = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&tab, sizeof(c128) * rp::stretch_table_elems(g));
  if (e == cudaSuccess) {
    if (h->p.form == 1)
      e = rp::launch_global_stencil_w(g, rp::Stencil7W{h->D, h->CW, h->CE, h->CS, h->CN, h->CSW, h->CNE}, h->st);
    else
      e = rp::launch_global_stencil(g, tab, h->D, h->CW, h->CS, h->CSW, h->st);
  }
  if (e == cudaSuccess && h->p.ortho >= 3) {
    // the Arnoldi products of the double-float forms use the split coefficients
    c128* src[4] = {h->D, h->CW, h->CS, h->CSW};
    c128** dst[4] = {&h->Ddf, &h->CWdf, &h->CSdf, &h->CSWdf};
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
      e = cudaMalloc((void**)dst[q], sizeof(c128) * h->n);
      if (e == cudaSuccess) e = rp::launch_split(src[q], *dst[q], h->n, nullptr, h->st);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (tab) cudaFree(tab);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "raspml: setup: %s\n", cudaGetErrorString(e));
    ras_pml_destroy(h);
    return RASPML_ECUDA;
  }
  *out = h;
  return RASPML_OK;
}

int ras_pml_num_unknowns(const ras_pml_handle* h, int64_t* n) {
  if (!h || !n) return RASPML_EBADARG;
  *n = h->n;
  return RASPML_OK;
}

int ras_pml_info(const ras_pml_handle* h, ras_pml_info_t* info) {
  if (!h || !info) return RASPML_EBADARG;
  std::memset(info, 0, sizeof(*info));
  const double es = h->p.factor_prec == 0 ? 16.0 : 8.0;          // D^-1 and work vector
  const double esl = h->p.factor_prec == 0 ? 16.0 : h->p.factor_prec == 1 ? 8.0 : 4.0;   // L entries
  info->n = h->n;
  info->Mx = h->geo.Mx;
  info->My = h->geo.My;
  info->num_sub = h->nsub;
  info->ovlp_cells = h->geo.ovlp;
  info->pml_cells = h->geo.pml;
  info->max_local_n = h->max_n;
  info->max_band = h->max_b;
  info->sum_local_n = h->sum_n;
  info->sum_band_n = h->sum_bn;
  info->factor_bytes = (int64_t)(2 * h->sum_l * esl + h->sum_npad * es);   // L, its reversed row copy, D^-1
  // L read in the forward and in the backward sweep, D^-1 once, r read once, z written once
  info->apply_bytes = 2.0 * esl * (double)h->sum_bn + es * (double)h->sum_n + 32.0 * (double)h->n;
  info->min_pivot_ratio = h->min_pivot_ratio;
  info->factored = h->factored ? 1 : 0;
  info->factor_prec = h->p.factor_prec;
  info->bad_subdomain = h->bad_sub;
  info->last_iters = h->last_iters;
  return RASPML_OK;
}

int ras_pml_assemble_rhs(ras_pml_handle* h, const double* centres, const double* amps, int ns, double width,
                         rp_c128* b_dev) {
  if (!h || !b_dev || ns < 0 || (ns > 0 && (!centres || !amps)) || !(width > 0.0)) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  double* buf = nullptr;
  RP_ALLOC(buf, (size_t)3 * (ns > 0 ? ns : 1));
  cudaError_t e = cudaSuccess;
  if (ns > 0) {
    e = cudaMemcpyAsync(buf, centres, sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(buf + 2 * ns, amps, sizeof(double) * ns, cudaMemcpyHostToDevice, h->st);
  }
  if (e == cudaSuccess) e = rp::launch_rhs(h->geo, buf, buf + 2 * ns, ns, width, (c128*)b_dev, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFree(buf);
  if (e != cudaSuccess) return RASPML_ECUDA;
  return RASPML_OK;
}

int ras_pml_factor(ras_pml_handle* h) {
  if (!h) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  const size_t es = h->p.factor_prec == 0 ? sizeof(c128) : sizeof(c64);
  const size_t esl = h->p.factor_prec == 0 ? 16 : h->p.factor_prec == 1 ? 8 : 4;   // L entry storage
  {
    const int sa = rp::alloc_factor_buffers(&h->L, &h->Lrev, &h->dinv, &h->Y, (size_t)h->sum_l * esl,
                                            (size_t)h->sum_npad * es);
    if (sa != RASPML_OK) return sa;
  }
  const bool weak = h->p.form == 1;   // seven couplings per local row, L D U factors
  c128* Aloc = nullptr;
  RP_ALLOC(Aloc, (size_t)(weak ? 7 : 4) * h->sum_npad);
  void* wscratch = nullptr;
  if (const int sw = rp::alloc_wide_scratch(&wscratch, h->nwslot, h->p.factor_prec, h->max_b); sw != RASPML_OK) {
    cudaFree(Aloc);
    return sw;
  }
  if (h->timing) {
    int es_ = ensure_events(h, 2);
    if (es_) return es_;
  }
  rp::DevStatus s0{-1, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(h->status, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess && h->timing) e = cudaEventRecord(h->ev[0], h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->Lrev, 0, (size_t)h->sum_l * esl, h->st);
  if (e == cudaSuccess && weak) {
    e = rp::launch_local_rows_w(h->p.factor_prec, h->geo_d, h->subs_d, h->nsub, h->max_npad, Aloc, h->st);
    if (e == cudaSuccess)
      e = rp::launch_factor_lu(h->p.factor_prec, h->subs_d, h->nsub, h->max_b, Aloc, h->L, h->Lrev, h->dinv,
                               h->pivstats, h->status, h->st);
  }
  if (e == cudaSuccess && !weak)
    e = rp::launch_local_rows(h->p.factor_prec, h->geo_d, h->subs_d, h->nsub, h->max_npad, h->max_b, Aloc, h->st);
  if (e == cudaSuccess && !weak)
    e = rp::launch_factor(h->p.factor_prec, h->tune.factor_threads, h->tune.factor_rank, h->subs_d, h->nsub, h->max_b, Aloc, h->L, h->Lrev, h->dinv,
                          h->pivstats, h->status, h->st, h->split, wscratch, false, h->tune.wide_cluster);
  if (e == cudaSuccess && h->timing) e = cudaEventRecord(h->ev[1], h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess && h->timing) h->tm.factor_ms = ev_ms(h->ev[0], h->ev[1]);
  cudaFree(Aloc);
  if (wscratch) cudaFree(wscratch);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "raspml: factor: %s\n", cudaGetErrorString(e));
    return RASPML_ECUDA;
  }
  rp::DevStatus st;
  std::vector<double> piv(2 * h->nsub);
  RP_CUDA(cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  RP_CUDA(cudaMemcpy(piv.data(), h->pivstats, sizeof(double) * piv.size(), cudaMemcpyDeviceToHost));
  double mr = 1e300;
  for (int j = 0; j < h->nsub; ++j) mr = std::min(mr, piv[2 * j] / piv[2 * j + 1]);
  h->min_pivot_ratio = mr;
  h->bad_sub = st.pivot_bad_sub;
  if (st.timeout) {
    h->factored = false;
    return RASPML_ETIMEOUT;
  }
  if (st.pivot_bad_sub >= 0) {
    h->factored = false;
    return RASPML_EPIVOT;
  }
  h->factored = true;
  return RASPML_OK;
}

int ras_pml_tune(ras_pml_handle* h, ras_pml_tune_t* report) {
  if (!h) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  int s = ras_pml_factor(h);
  if (s != RASPML_OK) return s;
  if (h->p.form == 1) {
    // one factor shape (the L D U kernel); the apply shape stays as set
    if (report) {
      std::memset(report, 0, sizeof(*report));
      report->factor_threads = h->tune.factor_threads;
      report->factor_rank = h->tune.factor_rank;
      report->apply_cols = h->tune.apply_cols;
    }
    return RASPML_OK;
  }
  c128 *Aloc = nullptr, *r = nullptr;
  RP_ALLOC(Aloc, (size_t)4 * h->sum_npad);
  if ((s = dalloc(&r, (size_t)h->n)) != RASPML_OK) { dfree(Aloc); return s; }
  cudaError_t e = cudaMemsetAsync(r, 0, sizeof(c128) * h->n, h->st);
  if (e == cudaSuccess)
    e = rp::launch_local_rows(h->p.factor_prec, h->geo_d, h->subs_d, h->nsub, h->max_npad, h->max_b, Aloc, h->st);
  if (e != cudaSuccess) {
    dfree(Aloc); dfree(r);
    return RASPML_ECUDA;
  }
  void* wscratch = nullptr;
  if ((s = rp::alloc_wide_scratch(&wscratch, h->nwslot, h->p.factor_prec, h->max_b)) != RASPML_OK) {
    dfree(Aloc); dfree(r);
    return s;
  }
  rp::TuneTarget t{h->p.factor_prec, h->geo_d, h->subs_d, h->nsub, h->max_b, h->max_bp, h->max_npad, h->sum_npad,
                   h->sum_l, Aloc, h->L, h->Lrev, h->dinv, h->Y, h->pivstats, h->status, r, h->st, h->split,
                   wscratch};
  s = rp::tune_shapes(t, 3, &h->tune, report);
  cudaStreamSynchronize(h->st);
  dfree(Aloc); dfree(r);
  if (wscratch) cudaFree(wscratch);
  return s;
}

int ras_pml_set_shapes(ras_pml_handle* h, int factor_threads, int factor_rank, int apply_cols, int wide_cluster) {
  if (!h ||
      !rp::factor_shape_valid(h->p.factor_prec, rp::narrow_band(h->p.factor_prec, h->max_b, h->split), factor_threads,
                              factor_rank) ||
      !rp::apply_cols_valid(h->p.factor_prec, apply_cols) ||
      !(wide_cluster == 0 || wide_cluster == 1 || wide_cluster == 2 || wide_cluster == 4 ||
        (wide_cluster == rp::kWideTensorCores && h->p.factor_prec >= 1)))
    return RASPML_EBADARG;
  h->tune.factor_threads = factor_threads;
  h->tune.factor_rank = factor_rank;
  h->tune.apply_cols = apply_cols;
  h->tune.wide_cluster = wide_cluster;
  return RASPML_OK;
}

int ras_pml_attach_net(ras_pml_handle* h, ras_pml_net* net) {
  if (!h) return RASPML_EBADARG;
  if (net && (rp::net_grid(net) > h->geo.nx || rp::net_grid(net) > h->geo.ny)) return RASPML_EBADARG;
  if (net) {   // each buffer on its own: a failed allocation leaves none half-set
    cudaSetDevice(h->dev);
    if (!h->lc) RP_ALLOC(h->lc, (size_t)h->n);
    if (!h->lac) RP_ALLOC(h->lac, (size_t)h->n);
    if (!h->lhv) RP_ALLOC(h->lhv, (size_t)3);
  }
  h->net = net;
  return RASPML_OK;
}

int ras_pml_net_correct(ras_pml_handle* h, ras_pml_net* net, const rp_c128* r, rp_c128* z) {
  if (!h || !net || !r || !z || (const void*)r == (const void*)z) return RASPML_EBADARG;
  if (rp::net_grid(net) > h->geo.nx || rp::net_grid(net) > h->geo.ny) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  const int s = rp::net_correct(net, (const c128*)r, (c128*)z, h->geo.nx, h->geo.ny, nullptr, h->st);
  if (s != RASPML_OK) return s;
  RP_CUDA(cudaStreamSynchronize(h->st));
  return RASPML_OK;
}

int ras_pml_set_copy_wait_limit(long long cycles) {
  RP_CUDA(rp::set_copy_wait_limit(cycles));
  return RASPML_OK;
}

int ras_pml_get_params(const ras_pml_handle* h, ras_pml_params* out) {
  if (!h || !out) return RASPML_EBADARG;
  *out = h->p;
  return RASPML_OK;
}

int ras_pml_apply(ras_pml_handle* h, const rp_c128* r, rp_c128* z) {
  if (!h || !r || !z || (const void*)r == (const void*)z) return RASPML_EBADARG;
  if (!h->factored) return RASPML_ESTATE;
  cudaSetDevice(h->dev);
  RP_CUDA(rp::launch_apply(h->p.factor_prec, h->tune.apply_cols, h->geo, h->geo_d, h->subs_d, h->nsub, h->max_b, h->max_bp, h->L, h->Lrev, h->dinv,
                           (const c128*)r, h->Y, (c128*)z, nullptr, h->status, h->st, rp::RK_C128, 0, &h->as));
  return RASPML_OK;
}

int ras_pml_matvec(ras_pml_handle* h, const rp_c128* x, rp_c128* y) {
  if (!h || !x || !y || (const void*)x == (const void*)y) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  RP_CUDA(spmv_A(h, (const c128*)x, nullptr, (c128*)y,
                          nullptr, h->st));
  return RASPML_OK;
}

int helmholtz_solve(ras_pml_handle* h, const rp_c128* b_dev, rp_c128* x_dev, double rtol, int maxit, int restart,
                    int* iters, double* relres) {
  if (!h || !b_dev || !x_dev || maxit < 1 || restart < 0 || !(rtol >= 0.0)) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  if (!h->factored) {
    int s = ras_pml_factor(h);
    if (s != RASPML_OK) return s;
  }
  int m = (restart > 0 && restart < maxit) ? restart : maxit;
  // The Krylov space (V: m+1 and Z: m vectors of n complex128) must fit in
  // the free device memory; beyond that the cycle is shortened (restarted
  // FGMRES) rather than failing.
  if (m > h->kcap) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const double per_vec = 16.0 * (double)h->n;
      const double held = h->kcap > 0 ? (2.0 * h->kcap + 2.0) * per_vec : 0.0;   // freed on regrowth
      const double avail = (double)free_b + held - 0.05 * (double)total_b - 512.0 * 1048576.0;
      const int fit = (int)std::max(1.0, std::floor(avail / (2.0 * per_vec) - 2.0));
      if (fit < m) m = fit;
    }
  }
  int s = ensure_krylov(h, m, maxit);
  if (s != RASPML_OK) return s;
  const long long n = h->n;
  const c128* b = (const c128*)b_dev;
  c128* x = (c128*)x_dev;
  cudaStream_t st = h->st;
  const int ldh = m + 1;
  const int batch = 4;
  // events: 4 per direction for two batch slots, solve start/end, batch-done x2
  if ((s = ensure_events(h, 8 * batch + 4)) != RASPML_OK) return s;
  double t_apply = 0.0, t_spmv = 0.0, t_ortho = 0.0;
  long long launches = 2, issued = 0, cycles = 0;
  if (h->timing) RP_CUDA(cudaEventRecord(h->ev[8 * batch], h->st));
  KState k0{};
  RP_CUDA(cudaMemcpyAsync(h->kst, &k0, sizeof(k0), cudaMemcpyHostToDevice, st));
  s = dev_norm(h, b, &h->kst->bnorm, nullptr, nullptr);
  if (s) return s;
  RP_CUDA(cudaMemcpyAsync(h->kst_host, h->kst, sizeof(KState), cudaMemcpyDeviceToHost, st));
  RP_CUDA(cudaStreamSynchronize(st));
  const double bnorm = h->kst_host->bnorm;
  h->hist_host.clear();
  if (!(bnorm > 0.0)) {
    RP_CUDA(cudaMemsetAsync(x, 0, sizeof(c128) * n, st));
    RP_CUDA(cudaStreamSynchronize(st));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    h->last_iters = 0;
    return std::isfinite(bnorm) ? RASPML_OK : RASPML_ENAN;
  }
  int status = RASPML_NOT_CONVERGED;
  double rel = NAN;
  const bool dfbasis = h->p.ortho == 3;   // V stored in double-float form
  const bool c64basis = h->p.ortho == 4;  // V stored as complex64, w in its own buffer
  // z_j in double-float form (prolongation to SpMV and to x += Z y), and w
  // with it through the step
  const int zdf = ((c64basis && h->p.factor_prec >= 1) || dfbasis) && h->Ddf ? 1 : 0;
  // The learned stage is gated: once it has corrected kGateDirs directions
  // without removing kGateGain of a residual's squared norm in any of them,
  // the host stops issuing it for the rest of the solve (read one batch late,
  // like the stop flag), so a stage that does not help costs a few
  // directions' worth of its kernels.
  constexpr int kGateDirs = 4;
  constexpr double kGateGain = 0.05;
  bool stage_on = h->net != nullptr;
  long long staged = 0;   // directions the stage corrected (about 20 launches each)
  const int bkind = dfbasis ? rp::RK_DF : c64basis ? rp::RK_C64 : rp::RK_C128;
  c64* V64 = reinterpret_cast<c64*>(h->V);
  for (;;) {
    // new cycle: V0 = b - A x, beta = ||V0||, g = beta e1, V0 /= beta
    c128* V0 = c64basis ? h->wdf : h->V;
    ++cycles;
    RP_CUDA(spmv_A(h, x, b, V0, nullptr, st));
    if ((s = dev_norm(h, V0, &h->kst->hnorm, nullptr, nullptr))) return s;
    RP_CUDA(rp::launch_cycle_init(h->kst, h->gvec, m, rtol, h->hist, st));
    if (dfbasis)
      RP_CUDA(rp::launch_scale_to_df(V0, n, &h->kst->hnorm, h->kst, st));
    else if (c64basis)
      RP_CUDA(rp::launch_scale_to_c64(V0, V64, n, &h->kst->hnorm, h->kst, st));
    else
      RP_CUDA(rp::launch_scale_inv(V0, n, &h->kst->hnorm, h->kst, st));
    // Batches of `batch` directions; batch b+1 is enqueued before the stop flag
    // of batch b is read back, so the device always has queued work while the
    // host waits. Kernels after a stop return at once.
    int slot = 0, pending = -1, pending_nb = 0;
    bool stopped = false;
    auto drain = [&](int sl, int cnt) -> int {
      RP_CUDA(cudaEventSynchronize(h->ev[8 * batch + 2 + sl]));
      if (h->timing) {
        for (int q = 0; q < cnt; ++q) {
          cudaEvent_t* evj = h->ev.data() + sl * 4 * batch + 4 * q;
          t_apply += ev_ms(evj[0], evj[1]);
          t_spmv += ev_ms(evj[1], evj[2]);
          t_ortho += ev_ms(evj[2], evj[3]);
        }
      }
      return RASPML_OK;
    };
    for (int j = 0; j < m && !stopped;) {
      const int nb = std::min(batch, m - j);
      for (int jj = j; jj < j + nb; ++jj) {
        c128* vj = c64basis ? reinterpret_cast<c128*>(V64 + (size_t)jj * n) : h->V + (size_t)jj * n;
        c128* zj = h->Z + (size_t)jj * n;
        c128* w = c64basis ? h->wdf : h->V + (size_t)(jj + 1) * n;
        c128* hcol = h->H + (size_t)jj * ldh;
        cudaEvent_t* evj = h->ev.data() + slot * 4 * batch + 4 * (jj - j);
        ++issued;
        if (h->timing) RP_CUDA(cudaEventRecord(evj[0], st));
        RP_CUDA(rp::launch_apply(h->p.factor_prec, h->tune.apply_cols, h->geo, h->geo_d, h->subs_d, h->nsub, h->max_b, h->max_bp, h->L, h->Lrev,
                                 h->dinv, vj, h->Y, zj, h->kst, h->status, st, bkind, zdf, &h->as));
        if (stage_on) {
          ++staged;
          // learned stage: c = correction of r1 = v_j - A z_j (r1 held in w), then
          // z_j += alpha c with the alpha minimising ||r1 - alpha A c||
          RP_CUDA(spmv_A(h, zj, vj, w, h->kst, st, bkind, zdf));
          RP_CUDA(cudaMemsetAsync(h->lc, 0, sizeof(c128) * n, st));
          const int cs = rp::net_correct(h->net, w, h->lc, h->geo.nx, h->geo.ny, h->kst, st);
          if (cs != RASPML_OK) return cs;
          RP_CUDA(spmv_A(h, h->lc, nullptr, h->lac, h->kst, st));
          RP_CUDA(rp::launch_dots(h->lac, n, 1, w, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, 1, h->lhv, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_dots(h->lac, n, 1, h->lac, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, 1, h->lhv + 1, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_dots(w, n, 1, w, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, 1, h->lhv + 2, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_mr_axpy(zj, h->lc, h->lhv, n, h->kst, st, zdf));
        }
        if (h->timing) RP_CUDA(cudaEventRecord(evj[1], st));
        if (h->Ddf)   // with the complex64 basis or zdf, w stays in double-float form through the step
          RP_CUDA(rp::launch_spmv_df(n, h->geo.nx, h->Ddf, h->CWdf, h->CSdf, h->CSWdf, zj, w, h->kst, st,
                                     (c64basis || zdf) ? 1 : 0, zdf));
        else
          RP_CUDA(spmv_A(h, zj, nullptr, w, h->kst, st));
        if (h->timing) RP_CUDA(cudaEventRecord(evj[2], st));
        if (h->p.ortho == 0) {
          // classical Gram-Schmidt, twice
          RP_CUDA(rp::launch_dots(h->V, n, jj + 1, w, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 1, hcol, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_axpys(h->V, n, jj + 1, hcol, -1.0, w, n, h->kst, 0, st));
          RP_CUDA(rp::launch_dots(h->V, n, jj + 1, w, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 1, h->hbuf, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_axpys(h->V, n, jj + 1, h->hbuf, -1.0, w, n, h->kst, 0, st));
          RP_CUDA(rp::launch_add(hcol, h->hbuf, jj + 1, h->kst, 0, st));
          if ((s = dev_norm(h, w, &h->kst->hnorm, hcol + jj + 1, h->kst))) return s;
        } else if (c64basis) {
          // one pass against the complex64 basis, double-float products and sums;
          // the update also leaves the partial sums of ||w||^2
          int nparts = 0;
          RP_CUDA(rp::launch_dots_c64b(V64, n, jj + 1, w, n, h->partial, h->kst, st, 1));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 1, hcol, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_axpys_c64b(V64, n, jj + 1, hcol, -1.0, w, n, h->kst, st, 1, h->partial, &nparts));
          RP_CUDA(rp::launch_norm_finish(h->partial, &h->kst->hnorm, hcol + jj + 1, h->kst, 0, st, nparts));
        } else if (dfbasis && zdf) {
          // one pass against the double-float basis with w in double-float form
          // (written so by the SpMV); the update also leaves the partial sums
          // of ||w||^2; no FP64 per element
          int nparts = 0;
          RP_CUDA(rp::launch_dots_dfb(h->V, n, jj + 1, w, n, h->partial, h->kst, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 1, hcol, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_axpys_dfb(h->V, n, jj + 1, hcol, -1.0, w, n, h->kst, st, h->partial, &nparts));
          RP_CUDA(rp::launch_norm_finish(h->partial, &h->kst->hnorm, hcol + jj + 1, h->kst, 0, st, nparts));
        } else if (h->p.ortho == 3) {
          // one pass against the double-float basis, products and sums on the FP32 pipe
          RP_CUDA(rp::launch_split(w, h->wdf, n, h->kst, st));
          RP_CUDA(rp::launch_dots_df(h->V, n, jj + 1, h->wdf, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 1, hcol, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_axpys_df(h->V, n, jj + 1, hcol, -1.0, w, n, h->kst, 0, st));
          if ((s = dev_norm(h, w, &h->kst->hnorm, hcol + jj + 1, h->kst))) return s;
        } else {
          // one pass; the projection also returns ||w||^2 (w is column jj+1 of V)
          RP_CUDA(rp::launch_dots(h->V, n, jj + 2, w, n, h->partial, h->kst, 0, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 2, hcol, 0, h->kst, 0, st));
          RP_CUDA(rp::launch_axpys(h->V, n, jj + 1, hcol, -1.0, w, n, h->kst, 0, st));
          if ((s = dev_norm(h, w, &h->kst->hnorm, nullptr, h->kst))) return s;
          RP_CUDA(rp::launch_reorth_decide(h->kst, hcol, jj, h->p.ortho == 1 ? 0.5 : 0.0, st));
          // second pass only where the DGKS test fired
          RP_CUDA(rp::launch_dots(h->V, n, jj + 1, w, n, h->partial, h->kst, 1, st));
          RP_CUDA(rp::launch_dots_finish(h->partial, jj + 1, h->hbuf, 0, h->kst, 1, st));
          RP_CUDA(rp::launch_axpys(h->V, n, jj + 1, h->hbuf, -1.0, w, n, h->kst, 1, st));
          RP_CUDA(rp::launch_add(hcol, h->hbuf, jj + 1, h->kst, 1, st));
          if ((s = dev_norm(h, w, &h->kst->hnorm, hcol + jj + 1, h->kst, 1))) return s;
        }
        RP_CUDA(rp::launch_givens(h->kst, h->H, ldh, h->cs, h->sn, h->gvec, jj, rtol, m, maxit, h->hist, st,
                                  c64basis ? kC64BasisFloor : 0.0));
        if (dfbasis && zdf)
          RP_CUDA(rp::launch_scale_df_to_df(w, w, n, &h->kst->hnorm, h->kst, st));
        else if (dfbasis)
          RP_CUDA(rp::launch_scale_to_df(w, n, &h->kst->hnorm, h->kst, st));
        else if (c64basis)
          RP_CUDA(rp::launch_scale_df_to_c64(w, V64 + (size_t)(jj + 1) * n, n, &h->kst->hnorm, h->kst, st));
        else
          RP_CUDA(rp::launch_scale_inv(w, n, &h->kst->hnorm, h->kst, st));
        if (h->timing) RP_CUDA(cudaEventRecord(evj[3], st));
      }
      RP_CUDA(cudaMemcpyAsync(h->kst_host + slot, h->kst, sizeof(KState), cudaMemcpyDeviceToHost, st));
      RP_CUDA(cudaEventRecord(h->ev[8 * batch + 2 + slot], st));
      if (pending >= 0) {
        if ((s = drain(pending, pending_nb))) return s;
        if (h->kst_host[pending].stop) stopped = true;
        if (stage_on && h->kst_host[pending].ldirs >= kGateDirs && h->kst_host[pending].lgain < kGateGain)
          stage_on = false;
      }
      pending = slot;
      pending_nb = nb;
      slot ^= 1;
      j += nb;
    }
    if ((s = drain(pending, pending_nb))) return s;
    *h->kst_host = h->kst_host[pending];
    const KState ks = *h->kst_host;
    // x += Z y with y = H^-1 g
    if (ks.jdone > 0) {
      RP_CUDA(rp::launch_backsolve(h->H, ldh, h->gvec, h->kst, h->yv, st));
      if (zdf)
        RP_CUDA(rp::launch_axpys_df(h->Z, n, ks.jdone, h->yv, 1.0, x, n, nullptr, 0, st));
      else
        RP_CUDA(rp::launch_axpys(h->Z, n, ks.jdone, h->yv, 1.0, x, n, nullptr, 0, st));
    }
    // true residual
    RP_CUDA(spmv_A(h, x, b, h->V, nullptr, st));
    if ((s = dev_norm(h, h->V, h->scal, nullptr, nullptr))) return s;
    double rn = 0.0;
    RP_CUDA(cudaMemcpyAsync(&rn, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    RP_CUDA(cudaStreamSynchronize(st));
    rel = rn / bnorm;
    if (!std::isfinite(rel) || ks.nan) { status = RASPML_ENAN; break; }
    if (rtol > 0.0 && rel <= rtol) { status = RASPML_OK; break; }
    if (ks.total >= maxit) { status = RASPML_NOT_CONVERGED; break; }
    if (ks.breakdown && ks.jdone == 0) { status = RASPML_NOT_CONVERGED; break; }
  }
  const int total = h->kst_host->total;
  h->last_iters = total;
  // launches: ||b|| (2); per cycle: residual, norm (2), init, scale, backsolve,
  // update, true residual, norm (2) = 10; per issued direction: 13 (CGS twice)
  // or 17 (one pass, test, gated second pass)
  launches += 10 * cycles + (h->p.ortho == 0 ? 13 : h->p.ortho == 3 ? (zdf ? 11 : 12) : h->p.ortho == 4 ? 11 : 17) * issued;
  launches += 20 * staged;
  h->tm.launches = (int32_t)launches;
  h->tm.learned_dirs = h->kst_host->ldirs;
  h->tm.learned_gain = h->kst_host->lgain;
  h->tm.applies = total;
  h->tm.reorths = h->p.ortho == 0 ? total : (h->p.ortho >= 3 ? 0 : h->kst_host->reorths);
  if (h->timing) {
    RP_CUDA(cudaEventRecord(h->ev[8 * batch + 1], st));
    RP_CUDA(cudaEventSynchronize(h->ev[8 * batch + 1]));
    h->tm.solve_ms = ev_ms(h->ev[8 * batch], h->ev[8 * batch + 1]);
    h->tm.apply_ms = t_apply;
    h->tm.spmv_ms = t_spmv;
    h->tm.ortho_ms = t_ortho;
  }
  h->hist_host.resize(total + 1);
  RP_CUDA(cudaMemcpy(h->hist_host.data(), h->hist, sizeof(double) * (total + 1), cudaMemcpyDeviceToHost));
  if (iters) *iters = total;
  if (relres) *relres = rel;
  int ts = check_status(h);
  if (ts != RASPML_OK) return ts;
  return status;
}

int helmholtz_solve_host(ras_pml_handle* h, const rp_c128* b_host, rp_c128* x_host, double rtol, int maxit,
                         int restart, int* iters, double* relres) {
  if (!h || !b_host || !x_host) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  if (!h->tmp_b) RP_ALLOC(h->tmp_b, (size_t)h->n);
  if (!h->tmp_x) RP_ALLOC(h->tmp_x, (size_t)h->n);
  const size_t bytes = sizeof(c128) * h->n;
  RP_CUDA(cudaMemcpyAsync(h->tmp_b, b_host, bytes, cudaMemcpyHostToDevice, h->st));
  RP_CUDA(cudaMemcpyAsync(h->tmp_x, x_host, bytes, cudaMemcpyHostToDevice, h->st));
  int s = helmholtz_solve(h, (const rp_c128*)h->tmp_b, (rp_c128*)h->tmp_x, rtol, maxit, restart, iters, relres);
  if (s < 0) return s;
  RP_CUDA(cudaMemcpyAsync(x_host, h->tmp_x, bytes, cudaMemcpyDeviceToHost, h->st));
  RP_CUDA(cudaStreamSynchronize(h->st));
  return s;
}

int ras_pml_richardson(ras_pml_handle* h, const rp_c128* b_dev, rp_c128* x_dev, double rtol, int maxit, int* iters,
                       double* relres) {
  if (!h || !b_dev || !x_dev || maxit < 0 || !(rtol >= 0.0)) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  if (!h->factored) {
    int s = ras_pml_factor(h);
    if (s != RASPML_OK) return s;
  }
  int s = ensure_krylov(h, 1, maxit);
  if (s) return s;
  if ((s = ensure_events(h, 2)) != RASPML_OK) return s;
  if (!h->tmp_r) RP_ALLOC(h->tmp_r, (size_t)h->n);
  const long long n = h->n;
  const c128* b = (const c128*)b_dev;
  c128* x = (c128*)x_dev;
  cudaStream_t st = h->st;
  // Sweeps in batches of four: each sweep is r = b - A x, ||r||, the check
  // (stop flag once rel <= rtol or after maxit sweeps), z = B^-1 r, x += z;
  // every kernel reads the stop flag first, and the host reads it one batch
  // late, so it synchronises once per four sweeps.
  KState k0{};
  RP_CUDA(cudaMemcpyAsync(h->kst, &k0, sizeof(k0), cudaMemcpyHostToDevice, st));
  if ((s = dev_norm(h, b, &h->kst->bnorm, nullptr, nullptr))) return s;
  const int batch = 4;
  int slot = 0, pending = -1;
  bool stopped = false;
  for (int it0 = 0; !stopped; it0 += batch) {
    for (int it = it0; it < it0 + batch && it <= maxit; ++it) {
      RP_CUDA(spmv_A(h, x, b, h->tmp_r, h->kst, st));
      if ((s = dev_norm(h, h->tmp_r, &h->kst->hnorm, nullptr, h->kst))) return s;
      RP_CUDA(rp::launch_rich_check(h->kst, rtol, maxit, it, h->hist, st));
      RP_CUDA(rp::launch_apply(h->p.factor_prec, h->tune.apply_cols, h->geo, h->geo_d, h->subs_d, h->nsub, h->max_b,
                               h->max_bp, h->L, h->Lrev, h->dinv, h->tmp_r, h->Y, h->V, h->kst, h->status, st,
                               rp::RK_C128, 0, &h->as));
      RP_CUDA(rp::launch_axpy_state(x, h->V, n, st, h->kst));
    }
    RP_CUDA(cudaMemcpyAsync(h->kst_host + slot, h->kst, sizeof(KState), cudaMemcpyDeviceToHost, st));
    RP_CUDA(cudaEventRecord(h->ev[slot], st));
    if (pending >= 0) {
      RP_CUDA(cudaEventSynchronize(h->ev[pending]));
      if (h->kst_host[pending].stop) stopped = true;
    }
    if (it0 + batch > maxit) {   // every sweep is enqueued: wait for the last batch
      RP_CUDA(cudaEventSynchronize(h->ev[slot]));
      stopped = true;
      pending = slot;
    }
    if (!stopped) {
      pending = slot;
      slot ^= 1;
    }
  }
  RP_CUDA(cudaStreamSynchronize(st));
  RP_CUDA(cudaMemcpy(h->kst_host, h->kst, sizeof(KState), cudaMemcpyDeviceToHost));
  const KState ks = *h->kst_host;
  const int it = ks.total;
  const double rel = ks.est;
  h->hist_host.resize(it + 1);
  RP_CUDA(cudaMemcpy(h->hist_host.data(), h->hist, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost));
  h->last_iters = it;
  if (iters) *iters = it;
  if (relres) *relres = rel;
  int ts = check_status(h);
  if (ts != RASPML_OK) return ts;
  if (ks.nan) return RASPML_ENAN;
  return ks.conv ? RASPML_OK : RASPML_NOT_CONVERGED;
}

int ras_pml_set_timing(ras_pml_handle* h, int enable) {
  if (!h) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  h->timing = enable != 0;
  if (h->timing && ensure_events(h, 36) != RASPML_OK) return RASPML_ECUDA;
  return RASPML_OK;
}

int ras_pml_get_timing(const ras_pml_handle* h, ras_pml_timing_t* t) {
  if (!h || !t) return RASPML_EBADARG;
  *t = h->tm;
  return RASPML_OK;
}

int ras_pml_history(const ras_pml_handle* h, double* hist_host, int cap, int* count) {
  if (!h || (!hist_host && cap > 0) || !count) return RASPML_EBADARG;
  int c = (int)std::min<size_t>(h->hist_host.size(), (size_t)std::max(cap, 0));
  if (c > 0) std::memcpy(hist_host, h->hist_host.data(), sizeof(double) * c);
  *count = (int)h->hist_host.size();
  return RASPML_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ras_pml_assemble_rhs_noalloc: the load-vector kernel with its source table
// in a fixed device array instead of a per-call cudaMalloc/cudaFree.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxSources = 1024;
constexpr int kNoAllocMaxDevices = 256;

// Source table shared by every call on a device: centres (x, y) of up to
// kNoAllocMaxSources sources, then their amplitudes. 24 KB per device that
// loads the library, held until the process exits.
__device__ __align__(256) double g_noalloc_sources[3 * kNoAllocMaxSources];

std::mutex g_noalloc_mu;
double* g_noalloc_table[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_sources on the current device. The host-side
// name of the array is only a stand-in; the address must come from the
// runtime, once per device, with that device current.
int noalloc_table(int dev, double** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return RASPML_EBADARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_table[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_sources);
    if (e != cudaSuccess || p == nullptr) {
      std::fprintf(stderr, "raspml: cudaGetSymbolAddress of the source table failed: %s\n",
                   cudaGetErrorString(e));
      return RASPML_ECUDA;
    }
    g_noalloc_table[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_table[dev];
  return RASPML_OK;
}

}  // namespace

extern "C" int ras_pml_assemble_rhs_noalloc(ras_pml_handle* h, const double* centres_host, const double* amps_host,
                                            int ns, double width, rp_c128* b_dev) {
  if (!h || !b_dev || ns < 0 || (ns > 0 && (!centres_host || !amps_host)) || !(width > 0.0)) return RASPML_EBADARG;
  if (ns > kNoAllocMaxSources) {
    std::fprintf(stderr, "raspml: ras_pml_assemble_rhs_noalloc takes at most %d sources (got %d)\n",
                 kNoAllocMaxSources, ns);
    return RASPML_EBADARG;
  }
  RP_CUDA(cudaSetDevice(h->dev));
  double* table = nullptr;
  int s = noalloc_table(h->dev, &table);
  if (s != RASPML_OK) return s;
  double* cen = table;
  double* amp = table + 2 * kNoAllocMaxSources;
  if (ns > 0) {
    RP_CUDA(cudaMemcpyAsync(cen, centres_host, sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, h->st));
    RP_CUDA(cudaMemcpyAsync(amp, amps_host, sizeof(double) * ns, cudaMemcpyHostToDevice, h->st));
  }
  RP_CUDA(rp::launch_rhs(h->geo, cen, amp, ns, width, (c128*)b_dev, h->st));
  return RASPML_OK;
}
