// Host side of the batched form: many independent problems, each built as
// ras_pml_setup builds one (Section 2's covering of its own domain), whose
// subdomains are factored and applied in single launches and whose FGMRES
// (Section 4.1) runs in lockstep, one Arnoldi step per replay of a captured
// CUDA graph. This file only sizes, launches and synchronises; the
// arithmetic is in assembly.cu, factor.cu, apply.cu and batch.cu.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "host.h"

using rp::BCtl;
using rp::c128;
using rp::dalloc;
using rp::dfree;
using rp::Geo;
using rp::KState;
using rp::SubDesc;

struct ras_pml_batch {
  int dev = 0;
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;    // private stream for graph capture
  int nprob = 0, prec = 0;
  std::vector<Geo> geos_h;
  std::vector<SubDesc> subs_h;      // launch order (decreasing factor cost)
  std::vector<int> sub_index_h;     // natural index -> launch position
  rp::BandSplit split;              // wide subdomains first in the launch order
  rp::ApplyStreams as{};            // band classes of the local solves, run concurrently
  std::vector<int> tile_prob_h, tile0_h, tile1_h;
  long long ntot = 0, sum_n = 0, sum_npad = 0, sum_l = 0, sum_bn = 0;
  int nsub = 0, max_b = 0, max_bp = 0, max_npad = 0, ntiles = 0;
  int nwslot = 0;                   // scratch slots (split.nblocked of them for b > max_band)
  Geo* geos_d = nullptr;
  SubDesc* subs_d = nullptr;
  int *sub_index_d = nullptr, *tile_prob_d = nullptr, *tile0_d = nullptr, *tile1_d = nullptr;
  c128 *D = nullptr, *CW = nullptr, *CS = nullptr, *CSW = nullptr;
  c128 *Ddf = nullptr, *CWdf = nullptr, *CSdf = nullptr, *CSWdf = nullptr;   // split, for the Arnoldi SpMV
  void *L = nullptr, *Lrev = nullptr, *dinv = nullptr, *Y = nullptr;
  double* pivstats = nullptr;
  rp::DevStatus* status = nullptr;
  rp::Tune tune{};
  bool factored = false;
  double min_pivot_ratio = 0.0;
  int bad_prob = -1, bad_sub = -1;
  // Krylov workspace
  int kcap = 0;
  void* V = nullptr;
  c128 *Z = nullptr, *w = nullptr, *partial = nullptr, *H = nullptr, *sn = nullptr, *gvec = nullptr, *yv = nullptr;
  double *cs = nullptr, *pnorm = nullptr;
  KState* kst = nullptr;
  KState* kst_host = nullptr;       // pinned, nprob entries
  BCtl* ctl = nullptr;
  int* active_host = nullptr;       // pinned, 2 slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int g_m = -1, g_maxit = -1, g_cols = -1;
  double g_rtol = -1.0;
  int steps = 0, cycles = 0;
};

namespace {

size_t entry_bytes(int prec) { return prec == 0 ? 16 : 8; }                          // D^-1, Y
size_t l_bytes(int prec) { return prec == 0 ? 16 : prec == 1 ? 8 : 4; }              // L entries

void free_krylov(ras_pml_batch* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  h->g_m = -1;
  dfree(h->V); dfree(h->Z); dfree(h->w); dfree(h->partial); dfree(h->H); dfree(h->sn); dfree(h->gvec);
  dfree(h->yv); dfree(h->cs); dfree(h->pnorm);
  h->kcap = 0;
}

int ensure_krylov(ras_pml_batch* h, int m) {
  if (h->kcap >= m) return RASPML_OK;
  free_krylov(h);
  int s;
#define BK_ALLOC(ptr, cnt) \
  if ((s = dalloc(&(ptr), (cnt))) != RASPML_OK) { free_krylov(h); return s; }
  rp::c64* v = nullptr;   // complex64 basis
  BK_ALLOC(v, (size_t)(m + 1) * h->ntot);
  h->V = v;
  BK_ALLOC(h->Z, (size_t)m * h->ntot);
  BK_ALLOC(h->w, (size_t)h->ntot);
  BK_ALLOC(h->partial, (size_t)(m + 1) * h->ntiles);
  BK_ALLOC(h->pnorm, (size_t)h->ntiles);
  BK_ALLOC(h->H, (size_t)h->nprob * (m + 1) * m);
  BK_ALLOC(h->cs, (size_t)h->nprob * m);
  BK_ALLOC(h->sn, (size_t)h->nprob * m);
  BK_ALLOC(h->gvec, (size_t)h->nprob * (m + 1));
  BK_ALLOC(h->yv, (size_t)h->nprob * m);
#undef BK_ALLOC
  h->kcap = m;
  return RASPML_OK;
}

rp::BStep step_args(ras_pml_batch* h, int m, double rtol, int maxit) {
  rp::BStep a{};
  a.prec = h->prec;
  a.cols = h->tune.apply_cols;
  a.nprob = h->nprob;
  a.nsub = h->nsub;
  a.ntiles = h->ntiles;
  a.max_b = h->max_b;
  a.max_bp = h->max_bp;
  a.m = m;
  a.maxit = maxit;
  a.rtol = rtol;
  a.geos = h->geos_d;
  a.subs = h->subs_d;
  a.sub_index = h->sub_index_d;
  a.tile_prob = h->tile_prob_d;
  a.tile0 = h->tile0_d;
  a.tile1 = h->tile1_d;
  a.L = h->L;
  a.Lrev = h->Lrev;
  a.dinv = h->dinv;
  a.Y = h->Y;
  a.D = h->D;
  a.CW = h->CW;
  a.CS = h->CS;
  a.CSW = h->CSW;
  a.Ddf = h->Ddf;
  a.CWdf = h->CWdf;
  a.CSdf = h->CSdf;
  a.CSWdf = h->CSWdf;
  a.V = h->V;
  a.Z = h->Z;
  a.ld = h->ntot;
  a.w = h->w;
  a.partial = h->partial;
  a.pnorm = h->pnorm;
  a.H = h->H;
  a.hstride = (long long)(m + 1) * m;
  a.cs = h->cs;
  a.sn = h->sn;
  a.gvec = h->gvec;
  a.yv = h->yv;
  a.kst = h->kst;
  a.ctl = h->ctl;
  a.status = h->status;
  a.as = &h->as;
  return a;
}

// The Arnoldi step as a graph, captured on the private stream; re-captured
// when the cycle length, rtol, maxit or a tile shape changes.
int ensure_graph(ras_pml_batch* h, const rp::BStep& a) {
  if (h->exec && h->g_m == a.m && h->g_rtol == a.rtol && h->g_maxit == a.maxit && h->g_cols == a.cols)
    return RASPML_OK;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  RP_CUDA(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed));
  cudaError_t e = rp::launch_bstep(a, h->cap_st);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->cap_st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    std::fprintf(stderr, "raspml: batch graph capture: %s\n", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return RASPML_ECUDA;
  }
  e = cudaGraphInstantiate(&h->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    std::fprintf(stderr, "raspml: batch graph instantiate: %s\n", cudaGetErrorString(e));
    return RASPML_ECUDA;
  }
  h->graph = g;
  h->g_m = a.m;
  h->g_rtol = a.rtol;
  h->g_maxit = a.maxit;
  h->g_cols = a.cols;
  return RASPML_OK;
}

}  // namespace

extern "C" {

void ras_pml_batch_destroy(ras_pml_batch* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->st) cudaStreamSynchronize(h->st);
  free_krylov(h);
  dfree(h->geos_d); dfree(h->subs_d); dfree(h->sub_index_d); dfree(h->tile_prob_d); dfree(h->tile0_d);
  dfree(h->tile1_d); dfree(h->D); dfree(h->CW); dfree(h->CS); dfree(h->CSW); dfree(h->L); dfree(h->Lrev);
  dfree(h->Ddf); dfree(h->CWdf); dfree(h->CSdf); dfree(h->CSWdf);
  dfree(h->dinv); dfree(h->Y); dfree(h->pivstats); dfree(h->status); dfree(h->kst); dfree(h->ctl);
  if (h->kst_host) cudaFreeHost(h->kst_host);
  if (h->active_host) cudaFreeHost(h->active_host);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  rp::destroy_apply_streams(&h->as);
  delete h;
}

int ras_pml_batch_setup(const ras_pml_params* params, int nprob, void* stream, ras_pml_batch** out) {
  if (!params || !out || nprob < 1) return RASPML_EBADARG;
  *out = nullptr;
  ras_pml_batch* h = new ras_pml_batch();
  h->nprob = nprob;
  h->prec = params[0].factor_prec;
  h->st = (cudaStream_t)stream;
  cudaGetDevice(&h->dev);
  std::vector<SubDesc> nat;   // natural order: problem by problem, x fastest
  long long goff = 0;
  for (int q = 0; q < nprob; ++q) {
    // the batched kernels take the symmetric form only
    if (params[q].factor_prec != h->prec || params[q].form != 0) { delete h; return RASPML_EBADARG; }
    Geo g{};
    const int s = rp::build_problem(params[q], q, g, nat);
    if (s != RASPML_OK) { delete h; return s; }
    g.goff = goff;
    g.sub0 = (int)(nat.size() - (size_t)g.px * g.py);
    const long long npad = ((long long)g.n + rp::kBatchTile - 1) / rp::kBatchTile * rp::kBatchTile;
    h->tile0_h.push_back((int)(goff / rp::kBatchTile));
    for (long long t = 0; t < npad / rp::kBatchTile; ++t) h->tile_prob_h.push_back(q);
    goff += npad;
    h->tile1_h.push_back((int)(goff / rp::kBatchTile));
    h->sum_n += g.n;
    h->geos_h.push_back(g);
  }
  h->ntot = goff;
  h->ntiles = (int)h->tile_prob_h.size();
  h->nsub = (int)nat.size();
  // launch order: the subdomains wider than the tensor-core factor's limit
  // first, then the others, each part by decreasing factor cost npad * b^2
  // (ties: natural order)
  std::vector<int> order(h->nsub);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const bool wa = nat[a].b > rp::kMaxBandTc, wb = nat[b].b > rp::kMaxBandTc;
    if (wa != wb) return wa;
    return (double)nat[a].npad * nat[a].b * nat[a].b > (double)nat[b].npad * nat[b].b * nat[b].b;
  });
  h->split.nwide = 0;
  h->split.max_b_tc = 0;
  for (int i = 0; i < h->nsub; ++i) {
    if (nat[i].b > rp::kMaxBandTc) ++h->split.nwide;
    else h->split.max_b_tc = std::max(h->split.max_b_tc, nat[i].b);
  }
  h->sub_index_h.assign(h->nsub, 0);
  long long l_off = 0, v_off = 0;
  for (int pos = 0; pos < h->nsub; ++pos) {
    SubDesc d = nat[order[pos]];
    h->sub_index_h[order[pos]] = pos;
    d.l_off = l_off;
    d.v_off = v_off;
    l_off += rp::sub_l_entries(d);
    v_off += d.npad;
    h->max_b = std::max(h->max_b, d.b);
    h->max_bp = std::max(h->max_bp, d.bp);
    h->max_npad = std::max(h->max_npad, d.npad);
    h->sum_bn += (long long)d.b * d.n;
    h->subs_h.push_back(d);
  }
  h->sum_npad = v_off;
  h->sum_l = l_off;
  // scratch slots: the subdomains wider than the shared-memory window, then
  // (complex64 arithmetic) those with kMaxBandTc < b <= max_band for the
  // blocked tensor-core shape (factor_rank kRankTcBlocked)
  h->nwslot = rp::assign_wide_slots(h->subs_h, h->prec, &h->split.max_b_narrow, &h->split.nblocked,
                                    h->prec >= 1 ? rp::kMaxBandTc : -1);
  if (const int sa = rp::make_apply_streams(&h->as, h->subs_h, h->prec); sa != RASPML_OK) {
    ras_pml_batch_destroy(h);
    return sa;
  }

  int s;
#define BS_ALLOC(ptr, cnt) \
  if ((s = dalloc(&(ptr), (cnt))) != RASPML_OK) { ras_pml_batch_destroy(h); return s; }
  BS_ALLOC(h->geos_d, (size_t)nprob);
  BS_ALLOC(h->subs_d, (size_t)h->nsub);
  BS_ALLOC(h->sub_index_d, (size_t)h->nsub);
  BS_ALLOC(h->tile_prob_d, (size_t)h->ntiles);
  BS_ALLOC(h->tile0_d, (size_t)nprob);
  BS_ALLOC(h->tile1_d, (size_t)nprob);
  BS_ALLOC(h->D, (size_t)h->ntot);
  BS_ALLOC(h->CW, (size_t)h->ntot);
  BS_ALLOC(h->CS, (size_t)h->ntot);
  BS_ALLOC(h->CSW, (size_t)h->ntot);
  BS_ALLOC(h->Ddf, (size_t)h->ntot);
  BS_ALLOC(h->CWdf, (size_t)h->ntot);
  BS_ALLOC(h->CSdf, (size_t)h->ntot);
  BS_ALLOC(h->CSWdf, (size_t)h->ntot);
  BS_ALLOC(h->pivstats, (size_t)2 * h->nsub);
  BS_ALLOC(h->status, (size_t)1);
  BS_ALLOC(h->kst, (size_t)nprob);
  BS_ALLOC(h->ctl, (size_t)1);
#undef BS_ALLOC
  cudaError_t e = cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->kst_host, sizeof(KState) * nprob);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->active_host, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st);
  };
  up(h->geos_d, h->geos_h.data(), sizeof(Geo) * nprob);
  up(h->subs_d, h->subs_h.data(), sizeof(SubDesc) * h->nsub);
  up(h->sub_index_d, h->sub_index_h.data(), sizeof(int) * h->nsub);
  up(h->tile_prob_d, h->tile_prob_h.data(), sizeof(int) * h->ntiles);
  up(h->tile0_d, h->tile0_h.data(), sizeof(int) * nprob);
  up(h->tile1_d, h->tile1_h.data(), sizeof(int) * nprob);
  rp::DevStatus s0{-1, 0, 0, 0};
  up(h->status, &s0, sizeof(s0));
  for (c128* a : {h->D, h->CW, h->CS, h->CSW})
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, sizeof(c128) * h->ntot, h->st);
  size_t tabn = 0;
  for (int q = 0; q < nprob; ++q) tabn = std::max(tabn, rp::stretch_table_elems(h->geos_h[q]));
  c128* tab = nullptr;   // one problem's stretching tables at a time (stream-ordered reuse)
  if (e == cudaSuccess) e = cudaMalloc((void**)&tab, sizeof(c128) * tabn);
  for (int q = 0; q < nprob && e == cudaSuccess; ++q) {
    const long long o = h->geos_h[q].goff;
    e = rp::launch_global_stencil(h->geos_h[q], tab, h->D + o, h->CW + o, h->CS + o, h->CSW + o, h->st);
  }
  if (e == cudaSuccess) e = rp::launch_split(h->D, h->Ddf, h->ntot, nullptr, h->st);
  if (e == cudaSuccess) e = rp::launch_split(h->CW, h->CWdf, h->ntot, nullptr, h->st);
  if (e == cudaSuccess) e = rp::launch_split(h->CS, h->CSdf, h->ntot, nullptr, h->st);
  if (e == cudaSuccess) e = rp::launch_split(h->CSW, h->CSWdf, h->ntot, nullptr, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (tab) cudaFree(tab);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "raspml: batch setup: %s\n", cudaGetErrorString(e));
    ras_pml_batch_destroy(h);
    return e == cudaErrorMemoryAllocation ? RASPML_ENOMEM : RASPML_ECUDA;
  }
  *out = h;
  return RASPML_OK;
}

int ras_pml_batch_info(const ras_pml_batch* h, ras_pml_batch_info_t* info) {
  if (!h || !info) return RASPML_EBADARG;
  std::memset(info, 0, sizeof(*info));
  info->nprob = h->nprob;
  info->num_sub = h->nsub;
  info->ntot = h->ntot;
  info->sum_n = h->sum_n;
  long long sl = 0;
  for (const SubDesc& d : h->subs_h) sl += d.n;
  info->sum_local_n = sl;
  info->max_band = h->max_b;
  info->factor_prec = h->prec;
  const double es = (double)entry_bytes(h->prec), esl = (double)l_bytes(h->prec);
  info->factor_bytes = (int64_t)(2 * h->sum_l * esl + h->sum_npad * es);
  // both sweeps read L (2 s sum b n), D^-1 once, r and z once each
  info->apply_bytes = 2.0 * esl * (double)h->sum_bn + es * (double)sl + 32.0 * (double)h->sum_n;
  info->min_pivot_ratio = h->min_pivot_ratio;
  info->factored = h->factored ? 1 : 0;
  info->bad_problem = h->bad_prob;
  info->bad_subdomain = h->bad_sub;
  info->factor_threads = h->tune.factor_threads;
  info->factor_rank = h->tune.factor_rank;
  info->apply_cols = h->tune.apply_cols;
  info->steps = h->steps;
  info->cycles = h->cycles;
  info->kcap = h->kcap;
  return RASPML_OK;
}

int ras_pml_batch_layout(const ras_pml_batch* h, int64_t* offsets, int64_t* sizes) {
  if (!h || !offsets || !sizes) return RASPML_EBADARG;
  for (int q = 0; q < h->nprob; ++q) {
    offsets[q] = h->geos_h[q].goff;
    sizes[q] = h->geos_h[q].n;
  }
  return RASPML_OK;
}

int ras_pml_batch_assemble_rhs(ras_pml_batch* h, const int32_t* ns, const double* centres, const double* amps,
                               const double* widths, rp_c128* b) {
  if (!h || !ns || !widths || !b) return RASPML_EBADARG;
  long long tot = 0;
  for (int q = 0; q < h->nprob; ++q) {
    if (ns[q] < 0 || !(widths[q] > 0.0)) return RASPML_EBADARG;
    tot += ns[q];
  }
  if (tot > 0 && (!centres || !amps)) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  double* src = nullptr;   // [2*tot centres | tot amps]
  RP_CUDA(cudaMalloc((void**)&src, sizeof(double) * (size_t)(3 * tot + 1)));
  cudaError_t e = cudaSuccess;
  if (tot > 0) {
    e = cudaMemcpyAsync(src, centres, sizeof(double) * 2 * tot, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(src + 2 * tot, amps, sizeof(double) * tot, cudaMemcpyHostToDevice, h->st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b, 0, sizeof(c128) * h->ntot, h->st);
  long long so = 0;
  for (int q = 0; q < h->nprob && e == cudaSuccess; ++q) {
    const Geo& g = h->geos_h[q];
    e = rp::launch_rhs(g, src + 2 * so, src + 2 * tot + so, ns[q], widths[q], (c128*)b + g.goff, h->st);
    so += ns[q];
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFree(src);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "raspml: batch rhs: %s\n", cudaGetErrorString(e));
    return RASPML_ECUDA;
  }
  return RASPML_OK;
}

namespace {

int batch_alloc_factors(ras_pml_batch* h) {
  const size_t esl = l_bytes(h->prec), es = entry_bytes(h->prec);
  return rp::alloc_factor_buffers(&h->L, &h->Lrev, &h->dinv, &h->Y, (size_t)h->sum_l * esl,
                                  (size_t)h->sum_npad * es);
}

// local rows of every subdomain into a fresh Aloc (caller frees)
int batch_local_rows(ras_pml_batch* h, c128** Aloc) {
  int s = dalloc(Aloc, (size_t)4 * h->sum_npad);
  if (s != RASPML_OK) return s;
  RP_CUDA(rp::launch_local_rows(h->prec, h->geos_d, h->subs_d, h->nsub, h->max_npad, h->max_b, *Aloc, h->st));
  return RASPML_OK;
}

}  // namespace

int ras_pml_batch_factor(ras_pml_batch* h) {
  if (!h) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  h->factored = false;
  int s = batch_alloc_factors(h);
  if (s != RASPML_OK) return s;
  rp::DevStatus s0{-1, 0, 0, 0};
  RP_CUDA(cudaMemcpyAsync(h->status, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->st));
  RP_CUDA(cudaMemsetAsync(h->Lrev, 0, (size_t)h->sum_l * l_bytes(h->prec), h->st));
  c128* Aloc = nullptr;
  s = batch_local_rows(h, &Aloc);
  if (s != RASPML_OK) { dfree(Aloc); return s; }
  void* wscratch = nullptr;
  const int slots = h->tune.factor_rank == rp::kRankTcBlocked ? h->nwslot : h->split.nblocked;
  if ((s = rp::alloc_wide_scratch(&wscratch, slots, h->prec, h->max_b)) != RASPML_OK) {
    dfree(Aloc);
    return s;
  }
  cudaError_t e = rp::launch_factor(h->prec, h->tune.factor_threads, h->tune.factor_rank, h->subs_d, h->nsub, h->max_b, Aloc, h->L,
                                    h->Lrev, h->dinv, h->pivstats, h->status, h->st, h->split, wscratch, false,
                                    h->tune.wide_cluster, &h->as);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  dfree(Aloc);
  if (wscratch) cudaFree(wscratch);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "raspml: batch factor: %s\n", cudaGetErrorString(e));
    return RASPML_ECUDA;
  }
  rp::DevStatus stt;
  std::vector<double> piv(2 * h->nsub);
  RP_CUDA(cudaMemcpy(&stt, h->status, sizeof(stt), cudaMemcpyDeviceToHost));
  RP_CUDA(cudaMemcpy(piv.data(), h->pivstats, sizeof(double) * piv.size(), cudaMemcpyDeviceToHost));
  double mr = 1e300;
  for (int j = 0; j < h->nsub; ++j) mr = std::min(mr, piv[2 * j] / piv[2 * j + 1]);
  h->min_pivot_ratio = mr;
  h->bad_prob = h->bad_sub = -1;
  if (stt.timeout) return RASPML_ETIMEOUT;
  if (stt.pivot_bad_sub >= 0) {
    const SubDesc& d = h->subs_h[stt.pivot_bad_sub];
    h->bad_prob = d.prob;
    for (int i = 0; i < h->nsub; ++i)
      if (h->sub_index_h[i] == stt.pivot_bad_sub) h->bad_sub = i - h->geos_h[d.prob].sub0;
    return RASPML_EPIVOT;
  }
  h->factored = true;
  return RASPML_OK;
}

int ras_pml_batch_tune(ras_pml_batch* h, ras_pml_tune_t* report) {
  if (!h) return RASPML_EBADARG;
  int s = ras_pml_batch_factor(h);
  if (s != RASPML_OK) return s;
  c128 *Aloc = nullptr, *r = nullptr;
  s = batch_local_rows(h, &Aloc);
  if (s == RASPML_OK) s = dalloc(&r, (size_t)h->ntot);
  if (s == RASPML_OK && cudaMemsetAsync(r, 0, sizeof(c128) * h->ntot, h->st) != cudaSuccess) s = RASPML_ECUDA;
  if (s == RASPML_OK) {
    void* wscratch = nullptr;
    s = rp::alloc_wide_scratch(&wscratch, h->nwslot, h->prec, h->max_b);
    rp::TuneTarget t{h->prec, h->geos_d, h->subs_d, h->nsub, h->max_b, h->max_bp, h->max_npad, h->sum_npad,
                     h->sum_l, Aloc, h->L, h->Lrev, h->dinv, h->Y, h->pivstats, h->status, r, h->st, h->split,
                     wscratch};
    if (s == RASPML_OK) s = rp::tune_shapes(t, 3, &h->tune, report);
    if (wscratch) cudaFree(wscratch);
  }
  cudaStreamSynchronize(h->st);
  dfree(Aloc);
  dfree(r);
  return s;
}

int ras_pml_batch_set_shapes(ras_pml_batch* h, int factor_threads, int factor_rank, int apply_cols, int wide_cluster) {
  if (!h ||
      !rp::factor_shape_valid(h->prec, rp::narrow_band(h->prec, h->max_b, h->split), factor_threads, factor_rank,
                              h->split) ||
      !rp::apply_cols_valid(h->prec, apply_cols) ||
      !(wide_cluster == 0 || wide_cluster == 1 || wide_cluster == 2 || wide_cluster == 4 ||
        (wide_cluster == rp::kWideTensorCores && h->prec >= 1)))
    return RASPML_EBADARG;
  h->tune.factor_threads = factor_threads;
  h->tune.factor_rank = factor_rank;
  h->tune.apply_cols = apply_cols;
  h->tune.wide_cluster = wide_cluster;
  return RASPML_OK;
}

int ras_pml_batch_apply(ras_pml_batch* h, const rp_c128* r, rp_c128* z) {
  if (!h || !r || !z || (const void*)r == (const void*)z) return RASPML_EBADARG;
  if (!h->factored) return RASPML_ESTATE;
  cudaSetDevice(h->dev);
  RP_CUDA(rp::launch_local_solves(h->prec, h->tune.apply_cols, h->geos_d, h->subs_d, h->nsub, h->max_b, h->max_bp,
                                  h->L, h->Lrev, h->dinv, (const c128*)r, 0, nullptr, h->Y, nullptr, h->status,
                                  h->st, rp::RK_C128, &h->as));
  RP_CUDA(rp::launch_bprolong(h->prec, h->ntiles, h->tile_prob_d, h->geos_d, h->subs_d, h->sub_index_d, h->Y,
                              (c128*)z, 0, nullptr, nullptr, 0, h->st));
  return RASPML_OK;
}

int ras_pml_batch_matvec(ras_pml_batch* h, const rp_c128* x, rp_c128* y) {
  if (!h || !x || !y || (const void*)x == (const void*)y) return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  RP_CUDA(rp::launch_bspmv(h->ntiles, h->tile_prob_d, h->geos_d, h->D, h->CW, h->CS, h->CSW, (const c128*)x, 0,
                           nullptr, nullptr, (c128*)y, nullptr, nullptr, 0, h->st));
  return RASPML_OK;
}

int ras_pml_batch_solve(ras_pml_batch* h, const rp_c128* b, rp_c128* x, double rtol, int maxit, int restart,
                        int32_t* iters, double* relres) {
  if (!h || !b || !x || (const void*)b == (const void*)x || !(rtol >= 0.0) || maxit < 1 || restart < 0 || !iters ||
      !relres)
    return RASPML_EBADARG;
  cudaSetDevice(h->dev);
  int s;
  if (!h->factored && (s = ras_pml_batch_factor(h)) != RASPML_OK) return s;
  // at most 1024 directions per cycle (the projection keeps per-warp sums of
  // every column in shared memory)
  int m = std::min(restart > 0 ? std::min(restart, maxit) : maxit, 1024);
  // cap the cycle at the Krylov space that fits in free memory (V and Z
  // take 8 + 16 bytes per element and direction)
  if (h->kcap < m) {
    free_krylov(h);
    size_t fr = 0, tot = 0;
    RP_CUDA(cudaMemGetInfo(&fr, &tot));
    const double reserve = 512.0 * (1 << 20) + 32.0 * (double)h->ntot;
    const double per = 24.0 * (double)h->ntot + 16.0 * h->ntiles + 80.0 * h->nprob;
    const double fit = ((double)fr - reserve) / per - 1.0;
    if (fit < 1.0) return RASPML_ENOMEM;
    m = std::min(m, (int)fit);
    if ((s = ensure_krylov(h, m)) != RASPML_OK) return s;
  }
  m = std::min(m, h->kcap);
  const rp::BStep a = step_args(h, m, rtol, maxit);
  if ((s = ensure_graph(h, a)) != RASPML_OK) return s;

  std::vector<KState> k0(h->nprob);
  for (KState& k : k0) {
    k = KState{};
    k.stop = 1;
    k.live = 1;
  }
  RP_CUDA(cudaMemcpyAsync(h->kst, k0.data(), sizeof(KState) * h->nprob, cudaMemcpyHostToDevice, h->st));
  RP_CUDA(cudaMemsetAsync(x, 0, sizeof(c128) * h->ntot, h->st));
  h->steps = 0;
  h->cycles = 0;
  const int kBatchSteps = 4;
  for (int cyc = 0; cyc <= maxit; ++cyc) {
    RP_CUDA(cudaMemsetAsync(h->ctl, 0, sizeof(BCtl), h->st));
    RP_CUDA(rp::launch_bcycle_start(a, (const c128*)b, (const c128*)x, cyc == 0 ? 1 : 0, h->st));
    RP_CUDA(cudaMemcpyAsync(h->active_host, &h->ctl->active, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    RP_CUDA(cudaStreamSynchronize(h->st));
    if (h->active_host[0] == 0) break;
    ++h->cycles;
    // replay the step graph; the count of running problems comes back once
    // per batch of steps, read one batch late so the device never idles
    int pending = -1;
    for (int j0 = 0; j0 < m; j0 += kBatchSteps) {
      const int j1 = std::min(m, j0 + kBatchSteps);
      for (int j = j0; j < j1; ++j) RP_CUDA(cudaGraphLaunch(h->exec, h->st));
      h->steps += j1 - j0;
      const int slot = (j0 / kBatchSteps) & 1;
      RP_CUDA(cudaMemcpyAsync(h->active_host + slot, &h->ctl->active, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      RP_CUDA(cudaEventRecord(h->ev[slot], h->st));
      if (pending >= 0) {
        RP_CUDA(cudaEventSynchronize(h->ev[pending]));
        if (h->active_host[pending] == 0) break;
      }
      pending = slot;
    }
    RP_CUDA(rp::launch_bcycle_end(a, (c128*)x, h->st));
  }
  RP_CUDA(cudaMemcpyAsync(h->kst_host, h->kst, sizeof(KState) * h->nprob, cudaMemcpyDeviceToHost, h->st));
  RP_CUDA(cudaStreamSynchronize(h->st));
  rp::DevStatus stt;
  RP_CUDA(cudaMemcpy(&stt, h->status, sizeof(stt), cudaMemcpyDeviceToHost));
  if (stt.timeout) return RASPML_ETIMEOUT;
  bool all = true, nan = false;
  for (int q = 0; q < h->nprob; ++q) {
    const KState& k = h->kst_host[q];
    iters[q] = k.total;
    relres[q] = k.relres;
    all = all && k.conv;
    nan = nan || k.nan;
  }
  if (nan) return RASPML_ENAN;
  return all ? RASPML_OK : RASPML_NOT_CONVERGED;
}

}  // extern "C"
