// Tile-shape tuner: times each candidate shape of the factor launch (threads
// per CTA, pivots per pass; the blocked tensor-core form where it applies),
// the wide-band factor's cluster size (CTAs per subdomain) where there are
// wide subdomains, and the local-solve launch (band columns per bulk copy) on the caller's
// own subdomains with CUDA events on its stream, and returns the fastest (the
// default shape unless another beats it by 2%). The factor runs last with
// the chosen shape, so the factors left behind are that shape's.
#include <algorithm>

#include "host.h"

namespace rp {

namespace {

float median(std::vector<float> v) {
  std::sort(v.begin(), v.end());
  return v.empty() ? 0.f : v[v.size() / 2];
}

}  // namespace

int tune_shapes(const TuneTarget& t, int reps, Tune* best, ras_pml_tune_t* report) {
  if (reps < 1) reps = 1;
  ras_pml_tune_t rep{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RP_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RASPML_ECUDA;
  }
  cudaError_t e = cudaSuccess;
  // the CUDA-core shapes, then the tensor-core forms: alone where every
  // band allows it, else mixed with the fastest two-pivot CUDA-core shape
  // on the wide subdomains (the batched form's order by band)
  // (the batched form, complex64: also the blocked tensor-core kernel for
  // kMaxBandTc < b <= max_band with the tensor-core kernel for the rest)
  int fthreads[9] = {128, 256, 512, 256, 512, 1024, 128, 128, 128};
  const int franks[9] = {1, 1, 1, 2, 2, 2, 8, 16, kRankTcBlocked};
  // shapes are judged and timed on the subdomains of the shared-memory
  // kernels (the blocked wide-band kernel, the same in every candidate, runs
  // only in the final factor); a CUDA-core shape with fewer threads than the
  // widest window needs is skipped
  const int nb = narrow_band(t.prec, t.max_b, t.split);
  const bool tc_all = t.max_b <= max_band(t.prec) && factor_tc_ok(t.prec, t.max_b);
  const bool tc_mixed = !tc_all && t.prec >= 1 && t.split.nwide >= 0 && t.split.nwide < t.nsub && nb > 0;
  const bool tc_blocked = tc_mixed && t.wscratch != nullptr;
  const int nfc = nb == 0 ? 0 : tc_blocked ? 9 : (tc_all || tc_mixed) ? 8 : 6;   // nb == 0: every subdomain is wide
  for (int c = 0; c < nfc && e == cudaSuccess; ++c) {
    if (c == 6 && tc_mixed) {
      int b2 = -1;   // the fastest two-pivot shape timed so far
      for (int i = 0; i < rep.n_factor; ++i)
        if (rep.factor_cand_rank[i] == 2 && (b2 < 0 || rep.factor_ms[i] < rep.factor_ms[b2])) b2 = i;
      if (b2 < 0) break;
      fthreads[6] = fthreads[7] = rep.factor_cand_threads[b2];
    }
    if (!factor_shape_valid(t.prec, nb, fthreads[c], franks[c], t.split)) continue;
    std::vector<float> ms;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, t.st);
      if (e == cudaSuccess)
        e = launch_factor(t.prec, fthreads[c], franks[c], t.subs, t.nsub, t.max_b, t.Aloc, t.L, t.Lrev, t.dinv,
                          t.pivstats, t.status, t.st, t.split, t.wscratch, /*skip_wide=*/true);
      if (e == cudaSuccess) e = cudaEventRecord(e1, t.st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) ms.push_back(ev_ms(e0, e1));
    }
    rep.factor_cand_threads[rep.n_factor] = fthreads[c];
    rep.factor_cand_rank[rep.n_factor] = franks[c];
    rep.factor_ms[rep.n_factor++] = median(ms);
  }
  // the wide-band factor's shape (cluster size on the CUDA cores, or the
  // tensor-core form): its launch alone, one run per candidate (each run
  // takes tens to hundreds of milliseconds)
  if (t.split.nblocked > 0 && t.wscratch != nullptr) {
    for (int cl : {1, 2, 4, kWideTensorCores}) {
      if (e != cudaSuccess) break;
      if (cl == kWideTensorCores && t.prec == 0) continue;   // complex64 arithmetic only
      e = cudaEventRecord(e0, t.st);
      if (e == cudaSuccess)
        e = launch_factor_wide(t.prec, t.subs, t.nsub, t.max_b, t.Aloc, t.L, t.Lrev, t.dinv, t.pivstats, t.status,
                               t.wscratch, t.st, cl);
      if (e == cudaSuccess) e = cudaEventRecord(e1, t.st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) {
        rep.wide_cand[rep.n_wide] = cl;
        rep.wide_ms[rep.n_wide++] = ev_ms(e0, e1);
      }
    }
  }
  std::vector<int> acand{8};
  if (t.prec == 1) { acand.push_back(4); acand.push_back(16); }
  for (int cols : acand) {
    if (e != cudaSuccess) break;
    if (apply_smem_bytes(t.max_bp, t.prec, cols) > 227 * 1024) continue;
    std::vector<float> ms;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // the first run warms up
      e = cudaEventRecord(e0, t.st);
      if (e == cudaSuccess)
        e = launch_local_solves(t.prec, cols, t.geos, t.subs, t.nsub, t.max_b, t.max_bp, t.L, t.Lrev, t.dinv, t.r, 0,
                                nullptr, t.Y, nullptr, t.status, t.st, RK_C128);
      if (e == cudaSuccess) e = cudaEventRecord(e1, t.st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess && r > 0) ms.push_back(ev_ms(e0, e1));
    }
    rep.apply_cand[rep.n_apply] = cols;
    rep.apply_ms[rep.n_apply++] = median(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "raspml: tune: %s\n", cudaGetErrorString(e));
    return RASPML_ECUDA;
  }
  // the fastest shape, but the default (256 x 2, 8 columns) unless another
  // beats it by 2%: near-ties are decided by timing noise, and the default
  // apply shape holds up better in the solves, where stopped problems drop out
  auto pick = [](const float* ms, int n, int def) {
    int b = def;
    for (int i = 0; i < n; ++i)
      if (ms[i] < ms[b] && ms[i] < 0.98f * ms[def]) b = i;
    return b;
  };
  int fdef = 0;
  for (int i = 0; i < rep.n_factor; ++i)
    if (rep.factor_cand_threads[i] == 256 && rep.factor_cand_rank[i] == 2) fdef = i;
  if (rep.n_factor == 0) {   // only wide subdomains: the shape does not matter
    rep.factor_cand_threads[0] = 256;
    rep.factor_cand_rank[0] = 2;
    rep.factor_ms[0] = 0.f;
    rep.n_factor = 1;
  }
  const int bf = pick(rep.factor_ms, rep.n_factor, fdef);
  const int ba = rep.n_apply > 0 ? pick(rep.apply_ms, rep.n_apply, 0) : 0;
  int wcl = 0;   // the automatic choice unless another cluster size beats it by 2%
  if (rep.n_wide > 0) {
    const int cauto = wide_cluster_auto(t.split.nblocked);
    int wdef = 0;
    for (int i = 0; i < rep.n_wide; ++i)
      if (rep.wide_cand[i] == cauto) wdef = i;
    wcl = rep.wide_cand[pick(rep.wide_ms, rep.n_wide, wdef)];
  }
  // leave the factors of the chosen shape
  cudaError_t e3 = launch_factor(t.prec, rep.factor_cand_threads[bf], rep.factor_cand_rank[bf], t.subs, t.nsub,
                                 t.max_b, t.Aloc, t.L, t.Lrev, t.dinv, t.pivstats, t.status, t.st, t.split,
                                 t.wscratch, false, wcl);
  if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(t.st);
  if (e3 != cudaSuccess) {
    std::fprintf(stderr, "raspml: tune: %s\n", cudaGetErrorString(e3));
    return RASPML_ECUDA;
  }
  best->factor_threads = rep.factor_cand_threads[bf];
  best->factor_rank = rep.factor_cand_rank[bf];
  best->apply_cols = rep.n_apply > 0 ? rep.apply_cand[ba] : 8;
  best->wide_cluster = wcl;
  rep.factor_threads = best->factor_threads;
  rep.factor_rank = best->factor_rank;
  rep.apply_cols = best->apply_cols;
  rep.wide_cluster = wcl > 0 ? wcl : (t.split.nblocked > 0 ? wide_cluster_auto(t.split.nblocked) : 0);
  if (report) *report = rep;
  return RASPML_OK;
}

}  // namespace rp
