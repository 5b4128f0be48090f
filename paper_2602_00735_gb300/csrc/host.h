// Host-side helpers shared by the one-problem and the batched handles:
// CUDA error mapping, device allocation, and the construction of one
// problem's geometry and covering (Section 2).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/raspml.h"
#include "common.cuh"
#include "kernels.h"

#define RP_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      std::fprintf(stderr, "raspml: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? RASPML_ENOMEM : RASPML_ECUDA;           \
    }                                                                                 \
  } while (0)

namespace rp {

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();   // an allocation failure is not sticky: keep it out of later launch checks
    return e == cudaErrorMemoryAllocation ? RASPML_ENOMEM : RASPML_ECUDA;
  }
  return RASPML_OK;
}

// Allocates whichever of a handle's factor buffers are still missing (L, its
// reversed band copy, D^-1, the work vector Y). After a failure the buffers
// already held stay with the handle, so a later call completes the set and
// ras_pml_destroy frees them; no buffer is ever left half-set.
inline int alloc_factor_buffers(void** L, void** Lrev, void** dinv, void** Y, size_t l_bytes, size_t v_bytes) {
  struct {
    void** p;
    size_t n;
  } bufs[4] = {{L, l_bytes}, {Lrev, l_bytes}, {dinv, v_bytes}, {Y, v_bytes}};
  for (auto& b : bufs) {
    if (*b.p) continue;
    if (cudaMalloc(b.p, b.n ? b.n : 1) != cudaSuccess) {
      *b.p = nullptr;
      cudaGetLastError();
      return RASPML_ENOMEM;
    }
  }
  return RASPML_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

inline float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.f;
  return ms;
}

// Validates p (the rules of ras_pml_setup), fills g (goff and sub0 left 0)
// and appends the descriptors of its subdomains in natural order (x fastest)
// with prob set; l_off and v_off are left for the caller. Returns a status.
int build_problem(const ras_pml_params& p, int prob, Geo& g, std::vector<SubDesc>& subs);

// Entry counts of one subdomain's factor (L: npad*bp) and per-row arrays (npad).
inline long long sub_l_entries(const SubDesc& d) { return (long long)d.npad * d.bp; }

// Scratch slots of the wide-band factor: SubDesc::wslot numbers the
// subdomains with b > max_band(prec) in order (slots 0 .. *nblocked - 1),
// then, when slot_bmin >= 0, those with slot_bmin < b <= max_band(prec) (the
// blocked tensor-core form of factor_rank kRankTcBlocked), -1 elsewhere.
// Returns the number of slots; *max_b_narrow is the widest subdomain at or
// below max_band(prec).
inline int assign_wide_slots(std::vector<SubDesc>& subs, int prec, int* max_b_narrow, int* nblocked,
                             int slot_bmin = -1) {
  int slots = 0, nb = 0;
  for (SubDesc& d : subs) {
    d.wslot = -1;
    if (d.b > max_band(prec)) d.wslot = slots++;
    else nb = std::max(nb, d.b);
  }
  *nblocked = slots;
  if (slot_bmin >= 0)
    for (SubDesc& d : subs)
      if (d.b > slot_bmin && d.b <= max_band(prec)) d.wslot = slots++;
  *max_b_narrow = nb;
  return slots;
}

// The local solves' band classes (see ApplyStreams): the slot mask of the
// subdomains and, when they fall in more than one class, two non-blocking
// side streams and the fork/join events that run the classes concurrently.
inline int make_apply_streams(ApplyStreams* as, const std::vector<SubDesc>& subs, int prec) {
  *as = ApplyStreams{};
  as->slot_mask = apply_slot_mask(subs.data(), (int)subs.size());
  const int smax = prec == 0 ? 6 : 8;
  const uint32_t lo4 = 0xFu, mid = ((1u << smax) - 1u) & ~lo4, hi = ~((1u << smax) - 1u);
  const int classes = ((as->slot_mask & lo4) != 0) + ((as->slot_mask & mid) != 0) + ((as->slot_mask & hi) != 0);
  if (classes < 2) return RASPML_OK;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&as->side[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&as->fork, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&as->join[i], cudaEventDisableTiming);
  return e == cudaSuccess ? RASPML_OK : RASPML_ECUDA;
}

inline void destroy_apply_streams(ApplyStreams* as) {
  for (int i = 0; i < 2; ++i) {
    if (as->side[i]) cudaStreamDestroy(as->side[i]);
    if (as->join[i]) cudaEventDestroy(as->join[i]);
  }
  if (as->fork) cudaEventDestroy(as->fork);
  *as = ApplyStreams{};
}

// Device scratch for the windows of the wide-band factor (nullptr and OK
// when there is no slot); the caller frees it after the factor has run.
inline int alloc_wide_scratch(void** p, int slots, int prec, int max_b) {
  *p = nullptr;
  if (slots <= 0) return RASPML_OK;
  const size_t bytes = (size_t)slots * factor_wide_slot_bytes(prec, max_b);
  if (bytes == 0) return RASPML_EBADARG;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return RASPML_ENOMEM;
  }
  return RASPML_OK;
}

// Times each tile shape of the factor and the apply on the given problem
// set (CUDA events, median of `reps`) and returns the fastest in *best.
struct TuneTarget {
  int prec;
  const Geo* geos;
  const SubDesc* subs;
  int nsub, max_b, max_bp, max_npad;
  long long sum_npad, sum_l;
  c128* Aloc;          // local rows, already assembled
  void *L, *Lrev, *dinv, *Y;
  double* pivstats;
  DevStatus* status;
  const c128* r;       // any input vector of the problems' layout
  cudaStream_t st;
  BandSplit split;     // the batched form's order by band (nwide < 0: none)
  void* wscratch;      // windows of the wide-band factor (nullptr: no wide subdomain)
};
int tune_shapes(const TuneTarget& t, int reps, Tune* best, ras_pml_tune_t* report);

}  // namespace rp
