// Host-side launchers of the libraspml kernels (internal interface).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace rp {

// largest local half-bandwidth b: the factor window, (b+1)(b+2)/2 entries in
// the arithmetic type, must fit in shared memory with its buffers
constexpr int kMaxBandC128 = 160;
constexpr int kMaxBandC64 = 232;
int max_band(int prec);
// Wider subdomains (b up to kMaxBandWide, both precisions) are factored by
// the blocked kernels of factor_wide.cu, with their window in device scratch,
// and solved by k_apply_mw (a register window of up to kApplyWideSlots =
// ceil((kMaxBandWide + 1) / 32) slots shared over kApplyWideWarps warps).
constexpr int kMaxBandWide = 900;
constexpr int kApplyWideSlots = 29;
// warps per subdomain of the wide-class sweep (k_apply_mw)
#ifndef RP_APPLY_WIDE_WARPS
#define RP_APPLY_WIDE_WARPS 2
#endif
constexpr int kApplyWideWarps = RP_APPLY_WIDE_WARPS;
constexpr int kDotBlocksPerSM = 2;

// Krylov control block in device memory.
struct KState {
  int stop;        // the current Arnoldi cycle has ended
  int conv;        // residual estimate <= rtol
  int total;       // directions taken over all cycles
  int jdone;       // directions in the current cycle
  int breakdown;   // ||w|| == 0
  int nan;         // non-finite residual estimate
  int reorth;      // the current direction needs a second Gram-Schmidt pass
  int reorths;     // second passes taken over the solve
  double bnorm;    // ||b||_2
  double est;      // latest |g_{j+1}| / ||b||
  double hnorm;    // latest ||w||_2
  double relres;   // true relative residual at the last cycle start (batch)
  double beta0;    // ||r|| at the start of the current cycle
  int live;        // batch: not yet finished (converged or out of iterations)
  int ldirs;       // directions the learned stage has corrected
  double lgain;    // largest fraction of ||r1||^2 one learned correction removed
};

// Tile shapes of the factor and apply launches (chosen by the tuner).
struct Tune {
  int factor_threads = 256;   // threads per factor CTA: 128, 256, 512 (1024 with rank 2)
  int factor_rank = 2;        // pivots per pass over the window: 1 or 2
  int apply_cols = 8;         // band columns per bulk copy: 8 (4 or 16 with complex64 storage)
  int wide_cluster = 0;       // wide-band factor: 1, 2, 4 CTAs per subdomain, 16 tensor cores; 0: wide_cluster_auto
};
// factor_rank 8 or 16 (with 128 threads): the blocked form on the tensor
// cores with that many pivots per panel, complex64 arithmetic (prec 1 and 2)
// and b <= kMaxBandTc
inline bool is_tc_rank(int rank) { return rank == 8 || rank == 16; }
constexpr int kMaxBandTc = 127;
// factor_rank kRankTcBlocked (with 128 threads; the batched form, complex64
// arithmetic): the subdomains with kMaxBandTc < b <= max_band(prec) on the
// blocked tensor-core kernel of factor_wide.cu (window in a scratch slot),
// those with b <= kMaxBandTc on the tensor-core kernel with 16 pivots per
// panel; wider ones as always on the wide-band factor's own shape.
constexpr int kRankTcBlocked = 24;
// Subdomains split by half-bandwidth for the mixed factor shape (factor_rank
// 8 or 16 with 256, 512 or 1024 threads): the first nwide entries of the
// launch order have b > kMaxBandTc and go to the CUDA-core kernel (two
// pivots per pass, that many threads), the others (largest band max_b_tc)
// to the tensor-core kernel. nwide < 0: no such order (the one-problem
// handle), and the mixed shape is not available.
// max_b_narrow: the widest subdomain at or below max_band(prec) (0: none),
// for the launch of the shared-memory kernels when wider subdomains exist;
// nblocked: the number of wider ones (the blocked kernel's subdomains).
struct BandSplit {
  int nwide = -1;
  int max_b_tc = 0;
  int max_b_narrow = 0;
  int nblocked = 0;
};
bool factor_tc_ok(int prec, int max_b);
bool factor_shape_valid(int prec, int max_b, int threads, int rank, BandSplit split = BandSplit{});
// the widest subdomain of the shared-memory factor kernels: max_b, or, when
// wider subdomains go to the blocked kernel, split.max_b_narrow
int narrow_band(int prec, int max_b, BandSplit split);
bool apply_cols_valid(int prec, int cols);

// assembly.cu
// tab: scratch of stretch_table_elems(g) complex128 values (stretching tables)
size_t stretch_table_elems(const Geo& g);
cudaError_t launch_global_stencil(const Geo& g, c128* tab, c128* D, c128* CW, c128* CS, c128* CSW, cudaStream_t st);
// Aloc: 4 couplings per local row; max_b: the widest subdomain of the launch
// (sizes the kernel's stretching table)
cudaError_t launch_local_rows(int prec, const Geo* geos, const SubDesc* subs, int nsub, int max_npad, int max_b,
                              c128* Aloc, cudaStream_t st);
cudaError_t launch_rhs(const Geo& g, const double* cen, const double* amp, int ns, double width, c128* b,
                       cudaStream_t st);

// Form 1, eq. weak as printed (not symmetric): the seven couplings of every
// global row, as stored (assembly.cu, written) and as read (weak.cu).
struct Stencil7W {
  c128 *D, *W, *E, *S, *N, *SW, *NE;
};
struct Stencil7 {
  const c128 *D, *W, *E, *S, *N, *SW, *NE;
};
// largest local half-bandwidth of the form-1 factor: its square window,
// (b+1)^2 entries in the arithmetic type, must fit in shared memory
constexpr int kMaxBandLuC128 = 112;
constexpr int kMaxBandLuC64 = 160;
int max_band_lu(int prec);
size_t factor_lu_smem_bytes(int b, int prec);
// assembly.cu
cudaError_t launch_global_stencil_w(const Geo& g, const Stencil7W& A, cudaStream_t st);
// Aw: 7 complex128 couplings per local row (D, W, E, S, N, SW, NE)
cudaError_t launch_local_rows_w(int prec, const Geo* geos, const SubDesc* subs, int nsub, int max_npad, c128* Aw,
                                cudaStream_t st);
// weak.cu: y = A x, or y = bsub - A x (bsub of kind bsub_kind)
cudaError_t launch_spmv7(long long n, int nx, const Stencil7& A, const c128* x, const c128* bsub, c128* y,
                         const KState* kst, cudaStream_t st, int bsub_kind);
// A_j = L D U without pivoting; writes L, the reversed band of U (the
// backward sweep's input, zero-filled by the caller) and D^-1 in the
// layout of launch_factor
cudaError_t launch_factor_lu(int prec, const SubDesc* subs, int nsub, int max_b, const c128* Aw, void* L, void* Urev,
                             void* dinv, double* pivstats, DevStatus* status, cudaStream_t st);

// factor_wide.cu: the subdomains with bmin < b <= bmax (bmin < 0: from
// max_band(prec); b up to kMaxBandWide), each factored by a cluster of cl
// CTAs (1, 2 or 4; only from max_band(prec)) on the CUDA cores, or, with
// cl = kWideTensorCores (complex64 arithmetic, prec 1 and 2; bmin down to
// kMaxBandTc), by one CTA with the trailing update on the tensor cores, in
// its own scratch slot (SubDesc::wslot) of factor_wide_slot_bytes(prec,
// max_b) bytes, max_b the widest band of all slots (one slot stride for every
// launch); the other subdomains of the launch return at once.
// wide_cluster_auto: the largest cl in {4, 2} for which all nblocked clusters
// are resident at once (one CTA per SM), else 1.
constexpr int kWideTensorCores = 16;
size_t factor_wide_slot_bytes(int prec, int max_b);
int wide_cluster_auto(int nblocked);
cudaError_t launch_factor_wide(int prec, const SubDesc* subs, int nsub, int max_b, const c128* Aloc, void* L,
                               void* Lrev, void* dinv, double* pivstats, DevStatus* status, void* scratch,
                               cudaStream_t st, int cl, int bmin = -1, int bmax = kMaxBandWide);

// factor.cu
size_t factor_smem_bytes(int b, int prec, int rank);
// Subdomains with b > max_band(prec) (up to kMaxBandWide) need wscratch of
// (slots) x factor_wide_slot_bytes(prec, max_b) bytes, SubDesc::wslot < slots;
// skip_wide leaves them out (the tuner times the other kernels' shapes);
// wide_cluster: CTAs per wide subdomain (0: wide_cluster_auto(split.nblocked)).

// apply.cu
size_t apply_smem_bytes(int max_bp, int prec, int cols);
// wait limit of the apply's bulk copies on the current device (<= 0: default)
cudaError_t set_copy_wait_limit(long long cycles);
// Input kinds of r: complex128, double-float (dfc) or complex64
enum : int { RK_C128 = 0, RK_DF = 1, RK_C64 = 2 };
// Local solves of all subdomains into Y. The input is r of kind rkind, or
// r + (*jptr) * r_ld when jptr is set.
// Band classes of the local solves (register slots S = (b + 32) / 32):
// slot_mask bit S-1 is set when some subdomain needs S slots (0: unknown,
// every class up to max_b is launched); with both side streams set, the
// classes run concurrently, forked from and joined back to the caller's
// stream by the events (timing disabled), which also works under stream
// capture.
struct ApplyStreams {
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[2] = {nullptr, nullptr};
  uint32_t slot_mask = 0;
};
uint32_t apply_slot_mask(const SubDesc* subs_host, int nsub);
// All local factors. With side streams (as, both set) and subdomains wider
// than the shared-memory window, the wide launch, the narrow CUDA-core launch
// and the narrow tensor-core launch run concurrently (forked from st, joined
// back into it), so that SMs the wide kernel's last CTAs leave idle take
// narrow subdomains; else one after the other on st.
cudaError_t launch_factor(int prec, int threads, int rank, const SubDesc* subs, int nsub, int max_b,
                          const c128* Aloc, void* L, void* Lrev, void* dinv, double* pivstats, DevStatus* status,
                          cudaStream_t st, BandSplit split = BandSplit{}, void* wscratch = nullptr,
                          bool skip_wide = false, int wide_cluster = 0, const ApplyStreams* as = nullptr);
cudaError_t launch_local_solves(int prec, int cols, const Geo* geos, const SubDesc* subs, int nsub, int max_b,
                                int max_bp, const void* Lf, const void* Lb, const void* dinv, const c128* r,
                                long long r_ld, const int* jptr, void* Y, const KState* kst, DevStatus* status,
                                cudaStream_t st, int rkind, const ApplyStreams* as = nullptr);
// z = sum_j R_j^T Y_j; with out_df (complex64 Y only) z is written in
// double-float form (dfc)
cudaError_t launch_prolong(int prec, const Geo& g, const SubDesc* subs, const void* Y, c128* z, const KState* kst,
                           cudaStream_t st, int out_df = 0);
// one problem: local solves + prolongation
cudaError_t launch_apply(int prec, int cols, const Geo& g, const Geo* geos, const SubDesc* subs, int nsub, int max_b,
                         int max_bp, const void* Lf, const void* Lb, const void* dinv, const c128* r, void* Y,
                         c128* z, const KState* kst, DevStatus* status, cudaStream_t st, int rkind = RK_C128,
                         int out_df = 0, const ApplyStreams* as = nullptr);

// krylov.cu
cudaError_t launch_spmv(long long n, int nx, const c128* D, const c128* CW, const c128* CS, const c128* CSW,
                        const c128* x, const c128* bsub, c128* y, const KState* kst, cudaStream_t st,
                        int bsub_kind = RK_C128, int xdf = 0);
// y = A x with double-float coefficients (dfc arrays from launch_split); y
// written as dfc (double-float form) when out_df is set, x read as dfc when
// in_df is set
cudaError_t launch_spmv_df(long long n, int nx, const void* D, const void* CW, const void* CS, const void* CSW,
                           const c128* x, c128* y, const KState* kst, cudaStream_t st, int out_df = 0,
                           int in_df = 0);
int dot_blocks();
cudaError_t launch_dots(const c128* V, long long ldv, int ncols, const c128* w, long long n, c128* partial,
                        const KState* kst, int gate, cudaStream_t st);
cudaError_t launch_dots_finish(const c128* partial, int ncols, c128* out, int accumulate, const KState* kst, int gate,
                               cudaStream_t st);
cudaError_t launch_axpys(const c128* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                         long long n, const KState* kst, int gate, cudaStream_t st);
// double-float Gram-Schmidt: V and wdf hold dfc values (16 bytes each)
cudaError_t launch_split(const c128* w, void* wdf, long long n, const KState* kst, cudaStream_t st);
cudaError_t launch_scale_to_df(c128* v, long long n, const double* nrm, const KState* kst, cudaStream_t st);
cudaError_t launch_dots_df(const void* V, long long ldv, int ncols, const void* wdf, long long n, c128* partial,
                           const KState* kst, int gate, cudaStream_t st);
cudaError_t launch_axpys_df(const void* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                            long long n, const KState* kst, int gate, cudaStream_t st);
cudaError_t launch_add(c128* dst, const c128* src, int cnt, const KState* kst, int gate, cudaStream_t st);
// complex64 Krylov basis (ortho = 4): v = fl32(w / nrm); projections of w
// on the basis and the update, double-float. w is complex128 (split in the
// kernels) or, with wdf, held in double-float form (dfc); the update can
// also leave the per-block sums of |w|^2 in pnorm (*nblocks of them) for
// launch_norm_finish.
cudaError_t launch_scale_to_c64(const c128* w, void* v, long long n, const double* nrm, const KState* kst,
                                cudaStream_t st);
cudaError_t launch_scale_df_to_c64(const void* w, void* v, long long n, const double* nrm, const KState* kst,
                                   cudaStream_t st);
cudaError_t launch_dots_c64b(const void* V, long long ldv, int ncols, const c128* w, long long n, c128* partial,
                             const KState* kst, cudaStream_t st, int wdf = 0);
cudaError_t launch_axpys_c64b(const void* V, long long ldv, int ncols, const c128* h, double sign, c128* w,
                              long long n, const KState* kst, cudaStream_t st, int wdf = 0, c128* pnorm = nullptr,
                              int* nblocks = nullptr);
// The same projection and update on a basis in double-float form (dfc, the
// split complex128 basis of ortho = 3), w held in double-float form; the
// update leaves the per-block sums of |w|^2 in pnorm
cudaError_t launch_dots_dfb(const void* V, long long ldv, int ncols, const void* wdf, long long n, c128* partial,
                            const KState* kst, cudaStream_t st);
cudaError_t launch_axpys_dfb(const void* V, long long ldv, int ncols, const c128* h, double sign, void* wdf,
                             long long n, const KState* kst, cudaStream_t st, c128* pnorm, int* nblocks);
// v = w / nrm, both in double-float form (in place allowed), on the FP32 pipe
cudaError_t launch_scale_df_to_df(const void* w, void* v, long long n, const double* nrm, const KState* kst,
                                  cudaStream_t st);
// ||.|| from nparts partial sums (default: dot_blocks() of them)
cudaError_t launch_norm_finish(const c128* partial, double* out, c128* hslot, const KState* kst, int gate,
                               cudaStream_t st, int nparts = 0);
cudaError_t launch_scale_inv(c128* v, long long n, const double* nrm, const KState* kst, cudaStream_t st);
cudaError_t launch_cycle_init(KState* kst, c128* gvec, int m, double rtol, double* hist, cudaStream_t st);
// the cycle also ends (without convergence) once |g_{j+1}| <= cfloor * beta0
cudaError_t launch_givens(KState* kst, c128* H, int ldh, double* cs, c128* sn, c128* gvec, int j, double rtol,
                          int mcycle, int maxit, double* hist, cudaStream_t st, double cfloor = 0.0);
cudaError_t launch_reorth_decide(KState* kst, c128* hcol, int j, double eta2, cudaStream_t st);
cudaError_t launch_backsolve(const c128* H, int ldh, const c128* gvec, const KState* kst, c128* y,
                             cudaStream_t st);
// x += v; nothing once kst->stop is set (kst may be null)
cudaError_t launch_axpy_state(c128* x, const c128* v, long long n, cudaStream_t st, const KState* kst = nullptr);
// the residual check of a sweep of Algorithm 1 (sets the stop flag)
cudaError_t launch_rich_check(KState* kst, double rtol, int maxit, int it, double* hist, cudaStream_t st);
// z += (hv[0] / hv[1]) c, skipped when hv[1] = 0 or kst->stop
// z += alpha c (the learned stage's minimal-residual step, hv: <Ac, r1>,
// ||Ac||^2, ||r1||^2); records the stage's gain in kst; z in double-float
// form with zdf
cudaError_t launch_mr_axpy(c128* z, const c128* c, const c128* hv, long long n, KState* kst, cudaStream_t st,
                           int zdf = 0);

}  // namespace rp

namespace rp {

// ---------------------------------------------------------------------------
// Batched form (batch.cu): vectors of many problems concatenated, each
// problem starting at a multiple of kBatchTile elements.
// ---------------------------------------------------------------------------
constexpr int kBatchTile = 2048;

// Lockstep control in device memory: the current Arnoldi step j and the
// number of problems whose cycle is still running.
struct BCtl {
  int j;
  int active;
  int pad0, pad1;
};

// Everything one lockstep Arnoldi step touches (device pointers).
struct BStep {
  int prec, cols, nprob, nsub, ntiles, max_b, max_bp, m, maxit;
  double rtol;
  const Geo* geos;
  const SubDesc* subs;
  const int* sub_index;   // natural subdomain index -> launch position
  const int* tile_prob;   // tile -> problem
  const int* tile0;       // problem -> first tile
  const int* tile1;       // problem -> one past its last tile
  const void *L, *Lrev, *dinv;
  void* Y;
  const c128 *D, *CW, *CS, *CSW;
  const void *Ddf, *CWdf, *CSdf, *CSWdf;   // the same, split into double-float form
  void* V;                // (m+1) x ld complex64 basis
  c128* Z;                // m x ld preconditioned directions
  long long ld;           // batch vector length
  c128* w;
  c128* partial;          // (m+1) x ntiles
  double* pnorm;          // ntiles
  c128* H;                // per problem (m+1) x m, column-major
  long long hstride;
  double* cs;
  c128 *sn, *gvec, *yv;
  KState* kst;            // per problem
  BCtl* ctl;
  DevStatus* status;
  const ApplyStreams* as;   // band classes of the local solves (may be null)
};

// with zdf (complex64 Y only) z is written in double-float form (dfc)
cudaError_t launch_bprolong(int prec, int ntiles, const int* tile_prob, const Geo* geos, const SubDesc* subs,
                            const int* sub_index, const void* Y, c128* z, long long ldz, const int* jptr,
                            const KState* kst, int gate, cudaStream_t st, int zdf = 0);
cudaError_t launch_bspmv(int ntiles, const int* tile_prob, const Geo* geos, const c128* D, const c128* CW,
                         const c128* CS, const c128* CSW, const c128* x, long long ldx, const int* jptr,
                         const c128* bsub, c128* y, double* pnorm, const KState* kst, int gate, cudaStream_t st);
// one Arnoldi step of every running problem (j read from ctl->j, then advanced)
cudaError_t launch_bstep(const BStep& a, cudaStream_t st);
// r = b - A x, beta, stop/start decisions, v_0 (problems still being solved)
cudaError_t launch_bcycle_start(const BStep& a, const c128* b, const c128* x, int first, cudaStream_t st);
// y = R^-1 g and x += Z y for the problems of the cycle
cudaError_t launch_bcycle_end(const BStep& a, c128* x, cudaStream_t st);

}  // namespace rp

namespace rp {

// ---------------------------------------------------------------------------
// Learned coarse correction (cnn.cu): 3x3 convolutions on tensor cores
// ---------------------------------------------------------------------------
// in: NHWC BF16 [nimg][H*X][ci]; wt: B tile (core-matrix order); bias ci/co
// padded channels; mask (NHWC BF16, co channels) multiplies the output by
// (mask > 0); relu: max(., 0); outputs NHWC BF16 and/or FP32 with co channels.
cudaError_t launch_conv(int ci, int co, const void* in, const void* wt, const float* bias, const void* mask, int relu,
                        int H, int X, int nimg, void* out_bf, float* out_f, DevStatus* status, cudaStream_t st);
// B tile of layer l from the FP32 master weights (transposed: data gradient)
cudaError_t launch_prep_weights(const float* W, int l, int transposed, void* tile, cudaStream_t st);
cudaError_t launch_pad_bias(const float* b, int l, float* bp, cudaStream_t st);
cudaError_t launch_to_nhwc16(const float* x, long long npix, int nimg, void* a, cudaStream_t st);
cudaError_t launch_from_nhwc16(const float* y, long long npix, int nimg, float* x, cudaStream_t st);
// loss of the last layer's output against t (NCHW, 2 channels), its gradient
// (BF16 NHWC, 16 channels); *nparts partial sums written to lossp
cudaError_t launch_loss_grad(const float* out, const float* t, long long npix, int nimg, void* g, double* lossp,
                             int* nparts, cudaStream_t st);
int wgrad_blocks(int H, int nimg);
// weight and bias gradients of layer l (master layout) from its input a and output gradient g
cudaError_t launch_wgrad(int l, const void* a, const void* g, int H, int X, int nimg, float* part, float* grad,
                         cudaStream_t st);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, long long t, cudaStream_t st);
// coarse grid transfers of the learned stage (kernels skip when kst->stop)
int restrict_blocks(int Nc);
// out (NCHW FP32, 2 channels) = pixel means of r; partial sums of their squares
cudaError_t launch_restrict(const c128* r, int nx, int ny, int Nc, float* out, double* partial, const KState* kst,
                            cudaStream_t st);
// s = ||out|| from the partials into *s_dev; out *= Nc / s (zero when s = 0)
cudaError_t launch_normalise(float* out, int Nc, const double* partial, double* s_dev, const KState* kst,
                             cudaStream_t st);
// z += gamma * s / Nc * bilinear(first two channels of out16 (NHWC, 16 channels))
cudaError_t launch_prolong_add(const float* out16, int Nc, int nx, int ny, const double* s_dev, double gamma, c128* z,
                               const KState* kst, cudaStream_t st);
cudaError_t launch_scale_f32(float* v, long long n, float f, cudaStream_t st);
cudaError_t launch_csub(const c128* a, const c128* b, c128* out, long long n, cudaStream_t st);

}  // namespace rp
