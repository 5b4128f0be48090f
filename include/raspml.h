/*
 * raspml.h -- C ABI of libraspml.so: the RAS-PML preconditioner and a
 * device-side flexible GMRES for P1 discretisations of the 2D Helmholtz
 * equation with a Cartesian PML, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Xie, Gong, Graham, Spence, Zhang, "Massively parallel Schwarz
 * methods for the high frequency Helmholtz equation".
 *   - Problem and PML truncation: Section 1 (eq. helmholtz0, the definitions
 *     of g, g_i, gamma_i and eq. weak).
 *   - Covering, local PML, local forms a_j, partition of unity: Section 2.
 *   - Preconditioner B^-1 = sum_j R~_j^T A_j^-1 R_j: Section 2 (the equation
 *     after eq. update1).
 *   - Impedance closure of the local problems (RAS-PML-Imp): Section 3 (ii),
 *     eq. impedance.
 *   - GMRES with B^-1 as preconditioner: Section 4.1; Algorithm 1 for the
 *     Richardson form.
 *
 * Discretisation (identical on every entry point):
 *   Omega = [x0-kappa_g, x1+kappa_g] x [y0-kappa_g, y1+kappa_g], Mx x My square
 *   cells of side h, each split along its (i,j)-(i+1,j+1) diagonal; P1
 *   elements; the gamma_1*gamma_2-multiplied (complex-symmetric) form of
 *   eq. weak; every element integral by the three-point edge-midpoint rule;
 *   impedance edges by 2-point Gauss. Unknowns are the (Mx-1)*(My-1) nodes not
 *   on the outer boundary, numbered x-fastest: node (i,j), 1<=i<=Mx-1,
 *   1<=j<=My-1, has index (j-1)*(Mx-1) + (i-1).
 *
 * Conventions:
 *   - Complex vectors are interleaved (re, im) doubles, i.e. the memory layout
 *     of torch.complex128 / std::complex<double>.
 *   - "_dev" pointers are device pointers on the handle's device; the caller
 *     owns them. They must be 16-byte aligned and hold n elements.
 *   - "_host" pointers are host pointers (pageable or pinned).
 *   - The library owns everything it allocates (factors, index tables,
 *     Krylov workspace) and frees it in ras_pml_destroy.
 *   - Work is enqueued on the stream given to ras_pml_setup. Calls return
 *     after enqueueing, except ras_pml_factor, helmholtz_solve and
 *     helmholtz_solve_host, which return when their result is known.
 *   - A handle is not thread-safe; use one handle per host thread.
 *
 * Status codes: 0 success; 1 not converged within maxit (outputs still
 * valid); negative values are errors, see ras_pml_error_string().
 */
#ifndef RASPML_H
#define RASPML_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RASPML_OK              0
#define RASPML_NOT_CONVERGED   1
#define RASPML_EBADARG        -1  /* invalid parameter or size            */
#define RASPML_ENOMEM         -2  /* device allocation failed             */
#define RASPML_ECUDA          -3  /* CUDA runtime error                   */
#define RASPML_EPIVOT         -4  /* zero/tiny pivot in a local factor    */
#define RASPML_ENAN           -5  /* NaN or Inf in a residual             */
#define RASPML_ETIMEOUT       -6  /* a bounded device-side wait gave up   */
#define RASPML_ESTATE         -7  /* call out of order (e.g. not factored)*/

/* One complex128 element; same layout as torch.complex128. */
typedef struct { double re, im; } rp_c128;

/* Problem and method parameters (Section 1 and Section 2 of the paper). */
typedef struct {
  double k;               /* wavenumber (wave speed c = 1), k >= 0               */
  double x0, y0, x1, y1;  /* Omega_int = (x0,x1) x (y0,y1)                       */
  double kappa_g;         /* global PML width around Omega_int                   */
  double h;               /* mesh size; (x1-x0+2 kappa_g)/h and (y1-y0+2
                             kappa_g)/h must be whole numbers (to 1e-9 rel)    */
  int    px, py;          /* subdomain grid over Omega (the non-overlapping
                             Cartesian partition of Section 2)                 */
  int    ovlp_cells;      /* overlap delta as a per-side extension in cells;
                             -1: 0.5*ln(k)/k rounded half up, at least 1       */
  int    pml_cells;       /* local PML width kappa in cells; -1: same law;
                             0: no local PML (RAS-Imp)                         */
  double g_amp, g_ramp;   /* stretching (g_profile 0): g'(d) = g_amp*(3t^2-2t^3),
                             t = min(d/g_ramp, 1), d = distance beyond the box  */
  int    local_bc;        /* 0: impedance closure (RAS-PML-Imp, Section 3 (ii));
                             1: Dirichlet closure (RAS-PML-Drch, Section 2)    */
  int    factor_prec;     /* local factors and solves: 0 complex128,
                             1 complex64, 2 complex64 arithmetic with the L
                             entries stored as pairs of IEEE halves (4 bytes);
                             the outer iteration stays complex128              */
  int    ortho;           /* Arnoldi orthogonalisation, all in complex128:
                             0 classical Gram-Schmidt applied twice;
                             1 classical Gram-Schmidt once, repeated only when
                             ||w'|| < ||w||/sqrt(2) (the DGKS test);
                             2 classical Gram-Schmidt once;
                             3 classical Gram-Schmidt once with the basis kept in
                               complex128 and its products and sums in
                               double-float arithmetic (two floats, about 46
                               bits) on the FP32 pipe;
                             4 as 3 with the basis vectors stored as their
                               complex64 roundings (8 bytes per entry; the
                               projections use those values exactly; the
                               rounding perturbs the Arnoldi relation by
                               ~1e-7 relative, which the true-residual check
                               at the end of each cycle catches).
                             With 3 and 4 the Arnoldi products w = A z_j are
                             double-float too (coefficients split once at
                             set-up); the true residual stays complex128.     */
  int    g_profile;       /* stretching: 0 g'(d) as above; 1 g(d) = g_amp d^3,
                             i.e. g'(d) = 3 g_amp d^2 (the paper's experiments
                             use g_amp = 10k, Section 4); g_ramp unused        */
  int    form;            /* bilinear form (Section 1, eq. weak):
                             0 eq. weak multiplied by gamma_1 gamma_2, complex
                               symmetric; local factors L D L^T (default);
                             1 eq. weak as printed, int (D grad u).grad v
                               - (beta.grad u) v - k^2 u v with D_ii =
                               gamma_i^-2, beta_i = gamma_i'/gamma_i^3: not
                               symmetric; local factors L D U without pivoting,
                               impedance closure -i k int gamma_n^-1 u v ds
                               (gamma_n: the stretch normal to the edge).
                               Needs ortho 0..2 and a local half-bandwidth of
                               at most 112 (factor_prec 0) or 160 (1 and 2);
                               not accepted by ras_pml_batch_setup.
                             Both discretise the same problem; their solutions
                             differ by the discretisation error.              */
} ras_pml_params;

/* Sizes and statistics of a handle (filled by ras_pml_info). */
typedef struct {
  int64_t n;              /* global unknowns, (Mx-1)*(My-1)                     */
  int32_t Mx, My;         /* cells per direction                                */
  int32_t num_sub;        /* px*py                                              */
  int32_t ovlp_cells, pml_cells;   /* resolved widths                           */
  int32_t max_local_n;    /* largest local unknown count                        */
  int32_t max_band;       /* largest local half-bandwidth b = nlx+1             */
  int64_t sum_local_n;    /* sum_j n_j                                          */
  int64_t sum_band_n;     /* sum_j b_j*n_j: entries of all L factors            */
  int64_t factor_bytes;   /* device bytes of the stored factors (L and D^-1)    */
  double  apply_bytes;    /* algorithmic bytes of one ras_pml_apply             */
  double  min_pivot_ratio;/* min_j min_k |d_k| / max_k |d_k| after factor       */
  int32_t factored;       /* 1 once ras_pml_factor succeeded                    */
  int32_t factor_prec;
  int32_t bad_subdomain;  /* subdomain of a RASPML_EPIVOT, else -1              */
  int32_t last_iters;     /* iterations of the last solve                       */
} ras_pml_info_t;

typedef struct ras_pml_handle ras_pml_handle;

/* Builds the mesh, the covering of Section 2 and the global matrix of
 * eq. weak on the current device, on `cuda_stream` (a cudaStream_t, may be
 * NULL for the legacy default stream). Validates params (RASPML_EBADARG when
 * Omega is not whole cells, 2*ovlp exceeds a box, or a local half-bandwidth nlx+1 exceeds
 * 160 for factor_prec 0 or 232 for factor_prec 1 and 2; with form 1, 112 and 160).
 * On success *out owns all device memory of the handle. */
int ras_pml_setup(const ras_pml_params* params, void* cuda_stream,
                  ras_pml_handle** out);

/* Fills *info (host struct). */
int ras_pml_info(const ras_pml_handle* h, ras_pml_info_t* info);

/* *n = number of global unknowns, (Mx-1)*(My-1): the interior nodes of the
 * mesh of Omega (Section 1, u in H^1_0), x fastest; the length of every
 * _dev vector of the handle. Host-only; RASPML_EBADARG on NULL arguments. */
int ras_pml_num_unknowns(const ras_pml_handle* h, int64_t* n);

/* Load vector F_i = int f phi_i (Section 1) of
 *   f(x) = sum_s amps[s] * exp(-|x - c_s|^2 / width^2) cut to Omega_int,
 * with c_s = (centres[2s], centres[2s+1]); centres and amps are host arrays of
 * ns entries (ns >= 0). Writes n complex values to b_dev. */
int ras_pml_assemble_rhs(ras_pml_handle* h, const double* centres_host,
                         const double* amps_host, int ns, double width,
                         rp_c128* b_dev);

/* ras_pml_assemble_rhs without any device allocation. The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc or
 * cudaFree at this point, e.g. applications whose caching allocator has
 * already reserved the device's memory (so cudaMalloc fails), or loops that
 * must not stall on the device-wide synchronisation cudaFree implies.
 * ras_pml_assemble_rhs allocates and frees a small device table of the
 * sources on every call; this variant copies the sources into a fixed
 * device array of the library instead (24 KB per device, held until the
 * process exits) and then runs the same kernel, so b_dev is identical.
 *   - At most 1024 sources; larger ns returns RASPML_EBADARG with a message.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any
 *     stream capture.
 *   - All calls on a device share the array, and each call overwrites the
 *     entries it uses (nothing needs clearing). Calls whose work overlaps on
 *     the GPU (different streams, not ordered) race on it.
 *   - Returns after enqueueing on the handle's stream. Pageable host arrays
 *     may be reused on return; pinned ones only after the stream has run
 *     the copy. */
int ras_pml_assemble_rhs_noalloc(ras_pml_handle* h, const double* centres_host,
                                 const double* amps_host, int ns, double width,
                                 rp_c128* b_dev);

/* Assembles every local operator A_j (Section 2; impedance term of
 * Section 3 (ii) when local_bc = 0) and factors it as A_j = L_j D_j L_j^T
 * (no pivoting; A_j is complex symmetric) in the handle's factor precision;
 * with form 1 as A_j = L_j D_j U_j (no pivoting, one CUDA-core shape).
 * Returns RASPML_EPIVOT if a pivot is zero or non-finite (see info.bad_subdomain),
 * RASPML_ETIMEOUT if the tensor-core form's bounded wait for its MMAs gave up.
 * Synchronises the stream. */
int ras_pml_factor(ras_pml_handle* h);

/* z = B^-1 r = sum_j R_j^T ( chi_j .* A_j^-1 (R_j r) )  (Section 2).
 * r_dev, z_dev: n complex128 on device; they must not overlap.
 * RASPML_ESTATE if not factored. */
int ras_pml_apply(ras_pml_handle* h, const rp_c128* r_dev, rp_c128* z_dev);

/* y = A x with the global matrix of eq. weak; x_dev, y_dev n complex128,
 * must not overlap. */
int ras_pml_matvec(ras_pml_handle* h, const rp_c128* x_dev, rp_c128* y_dev);

/* Flexible GMRES (Section 4.1) with B^-1 as right preconditioner, in
 * complex128 (Arnoldi by classical Gram-Schmidt applied twice, complex Givens
 * rotations), on the device. x_dev holds x0 on entry and the solution on exit.
 * Stops when the residual estimate ||b-Ax||/||b|| <= rtol or after maxit
 * preconditioned directions (restart = 0: no restart; else the Krylov space
 * is rebuilt every `restart` directions). The Krylov space takes
 * (2m+1)*n*16 bytes for a cycle of m directions; if that does not fit in
 * the free device memory, the cycle is shortened to what fits. rtol = 0 runs exactly maxit
 * directions. *iters gets the number of directions, *relres the final true
 * relative residual ||b - A x||_2 / ||b||_2 (computed in complex128).
 * Factors first if needed. Returns 0, RASPML_NOT_CONVERGED, or an error. */
int helmholtz_solve(ras_pml_handle* h, const rp_c128* b_dev, rp_c128* x_dev,
                    double rtol, int maxit, int restart,
                    int* iters, double* relres);

/* helmholtz_solve on host buffers: copies b_host (and x0 from x_host) to the
 * device, solves, and copies the solution back into x_host. */
int helmholtz_solve_host(ras_pml_handle* h, const rp_c128* b_host, rp_c128* x_host,
                         double rtol, int maxit, int restart,
                         int* iters, double* relres);

/* Algorithm 1 (discrete form): u <- u + B^-1 (b - A u) until
 * ||b - A u||/||b|| <= rtol or maxit sweeps. x_dev: u0 in, u out. */
int ras_pml_richardson(ras_pml_handle* h, const rp_c128* b_dev, rp_c128* x_dev,
                       double rtol, int maxit, int* iters, double* relres);

/* Copies up to `cap` entries of the last solve's residual-estimate history
 * (relative to ||b||; entry 0 is the initial residual) to hist_host and
 * returns the count through *count. */
int ras_pml_history(const ras_pml_handle* h, double* hist_host, int cap, int* count);

/* Device-time breakdown of the last ras_pml_factor / helmholtz_solve, from
 * CUDA events recorded on the handle's stream (recorded only while timing is
 * enabled with ras_pml_set_timing; disabled by default). */
typedef struct {
  double factor_ms;       /* local assembly + factorisation (L D L^T; L D U with form 1) */
  double solve_ms;        /* whole helmholtz_solve, first launch to last       */
  double apply_ms;        /* sum over the solve's applies of B^-1              */
  double spmv_ms;         /* sum over the solve's A z products                 */
  double ortho_ms;        /* Gram-Schmidt, norms, Givens, normalisation        */
  int32_t applies;        /* directions (applies) the solve took               */
  int32_t reorths;        /* second Gram-Schmidt passes taken (ortho = 1)      */
  int32_t launches;       /* kernels the solve launched, including those that
                             returned at once after convergence               */
  int32_t learned_dirs;   /* directions the learned stage corrected before its
                             gate closed (0 without a network); filled whether
                             or not timing is enabled                         */
  double learned_gain;    /* largest fraction of a residual's squared norm one
                             learned correction removed                       */
} ras_pml_timing_t;

/* Enables (1) or disables (0) event timing on the handle. */
int ras_pml_set_timing(ras_pml_handle* h, int enable);

/* Fills *t (host struct) for the last factor and solve. */
int ras_pml_get_timing(const ras_pml_handle* h, ras_pml_timing_t* t);

/* Failure injection for the device-side time-out path (failure detection;
 * the paper has no counterpart). Sets, for the current
 * device and every later launch on it, the limit in SM clock cycles of the
 * apply kernels' waits for their bulk copies of factor columns; cycles <= 0
 * restores the default (2^31 cycles, about a second); cycles = 1 makes every
 * such wait give up at its first check. With a limit shorter than a copy
 * takes, a warp's wait gives up: the warp records the time-out,
 * waits for its own copies still in flight with the default limit, and
 * returns, and the solve or apply reports RASPML_ETIMEOUT; the context stays
 * usable. A later ras_pml_factor clears the recorded time-out. Not for
 * production use; -3 if the device variable cannot be written. */
int ras_pml_set_copy_wait_limit(long long cycles);

/* Throughput of the FP64 (fp64 = 1) or FP32 (fp64 = 0) fused multiply-add
 * pipes of the current device, in TFLOP/s (2 flops per FMA), from a
 * microbenchmark of independent FMA chains on every SM timed with CUDA events:
 * the ALU roofline of the kernels whose arithmetic, not memory, bounds them.
 * The paper has no counterpart. Synchronises the device; -3 on a CUDA error. */
int ras_pml_fma_peak(int fp64, double* tflops);

/* Human-readable text for a status code (static storage). */
const char* ras_pml_error_string(int status);

/* Releases every device allocation of the handle (NULL is allowed). */
void ras_pml_destroy(ras_pml_handle* h);

/* ---------------------------------------------------------------------------
 * Tile-shape tuning. Not an operation of the paper (which fixes no kernel
 * shapes): times each candidate shape of the factor launch (threads per CTA
 * and pivots per pass over the window) and of the apply launch (band columns
 * per bulk copy) on the handle's own subdomains with CUDA events, keeps the
 * fastest for later calls (the default, 256 threads x 2 pivots and 8
 * columns, unless another shape beats it by 2%), and leaves the handle
 * factored (every shape
 * computes the same factors up to the rounding order of the rank-2 update).
 * Factor candidates: 128, 256, 512 threads with one pivot per pass, 256,
 * 512 and 1024 threads with two, and, when factor_prec >= 1 and every
 * half-bandwidth is <= 127, the blocked form on the tensor cores (128
 * threads, factor_rank 8 or 16: that many pivots per panel, the trailing
 * update as TF32 MMAs with a three-term split of each FP32 operand); in
 * the batched form with factor_prec >= 1 also the tensor-core form mixed
 * with two-pivot CUDA-core shapes for the half-bandwidths above 127, and
 * factor_rank 24 (128 threads): those half-bandwidths (up to the
 * shared-memory window's limit) on the blocked tensor-core kernel of the
 * wide bands, window in device scratch, the rest with 16 pivots per panel;
 * apply
 * columns 8, plus 4 and 16 when factor_prec = 1; where subdomains are wider
 * than the shared-memory window, the wide-band factor's shape: 1, 2 or 4
 * CTAs per subdomain on the CUDA cores, or (factor_prec >= 1) 16, the
 * trailing update on the tensor cores (kept: the automatic choice, the
 * largest cluster for which all wide subdomains' clusters are resident at
 * once, unless another shape beats it by 2%).
 * Synchronises the stream. With form 1 it factors once and times nothing
 * (one factor shape; the apply shape stays as set; n_factor = n_apply = 0).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t factor_threads;    /* chosen threads per factor CTA                 */
  int32_t factor_rank;       /* chosen pivots per pass (1, 2; 8, 16: tensor cores;
                                24: blocked tensor-core form, batched) */
  int32_t apply_cols;        /* chosen band columns per bulk copy             */
  int32_t n_factor;          /* factor candidates timed (entries below)       */
  int32_t n_apply;           /* apply candidates timed                        */
  int32_t factor_cand_threads[10];
  int32_t factor_cand_rank[10];
  float   factor_ms[10];     /* median time of each factor candidate          */
  int32_t apply_cand[4];
  float   apply_ms[4];       /* median time of each apply candidate (local
                                solves of all subdomains)                     */
  int32_t wide_cluster;      /* wide-band factor shape in use: 1, 2, 4 CTAs
                                per subdomain, 16 tensor cores (0: no wide
                                subdomain)                                    */
  int32_t n_wide;            /* wide shapes timed (entries below; 0 when no
                                subdomain is wider than the shared-memory
                                window)                                       */
  int32_t wide_cand[4];
  float   wide_ms[4];        /* time of the wide-band factor's launch        */
} ras_pml_tune_t;

int ras_pml_tune(ras_pml_handle* h, ras_pml_tune_t* report);

/* Sets the tile shapes directly (e.g. those a tuning run chose for another
 * handle of the same sizes): factor_threads 128, 256 or 512 with
 * factor_rank 1 or 2, 1024 with factor_rank 2, or 128 with factor_rank 8
 * or 16 (the tensor-core form: factor_prec >= 1 and every half-bandwidth
 * <= 127; in the batched form also 256, 512 or 1024 threads, mixed with
 * the CUDA-core kernel for half-bandwidths above 127, or 128 threads with
 * factor_rank 24, the blocked tensor-core kernel for those);
 * apply_cols 8, or 4 or 16 with factor_prec = 1; wide_cluster 1, 2 or 4
 * CTAs per subdomain of the wide-band factor on the CUDA cores, 16 for its
 * tensor-core form (factor_prec >= 1), or 0 for the automatic choice.
 * RASPML_EBADARG for other values. */
int ras_pml_set_shapes(ras_pml_handle* h, int factor_threads, int factor_rank, int apply_cols, int wide_cluster);

/* ---------------------------------------------------------------------------
 * Batched form: many independent problems in the same launches. The paper
 * solves one problem at a time; a batch holds nprob problems, each defined
 * by its own ras_pml_params exactly as ras_pml_setup would define it, and
 * runs every step of the method over all of them at once:
 *   - one local-assembly and one factor launch over the union of all
 *     subdomains (ordered by decreasing factor cost, so that the largest
 *     start first and the uneven sizes pack onto the SMs);
 *   - one local-solve launch and one prolongation launch per application
 *     of the preconditioners;
 *   - flexible GMRES run in lockstep: direction j of every unfinished
 *     problem in the same launches, each problem with its own Krylov
 *     space, Hessenberg matrix, rotations, residual estimate and stop
 *     flag; a finished problem's share of each launch returns at once.
 *     One Arnoldi step is a CUDA graph (its kernels read the step index
 *     from device memory) captured once and replayed for every step.
 * Vectors of a batch are concatenations: problem q occupies elements
 * [off_q, off_q + n_q) of a complex128 vector of ntot elements
 * (ras_pml_batch_layout); off_q is a multiple of 2048. Elements between
 * problems are ignored on input and written as zero on output.
 * All problems must share factor_prec; ortho is ignored (the Gram-Schmidt of
 * the batch is one classical pass in double-float arithmetic on a complex64
 * basis, as ortho = 4).
 * ------------------------------------------------------------------------- */
typedef struct ras_pml_batch ras_pml_batch;

typedef struct {
  int32_t nprob;
  int32_t num_sub;         /* subdomains over all problems                  */
  int64_t ntot;            /* length of a batch vector                      */
  int64_t sum_n;           /* unknowns over all problems                    */
  int64_t sum_local_n;     /* local unknowns over all subdomains            */
  int32_t max_band;
  int32_t factor_prec;
  int64_t factor_bytes;    /* device bytes of the stored factors            */
  double  apply_bytes;     /* algorithmic bytes of one batch apply          */
  double  min_pivot_ratio; /* over all subdomains                           */
  int32_t factored;
  int32_t bad_problem;     /* problem of a RASPML_EPIVOT subdomain, else -1 */
  int32_t bad_subdomain;   /* its subdomain index within that problem       */
  int32_t factor_threads;  /* tile shapes in use                            */
  int32_t factor_rank;
  int32_t apply_cols;
  int32_t steps;           /* lockstep Arnoldi steps of the last solve      */
  int32_t cycles;          /* restart cycles of the last solve              */
  int32_t kcap;            /* Krylov directions per cycle of the last solve */
} ras_pml_batch_info_t;

/* Builds every problem (params[q], q < nprob; RASPML_EBADARG if one is
 * invalid, as ras_pml_setup, or has form != 0) on the current device and
 * stream. */
int ras_pml_batch_setup(const ras_pml_params* params, int nprob, void* cuda_stream,
                        ras_pml_batch** out);

int ras_pml_batch_info(const ras_pml_batch* h, ras_pml_batch_info_t* info);

/* offsets_host[q] = off_q and sizes_host[q] = n_q for q < nprob (host arrays). */
int ras_pml_batch_layout(const ras_pml_batch* h, int64_t* offsets_host, int64_t* sizes_host);

/* Load vectors of all problems (the f of ras_pml_assemble_rhs): problem q
 * has ns_host[q] sources, taken in order from centres_host (2 doubles each)
 * and amps_host, and Gaussian width widths_host[q]. Writes ntot elements. */
int ras_pml_batch_assemble_rhs(ras_pml_batch* h, const int32_t* ns_host, const double* centres_host,
                               const double* amps_host, const double* widths_host, rp_c128* b_dev);

/* ras_pml_factor for all problems in one local-assembly and one factor
 * launch. RASPML_EPIVOT names the first failing (problem, subdomain) in info. */
int ras_pml_batch_factor(ras_pml_batch* h);

/* ras_pml_tune and ras_pml_set_shapes on the batch's subdomains. */
int ras_pml_batch_tune(ras_pml_batch* h, ras_pml_tune_t* report);
int ras_pml_batch_set_shapes(ras_pml_batch* h, int factor_threads, int factor_rank, int apply_cols,
                             int wide_cluster);

/* z = B_q^-1 r for every problem q (batch vectors, must not overlap). */
int ras_pml_batch_apply(ras_pml_batch* h, const rp_c128* r_dev, rp_c128* z_dev);

/* y = A_q x for every problem q (batch vectors, must not overlap). */
int ras_pml_batch_matvec(ras_pml_batch* h, const rp_c128* x_dev, rp_c128* y_dev);

/* helmholtz_solve for every problem, in lockstep, from x0 = 0 (x_dev is
 * overwritten). Each problem stops on its own residual estimate or after
 * maxit directions; restart = 0 keeps one cycle (shortened, as for
 * helmholtz_solve, to the Krylov space that fits in free memory, about
 * 24*m*ntot bytes, and to at most 1024 directions). iters_host[q] and relres_host[q] (host arrays) receive each
 * problem's directions and final true relative residual. Returns 0 when
 * every problem converged, RASPML_NOT_CONVERGED otherwise, or an error
 * (RASPML_ENAN if a problem's residual became non-finite). */
int ras_pml_batch_solve(ras_pml_batch* h, const rp_c128* b_dev, rp_c128* x_dev, double rtol,
                        int maxit, int restart, int32_t* iters_host, double* relres_host);

void ras_pml_batch_destroy(ras_pml_batch* h);

/* ---------------------------------------------------------------------------
 * Learned coarse correction. The paper has no learned component; this is an
 * extra stage of the flexible GMRES: after z = B^-1 r, the residual it
 * leaves, r1 = r - A z, is averaged onto an Nc x Nc coarse grid (pixel means
 * in index space, two real channels), normalised to norm Nc, mapped by a
 * 6-layer 3x3 convolutional network (channels 2-32-32-32-32-32-2, ReLU after
 * the first five, zero padding; BF16 weights and activations, FP32
 * accumulation, tensor cores), scaled back by gamma * ||R r1|| / Nc and
 * interpolated bilinearly to the fine grid, where it is added to z.
 * Parameters (FP32, ras_pml_net_param_count of them) are stored layer by
 * layer as W[co][ci][3][3] followed by b[co].
 * ------------------------------------------------------------------------- */
typedef struct ras_pml_net ras_pml_net;

/* Network for an Nc x Nc grid and batches of up to `cap` images, He-normal
 * weights from `seed`, zero biases; work on `cuda_stream`. */
int ras_pml_net_create(int Nc, int cap, uint64_t seed, void* cuda_stream, ras_pml_net** out);
int ras_pml_net_param_count(const ras_pml_net* net);
/* Host copies of all parameters (count = ras_pml_net_param_count). Setting
 * them also resets the optimiser state. */
int ras_pml_net_set_params(ras_pml_net* net, const float* params_host, int count);
int ras_pml_net_get_params(const ras_pml_net* net, float* params_host, int count);
/* y = net(x) for nimg <= cap images; x_dev and y_dev hold nimg x 2 x Nc x Nc
 * FP32 values (image, channel, row, column). */
int ras_pml_net_forward(ras_pml_net* net, const float* x_dev, float* y_dev, int nimg);
/* Loss L = (1/nimg) sum over images of mean over pixels and the two
 * channels of (net(x) - t)^2 / 2 into *loss_host, and its gradient with
 * respect to every parameter (kept on the device for
 * ras_pml_net_adam_step; copied to grad_host, in the parameter layout, when
 * that is not NULL). The backward pass: data gradients on the tensor cores
 * (transposed, tap-flipped weights; the ReLU mask applied in the epilogue),
 * weight gradients as FP32 sums over pixels. */
int ras_pml_net_loss_grad(ras_pml_net* net, const float* x_dev, const float* t_dev, int nimg,
                          double* loss_host, float* grad_host);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) with the last
 * gradients and learning rate lr. */
int ras_pml_net_adam_step(ras_pml_net* net, float lr);
/* Output scale gamma of the correction (set by ras_pml_net_train). */
int ras_pml_net_set_gamma(ras_pml_net* net, double gamma);
double ras_pml_net_get_gamma(const ras_pml_net* net);
/* Trains the network on residual/error pairs the method itself generates on
 * the handle's problem: for each of nrhs load vectors (1-8 Gaussian sources
 * of width 0.4 pi / k at random points of Omega_int, from `seed`) the
 * converged solution x* (FGMRES, rtol 1e-9) and, for every m in m_list, the
 * FGMRES iterate x_m after m directions give the pair (r_m = b - A x_m,
 * e_m = x* - x_m). Inputs restrict(r_m) Nc / ||restrict(r_m)||, targets
 * restrict(e_m) Nc / (gamma ||restrict(r_m)||) with gamma the median of
 * ||restrict(e_m)|| / ||restrict(r_m)||; then `epochs` passes of Adam (rate lr)
 * over shuffled minibatches of up to `cap` pairs. loss_hist_host receives the
 * mean loss of every epoch, *gamma_out (may be NULL) gamma. Detaches any
 * network from the handle while generating pairs. Synchronises. */
int ras_pml_net_train(ras_pml_net* net, ras_pml_handle* h, int nrhs, const int32_t* m_list, int nm, int epochs,
                      float lr, uint64_t seed, float* loss_hist_host, double* gamma_out);
void ras_pml_net_destroy(ras_pml_net* net);

/* Attaches a network as the learned stage of helmholtz_solve on this handle
 * (NULL detaches): every preconditioned direction becomes
 * z_j = z1 + alpha c, z1 = B^-1 v_j, c = c(r1) the correction of the
 * residual r1 = v_j - A z1 described above, and alpha = <A c, r1> / ||A c||^2
 * the step that minimises ||r1 - alpha A c|| (so the stage never increases
 * that residual); the flexible GMRES absorbs the nonlinearity. Costs two
 * more SpMVs and three inner products per direction. The stage is gated:
 * once it has corrected 4 directions of a solve without removing 5% of
 * ||r1||^2 in any of them, the solve stops issuing it (the host sees this one
 * batch of four directions late), so a stage that does not help costs about
 * eight directions' worth of its kernels; ras_pml_get_timing reports the
 * directions it corrected and its largest gain. The net must live as long
 * as it is attached; Nc must not exceed the unknowns per grid row or column. */
int ras_pml_attach_net(ras_pml_handle* h, ras_pml_net* net);
/* z += c(r): the learned correction of a fine residual r on the handle's
 * grid (n complex128 each, device, not overlapping). Synchronises. */
int ras_pml_net_correct(ras_pml_handle* h, ras_pml_net* net, const rp_c128* r_dev, rp_c128* z_dev);
/* The handle's parameters (ovlp_cells and pml_cells as resolved). */
int ras_pml_get_params(const ras_pml_handle* h, ras_pml_params* out);

#ifdef __cplusplus
}
#endif
#endif /* RASPML_H */
