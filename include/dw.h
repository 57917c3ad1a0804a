/*
 * dw.h -- C ABI of the GB300 (sm_103a) Wilson-Dirac conjugate-gradient library.
 *
 * The problem (Korcyl & Korcyl, SoftwareX, Sec. 1 and Sec. 3.2): solve the
 * large sparse linear system whose matrix is the Dirac-Wilson operator by
 * conjugate gradient, with most of the work in a low-precision data type and
 * occasional high-precision corrections (Sec. 2).  The operator, on an
 * Lx*Ly*Lz*Lt lattice with 12 complex components per site (4 spins x 3
 * colours) and one 3x3 complex link matrix per site and direction (Fig. 1
 * caption), is
 *
 *   D(x,y) = delta_xy - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                                      + (1 + gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} ]
 *
 * = 1 - kappa*H with the hopping term H.  Space is periodic; time is
 * antiperiodic when t_antiperiodic != 0 (sign -1 on links crossing
 * t = Lt-1 -> 0).  gamma basis: chiral, gamma_k = [[0, -i sigma_k],
 * [i sigma_k, 0]] (k = 1,2,3 for mu = x,y,z), gamma_t = [[0,1],[1,0]],
 * gamma_5 = diag(1,1,-1,-1).
 *
 * Even-odd split: sites have parity (x+y+z+t) mod 2.  With H_eo (odd -> even)
 * and H_oe, the Schur complement on even sites is
 *   Dhat = 1 - kappa^2 H_eo H_oe,   Dhat^dag = gamma_5 Dhat gamma_5.
 *
 * Conventions for every call
 *   - All device work is enqueued on `stream` (a cudaStream_t; NULL = the
 *     legacy default stream) and is asynchronous, except the solvers, which
 *     synchronise `stream` before returning so that they can fill statistics.
 *   - Inputs are never modified.  On DW_ERR_ARG / DW_ERR_SHAPE /
 *     DW_ERR_PRECISION nothing is enqueued and outputs are untouched.
 *   - The library owns the memory of fields made by dw_field_alloc; memory
 *     handed to dw_field_wrap stays owned by the caller and must outlive the
 *     field handle.
 *   - dw_last_error() returns a thread-local message for the last failure.
 *   - Solver calls (dw_cg_solve*, dw_cg_backward) from several host threads
 *     are serialised within a process: they share the cache of solver plans
 *     and working memory.
 *   - Dimensions must all be even and Lx*Ly*Lz*Lt/2 must be a multiple of 8.
 *
 * Host canonical layout (complex128 as interleaved re, im doubles):
 *   site s = x + Lx*(y + Ly*(z + Lz*t))
 *   gauge         U[s][mu][row][col]                 (V*4*9 complex)
 *   full spinor   psi[rhs][s][spin][colour]          (nrhs*V*12 complex)
 *   parity spinor psi[rhs][j][spin][colour], j = the sites of that parity in
 *                 increasing s order, i.e. j = s/2  (nrhs*V/2*12 complex)
 */
#ifndef DW_H
#define DW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st* dw_stream_t;

typedef enum {
  DW_OK = 0,
  DW_ERR_ARG = 1,           /* NULL pointer, bad enum, bad parameter value */
  DW_ERR_SHAPE = 2,         /* lattice / kind / nrhs mismatch between fields */
  DW_ERR_PRECISION = 3,     /* unsupported or mismatched storage precision */
  DW_ERR_OOM = 4,           /* device allocation failed */
  DW_ERR_CUDA = 5,          /* a CUDA runtime call failed (message in dw_last_error) */
  DW_ERR_NOT_CONVERGED = 6, /* maxiter reached; x holds the last FP64 iterate */
  DW_ERR_BREAKDOWN = 7,     /* CG breakdown (p^dag A p <= 0 or not finite) */
  DW_ERR_TIMEOUT = 8        /* device-side wall-time budget exhausted */
} dw_status;

/* DW_DF64: each real stored as the unevaluated sum hi + lo of two FP32
 * numbers (about 49 significant bits) with double-float arithmetic on the
 * FP32 pipes; same size as FP64.  On GB300 the FP64 pipe runs at 1/61 of the
 * FP32 rate, so FP64-class stencils are faster this way. */
/* DW_I16: 16-bit fixed point.  Spinor components are stored as
 * round(32767 * value / max|component of the site|) with one FP32 scale per
 * site (the layout of FP16 storage); link entries, which SU(3) bounds by 1 in
 * magnitude, as round(32767 * entry).  Arithmetic in FP32.  Relative
 * resolution 2^-15 of the site's largest component, against FP16's 2^-11 of
 * each value. */
typedef enum { DW_F64 = 0, DW_F32 = 1, DW_F16 = 2, DW_BF16 = 3, DW_DF64 = 4, DW_I16 = 5 } dw_prec;

typedef enum {
  DW_GAUGE = 0,       /* links U_mu(x), all sites */
  DW_SPINOR_FULL = 1, /* spinor on all sites */
  DW_SPINOR_EVEN = 2, /* spinor on even sites only */
  DW_SPINOR_ODD = 3   /* spinor on odd sites only */
} dw_kind;

typedef struct {
  int dims[4];        /* Lx, Ly, Lz, Lt (all even) */
  int t_antiperiodic; /* 1: antiperiodic in time, 0: periodic */
  double kappa;       /* hopping parameter (read from the gauge field's lattice) */
} dw_lattice;

typedef struct dw_field dw_field; /* opaque handle */

/* ------------------------------------------------------------------ fields */

/* Device bytes a field of this shape occupies (for dw_field_wrap).
 * 16-bit spinors store 24 halves plus one FP32 scale per site; 16-bit links
 * store the link entries directly (|U_ij| <= 1).  compress12 applies to
 * gauge fields: only rows 0 and 1 are stored and row 2 is rebuilt as
 * conj(row0 x row1), valid for SU(3) links.  nrhs: right-hand sides held by
 * a spinor field, 1..64 (gauge fields: 1); others return DW_ERR_SHAPE. */
dw_status dw_field_bytes(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs,
                         size_t* bytes);

/* Allocate a field in device memory (owned by the library, freed by dw_field_free). */
dw_status dw_field_alloc(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs,
                         dw_field** out);

/* Make a field handle over caller-owned device memory of at least
 * dw_field_bytes() bytes, 256-byte aligned (e.g. a torch tensor's storage).
 * The solvers keep copies of a gauge field's links in their inner and outer
 * storage formats (FP32, FP16, double-float, ...) on the handle and refresh
 * them only when the field has changed through the library (upload, import)
 * or through dw_field_mark_modified: a caller that rewrites a wrapped gauge
 * field's memory itself must call dw_field_mark_modified before the next
 * solve, or that solve runs on the old links (and fails its FP64
 * certification, which always reads the caller's memory). */
dw_status dw_field_wrap(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs,
                        void* dev_ptr, size_t bytes, dw_field** out);

/* Declare that the field's device memory was changed outside the library
 * (e.g. a wrapped tensor written in place): derived copies of its links are
 * rebuilt, on the solver's stream, by the next call that needs them.  Cheap;
 * enqueues nothing. */
dw_status dw_field_mark_modified(dw_field* f);

/* Release a handle (and its memory if it was made by dw_field_alloc).
 * Waits for the device to finish work that may use it. */
dw_status dw_field_free(dw_field* f);

/* Copy host canonical complex128 data into the field (converted to the
 * field's storage precision and layout): host-to-device copies into a
 * staging buffer, then the layout kernel; a gauge field's derived link copies
 * (see dw_field_wrap) are refreshed by the same call.  Transfers of 64 MiB
 * and more run in up to 8 chunks: the copies go on a copy stream owned by the
 * library, the kernels on `stream`, so that the kernels of one chunk overlap
 * the copy of the next; events order the copy stream after the work already
 * on `stream` and `stream` after the copies, so the call is ordered on
 * `stream` as one copy plus kernel would be.  (Under stream capture the call
 * issues one copy and one kernel on `stream`.)  `host` may be pageable or
 * pinned; from pinned (page-locked) memory the copies are asynchronous and the
 * buffer must stay valid and unchanged until the stream reaches this point.
 * Staging buffers come from a memory pool owned by the library, which keeps up
 * to 8 GiB per device reserved between calls. */
dw_status dw_field_upload(dw_field* f, const double* host, dw_stream_t stream);

/* Copy the field back to host canonical complex128 (layout kernel into a
 * staging buffer, then device-to-host copies, chunked as in dw_field_upload).
 * Data are valid once `stream` has been synchronised. */
dw_status dw_field_download(const dw_field* f, double* host, dw_stream_t stream);

/* As upload/download, with the canonical complex128 array in device memory
 * (one layout kernel on `stream`; import also refreshes derived link copies). */
dw_status dw_field_import(dw_field* f, const double* dev_canonical, dw_stream_t stream);
dw_status dw_field_export(const dw_field* f, double* dev_canonical, dw_stream_t stream);

/* Shape of a field. Any output pointer may be NULL. */
dw_status dw_field_info(const dw_field* f, dw_lattice* lat, dw_kind* kind, dw_prec* prec, int* compress12,
                        int* nrhs);

/* --------------------------------------------------------------- operators */

/* out = D in.  in/out FULL: the operator on all sites.  in/out EVEN (ODD):
 * the Schur complement on that parity, 1 - kappa^2 H_pq H_qp.  U, in and out
 * share one storage precision (FP64: IEEE binary64 throughout; FP32: binary32;
 * FP16/BF16: 16-bit storage, 16-bit operands, FP32 accumulation; I16:
 * 16-bit fixed point with FP32 arithmetic).  kappa and the boundary
 * condition come from U's lattice.  in and out must not alias. */
dw_status dw_apply(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream);

/* out = D^dag in (same rules as dw_apply). */
dw_status dw_apply_dag(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream);

/* out = D^dag D in, or Dhat^dag Dhat in for parity fields. */
dw_status dw_normal_apply(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream);

/* out = D in (dagger == 0) or D^dag in (dagger != 0), as dw_apply, and
 * norm2[r] = |out_r|^2 for every right-hand side r, summed in FP64 by the
 * library's deterministic two-level grid reduction inside the launch that
 * writes out -- the same fused epilogue (xpay plus squared norm) that forms
 * w = Dhat p and |w|^2 in every CG iteration (the per-iteration matrix-vector
 * product and residual norm of the paper's Sec. 3.1 and Sec. 3.1.1).  The squared norm is taken of
 * the output before it is rounded to the storage precision.  norm2: host
 * array of out->nrhs doubles.  Synchronises `stream` before returning. */
dw_status dw_apply_norm(const dw_field* U, const dw_field* in, dw_field* out, int dagger, double* norm2,
                        dw_stream_t stream);

/* A second stencil on the same fields: the gauge-covariant Laplacian in
 * hopping form, M = 1 - kappa K with
 *   K(x,y) = sum_mu [ eta U_mu(x) delta_{x+mu,y} + eta U_mu(x-mu)^dag delta_{x-mu,y} ]
 * acting on every spin component alike (eta: the boundary sign).  With
 * kappa = 1/(8 + m^2), M = (-Delta_U + m^2)/(8 + m^2); M is Hermitian, and
 * positive definite for kappa < 1/8.  The paper presents its CG as a backbone
 * for other stencil operators (Sec. 1, Fig. 1 caption, Sec. 3.2); this is one.
 * out = M in (FULL) or the Schur complement 1 - kappa^2 K_pq K_qp on parity
 * fields, as dw_apply.  Storage FP64, FP32, FP16 or double-float. */
dw_status dw_laplace_apply(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream);

/* dw_apply (dagger == 0) or dw_apply_dag (dagger != 0) without allocating any
 * device memory.  The paper has no counterpart: this is for callers that
 * cannot allocate GPU memory when they call -- code sharing the GPU with a
 * framework whose caching allocator already holds nearly all of it, latency-
 * critical loops where a cudaMalloc or cudaFree would synchronise the device,
 * and code held to a fixed, planned memory budget.
 * The Schur complement's intermediate parity field goes to one fixed 32 MiB
 * array in device memory that the library reserves on every GPU that loads
 * it, until the process exits.  Limit: nrhs * Vh * (bytes per site of the
 * storage precision: 192 FP64, 96 FP32, 52 FP16/BF16/I16) <= 32 MiB; larger
 * fields return DW_ERR_SHAPE with nothing enqueued (FULL fields need no
 * scratch).  All calls on a device share the array, which keeps the last
 * call's contents; calls whose kernels can run at the same time on the GPU
 * (e.g. on two unordered streams) race on it.  The first call on each device,
 * made with that device current, looks up the array's device address; make
 * that first call before any stream capture. */
dw_status dw_apply_noalloc(const dw_field* U, const dw_field* in, dw_field* out, int dagger, dw_stream_t stream);

/* ------------------------------------------------------------------ solvers */

typedef struct {
  double tol;          /* stop when |b - D x| / |b| <= tol, recomputed in FP64 */
  int maxiter;         /* CG iteration limit */
  dw_prec inner;       /* DW_F64: plain FP64 CG.  DW_DF64: plain CG in double-float.
                          DW_F32/F16/BF16/I16: mixed-precision CG with reliable updates
                          in the `outer` precision */
  double delta;        /* reliable update when |r| < delta * |r at last update|;
                          0 = by inner precision: 0.01 for FP16/BF16 storage, 1e-3
                          for I16, 1e-4 for FP32 (the low-precision recursion drifts by about
                          unit roundoff / delta between corrections; smaller values
                          mean fewer high-precision corrections until that drift
                          starts to cost iterations) */
  int eo;              /* 1: even-odd preconditioned (Schur system on even sites) */
  int compress12;      /* inner-precision links stored as 12 reals */
  int recompute_fwd;   /* dw_cg_backward: 1 = recompute the forward solution */
  int tile;            /* sites per thread block (0 = library choice) */
  int check_every;     /* host-stepped loop only: iterations per convergence poll
                          (0 = library choice); the default loop runs on the device */
  double timeout_s;    /* device-side time budget per solve (0 = none) */
  int verify_normal;   /* 1: also compute normal_rel_resid (two more FP64 operator
                          applications); 0: normal_rel_resid = -1 */
  dw_prec outer;       /* precision of the accumulator x, the recomputed residual, the
                          source preparation and reconstruction of a mixed solve:
                          DW_F64 (IEEE) or DW_DF64.  The final residual that
                          certifies every solve is IEEE FP64 either way. */
  int defect_correction; /* 1: the two-data-type scheme of Strzodka & Goeddeke (the
                          paper's Sec. 1): after every high-precision residual the
                          low-precision CG restarts (new search direction), i.e.
                          outer defect correction with inner solves to relative
                          accuracy delta.  0: reliable updates (the search
                          direction is kept across corrections). */
} dw_solver_params;

typedef struct {
  int iters;              /* CG iterations */
  int reliable_updates;   /* FP64 residual replacements */
  double true_rel_resid;  /* |b - D x| / |b| recomputed in FP64 on all sites */
  double normal_rel_resid;/* |D^dag (b - D x)| / |D^dag b| (FP64) */
  double time_ms;         /* wall time of the solve on the stream */
  double flops;           /* model flop count (1320 per site per hop) */
  double bytes;           /* model HBM bytes */
  int status;             /* dw_status of this system */
} dw_solver_stats;

/* Fill *p with defaults: tol 1e-10, maxiter 20000, inner DW_F32, delta 0 (automatic),
 * eo 1, compress12 0, recompute_fwd 1, tile 0, check_every 0, timeout 0,
 * verify_normal 0, outer DW_F64, defect_correction 0.
 * The CG loop runs as one CUDA graph: a device-side while-loop over the
 * iteration, with the FP64 reliable update in a conditional node; the host
 * waits once per solve.  While dw_profile_start is active the loop is stepped
 * from the host instead (one poll per iteration) so that every stencil launch
 * can be timed with events; the arithmetic is identical. */
dw_status dw_solver_params_default(dw_solver_params* p);

/* Solve D x = b by CG on the normal equations D^dag D x = D^dag b (with the
 * even-odd Schur system when p->eo).  U: FP64 gauge field (18 reals).  b, x:
 * FP64 FULL spinors of equal nrhs; every right-hand side is solved.  x holds
 * the initial guess on entry; a right-hand side with b = 0 returns x = 0.
 * stats: one entry per right-hand side (may be NULL).  Returns the worst
 * status over right-hand sides. */
dw_status dw_cg_solve(const dw_field* U, const dw_field* b, dw_field* x, const dw_solver_params* p,
                      dw_solver_stats* stats, dw_stream_t stream);

/* n independent systems (lattices of any sizes, each with its own gauge
 * field and kappa) solved together: every kernel launch of the iteration
 * covers all systems.  All b[i] must have the same nrhs.  stats: n*nrhs
 * entries, system-major (may be NULL). */
dw_status dw_cg_solve_batched(int n, const dw_field* const* U, const dw_field* const* b, dw_field* const* x,
                              const dw_solver_params* p, dw_solver_stats* stats, dw_stream_t stream);

/* x = (D^dag D)^{-1} b by plain CG on the normal operator (rhs b itself), all
 * sites; used for differentiation.  Same argument rules as dw_cg_solve. */
dw_status dw_cg_solve_normal(const dw_field* U, const dw_field* b, dw_field* x, const dw_solver_params* p,
                             dw_solver_stats* stats, dw_stream_t stream);

/* M x = b for the covariant Laplacian M of dw_laplace_apply: plain CG (no
 * normal equations: M is Hermitian positive definite; kappa < 1/8 required)
 * on the even-site Schur complement, then the odd sites, with the same
 * reliable updates and the same final IEEE-FP64 residual |b - M x| / |b| as
 * dw_cg_solve.  p->eo and p->verify_normal are ignored.  Inner precision:
 * DW_F64, DW_F32 with compress12 = 0, or DW_F16 with compress12 = 1 (other
 * choices return DW_ERR_PRECISION). */
dw_status dw_cg_solve_laplace(const dw_field* U, const dw_field* b, dw_field* x, const dw_solver_params* p,
                              dw_solver_stats* stats, dw_stream_t stream);

/* Gradients of the two differentiable forms (PyTorch convention for complex
 * numbers: for a real loss L, grad z = dL/dRe z + i dL/dIm z).
 *   grad_x != NULL:  forward x = (D^dag D)^{-1} b, incoming grad_x = dL/dx.
 *                    grad_b = (D^dag D)^{-1} grad_x (a second CG solve);
 *                    grad_U = F(D x, grad_b) + F(D grad_b, x).
 *   grad_x == NULL:  S = phi^dag (D^dag D)^{-1} phi with phi = phi_or_b.
 *                    grad_b = dS/dphi = 2 X, X = (D^dag D)^{-1} phi;
 *                    grad_U = 2 F(D X, X).
 * F(Y, X)_mu(x) = kappa eta_mu(x) sum_s [ w_s X(x+mu)_s^dag + X(x)_s w'_s^dag ],
 * w = (1 - gamma_mu) Y(x), w' = (1 + gamma_mu) Y(x+mu) (eta = boundary sign).
 * su3_project != 0 replaces grad_U by its su(3) projection P(G U^dag),
 * P(M) = (M - M^dag)/2 - tr(M - M^dag)/6, the derivative along U -> exp(eps T) U.
 * x_fwd: the forward solution (x, or X for the action) or NULL to recompute it.
 * grad_b: FP64 FULL spinor; grad_U: FP64 gauge field (18 reals). */
dw_status dw_cg_backward(const dw_field* U, const dw_field* phi_or_b, const dw_field* grad_x,
                         const dw_field* x_fwd, dw_field* grad_b, dw_field* grad_U, int su3_project,
                         const dw_solver_params* p, dw_solver_stats* stats, dw_stream_t stream);

/* ----------------------------------------------------------- instrumentation */

/* Launch accounting for measurement (no counterpart in the paper, whose
 * Fig. 2 is a simulated timeline).  Between start and stop every kernel
 * executed by the library is counted (kernels inside the solver's CUDA graph
 * from the device loop counters).  With time_stencils != 0 every stencil
 * launch is also bracketed by two CUDA events on its own stream, and solvers
 * step their loop from the host (events cannot live inside conditional graph
 * nodes).  Entries aggregate the timed stencil launches by (arithmetic
 * precision / link storage): launches, summed event time, algorithmic bytes
 * (8 links per output site, each spinor touched once) and model flops (1320
 * per output site).  stop synchronises the device. */
typedef struct {
  char name[64];
  long long launches;
  double total_ms;
  double bytes;
  double flops;
} dw_profile_entry;

dw_status dw_profile_start(int time_stencils);
dw_status dw_profile_stop(dw_profile_entry* entries, int max_entries, int* n_entries, long long* launches);

/* ------------------------------------------------------------------- misc */

const char* dw_last_error(void);

/* Library version string. */
const char* dw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DW_H */
