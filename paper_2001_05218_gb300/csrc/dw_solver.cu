// dw_solver.cu -- C ABI of the solvers: argument checks and precision dispatch.
#include <mutex>

#include "dw_solver.cuh"

namespace dw {

#define DW_CG_EXTERN(L, A, C, H) extern template struct CG<L, A, C, H>;
DW_CG_EXTERN(P64, P64, false, P64)
DW_CG_EXTERN(PDF, PDF, false, PDF)
DW_CG_EXTERN(P32, P32, false, P64)
DW_CG_EXTERN(P32, P32, true, P64)
DW_CG_EXTERN(P16, P32, false, P64)
DW_CG_EXTERN(P16, P32, true, P64)
DW_CG_EXTERN(PB16, P32, false, P64)
DW_CG_EXTERN(PB16, P32, true, P64)
DW_CG_EXTERN(P32, P32, false, PDF)
DW_CG_EXTERN(P32, P32, true, PDF)
DW_CG_EXTERN(P16, P32, false, PDF)
DW_CG_EXTERN(P16, P32, true, PDF)
DW_CG_EXTERN(PB16, P32, false, PDF)
DW_CG_EXTERN(PB16, P32, true, PDF)
DW_CG_EXTERN(PI16, P32, false, P64)
DW_CG_EXTERN(PI16, P32, true, P64)
DW_CG_EXTERN(PI16, P32, false, PDF)
DW_CG_EXTERN(PI16, P32, true, PDF)
#undef DW_CG_EXTERN
#define DW_CG_LAP_EXTERN(L, A, C, H) extern template struct CG<L, A, C, H, OP_LAPLACE>;
DW_CG_LAP_EXTERN(P64, P64, false, P64)
DW_CG_LAP_EXTERN(P32, P32, false, P64)
DW_CG_LAP_EXTERN(P32, P32, false, PDF)
DW_CG_LAP_EXTERN(P16, P32, true, P64)
DW_CG_LAP_EXTERN(P16, P32, true, PDF)
#undef DW_CG_LAP_EXTERN

// The covariant Laplacian (MODE_HERM): inner FP64, FP32 with 18-real links or
// FP16 with 12-real links.
template <int H>
static dw_status dispatch_laplace_inner(const SolveArgs& a) {
  if (a.p.inner == DW_F32 && !a.p.compress12) return CG<P32, P32, false, H, OP_LAPLACE>::run(a);
  if (a.p.inner == DW_F16 && a.p.compress12) return CG<P16, P32, true, H, OP_LAPLACE>::run(a);
  return set_error(DW_ERR_PRECISION,
                   "the Laplacian solver runs inner FP64, FP32 with 18-real links or FP16 with 12-real links");
}

template <int H>
static dw_status dispatch_inner(const SolveArgs& a) {
  const bool c = a.p.compress12 != 0;
  switch (a.p.inner) {
    case DW_F32: return c ? CG<P32, P32, true, H>::run(a) : CG<P32, P32, false, H>::run(a);
    case DW_F16: return c ? CG<P16, P32, true, H>::run(a) : CG<P16, P32, false, H>::run(a);
    case DW_BF16: return c ? CG<PB16, P32, true, H>::run(a) : CG<PB16, P32, false, H>::run(a);
    case DW_I16: return c ? CG<PI16, P32, true, H>::run(a) : CG<PI16, P32, false, H>::run(a);
    default: break;
  }
  return set_error(DW_ERR_PRECISION, "unknown inner precision %d", (int)a.p.inner);
}

static dw_status dispatch(const SolveArgs& a) {
  if (a.mode == MODE_HERM) {
    if (a.p.inner == DW_F64) return CG<P64, P64, false, P64, OP_LAPLACE>::run(a);
    return a.p.outer == DW_DF64 ? dispatch_laplace_inner<PDF>(a) : dispatch_laplace_inner<P64>(a);
  }
  if (a.p.inner == DW_F64) return CG<P64, P64, false, P64>::run(a);
  if (a.p.inner == DW_DF64) return CG<PDF, PDF, false, PDF>::run(a);
  return a.p.outer == DW_DF64 ? dispatch_inner<PDF>(a) : dispatch_inner<P64>(a);
}

static dw_status check_params(const dw_solver_params* p) {
  DW_CHECK(p != nullptr, DW_ERR_ARG, "params is NULL");
  DW_CHECK(p->tol > 0 && p->tol < 1, DW_ERR_ARG, "tol %g must lie in (0, 1)", p->tol);
  DW_CHECK(p->maxiter > 0, DW_ERR_ARG, "maxiter must be positive");
  DW_CHECK(p->inner >= DW_F64 && p->inner <= DW_I16, DW_ERR_PRECISION, "unknown inner precision");
  DW_CHECK(p->outer == DW_F64 || p->outer == DW_DF64, DW_ERR_PRECISION, "outer precision must be DW_F64 or DW_DF64");
  DW_CHECK(p->inner == DW_F64 || p->inner == DW_DF64 || (p->delta >= 0 && p->delta < 1), DW_ERR_ARG,
           "delta %g must lie in [0, 1) (0: chosen by inner precision)",
           p->delta);
  DW_CHECK(p->tile == 0 || (p->tile >= 32 && p->tile <= 256 && p->tile % 32 == 0), DW_ERR_ARG,
           "tile %d must be 0 or a multiple of 32 in [32, 256]", p->tile);
  DW_CHECK(p->check_every >= 0 && p->timeout_s >= 0, DW_ERR_ARG, "negative check_every / timeout");
  return DW_OK;
}

static dw_status check_system(const dw_field* U, const dw_field* b, const dw_field* x, int nrhs) {
  DW_CHECK(U && b && x, DW_ERR_ARG, "NULL field");
  DW_CHECK(U->kind == DW_GAUGE && U->prec == DW_F64 && !U->compress12, DW_ERR_PRECISION,
           "solvers take an FP64 18-real gauge field");
  DW_CHECK(b->kind == DW_SPINOR_FULL && x->kind == DW_SPINOR_FULL, DW_ERR_SHAPE, "b and x must be FULL spinors");
  DW_CHECK(b->prec == DW_F64 && x->prec == DW_F64, DW_ERR_PRECISION, "b and x must be FP64");
  DW_CHECK(same_dims(U->lat, b->lat) && same_dims(U->lat, x->lat), DW_ERR_SHAPE, "lattice dimensions differ");
  DW_CHECK(b->nrhs == nrhs && x->nrhs == nrhs, DW_ERR_SHAPE, "every b and x must have nrhs = %d", nrhs);
  DW_CHECK(b->ptr != x->ptr, DW_ERR_ARG, "b and x must not alias");
  return DW_OK;
}

// Solves share process-wide state (the plan cache, whose eviction frees the
// working memory of an entry, the tuning cache and the cached link copies on
// the gauge handles), so they run one at a time per process.  Recursive: the
// adjoint solver calls back into this function.
static std::recursive_mutex g_solve_mu;

dw_status solve_many(int n, const dw_field* const* U, const dw_field* const* b, dw_field* const* x,
                     const dw_solver_params* p, dw_solver_stats* stats, cudaStream_t st, int mode) {
  std::lock_guard<std::recursive_mutex> lock(g_solve_mu);
  DW_CHECK(n >= 1 && U && b && x, DW_ERR_ARG, "need n >= 1 systems and non-NULL arrays");
  DW_TRY(check_params(p));
  const int nrhs = b[0] ? b[0]->nrhs : 0;
  for (int i = 0; i < n; ++i) DW_TRY(check_system(U[i], b[i], x[i], nrhs));
  dw_status worst = DW_OK;
  for (int g = 0; g < n; g += kMaxSys) {
    SolveArgs a;
    a.n = n - g < kMaxSys ? n - g : kMaxSys;
    a.U = const_cast<dw_field* const*>(U + g);
    a.b = b + g;
    a.x = x + g;
    a.p = *p;
    if (a.p.delta <= 0.0)  // reliable-update threshold by inner precision
      a.p.delta = (a.p.inner == DW_F16 || a.p.inner == DW_BF16) ? 0.01 : a.p.inner == DW_I16 ? 1e-3 : 1e-4;
    if (mode == MODE_EO && !p->eo) mode = MODE_FULL;
    a.mode = mode;
    a.stats = stats ? stats + (size_t)g * nrhs : nullptr;
    a.st = st;
    dw_status s = dispatch(a);
    if (s != DW_OK && worst == DW_OK) worst = s;
    if (s != DW_OK && s != DW_ERR_NOT_CONVERGED && s != DW_ERR_BREAKDOWN && s != DW_ERR_TIMEOUT) return s;
  }
  return worst;
}

}  // namespace dw

using namespace dw;

extern "C" {

dw_status dw_solver_params_default(dw_solver_params* p) {
  DW_CHECK(p != nullptr, DW_ERR_ARG, "params is NULL");
  p->tol = 1e-10;
  p->maxiter = 20000;
  p->inner = DW_F32;
  p->delta = 0.0;  // automatic: 0.01 for 16-bit inner storage, 1e-4 for FP32
  p->eo = 1;
  p->compress12 = 0;
  p->recompute_fwd = 1;
  p->tile = 0;
  p->check_every = 0;
  p->timeout_s = 0;
  p->verify_normal = 0;
  p->outer = DW_F64;
  p->defect_correction = 0;
  return DW_OK;
}

dw_status dw_cg_solve(const dw_field* U, const dw_field* b, dw_field* x, const dw_solver_params* p,
                      dw_solver_stats* stats, dw_stream_t stream) {
  return solve_many(1, &U, &b, &x, p, stats, reinterpret_cast<cudaStream_t>(stream), MODE_EO);
}

dw_status dw_cg_solve_batched(int n, const dw_field* const* U, const dw_field* const* b, dw_field* const* x,
                              const dw_solver_params* p, dw_solver_stats* stats, dw_stream_t stream) {
  return solve_many(n, U, b, x, p, stats, reinterpret_cast<cudaStream_t>(stream), MODE_EO);
}

dw_status dw_cg_solve_normal(const dw_field* U, const dw_field* b, dw_field* x, const dw_solver_params* p,
                             dw_solver_stats* stats, dw_stream_t stream) {
  return solve_many(1, &U, &b, &x, p, stats, reinterpret_cast<cudaStream_t>(stream), MODE_NORMAL);
}

dw_status dw_cg_solve_laplace(const dw_field* U, const dw_field* b, dw_field* x, const dw_solver_params* p,
                              dw_solver_stats* stats, dw_stream_t stream) {
  return solve_many(1, &U, &b, &x, p, stats, reinterpret_cast<cudaStream_t>(stream), MODE_HERM);
}

}  // extern "C"
