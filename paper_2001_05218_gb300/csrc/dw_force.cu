// dw_force.cu -- dw_cg_backward: adjoint solves and the link force.
//
// For -Re<Y, dD X> = Re sum_{x,mu} tr(F_mu(x)^dag dU_mu(x)) the force is
//   F_mu(x) = kappa eta_mu(x) sum_s [ w_s X(x+mu)_s^dag + X(x)_s w'_s^dag ],
//   w = (1 - gamma_mu) Y(x),  w' = (1 + gamma_mu) Y(x+mu),
// an outer product of colour vectors summed over spins (derived from the
// operator D(x,y) given for the problem of Sec. 1; the paper has no
// differentiation, this is the gradient of its CG solution).
//   S = phi^dag (D^dag D)^{-1} phi:      grad_U = 2 F(D X, X), grad_phi = 2 X
//   x = (D^dag D)^{-1} b, g = dL/dx:     grad_b = l = (D^dag D)^{-1} g,
//                                        grad_U = F(D x, l) + F(D l, x)
// Optional su(3) projection P(G U^dag), P(M) = (M - M^dag)/2 - tr(M - M^dag)/6.
#include "dw_exec.cuh"

namespace dw {

dw_status solve_many(int n, const dw_field* const* U, const dw_field* const* b, dw_field* const* x,
                     const dw_solver_params* p, dw_solver_stats* stats, cudaStream_t st, int mode);

// MU-specific part of the force at one link: accumulates into f[9].
template <int MU>
__device__ __forceinline__ void force_dir(const Cx<double> (&Yx)[12], const Cx<double> (&Xx)[12],
                                          const Cx<double> (&Yf)[12], const Cx<double> (&Xf)[12], double c,
                                          Cx<double> (&f)[9]) {
  Cx<double> h[6], w[12], wp[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) w[k] = wp[k] = cx(0.0, 0.0);
  project<MU, -1>(Yx, h);
  accumulate<MU, -1>(w, h);   // w = (1 - gamma_mu) Y(x)
  project<MU, +1>(Yf, h);
  accumulate<MU, +1>(wp, h);  // w' = (1 + gamma_mu) Y(x+mu)
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<double> t = cx(0.0, 0.0);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        t = cjmadd(Xf[3 * s + b], w[3 * s + a], t);   // w_s[a] conj(X(x+mu)_s[b])
        t = cjmadd(wp[3 * s + b], Xx[3 * s + a], t);  // X(x)_s[a] conj(w'_s[b])
      }
      f[3 * a + b] = cx(f[3 * a + b].re + c * t.re, f[3 * a + b].im + c * t.im);
    }
}

struct ForceArgs {
  SysDesc S;        // geometry + slots: AUX0 = Y1, AUX1 = X1, AUX2 = Y2, AUX3 = X2, LHI = U, B = out (gauge)
  int two_terms;
  int project;
  double coef;
};

// One thread per (parity, eo site); all four directions.
__global__ void __launch_bounds__(128) k_force(const __grid_constant__ ForceArgs A) {
  const SysDesc& S = A.S;
  const int par = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S.vh) return;
  const Coord c = coord_of(S, s, par);
  const int q = par ^ 1;
  Cx<double> Y1[12], X1[12], Y2[12], X2[12];
  Spin<P64>::load(slot_ptr(S, S_AUX0, 0, par), S.vh, s, Y1);
  Spin<P64>::load(slot_ptr(S, S_AUX1, 0, par), S.vh, s, X1);
  if (A.two_terms) {
    Spin<P64>::load(slot_ptr(S, S_AUX2, 0, par), S.vh, s, Y2);
    Spin<P64>::load(slot_ptr(S, S_AUX3, 0, par), S.vh, s, X2);
  }
  const long long lb = (long long)Link<P64, false>::kBytes * S.vh;
  char* gout = slot_wptr(S, S_B, 0, par);
  const char* ul = slot_ptr(S, S_LHI, 0, par);
#define DW_FORCE_DIR(MU)                                                             \
  {                                                                                  \
    float eta;                                                                       \
    const int nf = neighbour<MU, +1>(S, c, s, &eta);                                 \
    const double cc = A.coef * S.kappa * (double)eta;                                \
    Cx<double> f[9], Yf[12], Xf[12];                                                 \
    _Pragma("unroll") for (int k = 0; k < 9; ++k) f[k] = cx(0.0, 0.0);              \
    Spin<P64>::load(slot_ptr(S, S_AUX0, 0, q), S.vh, nf, Yf);                        \
    Spin<P64>::load(slot_ptr(S, S_AUX1, 0, q), S.vh, nf, Xf);                        \
    force_dir<MU>(Y1, X1, Yf, Xf, cc, f);                                            \
    if (A.two_terms) {                                                               \
      Spin<P64>::load(slot_ptr(S, S_AUX2, 0, q), S.vh, nf, Yf);                      \
      Spin<P64>::load(slot_ptr(S, S_AUX3, 0, q), S.vh, nf, Xf);                      \
      force_dir<MU>(Y2, X2, Yf, Xf, cc, f);                                          \
    }                                                                                \
    if (A.project) {                                                                 \
      Cx<double> u[9], m[9];                                                         \
      Link<P64, false>::load(ul + MU * lb, S.vh, s, u);                              \
      _Pragma("unroll") for (int a = 0; a < 3; ++a)                                  \
      _Pragma("unroll") for (int b = 0; b < 3; ++b) {                                \
        Cx<double> t = cx(0.0, 0.0);                                                 \
        _Pragma("unroll") for (int k = 0; k < 3; ++k) t = cjmadd(u[3 * b + k], f[3 * a + k], t); \
        m[3 * a + b] = t;                                                            \
      }                                                                              \
      const double tri = (m[0].im + m[4].im + m[8].im) * (2.0 / 6.0);                \
      _Pragma("unroll") for (int a = 0; a < 3; ++a)                                  \
      _Pragma("unroll") for (int b = 0; b < 3; ++b) {                                \
        Cx<double> v = cx(0.5 * (m[3 * a + b].re - m[3 * b + a].re),                 \
                          0.5 * (m[3 * a + b].im + m[3 * b + a].im));                \
        if (a == b) v.im -= tri;                                                     \
        f[3 * a + b] = v;                                                            \
      }                                                                              \
    }                                                                                \
    Link<P64, false>::store(gout + MU * lb, S.vh, s, f);                             \
  }
  DW_FORCE_DIR(0)
  DW_FORCE_DIR(1)
  DW_FORCE_DIR(2)
  DW_FORCE_DIR(3)
#undef DW_FORCE_DIR
}

// out = a * X (FP64 spinor blocks, n doubles)
__global__ void k_scale(const double* __restrict__ x, double* __restrict__ out, double a, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i];
}

static dw_status temp_like(const dw_field* f, cudaStream_t st, dw_field* t) {
  *t = dw_field();
  t->lat = f->lat;
  t->kind = f->kind;
  t->prec = f->prec;
  t->compress12 = f->compress12;
  t->nrhs = f->nrhs;
  t->bytes = f->bytes;
  t->owned = 0;
  t->version = 1;
  DW_CUDA(cudaMallocAsync((void**)&t->ptr, f->bytes, st));
  return DW_OK;
}

static dw_status launch_force(const dw_field* U, const dw_field* Y1, const dw_field* X1, const dw_field* Y2,
                              const dw_field* X2, double coef, int project, dw_field* G, cudaStream_t st) {
  ForceArgs A;
  geometry(A.S, U->lat, 1);
  A.S.f[S_AUX0] = spinor_slot(Y1);
  A.S.f[S_AUX1] = spinor_slot(X1);
  A.two_terms = Y2 != nullptr;
  if (Y2) {
    A.S.f[S_AUX2] = spinor_slot(Y2);
    A.S.f[S_AUX3] = spinor_slot(X2);
  }
  A.S.f[S_LHI] = gauge_slot(U->ptr, U->lat, DW_F64, 0);
  A.S.f[S_B] = gauge_slot(G->ptr, G->lat, DW_F64, 0);
  A.project = project;
  A.coef = coef;
  dim3 b(128), g((A.S.vh + 127) / 128, 2);
  count_launch();
  k_force<<<g, b, 0, st>>>(A);
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

}  // namespace dw

using namespace dw;

extern "C" dw_status dw_cg_backward(const dw_field* U, const dw_field* phi_or_b, const dw_field* grad_x,
                                    const dw_field* x_fwd, dw_field* grad_b, dw_field* grad_U, int su3_project,
                                    const dw_solver_params* p, dw_solver_stats* stats, dw_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DW_CHECK(U && phi_or_b && p, DW_ERR_ARG, "NULL argument");
  DW_CHECK(U->kind == DW_GAUGE && U->prec == DW_F64 && !U->compress12, DW_ERR_PRECISION,
           "U must be an FP64 18-real gauge field");
  auto full64 = [&](const dw_field* f) {
    return f == nullptr || (f->kind == DW_SPINOR_FULL && f->prec == DW_F64 && f->nrhs == 1 && same_dims(f->lat, U->lat));
  };
  DW_CHECK(full64(phi_or_b) && full64(grad_x) && full64(x_fwd) && full64(grad_b), DW_ERR_SHAPE,
           "spinors must be FP64 FULL fields with nrhs = 1 on U's lattice");
  DW_CHECK(grad_U == nullptr || (grad_U->kind == DW_GAUGE && grad_U->prec == DW_F64 && !grad_U->compress12 &&
                                 same_dims(grad_U->lat, U->lat)),
           DW_ERR_SHAPE, "grad_U must be an FP64 18-real gauge field on U's lattice");
  DW_CHECK(grad_b || grad_U, DW_ERR_ARG, "nothing to compute (grad_b and grad_U are NULL)");
  dw_solver_stats st2[2];
  memset(st2, 0, sizeof st2);
  dw_field X, Y, L, DL;
  DW_TRY(temp_like(phi_or_b, st, &X));
  DW_TRY(temp_like(phi_or_b, st, &Y));
  const bool have_fwd = x_fwd != nullptr && !p->recompute_fwd;
  dw_status s = DW_OK;
  // forward solution X = (D^dag D)^{-1} phi_or_b (x in the x-mode)
  if (have_fwd) {
    s = cudaMemcpyAsync(X.ptr, x_fwd->ptr, X.bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess ? DW_OK : DW_ERR_CUDA;
  } else {
    cudaMemsetAsync(X.ptr, 0, X.bytes, st);
    dw_field* xp = &X;
    s = solve_many(1, &U, &phi_or_b, &xp, p, &st2[0], st, 2 /* MODE_NORMAL */);
  }
  if (s == DW_OK) s = dw_apply(U, &X, &Y, stream);  // Y = D X
  if (s == DW_OK && grad_x == nullptr) {
    // action: grad_phi = 2 X, grad_U = 2 F(Y, X)
    if (grad_b) {
      const long long n = (long long)(X.bytes / 8);
      count_launch();
      k_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double*)X.ptr, (double*)grad_b->ptr, 2.0, n);
    }
    if (grad_U) s = launch_force(U, &Y, &X, nullptr, nullptr, 2.0, su3_project, grad_U, st);
  } else if (s == DW_OK) {
    DW_TRY(temp_like(phi_or_b, st, &L));
    DW_TRY(temp_like(phi_or_b, st, &DL));
    cudaMemsetAsync(L.ptr, 0, L.bytes, st);
    dw_field* lp = &L;
    s = solve_many(1, &U, &grad_x, &lp, p, &st2[1], st, 2 /* MODE_NORMAL */);
    if (s == DW_OK) s = dw_apply(U, &L, &DL, stream);
    if (s == DW_OK && grad_b) {
      if (cudaMemcpyAsync(grad_b->ptr, L.ptr, L.bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) s = DW_ERR_CUDA;
    }
    if (s == DW_OK && grad_U) s = launch_force(U, &Y, &L, &DL, &X, 1.0, su3_project, grad_U, st);
    cudaFreeAsync(L.ptr, st);
    cudaFreeAsync(DL.ptr, st);
  }
  cudaFreeAsync(X.ptr, st);
  cudaFreeAsync(Y.ptr, st);
  if (stats) {
    stats[0] = st2[0];
    stats[1] = st2[1];
  }
  if (s == DW_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "backward", __FILE__, __LINE__);
  }
  return s;
}
