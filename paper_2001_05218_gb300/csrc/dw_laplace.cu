// dw_laplace.cu -- dw_laplace_apply: the covariant Laplacian 1 - kappa K.
//
// Full lattice: out = in - kappa * K in, one launch over both parities.
// Parity p (Schur complement, q = 1 - p):
//   tmp_q = K_qp in_p ;  out_p = in_p - kappa^2 K_pq tmp_q   (two launches).
#include "dw_exec.cuh"

namespace dw {

template <int P, bool C12>
static void laplace_launch(const Exec& E, dw_kind kind) {
  if (kind == DW_SPINOR_FULL) {
    hop<P, P, C12, false, OP_LAPLACE>(E, 2, S_LLO, InOne<P>{S_AUX0},
                                      EpiXpay<P, P, C_MK, false>{S_AUX2, S_AUX0, G_ALL});
  } else {
    const int p = kind == DW_SPINOR_EVEN ? 0 : 1;
    hop<P, P, C12, false, OP_LAPLACE>(E, 1 - p, S_LLO, InOne<P>{S_AUX0}, EpiOut<P, C_ONE>{S_AUX1, G_ALL});
    hop<P, P, C12, false, OP_LAPLACE>(E, p, S_LLO, InOne<P>{S_AUX1},
                                      EpiXpay<P, P, C_MK2, false>{S_AUX2, S_AUX0, G_ALL});
  }
}

}  // namespace dw

using namespace dw;

extern "C" dw_status dw_laplace_apply(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream) {
  DW_CHECK(U && in && out, DW_ERR_ARG, "NULL field");
  DW_CHECK(U->kind == DW_GAUGE, DW_ERR_ARG, "first argument must be a gauge field");
  DW_CHECK(in->kind != DW_GAUGE && out->kind == in->kind, DW_ERR_SHAPE, "in/out must be spinors of the same kind");
  DW_CHECK(same_dims(U->lat, in->lat) && same_dims(U->lat, out->lat), DW_ERR_SHAPE, "lattice dimensions differ");
  DW_CHECK(in->nrhs == out->nrhs, DW_ERR_SHAPE, "nrhs differs (%d vs %d)", in->nrhs, out->nrhs);
  DW_CHECK(U->prec == in->prec && U->prec == out->prec, DW_ERR_PRECISION,
           "gauge and spinor fields must share one storage precision");
  DW_CHECK(in->prec == DW_F64 || in->prec == DW_F32 || in->prec == DW_F16 || in->prec == DW_DF64, DW_ERR_PRECISION,
           "the Laplacian runs in FP64, FP32, FP16 or double-float storage");
  DW_CHECK(in->ptr != out->ptr, DW_ERR_ARG, "in and out must not alias");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Exec E;
  E.st = st;
  std::vector<dw_lattice> lats(1, U->lat);
  make_plan(E.P, lats, in->nrhs, 0);
  SysDesc& S = E.P.B.sd[0];
  S.f[S_LLO] = gauge_slot(U->ptr, U->lat, U->prec, U->compress12);
  S.f[S_AUX0] = spinor_slot(in);
  S.f[S_AUX2] = spinor_slot(out);
  char* tmp = nullptr;
  if (in->kind != DW_SPINOR_FULL) {
    const size_t nb = (size_t)in->nrhs * spin_bytes(in->prec) * vh_of(in->lat);
    DW_CUDA(cudaMallocAsync((void**)&tmp, nb, st));
    S.f[S_AUX1] = arena_slot(tmp, in->lat, in->prec, in->nrhs, 1);
  }
  const bool c12 = U->compress12 != 0;
  switch (in->prec) {
    case DW_F64: c12 ? laplace_launch<P64, true>(E, in->kind) : laplace_launch<P64, false>(E, in->kind); break;
    case DW_F32: c12 ? laplace_launch<P32, true>(E, in->kind) : laplace_launch<P32, false>(E, in->kind); break;
    case DW_F16: c12 ? laplace_launch<P16, true>(E, in->kind) : laplace_launch<P16, false>(E, in->kind); break;
    case DW_DF64: c12 ? laplace_launch<PDF, true>(E, in->kind) : laplace_launch<PDF, false>(E, in->kind); break;
    default: break;
  }
  cudaError_t e = cudaGetLastError();
  if (tmp) cudaFreeAsync(tmp, st);
  DW_CUDA(e);
  return DW_OK;
}
