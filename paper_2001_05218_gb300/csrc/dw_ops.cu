// dw_ops.cu -- dw_apply, dw_apply_dag, dw_normal_apply.
//
// Full lattice: out = in - kappa * H in, one launch over both parities.
// Parity p (Schur complement, q = 1 - p):
//   tmp_q = H_qp in_p ;  out_p = in_p - kappa^2 H_pq tmp_q   (two launches).
// The dagger uses the swapped projectors (gamma_5-conjugate operator).
#include "dw_exec.cuh"

namespace dw {

template <int P, bool C12, bool DAG>
static void apply_launch(const Exec& E, dw_kind kind) {
  if (kind == DW_SPINOR_FULL) {
    hop<P, P, C12, DAG>(E, 2, S_LLO, InOne<P>{S_AUX0}, EpiXpay<P, P, C_MK, false>{S_AUX2, S_AUX0, G_ALL});
  } else {
    const int p = kind == DW_SPINOR_EVEN ? 0 : 1;
    hop<P, P, C12, DAG>(E, 1 - p, S_LLO, InOne<P>{S_AUX0}, EpiOut<P, C_ONE>{S_AUX1, G_ALL});
    hop<P, P, C12, DAG>(E, p, S_LLO, InOne<P>{S_AUX1}, EpiXpay<P, P, C_MK2, false>{S_AUX2, S_AUX0, G_ALL});
  }
}

static dw_status check_op(const dw_field* U, const dw_field* in, const dw_field* out) {
  DW_CHECK(U && in && out, DW_ERR_ARG, "NULL field");
  DW_CHECK(U->kind == DW_GAUGE, DW_ERR_ARG, "first argument must be a gauge field");
  DW_CHECK(in->kind != DW_GAUGE && out->kind == in->kind, DW_ERR_SHAPE, "in/out must be spinors of the same kind");
  DW_CHECK(same_dims(U->lat, in->lat) && same_dims(U->lat, out->lat), DW_ERR_SHAPE, "lattice dimensions differ");
  DW_CHECK(in->nrhs == out->nrhs, DW_ERR_SHAPE, "nrhs differs (%d vs %d)", in->nrhs, out->nrhs);
  DW_CHECK(U->prec == in->prec && U->prec == out->prec, DW_ERR_PRECISION,
           "gauge and spinor fields must share one storage precision");
  DW_CHECK(in->ptr != out->ptr, DW_ERR_ARG, "in and out must not alias");
  return DW_OK;
}

// One application of D (or D^dag) with temporaries from the stream-ordered pool.
static dw_status apply_one(const dw_field* U, const dw_field* in, dw_field* out, int dag, cudaStream_t st) {
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
  const int c12 = U->compress12;
#define DW_APPLY_CASE(PP)                                                      \
  if (c12) {                                                                   \
    if (dag) apply_launch<PP, true, true>(E, in->kind);                        \
    else apply_launch<PP, true, false>(E, in->kind);                           \
  } else {                                                                     \
    if (dag) apply_launch<PP, false, true>(E, in->kind);                       \
    else apply_launch<PP, false, false>(E, in->kind);                          \
  }
  switch (in->prec) {
    case DW_F64: DW_APPLY_CASE(P64) break;
    case DW_F32: DW_APPLY_CASE(P32) break;
    case DW_F16: DW_APPLY_CASE(P16) break;
    case DW_BF16: DW_APPLY_CASE(PB16) break;
    case DW_DF64: DW_APPLY_CASE(PDF) break;
    case DW_I16: DW_APPLY_CASE(PI16) break;
  }
#undef DW_APPLY_CASE
  cudaError_t e = cudaGetLastError();
  if (tmp) cudaFreeAsync(tmp, st);
  DW_CUDA(e);
  return DW_OK;
}

}  // namespace dw

using namespace dw;

extern "C" {

dw_status dw_apply(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream) {
  DW_TRY(check_op(U, in, out));
  return apply_one(U, in, out, 0, reinterpret_cast<cudaStream_t>(stream));
}

dw_status dw_apply_dag(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream) {
  DW_TRY(check_op(U, in, out));
  return apply_one(U, in, out, 1, reinterpret_cast<cudaStream_t>(stream));
}

dw_status dw_normal_apply(const dw_field* U, const dw_field* in, dw_field* out, dw_stream_t stream) {
  DW_TRY(check_op(U, in, out));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  dw_field mid = *out;  // same shape as out, memory from the stream-ordered pool
  mid.derived.clear();
  mid.owned = 0;
  DW_CUDA(cudaMallocAsync((void**)&mid.ptr, out->bytes, st));
  dw_status s = apply_one(U, in, &mid, 0, st);
  if (s == DW_OK) s = apply_one(U, &mid, out, 1, st);
  cudaFreeAsync(mid.ptr, st);
  return s;
}

}  // extern "C"
