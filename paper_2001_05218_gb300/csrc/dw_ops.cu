// dw_ops.cu -- dw_apply, dw_apply_dag, dw_normal_apply.
#include "dw_apply.cuh"

namespace dw {

dw_status check_op(const dw_field* U, const dw_field* in, const dw_field* out) {
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

void apply_plan(Plan& P, const dw_field* U, const dw_field* in) {
  BlockShape shape{0, 0};
  tune_lookup(tune_key(&U->lat, 1, in->nrhs, U->prec, U->compress12), &shape);
  make_plan(P, &U->lat, 1, in->nrhs, shape.T, shape.RB);
  P.pair = shape.pair;
}

// One application of D (or D^dag) with temporaries from the stream-ordered pool.
static dw_status apply_one(const dw_field* U, const dw_field* in, dw_field* out, int dag, cudaStream_t st) {
  Exec E;
  E.st = st;
  apply_plan(E.P, U, in);
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
  dw_status s = apply_dispatch<false>(E, U, in, dag);
  if (tmp) cudaFreeAsync(tmp, st);
  return s;
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
