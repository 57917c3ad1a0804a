// dw_apply.cuh -- one application of D or D^dag on the caller's fields, with
// or without the FP64 grid reduction of |out|^2 per right-hand side.
//
// Full lattice: out = in - kappa * H in, one launch over both parities.
// Parity p (Schur complement, q = 1 - p):
//   tmp_q = H_qp in_p ;  out_p = in_p - kappa^2 H_pq tmp_q   (two launches).
// The dagger uses the swapped projectors (gamma_5-conjugate operator).  With
// the reduction the second launch is the solver's own reducing xpay epilogue
// (the kernel that forms w = Dhat p and |w|^2 in every CG iteration).
#pragma once

#include "dw_exec.cuh"

namespace dw {

template <int P, bool C12, bool DAG, bool RED>
void apply_launch(const Exec& E, dw_kind kind) {
  if (kind == DW_SPINOR_FULL) {
    hop<P, P, C12, DAG>(E, 2, S_LLO, InOne<P>{S_AUX0}, EpiXpay<P, P, C_MK, RED>{S_AUX2, S_AUX0, G_ALL}, FIN_STORE0);
  } else {
    const int p = kind == DW_SPINOR_EVEN ? 0 : 1;
    hop<P, P, C12, DAG>(E, 1 - p, S_LLO, InOne<P>{S_AUX0}, EpiOut<P, C_ONE>{S_AUX1, G_ALL});
    hop<P, P, C12, DAG>(E, p, S_LLO, InOne<P>{S_AUX1}, EpiXpay<P, P, C_MK2, RED>{S_AUX2, S_AUX0, G_ALL}, FIN_STORE0);
  }
}

dw_status check_op(const dw_field* U, const dw_field* in, const dw_field* out);

// Launch plan for one system: the autotuner's block shape for this lattice,
// storage and nrhs when the solver has tuned it, else the default.
void apply_plan(Plan& P, const dw_field* U, const dw_field* in);

template <bool RED>
dw_status apply_dispatch(const Exec& E, const dw_field* U, const dw_field* in, int dag) {
  const int c12 = U->compress12;
#define DW_APPLY_CASE(PP)                                                      \
  if (c12) {                                                                   \
    if (dag) apply_launch<PP, true, true, RED>(E, in->kind);                   \
    else apply_launch<PP, true, false, RED>(E, in->kind);                      \
  } else {                                                                     \
    if (dag) apply_launch<PP, false, true, RED>(E, in->kind);                  \
    else apply_launch<PP, false, false, RED>(E, in->kind);                     \
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
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

}  // namespace dw
