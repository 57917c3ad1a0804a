// dw_ops_norm.cu -- dw_apply_norm: out = D in (or D^dag in) and |out|^2 per
// right-hand side from the FP64 grid reduction of the output stencil launch.
#include <vector>

#include "dw_apply.cuh"

using namespace dw;

extern "C" dw_status dw_apply_norm(const dw_field* U, const dw_field* in, dw_field* out, int dagger, double* norm2,
                                   dw_stream_t stream) {
  DW_TRY(check_op(U, in, out));
  DW_CHECK(norm2 != nullptr, DW_ERR_ARG, "norm2 is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Exec E;
  E.st = st;
  apply_plan(E.P, U, in);
  SysDesc& S = E.P.B.sd[0];
  S.f[S_LLO] = gauge_slot(U->ptr, U->lat, U->prec, U->compress12);
  S.f[S_AUX0] = spinor_slot(in);
  S.f[S_AUX2] = spinor_slot(out);
  // one pool allocation: the Schur intermediate (parity fields) and the
  // reduction buffers (partial sums, column states, flags)
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t tmp_b =
      in->kind == DW_SPINOR_FULL ? 0 : al((size_t)in->nrhs * spin_bytes(in->prec) * vh_of(in->lat));
  const size_t part_b = al(sizeof(double) * E.P.partials);
  const size_t cols_b = al(sizeof(ColState) * E.P.ncols), flags_b = al(sizeof(Flags));
  char* buf = nullptr;
  DW_CUDA(cudaMallocAsync((void**)&buf, tmp_b + part_b + cols_b + flags_b, st));
  char* p = buf;
  if (tmp_b) S.f[S_AUX1] = arena_slot(p, in->lat, in->prec, in->nrhs, 1);
  p += tmp_b;
  E.rb.partial = reinterpret_cast<double*>(p);
  p += part_b;
  E.rb.cols = reinterpret_cast<ColState*>(p);
  p += cols_b;
  E.rb.flags = reinterpret_cast<Flags*>(p);
  std::vector<ColState> hc(E.P.ncols);
  dw_status s = apply_dispatch<true>(E, U, in, dagger);
  cudaError_t e;
  if (s == DW_OK) {
    e = cudaMemcpyAsync(hc.data(), E.rb.cols, sizeof(ColState) * hc.size(), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = cuda_error(e, "cudaMemcpyAsync(norms)", __FILE__, __LINE__);
  }
  cudaFreeAsync(buf, st);
  e = cudaStreamSynchronize(st);
  if (s == DW_OK && e != cudaSuccess) s = cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
  if (s == DW_OK)
    for (int r = 0; r < in->nrhs; ++r) norm2[r] = hc[r].store[0];
  return s;
}
