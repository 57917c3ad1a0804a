// dw_tune.cuh -- autotuner for the block shape of the inner stencil.
//
// For a batch of lattices with nrhs right-hand sides, candidate shapes (T sites
// per block x RB right-hand sides per block) are timed on the actual link
// field with CUDA events (one warm-up and three timed launches of the
// stencil each) and the fastest is kept, in memory and in the tuning file.
#pragma once

#include <cstdio>
#include <string>

#include "dw_exec.cuh"

namespace dw {

template <int L, bool C12>
BlockShape tune_inner_shape(const std::vector<dw_lattice>& lats, int nrhs, const std::vector<const char*>& links,
                            cudaStream_t st) {
  const std::string key = tune_key(lats.data(), (int)lats.size(), nrhs, L, C12 ? 1 : 0);
  BlockShape best{0, 0};
  if (tune_lookup(key, &best)) return best;

  // candidates: 32..256 sites per block; with several right-hand sides, RB of
  // them share a block (and its link loads through L1).  32-site blocks spread
  // small lattices over more SMs, which matters most where one SM's FP64 pipe
  // (two operations per clock on GB300) would otherwise carry a whole lattice.
  std::vector<BlockShape> cand;
  for (int T : {32, 64, 128, 256})
    for (int RB = 1; RB <= nrhs && RB <= 12; ++RB)
      if (nrhs % RB == 0 && T * RB <= 256) cand.push_back(BlockShape{T, RB});

  // temporary fields: one parity spinor per system (input and output)
  size_t per = 0;
  std::vector<size_t> off;
  for (auto& l : lats) {
    off.push_back(per);
    per += (((size_t)nrhs * spin_bytes(L) * vh_of(l)) + 255) & ~(size_t)255;
  }
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, 2 * per, st) != cudaSuccess) return BlockShape{0, 0};
  cudaMemsetAsync(buf, 0, 2 * per, st);
  Profiler& pr = profiler();
  const bool was_on = pr.on, was_timing = pr.timing;
  pr.on = false;
  pr.timing = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  for (const BlockShape& c : cand) {
    Exec E;
    E.st = st;
    make_plan(E.P, lats, nrhs, c.T, c.RB);
    for (size_t i = 0; i < lats.size(); ++i) {
      SysDesc& S = E.P.B.sd[i];
      S.f[S_LLO] = gauge_slot(links[i], lats[i], L, C12 ? 1 : 0);
      S.f[S_AUX0] = arena_slot(buf + off[i], lats[i], L, nrhs, 1);
      S.f[S_AUX1] = arena_slot(buf + per + off[i], lats[i], L, nrhs, 1);
    }
    hop<L, L, C12, false>(E, 1, S_LLO, InOne<L>{S_AUX0}, EpiOut<L, C_ONE>{S_AUX1, G_ALL});
    cudaEventRecord(e0, st);
    for (int k = 0; k < 3; ++k)
      hop<L, L, C12, false>(E, 1, S_LLO, InOne<L>{S_AUX0}, EpiOut<L, C_ONE>{S_AUX1, G_ALL});
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    if (cudaGetLastError() == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, st);
  pr.on = was_on;
  pr.timing = was_timing;
  if (best.T > 0) tune_store(key, best);
  return best;
}

}  // namespace dw
