// dw_tune.cuh -- autotuner for the block shape of the inner stencil.
//
// For a batch of lattices with nrhs right-hand sides, candidate shapes (T sites
// per block x RB right-hand sides per block) are timed on the actual link
// field with CUDA events, each on the pair of launches that forms w = Dhat p
// in every CG iteration (a plain hop, then the hop with the xpay epilogue and
// the FP64 grid reduction of |w|^2), one warm-up and three timed pairs, and
// the fastest is kept, in memory and in the tuning file.
#pragma once

#include <algorithm>
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
  // 16-bit storage, several right-hand sides: also two per thread (each link
  // loaded once for both), RB thread groups per block
  if ((L == P16 || L == PB16) && nrhs >= 2 && nrhs % 2 == 0)
    for (int T : {32, 64, 128, 256})
      for (int RB = 1; 2 * RB <= nrhs && RB <= 6; ++RB)
        if (nrhs % (2 * RB) == 0 && T * RB <= 256) {
          BlockShape b{T, RB};
          b.pair = 1;
          cand.push_back(b);
        }

  // temporary fields: three parity spinors per system (input, intermediate,
  // output) and the reduction buffers of the largest candidate plan
  size_t per = 0;
  std::vector<size_t> off;
  for (auto& l : lats) {
    off.push_back(per);
    per += (((size_t)nrhs * spin_bytes(L) * vh_of(l)) + 255) & ~(size_t)255;
  }
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  std::vector<Plan> plans(cand.size());
  size_t part_b = 0, cols_b = 0;
  for (size_t i = 0; i < cand.size(); ++i) {
    make_plan(plans[i], lats, nrhs, cand[i].T, cand[i].RB);
    part_b = std::max(part_b, al(sizeof(double) * plans[i].partials));
    cols_b = std::max(cols_b, al(sizeof(ColState) * plans[i].ncols));
  }
  const size_t red_b = part_b + cols_b + al(sizeof(Flags));
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, 3 * per + red_b, st) != cudaSuccess) return BlockShape{0, 0};
  cudaMemsetAsync(buf, 0, 3 * per + red_b, st);
  RedBuf rb;
  rb.partial = reinterpret_cast<double*>(buf + 3 * per);
  rb.cols = reinterpret_cast<ColState*>(buf + 3 * per + part_b);
  rb.flags = reinterpret_cast<Flags*>(buf + 3 * per + part_b + cols_b);
  Profiler& pr = profiler();
  const bool was_on = pr.on, was_timing = pr.timing;
  pr.on = false;
  pr.timing = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  for (size_t ci = 0; ci < cand.size(); ++ci) {
    const BlockShape& c = cand[ci];
    Exec E;
    E.st = st;
    E.P = plans[ci];
    E.P.pair = c.pair;
    E.rb = rb;
    for (size_t i = 0; i < lats.size(); ++i) {
      SysDesc& S = E.P.B.sd[i];
      S.f[S_LLO] = gauge_slot(links[i], lats[i], L, C12 ? 1 : 0);
      S.f[S_AUX0] = arena_slot(buf + off[i], lats[i], L, nrhs, 1);
      S.f[S_AUX1] = arena_slot(buf + per + off[i], lats[i], L, nrhs, 1);
      S.f[S_AUX2] = arena_slot(buf + 2 * per + off[i], lats[i], L, nrhs, 1);
    }
    auto pair = [&] {
      hop<L, L, C12, false>(E, 1, S_LLO, InOne<L>{S_AUX0}, EpiOut<L, C_ONE>{S_AUX1, G_ALL});
      hop<L, L, C12, false>(E, 0, S_LLO, InOne<L>{S_AUX1}, EpiXpay<L, L, C_MK2, true>{S_AUX2, S_AUX0, G_ALL},
                            FIN_STORE0);
    };
    pair();
    cudaEventRecord(e0, st);
    for (int k = 0; k < 3; ++k) pair();
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
