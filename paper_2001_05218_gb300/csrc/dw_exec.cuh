// dw_exec.cuh -- launch helpers shared by the operator and solver translation units.
#pragma once

#include <cstdio>
#include <string>
#include <type_traits>
#include <utility>

#include "dw_internal.h"

namespace dw {

// Launch instrumentation (dw_profile_start / dw_profile_stop): counts every
// kernel launch and brackets each stencil launch with CUDA events on its
// stream, with the launch's algorithmic bytes and model flops.
struct Profiler {
  bool on = false;      // count launches
  bool timing = false;  // also bracket stencil launches with events
  long long launches = 0;
  struct Rec {
    int cat;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  std::vector<std::string> names;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  int category(const std::string& n) {
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == n) return (int)i;
    names.push_back(n);
    return (int)names.size() - 1;
  }
  cudaEvent_t event() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
};
Profiler& profiler();
inline void count_launch() {
  Profiler& p = profiler();
  if (p.on) p.launches += 1;
}
inline const char* prec_name(int p) {
  return p == P64 ? "f64" : p == P32 ? "f32" : p == P16 ? "f16" : p == PB16 ? "bf16" : p == PI16 ? "i16" : "df64";
}

struct Exec {
  Plan P;
  RedBuf rb;
  cudaStream_t st = nullptr;
  // 1: the launches walk their grid from its end (Batch::rev).  Consecutive
  // kernels of a CG iteration alternate directions, so that each starts on
  // the sites (links, neighbour spinors, the vector just written) that its
  // predecessor touched last and that are still in L2 (measured on GB300:
  // FP16 stencils 1.8% and the 32^3x64 solve 0.9% faster; results unchanged,
  // since the block partials stay indexed by tile).
  int rev = 0;
  Batch batch() const {
    Batch b = P.B;
    b.rev = rev;
    return b;
  }
  Exec flipped() const {
    Exec e = *this;
    e.rev = 1 - rev;
    return e;
  }
  RedArgs ra(int fin) const {
    RedArgs a;
    a.partial = rb.partial;
    a.cols = rb.cols;
    a.flags = rb.flags;
    a.fin = fin;
    return a;
  }
  dim3 grid(int par_mode) const { return par_mode == 2 ? P.grid2 : P.grid1; }
};

// A solver plan kept across solves: launch plan with every field slot, the
// working arena and the instantiated CUDA graph of the CG loop.
struct SolveCacheEntry {
  std::vector<unsigned long long> key;
  Exec E;
  char* arena = nullptr;
  cudaGraphExec_t exec = nullptr;
  int body_k = 0, rel_k = 0;
  std::vector<std::pair<char*, size_t>> zero;  // ranges cleared at the start of every solve
};
// The entry with this key (moved to most recently used), or nullptr.
SolveCacheEntry* solve_cache_find(const std::vector<unsigned long long>& key);
// Inserts; evicts the least recently used entries beyond a small limit (after
// synchronising the device).  The returned pointer stays valid until the next insert.
SolveCacheEntry* solve_cache_insert(SolveCacheEntry&& e);

// The second kernel of a grid reduction: sums the partials of the kernel just
// launched (par_mode as that kernel's) per column and runs finalizer fin.
inline void finish(const Exec& E, int par_mode, int fin) {
  Profiler& pr = profiler();
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (pr.on) pr.launches += 1;
  if (pr.timing) {
    ea = pr.event();
    eb = pr.event();
    cudaEventRecord(ea, E.st);
  }
  k_finish<<<E.P.ncols, kFinishThreads, 0, E.st>>>(E.P.B, par_mode, E.ra(fin));
  if (pr.timing) {
    cudaEventRecord(eb, E.st);
    Profiler::Rec r;
    r.cat = pr.category("reduction finish");
    r.a = ea;
    r.b = eb;
    r.bytes = (double)E.P.partials * 8.0;
    r.flops = 0.0;
    pr.recs.push_back(r);
  }
}

template <int SPA, int LP, bool C12, bool DAG, int OP = OP_WILSON, class In, class Epi>
inline void hop(const Exec& E, int par_mode, int link_slot, In in, Epi epi, int fin = FIN_STORE0) {
  Profiler& pr = profiler();
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (pr.on) pr.launches += 1;
  if (pr.timing) {
    ea = pr.event();
    eb = pr.event();
    cudaEventRecord(ea, E.st);
  }
  bool launched = false;
  if constexpr ((SPA == P16 || SPA == PB16) && LP == SPA && OP == OP_WILSON && std::is_same<In, InOne<SPA>>::value) {
    if (E.P.pair && E.P.nrhs >= 2) {  // two right-hand sides per thread, each link loaded once for both
      const unsigned npar = par_mode == 2 ? 2u : 1u;
      const dim3 g(npar * E.P.B.ntot * ((E.P.nrhs + 2 * E.P.B.RB - 1) / (2 * E.P.B.RB)));
      k_hop_pair<SPA, C12, DAG, Epi><<<g, E.P.block, 0, E.st>>>(E.batch(), par_mode, link_slot, in.slot, epi, E.ra(fin));
      launched = true;
    }
  }
  if (!launched)
    k_hop<SPA, LP, C12, DAG, In, Epi, OP><<<E.grid(par_mode), E.P.block, 0, E.st>>>(E.batch(), par_mode, link_slot, in,
                                                                                    epi, E.ra(fin));
  if (pr.timing) {
    cudaEventRecord(eb, E.st);
    const int npar = par_mode == 2 ? 2 : 1;
    double bytes = 0, sites = 0;
    for (int i = 0; i < E.P.nsys; ++i) {
      const double v = (double)E.P.B.sd[i].vh * npar;
      bytes += v * 8.0 * Link<LP, C12>::kBytes + v * E.P.nrhs * (in.io_bytes() + epi.io_bytes());
      sites += v * E.P.nrhs;
    }
    char nm[64];
    snprintf(nm, sizeof nm, "%s %s/%s%s", OP == OP_LAPLACE ? "laplace" : "hop", prec_name(SPA), prec_name(LP),
             C12 ? "-c12" : "");
    Profiler::Rec r;
    r.cat = pr.category(nm);
    r.a = ea;
    r.b = eb;
    r.bytes = bytes;
    // Wilson: 8 x (12 projection + 2 x 66 mat-vec) + 7 x 24; Laplacian: 8 x 4 x 66 + 7 x 24
    r.flops = (OP == OP_LAPLACE ? 2280.0 : 1320.0) * sites;
    pr.recs.push_back(r);
  }
  if (Epi::kReduce) finish(E, par_mode, fin);
}

template <int SP>
inline void norm(const Exec& E, int par_mode, int slot, int fin) {
  count_launch();
  k_norm<SP><<<E.grid(par_mode), E.P.block, 0, E.st>>>(E.batch(), par_mode, slot, E.ra(fin));
  finish(E, par_mode, fin);
}

}  // namespace dw
