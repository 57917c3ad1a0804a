// dw_solver.cuh -- conjugate gradient on the GPU, mixed precision with FP64
// reliable updates.
//
// The paper (Sec. 2, Sec. 3.3) runs most CG iterations in a low-precision
// type and corrects "for a possible bias" in high precision now and then.
// Here the correction is the reliable update of Sleijpen & van der Vorst
// (1996): the low-precision recursion runs until its residual has fallen by
// delta since the last correction, then the FP64 accumulator absorbs the
// low-precision increment and the residual is recomputed in FP64 from the
// definition (b - A x).  With inner = FP64 the same code is plain FP64 CG
// whose residual is only recomputed at the convergence check.
//
// Three systems share the machinery (A = operator, r = b - A x tracked):
//   MODE_EO     CGNR on the even-site Schur complement Dhat = 1 - k^2 H_eo H_oe:
//               z = Dhat^dag r, w = Dhat p, alpha = |z|^2/|w|^2, beta = |z'|^2/|z|^2.
//               Source b_e + k H_eo b_o; after convergence x_o = b_o + k H_oe x_e.
//   MODE_FULL   CGNR on the full lattice (D = 1 - k H).
//   MODE_NORMAL plain CG on D^dag D x = b (z = r, w = D^dag D p, |Dp|^2 = p.Ap).
// Every CG scalar is formed on the device in FP64 by the finalizer of the
// reduction that produces it; the host only polls an "active columns" count.
#pragma once

#include <chrono>

#include "dw_exec.cuh"

namespace dw {

enum Mode { MODE_EO = 0, MODE_FULL = 1, MODE_NORMAL = 2 };

struct SolveArgs {
  int n;
  dw_field* const* U;
  const dw_field* const* b;
  dw_field* const* x;
  dw_solver_params p;
  dw_solver_stats* stats;
  cudaStream_t st;
  int mode;
};

// counts for the model flops / bytes of one solve
struct HopCount {
  double lo_sites = 0, hi_sites = 0;
};

static __global__ void k_set_deadline(ColState* cols, int n, unsigned long long budget_ns) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && budget_ns) cols[i].deadline_ns = globaltimer_ns() + budget_ns;
}

template <int L, int A, bool C12>
struct CG {
  static constexpr int kLinkHi = S_LHI;
  static constexpr int kLinkLo = S_LLO;

  // reliable update (gated by do_rel) and its finalizer
  static void reliable(const Exec& E, int mode) {
    if (mode == MODE_EO) {
      hop<P64, P64, false, false>(E, 1, kLinkHi, InSum<A>{S_X, S_XL}, EpiOut<P64, C_ONE>{S_RT, G_REL});
      hop<P64, P64, false, false>(E, 0, kLinkHi, InOne<P64>{S_RT}, EpiReliableEO<L, A>{G_REL}, FIN_RELIABLE);
    } else if (mode == MODE_FULL) {
      count_launch();
      k_fold_x<A><<<E.grid(2), E.P.block, 0, E.st>>>(E.P.B, 2, E.ra(FIN_STORE0));
      hop<P64, P64, false, false>(E, 2, kLinkHi, InOne<P64>{S_X}, EpiResidFull<L, true>{G_REL, S_RT, S_X, S_B},
                                  FIN_RELIABLE);
    } else {
      count_launch();
      k_fold_x<A><<<E.grid(2), E.P.block, 0, E.st>>>(E.P.B, 2, E.ra(FIN_STORE0));
      // t64 = D x ; r64 = b - D^dag t64
      hop<P64, P64, false, false>(E, 2, kLinkHi, InOne<P64>{S_X}, EpiXpay<P64, P64, C_MK, false>{S_AUX0, S_X, G_REL});
      hop<P64, P64, false, true>(E, 2, kLinkHi, InOne<P64>{S_AUX0},
                                 EpiResidFull<L, true>{G_REL, S_RT, S_AUX0, S_B}, FIN_RELIABLE);
    }
  }

  // z = A-side residual and its norm with finalizer fin (FIN_GAMMA0 / FIN_BETA)
  static void zstep(const Exec& E, int mode, int fin) {
    if (mode == MODE_EO) {
      hop<L, L, C12, true>(E, 1, kLinkLo, InOne<L>{S_R}, EpiOut<L, C_ONE>{S_T, G_ACTIVE});
      hop<L, L, C12, true>(E, 0, kLinkLo, InOne<L>{S_T}, EpiXpay<L, L, C_MK2, true>{S_Z, S_R, G_ACTIVE}, fin);
    } else if (mode == MODE_FULL) {
      hop<L, L, C12, true>(E, 2, kLinkLo, InOne<L>{S_R}, EpiXpay<L, L, C_MK, true>{S_Z, S_R, G_ACTIVE}, fin);
    } else {
      norm<L>(E, 2, S_R, fin);  // z aliases r
    }
  }

  static void wstep(const Exec& E, int mode) {
    if (mode == MODE_EO) {
      hop<L, L, C12, false>(E, 1, kLinkLo, InOne<L>{S_P}, EpiOut<L, C_ONE>{S_T, G_ACTIVE});
      hop<L, L, C12, false>(E, 0, kLinkLo, InOne<L>{S_T}, EpiXpay<L, L, C_MK2, true>{S_W, S_P, G_ACTIVE}, FIN_ALPHA);
    } else if (mode == MODE_FULL) {
      hop<L, L, C12, false>(E, 2, kLinkLo, InOne<L>{S_P}, EpiXpay<L, L, C_MK, true>{S_W, S_P, G_ACTIVE}, FIN_ALPHA);
    } else {
      // t = D p (|t|^2 = p^dag A p);  w = D^dag t
      hop<L, L, C12, false>(E, 2, kLinkLo, InOne<L>{S_P}, EpiXpay<L, L, C_MK, true>{S_T, S_P, G_ACTIVE}, FIN_ALPHA);
      hop<L, L, C12, true>(E, 2, kLinkLo, InOne<L>{S_T}, EpiXpay<L, L, C_MK, false>{S_W, S_T, G_ACTIVE});
    }
  }

  static void iteration(const Exec& E, int mode) {
    const int pm = mode == MODE_EO ? 0 : 2;
    wstep(E, mode);
    count_launch();
    k_update_xr<L, A><<<E.grid(pm), E.P.block, 0, E.st>>>(E.P.B, pm, E.ra(FIN_UPDATE));
    reliable(E, mode);
    zstep(E, mode, FIN_BETA);
    count_launch();
    k_update_p<L><<<E.grid(pm), E.P.block, 0, E.st>>>(E.P.B, pm, E.ra(FIN_STORE0));
  }

  static dw_status run(const SolveArgs& a);
};

// Bytes of one even-odd spinor block in each role, per system and rhs.
struct Arena {
  char* base = nullptr;
  size_t bytes = 0;
};

template <int L, int A, bool C12>
dw_status CG<L, A, C12>::run(const SolveArgs& a) {
  const int n = a.n;
  const int mode = a.mode;
  const int nrhs = a.b[0]->nrhs;
  const bool eo = mode == MODE_EO;
  const int fpar = eo ? 1 : 2;  // parities held by the inner vectors
  cudaStream_t st = a.st;

  Exec E;
  E.st = st;
  std::vector<dw_lattice> lats;
  for (int i = 0; i < n; ++i) lats.push_back(a.U[i]->lat);
  make_plan(E.P, lats, nrhs, a.p.tile);

  // ---- per-system arena layout (256-byte aligned pieces)
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  std::vector<size_t> off(n + 1, 0);
  struct Piece { int slot, prec, npar; };
  std::vector<Piece> pieces;
  if (eo) {
    pieces = {{S_BH, DW_F64, 1}, {S_RT, DW_F64, 2}, {S_XL, A, 1}, {S_R, L, 1},
              {S_P, L, 1},       {S_Z, L, 1},       {S_W, L, 1},  {S_T, L, 1}};
  } else if (mode == MODE_FULL) {
    pieces = {{S_RT, DW_F64, 2}, {S_XL, A, 2}, {S_R, L, 2}, {S_P, L, 2}, {S_Z, L, 2}, {S_W, L, 2}};
  } else {
    pieces = {{S_RT, DW_F64, 2}, {S_AUX0, DW_F64, 2}, {S_XL, A, 2}, {S_R, L, 2},
              {S_P, L, 2},       {S_W, L, 2},         {S_T, L, 2}};
  }
  size_t total = 0;
  std::vector<std::vector<size_t>> poff(n);
  for (int i = 0; i < n; ++i) {
    const long long vh = vh_of(lats[i]);
    for (auto& pc : pieces) {
      poff[i].push_back(total);
      total += al((size_t)nrhs * pc.npar * spin_bytes(pc.prec) * vh);
    }
  }
  const size_t red_bytes = al(sizeof(double) * E.P.partials) + al(sizeof(int) * kMaxSys) +
                           al(sizeof(ColState) * E.P.ncols) + al(sizeof(Flags));
  char* arena = nullptr;
  DW_CUDA(cudaMallocAsync((void**)&arena, total + red_bytes, st));
  char* rp = arena + total;
  E.rb.partial = reinterpret_cast<double*>(rp);
  rp += al(sizeof(double) * E.P.partials);
  E.rb.counter = reinterpret_cast<int*>(rp);
  rp += al(sizeof(int) * kMaxSys);
  E.rb.cols = reinterpret_cast<ColState*>(rp);
  rp += al(sizeof(ColState) * E.P.ncols);
  E.rb.flags = reinterpret_cast<Flags*>(rp);

  // ---- slots
  dw_status status = DW_OK;
  for (int i = 0; i < n && status == DW_OK; ++i) {
    SysDesc& S = E.P.B.sd[i];
    const char* lo = nullptr;
    status = derived_links(a.U[i], L, C12 ? 1 : 0, st, &lo);
    if (status != DW_OK) break;
    S.f[S_LLO] = gauge_slot(lo, lats[i], L, C12 ? 1 : 0);
    S.f[S_LHI] = gauge_slot(a.U[i]->ptr, lats[i], DW_F64, 0);
    S.f[S_B] = spinor_slot(a.b[i]);
    S.f[S_X] = spinor_slot(a.x[i]);
    for (size_t k = 0; k < pieces.size(); ++k)
      S.f[pieces[k].slot] = arena_slot(arena + poff[i][k], lats[i], pieces[k].prec, nrhs, pieces[k].npar);
    if (mode == MODE_NORMAL) S.f[S_Z] = S.f[S_R];
  }
  if (status != DW_OK) {
    cudaFreeAsync(arena, st);
    return status;
  }

  // ---- column state
  std::vector<ColState> hc(E.P.ncols);
  for (auto& c : hc) {
    memset(&c, 0, sizeof c);
    c.tol2 = a.p.tol * a.p.tol;
    c.delta2 = L == P64 ? 0.0 : a.p.delta * a.p.delta;
    c.maxiter = a.p.maxiter;
    c.active = 1;
    c.do_rel = 1;  // the first FP64 residual is a "reliable update"
    c.status = DW_ERR_NOT_CONVERGED;
  }
  Flags hf;
  hf.active = E.P.ncols;
  hf.err = 0;
  cudaEvent_t ev0, ev1;
  DW_CUDA(cudaEventCreate(&ev0));
  DW_CUDA(cudaEventCreate(&ev1));
  DW_CUDA(cudaEventRecord(ev0, st));
  DW_CUDA(cudaMemcpyAsync(E.rb.cols, hc.data(), sizeof(ColState) * hc.size(), cudaMemcpyHostToDevice, st));
  DW_CUDA(cudaMemcpyAsync(E.rb.flags, &hf, sizeof hf, cudaMemcpyHostToDevice, st));
  DW_CUDA(cudaMemsetAsync(E.rb.counter, 0, sizeof(int) * kMaxSys, st));
  if (a.p.timeout_s > 0)
    k_set_deadline<<<(E.P.ncols + 127) / 128, 128, 0, st>>>(E.rb.cols, E.P.ncols,
                                                           (unsigned long long)(a.p.timeout_s * 1e9));

  // ---- set-up
  norm<P64>(E, 2, S_B, FIN_BNORM);
  for (int i = 0; i < n; ++i) {
    const SysDesc& S = E.P.B.sd[i];
    for (auto pc : {S_XL, S_P}) {
      const size_t nb = (size_t)nrhs * fpar * (pc == S_XL ? spin_bytes(A) : spin_bytes(L)) * S.vh;
      DW_CUDA(cudaMemsetAsync(S.f[pc].p, 0, nb, st));
    }
  }
  if (eo) {
    // bh = b_e + kappa H_eo b_o
    hop<P64, P64, false, false>(E, 0, kLinkHi, InOne<P64>{S_B}, EpiXpay<P64, P64, C_PK, false>{S_BH, S_B, G_ALL});
  }
  reliable(E, mode);                 // r = b - A x in FP64, r_low = r
  zstep(E, mode, FIN_GAMMA0);        // z, gamma
  count_launch();
  k_update_p<L><<<E.grid(eo ? 0 : 2), E.P.block, 0, st>>>(E.P.B, eo ? 0 : 2, E.ra(FIN_STORE0));  // p = z
  DW_CUDA(cudaGetLastError());

  // ---- iterations: chunks of `chunk` iterations, host polls the active count
  // one chunk behind so the GPU never waits for the host.
  const int chunk = a.p.check_every > 0 ? a.p.check_every : 16;
  static Flags* hflags = nullptr;  // pinned, two slots
  if (!hflags) DW_CUDA(cudaMallocHost((void**)&hflags, 2 * sizeof(Flags)));
  cudaEvent_t evc[2];
  DW_CUDA(cudaEventCreateWithFlags(&evc[0], cudaEventDisableTiming));
  DW_CUDA(cudaEventCreateWithFlags(&evc[1], cudaEventDisableTiming));
  const long long max_chunks = (long long)a.p.maxiter / chunk + 3;
  long long k = 0;
  for (; k < max_chunks; ++k) {
    for (int it = 0; it < chunk; ++it) iteration(E, mode);
    DW_CUDA(cudaGetLastError());
    DW_CUDA(cudaMemcpyAsync(&hflags[k & 1], E.rb.flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
    DW_CUDA(cudaEventRecord(evc[k & 1], st));
    if (k >= 1) {
      DW_CUDA(cudaEventSynchronize(evc[(k - 1) & 1]));
      if (hflags[(k - 1) & 1].active == 0) break;
    }
  }
  DW_CUDA(cudaEventSynchronize(evc[k & 1]));

  // ---- finish: odd sites, true residual, normal residual
  if (eo) {
    hop<P64, P64, false, false>(E, 1, kLinkHi, InOne<P64>{S_X}, EpiXpay<P64, P64, C_PK, false>{S_X, S_B, G_ALL});
  }
  if (mode != MODE_NORMAL) {
    hop<P64, P64, false, false>(E, 2, kLinkHi, InOne<P64>{S_X}, EpiResidFull<L, false>{G_ALL, S_RT, S_X, S_B},
                                FIN_STORE0);
    hop<P64, P64, false, true>(E, 2, kLinkHi, InOne<P64>{S_RT}, EpiXpay<P64, P64, C_MK, true>{-1, S_RT, G_ALL},
                               FIN_STORE1);
    hop<P64, P64, false, true>(E, 2, kLinkHi, InOne<P64>{S_B}, EpiXpay<P64, P64, C_MK, true>{-1, S_B, G_ALL},
                               FIN_STORE2);
  } else {
    // |b - D^dag D x|^2
    hop<P64, P64, false, false>(E, 2, kLinkHi, InOne<P64>{S_X}, EpiXpay<P64, P64, C_MK, false>{S_AUX0, S_X, G_ALL});
    hop<P64, P64, false, true>(E, 2, kLinkHi, InOne<P64>{S_AUX0}, EpiResidFull<L, false>{G_ALL, S_RT, S_AUX0, S_B},
                               FIN_STORE0);
  }
  DW_CUDA(cudaEventRecord(ev1, st));
  DW_CUDA(cudaMemcpyAsync(hc.data(), E.rb.cols, sizeof(ColState) * hc.size(), cudaMemcpyDeviceToHost, st));
  cudaFreeAsync(arena, st);
  DW_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaEventDestroy(evc[0]);
  cudaEventDestroy(evc[1]);
  DW_CUDA(cudaGetLastError());

  // ---- statistics
  dw_status worst = DW_OK;
  for (int i = 0; i < n; ++i) {
    const SysDesc& S = E.P.B.sd[i];
    for (int r = 0; r < nrhs; ++r) {
      const ColState& c = hc[S.col0 + r];
      const double bn2 = c.bnorm2 > 0 ? c.bnorm2 : 1.0;
      dw_status s = (dw_status)c.status;
      const double true_rel = sqrt(c.store[0] / bn2);
      if (s == DW_OK && !(true_rel <= a.p.tol)) s = DW_ERR_NOT_CONVERGED;
      if (c.active) s = DW_ERR_NOT_CONVERGED;
      if (s != DW_OK && worst == DW_OK) worst = s;
      if (a.stats) {
        dw_solver_stats& o = a.stats[S.col0 + r];
        o.iters = c.iter;
        o.reliable_updates = c.nrel > 0 ? c.nrel - 1 : 0;
        o.true_rel_resid = true_rel;
        o.normal_rel_resid = mode == MODE_NORMAL ? true_rel : sqrt(c.store[1] / (c.store[2] > 0 ? c.store[2] : 1.0));
        o.time_ms = ms;
        const double vh = (double)S.vh;
        const double hops_lo = (mode == MODE_EO ? 4.0 : 4.0) * c.iter;  // parity-hops per iteration
        const double hops_hi = 2.0 * c.nrel + 6.0;
        o.flops = 1320.0 * vh * (hops_lo + hops_hi);
        const double lo_hop = 8.0 * link_bytes(L, C12) + 2.0 * spin_bytes(L);
        const double hi_hop = 8.0 * link_bytes(DW_F64, 0) + 2.0 * spin_bytes(DW_F64);
        o.bytes = vh * (hops_lo * lo_hop + hops_hi * hi_hop + c.iter * 12.0 * spin_bytes(L));
        o.status = s;
      }
    }
  }
  if (worst != DW_OK)
    set_error(worst, "solve ended with status %d (see per-system stats)", (int)worst);
  return worst;
}

}  // namespace dw
