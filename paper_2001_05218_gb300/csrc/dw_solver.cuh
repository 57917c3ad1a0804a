// dw_solver.cuh -- conjugate gradient on the GPU, mixed precision with
// high-precision reliable updates.
//
// The paper (Sec. 2, Sec. 3.2) runs most CG iterations in a low-precision
// type and corrects "for a possible bias" in high precision now and then.
// Here the correction is the reliable update of Sleijpen & van der Vorst
// (1996): the low-precision recursion runs until its residual has fallen by
// delta since the last correction, then the FP64 accumulator absorbs the
// low-precision increment and the residual is recomputed in FP64 from the
// definition (b - A x).  With inner = FP64 the same code is plain FP64 CG
// whose residual is only recomputed at the convergence check.
//
// The high precision H of the accumulator, the recomputed residual, the
// source preparation and the reconstruction is either IEEE FP64 or
// double-float (two FP32 numbers, ~49 bits, computed on the FP32 pipes: on
// GB300 the FP64 pipe runs at 1/61 of the FP32 rate).  The final residual
// that certifies the solve is always recomputed in IEEE FP64 from the
// caller's x, b and links.
//
// Four systems share the machinery (A = operator, r = b - A x tracked):
//   MODE_EO     CGNR on the even-site Schur complement Dhat = 1 - k^2 H_eo H_oe:
//               z = Dhat^dag r, w = Dhat p, alpha = |z|^2/|w|^2, beta = |z'|^2/|z|^2.
//               Source b_e + k H_eo b_o; after convergence x_o = b_o + k H_oe x_e.
//   MODE_FULL   CGNR on the full lattice (D = 1 - k H).
//   MODE_NORMAL plain CG on D^dag D x = b (z = r, w = D^dag D p, |Dp|^2 = p.Ap).
//   MODE_HERM   plain CG on the even-site Schur complement of a Hermitian
//               positive definite operator 1 - k K (the covariant Laplacian,
//               OP_LAPLACE): z = r, w = Mhat p, alpha = |r|^2 / Re(p.w);
//               source, reconstruction and certification as in MODE_EO.
// Every CG scalar is formed on the device in FP64 by the finalizer of the
// reduction that produces it; the host only polls an "active columns" count.
#pragma once

#include <chrono>

#include "dw_exec.cuh"
#include "dw_tune.cuh"

namespace dw {

enum Mode { MODE_EO = 0, MODE_FULL = 1, MODE_NORMAL = 2, MODE_HERM = 3 };
// modes whose CG vectors live on the even sites only
inline bool eo_mode(int mode) { return mode == MODE_EO || mode == MODE_HERM; }

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

template <int L, int A, bool C12, int H, int OP = OP_WILSON>
struct CG {
  static constexpr int kLinkHi = S_LHI;
  static constexpr int kLinkLo = S_LLO;

  // reliable update (gated by do_rel) and its finalizer
  static void reliable(const Exec& E, int mode) {
    // even-odd systems: x_e += xl_e (xl_e = 0); t_o = H_oe x_e; r_e = bh - x_e + k^2 H_eo t_o
    // (MODE_HERM: the same with the Laplacian's K)
    auto eo_reliable = [&] {
      count_launch();
      k_fold_x<L, A, H><<<E.grid(0), E.P.block, 0, E.st>>>(E.P.B, 0, E.ra(FIN_STORE0));
      // grid directions alternate: fold forwards, H_oe backwards, H_eo forwards
      // (the next stencil, z's first hop, walks backwards again)
      hop<H, H, false, false, OP>(E.flipped(), 1, kLinkHi, InOne<H>{S_X}, EpiOut<H, C_ONE>{S_RT, G_REL});
      hop<H, H, false, false, OP>(E, 0, kLinkHi, InOne<H>{S_RT}, EpiResidEO<L, H>{G_REL}, FIN_RELIABLE);
    };
    if constexpr (OP == OP_LAPLACE) {
      eo_reliable();
    } else if (mode == MODE_EO) {
      eo_reliable();
    } else if (mode == MODE_FULL) {
      count_launch();
      k_fold_x<L, A, H><<<E.grid(2), E.P.block, 0, E.st>>>(E.P.B, 2, E.ra(FIN_STORE0));
      hop<H, H, false, false, OP>(E, 2, kLinkHi, InOne<H>{S_X}, EpiResidFull<L, true, H>{G_REL, S_RT, S_X, S_B},
                              FIN_RELIABLE);
    } else {
      count_launch();
      k_fold_x<L, A, H><<<E.grid(2), E.P.block, 0, E.st>>>(E.P.B, 2, E.ra(FIN_STORE0));
      // t = D x ; r = b - D^dag t
      hop<H, H, false, false, OP>(E, 2, kLinkHi, InOne<H>{S_X}, EpiXpay<H, H, C_MK, false>{S_AUX0, S_X, G_REL});
      hop<H, H, false, true, OP>(E, 2, kLinkHi, InOne<H>{S_AUX0}, EpiResidFull<L, true, H>{G_REL, S_RT, S_AUX0, S_B},
                             FIN_RELIABLE);
    }
  }

  // z = A-side residual and its norm with finalizer fin (FIN_GAMMA0 / FIN_BETA)
  static void zstep(const Exec& E, int mode, int fin) {
    if constexpr (OP == OP_LAPLACE) {
      norm<L>(E, 0, S_R, fin);  // MODE_HERM: z aliases r
    } else if (mode == MODE_EO) {
      hop<L, L, C12, true, OP>(E.flipped(), 1, kLinkLo, InOne<L>{S_R}, EpiOut<L, C_ONE>{S_T, G_ACTIVE});
      hop<L, L, C12, true, OP>(E, 0, kLinkLo, InOne<L>{S_T}, EpiXpay<L, L, C_MK2, true>{S_Z, S_R, G_ACTIVE}, fin);
    } else if (mode == MODE_FULL) {
      hop<L, L, C12, true, OP>(E, 2, kLinkLo, InOne<L>{S_R}, EpiXpay<L, L, C_MK, true>{S_Z, S_R, G_ACTIVE}, fin);
    } else {
      norm<L>(E, 2, S_R, fin);  // z aliases r
    }
  }

  static void wstep(const Exec& E, int mode) {
    if constexpr (OP == OP_LAPLACE) {
      // MODE_HERM: w = Mhat p = p - k^2 K_eo K_oe p and p^dag w
      hop<L, L, C12, false, OP>(E, 1, kLinkLo, InOne<L>{S_P}, EpiOut<L, C_ONE>{S_T, G_ACTIVE});
      hop<L, L, C12, false, OP>(E, 0, kLinkLo, InOne<L>{S_T}, EpiXpayDot<L, L, C_MK2>{S_W, S_P, G_ACTIVE}, FIN_ALPHA);
    } else if (mode == MODE_EO) {
      hop<L, L, C12, false, OP>(E, 1, kLinkLo, InOne<L>{S_P}, EpiOut<L, C_ONE>{S_T, G_ACTIVE});
      hop<L, L, C12, false, OP>(E.flipped(), 0, kLinkLo, InOne<L>{S_T}, EpiXpay<L, L, C_MK2, true>{S_W, S_P, G_ACTIVE}, FIN_ALPHA);
    } else if (mode == MODE_FULL) {
      hop<L, L, C12, false, OP>(E, 2, kLinkLo, InOne<L>{S_P}, EpiXpay<L, L, C_MK, true>{S_W, S_P, G_ACTIVE}, FIN_ALPHA);
    } else {
      // t = D p (|t|^2 = p^dag A p);  w = D^dag t
      hop<L, L, C12, false, OP>(E, 2, kLinkLo, InOne<L>{S_P}, EpiXpay<L, L, C_MK, true>{S_T, S_P, G_ACTIVE}, FIN_ALPHA);
      hop<L, L, C12, true, OP>(E, 2, kLinkLo, InOne<L>{S_T}, EpiXpay<L, L, C_MK, false>{S_W, S_T, G_ACTIVE});
    }
  }

  static dw_status run(const SolveArgs& a);
  static dw_status build_graph(const Exec& E, int mode, cudaGraphExec_t* exec, int* body_kernels,
                               int* rel_kernels);
  static dw_status run_stepped(const Exec& E, int mode, int maxiter);
};

// Condition setters for the device-driven loop (one thread).
static __global__ void k_cond_rel(Flags* f, cudaGraphConditionalHandle h) {
  const bool run = f->rel_pending > 0;
  if (run) f->rel_runs += 1;
  cudaGraphSetConditional(h, run ? 1u : 0u);
}
static __global__ void k_cond_loop(Flags* f, cudaGraphConditionalHandle h) {
  const int loops = f->loops + 1;
  f->loops = loops;
  cudaGraphSetConditional(h, (f->active > 0 && loops < f->max_loops) ? 1u : 0u);
}

struct CaptureStreams {
  cudaStream_t a = nullptr, b = nullptr;
  CaptureStreams() {
    cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking);
  }
};

// The whole CG loop as one graph: while (active columns) { iteration with the
// reliable update in an if-node }.  Both conditions are set on the device,
// the loop is capped at maxiter + 2 passes, and every column also leaves the
// loop through its own maxiter / timeout / breakdown checks.
template <int L, int A, bool C12, int H, int OP>
dw_status CG<L, A, C12, H, OP>::build_graph(const Exec& E0, int mode, cudaGraphExec_t* exec, int* body_kernels,
                                        int* rel_kernels) {
  static thread_local CaptureStreams cs;
  const int pm = eo_mode(mode) ? 0 : 2;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  DW_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hw, hr;
  DW_CUDA(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn;
  DW_CUDA(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  DW_CUDA(cudaGraphConditionalHandleCreate(&hr, body, 0, cudaGraphCondAssignDefault));

  Exec E = E0;
  E.st = cs.a;
  // count the captured kernel nodes (and never record profiling events into
  // the graph: events cannot live inside conditional nodes)
  Profiler& pr = profiler();
  const bool was_on = pr.on, was_timing = pr.timing;
  pr.on = true;
  pr.timing = false;
  const long long c0 = pr.launches;
  long long c1 = c0, c2 = c0;
  DW_CUDA(cudaStreamBeginCaptureToGraph(cs.a, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  wstep(E, mode);
  count_launch();
  count_launch();
  k_update_r<L><<<E.grid(pm), E.P.block, 0, E.st>>>(E.P.B, pm, E.ra(FIN_UPDATE));
  finish(E, pm, FIN_UPDATE);
  k_cond_rel<<<1, 1, 0, E.st>>>(E.rb.flags, hr);
  {
    cudaStreamCaptureStatus cst;
    cudaGraph_t capg;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    DW_CUDA(cudaStreamGetCaptureInfo(cs.a, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hr;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t in;
    DW_CUDA(cudaGraphAddNode(&in, capg, deps, nullptr, ndeps, &ip));
    DW_CUDA(cudaStreamUpdateCaptureDependencies(cs.a, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    Exec R = E;
    R.st = cs.b;
    c1 = pr.launches;
    DW_CUDA(cudaStreamBeginCaptureToGraph(cs.b, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    reliable(R, mode);
    cudaGraph_t tmp;
    DW_CUDA(cudaStreamEndCapture(cs.b, &tmp));
    c2 = pr.launches;
  }
  zstep(E, mode, FIN_BETA);
  k_update_p<L, A><<<E.grid(pm), E.P.block, 0, E.st>>>(E.flipped().batch(), pm, E.ra(FIN_STORE0));
  k_cond_loop<<<1, 1, 0, E.st>>>(E.rb.flags, hw);
  count_launch();
  count_launch();
  cudaGraph_t tmp;
  DW_CUDA(cudaStreamEndCapture(cs.a, &tmp));
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    pr.on = was_on;
    pr.timing = was_timing;
    pr.launches = c0;
    return cuda_error(e, "CG graph", __FILE__, __LINE__);
  }
  *exec = ge;
  // kernel nodes per pass of the loop body and of the reliable-update branch;
  // the executed counts are added once the device counters are read back
  *body_kernels = (int)((c1 - c0) + (pr.launches - c2));
  *rel_kernels = (int)(c2 - c1);
  pr.launches = c0;
  pr.on = was_on;
  pr.timing = was_timing;
  return DW_OK;
}

// Host-stepped loop: identical kernels, the host reads the device counters
// after every update so that no launch is made without work; used while the
// launch profiler is active.
template <int L, int A, bool C12, int H, int OP>
dw_status CG<L, A, C12, H, OP>::run_stepped(const Exec& E, int mode, int maxiter) {
  static Flags* hf = nullptr;
  if (!hf) DW_CUDA(cudaMallocHost((void**)&hf, sizeof(Flags)));
  const int pm = eo_mode(mode) ? 0 : 2;
  for (int it = 0; it < maxiter + 2; ++it) {
    DW_CUDA(cudaMemcpyAsync(hf, E.rb.flags, sizeof(Flags), cudaMemcpyDeviceToHost, E.st));
    DW_CUDA(cudaStreamSynchronize(E.st));
    if (hf->active == 0) break;
    wstep(E, mode);
    count_launch();
    k_update_r<L><<<E.grid(pm), E.P.block, 0, E.st>>>(E.P.B, pm, E.ra(FIN_UPDATE));
    finish(E, pm, FIN_UPDATE);
    DW_CUDA(cudaMemcpyAsync(hf, E.rb.flags, sizeof(Flags), cudaMemcpyDeviceToHost, E.st));
    DW_CUDA(cudaStreamSynchronize(E.st));
    if (hf->rel_pending > 0) reliable(E, mode);
    if (hf->active == 0) continue;
    zstep(E, mode, FIN_BETA);
    count_launch();
    k_update_p<L, A><<<E.grid(pm), E.P.block, 0, E.st>>>(E.flipped().batch(), pm, E.ra(FIN_STORE0));
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}


template <int L, int A, bool C12, int H, int OP>
dw_status CG<L, A, C12, H, OP>::run(const SolveArgs& a) {
  const int n = a.n;
  const int mode = a.mode;
  const int nrhs = a.b[0]->nrhs;
  const bool eo = eo_mode(mode);
  const int fpar = eo ? 1 : 2;  // parities held by the inner vectors
  cudaStream_t st = a.st;

  std::vector<dw_lattice> lats;
  for (int i = 0; i < n; ++i) lats.push_back(a.U[i]->lat);

  // ---- plan, arena and graph: reused from the cache when every pointer,
  // shape and choice baked into them is the same
  std::vector<const char*> lo_links(n), hi_links(n);
  for (int i = 0; i < n; ++i) {
    DW_TRY(derived_links(a.U[i], L, C12 ? 1 : 0, st, &lo_links[i]));
    DW_TRY(derived_links(a.U[i], H, 0, st, &hi_links[i]));
  }
  std::vector<unsigned long long> key = {0xC6ull, (unsigned long long)OP, (unsigned long long)L, (unsigned long long)A,
                                         C12 ? 1ull : 0ull,
                                         (unsigned long long)H, (unsigned long long)mode, (unsigned long long)nrhs,
                                         (unsigned long long)a.p.tile, (unsigned long long)a.p.verify_normal,
                                         (unsigned long long)n};
  int dev = 0;
  cudaGetDevice(&dev);
  key.push_back((unsigned long long)dev);
  for (int i = 0; i < n; ++i) {
    unsigned long long kb;
    memcpy(&kb, &lats[i].kappa, sizeof kb);
    for (unsigned long long v :
         {(unsigned long long)(uintptr_t)a.U[i]->ptr, (unsigned long long)(uintptr_t)lo_links[i],
          (unsigned long long)(uintptr_t)hi_links[i], (unsigned long long)(uintptr_t)a.b[i]->ptr,
          (unsigned long long)(uintptr_t)a.x[i]->ptr, (unsigned long long)lats[i].dims[0],
          (unsigned long long)lats[i].dims[1], (unsigned long long)lats[i].dims[2],
          (unsigned long long)lats[i].dims[3], kb, (unsigned long long)lats[i].t_antiperiodic})
      key.push_back(v);
  }
  SolveCacheEntry* ent = solve_cache_find(key);
  if (ent == nullptr) {
    SolveCacheEntry fresh;
    fresh.key = key;
    Exec& F = fresh.E;
    BlockShape shape{a.p.tile, a.p.tile > 0 ? 1 : 0};
    if (a.p.tile <= 0) shape = tune_inner_shape<L, C12>(lats, nrhs, lo_links, st);
    make_plan(F.P, lats, nrhs, shape.T, shape.RB);
    F.P.pair = shape.pair;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    struct Piece { int slot, prec, npar; };
    std::vector<Piece> pieces;
    if (eo) {
      pieces = {{S_BH, H, 1}, {S_RT, H, 2}, {S_XL, A, 1}, {S_R, L, 1},
                {S_P, L, 1},  {S_Z, L, 1},  {S_W, L, 1},  {S_T, L, 1}};
    } else if (mode == MODE_FULL) {
      pieces = {{S_RT, H, 2}, {S_XL, A, 2}, {S_R, L, 2}, {S_P, L, 2}, {S_Z, L, 2}, {S_W, L, 2}};
    } else {
      pieces = {{S_RT, H, 2}, {S_AUX0, H, 2}, {S_XL, A, 2}, {S_R, L, 2},
                {S_P, L, 2},  {S_W, L, 2},    {S_T, L, 2}};
    }
    if (H != P64) {  // high-precision copies of the caller's x and b
      pieces.push_back({S_X, H, 2});
      pieces.push_back({S_B, H, 2});
    }
    // FP64 full temporary for the certification (the FP64 arena pieces serve when H = FP64)
    if (H != P64 && (a.p.verify_normal || mode == MODE_NORMAL)) pieces.push_back({S_AUX1, DW_F64, 2});
    size_t total = 0;
    std::vector<std::vector<size_t>> poff(n);
    for (int i = 0; i < n; ++i) {
      const long long vh = vh_of(lats[i]);
      for (auto& pc : pieces) {
        poff[i].push_back(total);
        total += al((size_t)nrhs * pc.npar * spin_bytes(pc.prec) * vh);
      }
    }
    const size_t red_bytes = al(sizeof(double) * F.P.partials) + al(sizeof(ColState) * F.P.ncols) + al(sizeof(Flags));
    DW_CUDA(cudaMalloc((void**)&fresh.arena, total + red_bytes));
    char* rp = fresh.arena + total;
    F.rb.partial = reinterpret_cast<double*>(rp);
    rp += al(sizeof(double) * F.P.partials);
    F.rb.cols = reinterpret_cast<ColState*>(rp);
    rp += al(sizeof(ColState) * F.P.ncols);
    F.rb.flags = reinterpret_cast<Flags*>(rp);
    for (int i = 0; i < n; ++i) {
      SysDesc& S = F.P.B.sd[i];
      S.f[S_LLO] = gauge_slot(lo_links[i], lats[i], L, C12 ? 1 : 0);
      S.f[S_LHI] = gauge_slot(hi_links[i], lats[i], H, 0);
      S.f[S_LF64] = gauge_slot(a.U[i]->ptr, lats[i], DW_F64, 0);
      S.f[S_BU] = spinor_slot(a.b[i]);
      S.f[S_XU] = spinor_slot(a.x[i]);
      S.f[S_B] = S.f[S_BU];
      S.f[S_X] = S.f[S_XU];
      for (size_t k = 0; k < pieces.size(); ++k)
        S.f[pieces[k].slot] = arena_slot(fresh.arena + poff[i][k], lats[i], pieces[k].prec, nrhs, pieces[k].npar);
      if (mode == MODE_NORMAL || mode == MODE_HERM) S.f[S_Z] = S.f[S_R];
      for (auto pc : {S_XL, S_P})
        fresh.zero.push_back({S.f[pc].p, (size_t)nrhs * fpar * (pc == S_XL ? spin_bytes(A) : spin_bytes(L)) * S.vh});
      // odd half of the high-precision temporary: holds H_oe x_e after every
      // reliable update and feeds the odd-site reconstruction; zero for a
      // column that converges before its first one (x_e = 0 there)
      if (eo)
        for (int r = 0; r < nrhs; ++r)
          fresh.zero.push_back({S.f[S_RT].p + r * S.f[S_RT].rhs_stride + S.f[S_RT].par_stride,
                                (size_t)spin_bytes(H) * S.vh});
    }
    F.st = st;
    dw_status gs = build_graph(F, mode, &fresh.exec, &fresh.body_k, &fresh.rel_k);
    if (gs != DW_OK) {
      cudaFree(fresh.arena);
      return gs;
    }
    ent = solve_cache_insert(std::move(fresh));
  }
  Exec E = ent->E;
  E.st = st;

  // ---- column state
  std::vector<ColState> hc(E.P.ncols);
  for (auto& c : hc) {
    memset(&c, 0, sizeof c);
    c.tol2 = a.p.tol * a.p.tol;
    c.delta2 = (L == P64 || L == PDF) ? 0.0 : a.p.delta * a.p.delta;
    c.maxiter = a.p.maxiter;
    c.defect = a.p.defect_correction ? 1 : 0;
    c.active = 1;
    c.do_rel = 1;  // the first FP64 residual is a "reliable update" unless x0 = 0
    c.status = DW_ERR_NOT_CONVERGED;
  }
  Flags hf;
  memset(&hf, 0, sizeof hf);
  hf.active = E.P.ncols;
  hf.rel_pending = E.P.ncols;
  hf.loops = 0;
  hf.max_loops = a.p.maxiter + 2;
  cudaEvent_t ev0, ev1;
  DW_CUDA(cudaEventCreate(&ev0));
  DW_CUDA(cudaEventCreate(&ev1));
  DW_CUDA(cudaEventRecord(ev0, st));
  DW_CUDA(cudaMemcpyAsync(E.rb.cols, hc.data(), sizeof(ColState) * hc.size(), cudaMemcpyHostToDevice, st));
  DW_CUDA(cudaMemcpyAsync(E.rb.flags, &hf, sizeof hf, cudaMemcpyHostToDevice, st));
  if (a.p.timeout_s > 0) {
    count_launch();
    k_set_deadline<<<(E.P.ncols + 127) / 128, 128, 0, st>>>(E.rb.cols, E.P.ncols,
                                                           (unsigned long long)(a.p.timeout_s * 1e9));
  }

  // ---- set-up
  norm<P64>(E, 2, S_BU, FIN_BNORM);
  norm<P64>(E, eo ? 0 : 2, S_XU, FIN_XNORM);
  if (H != P64) {
    count_launch();
    k_convert<H, P64><<<E.grid(2), E.P.block, 0, st>>>(E.P.B, 2, S_B, S_BU, E.ra(FIN_STORE0));
    count_launch();
    k_convert<H, P64><<<E.grid(2), E.P.block, 0, st>>>(E.P.B, 2, S_X, S_XU, E.ra(FIN_STORE0));
  }
  for (auto& z : ent->zero) DW_CUDA(cudaMemsetAsync(z.first, 0, z.second, st));
  if (eo) {
    // bh = b_e + kappa H_eo b_o
    hop<H, H, false, false, OP>(E, 0, kLinkHi, InOne<H>{S_B}, EpiXpay<H, H, C_PK, false>{S_BH, S_B, G_ALL});
  }
  // zero guess: r = source (bh or b); otherwise r = source - A x, recomputed
  count_launch();
  k_init_r<L, H><<<E.grid(eo ? 0 : 2), E.P.block, 0, st>>>(E.P.B, eo ? 0 : 2, eo ? S_BH : S_B, E.ra(FIN_RESID0));
  finish(E, eo ? 0 : 2, FIN_RESID0);
  if (profiler().timing) {
    // host-stepped (profiled) run: launch the first FP64-class residual only
    // when the guess is non-zero, so every timed launch does its work
    static Flags* hf0 = nullptr;
    if (!hf0) DW_CUDA(cudaMallocHost((void**)&hf0, sizeof(Flags)));
    DW_CUDA(cudaMemcpyAsync(hf0, E.rb.flags, sizeof(Flags), cudaMemcpyDeviceToHost, st));
    DW_CUDA(cudaStreamSynchronize(st));
    if (hf0->rel_pending > 0) reliable(E, mode);
  } else {
    reliable(E, mode);
  }
  zstep(E, mode, FIN_GAMMA0);  // z, gamma
  count_launch();
  k_update_p<L, A><<<E.grid(eo ? 0 : 2), E.P.block, 0, st>>>(E.P.B, eo ? 0 : 2, E.ra(FIN_STORE0));  // p = z
  DW_CUDA(cudaGetLastError());

  // ---- iterations
  const int body_k = ent->body_k, rel_k = ent->rel_k;
  const bool graph = !profiler().timing;
  if (graph) {
    DW_CUDA(cudaGraphLaunch(ent->exec, st));
  } else {
    DW_TRY(run_stepped(E, mode, a.p.maxiter));
  }

  // ---- finish: odd sites, then the IEEE FP64 residual from the caller's fields
  if (eo) {
    // x_o = b_o + kappa H_oe x_e, with H_oe x_e (the first hop of the column's
    // last reliable update, taken of its final x_e) read from the odd half of S_RT
    count_launch();
    k_recon_odd<H><<<E.grid(1), E.P.block, 0, st>>>(E.P.B, 1, E.ra(FIN_STORE0));
  }
  if (H != P64) {
    count_launch();
    k_convert<P64, H><<<E.grid(2), E.P.block, 0, st>>>(E.P.B, 2, S_XU, S_X, E.ra(FIN_STORE0));
  }
  count_launch();
  k_zero_zsrc<P64><<<E.grid(2), E.P.block, 0, st>>>(E.P.B, 2, S_XU, E.ra(FIN_STORE0));  // zero source: x = 0
  const int rt64 = H == P64 ? S_RT : S_AUX1;  // FP64 full temporary (verify_normal)
  if (mode != MODE_NORMAL) {
    hop<P64, P64, false, false, OP>(E, 2, S_LF64, InOne<P64>{S_XU},
                                EpiResidFull<L, false, P64>{G_ALL, a.p.verify_normal ? rt64 : -1, S_XU, S_BU},
                                FIN_STORE0);
    if constexpr (OP == OP_WILSON) {
      if (a.p.verify_normal) {
        hop<P64, P64, false, true, OP>(E, 2, S_LF64, InOne<P64>{rt64}, EpiXpay<P64, P64, C_MK, true>{-1, rt64, G_ALL},
                                       FIN_STORE1);
        hop<P64, P64, false, true, OP>(E, 2, S_LF64, InOne<P64>{S_BU}, EpiXpay<P64, P64, C_MK, true>{-1, S_BU, G_ALL},
                                       FIN_STORE2);
      }
    }
  } else {
    if constexpr (OP == OP_WILSON) {
      // |b - D^dag D x|^2 in FP64: t = D x into the FP64 temporary, then b - D^dag t
      const int t64 = H == P64 ? S_AUX0 : S_AUX1;
      hop<P64, P64, false, false, OP>(E, 2, S_LF64, InOne<P64>{S_XU},
                                      EpiXpay<P64, P64, C_MK, false>{t64, S_XU, G_ALL});
      hop<P64, P64, false, true, OP>(E, 2, S_LF64, InOne<P64>{t64}, EpiResidFull<L, false, P64>{G_ALL, -1, t64, S_BU},
                                     FIN_STORE0);
    }
  }
  DW_CUDA(cudaEventRecord(ev1, st));
  DW_CUDA(cudaMemcpyAsync(hc.data(), E.rb.cols, sizeof(ColState) * hc.size(), cudaMemcpyDeviceToHost, st));
  DW_CUDA(cudaMemcpyAsync(&hf, E.rb.flags, sizeof hf, cudaMemcpyDeviceToHost, st));
  DW_CUDA(cudaStreamSynchronize(st));
  if (graph && profiler().on) profiler().launches += (long long)hf.loops * body_k + (long long)hf.rel_runs * rel_k;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
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
        o.normal_rel_resid = mode == MODE_HERM     ? -1.0
                             : mode == MODE_NORMAL ? true_rel
                             : a.p.verify_normal ? sqrt(c.store[1] / (c.store[2] > 0 ? c.store[2] : 1.0))
                                                 : -1.0;
        o.time_ms = ms;
        const double vh = (double)S.vh;
        const double hops_lo = 4.0 * c.iter;  // parity-hops per iteration (D and D^dag, two each)
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
