/*
 * dw_oracle.c -- plain, slow, obviously-correct FP64 reference for the
 * Wilson-Dirac conjugate-gradient path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (the paper, Korcyl & Korcyl, "Optimized implementation of
 * the conjugate gradient algorithm for FPGA-based platforms using the
 * Dirac-Wilson operator as an example", SoftwareX):
 *   - Sec. 1 and Sec. 3.2 state the problem: solve a large sparse system whose
 *     matrix is the Dirac-Wilson operator, by conjugate gradient.  The paper
 *     prints no formula; the operator is the standard one,
 *       D(x,y) = delta_xy - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) delta_{x+mu,y}
 *                                        + (1 + gamma_mu) U_mu(x-mu)^dag delta_{x-mu,y} ],
 *     on an L_x*L_y*L_z*L_t lattice, periodic in space and (optionally)
 *     antiperiodic in time (a sign -1 on every link that crosses t=L_t-1 -> 0).
 *   - Fig. 1 caption: the per-site data are 3x3 complex link matrices U and
 *     12-component complex vectors psi (4 spins x 3 colours).
 *   - Sec. 3.1.1: the host-side CG loop owns solution, residual and search vectors and
 *     evaluates the stopping criterion on the full residual vector.
 *
 * Layout (canonical, host): site index  s = x + Lx*(y + Ly*(z + Lz*t));
 *   spinor  psi[s][spin][colour]        (complex double)
 *   gauge   U[s][mu][row][col]          (complex double), mu = 0..3 = x,y,z,t
 *
 * Gamma basis (the paper is silent): chiral,
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  for mu = 0,1,2 (k = mu+1),
 *   gamma_3 = [[0, 1], [1, 0]],  gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3
 *           = diag(1, 1, -1, -1).
 *
 * Every spin product here multiplies by the explicit 4x4 matrix (1 -/+ gamma);
 * no spin-projection shortcut is taken.  Site loops may run under OpenMP;
 * each output site is written by exactly one thread, so results do not
 * depend on the thread count.  Dot products are serial, in site order.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

static long volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int d[4], long s, int c[4]) {
  c[0] = (int)(s % d[0]); s /= d[0];
  c[1] = (int)(s % d[1]); s /= d[1];
  c[2] = (int)(s % d[2]); s /= d[2];
  c[3] = (int)s;
}

static long site_of(const int d[4], const int c[4]) {
  return c[0] + (long)d[0] * (c[1] + (long)d[1] * (c[2] + (long)d[2] * c[3]));
}

/* Neighbour of s one step in direction mu (dir = +1 or -1), periodic wrap.
 * *sign receives the boundary phase of the link crossed: -1 when the step
 * crosses the time boundary of an antiperiodic lattice, else +1. */
static long neighbour(const int d[4], int anti_t, long s, int mu, int dir, double* sign) {
  int c[4];
  coords(d, s, c);
  int v = c[mu] + dir;
  *sign = 1.0;
  if (v == d[mu]) { v = 0; if (mu == 3 && anti_t) *sign = -1.0; }
  if (v < 0) { v = d[mu] - 1; if (mu == 3 && anti_t) *sign = -1.0; }
  c[mu] = v;
  return site_of(d, c);
}

/* ------------------------------------------------------------------ */
/* Gamma matrices                                                      */
/* ------------------------------------------------------------------ */

static void pauli(int k, cplx p[2][2]) {
  /* k = 1, 2, 3 */
  if (k == 1) { p[0][0] = 0; p[0][1] = 1; p[1][0] = 1; p[1][1] = 0; }
  else if (k == 2) { p[0][0] = 0; p[0][1] = -I; p[1][0] = I; p[1][1] = 0; }
  else { p[0][0] = 1; p[0][1] = 0; p[1][0] = 0; p[1][1] = -1; }
}

void or_gamma(int mu, double* out /* 4x4 complex, row-major, re/im */) {
  cplx g[4][4];
  memset(g, 0, sizeof g);
  if (mu == 4) {
    /* gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3, formed by multiplication */
    cplx a[4][4], b[4][4], t[4][4];
    or_gamma(0, (double*)a);
    for (int m = 1; m < 4; ++m) {
      or_gamma(m, (double*)b);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          cplx acc = 0;
          for (int k = 0; k < 4; ++k) acc += a[i][k] * b[k][j];
          t[i][j] = acc;
        }
      memcpy(a, t, sizeof a);
    }
    memcpy(out, a, sizeof a);
    return;
  }
  if (mu == 3) {
    for (int i = 0; i < 2; ++i) { g[i][i + 2] = 1; g[i + 2][i] = 1; }
  } else {
    cplx p[2][2];
    pauli(mu + 1, p);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        g[i][j + 2] = -I * p[i][j];
        g[i + 2][j] = I * p[i][j];
      }
  }
  memcpy(out, g, sizeof g);
}

/* spin matrix (1 + s*gamma_mu), s = +1 or -1 */
static void one_plus_s_gamma(int mu, double s, cplx m[4][4]) {
  cplx g[4][4];
  or_gamma(mu, (double*)g);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m[i][j] = (i == j ? 1.0 : 0.0) + s * g[i][j];
}

/* ------------------------------------------------------------------ */
/* Hopping term and the Wilson-Dirac operator                          */
/* ------------------------------------------------------------------ */

/* out(x) = sum_mu [ (1 + sf*gamma_mu) eta U_mu(x) in(x+mu)
 *                 + (1 + sb*gamma_mu) eta U_mu(x-mu)^dag in(x-mu) ]
 * with (sf, sb) = (-1, +1) for H (the hopping term of D) and (+1, -1) for the
 * hopping term of D^dag (conjugate transpose of D, element by element). */
static void hop_general(const int d[4], int anti_t, const cplx* U, const cplx* in, cplx* out,
                        double sf, double sb) {
  const long V = volume(d);
  cplx Pf[4][4][4], Pb[4][4][4];
  for (int mu = 0; mu < 4; ++mu) { one_plus_s_gamma(mu, sf, Pf[mu]); one_plus_s_gamma(mu, sb, Pb[mu]); }
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    cplx acc[4][3];
    memset(acc, 0, sizeof acc);
    for (int mu = 0; mu < 4; ++mu) {
      double sgn;
      /* forward: U_mu(x) in(x+mu) */
      long f = neighbour(d, anti_t, s, mu, +1, &sgn);
      const cplx* u = U + ((s * 4 + mu) * 9);
      const cplx* pf = in + f * 12;
      cplx v[4][3];
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
          cplx t = 0;
          for (int b = 0; b < 3; ++b) t += u[a * 3 + b] * pf[sp * 3 + b];
          v[sp][a] = sgn * t;
        }
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a)
          for (int q = 0; q < 4; ++q) acc[sp][a] += Pf[mu][sp][q] * v[q][a];
      /* backward: U_mu(x-mu)^dag in(x-mu) */
      long bk = neighbour(d, anti_t, s, mu, -1, &sgn);
      const cplx* ub = U + ((bk * 4 + mu) * 9);
      const cplx* pb = in + bk * 12;
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
          cplx t = 0;
          for (int b = 0; b < 3; ++b) t += conj(ub[b * 3 + a]) * pb[sp * 3 + b];
          v[sp][a] = sgn * t;
        }
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a)
          for (int q = 0; q < 4; ++q) acc[sp][a] += Pb[mu][sp][q] * v[q][a];
    }
    memcpy(out + s * 12, acc, sizeof acc);
  }
}

/* H psi: hopping term, so that D = 1 - kappa*H */
void or_hop(const int* d, int anti_t, const double* U, const double* in, double* out) {
  hop_general(d, anti_t, (const cplx*)U, (const cplx*)in, (cplx*)out, -1.0, +1.0);
}

/* hopping term of D^dag, so that D^dag = 1 - kappa*Hdag */
void or_hop_dag(const int* d, int anti_t, const double* U, const double* in, double* out) {
  hop_general(d, anti_t, (const cplx*)U, (const cplx*)in, (cplx*)out, +1.0, -1.0);
}

static void dirac_general(const int* d, int anti_t, double kappa, const double* U, const double* in,
                          double* out, int dag) {
  const long n = volume(d) * 12;
  cplx* h = (cplx*)malloc(sizeof(cplx) * n);
  if (dag) or_hop_dag(d, anti_t, U, in, (double*)h);
  else or_hop(d, anti_t, U, in, (double*)h);
  const cplx* x = (const cplx*)in;
  cplx* o = (cplx*)out;
  for (long i = 0; i < n; ++i) o[i] = x[i] - kappa * h[i];
  free(h);
}

/* out = D psi */
void or_dirac(const int* d, int anti_t, double kappa, const double* U, const double* in, double* out) {
  dirac_general(d, anti_t, kappa, U, in, out, 0);
}

/* out = D^dag psi */
void or_dirac_dag(const int* d, int anti_t, double kappa, const double* U, const double* in, double* out) {
  dirac_general(d, anti_t, kappa, U, in, out, 1);
}

/* out = D^dag D psi */
void or_normal(const int* d, int anti_t, double kappa, const double* U, const double* in, double* out) {
  const long n = volume(d) * 12;
  double* t = (double*)malloc(sizeof(cplx) * n);
  or_dirac(d, anti_t, kappa, U, in, t);
  or_dirac_dag(d, anti_t, kappa, U, t, out);
  free(t);
}

/* ------------------------------------------------------------------ */
/* Even-odd (Schur complement) operator, by composition                */
/* ------------------------------------------------------------------ */

static int parity_of(const int d[4], long s) {
  int c[4];
  coords(d, s, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* Zero every site whose parity differs from `keep`. */
void or_mask_parity(const int* d, double* field, int keep) {
  const long V = volume(d);
  cplx* f = (cplx*)field;
  for (long s = 0; s < V; ++s)
    if (parity_of(d, s) != keep)
      for (int k = 0; k < 12; ++k) f[s * 12 + k] = 0;
}

/* Schur complement on parity p of D = [[1, -kappa H_pq], [-kappa H_qp, 1]]:
 *   Dhat psi_p = psi_p - kappa^2 H_pq H_qp psi_p      (dag = 0)
 *   Dhat^dag psi_p = psi_p - kappa^2 Hdag_pq Hdag_qp psi_p   (dag = 1)
 * Input and output are full-lattice arrays; only parity-p sites of the input
 * are read, and the output is zero on the other parity. */
void or_schur(const int* d, int anti_t, double kappa, const double* U, const double* in, double* out,
              int p, int dag) {
  const long n = volume(d) * 12;
  double* a = (double*)malloc(sizeof(cplx) * n);
  double* t = (double*)malloc(sizeof(cplx) * n);
  memcpy(a, in, sizeof(cplx) * n);
  or_mask_parity(d, a, p);
  if (dag) { or_hop_dag(d, anti_t, U, a, t); or_hop_dag(d, anti_t, U, t, out); }
  else { or_hop(d, anti_t, U, a, t); or_hop(d, anti_t, U, t, out); }
  cplx* o = (cplx*)out;
  const cplx* x = (const cplx*)a;
  for (long i = 0; i < n; ++i) o[i] = x[i] - kappa * kappa * o[i];
  or_mask_parity(d, out, p);
  free(a);
  free(t);
}

/* ------------------------------------------------------------------ */
/* Conjugate gradient (plain textbook forms, full lattice, FP64)      */
/* ------------------------------------------------------------------ */

static double norm2(const cplx* a, long n) {
  double s = 0;
  for (long i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
  return s;
}

/* CG on the normal equations D^dag D x = D^dag b (CGNR), full lattice.
 * x holds the initial guess on entry and the solution on exit.  Stops when
 * the true-recursion residual |b - D x| <= tol |b|.  Returns the iteration
 * count, or -1 if maxiter was reached first. */
int or_cgnr(const int* d, int anti_t, double kappa, const double* U, const double* b, double* x,
            double tol, int maxiter, double* final_rel_resid) {
  const long n = volume(d) * 12;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  cplx* z = (cplx*)malloc(sizeof(cplx) * n);
  cplx* p = (cplx*)malloc(sizeof(cplx) * n);
  cplx* w = (cplx*)malloc(sizeof(cplx) * n);
  cplx* X = (cplx*)x;
  const cplx* B = (const cplx*)b;
  or_dirac(d, anti_t, kappa, U, x, (double*)w);
  for (long i = 0; i < n; ++i) r[i] = B[i] - w[i];
  const double bn = sqrt(norm2(B, n));
  or_dirac_dag(d, anti_t, kappa, U, (double*)r, (double*)z);
  memcpy(p, z, sizeof(cplx) * n);
  double gam = norm2(z, n);
  double rn = sqrt(norm2(r, n));
  int it = 0;
  while (rn > tol * bn && it < maxiter) {
    or_dirac(d, anti_t, kappa, U, (double*)p, (double*)w);
    const double alpha = gam / norm2(w, n);
    for (long i = 0; i < n; ++i) { X[i] += alpha * p[i]; r[i] -= alpha * w[i]; }
    rn = sqrt(norm2(r, n));
    ++it;
    if (rn <= tol * bn) break;
    or_dirac_dag(d, anti_t, kappa, U, (double*)r, (double*)z);
    const double gnew = norm2(z, n);
    const double beta = gnew / gam;
    gam = gnew;
    for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  /* report the residual recomputed from scratch */
  or_dirac(d, anti_t, kappa, U, x, (double*)w);
  for (long i = 0; i < n; ++i) r[i] = B[i] - w[i];
  if (final_rel_resid) *final_rel_resid = sqrt(norm2(r, n)) / bn;
  free(r); free(z); free(p); free(w);
  return rn <= tol * bn ? it : -1;
}

/* Plain CG on A x = b with A = D^dag D (Hermitian positive definite).
 * Stops when |b - A x| <= tol |b| on the recursive residual. */
int or_cg_normal(const int* d, int anti_t, double kappa, const double* U, const double* b, double* x,
                 double tol, int maxiter, double* final_rel_resid) {
  const long n = volume(d) * 12;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  cplx* p = (cplx*)malloc(sizeof(cplx) * n);
  cplx* ap = (cplx*)malloc(sizeof(cplx) * n);
  cplx* X = (cplx*)x;
  const cplx* B = (const cplx*)b;
  or_normal(d, anti_t, kappa, U, x, (double*)ap);
  for (long i = 0; i < n; ++i) r[i] = B[i] - ap[i];
  memcpy(p, r, sizeof(cplx) * n);
  const double bn = sqrt(norm2(B, n));
  double rr = norm2(r, n);
  int it = 0;
  while (sqrt(rr) > tol * bn && it < maxiter) {
    or_normal(d, anti_t, kappa, U, (double*)p, (double*)ap);
    double pap = 0;
    for (long i = 0; i < n; ++i) pap += creal(conj(p[i]) * ap[i]);
    const double alpha = rr / pap;
    for (long i = 0; i < n; ++i) { X[i] += alpha * p[i]; r[i] -= alpha * ap[i]; }
    const double rnew = norm2(r, n);
    const double beta = rnew / rr;
    rr = rnew;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  or_normal(d, anti_t, kappa, U, x, (double*)ap);
  for (long i = 0; i < n; ++i) r[i] = B[i] - ap[i];
  if (final_rel_resid) *final_rel_resid = sqrt(norm2(r, n)) / bn;
  free(r); free(p); free(ap);
  return sqrt(rr) <= tol * bn ? it : -1;
}

/* ------------------------------------------------------------------ */
/* A second stencil: the gauge-covariant Laplacian                     */
/* ------------------------------------------------------------------ */
/* The same lattice, links and boundary signs with no spin structure
 * (another four-dimensional stencil behind the same CG, the generalisation
 * the paper points to in Sec. 1, the caption of Fig. 1 and Sec. 3.2):
 *   out = in - kappa * K in,
 *   K(x,y) = sum_mu [ eta U_mu(x) delta_{x+mu,y} + eta U_mu(x-mu)^dag delta_{x-mu,y} ]
 * acting on each spin component alike.  With kappa = 1/(8 + m^2) this is
 * (-Delta_U + m^2)/(8 + m^2); it is Hermitian, and positive definite for
 * kappa < 1/8 (|K| <= 8). */
void or_laplace(const int* d, int anti_t, double kappa, const double* Ud, const double* in_d, double* out_d) {
  const long V = volume(d);
  const cplx* U = (const cplx*)Ud;
  const cplx* in = (const cplx*)in_d;
  cplx* out = (cplx*)out_d;
#pragma omp parallel for schedule(static)
  for (long s = 0; s < V; ++s) {
    cplx acc[4][3];
    memset(acc, 0, sizeof acc);
    for (int mu = 0; mu < 4; ++mu) {
      double sgn;
      const long f = neighbour(d, anti_t, s, mu, +1, &sgn);
      const cplx* u = U + ((s * 4 + mu) * 9);
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
          cplx t = 0;
          for (int b = 0; b < 3; ++b) t += u[a * 3 + b] * in[f * 12 + sp * 3 + b];
          acc[sp][a] += sgn * t;
        }
      const long bk = neighbour(d, anti_t, s, mu, -1, &sgn);
      const cplx* ub = U + ((bk * 4 + mu) * 9);
      for (int sp = 0; sp < 4; ++sp)
        for (int a = 0; a < 3; ++a) {
          cplx t = 0;
          for (int b = 0; b < 3; ++b) t += conj(ub[b * 3 + a]) * in[bk * 12 + sp * 3 + b];
          acc[sp][a] += sgn * t;
        }
    }
    for (int sp = 0; sp < 4; ++sp)
      for (int a = 0; a < 3; ++a) out[s * 12 + sp * 3 + a] = in[s * 12 + sp * 3 + a] - kappa * acc[sp][a];
  }
}

/* Plain CG on the Laplacian system M x = b (Hermitian positive definite),
 * full lattice; stops when the recursive residual |r| <= tol |b|. */
int or_cg_laplace(const int* d, int anti_t, double kappa, const double* U, const double* b, double* x,
                  double tol, int maxiter, double* final_rel_resid) {
  const long n = volume(d) * 12;
  cplx* r = (cplx*)malloc(sizeof(cplx) * n);
  cplx* p = (cplx*)malloc(sizeof(cplx) * n);
  cplx* ap = (cplx*)malloc(sizeof(cplx) * n);
  cplx* X = (cplx*)x;
  const cplx* B = (const cplx*)b;
  or_laplace(d, anti_t, kappa, U, x, (double*)ap);
  for (long i = 0; i < n; ++i) r[i] = B[i] - ap[i];
  memcpy(p, r, sizeof(cplx) * n);
  const double bn = sqrt(norm2(B, n));
  double rr = norm2(r, n);
  int it = 0;
  while (sqrt(rr) > tol * bn && it < maxiter) {
    or_laplace(d, anti_t, kappa, U, (double*)p, (double*)ap);
    double pap = 0;
    for (long i = 0; i < n; ++i) pap += creal(conj(p[i]) * ap[i]);
    const double alpha = rr / pap;
    for (long i = 0; i < n; ++i) { X[i] += alpha * p[i]; r[i] -= alpha * ap[i]; }
    const double rnew = norm2(r, n);
    const double beta = rnew / rr;
    rr = rnew;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  or_laplace(d, anti_t, kappa, U, x, (double*)ap);
  for (long i = 0; i < n; ++i) r[i] = B[i] - ap[i];
  if (final_rel_resid) *final_rel_resid = sqrt(norm2(r, n)) / bn;
  free(r); free(p); free(ap);
  return sqrt(rr) <= tol * bn ? it : -1;
}

/* ------------------------------------------------------------------ */
/* Dense assembly (for LU cross-checks on tiny lattices)               */
/* ------------------------------------------------------------------ */

/* M is (12V) x (12V) complex, row-major; row = 12*x + 3*spin + colour.
 * Entries are accumulated from the operator's definition block by block;
 * on a lattice of extent 2 the forward and backward neighbours coincide and
 * both contributions land in the same block. */
void or_dense_dirac(const int* d, int anti_t, double kappa, const double* Ud, double* Md) {
  const long V = volume(d), N = 12 * V;
  const cplx* U = (const cplx*)Ud;
  cplx* M = (cplx*)Md;
  memset(M, 0, sizeof(cplx) * N * N);
  for (long i = 0; i < N; ++i) M[i * N + i] = 1.0;
  for (long x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      cplx Pm[4][4], Pp[4][4];
      one_plus_s_gamma(mu, -1.0, Pm);
      one_plus_s_gamma(mu, +1.0, Pp);
      double sf, sb;
      long yf = neighbour(d, anti_t, x, mu, +1, &sf);
      long yb = neighbour(d, anti_t, x, mu, -1, &sb);
      const cplx* uf = U + (x * 4 + mu) * 9;
      const cplx* ub = U + (yb * 4 + mu) * 9;
      for (int s1 = 0; s1 < 4; ++s1)
        for (int a = 0; a < 3; ++a)
          for (int s2 = 0; s2 < 4; ++s2)
            for (int b = 0; b < 3; ++b) {
              long row = 12 * x + 3 * s1 + a;
              M[row * N + 12 * yf + 3 * s2 + b] += -kappa * sf * Pm[s1][s2] * uf[a * 3 + b];
              M[row * N + 12 * yb + 3 * s2 + b] += -kappa * sb * Pp[s1][s2] * conj(ub[b * 3 + a]);
            }
    }
}

/* ------------------------------------------------------------------ */
/* Gauge force (derivative of Re<Y, dD X> with respect to the links)   */
/* ------------------------------------------------------------------ */

/* F[x][mu] = kappa * eta_mu(x) * sum_s [ w_s X(x+mu)_s^dag + X(x)_s w'_s^dag ],
 *   w = (1 - gamma_mu) Y(x),  w' = (1 + gamma_mu) Y(x+mu),
 * so that  -Re<Y, dD X> = Re sum_{x,mu} tr(F^dag dU_mu(x))  for any change dU
 * of the links (D depends linearly on U and U^dag).  With this,
 *   S = phi^dag (D^dag D)^{-1} phi:  dS/dU (PyTorch convention) = 2 F(D X, X),
 *     X = (D^dag D)^{-1} phi;
 *   L(x), x = (D^dag D)^{-1} b, g = dL/dx:  dL/dU = F(D x, l) + F(D l, x),
 *     l = (D^dag D)^{-1} g. */
void or_force(const int* d, int anti_t, double kappa, const double* Yd, const double* Xd, double* Fd) {
  const long V = volume(d);
  const cplx* Y = (const cplx*)Yd;
  const cplx* X = (const cplx*)Xd;
  cplx* F = (cplx*)Fd;
#pragma omp parallel for schedule(static)
  for (long x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      cplx Pm[4][4], Pp[4][4];
      one_plus_s_gamma(mu, -1.0, Pm);
      one_plus_s_gamma(mu, +1.0, Pp);
      double eta;
      long xf = neighbour(d, anti_t, x, mu, +1, &eta);
      cplx w[4][3], wp[4][3];
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
          cplx t1 = 0, t2 = 0;
          for (int q = 0; q < 4; ++q) {
            t1 += Pm[s][q] * Y[x * 12 + q * 3 + a];
            t2 += Pp[s][q] * Y[xf * 12 + q * 3 + a];
          }
          w[s][a] = t1;
          wp[s][a] = t2;
        }
      cplx* f = F + (x * 4 + mu) * 9;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cplx acc = 0;
          for (int s = 0; s < 4; ++s)
            acc += w[s][a] * conj(X[xf * 12 + s * 3 + b]) + X[x * 12 + s * 3 + a] * conj(wp[s][b]);
          f[a * 3 + b] = kappa * eta * acc;
        }
    }
}

/* su(3) projection of a link gradient: P(G U^dag) with
 * P(M) = (M - M^dag)/2 - tr(M - M^dag)/6 * 1  (traceless anti-Hermitian part).
 * Then for U -> exp(eps T) U, T in su(3):  dS/deps = Re tr(P^dag T). */
void or_su3_project(long nlinks, const double* Gd, const double* Ud, double* Pd) {
  const cplx* G = (const cplx*)Gd;
  const cplx* U = (const cplx*)Ud;
  cplx* P = (cplx*)Pd;
  for (long l = 0; l < nlinks; ++l) {
    cplx M[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        cplx t = 0;
        for (int c = 0; c < 3; ++c) t += G[l * 9 + a * 3 + c] * conj(U[l * 9 + b * 3 + c]);
        M[a][b] = t;
      }
    cplx tr = 0;
    for (int a = 0; a < 3; ++a) tr += M[a][a] - conj(M[a][a]);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        P[l * 9 + a * 3 + b] = 0.5 * (M[a][b] - conj(M[b][a])) - (a == b ? tr / 6.0 : 0.0);
  }
}

int or_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Thread count of the oracle's OpenMP loops (n >= 1); used to time the
 * oracle on one host core as well as on all of them. */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  omp_set_num_threads(n < 1 ? 1 : n);
#else
  (void)n;
#endif
}
