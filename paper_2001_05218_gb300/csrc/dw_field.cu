// dw_field.cu -- field handles, host/device transfers and the layout kernels
// that convert between the canonical (lexicographic, site-major complex128)
// order and the even-odd structure-of-arrays storage.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <sys/stat.h>
#include <mutex>

#include "dw_exec.cuh"

namespace dw {

static thread_local char g_err[1024] = "";

dw_status set_error(dw_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

dw_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_err, sizeof g_err, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file,
           line);
  return e == cudaErrorMemoryAllocation ? DW_ERR_OOM : DW_ERR_CUDA;
}

void clear_error() { g_err[0] = 0; }

int spin_bytes(int prec) {
  switch (prec) {
    case DW_F64: return Spin<P64>::kBytes;
    case DW_F32: return Spin<P32>::kBytes;
    case DW_F16: return Spin<P16>::kBytes;
    case DW_BF16: return Spin<PB16>::kBytes;
    case DW_DF64: return Spin<PDF>::kBytes;
    case DW_I16: return Spin<PI16>::kBytes;
  }
  return 0;
}

int link_bytes(int prec, int c12) {
  switch (prec) {
    case DW_F64: return c12 ? Link<P64, true>::kBytes : Link<P64, false>::kBytes;
    case DW_F32: return c12 ? Link<P32, true>::kBytes : Link<P32, false>::kBytes;
    case DW_F16: return c12 ? Link<P16, true>::kBytes : Link<P16, false>::kBytes;
    case DW_BF16: return c12 ? Link<PB16, true>::kBytes : Link<PB16, false>::kBytes;
    case DW_DF64: return c12 ? Link<PDF, true>::kBytes : Link<PDF, false>::kBytes;
    case DW_I16: return c12 ? Link<PI16, true>::kBytes : Link<PI16, false>::kBytes;
  }
  return 0;
}

dw_status check_lattice(const dw_lattice* l) {
  DW_CHECK(l != nullptr, DW_ERR_ARG, "lattice is NULL");
  for (int m = 0; m < 4; ++m)
    DW_CHECK(l->dims[m] >= 2 && (l->dims[m] % 2) == 0, DW_ERR_SHAPE,
             "lattice extent %d in direction %d must be even and >= 2", l->dims[m], m);
  const long long V = volume_of(*l);
  DW_CHECK(V / 2 <= (1ll << 30), DW_ERR_SHAPE, "lattice too large (%lld sites)", V);
  DW_CHECK((V / 2) % 8 == 0, DW_ERR_SHAPE, "half volume %lld must be a multiple of 8", V / 2);
  return DW_OK;
}

bool same_dims(const dw_lattice& a, const dw_lattice& b) {
  return a.dims[0] == b.dims[0] && a.dims[1] == b.dims[1] && a.dims[2] == b.dims[2] && a.dims[3] == b.dims[3];
}

Slot arena_slot(char* p, const dw_lattice& l, int prec, int nrhs, int npar) {
  (void)nrhs;
  Slot s;
  const long long blk = (long long)spin_bytes(prec) * vh_of(l);
  s.p = p;
  s.par_stride = npar == 2 ? blk : 0;
  s.rhs_stride = blk * npar;
  return s;
}

Slot spinor_slot(const dw_field* f) { return arena_slot(f->ptr, f->lat, f->prec, f->nrhs, npar_of(f->kind)); }

Slot gauge_slot(const char* p, const dw_lattice& l, int prec, int c12) {
  Slot s;
  s.p = const_cast<char*>(p);
  s.rhs_stride = 0;
  s.par_stride = 4ll * link_bytes(prec, c12) * vh_of(l);
  return s;
}

static FastDiv fast_div(int d) {
  int l = 0;
  while ((1ll << l) < d) ++l;
  FastDiv f;
  f.m = (unsigned)((((unsigned long long)1 << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l - 1 > 0 ? l - 1 : 0;
  return f;
}

void geometry(SysDesc& S, const dw_lattice& l, int nrhs) {
  memset(&S, 0, sizeof S);
  S.lxh = l.dims[0] / 2;
  S.ly = l.dims[1];
  S.lz = l.dims[2];
  S.lt = l.dims[3];
  S.div_lxh = fast_div(S.lxh);
  S.div_ly = fast_div(S.ly);
  S.div_lz = fast_div(S.lz);
  S.vh = (int)vh_of(l);
  S.nrhs = nrhs;
  S.anti_t = l.t_antiperiodic ? 1 : 0;
  S.kappa = l.kappa;
  const double k2 = l.kappa * l.kappa;
  S.kappa_f = (float)l.kappa;
  S.kappa_lo = (float)(l.kappa - (double)S.kappa_f);
  S.kappa2_f = (float)k2;
  S.kappa2_lo = (float)(k2 - (double)S.kappa2_f);
}

void default_block_shape(int nrhs, int* T, int* RB) {
  // 128 sites per block, or 64 sites x (the largest divisor of nrhs up to 4)
  *RB = 1;
  *T = 128;
  if (nrhs > 1) {
    *T = 64;
    for (int d = 4; d >= 1; --d)
      if (nrhs % d == 0) {
        *RB = d;
        break;
      }
  }
}

void make_plan(Plan& P, const dw_lattice* lats, int n, int nrhs, int T, int RB) {
  memset(&P.B, 0, sizeof P.B);
  P.pair = 0;
  P.nsys = n;
  P.nrhs = nrhs;
  if (T <= 0 || RB <= 0) default_block_shape(nrhs, &T, &RB);
  P.B.nsys = P.nsys;
  P.B.T = T;
  P.B.RB = RB;
  int tile = 0, part = 0;
  for (int i = 0; i < P.nsys; ++i) {
    SysDesc& S = P.B.sd[i];
    geometry(S, lats[i], nrhs);
    S.tpp = (S.vh + T - 1) / T;
    S.tile0 = tile;
    S.col0 = i * nrhs;
    S.part0 = part;
    S.sys = i;
    tile += S.tpp;
    part += nrhs * 2 * S.tpp;  // block partials (both-parity launches hold 2*tpp tiles)
  }
  P.B.ntot = tile;
  P.ncols = P.nsys * nrhs;
  P.partials = part;
  const int gy = (nrhs + RB - 1) / RB;
  P.block = dim3(T * RB);
  P.B.ny = gy;
  P.grid1 = dim3(tile * gy);
  P.grid2 = dim3(2 * tile * gy);
}

// ------------------------------------------------------------------ layout kernels
__host__ __device__ inline long long lex_of(const int* d, int par, long long j) {
  const int lxh = d[0] / 2;
  long long q = j / lxh;
  const int xh = (int)(j - q * lxh);
  const int y = (int)(q % d[1]);
  q /= d[1];
  const int z = (int)(q % d[2]);
  const int t = (int)(q / d[2]);
  const int x = 2 * xh + ((y + z + t + par) & 1);
  return x + (long long)d[0] * (y + (long long)d[1] * (z + (long long)d[2] * t));
}

struct Dims4 {
  int d[4];
};

// canonical (complex128, [rhs][site][12]) <-> storage.  Threads run over the
// canonical site order (lexicographic for full fields, j for parity fields) so
// that a warp touches one contiguous stretch of the canonical array -- which
// may be page-locked host memory read or written over the host link.
__host__ __device__ inline void site_to_eo(const int* d, long long lex, int* par, long long* j) {
  long long q = lex / d[0];
  const int x = (int)(lex - q * d[0]);
  const int y = (int)(q % d[1]);
  q /= d[1];
  const int z = (int)(q % d[2]);
  const int t = (int)(q / d[2]);
  *par = (x + y + z + t) & 1;
  *j = lex >> 1;
}

// Spinor kernels run over canonical elements e = rhs * nsite + site in
// [e0, e1); gauge kernels over canonical sites [s0, s1).  A host transfer in
// chunks launches one kernel per chunk.
template <int P>
__global__ void k_pack_spinor(Dims4 dm, int vh, int npar, int par0, long long e0, long long e1,
                              const double2* __restrict__ can, Slot dst) {
  const long long e = e0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= e1) return;
  const long long nsite = (long long)vh * npar;
  const int r = (int)(e / nsite);
  const long long site = e - r * nsite;
  int par = par0, pi = 0;
  long long j = site;
  if (npar == 2) {
    site_to_eo(dm.d, site, &par, &j);
    pi = par;
  }
  using R = typename Spin<P>::R;
  const double2* src = can + e * 12;
  Cx<R> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 t = src[k];
    v[k] = cx((R)t.x, (R)t.y);
  }
  Spin<P>::store(dst.p + r * dst.rhs_stride + pi * dst.par_stride, vh, (int)j, v);
}

template <int P>
__global__ void k_unpack_spinor(Dims4 dm, int vh, int npar, int par0, long long e0, long long e1, Slot srcs,
                                double2* __restrict__ can) {
  const long long e = e0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= e1) return;
  const long long nsite = (long long)vh * npar;
  const int r = (int)(e / nsite);
  const long long site = e - r * nsite;
  int par = par0, pi = 0;
  long long j = site;
  if (npar == 2) {
    site_to_eo(dm.d, site, &par, &j);
    pi = par;
  }
  using R = typename Spin<P>::R;
  Cx<R> v[12];
  Spin<P>::load(srcs.p + r * srcs.rhs_stride + pi * srcs.par_stride, vh, (int)j, v);
  double2* o = can + e * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) o[k] = make_double2((double)v[k].re, (double)v[k].im);
}

template <int P, bool C12>
__global__ void k_pack_gauge(Dims4 dm, int vh, long long s0, long long s1, const double2* __restrict__ can,
                             char* dst) {
  const long long site = s0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (site >= s1) return;
  int par;
  long long j;
  site_to_eo(dm.d, site, &par, &j);
  const long long lb = (long long)Link<P, C12>::kBytes * vh;
  using R = typename Link<P, C12>::R;
  for (int mu = 0; mu < 4; ++mu) {
    const double2* src = can + (site * 4 + mu) * 9;
    Cx<R> u[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 t = src[k];
      u[k] = cx((R)t.x, (R)t.y);
    }
    Link<P, C12>::store(dst + par * 4 * lb + mu * lb, vh, (int)j, u);
  }
}

template <int P, bool C12>
__global__ void k_unpack_gauge(Dims4 dm, int vh, long long s0, long long s1, const char* src,
                               double2* __restrict__ can) {
  const long long site = s0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (site >= s1) return;
  int par;
  long long j;
  site_to_eo(dm.d, site, &par, &j);
  const long long lb = (long long)Link<P, C12>::kBytes * vh;
  using R = typename Link<P, C12>::R;
  for (int mu = 0; mu < 4; ++mu) {
    Cx<R> u[9];
    Link<P, C12>::load(src + par * 4 * lb + mu * lb, vh, (int)j, u);
    double2* o = can + (site * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = make_double2((double)u[k].re, (double)u[k].im);
  }
}

// FP64 18-real links -> (P, C12) storage, checkerboard indexes [j0, j1) of
// all eight (parity, mu) planes
template <int P, bool C12>
__global__ void k_convert_gauge(int vh, long long j0, long long j1, const char* src, char* dst) {
  const long long j = j0 + blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int pm = blockIdx.y;  // parity*4 + mu
  if (j >= j1) return;
  const long long lsrc = (long long)Link<P64, false>::kBytes * vh;
  const long long ldst = (long long)Link<P, C12>::kBytes * vh;
  Cx<double> u[9];
  Link<P64, false>::load(src + pm * lsrc, vh, (int)j, u);
  using R = typename Link<P, C12>::R;
  Cx<R> v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = cx((R)u[k].re, (R)u[k].im);
  Link<P, C12>::store(dst + pm * ldst, vh, (int)j, v);
}

static Dims4 dims4(const dw_lattice& l) {
  Dims4 d;
  for (int m = 0; m < 4; ++m) d.d[m] = l.dims[m];
  return d;
}

#define DW_PREC_DISPATCH(prec, BODY)         \
  switch (prec) {                            \
    case DW_F64: { constexpr int PP = P64; BODY; } break;  \
    case DW_F32: { constexpr int PP = P32; BODY; } break;  \
    case DW_F16: { constexpr int PP = P16; BODY; } break;  \
    case DW_BF16: { constexpr int PP = PB16; BODY; } break; \
    case DW_DF64: { constexpr int PP = PDF; BODY; } break; \
    case DW_I16: { constexpr int PP = PI16; BODY; } break; \
  }

static unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

long long canonical_units(const dw_field* f) {
  const long long vh = vh_of(f->lat);
  if (f->kind == DW_GAUGE) return 2 * vh;
  return (long long)f->nrhs * vh * npar_of(f->kind);
}

size_t canonical_unit_bytes(const dw_field* f) { return f->kind == DW_GAUGE ? 4 * 9 * 16 : 12 * 16; }

dw_status pack_range(dw_field* f, const double* can, long long u0, long long u1, cudaStream_t st) {
  if (u1 <= u0) return DW_OK;
  const int vh = (int)vh_of(f->lat);
  const double2* c = reinterpret_cast<const double2*>(can);
  dim3 b(256), g(blocks_for(u1 - u0));
  if (f->kind == DW_GAUGE) {
    if (f->compress12) {
      DW_PREC_DISPATCH(f->prec, (count_launch(), k_pack_gauge<PP, true><<<g, b, 0, st>>>(dims4(f->lat), vh, u0, u1, c, f->ptr)));
    } else {
      DW_PREC_DISPATCH(f->prec, (count_launch(), k_pack_gauge<PP, false><<<g, b, 0, st>>>(dims4(f->lat), vh, u0, u1, c, f->ptr)));
    }
  } else {
    const int npar = npar_of(f->kind);
    const int par0 = f->kind == DW_SPINOR_ODD ? 1 : 0;
    Slot s = spinor_slot(f);
    DW_PREC_DISPATCH(f->prec, (count_launch(), k_pack_spinor<PP><<<g, b, 0, st>>>(dims4(f->lat), vh, npar, par0, u0, u1, c, s)));
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

dw_status unpack_range(const dw_field* f, double* can, long long u0, long long u1, cudaStream_t st) {
  if (u1 <= u0) return DW_OK;
  const int vh = (int)vh_of(f->lat);
  double2* c = reinterpret_cast<double2*>(can);
  dim3 b(256), g(blocks_for(u1 - u0));
  if (f->kind == DW_GAUGE) {
    if (f->compress12) {
      DW_PREC_DISPATCH(f->prec, (count_launch(), k_unpack_gauge<PP, true><<<g, b, 0, st>>>(dims4(f->lat), vh, u0, u1, f->ptr, c)));
    } else {
      DW_PREC_DISPATCH(f->prec, (count_launch(), k_unpack_gauge<PP, false><<<g, b, 0, st>>>(dims4(f->lat), vh, u0, u1, f->ptr, c)));
    }
  } else {
    const int npar = npar_of(f->kind);
    const int par0 = f->kind == DW_SPINOR_ODD ? 1 : 0;
    Slot s = spinor_slot(f);
    DW_PREC_DISPATCH(f->prec, (count_launch(), k_unpack_spinor<PP><<<g, b, 0, st>>>(dims4(f->lat), vh, npar, par0, u0, u1, s, c)));
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

static dw_status convert_links(const dw_field* U, const dw_field::Derived& d, long long j0, long long j1,
                               cudaStream_t st) {
  if (j1 <= j0) return DW_OK;
  const int vh = (int)vh_of(U->lat);
  dim3 b(256), g(blocks_for(j1 - j0), 8);
  if (d.c12) {
    DW_PREC_DISPATCH(d.prec, (count_launch(), k_convert_gauge<PP, true><<<g, b, 0, st>>>(vh, j0, j1, U->ptr, d.ptr)));
  } else {
    DW_PREC_DISPATCH(d.prec, (count_launch(), k_convert_gauge<PP, false><<<g, b, 0, st>>>(vh, j0, j1, U->ptr, d.ptr)));
  }
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}

dw_status refresh_derived_range(dw_field* U, long long s0, long long s1, cudaStream_t st) {
  if (U->kind != DW_GAUGE) return DW_OK;
  // lexicographic sites 2j and 2j+1 are the two parities of checkerboard index j
  for (auto& d : U->derived) DW_TRY(convert_links(U, d, s0 / 2, (s1 + 1) / 2, st));
  return DW_OK;
}

void mark_derived_current(dw_field* U) {
  for (auto& d : U->derived) d.version = U->version;
}

dw_status derived_links(dw_field* U, int prec, int c12, cudaStream_t st, const char** out) {
  if (prec == (int)U->prec && c12 == U->compress12) {
    *out = U->ptr;
    return DW_OK;
  }
  DW_CHECK(U->prec == DW_F64 && !U->compress12, DW_ERR_PRECISION,
           "derived link copies need an FP64 18-real gauge field");
  for (auto& d : U->derived)
    if (d.prec == prec && d.c12 == c12) {
      if (d.version != U->version) {
        DW_TRY(convert_links(U, d, 0, vh_of(U->lat), st));
        d.version = U->version;
      }
      *out = d.ptr;
      return DW_OK;
    }
  dw_field::Derived d;
  d.prec = prec;
  d.c12 = c12;
  d.bytes = 8ull * link_bytes(prec, c12) * vh_of(U->lat);
  DW_CUDA(cudaMalloc(&d.ptr, d.bytes));
  d.version = U->version - 1;  // force conversion below
  U->derived.push_back(d);
  return derived_links(U, prec, c12, st, out);
}

}  // namespace dw

namespace dw {
Profiler& profiler() {
  static Profiler p;
  return p;
}

// ------------------------------------------------------------------ autotuning cache
static std::mutex g_tune_mu;
static std::map<std::string, BlockShape>& tune_table() {
  static std::map<std::string, BlockShape> t;
  return t;
}
static std::string tune_path() {
  const char* e = getenv("DW_TUNE_CACHE");
  if (e && *e) return e;
  const char* h = getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/dwsolve/tune.txt";
}
static void tune_load_once() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  FILE* f = fopen(tune_path().c_str(), "r");
  if (!f) return;
  char line[640], key[512];
  int T, RB, pair;
  while (fgets(line, sizeof line, f)) {
    if (sscanf(line, "%511s %d %d %d", key, &T, &RB, &pair) != 4) continue;
    if (T >= 32 && T <= 256 && T % 32 == 0 && RB >= 1 && T * RB <= 256 && (pair == 0 || pair == 1)) {
      BlockShape b{T, RB};
      b.pair = pair;
      tune_table()[key] = b;
    }
  }
  fclose(f);
}
std::string tune_key(const dw_lattice* lats, int n, int nrhs, int prec, int c12) {
  char dev_name[256] = "gpu";
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    snprintf(dev_name, sizeof dev_name, "%s", prop.name);
  for (char* c = dev_name; *c; ++c)
    if (*c == ' ') *c = '_';
  std::string key = std::string(dev_name) + "/v5/" + prec_name(prec) + (c12 ? "c12" : "c18") + "/r" +
                    std::to_string(nrhs);
  for (int i = 0; i < n; ++i)
    key += "/" + std::to_string(lats[i].dims[0]) + "x" + std::to_string(lats[i].dims[1]) + "x" +
           std::to_string(lats[i].dims[2]) + "x" + std::to_string(lats[i].dims[3]);
  return key;
}
bool tune_lookup(const std::string& key, BlockShape* out) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_once();
  auto it = tune_table().find(key);
  if (it == tune_table().end()) return false;
  *out = it->second;
  return true;
}
void tune_store(const std::string& key, BlockShape v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load_once();
  tune_table()[key] = v;
  const std::string path = tune_path();
  const std::string dir = path.substr(0, path.find_last_of('/'));
  std::string cmd_dir = dir;
  // create the directory chain (best effort), then append
  for (size_t pos = 1; pos < cmd_dir.size(); ++pos)
    if (cmd_dir[pos] == '/') mkdir(cmd_dir.substr(0, pos).c_str(), 0755);
  mkdir(cmd_dir.c_str(), 0755);
  FILE* f = fopen(path.c_str(), "a");
  if (f) {
    fprintf(f, "%s %d %d %d\n", key.c_str(), v.T, v.RB, v.pair);
    fclose(f);
  }
}

static constexpr size_t kSolveCacheMax = 4;
static std::list<SolveCacheEntry>& solve_cache() {
  static std::list<SolveCacheEntry> c;
  return c;
}

SolveCacheEntry* solve_cache_find(const std::vector<unsigned long long>& key) {
  auto& c = solve_cache();
  for (auto it = c.begin(); it != c.end(); ++it)
    if (it->key == key) {
      c.splice(c.begin(), c, it);
      return &c.front();
    }
  return nullptr;
}

SolveCacheEntry* solve_cache_insert(SolveCacheEntry&& e) {
  auto& c = solve_cache();
  c.push_front(std::move(e));
  while (c.size() > kSolveCacheMax) {
    SolveCacheEntry& old = c.back();
    cudaDeviceSynchronize();
    if (old.exec) cudaGraphExecDestroy(old.exec);
    if (old.arena) cudaFree(old.arena);
    c.pop_back();
  }
  return &c.front();
}
}  // namespace dw

using namespace dw;

extern "C" {

const char* dw_last_error(void) { return g_err; }

dw_status dw_profile_start(int time_stencils) {
  Profiler& p = profiler();
  p.on = true;
  p.timing = time_stencils != 0;
  p.launches = 0;
  p.recs.clear();
  p.next = 0;
  return DW_OK;
}

dw_status dw_profile_stop(dw_profile_entry* out, int max_entries, int* n_entries, long long* launches) {
  Profiler& p = profiler();
  DW_CUDA(cudaDeviceSynchronize());
  std::vector<dw_profile_entry> agg(p.names.size());
  for (size_t i = 0; i < agg.size(); ++i) {
    memset(&agg[i], 0, sizeof agg[i]);
    snprintf(agg[i].name, sizeof agg[i].name, "%s", p.names[i].c_str());
  }
  for (auto& r : p.recs) {
    float ms = 0.f;
    DW_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    dw_profile_entry& e = agg[r.cat];
    e.launches += 1;
    e.total_ms += ms;
    e.bytes += r.bytes;
    e.flops += r.flops;
  }
  int n = 0;
  for (auto& e : agg)
    if (e.launches > 0) {
      if (out && n < max_entries) out[n] = e;
      ++n;
    }
  if (n_entries) *n_entries = n;
  if (launches) *launches = p.launches;
  p.on = false;
  p.timing = false;
  p.recs.clear();
  p.next = 0;
  return DW_OK;
}

const char* dw_version(void) { return "dw 1.0 (sm_103a)"; }

dw_status dw_field_bytes(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs,
                         size_t* bytes) {
  DW_TRY(check_lattice(lat));
  DW_CHECK(bytes != nullptr, DW_ERR_ARG, "bytes is NULL");
  DW_CHECK(prec >= DW_F64 && prec <= DW_I16, DW_ERR_PRECISION, "unknown precision %d", (int)prec);
  DW_CHECK(kind >= DW_GAUGE && kind <= DW_SPINOR_ODD, DW_ERR_ARG, "unknown field kind %d", (int)kind);
  const long long vh = vh_of(*lat);
  if (kind == DW_GAUGE) {
    DW_CHECK(nrhs == 1 || nrhs == 0, DW_ERR_SHAPE, "gauge fields have nrhs = 1");
    *bytes = 8ull * link_bytes(prec, compress12 ? 1 : 0) * vh;
  } else {
    DW_CHECK(nrhs >= 1 && nrhs <= 64, DW_ERR_SHAPE, "nrhs %d out of range 1..64", nrhs);
    DW_CHECK(!compress12, DW_ERR_ARG, "compress12 applies to gauge fields only");
    *bytes = (size_t)nrhs * npar_of(kind) * spin_bytes(prec) * vh;
  }
  return DW_OK;
}

static dw_status make_field(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs, void* ptr,
                            size_t have, int owned, dw_field** out) {
  size_t need = 0;
  DW_TRY(dw_field_bytes(lat, kind, prec, compress12, nrhs, &need));
  DW_CHECK(out != nullptr, DW_ERR_ARG, "out is NULL");
  dw_field* f = new dw_field();
  f->lat = *lat;
  f->kind = kind;
  f->prec = prec;
  f->compress12 = compress12 ? 1 : 0;
  f->nrhs = kind == DW_GAUGE ? 1 : nrhs;
  f->bytes = need;
  f->owned = owned;
  f->version = 1;
  cudaGetDevice(&f->device);
  if (owned) {
    cudaError_t e = cudaMalloc(&f->ptr, need);
    if (e != cudaSuccess) {
      delete f;
      return cuda_error(e, "cudaMalloc(field)", __FILE__, __LINE__);
    }
  } else {
    if (ptr == nullptr || have < need || (reinterpret_cast<uintptr_t>(ptr) & 255) != 0) {
      delete f;
      return set_error(DW_ERR_ARG, "wrapped memory must be non-NULL, 256-byte aligned and >= %zu bytes", need);
    }
    f->ptr = static_cast<char*>(ptr);
  }
  *out = f;
  return DW_OK;
}

dw_status dw_field_alloc(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs,
                         dw_field** out) {
  return make_field(lat, kind, prec, compress12, nrhs, nullptr, 0, 1, out);
}

dw_status dw_field_wrap(const dw_lattice* lat, dw_kind kind, dw_prec prec, int compress12, int nrhs, void* dev_ptr,
                        size_t bytes, dw_field** out) {
  return make_field(lat, kind, prec, compress12, nrhs, dev_ptr, bytes, 0, out);
}

dw_status dw_field_mark_modified(dw_field* f) {
  DW_CHECK(f != nullptr, DW_ERR_ARG, "field is NULL");
  f->version += 1;
  return DW_OK;
}

dw_status dw_field_free(dw_field* f) {
  if (f == nullptr) return DW_OK;
  cudaDeviceSynchronize();
  for (auto& d : f->derived) cudaFree(d.ptr);
  if (f->owned) cudaFree(f->ptr);
  delete f;
  return DW_OK;
}

dw_status dw_field_info(const dw_field* f, dw_lattice* lat, dw_kind* kind, dw_prec* prec, int* compress12,
                        int* nrhs) {
  DW_CHECK(f != nullptr, DW_ERR_ARG, "field is NULL");
  if (lat) *lat = f->lat;
  if (kind) *kind = f->kind;
  if (prec) *prec = f->prec;
  if (compress12) *compress12 = f->compress12;
  if (nrhs) *nrhs = f->nrhs;
  return DW_OK;
}

dw_status dw_field_import(dw_field* f, const double* dev, dw_stream_t stream) {
  DW_CHECK(f != nullptr && dev != nullptr, DW_ERR_ARG, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  f->version += 1;
  const long long nu = canonical_units(f);
  DW_TRY(pack_range(f, dev, 0, nu, st));
  DW_TRY(refresh_derived_range(f, 0, nu, st));
  mark_derived_current(f);
  return DW_OK;
}

dw_status dw_field_export(const dw_field* f, double* dev, dw_stream_t stream) {
  DW_CHECK(f != nullptr && dev != nullptr, DW_ERR_ARG, "NULL argument");
  return unpack_range(f, dev, 0, canonical_units(f), reinterpret_cast<cudaStream_t>(stream));
}

// Staging buffers for host transfers come from a stream-ordered memory pool
// owned by the library (one per device), which keeps up to kStagingKeep bytes
// reserved between calls so that repeated transfers do not reallocate.
static constexpr uint64_t kStagingKeep = 8ull << 30;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static dw_status staging_pool(cudaMemPool_t* out) {
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  DW_CHECK(dev >= 0 && dev < 64, DW_ERR_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    DW_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = kStagingKeep;
    DW_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return DW_OK;
}

// Large host transfers run in chunks: the DMA copies go on a copy stream owned
// by the library (one per device) and the layout kernels on the caller's
// stream, so that the kernels of one chunk run under the copy of the next.
// Events order the two streams both ways, which keeps the call ordered on the
// caller's stream exactly as a single copy plus kernel would be.
static constexpr int kMaxChunks = 8;
static constexpr size_t kChunkMinBytes = 32ull << 20;
struct CopyLane {
  cudaStream_t s = nullptr;
  cudaEvent_t ev[kMaxChunks + 1] = {};
};
static std::mutex g_lane_mu;  // held while a transfer enqueues (the events are reused)
static CopyLane g_lane[64];

static dw_status copy_lane(CopyLane** out) {
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  DW_CHECK(dev >= 0 && dev < 64, DW_ERR_ARG, "device index %d out of range", dev);
  CopyLane& l = g_lane[dev];
  if (!l.s) {
    DW_CUDA(cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking));
    for (auto& e : l.ev) DW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  *out = &l;
  return DW_OK;
}

// Number of chunks for a transfer of nb bytes on stream st: one (a single copy
// and kernel on st) for small transfers and while st is being captured.
static int transfer_chunks(size_t nb, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 1;
  const size_t n = nb / kChunkMinBytes;
  return n < 2 ? 1 : (int)(n < (size_t)kMaxChunks ? n : kMaxChunks);
}

// First canonical unit of chunk k of n (gauge fields: an even site, so that a
// chunk holds both parities of each of its checkerboard indexes)
static long long chunk_start(const dw_field* f, long long nu, int k, int n) {
  long long u = nu * k / n;
  if (f->kind == DW_GAUGE) u &= ~1ll;
  return u;
}

dw_status dw_field_upload(dw_field* f, const double* host, dw_stream_t stream) {
  DW_CHECK(f != nullptr && host != nullptr, DW_ERR_ARG, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // DMA copies into a device staging buffer, then the layout kernel (and the
  // refresh of derived link copies) on the device (measured on a
  // Grace-Blackwell node: about 200 GB/s from pinned memory, against about
  // 140 GB/s for a kernel reading host memory directly)
  const long long nu = canonical_units(f);
  const size_t ub = canonical_unit_bytes(f);
  const size_t nb = (size_t)nu * ub;
  cudaMemPool_t pool;
  DW_TRY(staging_pool(&pool));
  char* tmp = nullptr;
  DW_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&tmp), nb, pool, st));
  const char* h = reinterpret_cast<const char*>(host);
  f->version += 1;
  const int n = transfer_chunks(nb, st);
  dw_status s = DW_OK;
  if (n == 1) {
    cudaError_t e = cudaMemcpyAsync(tmp, h, nb, cudaMemcpyHostToDevice, st);
    s = e == cudaSuccess ? pack_range(f, reinterpret_cast<const double*>(tmp), 0, nu, st)
                         : cuda_error(e, "cudaMemcpyAsync(host to device)", __FILE__, __LINE__);
    if (s == DW_OK) s = refresh_derived_range(f, 0, nu, st);
  } else {
    std::lock_guard<std::mutex> lock(g_lane_mu);
    CopyLane* l = nullptr;
    s = copy_lane(&l);
    cudaError_t e = cudaSuccess;
    if (s == DW_OK) e = cudaEventRecord(l->ev[0], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(l->s, l->ev[0], 0);
    for (int k = 0; k < n && s == DW_OK && e == cudaSuccess; ++k) {
      const long long u0 = chunk_start(f, nu, k, n), u1 = chunk_start(f, nu, k + 1, n);
      e = cudaMemcpyAsync(tmp + u0 * ub, h + u0 * ub, (u1 - u0) * ub, cudaMemcpyHostToDevice, l->s);
      if (e == cudaSuccess) e = cudaEventRecord(l->ev[k + 1], l->s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, l->ev[k + 1], 0);
      if (e == cudaSuccess) s = pack_range(f, reinterpret_cast<const double*>(tmp), u0, u1, st);
      if (e == cudaSuccess && s == DW_OK) s = refresh_derived_range(f, u0, u1, st);
    }
    if (l != nullptr && (s != DW_OK || e != cudaSuccess)) {
      // an error part way: the staging buffer's release still waits for the copies issued
      if (cudaEventRecord(l->ev[kMaxChunks], l->s) == cudaSuccess) cudaStreamWaitEvent(st, l->ev[kMaxChunks], 0);
    }
    if (s == DW_OK && e != cudaSuccess) s = cuda_error(e, "chunked host-to-device copy", __FILE__, __LINE__);
  }
  if (s == DW_OK) mark_derived_current(f);
  cudaFreeAsync(tmp, st);
  return s;
}

dw_status dw_field_download(const dw_field* f, double* host, dw_stream_t stream) {
  DW_CHECK(f != nullptr && host != nullptr, DW_ERR_ARG, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // layout kernel into a device staging buffer, then DMA copies (kernel
  // writes into host memory reach only about a quarter of the DMA rate)
  const long long nu = canonical_units(f);
  const size_t ub = canonical_unit_bytes(f);
  const size_t nb = (size_t)nu * ub;
  cudaMemPool_t pool;
  DW_TRY(staging_pool(&pool));
  char* tmp = nullptr;
  DW_CUDA(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&tmp), nb, pool, st));
  char* h = reinterpret_cast<char*>(host);
  const int n = transfer_chunks(nb, st);
  dw_status s = DW_OK;
  if (n == 1) {
    s = unpack_range(f, reinterpret_cast<double*>(tmp), 0, nu, st);
    if (s == DW_OK) {
      cudaError_t e = cudaMemcpyAsync(h, tmp, nb, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) s = cuda_error(e, "cudaMemcpyAsync(device to host)", __FILE__, __LINE__);
    }
  } else {
    std::lock_guard<std::mutex> lock(g_lane_mu);
    CopyLane* l = nullptr;
    s = copy_lane(&l);
    cudaError_t e = cudaSuccess;
    int issued = 0;  // chunks whose copy is on the copy stream
    for (int k = 0; k < n && s == DW_OK && e == cudaSuccess; ++k) {
      const long long u0 = chunk_start(f, nu, k, n), u1 = chunk_start(f, nu, k + 1, n);
      s = unpack_range(f, reinterpret_cast<double*>(tmp), u0, u1, st);
      if (s != DW_OK) break;
      e = cudaEventRecord(l->ev[k], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(l->s, l->ev[k], 0);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h + u0 * ub, tmp + u0 * ub, (u1 - u0) * ub, cudaMemcpyDeviceToHost, l->s);
      if (e == cudaSuccess) issued = k + 1;
    }
    // the caller's stream (and the staging buffer's release) waits for every copy issued
    if (issued > 0) {
      cudaError_t e2 = cudaEventRecord(l->ev[kMaxChunks], l->s);
      if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, l->ev[kMaxChunks], 0);
      if (e == cudaSuccess) e = e2;
    }
    if (s == DW_OK && e != cudaSuccess) s = cuda_error(e, "chunked device-to-host copy", __FILE__, __LINE__);
  }
  cudaFreeAsync(tmp, st);
  return s;
}

}  // extern "C"
