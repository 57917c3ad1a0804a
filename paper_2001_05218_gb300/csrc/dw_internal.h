// dw_internal.h -- host-side internals shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "dw.h"
#include "dw_kernels.cuh"

struct dw_field {
  dw_lattice lat;
  dw_kind kind;
  dw_prec prec;
  int compress12;
  int nrhs;
  char* ptr;
  size_t bytes;
  int owned;
  int device;
  unsigned long long version;  // bumped by every upload/import and by dw_field_mark_modified
  // gauge fields: cached copies in other storage formats (solver inner links)
  struct Derived {
    int prec, c12;
    char* ptr;
    size_t bytes;
    unsigned long long version;
  };
  std::vector<Derived> derived;
};

namespace dw {

dw_status set_error(dw_status st, const char* fmt, ...);
dw_status cuda_error(cudaError_t e, const char* what, const char* file, int line);
void clear_error();

#define DW_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return ::dw::cuda_error(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define DW_CHECK(cond, st, ...)                          \
  do {                                                   \
    if (!(cond)) return ::dw::set_error(st, __VA_ARGS__); \
  } while (0)

#define DW_TRY(expr)                   \
  do {                                 \
    dw_status s_ = (expr);             \
    if (s_ != DW_OK) return s_;        \
  } while (0)

inline long long volume_of(const dw_lattice& l) {
  return (long long)l.dims[0] * l.dims[1] * l.dims[2] * l.dims[3];
}
inline long long vh_of(const dw_lattice& l) { return volume_of(l) / 2; }

int spin_bytes(int prec);             // bytes per site of one spinor
int link_bytes(int prec, int c12);    // bytes per site per direction
dw_status check_lattice(const dw_lattice* l);
bool same_dims(const dw_lattice& a, const dw_lattice& b);
inline int npar_of(dw_kind k) { return k == DW_SPINOR_FULL ? 2 : 1; }

// Slot of a spinor field: rhs and parity strides in bytes.
Slot spinor_slot(const dw_field* f);
// Slot of a spinor arena laid out like a field of the given kind/prec.
Slot arena_slot(char* p, const dw_lattice& l, int prec, int nrhs, int npar);
// Slot of a gauge field stored at p (parity stride = 4 directions).
Slot gauge_slot(const char* p, const dw_lattice& l, int prec, int c12);
void geometry(SysDesc& S, const dw_lattice& l, int nrhs);

// Launch plan for a set of systems sharing nrhs.
struct Plan {
  Batch B;
  int pair = 0;      // 16-bit Wilson stencils: two right-hand sides per thread (k_hop_pair)
  int nsys = 0, nrhs = 1, ncols = 0;
  int partials = 0;  // doubles in the partial-sum buffer (one per block and column)
  dim3 block, grid1, grid2;  // one parity / both parities
};
// T sites per block and RB right-hand sides per block (T*RB <= 256, T a
// multiple of 32); T <= 0 or RB <= 0 selects the defaults.  Allocates nothing.
void make_plan(Plan& P, const dw_lattice* lats, int n, int nrhs, int T, int RB = 0);
inline void make_plan(Plan& P, const std::vector<dw_lattice>& lats, int nrhs, int T, int RB = 0) {
  make_plan(P, lats.data(), (int)lats.size(), nrhs, T, RB);
}
// The default block shape for nrhs right-hand sides.
void default_block_shape(int nrhs, int* T, int* RB);

// Autotuned block shape (T, RB) for the inner stencil of a batch, cached per
// (lattices, nrhs, storage, link compression, device) in memory and in the
// file named by DW_TUNE_CACHE (default ~/.cache/dwsolve/tune.txt).
struct BlockShape {
  int T, RB;
  int pair = 0;  // 16-bit stencils: each thread group takes two right-hand sides (grid.y halves)
};
bool tune_lookup(const std::string& key, BlockShape* out);
void tune_store(const std::string& key, BlockShape v);
// Key of the tuning cache: device name, storage, nrhs and every lattice.
std::string tune_key(const dw_lattice* lats, int n, int nrhs, int prec, int c12);

// Device scratch for reductions of one plan.
struct RedBuf {
  double* partial = nullptr;
  ColState* cols = nullptr;
  Flags* flags = nullptr;
};

// Gauge field copy in (prec, c12) storage, cached on the handle.
dw_status derived_links(dw_field* U, int prec, int c12, cudaStream_t st, const char** out);

// Canonical layout <-> storage over a range of canonical units: sites for
// gauge fields, (rhs, site) pairs for spinor fields (canonical_units of them,
// canonical_unit_bytes each).  can points at unit 0 of the canonical array.
long long canonical_units(const dw_field* f);
size_t canonical_unit_bytes(const dw_field* f);
dw_status pack_range(dw_field* f, const double* can, long long u0, long long u1, cudaStream_t st);
dw_status unpack_range(const dw_field* f, double* can, long long u0, long long u1, cudaStream_t st);
// Gauge fields: converts the derived link copies over canonical sites [s0, s1)
// (s0 even); mark_derived_current then records them as up to date.
dw_status refresh_derived_range(dw_field* U, long long s0, long long s1, cudaStream_t st);
void mark_derived_current(dw_field* U);

}  // namespace dw
