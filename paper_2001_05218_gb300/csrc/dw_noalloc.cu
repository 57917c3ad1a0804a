// dw_noalloc.cu -- dw_apply_noalloc: the operator application without any
// device allocation, for callers that must not allocate GPU memory at call
// time.
//
// Who needs it: code that shares the GPU with a framework whose caching
// allocator already holds nearly all device memory, code inside a latency-
// critical loop where a cudaMalloc/cudaFree would synchronise the device, and
// code with a fixed, planned memory budget.  dw_apply takes its temporary
// (the intermediate parity field of the Schur complement) from the
// stream-ordered pool; this variant takes it from one fixed array in device
// global memory instead.
//
// The array below is reserved on every GPU that loads this library, for the
// life of the process.  Every call on a device uses the same array and it
// keeps whatever the last call left in it; calls whose kernels overlap on the
// GPU (for example on two streams without an ordering between them) race on
// it.  Host code cannot pass the array's name to a kernel (in host code the
// name is only a stand-in, not a device address), so the device address is
// looked up once per device with cudaGetSymbolAddress, by the first call made
// with that device current.  Make that first call before any stream capture.
// The address is kept for the life of the process: after cudaDeviceReset the
// array lives at a new address in the new context, so a process that resets a
// device must not call this function on that device again.
#include <mutex>

#include "dw_exec.cuh"

namespace dw {

static constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB
static __device__ __align__(256) char dw_noalloc_scratch[kNoAllocScratchBytes];

static constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

static dw_status scratch_address(void** out) {
  int dev = 0;
  DW_CUDA(cudaGetDevice(&dev));
  DW_CHECK(dev >= 0 && dev < kMaxDevices, DW_ERR_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, dw_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(dw_noalloc_scratch)", __FILE__, __LINE__);
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return DW_OK;
}

template <int P, bool C12, bool DAG>
static void noalloc_launch(const Exec& E, dw_kind kind) {
  if (kind == DW_SPINOR_FULL) {
    hop<P, P, C12, DAG>(E, 2, S_LLO, InOne<P>{S_AUX0}, EpiXpay<P, P, C_MK, false>{S_AUX2, S_AUX0, G_ALL});
  } else {
    const int p = kind == DW_SPINOR_EVEN ? 0 : 1;
    hop<P, P, C12, DAG>(E, 1 - p, S_LLO, InOne<P>{S_AUX0}, EpiOut<P, C_ONE>{S_AUX1, G_ALL});
    hop<P, P, C12, DAG>(E, p, S_LLO, InOne<P>{S_AUX1}, EpiXpay<P, P, C_MK2, false>{S_AUX2, S_AUX0, G_ALL});
  }
}

}  // namespace dw

using namespace dw;

extern "C" dw_status dw_apply_noalloc(const dw_field* U, const dw_field* in, dw_field* out, int dagger,
                                      dw_stream_t stream) {
  DW_CHECK(U && in && out, DW_ERR_ARG, "NULL field");
  DW_CHECK(U->kind == DW_GAUGE, DW_ERR_ARG, "first argument must be a gauge field");
  DW_CHECK(in->kind != DW_GAUGE && out->kind == in->kind, DW_ERR_SHAPE, "in/out must be spinors of the same kind");
  DW_CHECK(same_dims(U->lat, in->lat) && same_dims(U->lat, out->lat), DW_ERR_SHAPE, "lattice dimensions differ");
  DW_CHECK(in->nrhs == out->nrhs, DW_ERR_SHAPE, "nrhs differs (%d vs %d)", in->nrhs, out->nrhs);
  DW_CHECK(U->prec == in->prec && U->prec == out->prec, DW_ERR_PRECISION,
           "gauge and spinor fields must share one storage precision");
  DW_CHECK(in->ptr != out->ptr, DW_ERR_ARG, "in and out must not alias");
  const size_t need =
      in->kind == DW_SPINOR_FULL ? 0 : (size_t)in->nrhs * spin_bytes(in->prec) * (size_t)vh_of(in->lat);
  DW_CHECK(need <= kNoAllocScratchBytes, DW_ERR_SHAPE,
           "dw_apply_noalloc needs %zu bytes of scratch for this field, more than its fixed %zu-byte array; "
           "use dw_apply", need, kNoAllocScratchBytes);
  void* scratch = nullptr;
  if (need > 0) DW_TRY(scratch_address(&scratch));

  // single-system launch plan with the default block shape (the plan builder
  // allocates nothing)
  Exec E;
  E.st = reinterpret_cast<cudaStream_t>(stream);
  make_plan(E.P, &U->lat, 1, in->nrhs, 0, 0);
  SysDesc& S = E.P.B.sd[0];
  S.f[S_LLO] = gauge_slot(U->ptr, U->lat, U->prec, U->compress12);
  S.f[S_AUX0] = spinor_slot(in);
  S.f[S_AUX2] = spinor_slot(out);
  if (scratch) S.f[S_AUX1] = arena_slot(static_cast<char*>(scratch), in->lat, in->prec, in->nrhs, 1);

  const int c12 = U->compress12;
#define DW_NOALLOC_CASE(PP)                                \
  if (c12) {                                               \
    if (dagger) noalloc_launch<PP, true, true>(E, in->kind);   \
    else noalloc_launch<PP, true, false>(E, in->kind);         \
  } else {                                                 \
    if (dagger) noalloc_launch<PP, false, true>(E, in->kind);  \
    else noalloc_launch<PP, false, false>(E, in->kind);        \
  }
  switch (in->prec) {
    case DW_F64: DW_NOALLOC_CASE(P64) break;
    case DW_F32: DW_NOALLOC_CASE(P32) break;
    case DW_F16: DW_NOALLOC_CASE(P16) break;
    case DW_BF16: DW_NOALLOC_CASE(PB16) break;
    case DW_DF64: DW_NOALLOC_CASE(PDF) break;
    case DW_I16: DW_NOALLOC_CASE(PI16) break;
  }
#undef DW_NOALLOC_CASE
  DW_CUDA(cudaGetLastError());
  return DW_OK;
}
