// loop_contract_local_noalloc: the local loop contraction without any device
// allocation.  Its two-stage reduction keeps the per-block partial sums in a
// fixed array that lives in the library's own device image instead of in
// stream-ordered scratch, so a call allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU on which the
// library is loaded holds kNoAllocScratchDoubles doubles (8 MiB) of it until
// the process exits.  Host code may not use the variable's name as a device
// address (it names a host-side shadow), so the device address is looked up
// once per device with cudaGetSymbolAddress and passed to the kernels.
#include <mutex>

#include "tm_host.h"

namespace tml {

size_t local_scratch_bytes(const Geom& g, int nrhs);
tm_status_t local_contract_into(const Geom& g, const void* left, const void* right, tm_prec_t prec,
                                int nrhs, int p_g5, double* out, double* scratch, cudaStream_t s);

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call for that device).
static tm_status_t noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("loop_contract_local_noalloc: cudaGetDevice failed: %s",
              cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("loop_contract_local_noalloc: device ordinal %d out of range", dev);
    return TM_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_error("loop_contract_local_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return TM_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return TM_OK;
}

}  // namespace tml

using namespace tml;

extern "C" tm_status_t loop_contract_local_noalloc(const tm_geom_t* gg, const void* left,
                                                   const void* right, tm_prec_t prec, int nrhs,
                                                   tm_loop_mode_t mode, double* out,
                                                   tm_stream_t strm) {
  if (!gg || !left || !right || !out || nrhs < 0) {
    set_error("loop_contract_local_noalloc: null argument");
    return TM_ERR_ARG;
  }
  if (mode != TM_LOOP_STD && mode != TM_LOOP_VV && mode != TM_LOOP_GEN) {
    set_error("loop_contract_local_noalloc: unknown mode %d", (int)mode);
    return TM_ERR_ARG;
  }
  if ((unsigned)prec >= (unsigned)kNumPrec) {
    set_error("loop_contract_local_noalloc: unknown precision %d", (int)prec);
    return TM_ERR_ARG;
  }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  if (nrhs > 65535) {
    set_error("loop_contract_local_noalloc: nrhs must be <= 65535");
    return TM_ERR_ARG;
  }
  if (2 * gg->L[3] > 65535) {
    set_error("loop_contract_local_noalloc: T = %d exceeds the launch grid (2 T <= 65535)", gg->L[3]);
    return TM_ERR_ARG;
  }
  const Geom g = make_geom(gg->L, 1);
  const size_t need = local_scratch_bytes(g, nrhs);
  if (need > kNoAllocScratchDoubles * sizeof(double)) {
    set_error("loop_contract_local_noalloc: needs %zu bytes of scratch, the fixed array holds %zu "
              "(64 * nrhs * T * ceil(X*Y*Z/2048) doubles must be <= 2^20)",
              need, kNoAllocScratchDoubles * sizeof(double));
    return TM_ERR_ARG;
  }
  double* scratch = nullptr;
  const tm_status_t st = noalloc_scratch(&scratch);
  if (st != TM_OK) return st;
  // Every scratch element the final kernel reads is written earlier in the
  // same call, so stale contents from a previous call need no clearing.
  return local_contract_into(g, left, right, prec, nrhs, mode != TM_LOOP_STD, out, scratch,
                             (cudaStream_t)strm);
}
