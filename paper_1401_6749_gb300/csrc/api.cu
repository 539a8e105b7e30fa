// Operator object, status/error reporting, launch counting, Dslash tracing and
// the tm_dslash entry point.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "tm_host.h"

namespace tml {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

static thread_local int t_capturing = 0;
static thread_local int t_captured = 0;

void count_launch(int n) {
  if (t_capturing) t_captured += n;
  else g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed);
}

void capture_begin() {
  t_capturing = 1;
  t_captured = 0;
}

int capture_end() {
  t_capturing = 0;
  return t_captured;
}

tm_status_t check_launch(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

tm_status_t check_geom(const int L[4]) {
  long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (L[i] < 2 || (L[i] & 1)) {
      set_error("lattice extent L[%d] = %d must be even and >= 2", i, L[i]);
      return TM_ERR_ARG;
    }
    V *= L[i];
  }
  if (V > (1L << 30)) {
    set_error("lattice volume %ld exceeds 2^30 sites", V);
    return TM_ERR_ARG;
  }
  return TM_OK;
}

// ------------------------------------------------------------ tracing
struct TraceRec {
  std::string name;
  cudaEvent_t a, b;
  int slot;        // device counter of active systems, or -1
  double bytes_per_rhs, fixed_bytes;
  int nrhs;        // systems counted as active when slot < 0
  double flops_per_rhs;
};
static std::mutex g_trace_mu;
static std::atomic<int> g_trace_on{0};
static std::vector<TraceRec> g_trace;
static int* g_trace_counts = nullptr;  // device: active systems per traced launch
static int g_trace_next = 0;
constexpr int kTraceSlots = 1 << 20;

static thread_local int t_tuning = 0;  // launches timed by the autotuner are not traced

int* trace_begin(cudaStream_t s, cudaEvent_t* ev0) {
  *ev0 = nullptr;
  if (t_capturing || t_tuning || !g_trace_on.load(std::memory_order_relaxed)) return nullptr;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_counts || g_trace_next >= kTraceSlots) return nullptr;
  if (cudaEventCreate(ev0) != cudaSuccess) { *ev0 = nullptr; return nullptr; }
  cudaEventRecord(*ev0, s);
  return g_trace_counts + g_trace_next++;  // slot reserved for this launch
}

void trace_end(cudaStream_t s, const char* name, cudaEvent_t ev0, int* slot, double bytes_per_rhs,
               double fixed_bytes, int nrhs_if_uncounted, double flops_per_rhs) {
  if (!ev0) return;
  cudaEvent_t ev1;
  if (cudaEventCreate(&ev1) != cudaSuccess) { cudaEventDestroy(ev0); return; }
  cudaEventRecord(ev1, s);
  std::lock_guard<std::mutex> lk(g_trace_mu);
  const int sl = slot ? (int)(slot - g_trace_counts) : -1;
  g_trace.push_back({name, ev0, ev1, sl, bytes_per_rhs, fixed_bytes, nrhs_if_uncounted, flops_per_rhs});
}

// Systems per thread of the FP32/FP16/BF16 Dslash (a tuning knob; results do
// not depend on it): TM_DSLASH_NR = 1, 2, 4 fixes them, "2p" two systems in
// packed FP32x2 arithmetic (returned as -2); unset leaves the choice to the
// autotuner.
int dslash_nr_override() {
  static const int v = [] {
    const char* e = getenv("TM_DSLASH_NR");
    if (!e) return 0;
    if (strcmp(e, "2p") == 0) return -2;
    const int n = atoi(e);
    return (n == 1 || n == 2 || n == 4) ? n : 0;
  }();
  return v;
}

// The FP16/BF16 Dslash with 18-real links on the tensor cores: off unless the
// environment sets TM_DSLASH_MMA=1; tm_dslash_mma_enable switches it at run
// time (it is slower than the CUDA-core kernel at the sizes measured).
static std::atomic<int> g_mma{-1};  // -1: not read from the environment yet

bool dslash_mma_on() {
  int v = g_mma.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("TM_DSLASH_MMA");
    v = (e && strcmp(e, "1") == 0) ? 1 : 0;
    int expect = -1;
    g_mma.compare_exchange_strong(expect, v);
    v = g_mma.load(std::memory_order_relaxed);
  }
  return v == 1;
}

static tm_status_t prepare_mma() {
  static const tm_status_t prep =
      dslash_mma_prepare<__half>() == TM_OK ? dslash_mma_prepare<__nv_bfloat16>() : TM_ERR_CUDA;
  return prep;
}

// ------------------------------------------------------------ autotuning
// Process-wide cache of the chosen Dslash launch shapes.  TM_TUNE=0 disables
// tuning (the built-in shape is used); tm_tune_enable overrides at run time.
bool TuneKey::operator<(const TuneKey& o) const {
  return std::tie(prec, recon, dag, epi, parity, centre, out_inv, vh, nrhs) <
         std::tie(o.prec, o.recon, o.dag, o.epi, o.parity, o.centre, o.out_inv, o.vh, o.nrhs);
}

static std::mutex g_tune_mu;
static std::map<TuneKey, TuneCfg> g_tune;
static std::atomic<int> g_tune_on{-1};

static bool tune_on() {
  int v = g_tune_on.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("TM_TUNE");
    v = (e && atoi(e) == 0) ? 0 : 1;
    g_tune_on.store(v, std::memory_order_relaxed);
  }
  return v == 1;
}

bool tune_active() { return !t_capturing && tune_on(); }

bool tune_lookup(const TuneKey& k, TuneCfg* c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *c = it->second;
  return true;
}

void tune_store(const TuneKey& k, const TuneCfg& c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[k] = c;
}

void tuning_begin() { ++t_tuning; }
void tuning_end() { --t_tuning; }

// ------------------------------------------------------------ memory
// One stream-ordered pool per device for everything the library allocates on
// it.  Its release threshold is unbounded, so memory freed by one operator or
// call stays mapped and the next allocation of similar size is served without
// the driver mapping fresh pages (cudaMalloc/cudaFree of the gigabytes an
// operator and its solver hold cost tens of milliseconds and synchronise the
// device).  tm_mem_trim hands the unused part back.
static std::mutex g_mem_mu;
static std::map<int, cudaMemPool_t> g_pools;
static std::multimap<int, int*> g_pinned;  // free pinned blocks by size (ints)

static tm_status_t pool_of_current_device(cudaMemPool_t* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    set_error("no CUDA device");
    return TM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mem_mu);
  auto it = g_pools.find(dev);
  if (it == g_pools.end()) {
    cudaMemPoolProps pr;
    memset(&pr, 0, sizeof pr);
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t pool;
    if (cudaMemPoolCreate(&pool, &pr) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMemPoolCreate failed on device %d", dev);
      return TM_ERR_CUDA;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    it = g_pools.emplace(dev, pool).first;
  }
  *out = it->second;
  return TM_OK;
}

tm_status_t dev_alloc(void** p, size_t bytes, cudaStream_t s, const char* what) {
  *p = nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  cudaError_t e;
  if (cs != cudaStreamCaptureStatusNone) {
    // inside a caller's graph capture: a graph memory node of the default pool
    e = cudaMallocAsync(p, bytes, s);
  } else {
    cudaMemPool_t pool;
    TM_TRY(pool_of_current_device(&pool));
    e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("%s: allocation of %zu bytes of device memory failed", what, bytes);
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int* pinned_take(int n, int* got) {
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    auto it = g_pinned.lower_bound(n);
    if (it != g_pinned.end()) {
      int* p = it->second;
      *got = it->first;
      g_pinned.erase(it);
      return p;
    }
  }
  int* p = nullptr;
  if (cudaMallocHost(&p, sizeof(int) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    *got = 0;
    return nullptr;
  }
  *got = n;
  return p;
}

void pinned_give(int* p, int n) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mem_mu);
  g_pinned.emplace(n, p);
}

// ------------------------------------------------------------ dispatch
tm_status_t dslash_dispatch(const tm_op* op, tm_prec_t prec, const DslashCall& c, cudaStream_t s) {
  if (c.il) return dslash_il_dispatch(op, prec, c, s);
  const bool r12 = (int)prec >= 0 && (int)prec < kNumPrec && op->recon_p[prec] == 12;
  switch (prec) {
    case TM_PREC_F64: return dslash_launch<double, 18>(op, c, s);
    case TM_PREC_FF: return dslash_launch<FFloat, 18>(op, c, s);
    case TM_PREC_F32: return r12 ? dslash_launch<float, 12>(op, c, s) : dslash_launch<float, 18>(op, c, s);
    case TM_PREC_F16: return r12 ? dslash_launch<__half, 12>(op, c, s) : dslash_launch<__half, 18>(op, c, s);
    case TM_PREC_BF16:
      return r12 ? dslash_launch<__nv_bfloat16, 12>(op, c, s) : dslash_launch<__nv_bfloat16, 18>(op, c, s);
    default: set_error("unknown precision %d", (int)prec); return TM_ERR_ARG;
  }
}

size_t link_bytes(const Geom& g, tm_prec_t p, int recon);
tm_status_t pack_links(const Geom& g, tm_prec_t p, int recon, void* out, const double* U,
                       cudaStream_t s);

}  // namespace tml

using namespace tml;

extern "C" const char* tm_last_error(void) { return g_last_error.c_str(); }
extern "C" uint64_t tm_launch_count(void) { return g_launches.load(); }

extern "C" tm_status_t tm_dslash_mma_enable(int on) {
  if (on) TM_TRY(prepare_mma());
  g_mma.store(on ? 1 : 0, std::memory_order_relaxed);
  return TM_OK;
}

extern "C" void tm_tune_enable(int on) { g_tune_on.store(on ? 1 : 0, std::memory_order_relaxed); }

extern "C" void tm_tune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

extern "C" int tm_tune_count(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}

extern "C" tm_status_t tm_tune_get(int i, int* key, int* nr, int* block, int* packed) {
  if (!key || !nr || !block || !packed) { set_error("tm_tune_get: null argument"); return TM_ERR_ARG; }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (i < 0 || i >= (int)g_tune.size()) { set_error("tm_tune_get: index %d out of range", i); return TM_ERR_ARG; }
  auto it = g_tune.begin();
  std::advance(it, i);
  const TuneKey& k = it->first;
  const int v[9] = {k.prec, k.recon, k.dag, k.epi, k.parity, k.centre, k.out_inv, k.vh, k.nrhs};
  for (int j = 0; j < 9; ++j) key[j] = v[j];
  *nr = it->second.nr;
  *block = it->second.bx;
  *packed = it->second.packed;
  return TM_OK;
}

extern "C" void tm_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (on && !g_trace_counts) {
    if (cudaMalloc(&g_trace_counts, sizeof(int) * kTraceSlots) != cudaSuccess) {
      cudaGetLastError();
      g_trace_counts = nullptr;
      set_error("tm_trace_enable: could not allocate the trace counters");
      return;
    }
  }
  g_trace_on.store(on ? 1 : 0);
}

extern "C" void tm_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (auto& r : g_trace) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_trace.clear();
  g_trace_next = 0;
}

static tm_status_t trace_sum(const char* name, int* launches, double* total_ms, double* total_bytes,
                             double* total_flops) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  std::vector<int> counts((size_t)g_trace_next);
  if (g_trace_next > 0) {
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(counts.data(), g_trace_counts, sizeof(int) * counts.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error("tm_trace_read: reading the trace counters failed");
      return TM_ERR_CUDA;
    }
  }
  int n = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
  // exact class name, or a prefix followed by '*'
  const std::string want(name);
  const bool prefix = !want.empty() && want.back() == '*';
  const std::string stem = prefix ? want.substr(0, want.size() - 1) : want;
  for (auto& r : g_trace) {
    if (prefix ? r.name.compare(0, stem.size(), stem) != 0 : r.name != want) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) { set_error("tm_trace_read: event sync failed"); return TM_ERR_CUDA; }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { set_error("tm_trace_read: elapsed time failed"); return TM_ERR_CUDA; }
    ms += t;
    const int act = r.slot < 0 ? r.nrhs : (r.slot < (int)counts.size() ? counts[r.slot] : 0);
    bytes += act > 0 ? act * r.bytes_per_rhs + r.fixed_bytes : 0.0;
    flops += act * r.flops_per_rhs;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  *total_bytes = bytes;
  if (total_flops) *total_flops = flops;
  return TM_OK;
}

extern "C" tm_status_t tm_trace_read(const char* name, int* launches, double* total_ms,
                                     double* total_bytes) {
  if (!name || !launches || !total_ms || !total_bytes) { set_error("tm_trace_read: null argument"); return TM_ERR_ARG; }
  return trace_sum(name, launches, total_ms, total_bytes, nullptr);
}

extern "C" tm_status_t tm_trace_read_flops(const char* name, double* total_flops) {
  if (!name || !total_flops) { set_error("tm_trace_read_flops: null argument"); return TM_ERR_ARG; }
  int n = 0;
  double ms = 0.0, bytes = 0.0;
  return trace_sum(name, &n, &ms, &bytes, total_flops);
}

namespace tml {
// One pass of the SMs over page-locked host memory into device memory (16-byte
// words, grid-stride).  Right after sustained GPU load the copy engine's first
// host-to-device transfer runs several times slower than these reads.
__global__ void pull_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
}  // namespace tml

// U_lex in page-locked host memory: pull it into a staging buffer of the pool
// (*staged, freed by the caller in stream order) and point *U at it; device
// memory passes through; other memory is an argument error.
static tm_status_t stage_links(const double* U_lex, size_t bytes, const double** U, double** staged,
                               cudaStream_t st) {
  *U = U_lex;
  *staged = nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, U_lex) != cudaSuccess) {
    cudaGetLastError();
    at.type = cudaMemoryTypeUnregistered;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return TM_OK;
  if (at.type != cudaMemoryTypeHost) {
    set_error("tm_op_create: U_lex must be device memory or page-locked host memory");
    return TM_ERR_ARG;
  }
  const void* src = at.devicePointer ? at.devicePointer : U_lex;
  if (reinterpret_cast<uintptr_t>(src) & 15u) {
    set_error("tm_op_create: page-locked host U_lex must be 16-byte aligned");
    return TM_ERR_ARG;
  }
  TM_TRY(dev_alloc((void**)staged, bytes, st, "tm_op_create"));
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
  pull_kernel<<<(unsigned)nsm * 8u, 256, 0, st>>>(static_cast<const uint4*>(src), reinterpret_cast<uint4*>(*staged),
                                                  bytes / 16);
  count_launch();
  const tm_status_t r = check_launch("tm_op_create: host links");
  if (r != TM_OK) {
    dev_free(*staged, st);
    *staged = nullptr;
    return r;
  }
  *U = *staged;
  return TM_OK;
}

extern "C" tm_status_t tm_op_create(tm_op_t** out, const tm_params_t* p, const double* U_lex,
                                    tm_stream_t s) {
  if (!out || !p || !U_lex) { set_error("tm_op_create: null argument"); return TM_ERR_ARG; }
  *out = nullptr;
  if (check_geom(p->L) != TM_OK) return TM_ERR_ARG;
  if (p->recon != 0 && p->recon != 12 && p->recon != 18) {
    set_error("recon must be 0, 12 or 18, got %d", p->recon);
    return TM_ERR_ARG;
  }
  if (dslash_mma_on()) {
    const tm_status_t prep = prepare_mma();
    if (prep != TM_OK) return prep;
  }
  tm_op* op = new tm_op();
  op->g = make_geom(p->L, p->antiperiodic_t ? 1 : 0);
  op->kappa = p->kappa;
  op->mu = p->mu;
  // per precision; F64 always stores the full matrix
  op->recon_p[TM_PREC_F64] = 18;
  op->recon_p[TM_PREC_FF] = 18;
  op->recon_p[TM_PREC_F32] = p->recon ? p->recon : 12;
  op->recon_p[TM_PREC_F16] = p->recon ? p->recon : 18;
  op->recon_p[TM_PREC_BF16] = p->recon ? p->recon : 18;
  op->work = nullptr;
  op->work_bytes = 0;
  op->host_flags = nullptr;
  op->host_flags_n = 0;
  op->owns_links = true;
  for (int i = 0; i < kNumPrec; ++i) op->links[i] = op->links_il[i] = nullptr;
  op->il_err = nullptr;
  const cudaStream_t st = (cudaStream_t)s;
  const double* U = nullptr;
  double* staged = nullptr;
  {
    const size_t ubytes = 4 * 2 * (size_t)op->g.Vh * 18 * sizeof(double);
    const tm_status_t ss = stage_links(U_lex, ubytes, &U, &staged, st);
    if (ss != TM_OK) { tm_op_destroy(op); return ss; }
  }
  for (int i = 0; i < kNumPrec; ++i) {
    const tm_prec_t pr = (tm_prec_t)i;
    const size_t nb = link_bytes(op->g, pr, op->recon_p[i]);
    const tm_status_t sa = dev_alloc(&op->links[i], nb, st, "tm_op_create");
    if (sa != TM_OK) { dev_free(staged, st); tm_op_destroy(op); return sa; }
    const tm_status_t st2 = pack_links(op->g, pr, op->recon_p[i], op->links[i], U, st);
    if (st2 != TM_OK) { dev_free(staged, st); tm_op_destroy(op); return st2; }
    // the interleaved (tensor-core) Dslash reads the 16-bit links site-major
    if ((pr == TM_PREC_F16 || pr == TM_PREC_BF16) && op->recon_p[i] == 18) {
      tm_status_t s3 = dev_alloc(&op->links_il[i], il_link_bytes(op->g), st, "tm_op_create");
      if (s3 == TM_OK) s3 = il_pack_links(op->g, op->links_il[i], op->links[i], st);
      if (s3 != TM_OK) { dev_free(staged, st); tm_op_destroy(op); return s3; }
      if (!op->il_err) {
        s3 = dev_alloc((void**)&op->il_err, sizeof(int), st, "tm_op_create");
        if (s3 == TM_OK && cudaMemsetAsync(op->il_err, 0, sizeof(int), st) != cudaSuccess) {
          set_error("tm_op_create: %s", cudaGetErrorString(cudaGetLastError()));
          s3 = TM_ERR_CUDA;
        }
        if (s3 != TM_OK) { dev_free(staged, st); tm_op_destroy(op); return s3; }
      }
    }
  }
  dev_free(staged, st);  // stream-ordered: after the packing that reads it
  if (op->il_err) {
    tm_status_t s4 = il_prepare();
    if (s4 == TM_OK) s4 = oned_il_prepare();
    if (s4 != TM_OK) { tm_op_destroy(op); return s4; }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("tm_op_create: %s", cudaGetErrorString(cudaGetLastError()));
    tm_op_destroy(op);
    return TM_ERR_CUDA;
  }
  *out = op;
  return TM_OK;
}

extern "C" tm_status_t tm_op_clone(tm_op_t** out, const tm_op_t* src) {
  if (!out || !src) { set_error("tm_op_clone: null argument"); return TM_ERR_ARG; }
  tm_op* op = new tm_op();
  *op = *src;
  op->work = nullptr;
  op->work_bytes = 0;
  op->host_flags = nullptr;
  op->host_flags_n = 0;
  op->owns_links = false;
  op->cg_graph = tm_cg_graph_cache{};  // the source's graph stays its own
  *out = op;
  return TM_OK;
}

extern "C" tm_status_t tm_op_destroy(tm_op_t* op) {
  if (!op) return TM_OK;
  // no work of the operator may still run: wait for the device (as cudaFree
  // would), then return the memory to the pool and wait for that too, so
  // that the next allocation on any stream can reuse it at once
  cudaDeviceSynchronize();
  for (int i = 0; i < kNumPrec; ++i)
    if (op->owns_links) {
      dev_free(op->links[i], nullptr);
      dev_free(op->links_il[i], nullptr);
    }
  if (op->owns_links) dev_free(op->il_err, nullptr);
  if (op->cg_graph.exec) cudaGraphExecDestroy(op->cg_graph.exec);
  dev_free(op->work, nullptr);
  cudaStreamSynchronize(nullptr);
  pinned_give(op->host_flags, op->host_flags_n);
  delete op;
  return TM_OK;
}

extern "C" tm_status_t tm_mem_trim(size_t keep_bytes) {
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("tm_mem_trim: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mem_mu);
  for (auto& kv : g_pools) cudaMemPoolTrimTo(kv.second, keep_bytes);
  for (auto& kv : g_pinned) cudaFreeHost(kv.second);
  g_pinned.clear();
  return TM_OK;
}

extern "C" tm_status_t tm_mem_reserved(size_t* bytes) {
  if (!bytes) { set_error("tm_mem_reserved: null argument"); return TM_ERR_ARG; }
  *bytes = 0;
  cudaMemPool_t pool;
  TM_TRY(pool_of_current_device(&pool));
  uint64_t v = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess) {
    set_error("tm_mem_reserved: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  *bytes = (size_t)v;
  return TM_OK;
}

extern "C" tm_status_t tm_dslash(tm_op_t* op, void* out, const void* in, int nrhs, int dagger,
                                 int mu_zero, tm_prec_t prec, tm_stream_t s) {
  if (!op || !out || !in || nrhs < 0) { set_error("tm_dslash: null argument"); return TM_ERR_ARG; }
  if (out == in) { set_error("tm_dslash: out and in must not overlap"); return TM_ERR_ARG; }
  if (nrhs == 0) return TM_OK;
  DslashCall c;
  c.in = in;
  c.out = out;
  c.nrhs = nrhs;
  c.dagger = dagger != 0;
  c.mu_zero = mu_zero != 0;
  c.epi = EPI_OUT;
  return dslash_dispatch(op, prec, c, (cudaStream_t)s);
}

extern "C" tm_status_t tm_dslash_g5(tm_op_t* op, void* out, const void* in, int nrhs, int dagger,
                                    int mu_zero, tm_prec_t prec, tm_stream_t s) {
  if (!op || !out || !in || nrhs < 0) { set_error("tm_dslash_g5: null argument"); return TM_ERR_ARG; }
  if (out == in) { set_error("tm_dslash_g5: out and in must not overlap"); return TM_ERR_ARG; }
  if (nrhs == 0) return TM_OK;
  DslashCall c;
  c.in = in;
  c.out = out;
  c.nrhs = nrhs;
  c.dagger = dagger != 0;
  c.mu_zero = mu_zero != 0;
  c.g5_out = true;
  c.epi = EPI_OUT;
  return dslash_dispatch(op, prec, c, (cudaStream_t)s);
}
