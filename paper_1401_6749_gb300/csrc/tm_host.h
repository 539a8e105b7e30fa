// Host-side internals of the tmloops library: the operator object, the
// Dslash call descriptor shared by the operator and the solver, and the
// per-precision launch entry points.
#pragma once

#include <cstddef>

#include "tm_core.cuh"

// The CUDA graph of a single-set solve's iterations between two polls, kept by
// the operator for the next solve whose captured launches would be the same
// (cg.cu): same work space, solution and flag buffers, systems, parameters.
struct tm_cg_graph_key {
  const void* x;
  const void* xs;
  const void* work;
  size_t work_bytes;
  const int* host_flags;
  int nrhs, k, il;
  double tol, delta;
  int max_iter, mode, prec, inner_prec, check_every, true_residual, schur, ru_prec;
};
struct tm_cg_graph_cache {
  bool valid;
  tm_cg_graph_key key;
  cudaGraphExec_t exec;
  int per_replay;  // kernel launches in one replay
};

struct tm_op {
  tml::Geom g;
  double kappa;
  double mu;
  int recon_p[tml::kNumPrec];  // link format (12 or 18 reals) of the copy of each precision
  void* links[tml::kNumPrec];  // indexed by tm_prec_t; F64 and FF always 18-real
  // solver work space, grown on demand, owned by the operator
  void* work;
  size_t work_bytes;
  // pinned host mirror of the solver's per-system flags
  int* host_flags;
  int host_flags_n;
  bool owns_links;    // false for clones, which share the links of their source
  // F16/BF16 links in the site-major layout of the interleaved Dslash
  // ([par][cb][mu][9 words + 3 zero], 48 bytes per direction), when the
  // 18-real copy exists; null otherwise
  void* links_il[tml::kNumPrec];
  // device flag: a bounded wait of the interleaved Dslash gave up (shared by clones)
  int* il_err;
  // the last single-set solve's iteration graph (owned; not shared by clones)
  tm_cg_graph_cache cg_graph;
};

namespace tml {

// Dslash launch-shape autotuning (cache in api.cu; selection in dslash.cuh)
int dslash_nr_override();
bool dslash_mma_on();  // FP16/BF16 with 18-real links on the tensor cores (api.cu)
struct TuneKey {
  int prec, recon, dag, epi, parity, centre, out_inv, vh, nrhs;
  bool operator<(const TuneKey& o) const;
};
struct TuneCfg {
  int nr, bx;
  int packed;  // 1: two systems per thread in packed FP32x2 arithmetic
};
bool tune_lookup(const TuneKey& k, TuneCfg* c);
void tune_store(const TuneKey& k, const TuneCfg& c);
bool tune_active();   // tuning enabled and this thread not capturing a graph
void tuning_begin();  // launches between these are timing runs (not traced)
void tuning_end();

#define TM_TRY(x)               \
  do {                          \
    const tm_status_t _s = (x); \
    if (_s != TM_OK) return _s; \
  } while (0)

// Device memory of the library (gauge-link copies, solver work spaces,
// contraction and HPE scratch): a stream-ordered pool of its own per device
// that keeps freed memory mapped for the next allocation (api.cu).
// dev_alloc reports failures through set_error with `what` in the message.
tm_status_t dev_alloc(void** p, size_t bytes, cudaStream_t s, const char* what);
void dev_free(void* p, cudaStream_t s);
// Pinned host blocks of at least n ints for the solver's flag mirrors, kept
// for reuse when given back.
int* pinned_take(int n, int* got);
void pinned_give(int* p, int n);

enum Epi { EPI_OUT = 0, EPI_CGUPD = 1, EPI_RESID = 2 };

// One Dslash application over nrhs fields, with an optional fused epilogue.
//   EPI_OUT   : out = D in;                 partial |out|^2 if partial != null
//   EPI_CGUPD : q = D in (not stored); r -= alpha q; x += alpha p;  partial |r|^2
//   EPI_RESID : out = b - D in;             partial |out|^2
// D = M, M^dag (dagger) or D_W (mu_zero).  Systems with active[rhs] == 0
// are skipped entirely (no stores, zero partial).  Partial sums are written
// per warp of 32 consecutive checkerboard sites: partial[(rhs*2 + par)*nwarp + cb/32].
struct DslashCall {
  const void* in = nullptr;
  void* out = nullptr;
  int nrhs = 1;
  bool dagger = false;
  bool mu_zero = false;
  // general form (custom = true): out = T_out(T_c(cfield) + hop_scale * H in)
  //   centre: 0 no centre term, 1 identity, 2 A = 1 + i nu g5;  out_inv: T_out = A^-1
  // default (custom = false): full M / M^dag / D_W on both parities
  bool custom = false;
  double nu = 0.0;
  double hop_scale = 0.0;
  int centre = 2;
  const void* cfield = nullptr;
  bool out_inv = false;
  bool g5_out = false;  // EPI_OUT: store gamma_5 times the result
  int parity = -1;  // output parity (0 even, 1 odd) or -1 for both
  int epi = EPI_OUT;
  double* partial = nullptr;
  const int* active = nullptr;
  const double* alpha = nullptr;
  const void* p = nullptr;
  void* x = nullptr;
  void* r = nullptr;
  const void* b = nullptr;
  bool il = false;  // fields in the system-interleaved 16-bit layout (dslash_il.cu)
};

inline int nwarp_of(const Geom& g) { return (g.Vh + 31) / 32; }

template <class S, int RECON>
tm_status_t dslash_launch(const tm_op* op, const DslashCall& c, cudaStream_t s);
// one-time set-up of the tensor-core Dslash kernels of a 16-bit format
// (their shared-memory limit); tm_op_create calls it outside any capture
template <class S>
tm_status_t dslash_mma_prepare();

tm_status_t dslash_dispatch(const tm_op* op, tm_prec_t prec, const DslashCall& c, cudaStream_t s);

// System-interleaved 16-bit layout (dslash_il.cu): bytes of nrhs systems,
// the tensor-core Dslash on it, conversions from/to the standard layout and
// the solver's BLAS on it; cg_il_on: the plain F16/BF16 solver runs on it.
size_t il_bytes(const Geom& g, int nrhs);
tm_status_t dslash_il_dispatch(const tm_op* op, tm_prec_t prec, const DslashCall& c, cudaStream_t s);
tm_status_t il_convert(const Geom& g, void* out, const void* in, int nrhs, bool to_il, cudaStream_t s);
tm_status_t il_xpay(const Geom& g, tm_prec_t prec, void* p, const void* r, const double* beta,
                    const int* active, int nrhs, int par0, int npar, cudaStream_t s);
tm_status_t il_twist(const Geom& g, tm_prec_t prec, void* out, const void* in, double nu, int inverse, int par,
                     int nrhs, cudaStream_t s);
bool cg_il_on();
size_t il_link_bytes(const Geom& g);
tm_status_t il_pack_links(const Geom& g, void* out, const void* links18, cudaStream_t s);
tm_status_t il_prepare();

// Loop contractions on the interleaved layout (loops_il.cu): set-up of the
// one-derivative kernel (its shared-memory limit), and the final reductions
// of the partial sums [rhs][t][par][chunk][32 | 128] (contract.cu).
tm_status_t oned_il_prepare();
tm_status_t local_final(const double* partial, int nchunk, const Geom& g, int nrhs, int p_g5, double* out,
                        cudaStream_t s);
tm_status_t oned_final(const double* partial, int nchunk, const Geom& g, int nrhs, int p_g5, double* out,
                       cudaStream_t s);

// per-warp partial sums -> result[rhs] (fixed summation order): system rhs sums
// partial[rhs * stride + i], i < nper (stride 0 means nper)
tm_status_t reduce_partials(const double* partial, int nper, int nrhs, double* result,
                            cudaStream_t s, size_t stride = 0);

tm_status_t check_geom(const int L[4]);

// ------------------------------------------------------- Gamma tables
// gamma_mu rows as (column, i^k): upper rows from A_mu, lower rows from B_mu.
struct GammaTab {
  unsigned char perm[16][4];
  unsigned char k[16][4];
};

inline GammaTab make_gamma_tab() {
  // DeGrand-Rossi gamma_1..4 as phased permutations (row -> column, phase i^k)
  const int gp[4][4] = {{3, 2, 1, 0}, {3, 2, 1, 0}, {2, 3, 0, 1}, {2, 3, 0, 1}};
  const int gk[4][4] = {{1, 1, 3, 3}, {2, 0, 0, 2}, {1, 3, 3, 1}, {0, 0, 0, 0}};
  GammaTab t;
  for (int n = 0; n < 16; ++n) {
    int perm[4] = {0, 1, 2, 3}, ph[4] = {0, 0, 0, 0};
    for (int m = 0; m < 4; ++m) {
      if (!((n >> m) & 1)) continue;
      // (X gamma_m): row a -> column gp[m][perm[a]], phase ph[a] + gk[m][perm[a]]
      for (int a = 0; a < 4; ++a) {
        const int c = perm[a];
        ph[a] = (ph[a] + gk[m][c]) & 3;
        perm[a] = gp[m][c];
      }
    }
    for (int a = 0; a < 4; ++a) {
      t.perm[n][a] = (unsigned char)perm[a];
      t.k[n][a] = (unsigned char)ph[a];
    }
  }
  return t;
}

inline const GammaTab& gamma_tab() {
  static const GammaTab t = make_gamma_tab();
  return t;
}


}  // namespace tml
