// Conjugate gradient on the normal equations M^dag M x = M^dag eta (Sec. 2.1:
// the paper inverts with CG, truncating the low-precision solves at a
// residual |r| ~ 1e-2).  Many independent systems run together: every kernel
// covers all right-hand sides, each system keeps its own scalars on the
// device and a mask retires it once it has converged, so the host only polls
// a flag array every `check_every` iterations.
//
// Per iteration (PLAIN, every vector in one precision):
//   t = M p                       Dslash, fused |t|^2 per-warp partials
//   alpha = |r|^2 / |t|^2         fixed-order reduction + scalar kernel
//   r -= alpha M^dag t, x += alpha p   Dslash with fused update, |r|^2 partials
//   beta = |r_new|^2 / |r|^2      fixed-order reduction + scalar kernel
//   p = r + beta p
// MIXED adds FP64 reliable updates (Sleijpen & van der Vorst): the iteration
// runs in inner precision on a correction y; when |r| drops below delta times
// its value at the last update (or the tolerance is reached), x += y in FP64,
// r = b - M^dag M x is recomputed in FP64 and the iteration continues from it.
// Convergence is only accepted on such a true residual.
//
// With schur = 1 the solve is even/odd preconditioned: with A = 1 + i nu g5 the
// diagonal blocks of M are M_ee = M_oo = A, and M s = eta is solved through
//   eta_hat_o = eta_o + kappa H_oe A^-1 eta_e,
//   M_hat s_o = eta_hat_o,   M_hat = A - kappa^2 H_oe A^-1 H_eo   (CG on M_hat^dag M_hat),
//   s_e = A^-1 (eta_e + kappa H_eo s_o),
// with M_hat^dag = A(-nu) - kappa^2 (H^dag)_oe A(-nu)^-1 (H^dag)_eo.  The CG vectors
// live on the odd sites; the even half of the vector an operator is applied to
// holds the intermediate A^-1 H_eo v.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tm_host.h"

namespace tml {

tm_status_t xpay(const Geom& g, tm_prec_t prec, void* p, const void* r, const double* beta,
                 const int* active, int nrhs, int par0, int npar, cudaStream_t s);
tm_status_t fold(const Geom& g, tm_prec_t prec, void* x64, void* y, const double* sigma,
                 const int* mask, int nrhs, int par0, int npar, cudaStream_t s, void* xff = nullptr);
tm_status_t rescale(const Geom& g, tm_prec_t prec, void* r, const void* r64, const double* sigma,
                    void* p, const double* ratio, const int* mask, int nrhs, int par0, int npar,
                    cudaStream_t s, bool r_ff = false);
tm_status_t convert_masked(const Geom& g, void* out, tm_prec_t po, const void* in, tm_prec_t pi,
                           int nrhs, const int* active, cudaStream_t s);
tm_status_t twist(const Geom& g, tm_prec_t prec, void* out, const void* in, double nu, int inverse,
                  int par, int nrhs, cudaStream_t s);

// The operator of the solve: M (both parities) or the odd-site Schur complement.
struct SolveOp {
  tm_op* op;
  bool schur;
  int nrhs;
  cudaStream_t s;
  bool il = false;  // vectors in the system-interleaved 16-bit layout
  double nu() const { return 2.0 * op->kappa * op->mu; }

  // t = Op v (+ |t|^2 partials); for the Schur operator v's even half is scratch
  tm_status_t apply(tm_prec_t prec, void* v, void* t, double* partial, const int* active) const {
    if (!schur) {
      DslashCall c;
      c.in = v; c.out = t; c.nrhs = nrhs; c.partial = partial; c.active = active; c.il = il;
      return dslash_dispatch(op, prec, c, s);
    }
    DslashCall c1;  // v_e = A^-1 H_eo v_o
    c1.custom = true; c1.in = v; c1.out = v; c1.nrhs = nrhs; c1.active = active;
    c1.parity = 0; c1.centre = 0; c1.hop_scale = 1.0; c1.out_inv = true; c1.nu = nu(); c1.il = il;
    const tm_status_t st = dslash_dispatch(op, prec, c1, s);
    if (st != TM_OK) return st;
    DslashCall c2;  // t_o = A v_o - kappa^2 H_oe v_e
    c2.custom = true; c2.in = v; c2.cfield = v; c2.out = t; c2.nrhs = nrhs; c2.active = active;
    c2.parity = 1; c2.centre = 2; c2.hop_scale = -op->kappa * op->kappa; c2.nu = nu();
    c2.partial = partial; c2.il = il;
    return dslash_dispatch(op, prec, c2, s);
  }

  // Op^dag t with the epilogue of `e` (EPI_OUT into e.out, EPI_CGUPD, EPI_RESID);
  // for the Schur operator t's even half is scratch
  tm_status_t apply_dag(tm_prec_t prec, void* t, DslashCall e) const {
    e.nrhs = nrhs;
    e.dagger = true;
    e.il = il;
    if (!schur) {
      e.in = t;
      return dslash_dispatch(op, prec, e, s);
    }
    DslashCall c1;  // t_e = A(-nu)^-1 (H^dag)_eo t_o
    c1.custom = true; c1.dagger = true; c1.in = t; c1.out = t; c1.nrhs = nrhs; c1.active = e.active;
    c1.parity = 0; c1.centre = 0; c1.hop_scale = 1.0; c1.out_inv = true; c1.nu = -nu(); c1.il = il;
    const tm_status_t st = dslash_dispatch(op, prec, c1, s);
    if (st != TM_OK) return st;
    e.custom = true; e.in = t; e.cfield = t; e.parity = 1; e.centre = 2;
    e.hop_scale = -op->kappa * op->kappa; e.nu = -nu();
    return dslash_dispatch(op, prec, e, s);
  }

  // eta_hat_o = eta_o + kappa H_oe A^-1 eta_e into dst (odd half; even half scratch)
  tm_status_t prepare(tm_prec_t prec, const void* eta, void* dst) const {
    tm_status_t st = il ? il_twist(op->g, prec, dst, eta, nu(), 1, 0, nrhs, s)
                        : twist(op->g, prec, dst, eta, nu(), 1, 0, nrhs, s);
    if (st != TM_OK) return st;
    DslashCall c;
    c.custom = true; c.in = dst; c.cfield = eta; c.out = dst; c.nrhs = nrhs;
    c.parity = 1; c.centre = 1; c.hop_scale = op->kappa; c.nu = nu(); c.il = il;
    return dslash_dispatch(op, prec, c, s);
  }

  // x_e = A^-1 (eta_e + kappa H_eo x_o)
  tm_status_t reconstruct(tm_prec_t prec, const void* eta, void* x) const {
    DslashCall c;
    c.custom = true; c.in = x; c.cfield = eta; c.out = x; c.nrhs = nrhs;
    c.parity = 0; c.centre = 1; c.hop_scale = op->kappa; c.out_inv = true; c.nu = nu(); c.il = il;
    return dslash_dispatch(op, prec, c, s);
  }
};

// per-system device state (structure of arrays)
struct CgState {
  double* bb;     // |b|^2
  double* rr;     // |r|^2 of the current residual
  double* red;    // output of the last reduction
  double* alpha;
  double* beta;
  double* maxr2;  // |r|^2 at the last reliable update (absolute)
  double* sigma;  // MIXED: inner vectors hold (true vector) / sigma
  double* ratio;  // MIXED: sigma_old / sigma_new of the last reliable update
  int* active;
  int* ru;        // reliable update pending
  int* iters;
  int* nru;
  int* status;
};

struct CgScalars {
  double tol2;
  double delta2;
  double n12;     // 12 V complex components per field
  int max_iter;
  int nrhs;
  int mixed;
};

__global__ void cg_init_kernel(CgState st, CgScalars sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.nrhs) return;
  const double bb = st.red[i];
  // MIXED: the inner iteration runs on b / sigma with entries of order one,
  // so that narrow formats (FP16) neither overflow nor underflow
  const double sg = (sc.mixed && bb > 0.0 && isfinite(bb)) ? sqrt(bb / sc.n12) : 1.0;
  st.bb[i] = bb;
  st.sigma[i] = sg;
  st.ratio[i] = 1.0;
  st.rr[i] = bb / (sg * sg);
  st.maxr2[i] = bb;
  st.iters[i] = 0;
  st.nru[i] = 0;
  st.ru[i] = 0;
  st.alpha[i] = 0.0;
  st.beta[i] = 0.0;
  if (!isfinite(bb)) {
    st.status[i] = TM_ERR_NAN;
    st.active[i] = 0;
  } else {
    st.status[i] = TM_OK;
    st.active[i] = (bb > 0.0 && sc.max_iter > 0) ? 1 : 0;
    if (bb > 0.0 && sc.max_iter == 0 && sc.tol2 < 1.0) st.status[i] = TM_ERR_NOCONV;
  }
}

__global__ void cg_alpha_kernel(CgState st, CgScalars sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.nrhs) return;
  st.ru[i] = 0;  // the reliable update of the previous iteration is complete
  if (!st.active[i]) return;
  const double pap = st.red[i];
  if (!isfinite(pap) || !(pap > 0.0)) {
    st.status[i] = TM_ERR_NAN;
    st.active[i] = 0;
    st.alpha[i] = 0.0;
    return;
  }
  st.alpha[i] = st.rr[i] / pap;
}

__global__ void cg_beta_plain_kernel(CgState st, CgScalars sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.nrhs || !st.active[i]) return;
  const double rn = st.red[i];
  const int it = ++st.iters[i];
  if (!isfinite(rn)) {
    st.status[i] = TM_ERR_NAN;
    st.active[i] = 0;
    return;
  }
  st.beta[i] = rn / st.rr[i];
  st.rr[i] = rn;
  if (rn <= sc.tol2 * st.bb[i]) {
    st.active[i] = 0;
    st.status[i] = TM_OK;
  } else if (it >= sc.max_iter) {
    st.active[i] = 0;
    st.status[i] = TM_ERR_NOCONV;
  }
}

__global__ void cg_beta_mixed_kernel(CgState st, CgScalars sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.nrhs || !st.active[i]) return;
  const double rn = st.red[i];
  const int it = ++st.iters[i];
  if (!isfinite(rn)) {
    st.status[i] = TM_ERR_NAN;
    st.active[i] = 0;
    return;
  }
  const double s2 = st.sigma[i] * st.sigma[i];
  const double rabs = rn * s2;
  if (rabs <= sc.tol2 * st.bb[i] || rabs < sc.delta2 * st.maxr2[i] || it >= sc.max_iter) {
    st.ru[i] = 1;  // beta follows from the true residual
    return;
  }
  st.beta[i] = rn / st.rr[i];
  st.rr[i] = rn;
}

__global__ void cg_ru_kernel(CgState st, CgScalars sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sc.nrhs || !st.ru[i]) return;
  const double rt = st.red[i];  // |b - M^dag M x|^2, absolute
  st.nru[i] += 1;
  if (!isfinite(rt)) {
    st.status[i] = TM_ERR_NAN;
    st.active[i] = 0;
    st.ratio[i] = 1.0;
    return;
  }
  const double s_old = st.sigma[i];
  const double s_new = rt > 0.0 ? sqrt(rt / sc.n12) : s_old;
  st.beta[i] = rt / (st.rr[i] * s_old * s_old);
  st.rr[i] = rt / (s_new * s_new);
  st.sigma[i] = s_new;
  st.ratio[i] = s_old / s_new;
  st.maxr2[i] = rt;
  if (rt <= sc.tol2 * st.bb[i]) {
    st.active[i] = 0;
    st.status[i] = TM_OK;
  } else if (st.iters[i] >= sc.max_iter) {
    st.active[i] = 0;
    st.status[i] = TM_ERR_NOCONV;
  }
}

static size_t align_up(size_t n) { return (n + 255) & ~(size_t)255; }

// Carve the operator's work space into the buffers a solve needs.
struct Carver {
  char* base;
  size_t off = 0;
  void* take(size_t n) {
    void* p = base ? base + off : nullptr;
    off += align_up(n);
    return p;
  }
};

static tm_status_t ensure_work(tm_op* op, size_t bytes, int nflags, cudaStream_t s) {
  if (op->work_bytes < bytes) {
    if (op->work) {
      cudaDeviceSynchronize();
      dev_free(op->work, s);
      op->work = nullptr;
      op->work_bytes = 0;
    }
    TM_TRY(dev_alloc(&op->work, bytes, s, "tm_cg_solve work space"));
    // the work space is used on other streams of the solve as well
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("tm_cg_solve: %s", cudaGetErrorString(cudaGetLastError()));
      return TM_ERR_CUDA;
    }
    op->work_bytes = bytes;
  }
  if (op->host_flags_n < nflags) {
    pinned_give(op->host_flags, op->host_flags_n);
    op->host_flags = pinned_take(nflags, &op->host_flags_n);
    if (!op->host_flags) {
      set_error("tm_cg_solve: pinned host allocation failed");
      return TM_ERR_CUDA;
    }
  }
  return TM_OK;
}

static tm_status_t scalar_launch(void (*k)(CgState, CgScalars), const CgState& st,
                                 const CgScalars& sc, cudaStream_t s) {
  const int nb = (sc.nrhs + 127) / 128;
  k<<<nb, 128, 0, s>>>(st, sc);
  count_launch();
  return check_launch("cg scalar kernel");
}

static tm_status_t memcpy_d2d(void* dst, const void* src, size_t n, cudaStream_t s) {
  if (cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    set_error("tm_cg_solve: device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

static tm_status_t memset_d(void* dst, size_t n, cudaStream_t s) {
  if (cudaMemsetAsync(dst, 0, n, s) != cudaSuccess) {
    set_error("tm_cg_solve: memset failed: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

// ---------------------------------------------------------------- one solve
// One batched solve (one operator, nrhs systems) split into stream-ordered
// phases, so that several solves can advance together and the iterations
// between two host polls can be captured into a CUDA graph.
struct CgRun {
  tm_op* op = nullptr;
  void* x = nullptr;
  const void* eta = nullptr;
  int nrhs = 0;
  tm_cg_params_t prm{};
  tm_cg_stats_t* stats = nullptr;
  cudaStream_t s = nullptr;

  bool mixed = false, schur = false;
  // plain F16/BF16 solves iterate on the system-interleaved layout (tensor-core
  // Dslash): eta is converted into eta_il at set-up, x_il back into x at the end
  bool il = false;
  void *eta_il = nullptr, *x_il = nullptr;
  bool x_is_il = false;  // the caller's x and eta are in the interleaved layout (tm_cg_solve_il)
  tm_prec_t lo = TM_PREC_F64, hi = TM_PREC_F64;
  int par0 = 0, npar = 2, nwarp = 0;
  void *b = nullptr, *r = nullptr, *p = nullptr, *t = nullptr, *y = nullptr;
  void *b64 = nullptr, *r64 = nullptr, *tmp64 = nullptr;
  // MIXED with ru_prec = FF: the true residuals in float-float from the
  // float-float copies of x (written by every fold) and b; r64 and tmp64 then
  // hold float-float fields of the same size
  bool ru_ff = false;
  void *xff = nullptr, *bff = nullptr;
  tm_prec_t ru = TM_PREC_F64;
  double* partial = nullptr;
  CgState st{};
  CgScalars sc{};
  void* xs = nullptr;          // iterate of the inner CG
  void* bb_field = nullptr;    // right-hand side Op^dag eta(_hat)
  void* scratch_hi = nullptr;
  const double* part0 = nullptr;
  int nper = 0;
  size_t pstride = 0;

  SolveOp A() const { return SolveOp{op, schur, nrhs, s, il}; }
  tm_status_t reduce() const { return reduce_partials(part0, nper, nrhs, st.red, s, pstride); }

  tm_status_t setup();
  tm_status_t iteration();
  tm_status_t poll() const;    // active flags -> the operator's pinned host flags
  bool any_active() const;
  bool timed_out() const;
  tm_status_t finish(tm_status_t* worst);
};

static tm_status_t check_params(const tm_cg_params_t* prm) {
  if (!prm) { set_error("tm_cg_solve: null argument"); return TM_ERR_ARG; }
  if (!(prm->tol >= 0.0) || prm->max_iter < 0) { set_error("tm_cg_solve: tol must be >= 0 and max_iter >= 0"); return TM_ERR_ARG; }
  const bool mixed = prm->mode == TM_CG_MIXED;
  if (prm->mode != TM_CG_PLAIN && !mixed) { set_error("tm_cg_solve: unknown mode %d", (int)prm->mode); return TM_ERR_ARG; }
  if (mixed && !(prm->delta > 0.0 && prm->delta < 1.0)) { set_error("tm_cg_solve: delta must be in (0, 1)"); return TM_ERR_ARG; }
  if (prm->schur != 0 && prm->schur != 1) { set_error("tm_cg_solve: schur must be 0 or 1"); return TM_ERR_ARG; }
  if (mixed && prm->ru_prec != TM_PREC_F64 && prm->ru_prec != TM_PREC_FF) {
    set_error("tm_cg_solve: ru_prec must be F64 or FF");
    return TM_ERR_ARG;
  }
  if (prm->graph != 0 && prm->graph != 1) { set_error("tm_cg_solve: graph must be 0 or 1"); return TM_ERR_ARG; }
  const tm_prec_t lo = mixed ? prm->inner_prec : prm->prec;
  if ((int)lo < 0 || (int)lo > 3) { set_error("tm_cg_solve: precision must be F64, F32, F16 or BF16"); return TM_ERR_ARG; }
  return TM_OK;
}

tm_status_t CgRun::setup() {
  mixed = prm.mode == TM_CG_MIXED;
  schur = prm.schur == 1;
  lo = mixed ? prm.inner_prec : prm.prec;
  hi = mixed ? TM_PREC_F64 : lo;
  const Geom& g = op->g;
  // the CG vectors cover both parities, or only the odd one (Schur)
  par0 = schur ? 1 : 0;
  npar = schur ? 1 : 2;
  const tm_geom_t gg = {{g.L[0], g.L[1], g.L[2], g.L[3]}};
  ru_ff = mixed && prm.ru_prec == TM_PREC_FF;
  ru = ru_ff ? TM_PREC_FF : TM_PREC_F64;
  il = !mixed && (lo == TM_PREC_F16 || lo == TM_PREC_BF16) && op->recon_p[lo] == 18 && cg_il_on();
  if (x_is_il && !il) {
    set_error("tm_cg_solve_il: needs a plain F16/BF16 solve with 18-real links and the interleaved solver enabled");
    return TM_ERR_UNSUPPORTED;
  }
  const size_t F = il ? il_bytes(g, nrhs) : tm_spinor_bytes(&gg, lo, nrhs);
  const size_t F64 = tm_spinor_bytes(&gg, TM_PREC_F64, nrhs);
  nwarp = nwarp_of(g);
  const size_t P = sizeof(double) * (size_t)nrhs * 2 * (size_t)nwarp;

  // lay out the work space (first pass sizes, second pass assigns)
  for (int pass = 0; pass < 2; ++pass) {
    Carver c{pass ? (char*)op->work : nullptr};
    if (mixed) {
      b64 = c.take(F64); r64 = c.take(F64); tmp64 = c.take(F64);
      if (ru_ff) { xff = c.take(F64); bff = c.take(F64); }
      y = c.take(F); r = c.take(F); p = c.take(F); t = c.take(F);
    } else {
      b = c.take(F); r = c.take(F); p = c.take(F); t = c.take(F);
      if (il) {
        eta_il = x_is_il ? const_cast<void*>(eta) : c.take(F);
        x_il = x_is_il ? x : c.take(F);
      }
    }
    partial = (double*)c.take(P);
    st.bb = (double*)c.take(sizeof(double) * nrhs);
    st.rr = (double*)c.take(sizeof(double) * nrhs);
    st.red = (double*)c.take(sizeof(double) * nrhs);
    st.alpha = (double*)c.take(sizeof(double) * nrhs);
    st.beta = (double*)c.take(sizeof(double) * nrhs);
    st.maxr2 = (double*)c.take(sizeof(double) * nrhs);
    st.sigma = (double*)c.take(sizeof(double) * nrhs);
    st.ratio = (double*)c.take(sizeof(double) * nrhs);
    st.active = (int*)c.take(sizeof(int) * nrhs);
    st.ru = (int*)c.take(sizeof(int) * nrhs);
    st.iters = (int*)c.take(sizeof(int) * nrhs);
    st.nru = (int*)c.take(sizeof(int) * nrhs);
    st.status = (int*)c.take(sizeof(int) * nrhs);
    if (pass == 0) TM_TRY(ensure_work(op, c.off, 5 * nrhs, s));
  }
  sc.tol2 = prm.tol * prm.tol;
  sc.delta2 = mixed ? prm.delta * prm.delta : 0.0;
  sc.n12 = 12.0 * (double)g.Vh * npar;
  sc.max_iter = prm.max_iter;
  sc.nrhs = nrhs;
  sc.mixed = mixed ? 1 : 0;
  // reductions over the parities the vectors live on
  part0 = partial + (schur ? nwarp : 0);
  nper = npar * nwarp;
  pstride = 2 * (size_t)nwarp;
  xs = mixed ? y : (il ? x_il : x);
  bb_field = mixed ? b64 : b;
  scratch_hi = mixed ? tmp64 : t;
  const SolveOp Op = A();

  if (il && !x_is_il) TM_TRY(il_convert(g, eta_il, eta, nrhs, true, s));
  const void* eta_in = il ? eta_il : eta;
  // b = Op^dag eta (Schur: Op^dag eta_hat), |b|^2
  {
    const void* src = eta_in;
    if (schur) {
      TM_TRY(Op.prepare(hi, eta_in, scratch_hi));
      src = scratch_hi;
    }
    DslashCall e;
    e.out = bb_field; e.partial = partial;
    if (schur) {
      TM_TRY(Op.apply_dag(hi, scratch_hi, e));
    } else {
      e.in = src;
      e.nrhs = nrhs;
      e.dagger = true;
      e.il = il;
      TM_TRY(dslash_dispatch(op, hi, e, s));
    }
    TM_TRY(reduce());
    TM_TRY(scalar_launch(cg_init_kernel, st, sc, s));
  }
  if (mixed) {
    TM_TRY(rescale(g, lo, r, b64, st.sigma, nullptr, nullptr, nullptr, nrhs, par0, npar, s));
    TM_TRY(memset_d(x, F64, s));
    TM_TRY(memset_d(y, F, s));
    if (ru_ff) {
      TM_TRY(convert_masked(g, bff, TM_PREC_FF, b64, TM_PREC_F64, nrhs, nullptr, s));
      TM_TRY(memset_d(xff, F64, s));
    }
  } else {
    TM_TRY(memcpy_d2d(r, b, F, s));
    TM_TRY(memset_d(xs, F, s));
  }
  TM_TRY(memcpy_d2d(p, r, F, s));
  return TM_OK;
}

// one CG iteration of every active system (inactive systems are masked out on
// the device, so extra iterations after convergence change nothing)
tm_status_t CgRun::iteration() {
  const Geom& g = op->g;
  const SolveOp Op = A();
  TM_TRY(Op.apply(lo, p, t, partial, st.active));  // t = Op p, |t|^2
  TM_TRY(reduce());
  TM_TRY(scalar_launch(cg_alpha_kernel, st, sc, s));
  DslashCall e;  // r -= alpha Op^dag t, x += alpha p, |r|^2
  e.epi = EPI_CGUPD; e.partial = partial; e.active = st.active; e.alpha = st.alpha;
  e.p = p; e.x = xs; e.r = r;
  TM_TRY(Op.apply_dag(lo, t, e));
  TM_TRY(reduce());
  if (!mixed) {
    TM_TRY(scalar_launch(cg_beta_plain_kernel, st, sc, s));
  } else {
    TM_TRY(scalar_launch(cg_beta_mixed_kernel, st, sc, s));
    // reliable update for the systems that asked for one: x += sigma y (FP64),
    // r = b - Op^dag Op x in FP64 or float-float (ru_prec)
    TM_TRY(fold(g, lo, x, y, st.sigma, st.ru, nrhs, par0, npar, s, ru_ff ? xff : nullptr));
    TM_TRY(Op.apply(ru, ru_ff ? xff : x, tmp64, nullptr, st.ru));
    DslashCall e4;
    e4.out = r64; e4.b = ru_ff ? bff : b64; e4.epi = EPI_RESID; e4.partial = partial; e4.active = st.ru;
    TM_TRY(Op.apply_dag(ru, tmp64, e4));
    TM_TRY(reduce());
    TM_TRY(scalar_launch(cg_ru_kernel, st, sc, s));
    TM_TRY(rescale(g, lo, r, r64, st.sigma, p, st.ratio, st.ru, nrhs, par0, npar, s, ru_ff));
  }
  if (il) return il_xpay(g, lo, p, r, st.beta, st.active, nrhs, par0, npar, s);
  return xpay(g, lo, p, r, st.beta, st.active, nrhs, par0, npar, s);
}

tm_status_t CgRun::poll() const {
  if (cudaMemcpyAsync(op->host_flags, st.active, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (il && cudaMemcpyAsync(op->host_flags + nrhs, op->il_err, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                 cudaSuccess)) {
    set_error("tm_cg_solve: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

// a bounded wait of the interleaved Dslash gave up (flag copied by poll())
bool CgRun::timed_out() const { return il && op->host_flags[nrhs] != 0; }

bool CgRun::any_active() const {
  for (int i = 0; i < nrhs; ++i)
    if (op->host_flags[i] != 0) return true;
  return false;
}

tm_status_t CgRun::finish(tm_status_t* worst_out) {
  const Geom& g = op->g;
  const SolveOp Op = A();
  if (mixed) TM_TRY(fold(g, lo, x, y, st.sigma, nullptr, nrhs, par0, npar, s, ru_ff ? xff : nullptr));
  std::vector<double> h_bb(nrhs), h_rr(nrhs), h_sig(nrhs);
  std::vector<int> h_it(nrhs), h_nru(nrhs), h_status(nrhs);
  auto fetch = [&]() -> bool {
    bool ok = cudaMemcpyAsync(h_bb.data(), st.bb, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h_rr.data(), st.rr, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h_sig.data(), st.sigma, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h_it.data(), st.iters, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h_nru.data(), st.nru, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h_status.data(), st.status, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    return ok && cudaStreamSynchronize(s) == cudaSuccess;
  };
  if (!fetch()) {
    set_error("tm_cg_solve: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  // true residual |b - Op^dag Op x| / |b|: a mixed solve that converged already
  // accepted it on such a residual (the last reliable update); otherwise, and
  // for plain solves that ask for it, it is recomputed here
  bool all_ok = true;
  for (int i = 0; i < nrhs; ++i) all_ok = all_ok && h_status[i] == TM_OK;
  const bool recompute = (mixed && !all_ok) || (!mixed && prm.true_residual);
  std::vector<double> h_true(nrhs, -1.0);
  if (mixed && all_ok) {
    for (int i = 0; i < nrhs; ++i) h_true[i] = h_rr[i] * h_sig[i] * h_sig[i];
  }
  if (recompute) {
    void* tmp = mixed ? tmp64 : t;
    void* res = mixed ? r64 : r;
    const tm_prec_t pr = mixed ? ru : hi;
    TM_TRY(Op.apply(pr, mixed ? (ru_ff ? xff : x) : xs, tmp, nullptr, nullptr));
    DslashCall e4;
    e4.out = res; e4.b = ru_ff ? bff : bb_field; e4.epi = EPI_RESID; e4.partial = partial;
    TM_TRY(Op.apply_dag(pr, tmp, e4));
    TM_TRY(reduce());
    if (cudaMemcpyAsync(h_true.data(), st.red, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("tm_cg_solve: %s", cudaGetErrorString(cudaGetLastError()));
      return TM_ERR_CUDA;
    }
  }
  if (schur) TM_TRY(Op.reconstruct(hi, il ? eta_il : eta, mixed ? x : xs));
  if (il && !x_is_il) TM_TRY(il_convert(g, x, x_il, nrhs, false, s));
  const bool want_true = mixed || prm.true_residual;
  tm_status_t worst = TM_OK;
  for (int i = 0; i < nrhs; ++i) {
    const double bbi = h_bb[i];
    if (stats) {
      stats[i].iters = h_it[i];
      stats[i].reliable_updates = h_nru[i];
      stats[i].status = h_status[i];
      stats[i].rel_res = bbi > 0 ? std::sqrt(h_rr[i] * h_sig[i] * h_sig[i] / bbi) : 0.0;
      stats[i].true_res = want_true ? (bbi > 0 ? std::sqrt(h_true[i] / bbi) : 0.0) : -1.0;
    }
    if (h_status[i] == TM_ERR_NAN) worst = TM_ERR_NAN;
    else if (h_status[i] == TM_ERR_NOCONV && worst == TM_OK) worst = TM_ERR_NOCONV;
  }
  *worst_out = worst;
  return TM_OK;
}

// ------------------------------------------------------------- the driver
// Streams and events of a group solve: one set runs on the caller's stream;
// several sets each get a stream forked from it (fork/join by events, which
// is also how the sets' branches enter one captured graph).
struct GroupStreams {
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> s;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  bool forked = false;

  tm_status_t init(cudaStream_t m, int n) {
    main = m;
    s.assign(n, m);
    if (n <= 1) return TM_OK;
    forked = true;
    join_ev.assign(n, nullptr);
    bool ok = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < n && ok; ++i) {
      ok = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&join_ev[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      set_error("tm_cg_solve_group: stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
      return TM_ERR_CUDA;
    }
    return TM_OK;
  }
  tm_status_t fork() {
    if (!forked) return TM_OK;
    bool ok = cudaEventRecord(fork_ev, main) == cudaSuccess;
    for (size_t i = 0; i < s.size() && ok; ++i) ok = cudaStreamWaitEvent(s[i], fork_ev, 0) == cudaSuccess;
    if (!ok) { set_error("tm_cg_solve_group: fork: %s", cudaGetErrorString(cudaGetLastError())); return TM_ERR_CUDA; }
    return TM_OK;
  }
  tm_status_t join() {
    if (!forked) return TM_OK;
    bool ok = true;
    for (size_t i = 0; i < s.size() && ok; ++i) {
      ok = cudaEventRecord(join_ev[i], s[i]) == cudaSuccess;
      ok = ok && cudaStreamWaitEvent(main, join_ev[i], 0) == cudaSuccess;
    }
    if (!ok) { set_error("tm_cg_solve_group: join: %s", cudaGetErrorString(cudaGetLastError())); return TM_ERR_CUDA; }
    return TM_OK;
  }
  ~GroupStreams() {
    if (!forked) return;
    for (size_t i = 0; i < s.size(); ++i) {
      if (s[i] && s[i] != main) cudaStreamDestroy(s[i]);
      if (join_ev[i]) cudaEventDestroy(join_ev[i]);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
  }
};

struct GraphHolder {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~GraphHolder() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// Enqueue k iterations of every set plus the poll of its flags.
static tm_status_t enqueue_block(std::vector<CgRun>& runs, GroupStreams& gs, int k) {
  TM_TRY(gs.fork());
  for (auto& run : runs) {
    for (int i = 0; i < k; ++i) TM_TRY(run.iteration());
    TM_TRY(run.poll());
  }
  return gs.join();
}

// A private stream ordered after the caller's (the legacy default stream
// cannot be captured); the caller's stream waits for it at the end.
struct PrivateStream {
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev = nullptr;
  tm_status_t open(cudaStream_t u) {
    user = u;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, user) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess) {
      set_error("tm_cg_solve: stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
      return TM_ERR_CUDA;
    }
    return TM_OK;
  }
  ~PrivateStream() {
    if (s && ev && cudaEventRecord(ev, s) == cudaSuccess) cudaStreamWaitEvent(user, ev, 0);
    if (s) cudaStreamDestroy(s);
    if (ev) cudaEventDestroy(ev);
  }
};

static tm_cg_graph_key graph_key(const CgRun& r, int k) {
  tm_cg_graph_key key{};
  key.x = r.x;
  key.xs = r.xs;
  key.work = r.op->work;
  key.work_bytes = r.op->work_bytes;
  key.host_flags = r.op->host_flags;
  key.nrhs = r.nrhs;
  key.k = k;
  key.il = r.il ? 1 : 0;
  key.tol = r.prm.tol;
  key.delta = r.prm.delta;
  key.max_iter = r.prm.max_iter;
  key.mode = (int)r.prm.mode;
  key.prec = (int)r.prm.prec;
  key.inner_prec = (int)r.prm.inner_prec;
  key.check_every = r.prm.check_every;
  key.true_residual = r.prm.true_residual;
  key.schur = r.prm.schur;
  key.ru_prec = (int)r.prm.ru_prec;
  return key;
}

static bool same_key(const tm_cg_graph_key& a, const tm_cg_graph_key& b) {
  return a.x == b.x && a.xs == b.xs && a.work == b.work && a.work_bytes == b.work_bytes &&
         a.host_flags == b.host_flags && a.nrhs == b.nrhs && a.k == b.k && a.il == b.il && a.tol == b.tol &&
         a.delta == b.delta && a.max_iter == b.max_iter && a.mode == b.mode && a.prec == b.prec &&
         a.inner_prec == b.inner_prec && a.check_every == b.check_every && a.true_residual == b.true_residual &&
         a.schur == b.schur && a.ru_prec == b.ru_prec;
}

static tm_status_t solve_group(std::vector<CgRun>& runs, const tm_cg_params_t* prm, cudaStream_t s_user,
                               tm_status_t* worst) {
  PrivateStream ps;
  cudaStream_t s0 = s_user;
  if (prm->graph) {
    TM_TRY(ps.open(s_user));
    s0 = ps.s;
  }
  GroupStreams gs;
  TM_TRY(gs.init(s0, (int)runs.size()));
  for (size_t i = 0; i < runs.size(); ++i) runs[i].s = gs.s[i];
  TM_TRY(gs.fork());
  for (auto& run : runs) TM_TRY(run.setup());
  TM_TRY(gs.join());

  const int check_every = prm->check_every > 0 ? prm->check_every : 1;
  GraphHolder gh;
  int per_replay = 0;
  // a single-set solve replays the graph its operator kept from the last solve
  // whose launches were the same (same buffers, systems and parameters): the
  // graph embeds nothing else, so the replay is the capture it would make
  tm_cg_graph_cache* cache = (prm->graph && runs.size() == 1) ? &runs[0].op->cg_graph : nullptr;
  const tm_cg_graph_key key = cache ? graph_key(runs[0], check_every) : tm_cg_graph_key{};
  cudaGraphExec_t exec = nullptr;
  if (cache && cache->valid && same_key(cache->key, key)) {
    exec = cache->exec;
    per_replay = cache->per_replay;
  }
  for (int done = 0; done < prm->max_iter;) {
    const int k = std::min(check_every, prm->max_iter - done);
    if (prm->graph && k == check_every) {
      if (!exec) {
        // capture k iterations of every set (and the flag copies) once; the
        // device-side masks make every replay the same sequence of launches
        capture_begin();
        tm_status_t cs = TM_OK;
        if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          capture_end();
          set_error("tm_cg_solve: graph capture failed: %s", cudaGetErrorString(cudaGetLastError()));
          return TM_ERR_CUDA;
        }
        cs = enqueue_block(runs, gs, k);
        const cudaError_t ce = cudaStreamEndCapture(s0, &gh.graph);
        per_replay = capture_end();
        if (cs != TM_OK) return cs;
        if (ce != cudaSuccess || cudaGraphInstantiate(&gh.exec, gh.graph, 0) != cudaSuccess) {
          set_error("tm_cg_solve: graph capture failed: %s", cudaGetErrorString(cudaGetLastError()));
          return TM_ERR_CUDA;
        }
        exec = gh.exec;
        if (cache) {
          // the operator keeps the new graph in place of the old one
          if (cache->exec) cudaGraphExecDestroy(cache->exec);
          cache->exec = gh.exec;
          cache->key = key;
          cache->per_replay = per_replay;
          cache->valid = true;
          gh.exec = nullptr;
        }
      }
      TraceScope ts(s0, "cg.graph", 0.0, 0.0, 0);
      if (cudaGraphLaunch(exec, s0) != cudaSuccess) {
        set_error("tm_cg_solve: graph launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return TM_ERR_CUDA;
      }
      count_launch(per_replay);
    } else {
      TM_TRY(enqueue_block(runs, gs, k));
    }
    if (cudaStreamSynchronize(s0) != cudaSuccess) {
      set_error("tm_cg_solve: %s", cudaGetErrorString(cudaGetLastError()));
      return TM_ERR_CUDA;
    }
    done += k;
    bool any = false;
    for (const auto& run : runs) {
      if (run.timed_out()) {
        set_error("tm_cg_solve: a bounded wait of the interleaved Dslash gave up");
        return TM_ERR_TIMEOUT;
      }
      any = any || run.any_active();
    }
    if (!any) break;
  }

  TM_TRY(gs.fork());
  *worst = TM_OK;
  for (auto& run : runs) {
    tm_status_t w = TM_OK;
    TM_TRY(run.finish(&w));
    if (w == TM_ERR_NAN) *worst = TM_ERR_NAN;
    else if (w == TM_ERR_NOCONV && *worst == TM_OK) *worst = TM_ERR_NOCONV;
  }
  return gs.join();
}

static tm_status_t report(tm_status_t worst) {
  if (worst == TM_ERR_NAN) set_error("tm_cg_solve: non-finite residual norm");
  else if (worst == TM_ERR_NOCONV) set_error("tm_cg_solve: max_iter reached before tolerance");
  return worst;
}

}  // namespace tml

using namespace tml;

extern "C" tm_status_t tm_cg_solve(tm_op_t* op, void* x, const void* eta, int nrhs,
                                   const tm_cg_params_t* prm, tm_cg_stats_t* stats, tm_stream_t strm) {
  if (!op || !x || !eta || !prm || nrhs < 0) { set_error("tm_cg_solve: null argument"); return TM_ERR_ARG; }
  if (x == eta) { set_error("tm_cg_solve: x and eta must not overlap"); return TM_ERR_ARG; }
  TM_TRY(check_params(prm));
  if (nrhs == 0) return TM_OK;
  std::vector<CgRun> runs(1);
  runs[0].op = op; runs[0].x = x; runs[0].eta = eta; runs[0].nrhs = nrhs;
  runs[0].prm = *prm; runs[0].stats = stats;
  tm_status_t worst = TM_OK;
  TM_TRY(solve_group(runs, prm, (cudaStream_t)strm, &worst));
  return report(worst);
}

extern "C" tm_status_t tm_cg_solve_il(tm_op_t* op, void* x_il, const void* eta_il, int nrhs,
                                      const tm_cg_params_t* prm, tm_cg_stats_t* stats, tm_stream_t strm) {
  if (!op || !x_il || !eta_il || !prm || nrhs < 0) { set_error("tm_cg_solve_il: null argument"); return TM_ERR_ARG; }
  if (x_il == eta_il) { set_error("tm_cg_solve_il: x and eta must not overlap"); return TM_ERR_ARG; }
  if ((reinterpret_cast<uintptr_t>(x_il) | reinterpret_cast<uintptr_t>(eta_il)) & 15u) {
    set_error("tm_cg_solve_il: x and eta must be 16-byte aligned");
    return TM_ERR_ARG;
  }
  TM_TRY(check_params(prm));
  const tm_prec_t lo = prm->prec;
  if (prm->mode != TM_CG_PLAIN || (lo != TM_PREC_F16 && lo != TM_PREC_BF16) || op->recon_p[lo] != 18 || !cg_il_on()) {
    set_error("tm_cg_solve_il: needs a plain F16/BF16 solve with 18-real links and the interleaved solver enabled");
    return TM_ERR_UNSUPPORTED;
  }
  if (nrhs == 0) return TM_OK;
  std::vector<CgRun> runs(1);
  runs[0].op = op; runs[0].x = x_il; runs[0].eta = eta_il; runs[0].nrhs = nrhs;
  runs[0].prm = *prm; runs[0].stats = stats; runs[0].x_is_il = true;
  tm_status_t worst = TM_OK;
  TM_TRY(solve_group(runs, prm, (cudaStream_t)strm, &worst));
  return report(worst);
}

extern "C" tm_status_t tm_cg_solve_group(int nsets, tm_op_t* const* ops, void* const* x,
                                         const void* const* eta, const int* nrhs,
                                         const tm_cg_params_t* prm, tm_cg_stats_t* const* stats,
                                         tm_stream_t strm) {
  if (nsets < 0 || (nsets > 0 && (!ops || !x || !eta || !nrhs))) {
    set_error("tm_cg_solve_group: null argument");
    return TM_ERR_ARG;
  }
  TM_TRY(check_params(prm));
  std::vector<CgRun> runs;
  for (int i = 0; i < nsets; ++i) {
    if (!ops[i] || !x[i] || !eta[i] || nrhs[i] < 0) { set_error("tm_cg_solve_group: null argument in set %d", i); return TM_ERR_ARG; }
    if (x[i] == eta[i]) { set_error("tm_cg_solve_group: x and eta of set %d overlap", i); return TM_ERR_ARG; }
    for (int j = 0; j < i; ++j)
      if (ops[j] == ops[i]) {
        set_error("tm_cg_solve_group: sets %d and %d share an operator handle (use tm_op_clone)", j, i);
        return TM_ERR_ARG;
      }
    if (nrhs[i] == 0) continue;
    CgRun r;
    r.op = ops[i]; r.x = x[i]; r.eta = eta[i]; r.nrhs = nrhs[i];
    r.prm = *prm; r.stats = stats ? stats[i] : nullptr;
    runs.push_back(r);
  }
  if (runs.empty()) return TM_OK;
  tm_status_t worst = TM_OK;
  TM_TRY(solve_group(runs, prm, (cudaStream_t)strm, &worst));
  return report(worst);
}
