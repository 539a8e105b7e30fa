// Hopping Parameter Expansion (Sec. 2.4, Eqs. 7-8).
//
// With M = B^-1 + H, B = (1 + i nu g5)^-1 (site-local, nu = 2 kappa mu) and H the
// hopping term (-kappa times the hops of M),
//   M^-1 = B - B H B + (BH)^2 B - (BH)^3 B + (BH)^4 M^-1.
// tm_hpe_apply computes (BH)^n v with the Dslash kernel in its general form
// (out = A^-1 (-kappa H v), no centre term).  tm_hpe_exact evaluates the exact
// terms for the local insertions: on a lattice whose extents are all >= 4 the
// odd orders have no site-diagonal part, and
//   [B + (BH)^2 B](x, x) = B + kappa^2 sum_mu [B (1 - g_mu) B (1 + g_mu) B + B (1 + g_mu) B (1 - g_mu) B]
// times the colour identity (the two hops of each closed path multiply
// U_mu(x) U_mu(x)^dag = 1, and the antiperiodic sign appears twice), so the
// traces are gauge independent and the same on every site.
#include <complex>

#include "tm_host.h"

namespace tml {

using cd = std::complex<double>;
struct M4 {
  cd m[4][4];
};

static M4 mul(const M4& a, const M4& b) {
  M4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd s = 0;
      for (int k = 0; k < 4; ++k) s += a.m[i][k] * b.m[k][j];
      c.m[i][j] = s;
    }
  return c;
}

static M4 add(const M4& a, const M4& b, double sb = 1.0) {
  M4 c;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) c.m[i][j] = a.m[i][j] + sb * b.m[i][j];
  return c;
}

static M4 identity4() {
  M4 c{};
  for (int i = 0; i < 4; ++i) c.m[i][i] = 1.0;
  return c;
}

// dense 4x4 form of Gamma_n from its phased-permutation table
static M4 gamma_dense(const GammaTab& t, int n) {
  static const cd ph[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
  M4 c{};
  for (int a = 0; a < 4; ++a) c.m[a][t.perm[n][a]] = ph[t.k[n][a]];
  return c;
}

}  // namespace tml

using namespace tml;

extern "C" tm_status_t tm_hpe_apply(tm_op_t* op, void* out, const void* in, int nrhs, int order,
                                    tm_prec_t prec, tm_stream_t strm) {
  if (!op || !out || !in || nrhs < 0 || order < 0) { set_error("tm_hpe_apply: bad argument"); return TM_ERR_ARG; }
  if (out == in) { set_error("tm_hpe_apply: out and in must not overlap"); return TM_ERR_ARG; }
  if ((int)prec < 0 || (int)prec >= kNumPrec) { set_error("tm_hpe_apply: unknown precision"); return TM_ERR_ARG; }
  if (nrhs == 0) return TM_OK;
  const cudaStream_t s = (cudaStream_t)strm;
  const tm_geom_t gg = {{op->g.L[0], op->g.L[1], op->g.L[2], op->g.L[3]}};
  const size_t F = tm_spinor_bytes(&gg, prec, nrhs);
  if (order == 0) {
    if (cudaMemcpyAsync(out, in, F, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      set_error("tm_hpe_apply: copy failed");
      return TM_ERR_CUDA;
    }
    return TM_OK;
  }
  // ping-pong so that the last application lands in out
  void* tmp = nullptr;
  if (order > 1) {
    const tm_status_t sa = dev_alloc(&tmp, F, s, "tm_hpe_apply");
    if (sa != TM_OK) return sa;
  }
  const void* src = in;
  tm_status_t st = TM_OK;
  for (int k = 0; k < order && st == TM_OK; ++k) {
    void* dst = ((order - 1 - k) % 2 == 0) ? out : tmp;
    DslashCall c;
    c.custom = true;
    c.in = src;
    c.out = dst;
    c.nrhs = nrhs;
    c.centre = 0;
    c.hop_scale = -op->kappa;
    c.out_inv = true;
    c.nu = 2.0 * op->kappa * op->mu;
    st = dslash_dispatch(op, prec, c, s);
    src = dst;
  }
  dev_free(tmp, s);
  return st;
}

extern "C" tm_status_t tm_hpe_exact(const tm_params_t* p, double* out) {
  if (!p || !out) { set_error("tm_hpe_exact: null argument"); return TM_ERR_ARG; }
  if (check_geom(p->L) != TM_OK) return TM_ERR_ARG;
  for (int i = 0; i < 4; ++i)
    if (p->L[i] < 4) {
      set_error("tm_hpe_exact: every extent must be >= 4 (got L[%d] = %d): with extent 2 the "
                "second-order term is gauge dependent", i, p->L[i]);
      return TM_ERR_UNSUPPORTED;
    }
  const GammaTab& tab = gamma_tab();
  const double nu = 2.0 * p->kappa * p->mu;
  const M4 g5 = gamma_dense(tab, 15);
  M4 B = add(identity4(), g5, 0.0);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) B.m[i][j] = (identity4().m[i][j] - cd(0, nu) * g5.m[i][j]) / (1.0 + nu * nu);
  M4 D{};
  for (int mu = 0; mu < 4; ++mu) {
    const M4 gm = gamma_dense(tab, 1 << mu);
    const M4 pm = add(identity4(), gm, -1.0), pp = add(identity4(), gm, 1.0);
    D = add(D, mul(mul(mul(mul(B, pm), B), pp), B));
    D = add(D, mul(mul(mul(mul(B, pp), B), pm), B));
  }
  const M4 E = add(B, D, p->kappa * p->kappa);
  const double v3 = (double)p->L[0] * p->L[1] * p->L[2];
  const int T = p->L[3];
  for (int n = 0; n < 16; ++n) {
    const M4 G = gamma_dense(tab, n);
    cd tr = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) tr += G.m[a][b] * E.m[b][a];
    tr *= 3.0 * v3;  // colour trace and the sites of a slice
    for (int t = 0; t < T; ++t) {
      out[2 * (n * T + t)] = tr.real();
      out[2 * (n * T + t) + 1] = tr.imag();
    }
  }
  return TM_OK;
}
