// Twisted-mass Wilson Dslash on the even/odd internal layout.
//
//   (M psi)(x) = psi(x) + i nu g5 psi(x)
//       - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x + mu) + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu) ]
//
// (twisted-mass formulation of Secs. 2.2/2.4, nu = 2 kappa mu, antiperiodic in
// time).  M^dag swaps (1 - g) <-> (1 + g) and nu -> -nu; D_W sets nu = 0.
//
// GB300 design: one thread per (site, right-hand side); the output site's
// neighbours live in the other parity, so each hop reads one 16-byte-chunked
// spinor and one link with fully coalesced 8/16-byte loads.  Each hop is spin
// projected: in the DeGrand-Rossi basis every g_mu is block off-diagonal,
// g_mu = [[0, A_mu], [B_mu, 0]] with A_mu, B_mu 2x2 phased permutations and
// B_mu A_mu = 1, so (1 + s g_mu) psi = (h, s B_mu h) with h = psi_up + s A_mu psi_dn:
// one 2-spinor goes through the link (two SU(3) mat-vecs) per hop.
// Right-hand sides of one block share the link loads through L1.
#pragma once

#include "tm_host.h"

namespace tml {

// A_mu / B_mu of the DeGrand-Rossi basis as (column, phase exponent k of i^k)
// for rows 0 and 1 of the upper-right (A) and lower-left (B) 2x2 blocks.
template <int MU> struct GBlock;
template <> struct GBlock<0> { static constexpr int ac0 = 1, ak0 = 1, ac1 = 0, ak1 = 1, bc0 = 1, bk0 = 3, bc1 = 0, bk1 = 3; };
template <> struct GBlock<1> { static constexpr int ac0 = 1, ak0 = 2, ac1 = 0, ak1 = 0, bc0 = 1, bk0 = 0, bc1 = 0, bk1 = 2; };
template <> struct GBlock<2> { static constexpr int ac0 = 0, ak0 = 1, ac1 = 1, ak1 = 3, bc0 = 0, bk0 = 3, bc1 = 1, bk1 = 1; };
template <> struct GBlock<3> { static constexpr int ac0 = 0, ak0 = 0, ac1 = 1, ak1 = 0, bc0 = 0, bk0 = 0, bc1 = 1, bk1 = 0; };

// acc += bsign * (1 + SGN g_MU) W psi, where W = U (ADJ = false) or U^dag.
template <int MU, int SGN, bool ADJ, class R>
__device__ __forceinline__ void hop(Cx<R> (&acc)[12], const Cx<R> (&psi)[12], const Mat3<R>& U,
                                    R bsign) {
  using G = GBlock<MU>;
  constexpr int s2 = SGN > 0 ? 0 : 2;  // extra phase i^2 = -1 for SGN = -1
  Cx<R> h0[3], h1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h0[c] = psi[c] + iphase<G::ak0 + s2>(psi[3 * (2 + G::ac0) + c]);
    h1[c] = psi[3 + c] + iphase<G::ak1 + s2>(psi[3 * (2 + G::ac1) + c]);
  }
  Cx<R> w0[3], w1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if constexpr (!ADJ) {
        s0 = s0 + U.m[a][b] * h0[b];
        s1 = s1 + U.m[a][b] * h1[b];
      } else {
        s0 = s0 + cmulc(U.m[b][a], h0[b]);
        s1 = s1 + cmulc(U.m[b][a], h1[b]);
      }
    }
    w0[a] = bsign * s0;
    w1[a] = bsign * s1;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = acc[c] + w0[c];
    acc[3 + c] = acc[3 + c] + w1[c];
    // lower rows: SGN * B_mu (w0, w1)
    const Cx<R> wb0 = G::bc0 == 0 ? w0[c] : w1[c];
    const Cx<R> wb1 = G::bc1 == 0 ? w0[c] : w1[c];
    acc[6 + c] = acc[6 + c] + iphase<G::bk0 + s2>(wb0);
    acc[9 + c] = acc[9 + c] + iphase<G::bk1 + s2>(wb1);
  }
}

struct DslashArgs {
  Geom g;
  const void* links;
  DslashCall c;
  double kappa;
  double nu;  // sign included: M uses +nu, M^dag -nu, D_W 0
  int nwarp;
  int rhs_groups;  // number of blockDim.y-wide right-hand-side groups
};

template <class R>
__device__ __forceinline__ R norm2_12(const Cx<R> (&v)[12]) {
  R s = 0;
#pragma unroll
  for (int j = 0; j < 12; ++j) s += v[j].re * v[j].re + v[j].im * v[j].im;
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class S, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128) dslash_kernel(const DslashArgs a) {
  using R = typename Prec<S>::R;
  const Geom& g = a.g;
  const int rg = blockIdx.x % a.rhs_groups;
  const int sb = blockIdx.x / a.rhs_groups;
  const int par = sb & 1;
  const int cb = (sb >> 1) * blockDim.x + threadIdx.x;
  const int rhs = rg * blockDim.y + threadIdx.y;
  const bool in_rhs = rhs < a.c.nrhs;
  const bool act = in_rhs && (a.c.active == nullptr || a.c.active[rhs] != 0);
  double part = 0.0;
  if (act && cb < g.Vh) {
    const Site s = site_of(g, par, cb);
    const int opar = par ^ 1;
    const size_t cs = (size_t)g.Vh;
    const size_t rbase = (size_t)rhs * 2;
    constexpr int NCH = spinor_chunks<S>();
    Cx<R> acc[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = {0, 0};
    // forward hops use (1 - g) for M and (1 + g) for M^dag; backward the opposite
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
#define TM_HOPS(MU)                                                                        \
    {                                                                                      \
      const int lf = lex_fwd(g, s, MU);                                                    \
      const int lb = lex_bwd(g, s, MU);                                                    \
      R sf = 1, sbk = 1;                                                                   \
      if (MU == 3 && g.antiperiodic) {                                                     \
        if (s.c[3] == g.L[3] - 1) sf = -1;                                                 \
        if (s.c[3] == 0) sbk = -1;                                                         \
      }                                                                                    \
      Cx<R> psi[12];                                                                       \
      load_spinor<S>(psi, a.c.in, ((rbase + opar) * NCH) * cs + (size_t)(lf >> 1), cs);    \
      const Mat3<R> Uf = load_link<S, RECON>(a.links, g, MU, par, cb);                     \
      hop<MU, SF, false>(acc, psi, Uf, sf);                                                \
      load_spinor<S>(psi, a.c.in, ((rbase + opar) * NCH) * cs + (size_t)(lb >> 1), cs);    \
      const Mat3<R> Ub = load_link<S, RECON>(a.links, g, MU, opar, lb >> 1);               \
      hop<MU, SB, true>(acc, psi, Ub, sbk);                                                \
    }
    TM_HOPS(0)
    TM_HOPS(1)
    TM_HOPS(2)
    TM_HOPS(3)
#undef TM_HOPS
    const size_t b0 = ((rbase + par) * NCH) * cs + (size_t)cb;
    Cx<R> out[12];
    load_spinor<S>(out, a.c.in, b0, cs);  // centre
    const R kap = (R)a.kappa;
    const R nu = (R)a.nu;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const R tw = j < 6 ? nu : -nu;  // gamma_5 = diag(1, 1, -1, -1)
      const Cx<R> c = out[j];
      out[j] = {c.re - tw * c.im - kap * acc[j].re, c.im + tw * c.re - kap * acc[j].im};
    }
    if constexpr (EPI == EPI_OUT) {
      store_spinor<S>(a.c.out, b0, cs, out);
      if (a.c.partial) part = (double)norm2_12(out);
    } else if constexpr (EPI == EPI_CGUPD) {
      const R al = (R)a.c.alpha[rhs];
      Cx<R> v[12], w[12];
      load_spinor<S>(v, a.c.r, b0, cs);
#pragma unroll
      for (int j = 0; j < 12; ++j) v[j] = v[j] - al * out[j];
      store_spinor<S>(a.c.r, b0, cs, v);
      part = (double)norm2_12(v);
      load_spinor<S>(v, a.c.x, b0, cs);
      load_spinor<S>(w, a.c.p, b0, cs);
#pragma unroll
      for (int j = 0; j < 12; ++j) v[j] = v[j] + al * w[j];
      store_spinor<S>(a.c.x, b0, cs, v);
    } else {  // EPI_RESID
      Cx<R> v[12];
      load_spinor<S>(v, a.c.b, b0, cs);
#pragma unroll
      for (int j = 0; j < 12; ++j) v[j] = v[j] - out[j];
      store_spinor<S>(a.c.out, b0, cs, v);
      part = (double)norm2_12(v);
    }
  }
  if (EPI != EPI_OUT || a.c.partial != nullptr) {
    part = warp_sum(part);
    if (threadIdx.x % 32 == 0 && in_rhs && cb < a.nwarp * 32)
      a.c.partial[((size_t)rhs * 2 + par) * a.nwarp + cb / 32] = part;
  }
}

template <class S, int RECON, bool DAG, int EPI>
tm_status_t launch_one(const tm_op* op, const DslashCall& c, cudaStream_t st) {
  DslashArgs a;
  a.g = op->g;
  a.links = op->links[Prec<S>::id];
  a.c = c;
  a.kappa = op->kappa;
  a.nu = c.mu_zero ? 0.0 : (DAG ? -2.0 * op->kappa * op->mu : 2.0 * op->kappa * op->mu);
  a.nwarp = nwarp_of(op->g);
  const int bx = 128;
  // several right-hand sides per block share link loads through L1; the
  // block stays at 128 threads
  int by = 1;
  while (by * 2 <= c.nrhs && by < 4) by *= 2;
  dim3 block(bx / by, by);
  a.rhs_groups = (c.nrhs + by - 1) / by;
  const int site_blocks = 2 * ((op->g.Vh + (int)block.x - 1) / (int)block.x);
  dim3 grid((unsigned)(site_blocks * a.rhs_groups));
  // trace class: dslash.<precision>.<epilogue>
  static const char* const kNames[4][3] = {
      {"dslash.f64.out", "dslash.f64.cgupd", "dslash.f64.resid"},
      {"dslash.f32.out", "dslash.f32.cgupd", "dslash.f32.resid"},
      {"dslash.f16.out", "dslash.f16.cgupd", "dslash.f16.resid"},
      {"dslash.bf16.out", "dslash.bf16.cgupd", "dslash.bf16.resid"}};
  const char* name = kNames[Prec<S>::id][EPI];
  cudaEvent_t ev = nullptr;
  trace_begin(st, name, &ev);
  dslash_kernel<S, RECON, DAG, EPI><<<grid, block, 0, st>>>(a);
  count_launch();
  trace_end(st, name, ev);
  return check_launch("dslash");
}

template <class S, int RECON>
tm_status_t dslash_launch(const tm_op* op, const DslashCall& c, cudaStream_t st) {
  if (c.dagger) {
    switch (c.epi) {
      case EPI_OUT: return launch_one<S, RECON, true, EPI_OUT>(op, c, st);
      case EPI_CGUPD: return launch_one<S, RECON, true, EPI_CGUPD>(op, c, st);
      default: return launch_one<S, RECON, true, EPI_RESID>(op, c, st);
    }
  }
  switch (c.epi) {
    case EPI_OUT: return launch_one<S, RECON, false, EPI_OUT>(op, c, st);
    case EPI_CGUPD: return launch_one<S, RECON, false, EPI_CGUPD>(op, c, st);
    default: return launch_one<S, RECON, false, EPI_RESID>(op, c, st);
  }
}

#define TM_INSTANTIATE_DSLASH(S)                                                           \
  template tm_status_t dslash_launch<S, 18>(const tm_op*, const DslashCall&, cudaStream_t); \
  template tm_status_t dslash_launch<S, 12>(const tm_op*, const DslashCall&, cudaStream_t);

}  // namespace tml
