// Twisted-mass Wilson Dslash on the even/odd internal layout.
//
//   (M psi)(x) = psi(x) + i nu g5 psi(x)
//       - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x + mu) + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu) ]
//
// (twisted-mass formulation of Secs. 2.2/2.4, nu = 2 kappa mu, antiperiodic in
// time).  M^dag swaps (1 - g) <-> (1 + g) and nu -> -nu; D_W sets nu = 0.
// The same kernel evaluates the pieces of the even/odd Schur complement
//   M_hat = A - kappa^2 H_oe A^-1 H_eo,   A = 1 + i nu g5,
// through a general form on one or both output parities:
//   out = T_out( T_c(c) + s_hop * H in ),   T_c in {0, 1, A},  T_out in {1, A^-1},
// with H the hopping term (dagger: swapped projectors) and c a centre field.
//
// GB300 design: one thread per site computes NR right-hand sides; the site's
// index arithmetic and its link loads (and 12-real reconstruction) are shared
// by the NR systems, which are read from their own fields with coalesced
// 8/16-byte loads.  Each hop is spin projected: in the DeGrand-Rossi basis
// every g_mu is block off-diagonal, g_mu = [[0, A_mu], [B_mu, 0]] with A_mu,
// B_mu 2x2 phased permutations and B_mu A_mu = 1, so
// (1 + s g_mu) psi = (h, s B_mu h) with h = psi_up + s A_mu psi_dn: one
// 2-spinor goes through the link (two SU(3) mat-vecs) per hop.  All floating
// point operations are explicit round-to-nearest intrinsics, so the result of
// one system does not depend on NR or on which systems share its launch.
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

// explicit round-to-nearest arithmetic
template <class R> struct Ar;
// norm: renormalise a float-float value at the end of a multiply-add chain
// (identity for the IEEE types)
template <> struct Ar<float> {
  static __device__ __forceinline__ float norm(float a) { return a; }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Ar<FF> {
  static __device__ __forceinline__ FF norm(FF a) { return ff_norm(a); }
  static __device__ __forceinline__ FF add(FF a, FF b) { return a + b; }
  static __device__ __forceinline__ FF sub(FF a, FF b) { return a - b; }
  static __device__ __forceinline__ FF mul(FF a, FF b) { return a * b; }
  static __device__ __forceinline__ FF fma(FF a, FF b, FF c) { return ff_fma(a, b, c); }
};
template <> struct Ar<double> {
  static __device__ __forceinline__ double norm(double a) { return a; }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// a + i^K b
template <int K, class R>
__device__ __forceinline__ Cx<R> add_ph(Cx<R> a, Cx<R> b) {
  using O = Ar<R>;
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return {O::add(a.re, b.re), O::add(a.im, b.im)};
  else if constexpr (k == 1) return {O::sub(a.re, b.im), O::add(a.im, b.re)};
  else if constexpr (k == 2) return {O::sub(a.re, b.re), O::sub(a.im, b.im)};
  else return {O::add(a.re, b.im), O::sub(a.im, b.re)};
}

// Spin projection h = psi_up + SGN A_mu psi_dn (rows 0 and 1 of (1 + SGN g_MU) psi).
template <int MU, int SGN, class R>
__device__ __forceinline__ void project(Cx<R> (&h0)[3], Cx<R> (&h1)[3], const Cx<R> (&psi)[12]) {
  using G = GBlock<MU>;
  constexpr int s2 = SGN > 0 ? 0 : 2;  // extra phase i^2 = -1 for SGN = -1
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h0[c] = add_ph<G::ak0 + s2>(psi[c], psi[3 * (2 + G::ac0) + c]);
    h1[c] = add_ph<G::ak1 + s2>(psi[3 + c], psi[3 * (2 + G::ac1) + c]);
  }
}

// FP16 / BF16 storage: sm_100+ adds a 16-bit operand to an FP32 one in one
// instruction with one rounding (add/sub.rn.f32.f16|bf16), so psi_up enters
// the projection unconverted: the result is bit-identical to converting it
// first, with 12 conversions fewer per hop.
template <class S> struct Mixed;
template <> struct Mixed<__half> {
  // a b + c with a, b 16-bit: the product is exact in FP32, one rounding
  static __device__ __forceinline__ float fma(unsigned short a, unsigned short b, float c) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
    return d;
  }
  static __device__ __forceinline__ float add(unsigned short a, float c) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
  }
  static __device__ __forceinline__ float sub(unsigned short a, float c) {
    float d;
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
  }
};
template <> struct Mixed<__nv_bfloat16> {
  static __device__ __forceinline__ float fma(unsigned short a, unsigned short b, float c) {
    float d;
    asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
    return d;
  }
  static __device__ __forceinline__ float add(unsigned short a, float c) {
    float d;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
  }
  static __device__ __forceinline__ float sub(unsigned short a, float c) {
    float d;
    asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
  }
};

// complex k (= 3 spin + colour) of a raw 16-bit spinor: one 32-bit word, re in
// the low half
__device__ __forceinline__ unsigned raw_word(const uint4 (&q)[3], int k) {
  const uint4& v = q[k >> 2];
  return (k & 3) == 0 ? v.x : (k & 3) == 1 ? v.y : (k & 3) == 2 ? v.z : v.w;
}

// a + i^K b with a raw (16-bit) and b in FP32
template <int K, class S>
__device__ __forceinline__ Cx<float> add_ph_raw(unsigned a, Cx<float> b) {
  using M = Mixed<S>;
  constexpr int k = ((K % 4) + 4) % 4;
  const unsigned short ar = (unsigned short)(a & 0xffffu), ai = (unsigned short)(a >> 16);
  if constexpr (k == 0) return {M::add(ar, b.re), M::add(ai, b.im)};
  else if constexpr (k == 1) return {M::sub(ar, b.im), M::add(ai, b.re)};
  else if constexpr (k == 2) return {M::sub(ar, b.re), M::sub(ai, b.im)};
  else return {M::add(ar, b.im), M::sub(ai, b.re)};
}

// a raw 16-bit complex (one 32-bit word) converted to FP32
template <class S>
__device__ __forceinline__ Cx<float> raw_to_f32(unsigned w) {
  const unsigned short lo = (unsigned short)(w & 0xffffu), hi = (unsigned short)(w >> 16);
  if constexpr (std::is_same<S, __half>::value)
    return {__half2float(__ushort_as_half(lo)), __half2float(__ushort_as_half(hi))};
  else
    return {__bfloat162float(__ushort_as_bfloat16(lo)), __bfloat162float(__ushort_as_bfloat16(hi))};
}

template <int MU, int SGN, class S>
__device__ __forceinline__ void project_raw(Cx<float> (&h0)[3], Cx<float> (&h1)[3], const uint4 (&q)[3]) {
  using G = GBlock<MU>;
  constexpr int s2 = SGN > 0 ? 0 : 2;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h0[c] = add_ph_raw<G::ak0 + s2, S>(raw_word(q, c), raw_to_f32<S>(raw_word(q, 3 * (2 + G::ac0) + c)));
    h1[c] = add_ph_raw<G::ak1 + s2, S>(raw_word(q, 3 + c), raw_to_f32<S>(raw_word(q, 3 * (2 + G::ac1) + c)));
  }
}

// 16-bit storage with 18-real links: every factor of a link product is a
// 16-bit number in memory, and the mixed-precision FMA (fma.rn.f32.f16|bf16)
// multiplies two of them exactly and adds in FP32 with one rounding.  The
// products therefore skip the conversions of the link and of the spinor and
// give the bits of link_times2 on converted operands: same operations in the
// same order, with each sign moved onto the spinor factor (exact).
template <class S, int RECON>
constexpr bool kRawLinks =
    (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) && RECON == 18;

// the 9 complex entries of a link (row-major), one 32-bit word each (re low)
template <class S>
__device__ __forceinline__ void load_link_raw(unsigned (&u)[9], const void* links, const Geom& g, int mu,
                                              int par, int cb) {
  using F = LinkFmt<S, 18>;
  const uint4* p = reinterpret_cast<const uint4*>(links);
  const size_t b0 = ((size_t)(mu * 2 + par) * F::NU) * (size_t)g.Vh + (size_t)cb;
  const size_t cs = (size_t)g.Vh;
  const uint4 a = p[b0], b = p[b0 + cs];
  u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
  u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
  u[8] = reinterpret_cast<const unsigned*>(p + b0 + 2 * cs)[0];
}

// components 6h .. 6h + 5 of a 16-bit spinor, one word per complex number
template <class S>
__device__ __forceinline__ void load_spins2_raw(unsigned (&x)[6], const void* field, size_t b0, size_t cs,
                                                int h) {
  const uint4* f = reinterpret_cast<const uint4*>(field);
  const uint4 a = f[b0 + h * cs], b = f[b0 + (h + 1) * cs];
  const unsigned e[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int j = 0; j < 6; ++j) x[j] = h ? e[2 + j] : e[j];
}

template <bool ADJ, bool SUB, class S>
__device__ __forceinline__ void link_times2_raw(Cx<float> (&w)[6], const unsigned (&u)[9], const unsigned (&x)[6]) {
  using M = Mixed<S>;
  // signs of Re u and Im u in (ADJ ? conj(U) : U), negated for SUB
  constexpr bool pre = !SUB, pim = ADJ == SUB;
  unsigned xn[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) xn[j] = x[j] ^ 0x80008000u;  // -x
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float zr = SUB ? w[3 * a + c].re : 0.0f, zi = SUB ? w[3 * a + c].im : 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const unsigned uw = ADJ ? u[3 * d + c] : u[3 * c + d];
        const unsigned short ur = (unsigned short)(uw & 0xffffu), ui = (unsigned short)(uw >> 16);
        const unsigned xp = x[3 * a + d], xm = xn[3 * a + d];
        const unsigned short xpr = (unsigned short)(xp & 0xffffu), xpi = (unsigned short)(xp >> 16);
        const unsigned short xmr = (unsigned short)(xm & 0xffffu), xmi = (unsigned short)(xm >> 16);
        zr = M::fma(ur, pre ? xpr : xmr, zr);    // Re u Re x
        zr = M::fma(ui, pim ? xmi : xpi, zr);    // -Im u Im x
        zi = M::fma(ur, pre ? xpi : xmi, zi);    // Re u Im x
        zi = M::fma(ui, pim ? xpr : xmr, zi);    // Im u Re x
      }
      w[3 * a + c] = {zr, zi};
    }
}

// Packed 16-bit pairs held as 32-bit words (low half = real part):
// f16x2 / bf16x2 add with round-to-nearest.
template <class S>
__device__ __forceinline__ unsigned hadd2_w(unsigned a, unsigned b) {
  unsigned d;
  if constexpr (std::is_same<S, __half>::value) asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  else asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// a + i^K b on 16-bit complex words, rounded once to the storage format: the
// i^K rotation only swaps halves and flips signs (exact), then one packed add
template <int K, class S>
__device__ __forceinline__ unsigned add_ph_w(unsigned a, unsigned b) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return hadd2_w<S>(a, b);
  else if constexpr (k == 2) return hadd2_w<S>(a, b ^ 0x80008000u);
  else if constexpr (k == 1) return hadd2_w<S>(a, __byte_perm(b, 0u, 0x1032) ^ 0x00008000u);  // (-b.im, b.re)
  else return hadd2_w<S>(a, __byte_perm(b, 0u, 0x1032) ^ 0x80000000u);                        // (b.im, -b.re)
}

// FP16/BF16 with 18-real links: one hop straight from the 16-bit words.  The
// projection h = psi_up + SGN A_mu psi_dn is one packed add per complex entry
// (one rounding to the storage format, like storing h), the link product
// multiplies the 16-bit link and h words exactly with the mixed FMA and
// accumulates in FP32, and the time-boundary sign flips h's sign bits.  No
// FP16 -> FP32 conversion at all.
template <class S, int MU, int SGN, bool ADJ>
__device__ __forceinline__ void hop_site_w(Cx<float> (&acc)[12], const void* field, size_t b0, size_t cs,
                                           const unsigned (&u)[9], unsigned negmask) {
  using G = GBlock<MU>;
  constexpr int s2 = SGN > 0 ? 0 : 2;
  const uint4* f = reinterpret_cast<const uint4*>(field);
  uint4 q[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) q[j] = f[b0 + j * cs];
  unsigned h[6];  // (h0[0..2], h1[0..2])
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h[c] = add_ph_w<G::ak0 + s2, S>(raw_word(q, c), raw_word(q, 3 * (2 + G::ac0) + c)) ^ negmask;
    h[3 + c] = add_ph_w<G::ak1 + s2, S>(raw_word(q, 3 + c), raw_word(q, 3 * (2 + G::ac1) + c)) ^ negmask;
  }
  Cx<float> w[6];
  link_times2_raw<ADJ, false, S>(w, u, h);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = add_ph<0>(acc[c], w[c]);
    acc[3 + c] = add_ph<0>(acc[3 + c], w[3 + c]);
    const Cx<float> wb0 = G::bc0 == 0 ? w[c] : w[3 + c];
    const Cx<float> wb1 = G::bc1 == 0 ? w[c] : w[3 + c];
    acc[6 + c] = add_ph<G::bk0 + s2>(acc[6 + c], wb0);
    acc[9 + c] = add_ph<G::bk1 + s2>(acc[9 + c], wb1);
  }
}

// acc += bsign * (1 + SGN g_MU) W psi given the projection (h0, h1) of psi,
// where W = U (ADJ = false) or U^dag.
template <int MU, int SGN, bool ADJ, class R>
__device__ __forceinline__ void hop_acc(Cx<R> (&acc)[12], const Cx<R> (&h0)[3], const Cx<R> (&h1)[3],
                                        const Mat3<R>& U, R bsign) {
  using G = GBlock<MU>;
  using O = Ar<R>;
  constexpr int s2 = SGN > 0 ? 0 : 2;
  Cx<R> w0[3], w1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R r0 = 0, i0 = 0, r1 = 0, i1 = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cx<R> u = ADJ ? conjx(U.m[b][a]) : U.m[a][b];
      if (b == 0) {
        r0 = O::mul(u.re, h0[b].re); i0 = O::mul(u.re, h0[b].im);
        r1 = O::mul(u.re, h1[b].re); i1 = O::mul(u.re, h1[b].im);
      } else {
        r0 = O::fma(u.re, h0[b].re, r0); i0 = O::fma(u.re, h0[b].im, i0);
        r1 = O::fma(u.re, h1[b].re, r1); i1 = O::fma(u.re, h1[b].im, i1);
      }
      r0 = O::fma(-u.im, h0[b].im, r0); i0 = O::fma(u.im, h0[b].re, i0);
      r1 = O::fma(-u.im, h1[b].im, r1); i1 = O::fma(u.im, h1[b].re, i1);
    }
    if (MU == 3) {
      r0 = O::mul(bsign, r0); i0 = O::mul(bsign, i0);
      r1 = O::mul(bsign, r1); i1 = O::mul(bsign, i1);
    }
    w0[a] = {r0, i0};
    w1[a] = {r1, i1};
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = add_ph<0>(acc[c], w0[c]);
    acc[3 + c] = add_ph<0>(acc[3 + c], w1[c]);
    // lower rows: SGN * B_mu (w0, w1)
    const Cx<R> wb0 = G::bc0 == 0 ? w0[c] : w1[c];
    const Cx<R> wb1 = G::bc1 == 0 ? w0[c] : w1[c];
    acc[6 + c] = add_ph<G::bk0 + s2>(acc[6 + c], wb0);
    acc[9 + c] = add_ph<G::bk1 + s2>(acc[9 + c], wb1);
  }
}

// acc += bsign * (1 + SGN g_MU) W psi with psi the field's site at b0
template <class S, int MU, int SGN, bool ADJ>
__device__ __forceinline__ void hop_site(Cx<typename Prec<S>::R> (&acc)[12], const void* field, size_t b0,
                                         size_t cs, const Mat3<typename Prec<S>::R>& U,
                                         typename Prec<S>::R bsign) {
  using R = typename Prec<S>::R;
  Cx<R> h0[3], h1[3];
  if constexpr (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) {
    const uint4* f = reinterpret_cast<const uint4*>(field);
    uint4 q[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) q[j] = f[b0 + j * cs];
    project_raw<MU, SGN, S>(h0, h1, q);
  } else {
    Cx<R> psi[12];
    load_spinor<S>(psi, field, b0, cs);
    project<MU, SGN>(h0, h1, psi);
  }
  hop_acc<MU, SGN, ADJ>(acc, h0, h1, U, bsign);
}

// Link product of a projected 2-spinor: w = W (h0, h1), W = U (ADJ = false) or
// U^dag; with START = false it accumulates onto w (w += W h).  w[0..2] is the
// product of h0, w[3..5] that of h1.
template <bool ADJ, bool START, class R>
__device__ __forceinline__ void link_mv2(Cx<R> (&w)[6], const Mat3<R>& U, const Cx<R> (&h0)[3],
                                         const Cx<R> (&h1)[3]) {
  using O = Ar<R>;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R r0, i0, r1, i1;
    if (!START) { r0 = w[a].re; i0 = w[a].im; r1 = w[3 + a].re; i1 = w[3 + a].im; }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cx<R> u = ADJ ? conjx(U.m[b][a]) : U.m[a][b];
      if (START && b == 0) {
        r0 = O::mul(u.re, h0[b].re); i0 = O::mul(u.re, h0[b].im);
        r1 = O::mul(u.re, h1[b].re); i1 = O::mul(u.re, h1[b].im);
      } else {
        r0 = O::fma(u.re, h0[b].re, r0); i0 = O::fma(u.re, h0[b].im, i0);
        r1 = O::fma(u.re, h1[b].re, r1); i1 = O::fma(u.re, h1[b].im, i1);
      }
      r0 = O::fma(-u.im, h0[b].im, r0); i0 = O::fma(u.im, h0[b].re, i0);
      r1 = O::fma(-u.im, h1[b].im, r1); i1 = O::fma(u.im, h1[b].re, i1);
    }
    w[a] = {O::norm(r0), O::norm(i0)};
    w[3 + a] = {O::norm(r1), O::norm(i1)};
  }
}

// Load the site at b0 and project it: (h0, h1) = rows 0, 1 of (1 + SGN g_MU) psi,
// negated when neg (the antiperiodic sign of a hop across the time boundary).
template <class S, int MU, int SGN>
__device__ __forceinline__ void load_project(Cx<typename Prec<S>::R> (&h0)[3], Cx<typename Prec<S>::R> (&h1)[3],
                                             const void* field, size_t b0, size_t cs, bool neg) {
  using R = typename Prec<S>::R;
  if constexpr (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) {
    const uint4* f = reinterpret_cast<const uint4*>(field);
    uint4 q[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) q[j] = f[b0 + j * cs];
    project_raw<MU, SGN, S>(h0, h1, q);
  } else {
    Cx<R> psi[12];
    load_spinor<S>(psi, field, b0, cs);
    project<MU, SGN>(h0, h1, psi);
  }
  if (MU == 3 && neg) {  // warp-uniform: only on the first and last time slice
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[c] = {-h0[c].re, -h0[c].im};
      h1[c] = {-h1[c].re, -h1[c].im};
    }
  }
}

// Both hops of direction MU together: with w_f the forward and w_b the backward
// link product (projection signs SF and SB = -SF), the upper spins receive
// w_f + w_b and the lower ones SF B_mu (w_f - w_b).  sum = w_f + w_b is
// accumulated onto w_f; w_f - w_b = 2 w_f - sum.
template <int MU, int SF, class R>
__device__ __forceinline__ void combine_dir(Cx<R> (&acc)[12], const Cx<R> (&wf)[6], const Cx<R> (&sum)[6]) {
  using G = GBlock<MU>;
  using O = Ar<R>;
  constexpr int s2 = SF > 0 ? 0 : 2;
  const R two = (R)2;
  Cx<R> d[6];
#pragma unroll
  for (int k = 0; k < 6; ++k)
    d[k] = {O::norm(O::fma(two, wf[k].re, -sum[k].re)), O::norm(O::fma(two, wf[k].im, -sum[k].im))};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = add_ph<0>(acc[c], sum[c]);
    acc[3 + c] = add_ph<0>(acc[3 + c], sum[3 + c]);
    const Cx<R> db0 = G::bc0 == 0 ? d[c] : d[3 + c];
    const Cx<R> db1 = G::bc1 == 0 ? d[c] : d[3 + c];
    acc[6 + c] = add_ph<G::bk0 + s2>(acc[6 + c], db0);
    acc[9 + c] = add_ph<G::bk1 + s2>(acc[9 + c], db1);
  }
}

struct DslashArgs {
  Geom g;
  const void* links;
  DslashCall c;
  double nu;         // twist of T_c / T_out
  double hop_scale;  // s_hop
  double inv;        // 1 / (1 + nu^2), the scale of A^-1
  float nu_f, hop_scale_f, inv_f;  // the same in FP32 for the narrow formats
  int nwarp;
  int rhs_groups;    // number of NR-wide right-hand-side groups
  int* trace_count;  // tracing: number of active systems of this launch
};

template <class R>
__device__ __forceinline__ R norm2_12(const Cx<R> (&v)[12]) {
  using O = Ar<R>;
  R s = 0;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    s = O::fma(v[j].re, v[j].re, s);
    s = O::fma(v[j].im, v[j].im, s);
  }
  return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Minimum resident blocks per SM requested from the compiler (caps the
// registers per thread).  The narrow formats are latency/issue bound and gain
// from occupancy: measured at 32^3 x 64, 16 systems, one system per thread, 7
// blocks (72 registers) is fastest for FP16/BF16 (8 blocks = 64 registers
// spills), 6 for FP32.  Several systems per thread need registers in
// proportion (4 blocks for 2, 2 for 4), so that the autotuner compares them
// without forced spills.  FP64 and float-float are arithmetic bound and keep
// their registers.  TM_DSLASH_MINBLOCKS (TM_DSLASH_MINBLOCKS_F32 for FP32
// only) overrides the one-system value at build time.
template <class S, int NR = 1>
constexpr int dslash_min_blocks() {
  if constexpr (std::is_same<S, double>::value) return 1;
  else if constexpr (std::is_same<S, FFloat>::value) return 2;
  else if constexpr (NR >= 4) return 2;
  else if constexpr (NR == 2) return 4;
#ifdef TM_DSLASH_MINBLOCKS_F32
  else if constexpr (std::is_same<S, float>::value) return TM_DSLASH_MINBLOCKS_F32;
#endif
#ifdef TM_DSLASH_MINBLOCKS
  else return TM_DSLASH_MINBLOCKS;
#else
  else return std::is_same<S, float>::value ? 6 : 7;
#endif
}

// Scalars of the epilogue in the arithmetic type (FP32 copies for the narrow
// formats: no FP64 arithmetic in their kernels)
template <class R>
struct EpiConsts {
  R shop, nu, inv;
  const void* cfield;
};
template <class R>
__device__ __forceinline__ EpiConsts<R> epi_consts(const DslashArgs& a) {
  EpiConsts<R> k;
  if constexpr (kWide<R>) {
    k.shop = (R)a.hop_scale; k.nu = (R)a.nu; k.inv = (R)a.inv;
  } else {
    k.shop = a.hop_scale_f; k.nu = a.nu_f; k.inv = a.inv_f;
  }
  k.cfield = a.c.cfield ? a.c.cfield : a.c.in;
  return k;
}

// Everything after the hopping sum acc = H in at output site cb of parity par
// for system r: out = T_out(T_c(c) + s_hop acc), then the epilogue of EPI.
// Returns the system's |.|^2 contribution to the partial sums (0 if none).
template <class S, int EPI, class R>
__device__ __forceinline__ double dslash_epilogue(const DslashArgs& a, const EpiConsts<R>& k, int r, int par,
                                                  int cb, const Cx<R> (&acc)[12]) {
  using O = Ar<R>;
  constexpr int NCH = spinor_chunks<S>();
  const size_t cs = (size_t)a.g.Vh;
  const R shop = k.shop, nu = k.nu, inv = k.inv;
  const size_t b0 = ((size_t)(r * 2 + par) * NCH) * cs + cb;
  Cx<R> out[12];
  if (a.c.centre != 0) {
    load_spinor<S>(out, k.cfield, b0, cs);
    if (a.c.centre == 2) {  // A c = c + i nu g5 c
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const R tw = q < 6 ? nu : -nu;  // gamma_5 = diag(1, 1, -1, -1)
        const Cx<R> c = out[q];
        out[q] = {O::fma(-tw, c.im, c.re), O::fma(tw, c.re, c.im)};
      }
    }
#pragma unroll
    for (int q = 0; q < 12; ++q)
      out[q] = {O::fma(shop, acc[q].re, out[q].re), O::fma(shop, acc[q].im, out[q].im)};
  } else {
#pragma unroll
    for (int q = 0; q < 12; ++q) out[q] = {O::mul(shop, acc[q].re), O::mul(shop, acc[q].im)};
  }
  if constexpr (std::is_same<R, FF>::value) {
#pragma unroll
    for (int q = 0; q < 12; ++q) out[q] = {O::norm(out[q].re), O::norm(out[q].im)};
  }
  if (a.c.out_inv) {  // A^-1 v = (v - i nu g5 v) / (1 + nu^2)
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const R tw = q < 6 ? nu : -nu;
      const Cx<R> v = out[q];
      out[q] = {O::mul(inv, O::norm(O::fma(tw, v.im, v.re))), O::mul(inv, O::norm(O::fma(-tw, v.re, v.im)))};
    }
  }
  double part = 0.0;
  if constexpr (EPI == EPI_OUT) {
    if (a.c.g5_out) {  // gamma_5 = diag(1, 1, -1, -1)
#pragma unroll
      for (int q = 6; q < 12; ++q) out[q] = {-out[q].re, -out[q].im};
    }
    store_spinor<S>(a.c.out, b0, cs, out);
    if (a.c.partial) part = (double)norm2_12(out);
  } else if constexpr (EPI == EPI_CGUPD) {
    const R al = (R)a.c.alpha[r];
    Cx<R> v[12];
    load_spinor<S>(v, a.c.r, b0, cs);
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = {O::fma(-al, out[q].re, v[q].re), O::fma(-al, out[q].im, v[q].im)};
    store_spinor<S>(a.c.r, b0, cs, v);
    part = (double)norm2_12(v);
    Cx<R> w[12];
    load_spinor<S>(v, a.c.x, b0, cs);
    load_spinor<S>(w, a.c.p, b0, cs);
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = {O::fma(al, w[q].re, v[q].re), O::fma(al, w[q].im, v[q].im)};
    store_spinor<S>(a.c.x, b0, cs, v);
  } else {  // EPI_RESID
    Cx<R> v[12];
    load_spinor<S>(v, a.c.b, b0, cs);
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = {O::sub(v[q].re, out[q].re), O::sub(v[q].im, out[q].im)};
    store_spinor<S>(a.c.out, b0, cs, v);
    part = (double)norm2_12(v);
  }
  return part;
}

template <class S, int RECON, bool DAG, int EPI, int NR>
__global__ void __launch_bounds__(128, (dslash_min_blocks<S, NR>())) dslash_kernel(const DslashArgs a) {
  using R = typename Prec<S>::R;
  using O = Ar<R>;
  const Geom& g = a.g;
  const int rg = blockIdx.x % a.rhs_groups;
  const int sb = blockIdx.x / a.rhs_groups;
  const int par = a.c.parity < 0 ? (sb & 1) : a.c.parity;
  const int cbb = a.c.parity < 0 ? (sb >> 1) : sb;
  const int cb = cbb * blockDim.x + threadIdx.x;
  const int nrhs = a.c.nrhs;
  int rhs[NR];
  bool act[NR];
  bool any = false;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int r = rg * NR + j;
    act[j] = r < nrhs && (a.c.active == nullptr || a.c.active[r] != 0);
    rhs[j] = r < nrhs ? r : rg * NR;  // padding systems are never loaded nor stored
    any = any || act[j];
  }
  double part[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) part[j] = 0.0;
  if (a.trace_count && blockIdx.x == 0 && threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < nrhs; ++r) n += (a.c.active == nullptr || a.c.active[r] != 0) ? 1 : 0;
    *a.trace_count = n;
  }
  if (any && cb < g.Vh) {
    const Site s = site_of(g, par, cb);
    const int opar = par ^ 1;
    const size_t cs = (size_t)g.Vh;
    constexpr int NCH = spinor_chunks<S>();
    Cx<R> acc[NR][12];
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[j][k] = {0, 0};
    // forward hops use (1 - g) for M and (1 + g) for M^dag; backward the opposite
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
// FP32/FP64/float-float: both hops of a direction combined (combine_dir), the
// time-boundary sign on the projected spinor.  FP16/BF16: one hop at a time,
// which holds fewer registers and spills less in this register-capped,
// issue-bound kernel (measured faster); with 18-real links entirely on the
// 16-bit words (hop_site_w), with 12-real links on converted values (hop_site).
#define TM_HOPS(MU)                                                                              \
    {                                                                                            \
      const int lf = lex_fwd(g, s, MU);                                                          \
      const int lb = lex_bwd(g, s, MU);                                                          \
      if constexpr (kRawLinks<S, RECON>) {                                                       \
        const unsigned negf = (MU == 3 && g.antiperiodic && s.c[3] == g.L[3] - 1) ? 0x80008000u : 0u; \
        const unsigned negb = (MU == 3 && g.antiperiodic && s.c[3] == 0) ? 0x80008000u : 0u;      \
        {                                                                                        \
          unsigned u[9];                                                                         \
          load_link_raw<S>(u, a.links, g, MU, par, cb);                                          \
          _Pragma("unroll") for (int j = 0; j < NR; ++j) {                                       \
            if (!act[j]) continue;                                                               \
            hop_site_w<S, MU, SF, false>(acc[j], a.c.in, ((size_t)(rhs[j] * 2 + opar) * NCH) * cs + (lf >> 1), \
                                         cs, u, negf);                                           \
          }                                                                                      \
        }                                                                                        \
        {                                                                                        \
          unsigned u[9];                                                                         \
          load_link_raw<S>(u, a.links, g, MU, opar, lb >> 1);                                    \
          _Pragma("unroll") for (int j = 0; j < NR; ++j) {                                       \
            if (!act[j]) continue;                                                               \
            hop_site_w<S, MU, SB, true>(acc[j], a.c.in, ((size_t)(rhs[j] * 2 + opar) * NCH) * cs + (lb >> 1), \
                                        cs, u, negb);                                            \
          }                                                                                      \
        }                                                                                        \
      } else if constexpr (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) { \
        R sf = 1, sbk = 1;                                                                       \
        if (MU == 3 && g.antiperiodic) {                                                         \
          if (s.c[3] == g.L[3] - 1) sf = -1;                                                     \
          if (s.c[3] == 0) sbk = -1;                                                             \
        }                                                                                        \
        {                                                                                        \
          const Mat3<R> Uf = load_link<S, RECON>(a.links, g, MU, par, cb);                       \
          _Pragma("unroll") for (int j = 0; j < NR; ++j) {                                       \
            if (!act[j]) continue;                                                               \
            hop_site<S, MU, SF, false>(acc[j], a.c.in, ((size_t)(rhs[j] * 2 + opar) * NCH) * cs + (lf >> 1), \
                                       cs, Uf, sf);                                              \
          }                                                                                      \
        }                                                                                        \
        {                                                                                        \
          const Mat3<R> Ub = load_link<S, RECON>(a.links, g, MU, opar, lb >> 1);                 \
          _Pragma("unroll") for (int j = 0; j < NR; ++j) {                                       \
            if (!act[j]) continue;                                                               \
            hop_site<S, MU, SB, true>(acc[j], a.c.in, ((size_t)(rhs[j] * 2 + opar) * NCH) * cs + (lb >> 1), \
                                      cs, Ub, sbk);                                              \
          }                                                                                      \
        }                                                                                        \
      } else {                                                                                   \
        const bool negf = MU == 3 && g.antiperiodic && s.c[3] == g.L[3] - 1;                     \
        const bool negb = MU == 3 && g.antiperiodic && s.c[3] == 0;                              \
        Cx<R> wf[NR][6];                                                                         \
        {                                                                                        \
          const Mat3<R> Uf = load_link<S, RECON>(a.links, g, MU, par, cb);                       \
          _Pragma("unroll") for (int j = 0; j < NR; ++j) {                                       \
            if (!act[j]) continue;                                                               \
            Cx<R> h0[3], h1[3];                                                                  \
            load_project<S, MU, SF>(h0, h1, a.c.in, ((size_t)(rhs[j] * 2 + opar) * NCH) * cs + (lf >> 1), \
                                    cs, negf);                                                   \
            link_mv2<false, true>(wf[j], Uf, h0, h1);                                            \
          }                                                                                      \
        }                                                                                        \
        {                                                                                        \
          const Mat3<R> Ub = load_link<S, RECON>(a.links, g, MU, opar, lb >> 1);                 \
          _Pragma("unroll") for (int j = 0; j < NR; ++j) {                                       \
            if (!act[j]) continue;                                                               \
            Cx<R> h0[3], h1[3];                                                                  \
            load_project<S, MU, SB>(h0, h1, a.c.in, ((size_t)(rhs[j] * 2 + opar) * NCH) * cs + (lb >> 1), \
                                    cs, negb);                                                   \
            Cx<R> sum[6];                                                                        \
            _Pragma("unroll") for (int k = 0; k < 6; ++k) sum[k] = wf[j][k];                     \
            link_mv2<true, false>(sum, Ub, h0, h1);                                              \
            combine_dir<MU, SF>(acc[j], wf[j], sum);                                             \
          }                                                                                      \
        }                                                                                        \
      }                                                                                          \
    }
    TM_HOPS(0)
    TM_HOPS(1)
    TM_HOPS(2)
    TM_HOPS(3)
#undef TM_HOPS
    const EpiConsts<R> k = epi_consts<R>(a);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (!act[j]) continue;
      part[j] = dslash_epilogue<S, EPI>(a, k, rhs[j], par, cb, acc[j]);
    }
  }
  if (EPI != EPI_OUT || a.c.partial != nullptr) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double ps = warp_sum(part[j]);
      const int r = rg * NR + j;
      if (threadIdx.x % 32 == 0 && r < nrhs && cb < a.nwarp * 32)
        a.c.partial[((size_t)r * 2 + par) * a.nwarp + cb / 32] = ps;
    }
  }
}

}  // namespace tml

#include "dslash_x2.cuh"
#include "dslash_mma.cuh"

namespace tml {

// X2: two systems per thread in packed FP32x2 arithmetic (FP16/BF16, NR = 2);
// MMA: the tensor-core kernel (FP16/BF16 with 18-real links, NR and bx unused)
template <class S, int RECON, bool DAG, int EPI, int NR, bool X2 = false, bool MMA = false>
tm_status_t launch_one(const tm_op* op, const DslashCall& c, cudaStream_t st, int bx = 128) {
  DslashArgs a;
  a.g = op->g;
  a.links = op->links[Prec<S>::id];
  a.c = c;
  if (c.custom) {
    a.nu = c.nu;
    a.hop_scale = c.hop_scale;
  } else {
    a.nu = c.mu_zero ? 0.0 : (DAG ? -2.0 * op->kappa * op->mu : 2.0 * op->kappa * op->mu);
    a.hop_scale = -op->kappa;
    a.c.centre = 2;
    a.c.cfield = nullptr;
    a.c.out_inv = false;
  }
  a.inv = 1.0 / (1.0 + a.nu * a.nu);
  a.nu_f = (float)a.nu;
  a.hop_scale_f = (float)a.hop_scale;
  a.inv_f = (float)a.inv;
  a.nwarp = nwarp_of(op->g);
  a.rhs_groups = (c.nrhs + NR - 1) / NR;
  const int per_par = (op->g.Vh + bx - 1) / bx;
  const int site_blocks = c.parity < 0 ? 2 * per_par : per_par;
  dim3 grid((unsigned)(site_blocks * a.rhs_groups));
  if constexpr (MMA) {
    const int tiles = (op->g.Vh + kMmaSites - 1) / kMmaSites;
    grid = dim3((unsigned)(c.parity < 0 ? 2 * tiles : tiles), (unsigned)((c.nrhs + kMmaRows - 1) / kMmaRows));
    if ((int)grid.y > 65535) {
      set_error("dslash: %d systems exceed the launch grid", c.nrhs);
      return TM_ERR_ARG;
    }
  }
  // trace class: dslash.<precision>.<epilogue>
  static const char* const kNames[5][3] = {
      {"dslash.f64.out", "dslash.f64.cgupd", "dslash.f64.resid"},
      {"dslash.f32.out", "dslash.f32.cgupd", "dslash.f32.resid"},
      {"dslash.f16.out", "dslash.f16.cgupd", "dslash.f16.resid"},
      {"dslash.bf16.out", "dslash.bf16.cgupd", "dslash.bf16.resid"},
      {"dslash.ff.out", "dslash.ff.cgupd", "dslash.ff.resid"}};
  const char* name = kNames[Prec<S>::id][EPI];
  // algorithmic bytes: every array once; per active system the neighbour field
  // (one parity's worth per output parity), the centre field, the epilogue's
  // streams; per launch the links of all sites
  const double e = (double)sizeof(S);
  const double out_sites = (c.parity < 0 ? 2.0 : 1.0) * op->g.Vh;
  // the centre field counts unless it is the input array read on both parities
  // (a full-lattice M: the centre reads are the neighbour reads of the other
  // output parity, the same bytes)
  const bool centre_is_in = a.c.cfield == nullptr || a.c.cfield == a.c.in;
  const int centre = (a.c.centre != 0 && !(c.parity < 0 && centre_is_in)) ? 1 : 0;
  const int epi_streams = EPI == EPI_OUT ? 1 : (EPI == EPI_CGUPD ? 5 : 2);
  const double per_rhs = out_sites * 24.0 * e * (1 + centre + epi_streams);
  const int link_reals = RECON;
  const double fixed = 4.0 * 2.0 * op->g.Vh * link_reals * e;
  cudaEvent_t ev = nullptr;
  a.trace_count = trace_begin(st, &ev);
  if constexpr (MMA) dslash_kernel_mma<S, DAG, EPI><<<grid, kMmaThreads, kMmaSmem, st>>>(a);
  else if constexpr (X2) dslash_kernel_x2<S, RECON, DAG, EPI><<<grid, bx, 0, st>>>(a);
  else dslash_kernel<S, RECON, DAG, EPI, NR><<<grid, bx, 0, st>>>(a);
  count_launch();
  // algorithmic flops per output site and system: the spin-projected hops
  // (8 x (12 projection + 132 link product + 24 accumulation) + 24 boundary
  // sign, counted as 1320 as usual), the hop scale and centre (48), the twist
  // A (48), A^-1 (72), the epilogue (CG update 144, residual 72, norm 48)
  const double site_flops = 1320.0 + 48.0 + (a.c.centre == 2 ? 48.0 : 0.0) + (a.c.out_inv ? 72.0 : 0.0) +
                            (EPI == EPI_CGUPD ? 144.0 : EPI == EPI_RESID ? 72.0 : (a.c.partial ? 48.0 : 0.0));
  trace_end(st, name, ev, a.trace_count, per_rhs, fixed, 0, out_sites * site_flops);
  return check_launch("dslash");
}

// ------------------------------------------------------------- autotuning
// Launch shape of the narrow-format Dslash: systems per thread (NR = 1, 2, 4:
// the site's index arithmetic, link loads and reconstruction shared by NR
// systems, against registers and occupancy; for FP16/BF16 also 2 systems in
// packed FP32x2 arithmetic, dslash_kernel_x2) and threads per block (32, 64,
// 128: small lattices fill more SMs with smaller blocks).  Results do not
// depend on either (explicit round-to-nearest arithmetic per system, partial
// sums per warp of 32 sites), so the first launch of each kind times every
// shape on its own arguments and keeps the fastest for the process.  Only
// launches that can be repeated without changing their result are timed
// (EPI_OUT, EPI_RESID: out is a function of inputs it does not overwrite);
// the CG-update launch takes the shape chosen for the plain launch of the same
// operator form.  No tuning while a CUDA graph is being captured, nor while
// TM_DSLASH_NR fixes NR.

// the packed kernel mirrors the 12-real-link 16-bit path (kRawLinks is the other)
template <class S, int RECON>
constexpr bool kPackable = (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) && RECON == 12;

template <class S, int RECON, bool DAG, int EPI>
tm_status_t launch_cfg(const tm_op* op, const DslashCall& c, cudaStream_t st, const TuneCfg& cfg) {
  if constexpr (kPackable<S, RECON>) {
    if (cfg.packed && c.nrhs >= 2) return launch_one<S, RECON, DAG, EPI, 2, true>(op, c, st, cfg.bx);
  }
  if (cfg.nr >= 4 && c.nrhs >= 4) return launch_one<S, RECON, DAG, EPI, 4>(op, c, st, cfg.bx);
  if (cfg.nr >= 2 && c.nrhs >= 2) return launch_one<S, RECON, DAG, EPI, 2>(op, c, st, cfg.bx);
  return launch_one<S, RECON, DAG, EPI, 1>(op, c, st, cfg.bx);
}

// time one launch shape: one warm-up launch, then the mean of three
template <class S, int RECON, bool DAG, int EPI>
float time_cfg(const tm_op* op, const DslashCall& c, cudaStream_t st, const TuneCfg& cfg) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.0f;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.0f; }
  float ms = -1.0f;
  if (launch_cfg<S, RECON, DAG, EPI>(op, c, st, cfg) == TM_OK && cudaEventRecord(e0, st) == cudaSuccess) {
    bool ok = true;
    for (int i = 0; i < 3 && ok; ++i) ok = launch_cfg<S, RECON, DAG, EPI>(op, c, st, cfg) == TM_OK;
    if (ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
      ms /= 3.0f;
    else
      ms = -1.0f;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

template <class S, int RECON, bool DAG, int EPI>
tm_status_t launch_nr(const tm_op* op, const DslashCall& c, cudaStream_t st) {
  if constexpr (std::is_same<S, double>::value || std::is_same<S, FFloat>::value) {
    // FP64 and float-float: arithmetic-bound and register-heavy, one system per thread
    return launch_one<S, RECON, DAG, EPI, 1>(op, c, st);
  } else {
    if constexpr (kRawLinks<S, RECON>) {
      if (dslash_mma_on()) return launch_one<S, RECON, DAG, EPI, 1, false, true>(op, c, st);
    }
    TuneCfg cfg{1, 128, 0};  // measured at 32^3 x 64 with 16 systems: NR = 1, 128 threads
    const int want = dslash_nr_override();
    if (want != 0) {
      cfg.nr = want > 0 ? want : 2;
      cfg.packed = want < 0 ? 1 : 0;
      return launch_cfg<S, RECON, DAG, EPI>(op, c, st, cfg);
    }
    const TuneKey key{(int)Prec<S>::id, RECON, DAG ? 1 : 0, EPI == EPI_CGUPD ? (int)EPI_OUT : EPI,
                      c.parity, c.centre, c.out_inv ? 1 : 0, op->g.Vh, c.nrhs};
    if (tune_lookup(key, &cfg) || EPI == EPI_CGUPD || !tune_active())
      return launch_cfg<S, RECON, DAG, EPI>(op, c, st, cfg);
    float best = -1.0f;
    TuneCfg pick = cfg;
    tuning_begin();
    // shapes: 1, 2 or 4 systems per thread, or 2 in packed FP32x2 (16-bit only)
    for (int v = 0; v < 4; ++v) {
      const int nr = v == 3 ? 2 : (1 << v);
      const int pk = v == 3 ? 1 : 0;
      if (nr > c.nrhs || (pk && !kPackable<S, RECON>)) continue;
      for (int bx : {128, 64, 32}) {
        const TuneCfg tc{nr, bx, pk};
        const float t = time_cfg<S, RECON, DAG, EPI>(op, c, st, tc);
        if (t > 0.0f && (best < 0.0f || t < best)) {
          best = t;
          pick = tc;
        }
      }
    }
    tuning_end();
    tune_store(key, pick);
    return launch_cfg<S, RECON, DAG, EPI>(op, c, st, pick);
  }
}

template <class S, int RECON>
tm_status_t dslash_launch(const tm_op* op, const DslashCall& c, cudaStream_t st) {
  if (c.dagger) {
    switch (c.epi) {
      case EPI_OUT: return launch_nr<S, RECON, true, EPI_OUT>(op, c, st);
      case EPI_CGUPD: return launch_nr<S, RECON, true, EPI_CGUPD>(op, c, st);
      default: return launch_nr<S, RECON, true, EPI_RESID>(op, c, st);
    }
  }
  switch (c.epi) {
    case EPI_OUT: return launch_nr<S, RECON, false, EPI_OUT>(op, c, st);
    case EPI_CGUPD: return launch_nr<S, RECON, false, EPI_CGUPD>(op, c, st);
    default: return launch_nr<S, RECON, false, EPI_RESID>(op, c, st);
  }
}

#define TM_INSTANTIATE_DSLASH(S)                                                           \
  template tm_status_t dslash_launch<S, 18>(const tm_op*, const DslashCall&, cudaStream_t); \
  template tm_status_t dslash_launch<S, 12>(const tm_op*, const DslashCall&, cudaStream_t);

#define TM_INSTANTIATE_DSLASH_MMA(S) template tm_status_t dslash_mma_prepare<S>();

}  // namespace tml
