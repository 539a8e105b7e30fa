// The Dslash for two systems per thread in packed FP32x2 arithmetic.
//
// sm_100+ issues one FFMA2 / FADD2 / FMUL2 for two FP32 lanes, so two
// systems at the same site share every arithmetic issue slot of the link
// products, accumulations and epilogue, besides the site indexing and the
// link loads and conversions.  Lane l of every packed value belongs to system
// 2 g + l.  Each lane performs exactly the operations, in exactly the order,
// of the one-system kernel (dslash_kernel with NR = 1), each rounded to
// nearest, so every system's result is bit-identical to it: the autotuner may
// pick either.  Loads, the FP16 conversions and the mixed-precision spin
// projection stay per system.
// Included by dslash.cuh after the one-system kernel.
#pragma once

namespace tml {

struct Cx2 {
  float2 re, im;
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// a + i^K b, lane by lane (add_ph)
template <int K>
__device__ __forceinline__ Cx2 add_ph2(Cx2 a, Cx2 b) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return {add2(a.re, b.re), add2(a.im, b.im)};
  else if constexpr (k == 1) return {sub2(a.re, b.im), add2(a.im, b.re)};
  else if constexpr (k == 2) return {sub2(a.re, b.re), sub2(a.im, b.im)};
  else return {add2(a.re, b.im), sub2(a.im, b.re)};
}

__device__ __forceinline__ Cx2 pack2(Cx<float> a, Cx<float> b) { return {f2(a.re, b.re), f2(a.im, b.im)}; }

// acc += bsign (1 + SGN g_MU) W psi for the two systems (hop_acc, lane-wise)
template <int MU, int SGN, bool ADJ>
__device__ __forceinline__ void hop_acc2(Cx2 (&acc)[12], const Cx2 (&h0)[3], const Cx2 (&h1)[3],
                                         const Mat3<float>& U, float2 bsign) {
  using G = GBlock<MU>;
  constexpr int s2 = SGN > 0 ? 0 : 2;
  Cx2 w0[3], w1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 r0, i0, r1, i1;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cx<float> u = ADJ ? conjx(U.m[b][a]) : U.m[a][b];
      const float2 ur = bc(u.re), ui = bc(u.im), nui = bc(-u.im);
      if (b == 0) {
        r0 = mul2(ur, h0[b].re); i0 = mul2(ur, h0[b].im);
        r1 = mul2(ur, h1[b].re); i1 = mul2(ur, h1[b].im);
      } else {
        r0 = fma2(ur, h0[b].re, r0); i0 = fma2(ur, h0[b].im, i0);
        r1 = fma2(ur, h1[b].re, r1); i1 = fma2(ur, h1[b].im, i1);
      }
      r0 = fma2(nui, h0[b].im, r0); i0 = fma2(ui, h0[b].re, i0);
      r1 = fma2(nui, h1[b].im, r1); i1 = fma2(ui, h1[b].re, i1);
    }
    if (MU == 3) {
      r0 = mul2(bsign, r0); i0 = mul2(bsign, i0);
      r1 = mul2(bsign, r1); i1 = mul2(bsign, i1);
    }
    w0[a] = {r0, i0};
    w1[a] = {r1, i1};
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c] = add_ph2<0>(acc[c], w0[c]);
    acc[3 + c] = add_ph2<0>(acc[3 + c], w1[c]);
    const Cx2 wb0 = G::bc0 == 0 ? w0[c] : w1[c];
    const Cx2 wb1 = G::bc1 == 0 ? w0[c] : w1[c];
    acc[6 + c] = add_ph2<G::bk0 + s2>(acc[6 + c], wb0);
    acc[9 + c] = add_ph2<G::bk1 + s2>(acc[9 + c], wb1);
  }
}

// the projected 2-spinor of one system's site (zero for an inactive system)
template <class S, int MU, int SGN>
__device__ __forceinline__ void project_site(Cx<float> (&h0)[3], Cx<float> (&h1)[3], const void* field,
                                             size_t b0, size_t cs, bool on) {
  if (!on) {
#pragma unroll
    for (int c = 0; c < 3; ++c) h0[c] = h1[c] = {0.0f, 0.0f};
    return;
  }
  const uint4* f = reinterpret_cast<const uint4*>(field);
  uint4 q[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) q[j] = f[b0 + j * cs];
  project_raw<MU, SGN, S>(h0, h1, q);
}

template <class S>
__device__ __forceinline__ void load_pair(Cx2 (&v)[12], const void* field, size_t b0, size_t b1, size_t cs,
                                          bool on0, bool on1) {
  Cx<float> a[12], b[12];
  if (on0) load_spinor<S>(a, field, b0, cs);
  else
#pragma unroll
    for (int k = 0; k < 12; ++k) a[k] = {0.0f, 0.0f};
  if (on1) load_spinor<S>(b, field, b1, cs);
  else
#pragma unroll
    for (int k = 0; k < 12; ++k) b[k] = {0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = pack2(a[k], b[k]);
}

template <class S>
__device__ __forceinline__ void store_pair(void* field, size_t b0, size_t b1, size_t cs, const Cx2 (&v)[12],
                                           bool on0, bool on1) {
  Cx<float> a[12], b[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    a[k] = {v[k].re.x, v[k].im.x};
    b[k] = {v[k].re.y, v[k].im.y};
  }
  if (on0) store_spinor<S>(field, b0, cs, a);
  if (on1) store_spinor<S>(field, b1, cs, b);
}

__device__ __forceinline__ float2 norm2_12x2(const Cx2 (&v)[12]) {
  float2 s = f2(0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    s = fma2(v[j].re, v[j].re, s);
    s = fma2(v[j].im, v[j].im, s);
  }
  return s;
}

template <class S>
constexpr int dslash_x2_min_blocks() { return 4; }

// FP16 / BF16 storage only: it mirrors their one-hop-at-a-time kernel
template <class S, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128, dslash_x2_min_blocks<S>()) dslash_kernel_x2(const DslashArgs a) {
  static_assert(std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value, "16-bit storage only");
  const Geom& g = a.g;
  const int rg = blockIdx.x % a.rhs_groups;
  const int sb = blockIdx.x / a.rhs_groups;
  const int par = a.c.parity < 0 ? (sb & 1) : a.c.parity;
  const int cbb = a.c.parity < 0 ? (sb >> 1) : sb;
  const int cb = cbb * blockDim.x + threadIdx.x;
  const int nrhs = a.c.nrhs;
  const int r0 = 2 * rg, r1 = 2 * rg + 1;
  const bool act0 = r0 < nrhs && (a.c.active == nullptr || a.c.active[r0] != 0);
  const bool act1 = r1 < nrhs && (a.c.active == nullptr || a.c.active[r1] != 0);
  const int rr1 = r1 < nrhs ? r1 : r0;  // padding system: never loaded nor stored
  double part0 = 0.0, part1 = 0.0;
  if (a.trace_count && blockIdx.x == 0 && threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < nrhs; ++r) n += (a.c.active == nullptr || a.c.active[r] != 0) ? 1 : 0;
    *a.trace_count = n;
  }
  if ((act0 || act1) && cb < g.Vh) {
    const Site s = site_of(g, par, cb);
    const int opar = par ^ 1;
    const size_t cs = (size_t)g.Vh;
    constexpr int NCH = spinor_chunks<S>();
    Cx2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {f2(0.0f, 0.0f), f2(0.0f, 0.0f)};
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const size_t base0 = ((size_t)(r0 * 2 + opar) * NCH) * cs, base1 = ((size_t)(rr1 * 2 + opar) * NCH) * cs;
#define TM_HOPS2(MU)                                                                             \
    {                                                                                            \
      const int lf = lex_fwd(g, s, MU);                                                          \
      const int lb = lex_bwd(g, s, MU);                                                          \
      float sf = 1, sbk = 1;                                                                     \
      if (MU == 3 && g.antiperiodic) {                                                           \
        if (s.c[3] == g.L[3] - 1) sf = -1;                                                       \
        if (s.c[3] == 0) sbk = -1;                                                               \
      }                                                                                          \
      {                                                                                          \
        const Mat3<float> Uf = load_link<S, RECON>(a.links, g, MU, par, cb);                     \
        Cx<float> h0a[3], h1a[3], h0b[3], h1b[3];                                                \
        project_site<S, MU, SF>(h0a, h1a, a.c.in, base0 + (lf >> 1), cs, act0);                   \
        project_site<S, MU, SF>(h0b, h1b, a.c.in, base1 + (lf >> 1), cs, act1);                   \
        Cx2 h0[3], h1[3];                                                                        \
        _Pragma("unroll") for (int c = 0; c < 3; ++c) {                                          \
          h0[c] = pack2(h0a[c], h0b[c]);                                                         \
          h1[c] = pack2(h1a[c], h1b[c]);                                                         \
        }                                                                                        \
        hop_acc2<MU, SF, false>(acc, h0, h1, Uf, bc(sf));                                        \
      }                                                                                          \
      {                                                                                          \
        const Mat3<float> Ub = load_link<S, RECON>(a.links, g, MU, opar, lb >> 1);               \
        Cx<float> h0a[3], h1a[3], h0b[3], h1b[3];                                                \
        project_site<S, MU, SB>(h0a, h1a, a.c.in, base0 + (lb >> 1), cs, act0);                   \
        project_site<S, MU, SB>(h0b, h1b, a.c.in, base1 + (lb >> 1), cs, act1);                   \
        Cx2 h0[3], h1[3];                                                                        \
        _Pragma("unroll") for (int c = 0; c < 3; ++c) {                                          \
          h0[c] = pack2(h0a[c], h0b[c]);                                                         \
          h1[c] = pack2(h1a[c], h1b[c]);                                                         \
        }                                                                                        \
        hop_acc2<MU, SB, true>(acc, h0, h1, Ub, bc(sbk));                                        \
      }                                                                                          \
    }
    TM_HOPS2(0)
    TM_HOPS2(1)
    TM_HOPS2(2)
    TM_HOPS2(3)
#undef TM_HOPS2
    const float2 shop = bc(a.hop_scale_f), nu = bc(a.nu_f), inv = bc(a.inv_f), nnu = bc(-a.nu_f);
    const void* cfield = a.c.cfield ? a.c.cfield : a.c.in;
    const size_t o0 = ((size_t)(r0 * 2 + par) * NCH) * cs + cb, o1 = ((size_t)(rr1 * 2 + par) * NCH) * cs + cb;
    Cx2 out[12];
    if (a.c.centre != 0) {
      load_pair<S>(out, cfield, o0, o1, cs, act0, act1);
      if (a.c.centre == 2) {  // A c = c + i nu g5 c
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float2 tw = k < 6 ? nu : nnu, ntw = k < 6 ? nnu : nu;
          const Cx2 c = out[k];
          out[k] = {fma2(ntw, c.im, c.re), fma2(tw, c.re, c.im)};
        }
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) out[k] = {fma2(shop, acc[k].re, out[k].re), fma2(shop, acc[k].im, out[k].im)};
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) out[k] = {mul2(shop, acc[k].re), mul2(shop, acc[k].im)};
    }
    if (a.c.out_inv) {  // A^-1 v = (v - i nu g5 v) / (1 + nu^2)
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float2 tw = k < 6 ? nu : nnu, ntw = k < 6 ? nnu : nu;
        const Cx2 v = out[k];
        out[k] = {mul2(inv, fma2(tw, v.im, v.re)), mul2(inv, fma2(ntw, v.re, v.im))};
      }
    }
    if constexpr (EPI == EPI_OUT) {
      if (a.c.g5_out) {
#pragma unroll
        for (int k = 6; k < 12; ++k) out[k] = {neg2(out[k].re), neg2(out[k].im)};
      }
      store_pair<S>(a.c.out, o0, o1, cs, out, act0, act1);
      if (a.c.partial) {
        const float2 n2 = norm2_12x2(out);
        part0 = (double)n2.x;
        part1 = (double)n2.y;
      }
    } else if constexpr (EPI == EPI_CGUPD) {
      const float al0 = act0 ? (float)a.c.alpha[r0] : 0.0f, al1 = act1 ? (float)a.c.alpha[rr1] : 0.0f;
      const float2 al = f2(al0, al1), nal = f2(-al0, -al1);
      Cx2 v[12];
      load_pair<S>(v, a.c.r, o0, o1, cs, act0, act1);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = {fma2(nal, out[k].re, v[k].re), fma2(nal, out[k].im, v[k].im)};
      store_pair<S>(a.c.r, o0, o1, cs, v, act0, act1);
      const float2 n2 = norm2_12x2(v);
      part0 = (double)n2.x;
      part1 = (double)n2.y;
      Cx2 w[12];
      load_pair<S>(v, a.c.x, o0, o1, cs, act0, act1);
      load_pair<S>(w, a.c.p, o0, o1, cs, act0, act1);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = {fma2(al, w[k].re, v[k].re), fma2(al, w[k].im, v[k].im)};
      store_pair<S>(a.c.x, o0, o1, cs, v, act0, act1);
    } else {  // EPI_RESID
      Cx2 v[12];
      load_pair<S>(v, a.c.b, o0, o1, cs, act0, act1);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = {sub2(v[k].re, out[k].re), sub2(v[k].im, out[k].im)};
      store_pair<S>(a.c.out, o0, o1, cs, v, act0, act1);
      const float2 n2 = norm2_12x2(v);
      part0 = (double)n2.x;
      part1 = (double)n2.y;
    }
  }
  if (EPI != EPI_OUT || a.c.partial != nullptr) {
    const double ps0 = warp_sum(part0), ps1 = warp_sum(part1);
    if (threadIdx.x % 32 == 0 && cb < a.nwarp * 32) {
      if (r0 < nrhs) a.c.partial[((size_t)r0 * 2 + par) * a.nwarp + cb / 32] = ps0;
      if (r1 < nrhs) a.c.partial[((size_t)r1 * 2 + par) * a.nwarp + cb / 32] = ps1;
    }
  }
}

}  // namespace tml
