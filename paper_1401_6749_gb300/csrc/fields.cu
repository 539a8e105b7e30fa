// Field utilities: layout packing, precision conversion, gamma_5, Z4 noise,
// gauge-link packing, the BLAS-1 updates of the solver and the fixed-order
// reduction of per-warp partial sums.
#include <cstdio>

#include "tm_host.h"

namespace tml {

// ------------------------------------------------ exact double <-> storage
// Stores from double values round once (round to nearest even) directly to
// the storage format.
template <class S>
__device__ __forceinline__ void store_spinor_f64(void* field, size_t b0, size_t cs,
                                                 const Cx<double> (&v)[12]) {
  if constexpr (std::is_same<S, double>::value) {
    store_spinor<double>(field, b0, cs, v);
  } else if constexpr (std::is_same<S, FFloat>::value) {
    Cx<FF> w[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) w[j] = {FF(v[j].re), FF(v[j].im)};
    store_spinor<FFloat>(field, b0, cs, w);
  } else if constexpr (std::is_same<S, float>::value) {
    Cx<float> w[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) w[j] = {(float)v[j].re, (float)v[j].im};
    store_spinor<float>(field, b0, cs, w);
  } else {
    uint4* f = reinterpret_cast<uint4*>(field);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint4 d;
      S* h = reinterpret_cast<S*>(&d);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if constexpr (std::is_same<S, __half>::value) {
          h[2 * k] = __double2half(v[4 * j + k].re);
          h[2 * k + 1] = __double2half(v[4 * j + k].im);
        } else {
          h[2 * k] = __double2bfloat16(v[4 * j + k].re);
          h[2 * k + 1] = __double2bfloat16(v[4 * j + k].im);
        }
      }
      f[b0 + j * cs] = d;
    }
  }
}

template <class S>
__device__ __forceinline__ void load_spinor_f64(Cx<double> (&v)[12], const void* field, size_t b0,
                                                size_t cs) {
  Cx<typename Prec<S>::R> w[12];
  load_spinor<S>(w, field, b0, cs);
#pragma unroll
  for (int j = 0; j < 12; ++j) v[j] = {(double)w[j].re, (double)w[j].im};
}

template <class F>
tm_status_t by_prec(tm_prec_t p, F&& f) {
  switch (p) {
    case TM_PREC_F64: return f(double{});
    case TM_PREC_F32: return f(float{});
    case TM_PREC_F16: return f(__half{});
    case TM_PREC_BF16: return f(__nv_bfloat16{});
    case TM_PREC_FF: return f(FFloat{});
    default: set_error("unknown precision %d", (int)p); return TM_ERR_ARG;
  }
}

static unsigned blocks_for(long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ------------------------------------------------------------- pack/unpack
template <class S>
__global__ void pack_kernel(Geom g, void* out, const double* in, int nrhs) {
  const long V = 2L * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * nrhs) return;
  const int rhs = (int)(i / V);
  const int lex = (int)(i % V);
  const int x = lex % g.L[0], y = (lex / g.stride[1]) % g.L[1];
  const int z = (lex / g.stride[2]) % g.L[2], t = lex / g.stride[3];
  const int par = (x + y + z + t) & 1;
  Cx<double> v[12];
  const double2* src = reinterpret_cast<const double2*>(in) + ((size_t)rhs * V + lex) * 12;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const double2 d = src[j];
    v[j] = {d.x, d.y};
  }
  store_spinor_f64<S>(out, SpinorRef<S>::base(g, rhs, par, lex >> 1), (size_t)g.Vh, v);
}

template <class S>
__global__ void unpack_kernel(Geom g, double* out, const void* in, int nrhs) {
  const long V = 2L * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * nrhs) return;
  const int rhs = (int)(i / V);
  const int lex = (int)(i % V);
  const int x = lex % g.L[0], y = (lex / g.stride[1]) % g.L[1];
  const int z = (lex / g.stride[2]) % g.L[2], t = lex / g.stride[3];
  const int par = (x + y + z + t) & 1;
  Cx<double> v[12];
  load_spinor_f64<S>(v, in, SpinorRef<S>::base(g, rhs, par, lex >> 1), (size_t)g.Vh);
  double2* dst = reinterpret_cast<double2*>(out) + ((size_t)rhs * V + lex) * 12;
#pragma unroll
  for (int j = 0; j < 12; ++j) dst[j] = make_double2(v[j].re, v[j].im);
}

template <class SO, class SI>
__global__ void convert_kernel(Geom g, void* out, const void* in, int nrhs, const int* active) {
  const long n = 2L * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int rhs = (int)(i / n);
  if (active && !active[rhs]) return;
  const int rem = (int)(i % n);
  const int par = rem / g.Vh, cb = rem % g.Vh;
  Cx<double> v[12];
  load_spinor_f64<SI>(v, in, SpinorRef<SI>::base(g, rhs, par, cb), (size_t)g.Vh);
  store_spinor_f64<SO>(out, SpinorRef<SO>::base(g, rhs, par, cb), (size_t)g.Vh, v);
}

template <class S>
__global__ void gamma5_kernel(Geom g, void* out, const void* in, int nrhs) {
  const long n = 2L * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int rhs = (int)(i / n);
  const int rem = (int)(i % n);
  const int par = rem / g.Vh, cb = rem % g.Vh;
  Cx<typename Prec<S>::R> v[12];
  const size_t b0 = SpinorRef<S>::base(g, rhs, par, cb);
  load_spinor<S>(v, in, b0, (size_t)g.Vh);
#pragma unroll
  for (int j = 6; j < 12; ++j) v[j] = {-v[j].re, -v[j].im};
  store_spinor<S>(out, b0, (size_t)g.Vh, v);
}

// ------------------------------------------------------------ Z4 noise
// Philox4x32 with 10 rounds (Salmon et al., SC'11): per round
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// keys advanced by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// dt > 0: time dilution, noise only on slices t = t0 (mod dt), zero elsewhere.
// One thread per (site, source): blockIdx.x covers the sites of both parities
// (parity = blockIdx.x & 1), blockIdx.y the source.  The entries i^k are
// built in the storage's own arithmetic (exact in every format), so no FP64
// conversion runs per entry.
template <class S>
__global__ void z4_kernel(Geom g, void* eta, uint2 key, uint32_t first, int t0, int dt) {
  using R = typename Prec<S>::R;
  const int par = blockIdx.x & 1;
  const int cb = (int)(blockIdx.x >> 1) * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  const int j = blockIdx.y;
  const Site st = site_of(g, par, cb);
  const int t = st.c[3];
  const bool on = dt <= 0 || ((t - t0) % dt + dt) % dt == 0;
  const uint4 w = on ? philox4x32_10(make_uint4((uint32_t)st.lex, first + (uint32_t)j, 0u, 0u), key)
                     : make_uint4(0u, 0u, 0u, 0u);
  const R one = (R)1, zero = (R)0;
  Cx<R> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int q = (int)((w.x >> (2 * k)) & 3u);  // component k = 3*alpha + colour
    v[k] = !on ? Cx<R>{zero, zero}
         : q == 0 ? Cx<R>{one, zero} : q == 1 ? Cx<R>{zero, one} : q == 2 ? Cx<R>{-one, zero}
                                                                       : Cx<R>{zero, -one};
  }
  store_spinor<S>(eta, SpinorRef<S>::base(g, j, par, cb), (size_t)g.Vh, v);
}

// The same noise written straight into the system-interleaved 16-bit layout
// ([block][parity][cb][k][slot], systems j and j + 8 on pair position j of
// rows k = 0, 1 (mod 3) and j ^ 4 of rows k = 2 (mod 3)).  One thread per
// (site, system of the block): a warp covers two sites, and each of its 12
// stores fills two 64-byte rows.  Systems >= nsrc are written as zero.  The
// entries are bit patterns of the format's +-1 (one = 0x3C00 FP16, 0x3F80
// BF16; sign bit 0x8000), re in the low half-word.
__global__ void __launch_bounds__(256) z4_il_kernel(Geom g, unsigned* __restrict__ eta, uint2 key,
                                                    uint32_t first, int nsrc, unsigned one) {
  const int par = blockIdx.y, blk = blockIdx.z;
  const int j = threadIdx.x & 15;
  const int cb = blockIdx.x * 16 + (threadIdx.x >> 4);
  if (cb >= g.Vh) return;
  const int r = blk * 16 + j;
  const Site st = site_of(g, par, cb);
  const uint32_t w = r < nsrc ? philox4x32_10(make_uint4((uint32_t)st.lex, first + (uint32_t)r, 0u, 0u), key).x
                              : 0u;
  const unsigned neg = one | 0x8000u;
  unsigned* o = eta + (((size_t)blk * 2 + par) * (size_t)g.Vh + (size_t)cb) * 192;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const unsigned q = (w >> (2 * k)) & 3u;
    const unsigned v = r >= nsrc ? 0u : q == 0 ? one : q == 1 ? one << 16 : q == 2 ? neg : neg << 16;
    const int slot = 2 * ((j & 7) ^ (k % 3 == 2 ? 4 : 0)) + (j >> 3);
    o[16 * k + slot] = v;
  }
}

// ------------------------------------------------------------ gauge packing
template <class S>
__device__ __forceinline__ S from_f64(double v) {
  if constexpr (std::is_same<S, double>::value) return v;
  else if constexpr (std::is_same<S, FFloat>::value) {
    const FF f(v);
    return FFloat{f.hi, f.lo};
  }
  else if constexpr (std::is_same<S, float>::value) return (float)v;
  else if constexpr (std::is_same<S, __half>::value) return __double2half(v);
  else return __double2bfloat16(v);
}

// canonical FP64 links -> internal format (LinkFmt), padding slots zeroed
template <class S, int RECON>
__global__ void pack_links_kernel(Geom g, void* out, const double* U) {
  using F = LinkFmt<S, RECON>;
  const long V = 2L * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * V) return;
  const int mu = (int)(i / V);
  const int lex = (int)(i % V);
  const int x = lex % g.L[0], y = (lex / g.stride[1]) % g.L[1];
  const int z = (lex / g.stride[2]) % g.L[2], t = lex / g.stride[3];
  const int par = (x + y + z + t) & 1;
  const int cb = lex >> 1;
  const double2* src = reinterpret_cast<const double2*>(U) + ((size_t)mu * V + lex) * 9;
  const size_t b0 = ((size_t)(mu * 2 + par) * F::NU) * (size_t)g.Vh + (size_t)cb;
  const size_t cs = (size_t)g.Vh;
  S* base = reinterpret_cast<S*>(out);
  constexpr int per_unit = 2 * F::kCplxPerUnit;  // S elements per unit
  for (int u = 0; u < F::NU; ++u) {
    S* q = base + (b0 + u * cs) * per_unit;
    for (int k = 0; k < F::kCplxPerUnit; ++k) {
      const int e = u * F::kCplxPerUnit + k;
      const double2 v = e < F::kCplx ? src[e] : make_double2(0.0, 0.0);
      q[2 * k] = from_f64<S>(v.x);
      q[2 * k + 1] = from_f64<S>(v.y);
    }
  }
}

template <class S, int RECON>
static size_t link_bytes_t(const Geom& g) {
  using F = LinkFmt<S, RECON>;
  return 4 * 2 * (size_t)g.Vh * F::NU * F::kUnitBytes;
}

size_t link_bytes(const Geom& g, tm_prec_t p, int recon) {
  const bool r12 = recon == 12;
  switch (p) {
    case TM_PREC_F64: return link_bytes_t<double, 18>(g);
    case TM_PREC_FF: return link_bytes_t<FFloat, 18>(g);
    case TM_PREC_F32: return r12 ? link_bytes_t<float, 12>(g) : link_bytes_t<float, 18>(g);
    case TM_PREC_F16: return r12 ? link_bytes_t<__half, 12>(g) : link_bytes_t<__half, 18>(g);
    default: return r12 ? link_bytes_t<__nv_bfloat16, 12>(g) : link_bytes_t<__nv_bfloat16, 18>(g);
  }
}

tm_status_t pack_links(const Geom& g, tm_prec_t p, int recon, void* out, const double* U,
                       cudaStream_t s) {
  const long n = 4L * 2 * g.Vh;
  const unsigned nb = blocks_for(n, 256);
  const bool r12 = recon == 12;
  if (p == TM_PREC_F64) pack_links_kernel<double, 18><<<nb, 256, 0, s>>>(g, out, U);
  else if (p == TM_PREC_FF) pack_links_kernel<FFloat, 18><<<nb, 256, 0, s>>>(g, out, U);
  else if (p == TM_PREC_F32 && r12) pack_links_kernel<float, 12><<<nb, 256, 0, s>>>(g, out, U);
  else if (p == TM_PREC_F32) pack_links_kernel<float, 18><<<nb, 256, 0, s>>>(g, out, U);
  else if (p == TM_PREC_F16 && r12) pack_links_kernel<__half, 12><<<nb, 256, 0, s>>>(g, out, U);
  else if (p == TM_PREC_F16) pack_links_kernel<__half, 18><<<nb, 256, 0, s>>>(g, out, U);
  else if (r12) pack_links_kernel<__nv_bfloat16, 12><<<nb, 256, 0, s>>>(g, out, U);
  else pack_links_kernel<__nv_bfloat16, 18><<<nb, 256, 0, s>>>(g, out, U);
  count_launch();
  return check_launch("pack_links");
}

// ------------------------------------------------------------ solver BLAS
// p = r + beta[rhs] p for active systems
template <class S>
__global__ void xpay_kernel(Geom g, void* p, const void* r, const double* beta, const int* active,
                            int nrhs, int par0, int npar) {
  const long n = (long)npar * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int rhs = (int)(i / n);
  if (!active[rhs]) return;
  const int rem = (int)(i % n);
  const size_t b0 = SpinorRef<S>::base(g, rhs, par0 + rem / g.Vh, rem % g.Vh);
  using R = typename Prec<S>::R;
  const R be = (R)beta[rhs];
  Cx<R> a[12], b[12];
  load_spinor<S>(a, r, b0, (size_t)g.Vh);
  load_spinor<S>(b, p, b0, (size_t)g.Vh);
#pragma unroll
  for (int j = 0; j < 12; ++j) a[j] = a[j] + be * b[j];
  store_spinor<S>(p, b0, (size_t)g.Vh, a);
}

// x64 += sigma[rhs] * y (exact widening), y = 0, for systems with mask[rhs] != 0;
// sigma may be null (scale 1); xff (may be null) receives x64 in float-float
template <class S>
__global__ void fold_kernel(Geom g, void* x64, void* y, const double* sigma, const int* mask,
                            int nrhs, int par0, int npar, void* xff) {
  const long n = (long)npar * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int rhs = (int)(i / n);
  if (mask && !mask[rhs]) return;
  const int rem = (int)(i % n);
  const int par = par0 + rem / g.Vh, cb = rem % g.Vh;
  const double sc = sigma ? sigma[rhs] : 1.0;
  Cx<double> a[12], b[12];
  const size_t bx = SpinorRef<double>::base(g, rhs, par, cb);
  const size_t by = SpinorRef<S>::base(g, rhs, par, cb);
  load_spinor<double>(a, x64, bx, (size_t)g.Vh);
  load_spinor_f64<S>(b, y, by, (size_t)g.Vh);
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    a[j] = a[j] + sc * b[j];
    b[j] = {0.0, 0.0};
  }
  store_spinor<double>(x64, bx, (size_t)g.Vh, a);
  store_spinor_f64<S>(y, by, (size_t)g.Vh, b);
  if (xff) store_spinor_f64<FFloat>(xff, SpinorRef<FFloat>::base(g, rhs, par, cb), (size_t)g.Vh, a);
}

// Reliable-update rescaling of the inner iteration (masked systems):
//   r = r64 / sigma[rhs]   and, if p != null,   p *= ratio[rhs]
// (r64 stored as SR: FP64, or float-float)
template <class S, class SR>
__global__ void rescale_kernel(Geom g, void* r, const void* r64, const double* sigma, void* p,
                               const double* ratio, const int* mask, int nrhs, int par0, int npar) {
  const long n = (long)npar * g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int rhs = (int)(i / n);
  if (mask && !mask[rhs]) return;
  const int rem = (int)(i % n);
  const int par = par0 + rem / g.Vh, cb = rem % g.Vh;
  const size_t b64 = SpinorRef<SR>::base(g, rhs, par, cb);
  const size_t bs = SpinorRef<S>::base(g, rhs, par, cb);
  const double inv = 1.0 / sigma[rhs];
  Cx<double> v[12];
  load_spinor_f64<SR>(v, r64, b64, (size_t)g.Vh);
#pragma unroll
  for (int j = 0; j < 12; ++j) v[j] = inv * v[j];
  store_spinor_f64<S>(r, bs, (size_t)g.Vh, v);
  if (p) {
    const double q = ratio[rhs];
    load_spinor_f64<S>(v, p, bs, (size_t)g.Vh);
#pragma unroll
    for (int j = 0; j < 12; ++j) v[j] = q * v[j];
    store_spinor_f64<S>(p, bs, (size_t)g.Vh, v);
  }
}

tm_status_t xpay(const Geom& g, tm_prec_t prec, void* p, const void* r, const double* beta,
                 const int* active, int nrhs, int par0, int npar, cudaStream_t s) {
  const unsigned nb = blocks_for((long)npar * g.Vh * nrhs, 256);
  TraceScope tr(s, "blas.xpay", 3.0 * 24.0 * prec_size(prec) * npar * g.Vh, 0.0, nrhs);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    xpay_kernel<S><<<nb, 256, 0, s>>>(g, p, r, beta, active, nrhs, par0, npar);
    count_launch();
    return check_launch("xpay");
  });
}

tm_status_t fold(const Geom& g, tm_prec_t prec, void* x64, void* y, const double* sigma,
                 const int* mask, int nrhs, int par0, int npar, cudaStream_t s, void* xff) {
  const unsigned nb = blocks_for((long)npar * g.Vh * nrhs, 256);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    fold_kernel<S><<<nb, 256, 0, s>>>(g, x64, y, sigma, mask, nrhs, par0, npar, xff);
    count_launch();
    return check_launch("fold");
  });
}

tm_status_t rescale(const Geom& g, tm_prec_t prec, void* r, const void* r64, const double* sigma,
                    void* p, const double* ratio, const int* mask, int nrhs, int par0, int npar,
                    cudaStream_t s, bool r_ff) {
  const unsigned nb = blocks_for((long)npar * g.Vh * nrhs, 256);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    if (r_ff)
      rescale_kernel<S, FFloat><<<nb, 256, 0, s>>>(g, r, r64, sigma, p, ratio, mask, nrhs, par0, npar);
    else
      rescale_kernel<S, double><<<nb, 256, 0, s>>>(g, r, r64, sigma, p, ratio, mask, nrhs, par0, npar);
    count_launch();
    return check_launch("rescale");
  });
}

tm_status_t convert_masked(const Geom& g, void* out, tm_prec_t po, const void* in, tm_prec_t pi,
                           int nrhs, const int* active, cudaStream_t s) {
  const unsigned nb = blocks_for(2L * g.Vh * nrhs, 256);
  return by_prec(po, [&](auto to) {
    using SO = decltype(to);
    return by_prec(pi, [&](auto ti) {
      using SI = decltype(ti);
      convert_kernel<SO, SI><<<nb, 256, 0, s>>>(g, out, in, nrhs, active);
      count_launch();
      return check_launch("convert");
    });
  });
}

// Site-local twist on one parity: out = A in (inverse = 0) or A^-1 in
// (inverse = 1), A = 1 + i nu g5, A^-1 = (1 - i nu g5) / (1 + nu^2).
template <class S>
__global__ void twist_kernel(Geom g, void* out, const void* in, double nu, int inverse, int par,
                             int nrhs) {
  using R = typename Prec<S>::R;
  const long n = (long)g.Vh;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nrhs) return;
  const int rhs = (int)(i / n);
  const int cb = (int)(i % n);
  const size_t b0 = SpinorRef<S>::base(g, rhs, par, cb);
  Cx<R> v[12];
  load_spinor<S>(v, in, b0, (size_t)g.Vh);
  const R sc = inverse ? (R)(1.0 / (1.0 + nu * nu)) : (R)1;
  const R tn = inverse ? (R)(-nu) : (R)nu;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const R tw = j < 6 ? tn : -tn;
    const Cx<R> c = v[j];
    v[j] = {sc * (c.re - tw * c.im), sc * (c.im + tw * c.re)};
  }
  store_spinor<S>(out, b0, (size_t)g.Vh, v);
}

tm_status_t twist(const Geom& g, tm_prec_t prec, void* out, const void* in, double nu, int inverse,
                  int par, int nrhs, cudaStream_t s) {
  const unsigned nb = blocks_for((long)g.Vh * nrhs, 256);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    twist_kernel<S><<<nb, 256, 0, s>>>(g, out, in, nu, inverse, par, nrhs);
    count_launch();
    return check_launch("twist");
  });
}

// ------------------------------------------------ fixed-order reductions
// One block per system; thread i sums entries i, i + 256, ... in order, then
// a fixed shared-memory tree.  The result depends only on the partial array.
__global__ void reduce_partials_kernel(const double* partial, int nper, size_t stride,
                                       double* result) {
  __shared__ double sh[256];
  const double* p = partial + (size_t)blockIdx.x * stride;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nper; i += 256) acc += p[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) result[blockIdx.x] = sh[0];
}

tm_status_t reduce_partials(const double* partial, int nper, int nrhs, double* result,
                            cudaStream_t s, size_t stride) {
  reduce_partials_kernel<<<nrhs, 256, 0, s>>>(partial, nper, stride ? stride : (size_t)nper, result);
  count_launch();
  return check_launch("reduce_partials");
}

}  // namespace tml

using namespace tml;

// ------------------------------------------------------------ C ABI
extern "C" size_t tm_spinor_bytes(const tm_geom_t* g, tm_prec_t prec, int nrhs) {
  if (!g || nrhs < 0) return 0;
  const size_t V = (size_t)g->L[0] * g->L[1] * g->L[2] * g->L[3];
  return V * 24 * prec_size(prec) * (size_t)nrhs;
}

extern "C" tm_status_t tm_spinor_pack(const tm_geom_t* gg, void* out, tm_prec_t prec,
                                      const double* in_lex, int nrhs, tm_stream_t s) {
  if (!gg || !out || !in_lex || nrhs < 0) { set_error("tm_spinor_pack: null argument"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  const Geom g = make_geom(gg->L, 1);
  const unsigned nb = blocks_for(2L * g.Vh * nrhs, 256);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    pack_kernel<S><<<nb, 256, 0, (cudaStream_t)s>>>(g, out, in_lex, nrhs);
    count_launch();
    return check_launch("pack");
  });
}

extern "C" tm_status_t tm_spinor_unpack(const tm_geom_t* gg, double* out_lex, const void* in,
                                        tm_prec_t prec, int nrhs, tm_stream_t s) {
  if (!gg || !out_lex || !in || nrhs < 0) { set_error("tm_spinor_unpack: null argument"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  const Geom g = make_geom(gg->L, 1);
  const unsigned nb = blocks_for(2L * g.Vh * nrhs, 256);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    unpack_kernel<S><<<nb, 256, 0, (cudaStream_t)s>>>(g, out_lex, in, nrhs);
    count_launch();
    return check_launch("unpack");
  });
}

extern "C" tm_status_t tm_spinor_convert(const tm_geom_t* gg, void* out, tm_prec_t out_prec,
                                         const void* in, tm_prec_t in_prec, int nrhs, tm_stream_t s) {
  if (!gg || !out || !in || nrhs < 0) { set_error("tm_spinor_convert: null argument"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  return convert_masked(make_geom(gg->L, 1), out, out_prec, in, in_prec, nrhs, nullptr,
                        (cudaStream_t)s);
}

extern "C" tm_status_t tm_gamma5(const tm_geom_t* gg, void* out, const void* in, tm_prec_t prec,
                                 int nrhs, tm_stream_t s) {
  if (!gg || !out || !in || nrhs < 0) { set_error("tm_gamma5: null argument"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  const Geom g = make_geom(gg->L, 1);
  const unsigned nb = blocks_for(2L * g.Vh * nrhs, 256);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    gamma5_kernel<S><<<nb, 256, 0, (cudaStream_t)s>>>(g, out, in, nrhs);
    count_launch();
    return check_launch("gamma5");
  });
}

static tm_status_t z4_launch(const tm_geom_t* gg, void* eta, tm_prec_t prec, uint64_t seed,
                             uint32_t first_src, int nsrc, int t0, int dt, tm_stream_t s);

extern "C" tm_status_t z4_noise(const tm_geom_t* gg, void* eta, tm_prec_t prec, uint64_t seed,
                                uint32_t first_src, int nsrc, tm_stream_t s) {
  return z4_launch(gg, eta, prec, seed, first_src, nsrc, 0, 0, s);
}

extern "C" tm_status_t z4_noise_diluted(const tm_geom_t* gg, void* eta, tm_prec_t prec, uint64_t seed,
                                        uint32_t first_src, int nsrc, int t0, int dt, tm_stream_t s) {
  if (!gg || dt < 1 || t0 < 0 || t0 >= dt) {
    set_error("z4_noise_diluted: need 1 <= dt and 0 <= t0 < dt");
    return TM_ERR_ARG;
  }
  return z4_launch(gg, eta, prec, seed, first_src, nsrc, t0, dt, s);
}

extern "C" tm_status_t z4_noise_il(const tm_geom_t* gg, void* eta_il, tm_prec_t prec, uint64_t seed,
                                   uint32_t first_src, int nsrc, tm_stream_t s) {
  if (!gg || !eta_il || nsrc < 0) { set_error("z4_noise_il: null argument"); return TM_ERR_ARG; }
  if (prec != TM_PREC_F16 && prec != TM_PREC_BF16) {
    set_error("z4_noise_il: the interleaved layout holds F16 or BF16 fields");
    return TM_ERR_ARG;
  }
  if (reinterpret_cast<uintptr_t>(eta_il) & 3u) { set_error("z4_noise_il: eta_il must be 4-byte aligned"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nsrc == 0) return TM_OK;
  const int nblk = (nsrc + 15) / 16;
  if (nblk > 65535) { set_error("z4_noise_il: too many sources (%d)", nsrc); return TM_ERR_ARG; }
  const Geom g = make_geom(gg->L, 1);
  const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  TraceScope tr((cudaStream_t)s, "z4_noise", 16.0 * 48.0 * 2.0 * g.Vh, 0.0, nblk);
  const dim3 grid((unsigned)((g.Vh + 15) / 16), 2, (unsigned)nblk);
  z4_il_kernel<<<grid, 256, 0, (cudaStream_t)s>>>(g, static_cast<unsigned*>(eta_il), key, first_src, nsrc,
                                                  prec == TM_PREC_F16 ? 0x3C00u : 0x3F80u);
  count_launch();
  return check_launch("z4_noise_il");
}

static tm_status_t z4_launch(const tm_geom_t* gg, void* eta, tm_prec_t prec, uint64_t seed,
                             uint32_t first_src, int nsrc, int t0, int dt, tm_stream_t s) {
  if (!gg || !eta || nsrc < 0) { set_error("z4_noise: null argument"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nsrc == 0) return TM_OK;
  const Geom g = make_geom(gg->L, 1);
  const unsigned nbx = 2 * blocks_for((long)g.Vh, 256);
  const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  const size_t per_src = tm_spinor_bytes(gg, prec, 1);
  TraceScope tr((cudaStream_t)s, "z4_noise", 24.0 * prec_size(prec) * 2.0 * g.Vh, 0.0, nsrc);
  return by_prec(prec, [&](auto tag) {
    using S = decltype(tag);
    // at most 65535 sources per launch (grid y)
    for (int j0 = 0; j0 < nsrc; j0 += 65535) {
      const int n = nsrc - j0 < 65535 ? nsrc - j0 : 65535;
      z4_kernel<S><<<dim3(nbx, n), 256, 0, (cudaStream_t)s>>>(g, (char*)eta + per_src * (size_t)j0, key,
                                                              first_src + (uint32_t)j0, t0, dt);
      count_launch();
      const tm_status_t st = check_launch("z4_noise");
      if (st != TM_OK) return st;
    }
    return TM_OK;
  });
}
