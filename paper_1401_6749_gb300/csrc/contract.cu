// Loop contractions (Sec. 2.2; Table 2 "local" and "one-derivative"
// operators) and the Truncated Solver Method combination (Sec. 2.1, Eq. 4).
//
// Both contractions first build, per time slice, the 4x4 Dirac matrices
//   S_{ab}(t) = sum_{x_t = t} sum_c conj(L_{ac}(x)) W_{bc}(x)
// (W = R for local insertions; W = U_mu(x) R(x+mu) or U_mu(x-mu)^dag R(x-mu) for
// the one-derivative ones) and only then project them on the 16 Gamma
// matrices: every Gamma_g of the DeGrand-Rossi basis is a phased permutation,
// so Tr[(P Gamma_g)^T S] = sum_a i^{k_ga} S_{a, pi_g(a)} costs four terms.
//
// Reductions are deterministic and independent of the batch: each block sums
// a fixed chunk of one (slice, parity) of one right-hand side; a warp
// butterfly (transpose-reduce) leaves lane j with component j, the eight warp
// results are added in order, and a final kernel adds the chunk partials in
// order.
#include <cmath>
#include <cstring>
#include <limits>

#include "dslash.cuh"

namespace tml {

// ------------------------------------------------------- warp butterfly
// v[0..31] per lane in, lane l returns the warp sum of component l.
template <class T>
__device__ __forceinline__ T warp_transpose_reduce(T (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const T send = up ? v[i] : v[i + w];
      const T keep = up ? v[i + w] : v[i];
      v[i] = keep + shfl_xor(send, w);
    }
  }
  return v[0];
}

// --------------------------------------------------------- local loops
constexpr int kLocalK = 4;          // sites per thread
constexpr int kLocalChunk = 256 * kLocalK;

// momenta of a projected contraction: p = 2 pi (n_x / X, n_y / Y, n_z / Z)
constexpr int kMaxMom = 64;
struct MomList {
  int n;
  int p[kMaxMom][3];
};

// MOM: the site's R is multiplied by exp(-i p.x), block z = rhs * n + momentum
template <class S, bool MOM = false>
__global__ void __launch_bounds__(256) local_partial_kernel(Geom g, const void* Lf, const void* Rf,
                                                            int nchunk, double* partial,
                                                            MomList mom = MomList{}) {
  using R = typename Prec<S>::R;
  // MOM: the momentum is the fastest block index, so the blocks of one chunk
  // (one set of sites) for all momenta run together and re-read L, R from L2
  const int q = MOM ? (int)blockIdx.x % mom.n : 0;
  const int chunk = MOM ? (int)blockIdx.x / mom.n : (int)blockIdx.x;
  const int t = blockIdx.y >> 1, par = blockIdx.y & 1;
  const int rhs = blockIdx.z;
  const int slot_rhs = MOM ? rhs * mom.n + q : rhs;  // index of this contraction's output
  R acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0;
#pragma unroll 1
  for (int k = 0; k < kLocalK; ++k) {
    const int i = chunk * kLocalChunk + k * 256 + (int)threadIdx.x;
    if (i < g.V3h) {
      const size_t b0 = SpinorRef<S>::base(g, rhs, par, t * g.V3h + i);
      Cx<R> l[12], r[12];
      load_spinor<S>(l, Lf, b0, (size_t)g.Vh);
      load_spinor<S>(r, Rf, b0, (size_t)g.Vh);
      if constexpr (MOM) {
        const Site st = site_of(g, par, t * g.V3h + i);
        // phase -2 pi sum_k n_k x_k / L_k, reduced exactly modulo one turn first
        const long num = (long)((mom.p[q][0] * st.c[0]) % g.L[0]) * g.L[1] * g.L[2] +
                         (long)((mom.p[q][1] * st.c[1]) % g.L[1]) * g.L[0] * g.L[2] +
                         (long)((mom.p[q][2] * st.c[2]) % g.L[2]) * g.L[0] * g.L[1];
        const long den = (long)g.L[0] * g.L[1] * g.L[2];
        const double frac = (double)(num % den) / (double)den;
        Cx<R> ph;
        if constexpr (kWide<R>) {
          double sn, cn;
          sincospi(-2.0 * frac, &sn, &cn);
          ph = {(R)cn, (R)sn};
        } else {
          float sn, cn;
          sincospif(-2.0f * (float)frac, &sn, &cn);
          ph = {cn, sn};
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) r[k] = ph * r[k];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const Cx<R> m = cmulc(l[3 * a + c], r[3 * b + c]);
            acc[2 * (4 * a + b)] += m.re;
            acc[2 * (4 * a + b) + 1] += m.im;
          }
    }
  }
  const R v = warp_transpose_reduce(acc);
  __shared__ double sh[8][32];
  sh[threadIdx.x >> 5][threadIdx.x & 31] = (double)v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += sh[w][threadIdx.x];
    const size_t slot = (((size_t)slot_rhs * g.L[3] + t) * 2 + par) * nchunk + chunk;
    partial[slot * 32 + threadIdx.x] = s;
  }
}

// Gamma projection of a 4x4 complex matrix stored as 32 doubles (row-major, re/im).
__device__ __forceinline__ Cx<double> gamma_project(const double* S, const GammaTab& tab, int gidx,
                                                    int p_g5) {
  Cx<double> acc = {0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int b = tab.perm[gidx][a];
    const int k = tab.k[gidx][a] + ((p_g5 && a >= 2) ? 2 : 0);
    const Cx<double> s = {S[2 * (4 * a + b)], S[2 * (4 * a + b) + 1]};
    acc = acc + iphase_rt(k, s);
  }
  return acc;
}

__global__ void local_final_kernel(const double* partial, int nchunk, int T, GammaTab tab,
                                   int p_g5, double* out) {
  const int t = blockIdx.x, rhs = blockIdx.y;
  __shared__ double S[32];
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int par = 0; par < 2; ++par) {
      const size_t slot0 = (((size_t)rhs * T + t) * 2 + par) * nchunk;
      for (int c = 0; c < nchunk; ++c) s += partial[(slot0 + c) * 32 + threadIdx.x];
    }
    S[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    const Cx<double> v = gamma_project(S, tab, threadIdx.x, p_g5);
    const size_t o = (((size_t)rhs * 16 + threadIdx.x) * T + t) * 2;
    out[o] = v.re;
    out[o + 1] = v.im;
  }
}

// ----------------------------------------------------- one-derivative loops
// With A_mu(x) = Lb(x) G U_mu(x) R(x+mu) and B_mu(x) = Lb(x) G U_mu(x-mu)^dag R(x-mu)
// the symmetric-derivative loop of slice t is
//   spatial mu:  1/4 sum_{x_t=t} [A(x) + A(x-mu) - B(x) - B(x+mu)] = 1/2 sum_{x_t=t} (A - B)(x),
//   mu = t:      1/4 [C(t) + C(t-1)],  C(t) = sum_{x_t=t} C(x),  C(x) = A(x) - B(x+t),
// since x -> x +/- mu permutes a time slice for spatial mu, and A(x), B(x+t)
// both live on the link (x, x+t).  So one 4x4 accumulator per direction:
//   spatial: L^dag(x) [U_mu(x) R(x+mu) - U_mu(x-mu)^dag R(x-mu)]
//   time:    L^dag(x) U_t(x) R(x+t) - L^dag(x+t) U_t(x)^dag R(x)   (boundary sign on both)
// Work split: a warp handles 32 sites of one direction mu and one half h of the
// column index b (b = 2h, 2h + 1), so the link products are computed for two
// spins only and each thread keeps 16 accumulators; FP64 loads L one Dirac row
// at a time to stay within two resident blocks per SM.
constexpr int kOneDK = 8;           // sites per thread
constexpr int kOneDLanes = 32;      // sites side by side in a block (x 8 warps)
constexpr int kOneDChunk = kOneDLanes * kOneDK;


__device__ __forceinline__ int sel4(const int (&a)[4], int mu) {
  return mu == 0 ? a[0] : mu == 1 ? a[1] : mu == 2 ? a[2] : a[3];
}

// components 6h .. 6h + 5 (spins 2h, 2h + 1) of a site's spinor
template <class S>
__device__ __forceinline__ void load_spins2(Cx<typename Prec<S>::R> (&v)[6], const void* field, size_t b0,
                                           size_t cs, int h) {
  using R = typename Prec<S>::R;
  const uint4* f = reinterpret_cast<const uint4*>(field);
  if constexpr (std::is_same<S, double>::value) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const double2 d = reinterpret_cast<const double2*>(f)[b0 + (6 * h + j) * cs];
      v[j] = {d.x, d.y};
    }
  } else if constexpr (std::is_same<S, FFloat>::value) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 d = reinterpret_cast<const float4*>(f)[b0 + (6 * h + j) * cs];
      v[j] = {FF{d.x, d.y}, FF{d.z, d.w}};
    }
  } else if constexpr (std::is_same<S, float>::value) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float4 d = reinterpret_cast<const float4*>(f)[b0 + (3 * h + j) * cs];
      v[2 * j] = {d.x, d.y};
      v[2 * j + 1] = {d.z, d.w};
    }
  } else {
    using P2 = typename Pair<S>::T;
    Cx<R> e[8];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint4 d = f[b0 + (h + j) * cs];
      const P2* q = reinterpret_cast<const P2*>(&d);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 z = h2f(q[k]);
        e[4 * j + k] = {z.x, z.y};
      }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = h ? e[2 + j] : e[j];
  }
}

// w (+/-)= U r or U^dag r for two spins (four FMAs per complex multiply-add)
template <bool ADJ, bool SUB, class R>
__device__ __forceinline__ void link_times2(Cx<R> (&w)[6], const Mat3<R>& U, const Cx<R> (&r)[6]) {
  using O = Ar<R>;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R zr = SUB ? w[3 * a + c].re : (R)0, zi = SUB ? w[3 * a + c].im : (R)0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const Cx<R> u0 = ADJ ? conjx(U.m[d][c]) : U.m[c][d];
        const Cx<R> u = SUB ? Cx<R>{-u0.re, -u0.im} : u0;  // subtract: negated (exactly) link
        const Cx<R> x = r[3 * a + d];
        zr = O::fma(u.re, x.re, zr);
        zr = O::fma(-u.im, x.im, zr);
        zi = O::fma(u.re, x.im, zi);
        zi = O::fma(u.im, x.re, zi);
      }
      w[3 * a + c] = {O::norm(zr), O::norm(zi)};
    }
}

// acc_{a, bb} += sgn * sum_c conj(l_{a c}) w_{bb c}, a = 0..3, bb = 0..1; FP64 reads
// one row of L at a time
template <class S, class R>
__device__ __forceinline__ void outer_acc2(R (&acc)[16], const void* Lf, size_t b0, size_t cs,
                                           const Cx<R> (&w)[6], R sgn) {
  using O = Ar<R>;
  Cx<R> ws[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) ws[j] = {sgn * w[j].re, sgn * w[j].im};
  if constexpr (kWide<R>) {
#pragma unroll 1
    for (int a = 0; a < 4; ++a) {
      Cx<R> l[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (std::is_same<S, double>::value) {
          const double2 d = reinterpret_cast<const double2*>(Lf)[b0 + (3 * a + c) * cs];
          l[c] = {d.x, d.y};
        } else {
          const float4 d = reinterpret_cast<const float4*>(Lf)[b0 + (3 * a + c) * cs];
          l[c] = {FF{d.x, d.y}, FF{d.z, d.w}};
        }
      }
      // a runtime index into acc would move it to local memory: select instead
#pragma unroll
      for (int aa = 0; aa < 4; ++aa) {
        if (aa != a) continue;
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
          R mr = acc[2 * (2 * aa + bb)], mi = acc[2 * (2 * aa + bb) + 1];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            mr = O::fma(l[c].re, ws[3 * bb + c].re, mr);
            mr = O::fma(l[c].im, ws[3 * bb + c].im, mr);
            mi = O::fma(l[c].re, ws[3 * bb + c].im, mi);
            mi = O::fma(-l[c].im, ws[3 * bb + c].re, mi);
          }
          acc[2 * (2 * aa + bb)] = mr;
          acc[2 * (2 * aa + bb) + 1] = mi;
        }
      }
    }
  } else {
    Cx<R> l[12];
    load_spinor<S>(l, Lf, b0, cs);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        R mr = acc[2 * (2 * a + bb)], mi = acc[2 * (2 * a + bb) + 1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const Cx<R> x = l[3 * a + c];
          mr = O::fma(x.re, ws[3 * bb + c].re, mr);
          mr = O::fma(x.im, ws[3 * bb + c].im, mr);
          mi = O::fma(x.re, ws[3 * bb + c].im, mi);
          mi = O::fma(-x.im, ws[3 * bb + c].re, mi);
        }
        acc[2 * (2 * a + bb)] = mr;
        acc[2 * (2 * a + bb) + 1] = mi;
      }
  }
}

// v[0..15] per lane in; lane l returns the warp sum of component l & 15
template <class T>
__device__ __forceinline__ T warp_transpose_reduce16(T (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] += shfl_xor(v[i], 16);
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const T send = up ? v[i] : v[i + w];
      const T keep = up ? v[i + w] : v[i];
      v[i] = keep + shfl_xor(send, w);
    }
  }
  return v[0];
}

template <class S>
constexpr int oned_min_blocks() { return std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value ? 3 : 2; }

template <class S, int RECON>
__global__ void __launch_bounds__(256, oned_min_blocks<S>()) oneD_partial_kernel(
    Geom g, const void* links, const void* Lf, const void* Rf, int nchunk, double* partial) {
  using R = typename Prec<S>::R;
  // the system index is the fastest block index: the blocks of all systems
  // for one set of sites run together and share its links through L2
  const int rhs = blockIdx.x;
  const int chunk = blockIdx.y;
  const int t = blockIdx.z >> 1, par = blockIdx.z & 1;
  const int mu = threadIdx.y >> 1, h = threadIdx.y & 1;
  const int opar = par ^ 1;
  const size_t cs = (size_t)g.Vh;
  R acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0;
  const int Lmu = sel4(g.L, mu), smu = sel4(g.stride, mu);
#pragma unroll 1
  for (int k = 0; k < kOneDK; ++k) {
    const int i = chunk * kOneDChunk + k * kOneDLanes + (int)threadIdx.x;
    if (i >= g.V3h) continue;
    const int cb = t * g.V3h + i;
    const Site s = site_of(g, par, cb);
    const int cmu = sel4(s.c, mu);
    const int lf = cmu + 1 < Lmu ? s.lex + smu : s.lex - (Lmu - 1) * smu;
    const size_t bx = SpinorRef<S>::base(g, rhs, par, cb);
    const size_t bf = SpinorRef<S>::base(g, rhs, opar, lf >> 1);
    Cx<R> w[6];
    if constexpr (kRawLinks<S, RECON>) {
      unsigned u[9], x[6];
      if (mu < 3) {
        const int lb = cmu > 0 ? s.lex - smu : s.lex + (Lmu - 1) * smu;
        load_link_raw<S>(u, links, g, mu, par, cb);
        load_spins2_raw<S>(x, Rf, bf, cs, h);
        link_times2_raw<false, false, S>(w, u, x);
        load_link_raw<S>(u, links, g, mu, opar, lb >> 1);
        load_spins2_raw<S>(x, Rf, SpinorRef<S>::base(g, rhs, opar, lb >> 1), cs, h);
        link_times2_raw<true, true, S>(w, u, x);
        outer_acc2<S>(acc, Lf, bx, cs, w, (R)1);
      } else {
        const R sf = (g.antiperiodic && cmu == Lmu - 1) ? (R)-1 : (R)1;
        load_link_raw<S>(u, links, g, mu, par, cb);
        load_spins2_raw<S>(x, Rf, bf, cs, h);
        link_times2_raw<false, false, S>(w, u, x);
        outer_acc2<S>(acc, Lf, bx, cs, w, sf);
        load_spins2_raw<S>(x, Rf, bx, cs, h);
        link_times2_raw<true, false, S>(w, u, x);
        outer_acc2<S>(acc, Lf, bf, cs, w, -sf);
      }
    } else {
      Cx<R> r[6];
      if (mu < 3) {
        const int lb = cmu > 0 ? s.lex - smu : s.lex + (Lmu - 1) * smu;
        {
          const Mat3<R> U = load_link<S, RECON>(links, g, mu, par, cb);
          load_spins2<S>(r, Rf, bf, cs, h);
          link_times2<false, false>(w, U, r);
        }
        {
          const Mat3<R> Ub = load_link<S, RECON>(links, g, mu, opar, lb >> 1);
          load_spins2<S>(r, Rf, SpinorRef<S>::base(g, rhs, opar, lb >> 1), cs, h);
          link_times2<true, true>(w, Ub, r);
        }
        outer_acc2<S>(acc, Lf, bx, cs, w, (R)1);
      } else {
        const R sf = (g.antiperiodic && cmu == Lmu - 1) ? (R)-1 : (R)1;
        const Mat3<R> U = load_link<S, RECON>(links, g, mu, par, cb);
        load_spins2<S>(r, Rf, bf, cs, h);
        link_times2<false, false>(w, U, r);
        outer_acc2<S>(acc, Lf, bx, cs, w, sf);
        load_spins2<S>(r, Rf, bx, cs, h);
        link_times2<true, false>(w, U, r);
        outer_acc2<S>(acc, Lf, bf, cs, w, -sf);
      }
    }
  }
  {
    using O = Ar<R>;
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = O::norm(acc[j]);
  }
  const R v = warp_transpose_reduce16(acc);
  const int lane = threadIdx.x & 31;
  if (lane < 16) {
    // local component 2 (2a + bb) + re/im  ->  global 2 (4a + 2h + bb) + re/im
    const int ab = lane >> 1, a = ab >> 1, bb = ab & 1;
    const int comp = 2 * (4 * a + 2 * h + bb) + (lane & 1);
    const size_t slot = (((size_t)rhs * g.L[3] + t) * 2 + par) * nchunk + chunk;
    partial[slot * 128 + mu * 32 + comp] = (double)v;
  }
}

// block per (t, rhs), 160 threads: 128 sums of slice t, 32 of C_t(t - 1)
__global__ void oneD_final_kernel(const double* partial, int nchunk, int T, GammaTab tab, int p_g5,
                                  double* out) {
  const int t = blockIdx.x, rhs = blockIdx.y;
  __shared__ double Q[4][32];
  __shared__ double Cm[32];
  const int tid = threadIdx.x;
  const int slice = tid < 128 ? t : (t + T - 1) % T;
  const int comp = tid < 128 ? tid : 3 * 32 + (tid - 128);
  double s = 0.0;
  for (int par = 0; par < 2; ++par) {
    const size_t slot0 = (((size_t)rhs * T + slice) * 2 + par) * nchunk;
    for (int c = 0; c < nchunk; ++c) s += partial[(slot0 + c) * 128 + comp];
  }
  if (tid < 128) Q[tid >> 5][tid & 31] = s;
  else Cm[tid - 128] = s;
  __syncthreads();
  __shared__ double D[4][32];
  if (tid < 128) {
    const int mu = tid >> 5, e = tid & 31;
    D[mu][e] = mu < 3 ? 0.5 * Q[mu][e] : 0.25 * (Q[3][e] + Cm[e]);
  }
  __syncthreads();
  if (tid < 64) {
    const int mu = tid >> 4, gi = tid & 15;
    const Cx<double> v = gamma_project(D[mu], tab, gi, p_g5);
    const size_t o = ((((size_t)rhs * 4 + mu) * 16 + gi) * T + t) * 2;
    out[o] = v.re;
    out[o + 1] = v.im;
  }
}

// --------------------------------------------------------- TSM combine
__device__ __forceinline__ Cx<double> scaled(const double* a, size_t idx, Cx<double> c) {
  return c * Cx<double>{a[2 * idx], a[2 * idx + 1]};
}

__global__ void tsm_kernel(const double* hp, const double* lphp, int n_hp, const double* lp, int n_lp,
                           size_t len, Cx<double> c, double* mean, double* err) {
  const size_t j = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  // biased estimate over the low-precision-only sources
  double mr = 0, mi = 0;
  for (int i = 0; i < n_lp; ++i) {
    const Cx<double> v = scaled(lp, (size_t)i * len + j, c);
    mr += v.re;
    mi += v.im;
  }
  mr /= n_lp;
  mi /= n_lp;
  double e2r, e2i;
  if (n_lp > 1) {
    double vr = 0, vi = 0;
    for (int i = 0; i < n_lp; ++i) {
      const Cx<double> v = scaled(lp, (size_t)i * len + j, c);
      vr += (v.re - mr) * (v.re - mr);
      vi += (v.im - mi) * (v.im - mi);
    }
    e2r = vr / (n_lp - 1) / n_lp;
    e2i = vi / (n_lp - 1) / n_lp;
  } else {
    e2r = e2i = nan;
  }
  if (n_hp > 0) {
    double dr = 0, di = 0;
    for (int i = 0; i < n_hp; ++i) {
      const size_t q = (size_t)i * len + j;
      const Cx<double> v = scaled(hp, q, c) - scaled(lphp, q, c);
      dr += v.re;
      di += v.im;
    }
    dr /= n_hp;
    di /= n_hp;
    if (n_hp > 1) {
      double vr = 0, vi = 0;
      for (int i = 0; i < n_hp; ++i) {
        const size_t q = (size_t)i * len + j;
        const Cx<double> v = scaled(hp, q, c) - scaled(lphp, q, c);
        vr += (v.re - dr) * (v.re - dr);
        vi += (v.im - di) * (v.im - di);
      }
      e2r += vr / (n_hp - 1) / n_hp;
      e2i += vi / (n_hp - 1) / n_hp;
    } else {
      e2r = e2i = nan;
    }
    mr += dr;
    mi += di;
  }
  mean[2 * j] = mr;
  mean[2 * j + 1] = mi;
  err[2 * j] = sqrt(e2r);
  err[2 * j + 1] = sqrt(e2i);
}

template <class F>
static tm_status_t by_prec_c(tm_prec_t p, F&& f) {
  switch (p) {
    case TM_PREC_F64: return f(double{});
    case TM_PREC_F32: return f(float{});
    case TM_PREC_F16: return f(__half{});
    case TM_PREC_BF16: return f(__nv_bfloat16{});
    case TM_PREC_FF: return f(FFloat{});
    default: set_error("unknown precision %d", (int)p); return TM_ERR_ARG;
  }
}

static const char* prec_name(const char* const (&names)[kNumPrec], tm_prec_t p) {
  return names[(unsigned)p < (unsigned)kNumPrec ? (int)p : 0];
}

static tm_status_t scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
  return dev_alloc(p, bytes, s, "contraction scratch");
}

// local contraction with caller-chosen scratch (>= local_scratch_bytes)
size_t local_scratch_bytes(const Geom& g, int nrhs) {
  const int nchunk = (g.V3h + kLocalChunk - 1) / kLocalChunk;
  return sizeof(double) * 32 * (size_t)nrhs * g.L[3] * 2 * nchunk;
}

tm_status_t local_contract_into(const Geom& g, const void* left, const void* right, tm_prec_t prec,
                                int nrhs, int p_g5, double* out, double* scratch, cudaStream_t s) {
  const int nchunk = (g.V3h + kLocalChunk - 1) / kLocalChunk;
  const dim3 grid(nchunk, 2 * g.L[3], nrhs);
  static const char* const kNames[kNumPrec] = {"local.f64", "local.f32", "local.f16", "local.bf16", "local.ff"};
  TraceScope tr(s, prec_name(kNames, prec), 2.0 * 24.0 * prec_size(prec) * 2.0 * g.Vh, 0.0, nrhs);
  tm_status_t st = by_prec_c(prec, [&](auto tag) {
    using S = decltype(tag);
    local_partial_kernel<S><<<grid, 256, 0, s>>>(g, left, right, nchunk, scratch);
    count_launch();
    return check_launch("loop_contract_local");
  });
  if (st != TM_OK) return st;
  local_final_kernel<<<dim3(g.L[3], nrhs), 32, 0, s>>>(scratch, nchunk, g.L[3], gamma_tab(), p_g5, out);
  count_launch();
  return check_launch("loop_contract_local final");
}

// The final reductions as host entry points (the interleaved contractions of
// loops_il.cu write partial sums in the layouts of these kernels).
tm_status_t local_final(const double* partial, int nchunk, const Geom& g, int nrhs, int p_g5, double* out,
                        cudaStream_t s) {
  local_final_kernel<<<dim3(g.L[3], nrhs), 32, 0, s>>>(partial, nchunk, g.L[3], gamma_tab(), p_g5, out);
  count_launch();
  return check_launch("local loops final");
}

tm_status_t oned_final(const double* partial, int nchunk, const Geom& g, int nrhs, int p_g5, double* out,
                       cudaStream_t s) {
  oneD_final_kernel<<<dim3(g.L[3], nrhs), 160, 0, s>>>(partial, nchunk, g.L[3], gamma_tab(), p_g5, out);
  count_launch();
  return check_launch("one-derivative loops final");
}

}  // namespace tml

using namespace tml;

static bool valid_mode(tm_loop_mode_t m) { return m == TM_LOOP_STD || m == TM_LOOP_VV || m == TM_LOOP_GEN; }

extern "C" tm_status_t loop_contract_local(const tm_geom_t* gg, const void* left, const void* right,
                                           tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                                           double* out, tm_stream_t strm) {
  if (!gg || !left || !right || !out || nrhs < 0) { set_error("loop_contract_local: null argument"); return TM_ERR_ARG; }
  if (!valid_mode(mode)) { set_error("loop_contract_local: unknown mode %d", (int)mode); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  if (nrhs > 65535) { set_error("loop_contract_local: nrhs must be <= 65535"); return TM_ERR_ARG; }
  if (2 * gg->L[3] > 65535) { set_error("loop_contract_local: T = %d exceeds the launch grid (2 T <= 65535)", gg->L[3]); return TM_ERR_ARG; }
  const cudaStream_t s = (cudaStream_t)strm;
  const Geom g = make_geom(gg->L, 1);
  double* scratch = nullptr;
  tm_status_t st = scratch_alloc((void**)&scratch, local_scratch_bytes(g, nrhs), s);
  if (st != TM_OK) return st;
  st = local_contract_into(g, left, right, prec, nrhs, mode != TM_LOOP_STD, out, scratch, s);
  dev_free(scratch, s);
  return st;
}

extern "C" tm_status_t loop_contract_local_mom(const tm_geom_t* gg, const void* left, const void* right,
                                               tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                                               const int* mom, int n_mom, double* out, tm_stream_t strm) {
  if (!gg || !left || !right || !out || !mom || nrhs < 0) { set_error("loop_contract_local_mom: null argument"); return TM_ERR_ARG; }
  if (!valid_mode(mode)) { set_error("loop_contract_local_mom: unknown mode %d", (int)mode); return TM_ERR_ARG; }
  if (n_mom < 1 || n_mom > kMaxMom) { set_error("loop_contract_local_mom: 1 <= n_mom <= %d", kMaxMom); return TM_ERR_ARG; }
  if ((int)prec < 0 || (int)prec >= kNumPrec) { set_error("loop_contract_local_mom: unknown precision"); return TM_ERR_ARG; }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  if ((long)nrhs * n_mom > 65535) { set_error("loop_contract_local_mom: nrhs * n_mom must be <= 65535"); return TM_ERR_ARG; }
  if (2 * gg->L[3] > 65535) { set_error("loop_contract_local_mom: T = %d exceeds the launch grid (2 T <= 65535)", gg->L[3]); return TM_ERR_ARG; }
  const cudaStream_t s = (cudaStream_t)strm;
  const Geom g = make_geom(gg->L, 1);
  MomList ml;
  ml.n = n_mom;
  for (int q = 0; q < n_mom; ++q)
    for (int k = 0; k < 3; ++k) {
      const int Lk = g.L[k];
      ml.p[q][k] = ((mom[3 * q + k] % Lk) + Lk) % Lk;  // p and p + L are the same momentum
    }
  const int n2 = nrhs * n_mom;
  double* scratch = nullptr;
  tm_status_t st = scratch_alloc((void**)&scratch, local_scratch_bytes(g, n2), s);
  if (st != TM_OK) return st;
  const int nchunk = (g.V3h + kLocalChunk - 1) / kLocalChunk;
  const dim3 grid(nchunk * n_mom, 2 * g.L[3], nrhs);
  {
    static const char* const kNames[kNumPrec] = {"localmom.f64", "localmom.f32", "localmom.f16", "localmom.bf16",
                                                  "localmom.ff"};
    TraceScope tr(s, prec_name(kNames, prec), 2.0 * 24.0 * prec_size(prec) * 2.0 * g.Vh, 0.0, n2);
    st = by_prec_c(prec, [&](auto tag) {
      using S = decltype(tag);
      local_partial_kernel<S, true><<<grid, 256, 0, s>>>(g, left, right, nchunk, scratch, ml);
      count_launch();
      return check_launch("loop_contract_local_mom");
    });
  }
  if (st == TM_OK) {
    local_final_kernel<<<dim3(g.L[3], n2), 32, 0, s>>>(scratch, nchunk, g.L[3], gamma_tab(),
                                                        mode != TM_LOOP_STD, out);
    count_launch();
    st = check_launch("loop_contract_local_mom final");
  }
  dev_free(scratch, s);
  return st;
}

extern "C" tm_status_t loop_contract_oneD(tm_op_t* op, const void* left, const void* right,
                                          tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                                          double* out, tm_stream_t strm) {
  if (!op || !left || !right || !out || nrhs < 0) { set_error("loop_contract_oneD: null argument"); return TM_ERR_ARG; }
  if (!valid_mode(mode)) { set_error("loop_contract_oneD: unknown mode %d", (int)mode); return TM_ERR_ARG; }
  if ((int)prec < 0 || (int)prec >= kNumPrec) { set_error("loop_contract_oneD: unknown precision %d", (int)prec); return TM_ERR_ARG; }
  if (nrhs == 0) return TM_OK;
  const cudaStream_t s = (cudaStream_t)strm;
  const Geom& g = op->g;
  const int nchunk = (g.V3h + kOneDChunk - 1) / kOneDChunk;
  if (nchunk > 65535 || 2 * g.L[3] > 65535) { set_error("loop_contract_oneD: lattice too large for the grid"); return TM_ERR_ARG; }
  double* scratch = nullptr;
  tm_status_t st = scratch_alloc((void**)&scratch, sizeof(double) * 128 * (size_t)nrhs * g.L[3] * 2 * nchunk, s);
  if (st != TM_OK) return st;
  const dim3 grid(nrhs, nchunk, 2 * g.L[3]);
  const dim3 block(kOneDLanes, 8);
  const bool r12 = op->recon_p[prec] == 12;
  const void* links = op->links[prec];
  static const char* const kNames[kNumPrec] = {"oneD.f64", "oneD.f32", "oneD.f16", "oneD.bf16", "oneD.ff"};
  const double esz = (double)prec_size(prec);
  const double lreals = r12 ? 12.0 : 18.0;
  TraceScope tr(s, prec_name(kNames, prec), 2.0 * 24.0 * esz * 2.0 * g.Vh, 4.0 * lreals * esz * 2.0 * g.Vh, nrhs);
  switch (prec) {
    case TM_PREC_F64:
      oneD_partial_kernel<double, 18><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch); break;
    case TM_PREC_FF:
      oneD_partial_kernel<FFloat, 18><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch); break;
    case TM_PREC_F32:
      if (r12) oneD_partial_kernel<float, 12><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch);
      else oneD_partial_kernel<float, 18><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch);
      break;
    case TM_PREC_F16:
      if (r12) oneD_partial_kernel<__half, 12><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch);
      else oneD_partial_kernel<__half, 18><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch);
      break;
    case TM_PREC_BF16:
      if (r12) oneD_partial_kernel<__nv_bfloat16, 12><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch);
      else oneD_partial_kernel<__nv_bfloat16, 18><<<grid, block, 0, s>>>(g, links, left, right, nchunk, scratch);
      break;
    default:
      dev_free(scratch, s);
      set_error("loop_contract_oneD: unknown precision %d", (int)prec);
      return TM_ERR_ARG;
  }
  count_launch();
  st = check_launch("loop_contract_oneD");
  if (st == TM_OK) {
    oneD_final_kernel<<<dim3(g.L[3], nrhs), 160, 0, s>>>(scratch, nchunk, g.L[3], gamma_tab(),
                                                          mode != TM_LOOP_STD, out);
    count_launch();
    st = check_launch("loop_contract_oneD final");
  }
  dev_free(scratch, s);
  return st;
}

// The same combination on host arrays: the per-source loop sets are small
// (kilobytes per source), so a caller that gathered them on the host (or
// across processes) combines them without a device round trip.  Each
// component is computed with the device kernel's formula in the same order.
extern "C" tm_status_t tsm_combine_host(const double* l_hp, const double* l_lp_on_hp, int n_hp,
                                        const double* l_lp, int n_lp, size_t len, double scale_re,
                                        double scale_im, double* mean, double* err) {
  if (!l_lp || !mean || !err || n_hp < 0) { set_error("tsm_combine_host: null argument"); return TM_ERR_ARG; }
  if (n_lp < 1) { set_error("tsm_combine_host: the estimator needs n_lp >= 1"); return TM_ERR_ARG; }
  if (n_hp > 0 && (!l_hp || !l_lp_on_hp)) { set_error("tsm_combine_host: null high-precision arrays"); return TM_ERR_ARG; }
  const double nan = std::numeric_limits<double>::quiet_NaN();
  auto sc = [&](const double* a, size_t idx, double& re, double& im) {
    const double xr = a[2 * idx], xi = a[2 * idx + 1];
    re = scale_re * xr - scale_im * xi;
    im = scale_re * xi + scale_im * xr;
  };
  for (size_t j = 0; j < len; ++j) {
    double mr = 0, mi = 0, re, im;
    for (int i = 0; i < n_lp; ++i) { sc(l_lp, (size_t)i * len + j, re, im); mr += re; mi += im; }
    mr /= n_lp;
    mi /= n_lp;
    double e2r = nan, e2i = nan;
    if (n_lp > 1) {
      double vr = 0, vi = 0;
      for (int i = 0; i < n_lp; ++i) {
        sc(l_lp, (size_t)i * len + j, re, im);
        vr += (re - mr) * (re - mr);
        vi += (im - mi) * (im - mi);
      }
      e2r = vr / (n_lp - 1) / n_lp;
      e2i = vi / (n_lp - 1) / n_lp;
    }
    if (n_hp > 0) {
      double dr = 0, di = 0, hr, hi;
      for (int i = 0; i < n_hp; ++i) {
        sc(l_hp, (size_t)i * len + j, hr, hi);
        sc(l_lp_on_hp, (size_t)i * len + j, re, im);
        dr += hr - re;
        di += hi - im;
      }
      dr /= n_hp;
      di /= n_hp;
      if (n_hp > 1) {
        double vr = 0, vi = 0;
        for (int i = 0; i < n_hp; ++i) {
          sc(l_hp, (size_t)i * len + j, hr, hi);
          sc(l_lp_on_hp, (size_t)i * len + j, re, im);
          vr += (hr - re - dr) * (hr - re - dr);
          vi += (hi - im - di) * (hi - im - di);
        }
        e2r += vr / (n_hp - 1) / n_hp;
        e2i += vi / (n_hp - 1) / n_hp;
      } else {
        e2r = e2i = nan;
      }
      mr += dr;
      mi += di;
    }
    mean[2 * j] = mr;
    mean[2 * j + 1] = mi;
    err[2 * j] = std::sqrt(e2r);
    err[2 * j + 1] = std::sqrt(e2i);
  }
  return TM_OK;
}

extern "C" tm_status_t tsm_combine(const double* l_hp, const double* l_lp_on_hp, int n_hp,
                                   const double* l_lp, int n_lp, size_t len, double scale_re,
                                   double scale_im, double* mean, double* err, tm_stream_t strm) {
  if (!l_lp || !mean || !err || n_hp < 0) { set_error("tsm_combine: null argument"); return TM_ERR_ARG; }
  if (n_lp < 1) { set_error("tsm_combine: the estimator needs n_lp >= 1"); return TM_ERR_ARG; }
  if (n_hp > 0 && (!l_hp || !l_lp_on_hp)) { set_error("tsm_combine: null high-precision arrays"); return TM_ERR_ARG; }
  if (len == 0) return TM_OK;
  const cudaStream_t s = (cudaStream_t)strm;
  const unsigned nb = (unsigned)((len + 127) / 128);
  tsm_kernel<<<nb, 128, 0, s>>>(l_hp, l_lp_on_hp, n_hp, l_lp, n_lp, len, Cx<double>{scale_re, scale_im},
                                mean, err);
  count_launch();
  return check_launch("tsm_combine");
}
