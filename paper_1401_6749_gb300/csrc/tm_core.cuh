// Shared device-side building blocks of the tmloops library: complex
// arithmetic, storage-precision traits, the even/odd site geometry, spinor
// and link accessors for the internal layouts, and launch bookkeeping.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <type_traits>

#include "tmloops.h"

namespace tml {

// ---------------------------------------------------------------- complex
template <class R>
struct Cx {
  R re, im;
};

template <class R>
__device__ __forceinline__ Cx<R> cx(R re, R im) { return Cx<R>{re, im}; }
template <class R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return {s * a.re, s * a.im}; }
// conj(a) * b
template <class R>
__device__ __forceinline__ Cx<R> cmulc(Cx<R> a, Cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class R>
__device__ __forceinline__ Cx<R> conjx(Cx<R> a) { return {a.re, -a.im}; }
// i^k * a for a compile-time k in 0..3
template <int K, class R>
__device__ __forceinline__ Cx<R> iphase(Cx<R> a) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return a;
  else if constexpr (k == 1) return {-a.im, a.re};
  else if constexpr (k == 2) return {-a.re, -a.im};
  else return {a.im, -a.re};
}
// runtime version (k in 0..3)
template <class R>
__device__ __forceinline__ Cx<R> iphase_rt(int k, Cx<R> a) {
  switch (k & 3) {
    case 0: return a;
    case 1: return {-a.im, a.re};
    case 2: return {-a.re, -a.im};
    default: return {a.im, -a.re};
  }
}

// ------------------------------------------------------------ float-float
// A real number as the unevaluated sum hi + lo of two FP32 values (|lo| at most
// half an ulp of hi): about 48 significant bits with the FP32 exponent range,
// computed on the FP32 pipes, which on GB300 run 64x the FP64 rate.  Built on
// the error-free transformations of Knuth (two-sum: s + e = a + b exactly)
// and Dekker (fast two-sum for |a| >= |b|; the exact product a b = p + e with
// e = fma(a, b, -p)).  The low parts are added without compensation (the
// "sloppy" addition of the double-double literature), so each operation errs
// by a few 2^-47 of the size of its operands rather than of its result.  Every
// step uses an explicit round-to-nearest intrinsic, so the compiler can
// neither contract nor reorder it.
struct FF {
  float hi, lo;
  FF() = default;
  __host__ __device__ constexpr FF(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ constexpr FF(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ constexpr FF(float h, float l) : hi(h), lo(l) {}
  // hi: d rounded to the nearest FP32; lo: the (exact) remainder, rounded
  __host__ __device__ explicit FF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
__device__ __forceinline__ FF operator-(FF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ FF operator+(FF a, FF b) {
  const FF s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF operator-(FF a, FF b) { return a + (-b); }
__device__ __forceinline__ FF operator*(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
// a b + c as one step of a compensated dot product (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005: Dot2): the
// exact product of the high parts plus its cross terms, the high part of the
// sum by an exact two-sum, and every error term added into the low part in
// FP32.  The result is left unnormalised (its low part may exceed half an
// ulp of the high part), so a chain of these depends on the previous step
// through one addition per part; ff_norm renormalises at the end of a chain,
// before the value is used as a factor or stored.
__device__ __forceinline__ FF ff_fma(FF a, FF b, FF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const FF s = ff_two_sum(c.hi, p);
  return {s.hi, __fadd_rn(c.lo, __fadd_rn(s.lo, e))};
}
__device__ __forceinline__ FF ff_norm(FF a) { return ff_two_sum(a.hi, a.lo); }
__device__ __forceinline__ FF& operator+=(FF& a, FF b) { return a = a + b; }
__device__ __forceinline__ FF shfl_xor(FF v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}
template <class T>
__device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// Storage of a float-float real: the pair (hi, lo), 8 bytes like FP64.
struct FFloat {
  float hi, lo;
};

// ------------------------------------------------------- storage precisions
// Storage type S -> arithmetic type R and how many reals one 16-byte chunk holds.
template <class S> struct Prec;
template <> struct Prec<double> { using R = double; static constexpr int kChunkReals = 2; static constexpr tm_prec_t id = TM_PREC_F64; };
template <> struct Prec<float> { using R = float; static constexpr int kChunkReals = 4; static constexpr tm_prec_t id = TM_PREC_F32; };
template <> struct Prec<__half> { using R = float; static constexpr int kChunkReals = 8; static constexpr tm_prec_t id = TM_PREC_F16; };
template <> struct Prec<__nv_bfloat16> { using R = float; static constexpr int kChunkReals = 8; static constexpr tm_prec_t id = TM_PREC_BF16; };
template <> struct Prec<FFloat> { using R = FF; static constexpr int kChunkReals = 2; static constexpr tm_prec_t id = TM_PREC_FF; };

// arithmetic wider than FP32 (kernel constants are taken in FP64 for these)
template <class R>
constexpr bool kWide = std::is_same<R, double>::value || std::is_same<R, FF>::value;

template <class S>
__host__ __device__ constexpr int spinor_chunks() { return 24 / Prec<S>::kChunkReals; }

// number of storage precisions (tm_prec_t values 0 .. kNumPrec - 1)
constexpr int kNumPrec = 5;

inline size_t prec_size(tm_prec_t p) {
  switch (p) {
    case TM_PREC_F64: return 8;
    case TM_PREC_FF: return 8;
    case TM_PREC_F32: return 4;
    default: return 2;
  }
}

// two reals <-> storage pair
__device__ __forceinline__ float2 h2f(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 h2f(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <class S> __device__ __forceinline__ S f2h(float2 v);
template <> __device__ __forceinline__ __half2 f2h<__half2>(float2 v) { return __float22half2_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat162 f2h<__nv_bfloat162>(float2 v) { return __float22bfloat162_rn(v); }
template <class S> struct Pair;
template <> struct Pair<__half> { using T = __half2; };
template <> struct Pair<__nv_bfloat16> { using T = __nv_bfloat162; };

// ----------------------------------------------------------------- geometry
// Division of a 32-bit unsigned n by an invariant d with one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> 1)) >> (l - 1),
// t = mulhi(m, n), exact for every n < 2^32 and d >= 2.
struct FastDiv {
  uint32_t d, m, l;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.l = l;
  f.m = d <= 1 ? 0u : (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  if (f.d == 1) return n;
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> 1)) >> (f.l - 1);
}

struct Geom {
  int L[4];   // X, Y, Z, T
  int Xh;     // X / 2
  int Vh;     // V / 2 (sites per parity)
  int V3h;    // X*Y*Z / 2 (sites per parity and time slice)
  int stride[4];  // lexicographic strides 1, X, XY, XYZ
  int antiperiodic;
  FastDiv dXh, dY, dZ;  // dividers for the checkerboard-index decomposition
};

inline Geom make_geom(const int L[4], int antiperiodic) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = L[i];
  g.Xh = L[0] / 2;
  g.stride[0] = 1;
  g.stride[1] = L[0];
  g.stride[2] = L[0] * L[1];
  g.stride[3] = L[0] * L[1] * L[2];
  g.V3h = g.stride[3] / 2;
  g.Vh = g.V3h * L[3];
  g.antiperiodic = antiperiodic;
  g.dXh = make_fastdiv((uint32_t)g.Xh);
  g.dY = make_fastdiv((uint32_t)L[1]);
  g.dZ = make_fastdiv((uint32_t)L[2]);
  return g;
}

// Site of parity `par` with checkerboard index cb: coordinates and lex index.
struct Site {
  int c[4];
  int lex;
};

__device__ __forceinline__ Site site_of(const Geom& g, int par, int cb) {
  Site s;
  const uint32_t q0 = fdiv((uint32_t)cb, g.dXh);
  const int xh = cb - (int)q0 * g.Xh;
  const uint32_t q1 = fdiv(q0, g.dY);
  s.c[1] = (int)q0 - (int)q1 * g.L[1];
  const uint32_t q2 = fdiv(q1, g.dZ);
  s.c[2] = (int)q1 - (int)q2 * g.L[2];
  s.c[3] = (int)q2;
  s.c[0] = 2 * xh + ((par + s.c[1] + s.c[2] + s.c[3]) & 1);
  s.lex = s.c[0] + g.stride[1] * s.c[1] + g.stride[2] * s.c[2] + g.stride[3] * s.c[3];
  return s;
}

// lex index of x +/- mu_hat (periodic wrap), and whether the hop crossed the
// time boundary.
__device__ __forceinline__ int lex_fwd(const Geom& g, const Site& s, int mu) {
  return (s.c[mu] + 1 < g.L[mu]) ? s.lex + g.stride[mu] : s.lex - (g.L[mu] - 1) * g.stride[mu];
}
__device__ __forceinline__ int lex_bwd(const Geom& g, const Site& s, int mu) {
  return (s.c[mu] > 0) ? s.lex - g.stride[mu] : s.lex + (g.L[mu] - 1) * g.stride[mu];
}

// --------------------------------------------------------- spinor accessors
// A field of nrhs spinors in the internal layout:
//   chunk index ((rhs * 2 + par) * NCH + j) * Vh + cb, each chunk 16 bytes.
template <class S>
struct SpinorRef {
  using R = typename Prec<S>::R;
  static constexpr int NCH = spinor_chunks<S>();
  __device__ __forceinline__ static size_t base(const Geom& g, int rhs, int par, int cb) {
    return ((size_t)(rhs * 2 + par) * NCH) * (size_t)g.Vh + (size_t)cb;
  }
};

// Load the 12 complex components (index 3*spin + colour) of one site.
template <class S>
__device__ __forceinline__ void load_spinor(Cx<typename Prec<S>::R> (&v)[12], const void* field,
                                            size_t b0, size_t cs) {
  const uint4* f = reinterpret_cast<const uint4*>(field);
  if constexpr (std::is_same<S, double>::value) {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const double2 d = reinterpret_cast<const double2*>(f)[b0 + j * cs];
      v[j] = {d.x, d.y};
    }
  } else if constexpr (std::is_same<S, FFloat>::value) {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const float4 d = reinterpret_cast<const float4*>(f)[b0 + j * cs];
      v[j] = {FF{d.x, d.y}, FF{d.z, d.w}};
    }
  } else if constexpr (std::is_same<S, float>::value) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 d = reinterpret_cast<const float4*>(f)[b0 + j * cs];
      v[2 * j] = {d.x, d.y};
      v[2 * j + 1] = {d.z, d.w};
    }
  } else {
    using P2 = typename Pair<S>::T;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint4 d = f[b0 + j * cs];
      const P2* h = reinterpret_cast<const P2*>(&d);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 q = h2f(h[k]);
        v[4 * j + k] = {q.x, q.y};
      }
    }
  }
}

template <class S>
__device__ __forceinline__ void store_spinor(void* field, size_t b0, size_t cs,
                                             const Cx<typename Prec<S>::R> (&v)[12]) {
  uint4* f = reinterpret_cast<uint4*>(field);
  if constexpr (std::is_same<S, double>::value) {
#pragma unroll
    for (int j = 0; j < 12; ++j)
      reinterpret_cast<double2*>(f)[b0 + j * cs] = make_double2(v[j].re, v[j].im);
  } else if constexpr (std::is_same<S, FFloat>::value) {
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const FF re = ff_norm(v[j].re), im = ff_norm(v[j].im);
      reinterpret_cast<float4*>(f)[b0 + j * cs] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
  } else if constexpr (std::is_same<S, float>::value) {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      reinterpret_cast<float4*>(f)[b0 + j * cs] =
          make_float4(v[2 * j].re, v[2 * j].im, v[2 * j + 1].re, v[2 * j + 1].im);
  } else {
    using P2 = typename Pair<S>::T;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint4 d;
      P2* h = reinterpret_cast<P2*>(&d);
#pragma unroll
      for (int k = 0; k < 4; ++k) h[k] = f2h<P2>(make_float2(v[4 * j + k].re, v[4 * j + k].im));
      f[b0 + j * cs] = d;
    }
  }
}

// ----------------------------------------------------------- link accessors
// Links of direction mu at site (par, cb): unit index ((mu * 2 + par) * NU + u) * Vh + cb.
// A link is 9 complex numbers (RECON 18) or its first two rows (RECON 12; the
// third row is conj(row0 x row1)), packed row-major into units of
// kCplxPerUnit complex numbers, the last unit zero-padded:
//   F64: double2 units (1 complex): 9 or 6 units of 16 bytes.
//   FF: (re.hi, re.lo, im.hi, im.lo) units (1 complex): 9 units of 16 bytes.
//   F32: float4 units (2 complex): 5 (18) or 3 (12) units of 16 bytes.
//   F16/BF16: RECON 18 -> 16-byte units of 4 complex (3 units),
//             RECON 12 -> 8-byte units of 2 complex (3 units).
template <class S, int RECON>
struct LinkFmt {
  static constexpr bool kF64 = std::is_same<S, double>::value;
  static constexpr bool kFF = std::is_same<S, FFloat>::value;
  static constexpr bool kF32 = std::is_same<S, float>::value;
  static constexpr int kCplx = RECON == 18 ? 9 : 6;
  static constexpr int kCplxPerUnit = (kF64 || kFF) ? 1 : (kF32 ? 2 : (RECON == 18 ? 4 : 2));
  static constexpr int NU = (kCplx + kCplxPerUnit - 1) / kCplxPerUnit;
  static constexpr int kUnitBytes = kCplxPerUnit * 2 * (int)sizeof(S);
};

template <class R>
struct Mat3 {
  Cx<R> m[3][3];
};

template <class S, int RECON>
__device__ __forceinline__ Mat3<typename Prec<S>::R> load_link(const void* links, const Geom& g,
                                                                int mu, int par, int cb) {
  using R = typename Prec<S>::R;
  using F = LinkFmt<S, RECON>;
  Mat3<R> U;
  Cx<R> e[F::NU * F::kCplxPerUnit];
  const size_t b0 = ((size_t)(mu * 2 + par) * F::NU) * (size_t)g.Vh + (size_t)cb;
  const size_t cs = (size_t)g.Vh;
  if constexpr (F::kF64) {
    const double2* p = reinterpret_cast<const double2*>(links);
#pragma unroll
    for (int u = 0; u < F::NU; ++u) {
      const double2 d = p[b0 + u * cs];
      e[u] = {d.x, d.y};
    }
  } else if constexpr (F::kFF) {
    const float4* p = reinterpret_cast<const float4*>(links);
#pragma unroll
    for (int u = 0; u < F::NU; ++u) {
      const float4 d = p[b0 + u * cs];
      e[u] = {FF{d.x, d.y}, FF{d.z, d.w}};
    }
  } else if constexpr (F::kF32) {
    const float4* p = reinterpret_cast<const float4*>(links);
#pragma unroll
    for (int u = 0; u < F::NU; ++u) {
      const float4 d = p[b0 + u * cs];
      e[2 * u] = {d.x, d.y};
      e[2 * u + 1] = {d.z, d.w};
    }
  } else {
    using P2 = typename Pair<S>::T;
    if constexpr (RECON == 18) {
      const uint4* p = reinterpret_cast<const uint4*>(links);
#pragma unroll
      for (int u = 0; u < F::NU; ++u) {
        const uint4 d = p[b0 + u * cs];
        const P2* h = reinterpret_cast<const P2*>(&d);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 q = h2f(h[k]);
          e[4 * u + k] = {q.x, q.y};
        }
      }
    } else {
      const uint2* p = reinterpret_cast<const uint2*>(links);
#pragma unroll
      for (int u = 0; u < F::NU; ++u) {
        const uint2 d = p[b0 + u * cs];
        const P2* h = reinterpret_cast<const P2*>(&d);
        const float2 q0 = h2f(h[0]), q1 = h2f(h[1]);
        e[2 * u] = {q0.x, q0.y};
        e[2 * u + 1] = {q1.x, q1.y};
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) U.m[i][j] = e[3 * i + j];
  if constexpr (RECON == 18) {
#pragma unroll
    for (int j = 0; j < 3; ++j) U.m[2][j] = e[6 + j];
  } else {
    // third row of an SU(3) matrix: complex conjugate of row0 x row1
    U.m[2][0] = conjx(U.m[0][1] * U.m[1][2] - U.m[0][2] * U.m[1][1]);
    U.m[2][1] = conjx(U.m[0][2] * U.m[1][0] - U.m[0][0] * U.m[1][2]);
    U.m[2][2] = conjx(U.m[0][0] * U.m[1][1] - U.m[0][1] * U.m[1][0]);
  }
  return U;
}

// ------------------------------------------------------------ bookkeeping
// While this thread captures a CUDA graph, launches are counted per captured
// graph (capture_begin / capture_end return how many one replay runs) and are
// not traced; the caller counts each replay.
void count_launch(int n = 1);
void capture_begin();
int capture_end();
void set_error(const char* fmt, ...);
tm_status_t check_launch(const char* what);
// Tracing of Dslash launches (tm_trace_enable): trace_begin records a start
// event and returns a device slot in which the kernel stores how many of its
// systems were active (nullptr when tracing is off); trace_end records the end
// event with the launch's algorithmic bytes per active system and per launch,
// and its algorithmic flops per active system.
int* trace_begin(cudaStream_t s, cudaEvent_t* ev0);
void trace_end(cudaStream_t s, const char* name, cudaEvent_t ev0, int* slot, double bytes_per_rhs,
               double fixed_bytes, int nrhs_if_uncounted = 0, double flops_per_rhs = 0.0);

// RAII form for kernels that do not count their active systems: all nrhs
// systems are taken as active.
struct TraceScope {
  cudaStream_t s;
  const char* name;
  cudaEvent_t ev = nullptr;
  double per_rhs, fixed;
  int nrhs;
  TraceScope(cudaStream_t st, const char* n, double bytes_per_rhs, double fixed_bytes, int nr)
      : s(st), name(n), per_rhs(bytes_per_rhs), fixed(fixed_bytes), nrhs(nr) {
    trace_begin(s, &ev);
  }
  ~TraceScope() { trace_end(s, name, ev, nullptr, per_rhs, fixed, nrhs); }
};


}  // namespace tml
