// Shared pieces of the kernels on the system-interleaved 16-bit layout
// (IL16): the packed 16-bit complex words, the warp-level MMA, the layout's
// constants and the bulk-copy / mbarrier staging primitives.
//
// Layout IL16: a set of nrhs 16-bit spinor fields stored as ceil(nrhs / 16)
// blocks of 16 systems, [block][parity][cb][k = 3 spin + colour][slot 0..15]
// x 4 bytes, one complex number (re in the low half) per slot, 64 bytes per
// (site, k) and 768 contiguous bytes per site.  Systems j and j + 8
// (j = 0..7) share one 8-byte pair of slots, at pair position j in rows
// k = 0, 1 (mod 3) and j ^ 4 in rows k = 2 (mod 3).
#pragma once

#include <cuda.h>

#include "tm_host.h"

namespace tml {

constexpr int kIlRows = 16;   // systems per interleaved block (MMA rows)
// ----------------------------------------------------------- 16-bit words
template <class S> struct H16;
template <> struct H16<__half> {
  static constexpr unsigned kMinusPlus = 0x3C00BC00u;  // (re -1, im +1)
  static constexpr unsigned kPlusMinus = 0xBC003C00u;  // (re +1, im -1)
  static __device__ __forceinline__ unsigned add(unsigned a, unsigned b) {
    unsigned d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
  }
  static __device__ __forceinline__ unsigned sub(unsigned a, unsigned b) {
    unsigned d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
  }
  static __device__ __forceinline__ unsigned fma(unsigned a, unsigned b, unsigned c) {
    unsigned d;
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
  }
  static __device__ __forceinline__ float2 to_f2(unsigned w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
  }
  static __device__ __forceinline__ unsigned pack(float re, float im) {
    const __half2 h = __floats2half2_rn(re, im);
    return *reinterpret_cast<const unsigned*>(&h);
  }
};
template <> struct H16<__nv_bfloat16> {
  static constexpr unsigned kMinusPlus = 0x3F80BF80u;
  static constexpr unsigned kPlusMinus = 0xBF803F80u;
  static __device__ __forceinline__ unsigned add(unsigned a, unsigned b) {
    unsigned d;
    asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
  }
  static __device__ __forceinline__ unsigned sub(unsigned a, unsigned b) {
    unsigned d;
    asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
  }
  static __device__ __forceinline__ unsigned fma(unsigned a, unsigned b, unsigned c) {
    unsigned d;
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
  }
  static __device__ __forceinline__ float2 to_f2(unsigned w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  static __device__ __forceinline__ unsigned pack(float re, float im) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<const unsigned*>(&h);
  }
};

// a + i^K b, rounded once to the storage format (the phase is exact: a swap
// of halves and a sign, as a product by (+-1, +-1) inside one packed FMA)
template <int K, class S>
__device__ __forceinline__ unsigned proj_w(unsigned a, unsigned b) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return H16<S>::add(a, b);
  else if constexpr (k == 2) return H16<S>::sub(a, b);
  else if constexpr (k == 1) return H16<S>::fma(__byte_perm(b, 0u, 0x1032), H16<S>::kMinusPlus, a);
  else return H16<S>::fma(__byte_perm(b, 0u, 0x1032), H16<S>::kPlusMinus, a);
}

// i^K times a 16-bit complex word: swap halves and flip signs, exact
template <int K>
__device__ __forceinline__ unsigned il_rot(unsigned h) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return h;
  else if constexpr (k == 2) return h ^ 0x80008000u;
  else if constexpr (k == 1) return __byte_perm(h, 0u, 0x1032) ^ 0x00008000u;  // (-im, re)
  else return __byte_perm(h, 0u, 0x1032) ^ 0x80000000u;                        // (im, -re)
}

template <class S>
__device__ __forceinline__ void il_mma(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                       unsigned b0, unsigned b1) {
  if constexpr (std::is_same<S, __half>::value)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  else
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// D = A B (the accumulators' first product: C = 0, which the tensor core adds
// exactly as it would add zeroed registers)
template <class S>
__device__ __forceinline__ void il_mma0(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                        unsigned b0, unsigned b1) {
  const float z = 0.0f;
  if constexpr (std::is_same<S, __half>::value)
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(z));
  else
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%10,%10,%10};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(z));
}

// first product into an accumulator (FIRST) or one more
template <class S, bool FIRST>
__device__ __forceinline__ void il_mma_acc(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                           unsigned b0, unsigned b1) {
  if constexpr (FIRST) il_mma0<S>(d, a0, a1, a2, a3, b0, b1);
  else il_mma<S>(d, a0, a1, a2, a3, b0, b1);
}

// Words of one site in uint2 units: site cb of parity par in block blk starts
// at ((blk * 2 + par) * Vh + cb) * 96; lane (g, t) reads spin s at + (3 s + t) * 8 + g.
constexpr int kIlSiteU2 = 96;
constexpr int kIlSiteBytes = 768;
constexpr int kIlLinkBytes = 48;                 // one direction of one site: 9 words + 3 pad
constexpr int kIlLinkSiteBytes = 4 * kIlLinkBytes;
constexpr unsigned kIlWaitLimit = 1u << 22;      // try_wait rounds before a wait gives up
constexpr unsigned long long kIlWaitNs = 1000000000ull;  // global time before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar), "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// rows of row_words 4-byte words at base as a 2-D tensor whose box is one
// whole row, for the gather4 copies (host; dslash_il.cu)
tm_status_t il_row_map(CUtensorMap* m, const void* base, unsigned row_words, size_t rows);

// four rows of a 2-D tensor (rows r0..r3, the whole box of columns from
// column 0) into consecutive rows at dst: one tensor copy in gather4 mode
__device__ __forceinline__ void gather4_g2s(unsigned dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

// bounded wait for a stage; false (and the launch's error flag set) if it
// gave up, after kIlWaitNs of global time or kIlWaitLimit rounds
__device__ __forceinline__ bool il_wait(unsigned bar, unsigned phase, int* err) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0; it < kIlWaitLimit; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if (global_ns() - t0 > kIlWaitNs) break;
  }
  if (err) atomicExch(err, 1);
  return false;
}

}  // namespace tml
