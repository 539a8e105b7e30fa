// Local and one-derivative loop contractions (Sec. 2.2; Table 2) on the
// system-interleaved 16-bit layout (IL16, il_core.cuh).
//
// Both produce the per-(slice, parity, chunk) partial sums of the standard
// contractions (contract.cu), in the same layout, and share their final
// kernels: per time slice t and system the 4x4 Dirac matrices
//   local:  S_ab(t)      = sum_{x_t = t} sum_c conj(L_ac(x)) R_bc(x)
//   oneD:   S^mu_ab(t)   = sum_{x_t = t} sum_c conj(L_ac(x)) W^mu_bc(x)
//   spatial mu: W = U_mu(x) R(x+mu) - U_mu(x-mu)^dag R(x-mu)
//   mu = t:     C(x) = L^dag(x) U_t(x) R(x+t) - L^dag(x+t) U_t(x)^dag R(x)
// (antiperiodic sign on both terms of the links that cross the boundary);
// the final kernel forms the symmetric derivative and projects on the 16
// Gamma matrices.  With right_g5 the right field enters as gamma_5 R, i.e.
// the columns b = 2, 3 change sign (gamma_5 = diag(1, 1, -1, -1)).
//
// One-derivative kernel, per site x and block of 16 systems, two tensor-core
// stages:
//  1. link products, rows = systems (as in the interleaved Dslash): per
//     spin b one mma.sync.m16n8k16 per direction with
//       A[system][(hop, colour, re/im)] = R_b(x+mu) words (k 0..7) and
//         R_b(x-mu) words (k 8..15), straight from the staged sites,
//       B = the real form of [U_mu(x); -U_mu(x-mu)^dag];
//     for mu = t the two terms of C(x) are separate products on A = [R_b(x+t);
//     R_b(x)] with B = [U_t(x); 0] and [0; -U_t(x)^dag].  20 MMAs, D rows =
//     systems, columns = (colour, re/im).
//  2. spin outer products, rows = (mu, b), one system per MMA: after the
//     products are rounded to the storage format and transposed through
//     shared memory, system s takes
//       A[(mu, b)][(term, colour, re/im)] = W^s (term 1) and the second time
//         term (rows (t, b) only),
//       B[(term, colour, re/im)][(a, re/im)] = the real form of conj(L^s(x))
//         (term 1) and conj(L^s(x+t)) (term 2): column (a, re) the word
//         L_ac itself, column (a, im) i L_ac,
//     so D[(mu, b)][(a, re/im)] accumulates Re / Im sum conj(L_ac) W_bc over
//     the warp's sites in the FP32 accumulators of 16 MMA tiles.
// Rows of stage 1 and tiles of stage 2 never mix systems, and every sum runs
// in a fixed order, so each system's loops depend on its own fields only.
//
// Staging: each warp owns two stages in shared memory (site m + 1 is in
// flight while m is computed); a stage holds the ten sites R(x +- mu)
// (spatial), R(x + t), R(x), L(x), L(x + t) and the links U_mu(x) (192
// bytes) and U_mu(x - mu) (3 x 48 bytes): fourteen bulk copies, one per lane
// role, completing on the stage's mbarrier; every wait is bounded and sets
// the operator's flag when it gives up.  The rounded products of a direction
// overwrite that direction's own neighbour sites once they are read.
#include "il_core.cuh"

namespace tml {

// sites of one (slice, parity) per block (a tuning build may set TM_OD_CHUNK:
// smaller blocks keep fewer sites in flight in L2, larger ones write fewer partial sums)
#ifndef TM_OD_CHUNK
#define TM_OD_CHUNK 512
#endif
constexpr int kOdWarps = 4;
constexpr int kOdChunk = TM_OD_CHUNK;
constexpr int kOdWarpSites = kOdChunk / kOdWarps;   // sites per warp
static_assert(kOdChunk % (32 * kOdWarps) == 0, "whole 32-site groups per warp");

struct OdStage {
  static constexpr int kLinkOff = 10 * kIlSiteBytes;                 // ten sites, then U_mu(x)
  // U_mu(x - mu), mu < 3, and a fourth row (a copy of mu = 2) that fills the
  // gather4 copy; on a 128-byte line, as tensor copies need
  static constexpr int kBwdOff = kLinkOff + 256;
  static constexpr int kCopyBytes = 10 * kIlSiteBytes + kIlLinkSiteBytes + 4 * kIlLinkBytes;  // 8064 per site
  // stages start on 128-byte lines, so that every stage has the bank
  // alignment of the zero block's line
  static constexpr int kBytes = kBwdOff + 256;                        // 8192
  static constexpr int kStages = 2;
  static constexpr int kWarpBytes = kStages * kBytes;
  // zero words for the lanes without a product word: 48 bytes into a line,
  // so that system s's zero word sits in bank 12 s + 12 (mod 32) of the
  // stage's alignment, which no product word read by the same instruction
  // occupies
  static constexpr int kZeroOff = kOdWarps * kWarpBytes + 48;
  static constexpr int kSmem = kZeroOff + kIlSiteBytes;
  // stage slots: 2 mu / 2 mu + 1 = R(x + mu) / R(x - mu) (mu < 3), 6 R(x + t),
  // 7 R(x), 8 L(x), 9 L(x + t).  Rounded products of class q (q = mu, and 4
  // for the second time term), [system][colour][b] words, 768 bytes each,
  // over the slots of their own direction; the 64-byte shifts put the
  // classes read together (0 / 1, 2 / 3) in different banks.
  static __host__ __device__ constexpr int w(int q) {
    return q == 0 ? 0 : q == 1 ? 2 * kIlSiteBytes + 64 : q == 2 ? 4 * kIlSiteBytes + 64 : q == 3 ? 6 * kIlSiteBytes
                                                                                                 : 7 * kIlSiteBytes;
  }
};
static_assert(OdStage::kBytes % 128 == 0 && OdStage::kWarpBytes % 128 == 0, "stages on 128-byte lines");
static_assert(OdStage::w(1) + kIlSiteBytes <= 4 * kIlSiteBytes && OdStage::w(2) + kIlSiteBytes <= 6 * kIlSiteBytes,
              "product classes inside their slots");

struct OdArgs {
  Geom g;
  const void* links_il;
  int* err;
  const unsigned char* L;
  const unsigned char* R;
  double* partial;
  int nrhs, nblk, nchunk, right_g5;
};

__device__ __forceinline__ unsigned lds32(const unsigned char* p) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ uint2 lds64(const unsigned char* p) { return *reinterpret_cast<const uint2*>(p); }

// D (rows g, g + 8; columns colour t re, im) of the four spins -> the 16-byte
// words [b = 0..3] of systems g and g + 8 at colour t
template <class S>
__device__ __forceinline__ void od_store(unsigned char* w, const float (&d)[4][4]) {
  using H = H16<S>;
  *reinterpret_cast<uint4*>(w) =
      make_uint4(H::pack(d[0][0], d[0][1]), H::pack(d[1][0], d[1][1]), H::pack(d[2][0], d[2][1]), H::pack(d[3][0], d[3][1]));
  *reinterpret_cast<uint4*>(w + 8 * 48) =
      make_uint4(H::pack(d[0][2], d[0][3]), H::pack(d[1][2], d[1][3]), H::pack(d[2][2], d[2][3]), H::pack(d[3][2], d[3][3]));
}

template <class S>
__global__ void __launch_bounds__(kOdWarps * 32, 3)
    oneD_il_kernel(const OdArgs a, const __grid_constant__ CUtensorMap tr, const __grid_constant__ CUtensorMap tlk) {
  using ST = OdStage;
  extern __shared__ __align__(128) unsigned char od_smem[];
  __shared__ __align__(8) unsigned long long bars[kOdWarps][ST::kStages];
  __shared__ __align__(16) int rowbuf[kOdWarps][12];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  // the tensor copies need 128-byte aligned destinations: a block whose
  // dynamic shared memory is not (never expected) flags the error and stops
  if (smem_u32(od_smem) & 127u) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    return;
  }
  const int blk = blockIdx.x % a.nblk, chunk = blockIdx.x / a.nblk;
  const int t = blockIdx.y >> 1, par = blockIdx.y & 1, opar = par ^ 1;
  const size_t Vh = (size_t)g.Vh;
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < ST::kStages; ++st) mbar_init(smem_u32(&bars[wq][st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kIlSiteBytes / 4; i += blockDim.x)
    reinterpret_cast<unsigned*>(od_smem + ST::kZeroOff)[i] = 0u;
  __syncthreads();
  // sites of this warp: i0 + 4 m (m < nsite) of slice t
  const int i0 = chunk * kOdChunk + wq;
  const int nsite = i0 >= g.V3h ? 0 : min(kOdWarpSites, (g.V3h - i0 + kOdWarps - 1) / kOdWarps);
  const int cb0 = t * g.V3h + i0;
  float acc[kIlRows][4];
#pragma unroll
  for (int s = 0; s < kIlRows; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = 0.0f;
  const int gq = lane >> 2, tq = lane & 3;
  if (nsite > 0) {
    // row role of this lane: 0..5 R(x +- mu), 6 R(x + t), 7 R(x), rows
    // (blk * 2 + parity) * Vh + cb of the field; 8..11 U_mu(x - mu) (lane 11
    // repeats mu = 2), rows (opar * Vh + cb') * 4 + mu of the links.  Hop roles
    // add the neighbour's lex step (or its wrap), R(x) takes the site itself.
    // L(x) and L(x + t) are the rows of R(x) and R(x + t) in the left field.
    const bool hop = lane != 7;
    const int rmu = lane < 6 ? (lane >> 1) : lane == 6 ? 3 : (lane >= 8 && lane < 12 ? min(lane - 8, 2) : 0);
    const bool rbwd = lane < 6 ? (lane & 1) != 0 : lane >= 8;
    const int rbit = 2 * rmu + (rbwd ? 1 : 0);
    const int rstep = rbwd ? -g.stride[rmu] : g.stride[rmu];
    const int rwrap = rbwd ? (g.L[rmu] - 1) * g.stride[rmu] : -(g.L[rmu] - 1) * g.stride[rmu];
    const int rrow0 = lane < 8 ? (blk * 2 + (lane == 7 ? par : opar)) * g.Vh : opar * g.Vh * 4 + rmu;
    const int rrmul = lane < 8 ? 1 : 4;
    const unsigned char* lk = reinterpret_cast<const unsigned char*>(a.links_il) + (size_t)par * Vh * kIlLinkSiteBytes;
    constexpr unsigned total = ST::kCopyBytes;
    static_assert(ST::kLinkOff % 128 == 0 && ST::kBwdOff % 128 == 0 && ST::kBytes % 128 == 0 &&
                      ST::kBwdOff >= ST::kLinkOff + kIlLinkSiteBytes && ST::kBytes >= ST::kBwdOff + 4 * kIlLinkBytes,
                  "stage layout");
    unsigned char* ring = od_smem + wq * ST::kWarpBytes;
    const unsigned ring_s = smem_u32(ring);
    const unsigned bar0 = smem_u32(&bars[wq][0]);
    // lane m of the current group of 32 sites: lex index and the mask of the
    // hops that wrap (bit 2 mu forward, 2 mu + 1 backward)
    int lexl = 0;
    unsigned bml = 0u;
    auto site_info = [&](int grp) {
      const int mm = grp * 32 + lane;
      lexl = 0;
      bml = 0u;
      if (mm < nsite) {
        const Site s = site_of(g, par, cb0 + kOdWarps * mm);
        lexl = s.lex;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
          bml |= (s.c[mu] == g.L[mu] - 1 ? 1u : 0u) << (2 * mu) | (s.c[mu] == 0 ? 2u : 0u) << (2 * mu);
      }
    };
    auto issue = [&](int m, int st) {
      const int lex = __shfl_sync(0xffffffffu, lexl, m & 31);
      const unsigned msk = __shfl_sync(0xffffffffu, bml, m & 31);
      const int nlex = lex + (((msk >> rbit) & 1u) ? rwrap : rstep);
      const int cb = cb0 + kOdWarps * m;
      if (lane < 12) rowbuf[wq][lane] = rrow0 + (hop ? (nlex >> 1) : cb) * rrmul;
      const unsigned bar = bar0 + st * 8;
      __syncwarp();
      if (lane == 0) {
        // every copy of the stage from one lane: gather4 of R's eight rows,
        // the two rows of L, the site's links, gather4 of the backward links
        const int4 q0 = *reinterpret_cast<const int4*>(&rowbuf[wq][0]);
        const int4 q1 = *reinterpret_cast<const int4*>(&rowbuf[wq][4]);
        const int4 q2 = *reinterpret_cast<const int4*>(&rowbuf[wq][8]);
        const unsigned sb = ring_s + st * ST::kBytes;
        mbar_expect_tx(bar, total);
        gather4_g2s(sb, &tr, q0.x, q0.y, q0.z, q0.w, bar);
        gather4_g2s(sb + 4 * kIlSiteBytes, &tr, q1.x, q1.y, q1.z, q1.w, bar);
        bulk_g2s(sb + 8 * kIlSiteBytes, a.L + (size_t)q1.w * kIlSiteBytes, kIlSiteBytes, bar);
        bulk_g2s(sb + 9 * kIlSiteBytes, a.L + (size_t)q1.z * kIlSiteBytes, kIlSiteBytes, bar);
        bulk_g2s(sb + ST::kLinkOff, lk + (size_t)cb * kIlLinkSiteBytes, kIlLinkSiteBytes, bar);
        gather4_g2s(sb + ST::kBwdOff, &tlk, q2.x, q2.y, q2.z, q2.w, bar);
      }
    };
    // stage 1 lane constants (as the interleaved Dslash): A words of rows
    // g, g + 8 at colour t (lanes t = 3 read colour 0 against zero B rows);
    // link words, forward U[g/2][t], adjoint U[t][g/2], loaded by every lane
    // (lanes t = 3 those of t = 0, zeroed by the byte selector psel; lanes
    // g = 6, 7 pad or colour words into the B columns of output colour 3,
    // which no lane stores); B word transforms
    const int teff = tq < 3 ? tq : 0;
    const int woff = teff * 64 + (teff == 2 ? gq ^ 4 : gq) * 8;
    const int lf_off = (3 * (gq >> 1) + teff) * 4, lb_off = (3 * teff + (gq >> 1)) * 4;
    const bool odd = (gq & 1) != 0;
    const unsigned psel = tq == 3 ? 0x4444u : odd ? 0x1032u : 0x3210u;
    const unsigned pfw = odd ? 0u : 0x80000000u;   // forward:  conj(u) / (u_im, u_re)
    const unsigned pad = odd ? 0x00008000u : 0u;   // adjoint:  u / (-u_im, u_re)
    // stage 2 lane constants: A words (row g' = 4 mu + b of class g' >> 2 and
    // 2 + (g' >> 2), colour t') and the second time term (rows 12..15 = lanes
    // g' >= 4); lanes without a word read the zero block.  B: L word of spin
    // a = g' >> 1 at colour t', i L on odd columns.
    const int offa0 = tq < 3 ? ST::w(gq >> 2) + tq * 16 + (gq & 3) * 4 : -1;
    const int offa1 = tq < 3 ? ST::w(2 + (gq >> 2)) + tq * 16 + (gq & 3) * 4 : -1;
    const int offa3 = (tq < 3 && gq >= 4) ? ST::w(4) + tq * 16 + (gq - 4) * 4 : -1;
    const unsigned char* zero = od_smem + ST::kZeroOff;
    const int lrow = (3 * (gq >> 1) + teff) * 64;
    const int x4 = teff == 2 ? 32 : 0;  // the XOR of colour-2 rows on pair positions 0..3 / 4..7
    const int loff_lo = lrow + x4, loff_hi = lrow - x4;
    const unsigned rsel = odd ? 0x1032u : 0x3210u, rmsk = odd ? 0x00008000u : 0u;
    site_info(0);
    issue(0, 0);
    for (int m = 0; m < nsite; ++m) {
      const int st = m & 1;
      const unsigned msk_m = __shfl_sync(0xffffffffu, bml, m & 31);
      if (m + 1 < nsite) {
        if (((m + 1) & 31) == 0) site_info((m + 1) >> 5);
        // the stage was last read (and written) by this warp's generic
        // accesses, ordered before this copy by the fence and barrier below
        issue(m + 1, st ^ 1);
      }
      if (!__all_sync(0xffffffffu, il_wait(bar0 + st * 8, (unsigned)((m >> 1) & 1), a.err))) {
        if (m + 1 < nsite) il_wait(bar0 + (st ^ 1) * 8, (unsigned)(((m + 1) >> 1) & 1), nullptr);
        break;
      }
      unsigned char* sd = ring + st * ST::kBytes;
      // ---- stage 1: link products, rounded, over their own neighbour slots
#pragma unroll
      for (int mu = 0; mu < 3; ++mu) {
        uint2 pf[4], pb[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          pf[s] = lds64(sd + (2 * mu) * kIlSiteBytes + woff + 192 * s);
          pb[s] = lds64(sd + (2 * mu + 1) * kIlSiteBytes + woff + 192 * s);
        }
        const unsigned uf = lds32(sd + ST::kLinkOff + mu * kIlLinkBytes + lf_off);
        const unsigned ub = lds32(sd + ST::kBwdOff + mu * kIlLinkBytes + lb_off);
        const unsigned b0 = __byte_perm(uf, 0u, psel) ^ pfw;
        const unsigned b1 = __byte_perm(ub, 0u, psel) ^ pad ^ 0x80008000u;
        float d[4][4];
#pragma unroll
        for (int s = 0; s < 4; ++s) il_mma0<S>(d[s], pf[s].x, pf[s].y, pb[s].x, pb[s].y, b0, b1);
        __syncwarp();  // every lane has read the slots before they are overwritten
        if (tq < 3) od_store<S>(sd + ST::w(mu) + gq * 48 + tq * 16, d);
      }
      {
        uint2 pf[4], pc[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          pf[s] = lds64(sd + 6 * kIlSiteBytes + woff + 192 * s);
          pc[s] = lds64(sd + 7 * kIlSiteBytes + woff + 192 * s);
        }
        const unsigned ut = lds32(sd + ST::kLinkOff + 3 * kIlLinkBytes + lf_off);
        const unsigned ua = lds32(sd + ST::kLinkOff + 3 * kIlLinkBytes + lb_off);
        const unsigned neg = (g.antiperiodic && (msk_m & 0x40u)) ? 0x80008000u : 0u;
        const unsigned bt = __byte_perm(ut, 0u, psel) ^ pfw ^ neg;
        const unsigned ba = __byte_perm(ua, 0u, psel) ^ pad ^ 0x80008000u ^ neg;
        float d1[4][4], d2[4][4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          il_mma0<S>(d1[s], pf[s].x, pf[s].y, pc[s].x, pc[s].y, bt, 0u);
          il_mma0<S>(d2[s], pf[s].x, pf[s].y, pc[s].x, pc[s].y, 0u, ba);
        }
        __syncwarp();
        if (tq < 3) {
          od_store<S>(sd + ST::w(3) + gq * 48 + tq * 16, d1);
          od_store<S>(sd + ST::w(4) + gq * 48 + tq * 16, d2);
        }
      }
      __syncwarp();  // the rounded products of every lane are in place
      // ---- stage 2: spin outer products, one MMA per system
      const unsigned char* pa0 = offa0 >= 0 ? sd + offa0 : zero;
      const unsigned char* pa1 = offa1 >= 0 ? sd + offa1 : zero;
      const unsigned char* pa3 = offa3 >= 0 ? sd + offa3 : zero;
      const unsigned char* lx = sd + 8 * kIlSiteBytes;
      const unsigned char* lt = sd + 9 * kIlSiteBytes;
#pragma unroll
      for (int p = 0; p < 8; p += 2) {
        // systems p, p + 8, p + 1, p + 9 of L(x) and L(x + t)
        const int lo = (p < 4 ? loff_lo : loff_hi) + p * 8;
        const uint4 qx = *reinterpret_cast<const uint4*>(lx + lo);
        const uint4 qt = *reinterpret_cast<const uint4*>(lt + lo);
        const unsigned wx[4] = {qx.x, qx.y, qx.z, qx.w}, wt[4] = {qt.x, qt.y, qt.z, qt.w};
        const int sys[4] = {p, p + 8, p + 1, p + 9};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int s = sys[j];
          const unsigned b0 = __byte_perm(wx[j], 0u, rsel) ^ rmsk;
          const unsigned b1 = __byte_perm(wt[j], 0u, rsel) ^ rmsk;
          il_mma<S>(acc[s], lds32(pa0 + s * 48), lds32(pa1 + s * 48), 0u, lds32(pa3 + s * 48), b0, b1);
        }
      }
      // order this warp's generic accesses to the stage before the next bulk
      // copy into it (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
    }
  }
  // ---- per-block sums: warp tiles -> shared memory (the stages are idle:
  // every copy issued was waited for) -> FP64 over the warps in order
  __syncthreads();
  float* red = reinterpret_cast<float*>(od_smem);  // [warp][system][128]
  {
    const int b = gq & 3, mu0 = gq >> 2;
    const float sg = (a.right_g5 && b >= 2) ? -1.0f : 1.0f;
    const int c0 = mu0 * 32 + 2 * (4 * tq + b);
#pragma unroll
    for (int s = 0; s < kIlRows; ++s) {
      float* r = red + (wq * kIlRows + s) * 128;
      r[c0] = sg * acc[s][0];
      r[c0 + 1] = sg * acc[s][1];
      r[c0 + 64] = sg * acc[s][2];
      r[c0 + 65] = sg * acc[s][3];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kIlRows * 128; i += blockDim.x) {
    const int s = i >> 7, comp = i & 127;
    const int rhs = blk * kIlRows + s;
    if (rhs >= a.nrhs) continue;
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kOdWarps; ++w) v += (double)red[(w * kIlRows + s) * 128 + comp];
    const size_t slot = (((size_t)rhs * g.L[3] + t) * 2 + par) * a.nchunk + chunk;
    a.partial[slot * 128 + comp] = v;
  }
}

// ----------------------------------------------------------------- local
// A warp takes two sites at a time: lane 16 h + j holds system j of site h,
// whose word of row k sits in slot 2 ((j & 7) ^ (k = 2 mod 3 ? 4 : 0)) + j / 8,
// so each half-warp reads one 64-byte row per load.  A lane keeps the 16
// products conj(L_a) R_b of its system summed over the colours in FP32
// (mixed-precision FMAs on the 16-bit halves: exact products); the two
// half-warps' sums are added at the end.  The next site's 24 words are in
// flight while one site is computed.
constexpr int kLcWarps = 4;
constexpr int kLcChunk = 512;

template <class S>
__device__ __forceinline__ void mfma(float& d, unsigned short a, unsigned short b) {
  if constexpr (std::is_same<S, __half>::value)
    asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(d) : "h"(a), "h"(b));
  else
    asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(d) : "h"(a), "h"(b));
}

template <class S>
__global__ void __launch_bounds__(kLcWarps * 32) local_il_kernel(Geom g, const unsigned* L, const unsigned* R,
                                                                 int nrhs, int nblk, int nchunk, int right_g5,
                                                                 double* partial) {
  __shared__ float red[kLcWarps][kIlRows][32];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int blk = blockIdx.x % nblk, chunk = blockIdx.x / nblk;
  const int t = blockIdx.y >> 1, par = blockIdx.y & 1;
  const int h = lane >> 4, j = lane & 15;
  const int slot01 = 2 * (j & 7) + (j >> 3), slot2 = 2 * ((j & 7) ^ 4) + (j >> 3);
  float acc[16][2];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q][0] = acc[q][1] = 0.0f;
  const size_t plane = ((size_t)blk * 2 + par) * (size_t)g.Vh * (kIlSiteBytes / 4);
  const unsigned* lp = L + plane;
  const unsigned* rp = R + plane;
  const int i0 = chunk * kLcChunk, iend = min(g.V3h, i0 + kLcChunk);
  // site i0 + 2 (wq + 4 m) + h of slice t
  unsigned ln[12], rn[12];
  auto fetch = [&](int i) {
    const size_t w = (size_t)(t * g.V3h + i) * (kIlSiteBytes / 4);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int sl = k % 3 == 2 ? slot2 : slot01;
      ln[k] = lp[w + 16 * k + sl];
      rn[k] = rp[w + 16 * k + sl];
    }
  };
  int i = i0 + 2 * wq + h;
  if (i < iend) fetch(i);
  for (; i < iend; i += 2 * kLcWarps) {
    unsigned l[12], r[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      l[k] = ln[k];
      r[k] = rn[k];
    }
    if (i + 2 * kLcWarps < iend) fetch(i + 2 * kLcWarps);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const unsigned lw = l[3 * a + c], rw = r[3 * b + c];
          const unsigned short lre = (unsigned short)(lw & 0xffffu), lim = (unsigned short)(lw >> 16);
          const unsigned short rre = (unsigned short)(rw & 0xffffu), rim = (unsigned short)(rw >> 16);
          // conj(l) r = (lre rre + lim rim) + i (lre rim - lim rre)
          mfma<S>(acc[4 * a + b][0], lre, rre);
          mfma<S>(acc[4 * a + b][0], lim, rim);
          mfma<S>(acc[4 * a + b][1], lre, rim);
          mfma<S>(acc[4 * a + b][1], (unsigned short)(lim ^ 0x8000u), rre);
        }
  }
  // the two sites of a step hold the same system: add the half-warps
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    acc[q][0] += __shfl_xor_sync(0xffffffffu, acc[q][0], 16);
    acc[q][1] += __shfl_xor_sync(0xffffffffu, acc[q][1], 16);
  }
  if (h == 0) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float sg = (right_g5 && (q & 3) >= 2) ? -1.0f : 1.0f;  // q = 4 a + b
      red[wq][j][2 * q] = sg * acc[q][0];
      red[wq][j][2 * q + 1] = sg * acc[q][1];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kIlRows * 32; k += blockDim.x) {
    const int sy = k >> 5, comp = k & 31;
    const int rhs = blk * kIlRows + sy;
    if (rhs >= nrhs) continue;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < kLcWarps; ++q) v += (double)red[q][sy][comp];
    const size_t slot = (((size_t)rhs * g.L[3] + t) * 2 + par) * nchunk + chunk;
    partial[slot * 32 + comp] = v;
  }
}

static tm_status_t il_fields_ok(const char* what, const void* left, const void* right, tm_prec_t prec) {
  if (prec != TM_PREC_F16 && prec != TM_PREC_BF16) {
    set_error("%s: the interleaved layout holds F16 or BF16 fields", what);
    return TM_ERR_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(left) | reinterpret_cast<uintptr_t>(right)) & 15u) {
    set_error("%s: fields must be 16-byte aligned", what);
    return TM_ERR_ARG;
  }
  return TM_OK;
}

tm_status_t oned_il_prepare() {
  const int smem = OdStage::kSmem;
  if (cudaFuncSetAttribute(oneD_il_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaFuncSetAttribute(oneD_il_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess) {
    set_error("interleaved one-derivative kernel: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

}  // namespace tml

using namespace tml;

static bool valid_mode_il(tm_loop_mode_t m) { return m == TM_LOOP_STD || m == TM_LOOP_VV || m == TM_LOOP_GEN; }

extern "C" tm_status_t loop_contract_local_il(const tm_geom_t* gg, const void* left, const void* right,
                                              tm_prec_t prec, int nrhs, tm_loop_mode_t mode, int right_g5,
                                              double* out, tm_stream_t strm) {
  const char* what = "loop_contract_local_il";
  if (!gg || !left || !right || !out || nrhs < 0) { set_error("%s: null argument", what); return TM_ERR_ARG; }
  if (!valid_mode_il(mode)) { set_error("%s: unknown mode %d", what, (int)mode); return TM_ERR_ARG; }
  TM_TRY(il_fields_ok(what, left, right, prec));
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  if (nrhs == 0) return TM_OK;
  const Geom g = make_geom(gg->L, 1);
  const int nblk = (nrhs + kIlRows - 1) / kIlRows;
  const int nchunk = (g.V3h + kLcChunk - 1) / kLcChunk;
  if ((long)nblk * nchunk > 0x7fffffffL || 2 * g.L[3] > 65535) {
    set_error("%s: lattice too large for the grid", what);
    return TM_ERR_ARG;
  }
  const cudaStream_t s = (cudaStream_t)strm;
  double* scratch = nullptr;
  TM_TRY(dev_alloc((void**)&scratch, sizeof(double) * 32 * (size_t)nrhs * g.L[3] * 2 * nchunk, s,
                   "contraction scratch"));
  const dim3 grid((unsigned)(nblk * nchunk), (unsigned)(2 * g.L[3]));
  tm_status_t st;
  {
    TraceScope tr(s, prec == TM_PREC_F16 ? "local.f16il" : "local.bf16il", 2.0 * 24.0 * 2.0 * 2.0 * g.Vh, 0.0,
                  nrhs);
    const unsigned* l = static_cast<const unsigned*>(left);
    const unsigned* r = static_cast<const unsigned*>(right);
    if (prec == TM_PREC_F16)
      local_il_kernel<__half><<<grid, kLcWarps * 32, 0, s>>>(g, l, r, nrhs, nblk, nchunk, right_g5 != 0, scratch);
    else
      local_il_kernel<__nv_bfloat16><<<grid, kLcWarps * 32, 0, s>>>(g, l, r, nrhs, nblk, nchunk, right_g5 != 0,
                                                                    scratch);
    count_launch();
    st = check_launch(what);
  }
  if (st == TM_OK) st = local_final(scratch, nchunk, g, nrhs, mode != TM_LOOP_STD, out, s);
  dev_free(scratch, s);
  return st;
}

extern "C" tm_status_t loop_contract_oneD_il(tm_op_t* op, const void* left, const void* right, tm_prec_t prec,
                                             int nrhs, tm_loop_mode_t mode, int right_g5, double* out,
                                             tm_stream_t strm) {
  const char* what = "loop_contract_oneD_il";
  if (!op || !left || !right || !out || nrhs < 0) { set_error("%s: null argument", what); return TM_ERR_ARG; }
  if (!valid_mode_il(mode)) { set_error("%s: unknown mode %d", what, (int)mode); return TM_ERR_ARG; }
  TM_TRY(il_fields_ok(what, left, right, prec));
  if (!op->links_il[prec]) {
    set_error("%s: needs the 18-real 16-bit links (recon 18 or 0)", what);
    return TM_ERR_UNSUPPORTED;
  }
  if (nrhs == 0) return TM_OK;
  const Geom& g = op->g;
  const int nblk = (nrhs + kIlRows - 1) / kIlRows;
  const int nchunk = (g.V3h + kOdChunk - 1) / kOdChunk;
  if ((long)nblk * nchunk > 0x7fffffffL || 2 * g.L[3] > 65535) {
    set_error("%s: lattice too large for the grid", what);
    return TM_ERR_ARG;
  }
  const cudaStream_t s = (cudaStream_t)strm;
  double* scratch = nullptr;
  TM_TRY(dev_alloc((void**)&scratch, sizeof(double) * 128 * (size_t)nrhs * g.L[3] * 2 * nchunk, s,
                   "contraction scratch"));
  OdArgs a;
  a.g = g;
  a.links_il = op->links_il[prec];
  a.err = op->il_err;
  a.L = static_cast<const unsigned char*>(left);
  a.R = static_cast<const unsigned char*>(right);
  a.partial = scratch;
  a.nrhs = nrhs;
  a.nblk = nblk;
  a.nchunk = nchunk;
  a.right_g5 = right_g5 != 0;
  const dim3 grid((unsigned)(nblk * nchunk), (unsigned)(2 * g.L[3]));
  if ((size_t)nblk * 2 * g.Vh >= ((size_t)1 << 31) || (size_t)g.Vh * 8 >= ((size_t)1 << 31)) {
    set_error("%s: lattice too large for the interleaved kernel (rows >= 2^31)", what);
    dev_free(scratch, s);
    return TM_ERR_UNSUPPORTED;
  }
  // R's rows (768 bytes per site) and the backward links' rows (48 bytes
  // per site and direction) as tensors of the gather4 copies
  CUtensorMap tmr, tlk;
  tm_status_t mst = il_row_map(&tmr, right, kIlSiteBytes / 4, (size_t)nblk * 2 * g.Vh);
  if (mst == TM_OK) mst = il_row_map(&tlk, a.links_il, kIlLinkBytes / 4, (size_t)g.Vh * 8);
  if (mst != TM_OK) {
    dev_free(scratch, s);
    return mst;
  }
  tm_status_t st;
  {
    // algorithmic bytes: both fields once (16 systems per 768-byte site) and
    // the links once per site (4 x 18 16-bit reals)
    TraceScope tr(s, prec == TM_PREC_F16 ? "oneD.f16il" : "oneD.bf16il", 2.0 * 24.0 * 2.0 * 2.0 * g.Vh,
                  4.0 * 18.0 * 2.0 * 2.0 * g.Vh, nrhs);
    if (prec == TM_PREC_F16)
      oneD_il_kernel<__half><<<grid, kOdWarps * 32, OdStage::kSmem, s>>>(a, tmr, tlk);
    else
      oneD_il_kernel<__nv_bfloat16><<<grid, kOdWarps * 32, OdStage::kSmem, s>>>(a, tmr, tlk);
    count_launch();
    st = check_launch(what);
  }
  if (st == TM_OK) st = oned_final(scratch, nchunk, g, nrhs, mode != TM_LOOP_STD, out, s);
  dev_free(scratch, s);
  return st;
}
