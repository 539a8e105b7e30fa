// FP16/BF16 Dslash on the tensor cores, on the system-interleaved field
// layout IL16 (il_core.cuh: 16 systems per block, 768 contiguous bytes per
// site, systems j and j + 8 in one 8-byte pair of slots).
//
// Every hop of a site is a small dense contraction over the 16 systems: with
// the spin projection h_s = psi_s + SGN i^ak psi_{2+ac} (s = 0, 1; the upper
// rows of (1 + SGN g_mu), DeGrand-Rossi basis) of the neighbour,
//   upper spins  out_s     += W_f h_f,s + W_b h_b,s
//   lower spins  out_{2+r} += SF i^bk_r W_f h_f,bc_r + SB i^bk_r W_b h_b,bc_r
// (W_f = U_mu(x), W_b = U_mu(x - mu)^dag, SF / SB the forward / backward
// projection signs, B_mu the lower-left block of g_mu).  One
// mma.sync.m16n8k16 (FP32 accumulation) per output spin and direction takes
//   A[system][(hop, colour, re/im)] = the projected words h (rows = systems),
//   B[(hop, colour, re/im)][(colour', re/im)] = the real form of the phased
//     links, forward hop in k = 0..7 and backward hop in k = 8..15,
// so the forward and backward hops of a direction are one product and the
// accumulators stay in registers across the four directions: 16 MMAs per
// site for 16 systems.  Lane (g, t) of a warp holds A rows g and g + 8 at
// colour t (one 8-byte load per spin and hop from the staged site), B column
// g (output colour g/2, part g&1) at colour t (one link word per hop,
// rotated by a lane-dependent phase so that every B word is a fixed swap or
// sign flip of it), and D rows g, g + 8 at output colour t: exactly the words
// it stores in the epilogue.
//
// A block of four warps takes 64 consecutive sites of one parity and one
// block of systems, warp q the sites q, q + 4, ..., q + 60; blocks are
// dispatched in site order with the systems' blocks fastest, so the sites in
// flight at one time are few and adjacent and their neighbours meet in L2.
// Each warp stages every site's neighbours and links in shared memory with
// bulk asynchronous copies (below), one site ahead of the one it computes.
// The block writes one partial sum per system and 32 sites (FP32 per warp,
// then FP64 over the lanes and the warps in a fixed order), in the per-warp
// layout of the CUDA-core kernel.  A system's result depends only on its own
// MMA row: rows do not mix in the products, and the per-lane sums run in a
// fixed order, whatever the other systems of the block are.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>

#include <cudaTypedefs.h>

#include "il_core.cuh"

namespace tml {

constexpr int kIlWarps = 4;   // warps per block

static std::atomic<int> g_il_on{-1};

bool cg_il_on() {
  int v = g_il_on.load();
  if (v < 0) {
    const char* e = getenv("TM_CG_IL");
    v = (e && e[0] == '0') ? 0 : 1;
    g_il_on.store(v);
  }
  return v != 0;
}

size_t il_bytes(const Geom& g, int nrhs) {
  const size_t nblk = (size_t)((nrhs + kIlRows - 1) / kIlRows);
  return nblk * 2 * (size_t)g.Vh * 12 * kIlRows * 4;
}


// A-side phases: the DeGrand-Rossi gamma_mu = [[0, A_mu], [B_mu, 0]] as
// (column, i^k) per row of A_mu and B_mu
template <int MU> struct IlG;
template <> struct IlG<0> { static constexpr int ac0 = 1, ak0 = 1, ac1 = 0, ak1 = 1, bc0 = 1, bk0 = 3, bc1 = 0, bk1 = 3; };
template <> struct IlG<1> { static constexpr int ac0 = 1, ak0 = 2, ac1 = 0, ak1 = 0, bc0 = 1, bk0 = 0, bc1 = 0, bk1 = 2; };
template <> struct IlG<2> { static constexpr int ac0 = 0, ak0 = 1, ac1 = 1, ak1 = 3, bc0 = 0, bk0 = 3, bc1 = 1, bk1 = 1; };
template <> struct IlG<3> { static constexpr int ac0 = 0, ak0 = 0, ac1 = 1, ak1 = 0, bc0 = 0, bk0 = 0, bc1 = 1, bk1 = 0; };

struct IlArgs {
  Geom g;
  const void* links_il;   // links in the site-major layout [par][cb][mu][12 words]
  int* err;               // set to 1 when a staging wait gave up
  const uint2* in;
  uint2* out;
  const uint2* cfield;    // centre field (null: in)
  const uint2* p;
  uint2* x;
  uint2* r;
  const uint2* b;
  const int* active;
  const double* alpha;
  double* partial;
  int* trace_count;
  int nrhs, nblk, parity, nwarp;
  int centre, out_inv;
  float nu, shop, inv, sinv;  // sinv = shop * inv
};

// per-lane constants of a warp
struct IlLane {
  int gq, tq;
  bool ld;         // lane loads spinor words (colour t < 3)
  // lane phase of the link words: swap halves on odd columns; lanes t = 3
  // (B rows of colour 3) select zero bytes
  unsigned psel;
  // lane phase (odd columns: forward words times -i, backward words times
  // +i) combined with the fixed sign flips of the four B words: forward
  // conj(u) for the upper spins, SF-signed for the lower ones; backward u,
  // SB-signed
  unsigned fup, fm, bup, bm;
};


// Lower-spin accumulators by phase class.  Lower spin 2 + r receives, from
// direction mu, i^bk_r(mu) (SF W_f h_f + SB W_b h_b)_bc_r(mu): one product per
// (r, mu) with the un-phased B = [SF U_f; SB U_b^dag], accumulated into the
// quad of its phase; the epilogue multiplies each quad by its phase (a swap
// and sign of FP32 values) and adds.  In the DeGrand-Rossi basis r = 0 meets
// the phases i^3, i^0 and r = 1 all four.
__host__ __device__ constexpr int il_quad(int r, int k) {
  return r == 0 ? (k == 3 ? 0 : 1) : (k == 3 ? 2 : k == 2 ? 3 : k == 1 ? 4 : 5);
}

// The direction whose product reaches a phase quad first (directions run 0..3)
__host__ __device__ constexpr int il_quad_first(int q) {
  int first = 4;
  for (int mu = 3; mu >= 0; --mu) {
    const int k0 = mu == 0 ? IlG<0>::bk0 : mu == 1 ? IlG<1>::bk0 : mu == 2 ? IlG<2>::bk0 : IlG<3>::bk0;
    const int k1 = mu == 0 ? IlG<0>::bk1 : mu == 1 ? IlG<1>::bk1 : mu == 2 ? IlG<2>::bk1 : IlG<3>::bk1;
    if (il_quad(0, k0) == q || il_quad(1, k1) == q) first = mu;
  }
  return first;
}
static_assert(il_quad_first(0) < 4 && il_quad_first(1) < 4 && il_quad_first(2) < 4 && il_quad_first(3) < 4 &&
                  il_quad_first(4) < 4 && il_quad_first(5) < 4,
              "every phase quad receives a product");

// One direction: both hops of 16 systems into the upper-spin accumulators
// up (spins 0, 1) and the lower-spin phase quads q, from the loaded neighbour
// words pf / pb (spins 0..3, systems g and g + 8) and link words uf / ub;
// negf / negb the antiperiodic signs (0 or 0x80008000).
template <class S, int MU, int SF>
__device__ __forceinline__ void il_dir(float (&up)[2][4], float (&q)[6][4], const IlLane& l, const uint2 (&pf)[4],
                                       const uint2 (&pb)[4], unsigned uf, unsigned ub, unsigned negf,
                                       unsigned negb) {
  using G = IlG<MU>;
  constexpr int SB = -SF;
  constexpr int pf2 = SF < 0 ? 2 : 0, pb2 = SB < 0 ? 2 : 0;
  // lane swap of the link words (odd columns); the lane's sign patterns and
  // the time-boundary sign follow in one logic operation per B word
  uf = __byte_perm(uf, 0u, l.psel);
  ub = __byte_perm(ub, 0u, l.psel);
  // projected words (rows g, g + 8) of the two upper spins for both hops
  const unsigned h0f0 = proj_w<G::ak0 + pf2, S>(pf[0].x, pf[2 + G::ac0].x);
  const unsigned h0f1 = proj_w<G::ak0 + pf2, S>(pf[0].y, pf[2 + G::ac0].y);
  const unsigned h0b0 = proj_w<G::ak0 + pb2, S>(pb[0].x, pb[2 + G::ac0].x);
  const unsigned h0b1 = proj_w<G::ak0 + pb2, S>(pb[0].y, pb[2 + G::ac0].y);
  const unsigned h1f0 = proj_w<G::ak1 + pf2, S>(pf[1].x, pf[2 + G::ac1].x);
  const unsigned h1f1 = proj_w<G::ak1 + pf2, S>(pf[1].y, pf[2 + G::ac1].y);
  const unsigned h1b0 = proj_w<G::ak1 + pb2, S>(pb[1].x, pb[2 + G::ac1].x);
  const unsigned h1b1 = proj_w<G::ak1 + pb2, S>(pb[1].y, pb[2 + G::ac1].y);
  // B words: [U_f; U_b^dag] (forward conj(u), backward u) and the signed
  // [SF U_f; SB U_b^dag]
  const unsigned bf_up = uf ^ l.fup ^ negf, bb_up = ub ^ l.bup ^ negb;
  const unsigned bf_m = SF < 0 ? uf ^ l.fm ^ negf : bf_up;
  const unsigned bb_m = SB < 0 ? ub ^ l.bm ^ negb : bb_up;
  // the first product into each accumulator of the site seeds it (direction 0
  // for the upper spins, il_quad_first for the quads)
  constexpr int q0 = il_quad(0, G::bk0), q1 = il_quad(1, G::bk1);
  il_mma_acc<S, (MU == 0)>(up[0], h0f0, h0f1, h0b0, h0b1, bf_up, bb_up);
  il_mma_acc<S, (MU == 0)>(up[1], h1f0, h1f1, h1b0, h1b1, bf_up, bb_up);
  if constexpr (G::bc0 == 0) il_mma_acc<S, il_quad_first(q0) == MU>(q[q0], h0f0, h0f1, h0b0, h0b1, bf_m, bb_m);
  else il_mma_acc<S, il_quad_first(q0) == MU>(q[q0], h1f0, h1f1, h1b0, h1b1, bf_m, bb_m);
  if constexpr (G::bc1 == 0) il_mma_acc<S, il_quad_first(q1) == MU>(q[q1], h0f0, h0f1, h0b0, h0b1, bf_m, bb_m);
  else il_mma_acc<S, il_quad_first(q1) == MU>(q[q1], h1f0, h1f1, h1b0, h1b1, bf_m, bb_m);
}

// store one 8-byte pair of words, only the halves of active systems
__device__ __forceinline__ void il_store(uint2* p, unsigned w0, unsigned w1, bool a0, bool a1) {
  if (a0 && a1) *p = make_uint2(w0, w1);
  else if (a0) reinterpret_cast<unsigned*>(p)[0] = w0;
  else if (a1) reinterpret_cast<unsigned*>(p)[1] = w1;
}

// ------------------------------------------------- staging (TMA, mbarrier)
// Each warp owns a ring of two stages in shared memory; a stage holds what
// the hops of one output site need: its eight neighbour sites (768 bytes
// each, copied whole), its forward links (4 directions x 48 bytes) and the
// four backward links.  Four asynchronous copies fill a stage: two tensor
// copies in gather4 mode (four neighbour sites each, rows of the field seen
// as a 2-D tensor of 768-byte rows), one bulk copy of the forward links and
// one gather4 copy of the backward links (rows of 48 bytes, one per site and
// direction).  Every lane computes the row of one neighbour or backward link
// and lane 0 issues the four copies, which complete on the stage's mbarrier;
// every lane waits on the barrier's phase before reading its words.  (Copies
// issued by several lanes at once execute one lane after another, each with
// its own operand set-up: thirteen per-lane copies per site cost about a
// quarter of the kernel's instructions.)  The copies of site m + 1 are in
// flight while site m is computed.  The words of the output site itself
// (centre, residual, solution, search direction) are read straight into
// registers, issued right after the previous site's epilogue.
constexpr int kIlGroups = 2;                     // 32-site groups per block

template <int EPI>
struct IlStage {
  static constexpr int kLinkOff = 8 * kIlSiteBytes;     // after the eight neighbours
  static constexpr int kBwdOff = kLinkOff + 256;        // tensor copies land on 128-byte boundaries
  static constexpr int kBytes = kBwdOff + 256;          // so do the stages
  static constexpr int kStages = 2;
  static constexpr int kWarpBytes = kStages * kBytes;
  static constexpr int kSmem = kIlWarps * kWarpBytes;
};


// FORM = 8 * norm + 2 * centre + out_inv: centre 0 (none), 1 (c), 2 (A c);
// out_inv: A^-1 on the result; norm: the plain output also writes |out|^2
// partial sums (the CG update and the residual always do)
constexpr int kIlNorm = 8;
template <class S, bool DAG, int EPI, int FORM>
__global__ void __launch_bounds__(kIlWarps * 32, EPI == EPI_CGUPD ? 3 : 4)
    dslash_il_kernel(const IlArgs a, const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tlk) {
  using H = H16<S>;
  constexpr int CENTRE = (FORM & 7) >> 1;
  constexpr bool INV = (FORM & 1) != 0;
  constexpr bool want_norm = EPI != EPI_OUT || (FORM & kIlNorm) != 0;
  using ST = IlStage<EPI>;
  extern __shared__ __align__(128) unsigned char il_smem[];
  __shared__ __align__(8) unsigned long long bars[kIlWarps][ST::kStages];
  __shared__ float red[kIlWarps][kIlGroups][kIlRows];
  __shared__ __align__(16) int rowbuf[kIlWarps][12];
  const Geom& g = a.g;
  const int lane = threadIdx.x & 31;
  const int wq = threadIdx.x >> 5;
  const int blk = blockIdx.x % a.nblk;
  const int rest = blockIdx.x / a.nblk;
  // the tensor copies need 128-byte aligned destinations: a block whose
  // dynamic shared memory is not (never expected) flags the error and stops
  if (smem_u32(il_smem) & 127u) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    return;
  }
  if (a.trace_count && blockIdx.x == 0 && threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < a.nrhs; ++r) n += (a.active == nullptr || a.active[r] != 0) ? 1 : 0;
    *a.trace_count = n;
  }
  // both parities: alternate them block by block (the centre reads of one are
  // the neighbour reads of the other)
  const int par = a.parity < 0 ? (rest & 1) : a.parity;
  const int cg = a.parity < 0 ? (rest >> 1) : rest;  // the block's 128-site chunk
  const int opar = par ^ 1;
  IlLane l;
  l.gq = lane >> 2;
  l.tq = lane & 3;
  const int r0 = blk * kIlRows + l.gq, r1 = r0 + 8;
  const bool act0 = r0 < a.nrhs && (a.active == nullptr || a.active[r0] != 0);
  const bool act1 = r1 < a.nrhs && (a.active == nullptr || a.active[r1] != 0);
  if (lane == 0) {
#pragma unroll
    for (int st = 0; st < ST::kStages; ++st) mbar_init(smem_u32(&bars[wq][st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kIlWarps * kIlGroups * kIlRows; i += blockDim.x) (&red[0][0][0])[i] = 0.0f;
  __syncthreads();
  const size_t Vh = (size_t)g.Vh;
  const int base = cg * (kIlGroups * 32);
  // sites of this warp: base + wq + 4 m, m = 0 .. nsite - 1
  const int left = g.Vh - base - wq;
  constexpr int kWarpSites = kIlGroups * 32 / kIlWarps;  // sites of one warp in a full block
  const int nsite = left <= 0 ? 0 : min(kWarpSites, (left + kIlWarps - 1) / kIlWarps);
  if (__any_sync(0xffffffffu, act0 || act1) && nsite > 0) {
    // lane m: the warp's site m: lex index and a mask of the hops that wrap
    // around the lattice (bit 2 mu: forward, 2 mu + 1: backward)
    int lexl = 0;
    unsigned bml = 0u;
    if (lane < nsite) {
      const Site s = site_of(g, par, base + wq + kIlWarps * lane);
      lexl = s.lex;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu)
        bml |= (s.c[mu] == g.L[mu] - 1 ? 1u : 0u) << (2 * mu) | (s.c[mu] == 0 ? 2u : 0u) << (2 * mu);
    }
    const size_t obase = ((size_t)blk * 2 + par) * Vh * kIlSiteBytes;
    // row role of this lane: lanes 0..7 the neighbour of direction lane / 2
    // (forward for even lanes), a row (blk * 2 + opar) * Vh + cb' of the
    // field; lanes 8..11 the backward link of direction lane - 8, row
    // (opar * Vh + cb') * 4 + mu of the links; cb' the neighbour's
    // checkerboard index
    const int rmu = lane < 8 ? (lane >> 1) : (lane < 12 ? lane - 8 : 0);
    const bool rbwd = lane < 8 ? (lane & 1) != 0 : true;
    // the role's hop: lex step, and the step when it wraps around
    const int rbit = 2 * rmu + (rbwd ? 1 : 0);
    const int rstep = rbwd ? -g.stride[rmu] : g.stride[rmu];
    const int rwrap = rbwd ? (g.L[rmu] - 1) * g.stride[rmu] : -(g.L[rmu] - 1) * g.stride[rmu];
    const int rrow0 = lane < 8 ? (blk * 2 + opar) * g.Vh : opar * g.Vh * 4 + rmu;
    const int rrmul = lane < 8 ? 1 : 4;
    const unsigned char* lk = reinterpret_cast<const unsigned char*>(a.links_il) + (size_t)par * Vh * kIlLinkSiteBytes;
    l.ld = l.tq < 3;
    const bool odd = (l.gq & 1) != 0;
    l.psel = l.tq == 3 ? 0x4444u : odd ? 0x1032u : 0x3210u;
    {
      constexpr int SFl = DAG ? +1 : -1;
      const unsigned pmf = odd ? 0x80000000u : 0u, pmb = odd ? 0x00008000u : 0u;
      l.fup = pmf ^ 0x80000000u;
      l.fm = SFl < 0 ? pmf ^ 0x00008000u : l.fup;
      l.bup = pmb;
      l.bm = SFl > 0 ? pmb ^ 0x80008000u : pmb;
    }
    // lane offsets in a stage: spinor words (3 s + t) * 64 + pair * 8 (pair
    // position g, XOR 4 on colour 2).  Lanes t = 3 (no colour) read the words
    // of t = 0: finite values against the zero B rows of colour 3.
    const int teff = l.tq < 3 ? l.tq : 0;
    const int woff = teff * 64 + ((teff == 2 ? l.gq ^ 4 : l.gq) * 8);
    // link words: entry (g / 2, t) forward, (t, g / 2) backward.  Every lane
    // loads a word of its direction's 48 bytes (lanes t = 3 that of t = 0,
    // zeroed by psel); lanes g = 6, 7 read pad or colour words into B
    // columns of output colour 3, which no lane stores.
    const int lf_off = (3 * (l.gq >> 1) + teff) * 4, lb_off = (3 * teff + (l.gq >> 1)) * 4;
    const float nu = a.nu, shop = a.shop, inv = a.inv, sinv = a.sinv;
    const float2 shop2 = make_float2(shop, shop);
    float al0 = 0.0f, al1 = 0.0f;
    if constexpr (EPI == EPI_CGUPD) {
      al0 = act0 ? (float)a.alpha[r0] : 0.0f;
      al1 = act1 ? (float)a.alpha[r1] : 0.0f;
    }
    const float2 pal0 = make_float2(al0, al0), pal1 = make_float2(al1, al1);
    const float2 nal0 = make_float2(-al0, -al0), nal1 = make_float2(-al1, -al1);
    unsigned char* ring = il_smem + wq * ST::kWarpBytes;
    const unsigned ring_s = smem_u32(ring);
    const unsigned bar0 = smem_u32(&bars[wq][0]);
    constexpr int SF = DAG ? +1 : -1;
    constexpr unsigned total = 8 * kIlSiteBytes + kIlLinkSiteBytes + 4 * kIlLinkBytes;
    static_assert(ST::kBwdOff % 128 == 0 && ST::kBytes % 128 == 0 && ST::kBwdOff >= ST::kLinkOff + kIlLinkSiteBytes &&
                      ST::kBytes >= ST::kBwdOff + 4 * kIlLinkBytes,
                  "stage layout");
    // the output site's own words (centre, r, x, p or b), straight into
    // registers; per-lane base pointers of the output parity, so that a site
    // adds one offset and the spins are immediate offsets
    const size_t lbase = (obase + woff) / 8;
    const uint2* cf = (a.cfield ? a.cfield : a.in) + lbase;
    const uint2* rp = (EPI == EPI_RESID ? a.b : a.r) + lbase;
    const uint2* xp = a.x + lbase;
    const uint2* pp = a.p + lbase;
    uint2* op = (EPI == EPI_CGUPD ? a.r : a.out) + lbase;
    uint2* oxp = a.x + lbase;
    uint2 cw[4], rw[4], xw[4], pw[4];
    auto fetch_site = [&](int m) {
      const unsigned w = (unsigned)(base + wq + kIlWarps * m) * (kIlSiteBytes / 8);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if constexpr (CENTRE != 0) cw[s] = cf[w + 24 * s];
        if constexpr (EPI == EPI_CGUPD) {
          rw[s] = rp[w + 24 * s];
          xw[s] = xp[w + 24 * s];
          pw[s] = pp[w + 24 * s];
        } else if constexpr (EPI == EPI_RESID) {
          rw[s] = rp[w + 24 * s];
        }
      }
    };
    // returns the site's wrap mask (the next iteration's time-boundary signs)
    auto issue = [&](int m, int st) -> unsigned {
      const int lex = __shfl_sync(0xffffffffu, lexl, m);
      const unsigned msk = __shfl_sync(0xffffffffu, bml, m);
      const int nlex = lex + (((msk >> rbit) & 1u) ? rwrap : rstep);
      if (lane < 12) rowbuf[wq][lane] = rrow0 + (nlex >> 1) * rrmul;
      const unsigned bar = bar0 + st * 8;
      // the stage was last read by this warp (generic proxy): order those reads
      // before the copies' writes (async proxy), every lane before lane 0 issues
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        const int4 q0 = *reinterpret_cast<const int4*>(&rowbuf[wq][0]);
        const int4 q1 = *reinterpret_cast<const int4*>(&rowbuf[wq][4]);
        const int4 q2 = *reinterpret_cast<const int4*>(&rowbuf[wq][8]);
        const unsigned sb = ring_s + st * ST::kBytes;
        mbar_expect_tx(bar, total);
        gather4_g2s(sb, &tin, q0.x, q0.y, q0.z, q0.w, bar);
        gather4_g2s(sb + 4 * kIlSiteBytes, &tin, q1.x, q1.y, q1.z, q1.w, bar);
        bulk_g2s(sb + ST::kLinkOff, lk + (size_t)(base + wq + kIlWarps * m) * kIlLinkSiteBytes, kIlLinkSiteBytes,
                 bar);
        gather4_g2s(sb + ST::kBwdOff, &tlk, q2.x, q2.y, q2.z, q2.w, bar);
      }
      return msk;
    };
    static_assert(ST::kStages == 2, "one site in flight while one is computed");
    unsigned mskc = issue(0, 0);
    fetch_site(0);
    float nacc0 = 0.0f, nacc1 = 0.0f;  // norms of the current 32-site group
    for (int m = 0; m < nsite; ++m) {
      const int st = m % ST::kStages;
      const unsigned mskn = m + 1 < nsite ? issue(m + 1, st ^ 1) : 0u;
      // antiperiodic time boundary: the hops that wrap in direction 3
      const unsigned bf = g.antiperiodic ? (mskc >> 6) & 3u : 0u;
      mskc = mskn;
      if (!__all_sync(0xffffffffu, il_wait(bar0 + st * 8, (unsigned)((m / ST::kStages) & 1), a.err))) {
        // a wait gave up: wait (bounded) for this warp's copies still in
        // flight (sites m .. m + kStages - 2), then stop
        for (int mm = m; mm < min(m + ST::kStages - 1, nsite); ++mm)
          il_wait(bar0 + (mm % ST::kStages) * 8, (unsigned)((mm / ST::kStages) & 1), nullptr);
        break;
      }
      const unsigned char* sd = ring + st * ST::kBytes;
      // upper spins: one accumulator pair over the four directions; lower
      // spins: the six phase quads
      float ua[2][4], qq[6][4];  // seeded by their first products
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        uint2 pf[4], pb[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          pf[s] = *reinterpret_cast<const uint2*>(sd + (2 * mu) * kIlSiteBytes + woff + 192 * s);
          pb[s] = *reinterpret_cast<const uint2*>(sd + (2 * mu + 1) * kIlSiteBytes + woff + 192 * s);
        }
        const unsigned uf = *reinterpret_cast<const unsigned*>(sd + ST::kLinkOff + mu * kIlLinkBytes + lf_off);
        const unsigned ub = *reinterpret_cast<const unsigned*>(sd + ST::kBwdOff + mu * kIlLinkBytes + lb_off);
        const unsigned negf = (mu == 3 && (bf & 1u)) ? 0x80008000u : 0u;
        const unsigned negb = (mu == 3 && (bf & 2u)) ? 0x80008000u : 0u;
        if (mu == 0) il_dir<S, 0, SF>(ua, qq, l, pf, pb, uf, ub, negf, negb);
        else if (mu == 1) il_dir<S, 1, SF>(ua, qq, l, pf, pb, uf, ub, negf, negb);
        else if (mu == 2) il_dir<S, 2, SF>(ua, qq, l, pf, pb, uf, ub, negf, negb);
        else il_dir<S, 3, SF>(ua, qq, l, pf, pb, uf, ub, negf, negb);
      }
      // epilogue: out = T_out(T_c(c) + s_hop H in), then the CG update / residual;
      // lanes t = 3 compute on the words of t = 0 and store nothing
      uint2* const ost = op + (unsigned)(base + wq + kIlWarps * m) * (kIlSiteBytes / 8);
      uint2* const xst = oxp + (unsigned)(base + wq + kIlWarps * m) * (kIlSiteBytes / 8);
      // the hopping sum of each spin (rows g, g + 8: re, im, re, im)
      float hs[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        hs[0][c] = ua[0][c];
        hs[1][c] = ua[1][c];
      }
#pragma unroll
      for (int rr = 0; rr < 4; rr += 2) {
        // spin 2: i^3 q0 + q1;  spin 3: i^3 q2 + i^2 q3 + i q4 + q5
        hs[2][rr] = __fadd_rn(qq[0][rr + 1], qq[1][rr]);
        hs[2][rr + 1] = __fsub_rn(qq[1][rr + 1], qq[0][rr]);
        hs[3][rr] = __fadd_rn(__fsub_rn(__fsub_rn(qq[2][rr + 1], qq[3][rr]), qq[4][rr + 1]), qq[5][rr]);
        hs[3][rr + 1] = __fadd_rn(__fsub_rn(qq[4][rr], __fadd_rn(qq[2][rr], qq[3][rr + 1])), qq[5][rr + 1]);
      }
      // (re, im) pairs in packed FP32x2 operations where both parts take the
      // same factor (each lane an ordinary round-to-nearest FMA)
      float2 n0 = make_float2(0.0f, 0.0f), n1 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float tw = s < 2 ? nu : -nu;  // gamma_5 = diag(1, 1, -1, -1)
        const float h0r = hs[s][0], h0i = hs[s][1], h1r = hs[s][2], h1i = hs[s][3];
        float2 o0, o1;
        if constexpr (CENTRE != 0) {
          float2 c0 = H::to_f2(cw[s].x), c1 = H::to_f2(cw[s].y);
          if constexpr (CENTRE == 2) {
            c0 = make_float2(__fmaf_rn(-tw, c0.y, c0.x), __fmaf_rn(tw, c0.x, c0.y));
            c1 = make_float2(__fmaf_rn(-tw, c1.y, c1.x), __fmaf_rn(tw, c1.x, c1.y));
          }
          o0 = __ffma2_rn(shop2, make_float2(h0r, h0i), c0);
          o1 = __ffma2_rn(shop2, make_float2(h1r, h1i), c1);
        } else if constexpr (INV) {
          // A^-1 s_hop h = (s_hop / (1 + nu^2)) (h - i nu g5 h): one scale
          o0 = make_float2(__fmul_rn(sinv, __fmaf_rn(tw, h0i, h0r)), __fmul_rn(sinv, __fmaf_rn(-tw, h0r, h0i)));
          o1 = make_float2(__fmul_rn(sinv, __fmaf_rn(tw, h1i, h1r)), __fmul_rn(sinv, __fmaf_rn(-tw, h1r, h1i)));
        } else {
          o0 = make_float2(__fmul_rn(shop, h0r), __fmul_rn(shop, h0i));
          o1 = make_float2(__fmul_rn(shop, h1r), __fmul_rn(shop, h1i));
        }
        if constexpr (INV && CENTRE != 0) {  // A^-1 v = (v - i nu g5 v) / (1 + nu^2)
          o0 = make_float2(__fmul_rn(inv, __fmaf_rn(tw, o0.y, o0.x)), __fmul_rn(inv, __fmaf_rn(-tw, o0.x, o0.y)));
          o1 = make_float2(__fmul_rn(inv, __fmaf_rn(tw, o1.y, o1.x)), __fmul_rn(inv, __fmaf_rn(-tw, o1.x, o1.y)));
        }
        if constexpr (EPI == EPI_OUT) {
          // every system's output (inactive and padding systems get the
          // operator applied to their own unchanged input)
          if (l.ld) ost[24 * s] = make_uint2(H::pack(o0.x, o0.y), H::pack(o1.x, o1.y));
          if constexpr (want_norm) {
            n0 = __ffma2_rn(o0, o0, n0);
            n1 = __ffma2_rn(o1, o1, n1);
          }
        } else if constexpr (EPI == EPI_CGUPD) {
          // r and x of inactive systems keep their bits
          float2 q0 = H::to_f2(rw[s].x), q1 = H::to_f2(rw[s].y);
          q0 = __ffma2_rn(nal0, o0, q0);
          q1 = __ffma2_rn(nal1, o1, q1);
          const uint2 rn = make_uint2(act0 ? H::pack(q0.x, q0.y) : rw[s].x, act1 ? H::pack(q1.x, q1.y) : rw[s].y);
          n0 = __ffma2_rn(q0, q0, n0);
          n1 = __ffma2_rn(q1, q1, n1);
          const float2 x0 = __ffma2_rn(pal0, H::to_f2(pw[s].x), H::to_f2(xw[s].x));
          const float2 x1 = __ffma2_rn(pal1, H::to_f2(pw[s].y), H::to_f2(xw[s].y));
          const uint2 xn = make_uint2(act0 ? H::pack(x0.x, x0.y) : xw[s].x, act1 ? H::pack(x1.x, x1.y) : xw[s].y);
          if (l.ld) {
            ost[24 * s] = rn;
            xst[24 * s] = xn;
          }
        } else {  // EPI_RESID: out = b - D in
          const float2 m1 = make_float2(-1.0f, -1.0f);  // b - o, rounded once as by a subtraction
          o0 = __ffma2_rn(m1, o0, H::to_f2(rw[s].x));
          o1 = __ffma2_rn(m1, o1, H::to_f2(rw[s].y));
          if (l.ld) ost[24 * s] = make_uint2(H::pack(o0.x, o0.y), H::pack(o1.x, o1.y));
          n0 = __ffma2_rn(o0, o0, n0);
          n1 = __ffma2_rn(o1, o1, n1);
        }
      }
      if constexpr (want_norm) {
        if (l.ld && act0) nacc0 = __fadd_rn(nacc0, __fadd_rn(n0.x, n0.y));
        if (l.ld && act1) nacc1 = __fadd_rn(nacc1, __fadd_rn(n1.x, n1.y));
        // site base + wq + 4 m lies in 32-site group m / 8: flush at the group's end
        static_assert(kIlWarps == 4, "a warp takes 8 sites of each 32-site group");
        if ((m & 7) == 7 || m == nsite - 1) {
          nacc0 = __fadd_rn(nacc0, __shfl_xor_sync(0xffffffffu, nacc0, 1));
          nacc0 = __fadd_rn(nacc0, __shfl_xor_sync(0xffffffffu, nacc0, 2));
          nacc1 = __fadd_rn(nacc1, __shfl_xor_sync(0xffffffffu, nacc1, 1));
          nacc1 = __fadd_rn(nacc1, __shfl_xor_sync(0xffffffffu, nacc1, 2));
          if (l.tq == 0) {
            red[wq][m >> 3][l.gq] = nacc0;
            red[wq][m >> 3][l.gq + 8] = nacc1;
          }
          nacc0 = nacc1 = 0.0f;
        }
      }
      if (m + 1 < nsite) fetch_site(m + 1);
      __syncwarp();  // every lane is done with the stage before it is refilled
    }
  }
  if constexpr (want_norm) {
    // the warps' sums of each 32-site group, fixed order
    __syncthreads();
    if (threadIdx.x < kIlGroups * kIlRows) {
      const int j = threadIdx.x / kIlRows, sy = threadIdx.x % kIlRows;
      const int r = blk * kIlRows + sy;
      const int grp = cg * kIlGroups + j;
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < kIlWarps; ++q) t += (double)red[q][j][sy];
      if (r < a.nrhs && grp < a.nwarp) a.partial[((size_t)r * 2 + par) * a.nwarp + grp] = t;
    }
  }
}

template <class S, bool DAG, int EPI, int FORM>
static tm_status_t il_prepare_t() {
  const cudaError_t e = cudaFuncSetAttribute(dslash_il_kernel<S, DAG, EPI, FORM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, IlStage<EPI>::kSmem);
  if (e != cudaSuccess) {
    set_error("dslash_il: shared-memory limit: %s", cudaGetErrorString(e));
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

// the instantiated forms: every (centre, A^-1) combination for the plain
// output, the twisted centre without A^-1 with norms (the solver's M) and
// for the CG update and the residual
template <class S, bool DAG>
static tm_status_t il_prepare_sd() {
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, 0>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, 1>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, 2>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, 3>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, 4>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, 5>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_OUT, kIlNorm + 4>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_CGUPD, 4>()));
  TM_TRY((il_prepare_t<S, DAG, EPI_RESID, 4>()));
  return TM_OK;
}

// raise the dynamic shared-memory limit of every instantiation (once)
tm_status_t il_prepare() {
  static std::mutex mu;
  static bool done = false;
  std::lock_guard<std::mutex> lk(mu);
  if (done) return TM_OK;
  TM_TRY((il_prepare_sd<__half, false>()));
  TM_TRY((il_prepare_sd<__half, true>()));
  TM_TRY((il_prepare_sd<__nv_bfloat16, false>()));
  TM_TRY((il_prepare_sd<__nv_bfloat16, true>()));
  done = true;
  return TM_OK;
}

// ------------------------------------------------ tensor maps (host)
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 il_encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// rows of row_words 4-byte words at base as a 2-D tensor whose box is one
// whole row (the gather4 copies take four rows at a time)
tm_status_t il_row_map(CUtensorMap* m, const void* base, unsigned row_words, size_t rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = il_encode_fn();
  if (!enc) {
    set_error("dslash_il: cuTensorMapEncodeTiled is not available");
    return TM_ERR_CUDA;
  }
  const cuuint64_t dim[2] = {row_words, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)row_words * 4};
  const cuuint32_t box[2] = {row_words, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dim, stride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("dslash_il: tensor map encoding failed (%d)", (int)r);
    return TM_ERR_CUDA;
  }
  return TM_OK;
}

template <class S, bool DAG, int EPI>
static tm_status_t il_launch_t(const tm_op* op, const DslashCall& c, cudaStream_t st, tm_prec_t prec) {
  IlArgs a{};
  const Geom& g = op->g;
  a.g = g;
  a.links_il = op->links_il[prec];
  a.err = op->il_err;
  a.in = static_cast<const uint2*>(c.in);
  a.out = static_cast<uint2*>(c.out);
  a.cfield = static_cast<const uint2*>(c.cfield);
  a.p = static_cast<const uint2*>(c.p);
  a.x = static_cast<uint2*>(c.x);
  a.r = static_cast<uint2*>(c.r);
  a.b = static_cast<const uint2*>(c.b);
  a.active = c.active;
  a.alpha = c.alpha;
  a.partial = c.partial;
  a.nrhs = c.nrhs;
  a.nblk = (c.nrhs + kIlRows - 1) / kIlRows;
  a.parity = c.parity;
  a.nwarp = nwarp_of(g);
  double nu, hop;
  if (c.custom) {
    nu = c.nu;
    hop = c.hop_scale;
    a.centre = c.centre;
    a.out_inv = c.out_inv ? 1 : 0;
  } else {
    nu = c.mu_zero ? 0.0 : (DAG ? -2.0 * op->kappa * op->mu : 2.0 * op->kappa * op->mu);
    hop = -op->kappa;
    a.centre = 2;
    a.cfield = nullptr;
    a.out_inv = 0;
  }
  a.nu = (float)nu;
  a.shop = (float)hop;
  a.inv = (float)(1.0 / (1.0 + nu * nu));
  a.sinv = (float)(hop / (1.0 + nu * nu));
  // every field the bulk copies read must sit on a 16-byte boundary
  const void* ptrs[6] = {a.in, a.cfield, a.p, a.x, a.r, a.b};
  for (const void* q : ptrs)
    if (q && ((uintptr_t)q & 15u)) {
      set_error("dslash_il: fields must be 16-byte aligned");
      return TM_ERR_ARG;
    }
  if ((size_t)g.Vh * kIlSiteBytes / 8 >= (size_t)0xffffffffu || (size_t)a.nblk * 2 * g.Vh >= ((size_t)1 << 31) ||
      (size_t)g.Vh * 8 >= ((size_t)1 << 31)) {
    set_error("dslash_il: lattice too large for the interleaved kernel (V/2 * 96 >= 2^32 or rows >= 2^31)");
    return TM_ERR_UNSUPPORTED;
  }
  // the neighbours' rows (768 bytes per site) and the backward links' rows
  // (48 bytes per site and direction) as tensors of the gather4 copies
  CUtensorMap tin, tlk;
  TM_TRY(il_row_map(&tin, a.in, kIlSiteBytes / 4, (size_t)a.nblk * 2 * g.Vh));
  TM_TRY(il_row_map(&tlk, a.links_il, kIlLinkBytes / 4, (size_t)g.Vh * 8));
  const int npar = c.parity < 0 ? 2 : 1;
  const long chunks = ((long)g.Vh + kIlGroups * 32 - 1) / (kIlGroups * 32);
  const long blocks = (long)a.nblk * npar * chunks;  // one block per 128 sites and 16 systems
  if (blocks > 0x7fffffffL) {
    set_error("dslash_il: launch grid too large");
    return TM_ERR_ARG;
  }
  TM_TRY(il_prepare());
  static const char* const kNames[2][3] = {{"dslash.f16il.out", "dslash.f16il.cgupd", "dslash.f16il.resid"},
                                           {"dslash.bf16il.out", "dslash.bf16il.cgupd", "dslash.bf16il.resid"}};
  const char* name = kNames[std::is_same<S, __half>::value ? 0 : 1][EPI];
  // algorithmic bytes as for the CUDA-core kernel: per active system the
  // neighbour field (one parity per output parity), the centre field unless it
  // is the input read on both parities, the epilogue's streams; per launch the
  // links of all sites (18 reals)
  const double e = 2.0;
  const double out_sites = (double)npar * g.Vh;
  const bool centre_is_in = a.cfield == nullptr || a.cfield == a.in;
  const int centre = (a.centre != 0 && !(c.parity < 0 && centre_is_in)) ? 1 : 0;
  const int epi_streams = EPI == EPI_OUT ? 1 : (EPI == EPI_CGUPD ? 5 : 2);
  const double per_rhs = out_sites * 24.0 * e * (1 + centre + epi_streams);
  const double fixed = 4.0 * 2.0 * g.Vh * 18.0 * e;
  const double site_flops = 1320.0 + 48.0 + (a.centre == 2 ? 48.0 : 0.0) + (a.out_inv ? 72.0 : 0.0) +
                            (EPI == EPI_CGUPD ? 144.0 : EPI == EPI_RESID ? 72.0 : (a.partial ? 48.0 : 0.0));
  const int form = 2 * a.centre + a.out_inv;
  if (EPI != EPI_OUT && form != 4) {
    set_error("dslash_il: the CG update and residual forms need the twisted centre without A^-1");
    return TM_ERR_UNSUPPORTED;
  }
  if (EPI == EPI_OUT && a.partial && form != 4) {
    set_error("dslash_il: norms of the plain output only with the twisted centre without A^-1");
    return TM_ERR_UNSUPPORTED;
  }
  cudaEvent_t ev = nullptr;
  a.trace_count = trace_begin(st, &ev);
  const dim3 grid((unsigned)blocks);
  constexpr int kT = kIlWarps * 32, kM = IlStage<EPI>::kSmem;
  if constexpr (EPI == EPI_OUT) {
    switch (form) {
      case 0: dslash_il_kernel<S, DAG, EPI, 0><<<grid, kT, kM, st>>>(a, tin, tlk); break;
      case 1: dslash_il_kernel<S, DAG, EPI, 1><<<grid, kT, kM, st>>>(a, tin, tlk); break;
      case 2: dslash_il_kernel<S, DAG, EPI, 2><<<grid, kT, kM, st>>>(a, tin, tlk); break;
      case 3: dslash_il_kernel<S, DAG, EPI, 3><<<grid, kT, kM, st>>>(a, tin, tlk); break;
      case 4:
        if (a.partial) dslash_il_kernel<S, DAG, EPI, kIlNorm + 4><<<grid, kT, kM, st>>>(a, tin, tlk);
        else dslash_il_kernel<S, DAG, EPI, 4><<<grid, kT, kM, st>>>(a, tin, tlk);
        break;
      default: dslash_il_kernel<S, DAG, EPI, 5><<<grid, kT, kM, st>>>(a, tin, tlk); break;
    }
  } else {
    dslash_il_kernel<S, DAG, EPI, 4><<<grid, kT, kM, st>>>(a, tin, tlk);
  }
  count_launch();
  trace_end(st, name, ev, a.trace_count, per_rhs, fixed, 0, out_sites * site_flops);
  return check_launch("dslash_il");
}

template <class S>
static tm_status_t il_launch_s(const tm_op* op, const DslashCall& c, cudaStream_t st, tm_prec_t prec) {
  if (c.dagger) {
    switch (c.epi) {
      case EPI_OUT: return il_launch_t<S, true, EPI_OUT>(op, c, st, prec);
      case EPI_CGUPD: return il_launch_t<S, true, EPI_CGUPD>(op, c, st, prec);
      default: return il_launch_t<S, true, EPI_RESID>(op, c, st, prec);
    }
  }
  switch (c.epi) {
    case EPI_OUT: return il_launch_t<S, false, EPI_OUT>(op, c, st, prec);
    case EPI_CGUPD: return il_launch_t<S, false, EPI_CGUPD>(op, c, st, prec);
    default: return il_launch_t<S, false, EPI_RESID>(op, c, st, prec);
  }
}

tm_status_t dslash_il_dispatch(const tm_op* op, tm_prec_t prec, const DslashCall& c, cudaStream_t s) {
  if (prec != TM_PREC_F16 && prec != TM_PREC_BF16) {
    set_error("dslash_il: the interleaved layout holds F16 or BF16 fields");
    return TM_ERR_ARG;
  }
  if (op->recon_p[prec] != 18 || !op->links_il[prec] || !op->il_err) {
    set_error("dslash_il: needs the 18-real 16-bit link copy (recon 18 or 0)");
    return TM_ERR_UNSUPPORTED;
  }
  if (c.g5_out || (c.custom && (c.centre < 0 || c.centre > 2))) {
    set_error("dslash_il: unsupported output form");
    return TM_ERR_UNSUPPORTED;
  }
  if (c.nrhs <= 0) return TM_OK;
  return prec == TM_PREC_F16 ? il_launch_s<__half>(op, c, s, prec) : il_launch_s<__nv_bfloat16>(op, c, s, prec);
}

// ------------------------------------------------ site-major links
// [mu][par][unit][cb] (three 16-byte units of the 18-real 16-bit copy, the
// last word pair zero) -> [par][cb][mu][unit]: one site's forward links are
// 192 contiguous bytes, one direction 48.
size_t il_link_bytes(const Geom& g) { return 2 * (size_t)g.Vh * kIlLinkSiteBytes; }

__global__ void il_pack_links_kernel(size_t Vh, uint4* __restrict__ out, const uint4* __restrict__ in) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (par, cb, mu)
  if (i >= 2 * Vh * 4) return;
  const int mu = (int)(i & 3);
  const size_t pc = i >> 2;  // par * Vh + cb
  const int par = (int)(pc / Vh);
  const size_t cb = pc % Vh;
#pragma unroll
  for (int u = 0; u < 3; ++u) out[i * 3 + u] = in[((size_t)(mu * 2 + par) * 3 + u) * Vh + cb];
}

tm_status_t il_pack_links(const Geom& g, void* out, const void* links18, cudaStream_t s) {
  const size_t n = 2 * (size_t)g.Vh * 4;
  il_pack_links_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((size_t)g.Vh, static_cast<uint4*>(out),
                                                                    static_cast<const uint4*>(links18));
  count_launch();
  return check_launch("interleaved link packing");
}

// ------------------------------------------------- layout conversions
// 32 sites x 16 systems per block of 512 threads, through shared memory:
// reads of the standard layout (warp = system, lane = site: 512 contiguous
// bytes per chunk) and writes of the interleaved rows (thread = 4-byte slot
// of 32 consecutive 64-byte rows) are both coalesced.  The 16-bit formats
// move as bytes; slots of systems >= nrhs are written as zero.
constexpr int kIlCvSites = 32;

// system (0..15 in its block) held by slot 0..15 of row k of a site
__device__ __forceinline__ int il_system(int k, int slot) {
  const int pos = (slot >> 1) ^ (k % 3 == 2 ? 4 : 0);
  return (slot & 1) ? pos + 8 : pos;
}

__global__ void __launch_bounds__(512) il_from_std_kernel(Geom g, uint4* __restrict__ out,
                                                          const uint4* __restrict__ in, int nrhs) {
  __shared__ unsigned sm[kIlRows][kIlCvSites + 1][13];
  const int blk = blockIdx.z, par = blockIdx.y;
  const int cb0 = blockIdx.x * kIlCvSites;
  const int tid = threadIdx.x;
  const size_t Vh = (size_t)g.Vh;
  {
    const int s = tid >> 5, j = tid & 31;
    const int r = blk * kIlRows + s;
    const int cb = cb0 + j;
    uint4 q[3] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
    if (r < nrhs && cb < g.Vh) {
#pragma unroll
      for (int c = 0; c < 3; ++c) q[c] = in[(((size_t)r * 2 + par) * 3 + c) * Vh + cb];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sm[s][j][4 * c] = q[c].x;
      sm[s][j][4 * c + 1] = q[c].y;
      sm[s][j][4 * c + 2] = q[c].z;
      sm[s][j][4 * c + 3] = q[c].w;
    }
  }
  __syncthreads();
  // the block's 32 sites are 32 x 192 contiguous words of the interleaved field
  unsigned* o = reinterpret_cast<unsigned*>(out) + (((size_t)blk * 2 + par) * Vh + cb0) * 192;
#pragma unroll
  for (int m = 0; m < 12; ++m) {
    const int w = tid + 512 * m;
    const int j = w / 192, k = (w % 192) >> 4, slot = w & 15;
    const int s = il_system(k, slot);
    if (cb0 + j < g.Vh) o[w] = sm[s][j][k];
  }
}

__global__ void __launch_bounds__(512) il_to_std_kernel(Geom g, uint4* __restrict__ out,
                                                        const uint4* __restrict__ in, int nrhs) {
  __shared__ unsigned sm[kIlRows][kIlCvSites + 1][13];
  const int blk = blockIdx.z, par = blockIdx.y;
  const int cb0 = blockIdx.x * kIlCvSites;
  const int tid = threadIdx.x;
  const size_t Vh = (size_t)g.Vh;
  {
    const unsigned* ip = reinterpret_cast<const unsigned*>(in) + (((size_t)blk * 2 + par) * Vh + cb0) * 192;
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      const int w = tid + 512 * m;
      const int j = w / 192, k = (w % 192) >> 4, slot = w & 15;
      const int s = il_system(k, slot);
      sm[s][j][k] = cb0 + j < g.Vh ? ip[w] : 0u;
    }
  }
  __syncthreads();
  const int s = tid >> 5, j = tid & 31;
  const int r = blk * kIlRows + s;
  const int cb = cb0 + j;
  if (r >= nrhs || cb >= g.Vh) return;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    out[(((size_t)r * 2 + par) * 3 + c) * Vh + cb] =
        make_uint4(sm[s][j][4 * c], sm[s][j][4 * c + 1], sm[s][j][4 * c + 2], sm[s][j][4 * c + 3]);
}

tm_status_t il_convert(const Geom& g, void* out, const void* in, int nrhs, bool to_il, cudaStream_t s) {
  if (nrhs <= 0) return TM_OK;
  const int nblk = (nrhs + kIlRows - 1) / kIlRows;
  if (nblk > 65535) {
    set_error("interleaved layout: too many systems (%d)", nrhs);
    return TM_ERR_ARG;
  }
  const dim3 grid((unsigned)((g.Vh + kIlCvSites - 1) / kIlCvSites), 2, (unsigned)nblk);
  if (to_il)
    il_from_std_kernel<<<grid, 512, 0, s>>>(g, static_cast<uint4*>(out), static_cast<const uint4*>(in), nrhs);
  else
    il_to_std_kernel<<<grid, 512, 0, s>>>(g, static_cast<uint4*>(out), static_cast<const uint4*>(in), nrhs);
  count_launch();
  return check_launch("interleaved layout conversion");
}

// ------------------------------------------------ solver BLAS on IL16
// p = r + beta p for the active systems on parities par0 .. par0 + npar - 1.
// One plane (block of systems, parity) per grid row; a thread takes 16-byte
// words (pair positions 2q, 2q + 1 of a row), the systems' beta and flags
// come from shared memory.
template <class S>
__global__ void il_xpay_kernel(uint4* p, const uint4* r, const double* beta, const int* active, int nrhs,
                               int par0, int npar, unsigned plane_u4) {
  using H = H16<S>;
  __shared__ float sb[kIlRows];
  __shared__ int sa[kIlRows];
  const int blk = blockIdx.y / npar, pi = blockIdx.y % npar;
  if (threadIdx.x < kIlRows) {
    const int rr = blk * kIlRows + threadIdx.x;
    const int on = rr < nrhs && active[rr] != 0;
    sa[threadIdx.x] = on;
    sb[threadIdx.x] = on ? (float)beta[rr] : 0.0f;
  }
  __syncthreads();
  uint4* pp = p + ((size_t)blk * 2 + par0 + pi) * plane_u4;
  const uint4* rp = r + ((size_t)blk * 2 + par0 + pi) * plane_u4;
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < plane_u4; j += gridDim.x * blockDim.x) {
    const unsigned k = (j >> 2) % 12u;  // row j / 4 = site * 12 + k
    const int sw = k % 3u == 2u ? 4 : 0;
    const int g0 = (int)(2 * (j & 3)) ^ sw, g1 = (int)(2 * (j & 3) + 1) ^ sw;
    const bool a0 = sa[g0], a1 = sa[g0 + 8], a2 = sa[g1], a3 = sa[g1 + 8];
    if (!(a0 || a1 || a2 || a3)) continue;
    const float b0 = sb[g0], b1 = sb[g0 + 8], b2 = sb[g1], b3 = sb[g1 + 8];
    const uint4 rv = rp[j], pv = pp[j];
    auto upd = [&](unsigned rw, unsigned pw, float b, bool on) -> unsigned {
      const float2 x = H::to_f2(rw), y = H::to_f2(pw);
      return on ? H::pack(__fmaf_rn(b, y.x, x.x), __fmaf_rn(b, y.y, x.y)) : pw;
    };
    pp[j] = make_uint4(upd(rv.x, pv.x, b0, a0), upd(rv.y, pv.y, b1, a1), upd(rv.z, pv.z, b2, a2),
                       upd(rv.w, pv.w, b3, a3));
  }
}

tm_status_t il_xpay(const Geom& g, tm_prec_t prec, void* p, const void* r, const double* beta,
                    const int* active, int nrhs, int par0, int npar, cudaStream_t s) {
  const int nblk = (nrhs + kIlRows - 1) / kIlRows;
  const unsigned plane_u4 = (unsigned)((size_t)g.Vh * (kIlSiteBytes / 16));
  const unsigned gx = std::min<unsigned>((plane_u4 + 255) / 256, 152u * 8u);
  const dim3 grid(gx, (unsigned)(nblk * npar));
  TraceScope tr(s, "blas.xpay", 3.0 * 24.0 * 2.0 * npar * g.Vh, 0.0, nrhs);
  if (prec == TM_PREC_F16)
    il_xpay_kernel<__half><<<grid, 256, 0, s>>>(static_cast<uint4*>(p), static_cast<const uint4*>(r), beta, active,
                                                nrhs, par0, npar, plane_u4);
  else
    il_xpay_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<uint4*>(p), static_cast<const uint4*>(r), beta,
                                                       active, nrhs, par0, npar, plane_u4);
  count_launch();
  return check_launch("xpay (interleaved)");
}

// out = A in (inverse = 0) or A^-1 in (inverse = 1) on one parity, as twist()
template <class S>
__global__ void il_twist_kernel(size_t Vh, uint2* out, const uint2* in, float tn, float sc, int nblk, int par) {
  using H = H16<S>;
  const size_t per_blk = Vh * kIlSiteU2;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= per_blk * nblk) return;
  const int blk = (int)(i / per_blk);
  const size_t rem = i % per_blk;
  const int k = (int)((rem >> 3) % 12);
  const size_t w = ((size_t)blk * 2 + par) * per_blk + rem;
  const float tw = k < 6 ? tn : -tn;
  const uint2 v = in[w];
  const float2 c0 = H::to_f2(v.x), c1 = H::to_f2(v.y);
  out[w] = make_uint2(H::pack(__fmul_rn(sc, __fmaf_rn(-tw, c0.y, c0.x)), __fmul_rn(sc, __fmaf_rn(tw, c0.x, c0.y))),
                      H::pack(__fmul_rn(sc, __fmaf_rn(-tw, c1.y, c1.x)), __fmul_rn(sc, __fmaf_rn(tw, c1.x, c1.y))));
}

tm_status_t il_twist(const Geom& g, tm_prec_t prec, void* out, const void* in, double nu, int inverse, int par,
                     int nrhs, cudaStream_t s) {
  const int nblk = (nrhs + kIlRows - 1) / kIlRows;
  const size_t n = (size_t)nblk * (size_t)g.Vh * kIlSiteU2;
  const unsigned nb = (unsigned)((n + 255) / 256);
  const float sc = inverse ? (float)(1.0 / (1.0 + nu * nu)) : 1.0f;
  const float tn = inverse ? (float)(-nu) : (float)nu;
  if (prec == TM_PREC_F16)
    il_twist_kernel<__half><<<nb, 256, 0, s>>>((size_t)g.Vh, static_cast<uint2*>(out),
                                                static_cast<const uint2*>(in), tn, sc, nblk, par);
  else
    il_twist_kernel<__nv_bfloat16><<<nb, 256, 0, s>>>((size_t)g.Vh, static_cast<uint2*>(out),
                                                       static_cast<const uint2*>(in), tn, sc, nblk, par);
  count_launch();
  return check_launch("twist (interleaved)");
}

}  // namespace tml

using namespace tml;

// ------------------------------------------------------------ C ABI
extern "C" size_t tm_spinor_bytes_il(const tm_geom_t* gg, int nrhs) {
  if (!gg || nrhs < 0 || check_geom(gg->L) != TM_OK) return 0;
  return il_bytes(make_geom(gg->L, 1), nrhs);
}

static tm_status_t il_conv_api(const char* what, const tm_geom_t* gg, void* out, const void* in, tm_prec_t prec,
                               int nrhs, bool to_il, tm_stream_t s) {
  if (!gg || !out || !in || nrhs < 0) {
    set_error("%s: null argument", what);
    return TM_ERR_ARG;
  }
  if (prec != TM_PREC_F16 && prec != TM_PREC_BF16) {
    set_error("%s: the interleaved layout holds F16 or BF16 fields", what);
    return TM_ERR_ARG;
  }
  if (out == in) {
    set_error("%s: out and in must not overlap", what);
    return TM_ERR_ARG;
  }
  if (check_geom(gg->L) != TM_OK) return TM_ERR_ARG;
  return il_convert(make_geom(gg->L, 1), out, in, nrhs, to_il, (cudaStream_t)s);
}

extern "C" tm_status_t tm_spinor_to_il(const tm_geom_t* gg, void* out_il, const void* in, tm_prec_t prec,
                                       int nrhs, tm_stream_t s) {
  return il_conv_api("tm_spinor_to_il", gg, out_il, in, prec, nrhs, true, s);
}

extern "C" tm_status_t tm_spinor_from_il(const tm_geom_t* gg, void* out, const void* in_il, tm_prec_t prec,
                                         int nrhs, tm_stream_t s) {
  return il_conv_api("tm_spinor_from_il", gg, out, in_il, prec, nrhs, false, s);
}

extern "C" tm_status_t tm_dslash_il(tm_op_t* op, void* out_il, const void* in_il, int nrhs, int dagger,
                                    int mu_zero, tm_prec_t prec, tm_stream_t s) {
  if (!op || !out_il || !in_il || nrhs < 0) {
    set_error("tm_dslash_il: null argument");
    return TM_ERR_ARG;
  }
  if (out_il == in_il) {
    set_error("tm_dslash_il: out and in must not overlap");
    return TM_ERR_ARG;
  }
  DslashCall c;
  c.in = in_il;
  c.out = out_il;
  c.nrhs = nrhs;
  c.dagger = dagger != 0;
  c.mu_zero = mu_zero != 0;
  return dslash_il_dispatch(op, prec, c, (cudaStream_t)s);
}

extern "C" tm_status_t tm_op_check(tm_op_t* op) {
  if (!op) {
    set_error("tm_op_check: null argument");
    return TM_ERR_ARG;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("tm_op_check: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  if (!op->il_err) return TM_OK;
  int v = 0;
  if (cudaMemcpy(&v, op->il_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("tm_op_check: %s", cudaGetErrorString(cudaGetLastError()));
    return TM_ERR_CUDA;
  }
  if (v != 0) {
    cudaMemset(op->il_err, 0, sizeof(int));
    set_error("tm_op_check: a bounded wait of the interleaved Dslash gave up");
    return TM_ERR_TIMEOUT;
  }
  return TM_OK;
}

extern "C" tm_status_t tm_cg_il_enable(int on) {
  g_il_on.store(on ? 1 : 0);
  return TM_OK;
}
