// FP16/BF16 Dslash with 18-real links on the tensor cores (warp-level MMA).
//
// Sixteen systems share every link of the lattice, so each hop of a site is a
// small dense contraction: with the projected 2-spinor h_s = psi_up + SGN
// A_mu psi_dn of the neighbour (s = 0, 1), the four output spins receive
//   out_0 += W h_0,  out_1 += W h_1,  out_2 += i^k2 W h_b0,  out_3 += i^k3 W h_b1
// (W = U or U^dag, the lower spins from the lower-left block B_mu of g_mu).
// The phase i^k and the choice of h are exact operations on the 16-bit words
// (swap halves, flip signs), so every output spin takes the same right
// operand W per hop, and the forward and backward hops of a direction form
// one m16n8k16 MMA per output spin:
//   D[rhs][(c_out, re/im)] += A[rhs][(hop, c_in, re/im)] * B[(hop, c_in, re/im)][(c_out, re/im)]
// with rows = 16 systems, k = (forward, backward) x 3 colours (+1 zero) x
// (re, im) of the rotated h, n = 3 colours (+1 zero) x (re, im) of the
// output, B the real form of W: B[(c, re)][(d, re)] = Re W_dc,
// B[(c, im)][(d, re)] = -Im W_dc, B[(c, re)][(d, im)] = Im W_dc,
// B[(c, im)][(d, im)] = Re W_dc.  Lane (g, t) holds A rows g and g + 8 at
// colour t of both hops, B column g (colour g/2, part g&1) at colour t, and
// D rows g, g + 8 at output colour t: one link entry per lane and hop, no
// lane-dependent register indexing; 16 MMAs per site.  The products of 16-bit
// numbers are exact, accumulation is in FP32; the projection h is one packed
// 16-bit add per entry, as in the CUDA-core 16-bit kernel, and the time
// boundary sign goes onto W.
//
// A block of 256 threads takes 32 consecutive output sites of one parity and
// 16 systems, one direction at a time through two shared-memory buffers: the
// neighbour spinors of the 32 sites (16 systems x 3 chunks, both hops) and
// their links are staged with 16-byte asynchronous copies, lane = site as in
// the CUDA-core kernel (coalesced: consecutive sites share cache lines), and
// direction mu + 1 is copied while the warps run the MMAs of direction mu,
// 4 sites per warp.  The staging layout [hop][row][chunk][site ^ (row & 7)][4
// words] keeps both the copies (lane = site) and the fragment reads (8 rows
// per instruction) free of bank conflicts.  The time-boundary sign comes from
// a per-site flag.  The accumulators stay in registers across the directions;
// the sums go through shared memory, and each thread runs the common epilogue
// (dslash_epilogue) for one (site, system), 32 consecutive sites per warp, so
// the per-warp partial sums are the same as the CUDA-core kernel's.  A
// system's result depends only on its own row.
#pragma once

namespace tml {

constexpr int kMmaSites = 32;    // output sites per block
constexpr int kMmaRows = 16;     // systems per block (MMA rows)
constexpr int kMmaThreads = 256;
constexpr int kMmaHops = 4;      // hops staged at a time: two buffers of one direction (fwd, bwd)
// shared memory: spinor words [hop][row][chunk][site][4] and link words
// [hop][unit][site][4] (both site-swizzled), then one boundary flag per site
constexpr int kMmaSpinWords = kMmaHops * kMmaSites * kMmaRows * 12;
constexpr int kMmaLinkWords = kMmaHops * kMmaSites * 12;
constexpr size_t kMmaSmem = sizeof(unsigned) * (kMmaSpinWords + kMmaLinkWords + kMmaSites);  // 102 KB
static_assert(sizeof(float2) * kMmaRows * 12 * kMmaSites <= sizeof(unsigned) * kMmaSpinWords,
              "the sums are staged in the spinor area");

// staging index of entry e (0..11) of row r at site sl: rows of 32 float2 with
// the site XOR-swizzled by the row, so that the lanes of one MMA (different
// rows, same site) and the lanes of the epilogue (same row, 32 sites) both hit
// distinct banks (up to the two wavefronts of a 64-bit access)
__device__ __forceinline__ int stage_idx(int r, int e, int sl) {
  const int row = r * 12 + e;
  return (row << 5) + (sl ^ (row & 31));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class S>
__device__ __forceinline__ void mma_m16n8k16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                             unsigned b0, unsigned b1);
template <>
__device__ __forceinline__ void mma_m16n8k16<__half>(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                                     unsigned a3, unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma_m16n8k16<__nv_bfloat16>(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                                            unsigned a3, unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// i^K times a 16-bit complex word (re low): swap halves and flip signs, exact
template <int K>
__device__ __forceinline__ unsigned rot_w(unsigned h) {
  constexpr int k = ((K % 4) + 4) % 4;
  if constexpr (k == 0) return h;
  else if constexpr (k == 2) return h ^ 0x80008000u;
  else if constexpr (k == 1) return __byte_perm(h, 0u, 0x1032) ^ 0x00008000u;  // (-im, re)
  else return __byte_perm(h, 0u, 0x1032) ^ 0x80000000u;                        // (im, -re)
}

// staged spinor word k (0..11) of row r at site sl, in the plane of one hop
__device__ __forceinline__ int spin_word(int r, int k, int sl) {
  return (((r * 3 + (k >> 2)) * kMmaSites + (sl ^ (r & 7))) << 2) + (k & 3);
}
constexpr int kMmaHopWords = kMmaRows * 12 * kMmaSites;  // one hop's plane
// staged link word i (0..8) at site sl, in the plane of one hop
__device__ __forceinline__ int link_word_idx(int i, int sl) {
  return (((i >> 2) * kMmaSites + (sl ^ (i >> 2))) << 2) + (i & 3);
}
constexpr int kMmaLinkHopWords = 12 * kMmaSites;

// Per-lane constants of the MMA phase.  Lane (g, t) reads spinor words
// k = 3 s + t (s = 0..3) of rows g and g + 8 and link word W_{g/2, t}; the
// site-independent parts of those shared-memory offsets are computed once.
struct MmaLane {
  int gq, tq;
  bool ulane;    // the lane's B column and row are not padding
  bool odd_col;  // B column part: im (odd) or re (even)
  int koff[4];   // rows' chunk/word offset of spin s: (k >> 2) * 128 + (k & 3)
  int rbase;     // offset of row g (row g + 8 is rbase + kMmaRow8)
  int uf, cf, ub, cb;  // link unit and offset of U_{g/2, t} (forward) and U_{t, g/2} (backward)
};
constexpr int kMmaRow8 = 8 * 3 * kMmaSites * 4;  // spin_word offset between rows r and r + 8

__device__ __forceinline__ MmaLane mma_lane() {
  MmaLane l;
  const int lane = threadIdx.x & 31;
  l.gq = lane >> 2;
  l.tq = lane & 3;
  l.ulane = l.gq < 6 && l.tq < 3;
  l.odd_col = (l.gq & 1) != 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int k = 3 * s + l.tq;
    l.koff[s] = (k >> 2) * (kMmaSites * 4) + (k & 3);
  }
  l.rbase = l.gq * 3 * (kMmaSites * 4);
  const int co = l.gq >> 1;
  const int i_f = 3 * co + l.tq, i_b = 3 * l.tq + co;
  l.uf = i_f >> 2;
  l.cf = l.uf * (kMmaSites * 4) + (i_f & 3);
  l.ub = i_b >> 2;
  l.cb = l.ub * (kMmaSites * 4) + (i_b & 3);
  return l;
}

// The projected words (h0, h1) of rows g and g + 8 at colour t of one hop
// (zero in the padding column t = 3); o[s]: offsets of spin s in row g.
template <class S, int MU, int SGN>
__device__ __forceinline__ void project_rows(unsigned (&h)[2][2], const unsigned* sp, const int (&o)[4], int t) {
  using G = GBlock<MU>;
  constexpr int s2 = SGN > 0 ? 0 : 2;
  unsigned q[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
  if (t < 3) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      q[0][s] = sp[o[s]];
      q[1][s] = sp[o[s] + kMmaRow8];
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    h[r][0] = add_ph_w<G::ak0 + s2, S>(q[r][0], q[r][2 + G::ac0]);
    h[r][1] = add_ph_w<G::ak1 + s2, S>(q[r][1], q[r][2 + G::ac1]);
  }
}

// Real form of W_{c_out, c_in} for this lane's B column (part re: even column,
// im: odd); u = U_{c_out, c_in} (forward) or U_{c_in, c_out} (W = U^dag).
template <bool ADJ>
__device__ __forceinline__ unsigned b_word(unsigned u, bool odd_col) {
  if constexpr (!ADJ) return odd_col ? __byte_perm(u, 0u, 0x1032) : (u ^ 0x80000000u);
  else return odd_col ? (__byte_perm(u, 0u, 0x1032) ^ 0x00008000u) : u;
}

// Both hops of direction MU for a staged site (spinor planes spf, spb, link
// planes suf, sub; o, lf, lb the lane's offsets for the site): for the lane's
// rows, d[s] += rows of spin s of
//   (1 + SF g_MU) U_MU(x) psi(x + MU) + (1 + SB g_MU) U_MU(x - MU)^dag psi(x - MU)
// (SF = -1 for M, +1 for M^dag; SB = -SF); negf / negb negate a hop across the
// antiperiodic time boundary.
template <class S, int MU, bool DAG>
__device__ __forceinline__ void dir_mma(float (&d)[4][4], const unsigned* spf, const unsigned* spb,
                                        const unsigned* suf, const unsigned* sub, const int (&o)[4], int lf, int lb,
                                        const MmaLane& l, unsigned negf, unsigned negb) {
  using G = GBlock<MU>;
  constexpr int SF = DAG ? +1 : -1;
  constexpr int SB = -SF;
  constexpr int s2f = SF > 0 ? 0 : 2, s2b = SB > 0 ? 0 : 2;
  const unsigned bf = b_word<false>(l.ulane ? suf[lf] : 0u, l.odd_col) ^ negf;
  const unsigned bb = b_word<true>(l.ulane ? sub[lb] : 0u, l.odd_col) ^ negb;
  unsigned hf[2][2], hb[2][2];  // [row g / g + 8][h0 / h1]
  project_rows<S, MU, SF>(hf, spf, o, l.tq);
  project_rows<S, MU, SB>(hb, spb, o, l.tq);
  mma_m16n8k16<S>(d[0], hf[0][0], hf[1][0], hb[0][0], hb[1][0], bf, bb);
  mma_m16n8k16<S>(d[1], hf[0][1], hf[1][1], hb[0][1], hb[1][1], bf, bb);
  mma_m16n8k16<S>(d[2], rot_w<G::bk0 + s2f>(hf[0][G::bc0]), rot_w<G::bk0 + s2f>(hf[1][G::bc0]),
                  rot_w<G::bk0 + s2b>(hb[0][G::bc0]), rot_w<G::bk0 + s2b>(hb[1][G::bc0]), bf, bb);
  mma_m16n8k16<S>(d[3], rot_w<G::bk1 + s2f>(hf[0][G::bc1]), rot_w<G::bk1 + s2f>(hf[1][G::bc1]),
                  rot_w<G::bk1 + s2b>(hb[0][G::bc1]), rot_w<G::bk1 + s2b>(hb[1][G::bc1]), bf, bb);
}

// What a block needs in every stage
struct MmaCtx {
  int par, cb0, r0;
  unsigned amask;   // active rows of the block (bit row)
  bool site_ok;     // this lane's staging site is on the lattice
  Site s;           // this lane's staging site (cb0 + lane)
};

// Stage direction MU into buffer buf (hop planes 2 buf: forward, 2 buf + 1:
// backward): lane = site; warp w copies rows w and w + 8 (3 chunks each) of
// both hops, warps 0..5 one (hop, link unit) each.  Asynchronous 16-byte
// copies, committed as one group.
template <class S, int MU>
__device__ __forceinline__ void mma_stage(const DslashArgs& a, const MmaCtx& x, unsigned* sA, unsigned* sU,
                                          int buf) {
  const Geom& g = a.g;
  constexpr int NCH = spinor_chunks<S>();
  using F = LinkFmt<S, 18>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int opar = x.par ^ 1;
  const size_t cs = (size_t)g.Vh;
  if (x.site_ok) {
    const int rowA = warp, rowB = warp + 8;
    const bool actA = (x.amask >> rowA) & 1u, actB = (x.amask >> rowB) & 1u;
    const uint4* fin = reinterpret_cast<const uint4*>(a.c.in);
    const uint4* srcA = actA ? fin + ((size_t)((x.r0 + rowA) * 2 + opar) * NCH) * cs : fin;
    const uint4* srcB = actB ? fin + ((size_t)((x.r0 + rowB) * 2 + opar) * NCH) * cs : fin;
    const int dstA = rowA * 3 * (kMmaSites * 4) + ((lane ^ warp) << 2);  // spin_word(rowA, 0, lane)
    const uint4* lk = reinterpret_cast<const uint4*>(a.links);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool fwd = h == 0;
      const int nb = (fwd ? lex_fwd(g, x.s, MU) : lex_bwd(g, x.s, MU)) >> 1;
      unsigned* dst = sA + (2 * buf + h) * kMmaHopWords + dstA;
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        if (actA) cp_async16(dst + j * (kMmaSites * 4), srcA + j * cs + nb);
        if (actB) cp_async16(dst + j * (kMmaSites * 4) + kMmaRow8, srcB + j * cs + nb);
      }
      const int lpar = fwd ? x.par : opar;
      const int lcb = fwd ? x.cb0 + lane : nb;
#pragma unroll
      for (int u = 0; u < F::NU; ++u) {
        if (h * F::NU + u != warp) continue;
        cp_async16(sU + (2 * buf + h) * kMmaLinkHopWords + link_word_idx(4 * u, lane),
                   lk + ((size_t)(MU * 2 + lpar) * F::NU + u) * cs + lcb);
      }
    }
  }
  cp_async_commit();
}

// The MMAs of direction MU from buffer buf: warp w takes sites 4 w .. 4 w + 3.
template <class S, bool DAG, int MU>
__device__ __forceinline__ void mma_compute(const MmaCtx& x, const MmaLane& l, const unsigned* sA,
                                            const unsigned* sU, const unsigned* sNeg, int buf, int Vh,
                                            float (&d)[4][4][4]) {
  const int warp = threadIdx.x >> 5;
  const unsigned* spf = sA + (2 * buf) * kMmaHopWords;
  const unsigned* suf = sU + (2 * buf) * kMmaLinkHopWords;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int sl = warp * 4 + i;
    if (x.cb0 + sl >= Vh) continue;
    int o[4];
    const int base = l.rbase + ((sl ^ l.gq) << 2);
#pragma unroll
    for (int s = 0; s < 4; ++s) o[s] = base + l.koff[s];
    const int lf = l.cf + ((sl ^ l.uf) << 2), lb = l.cb + ((sl ^ l.ub) << 2);
    unsigned negf = 0u, negb = 0u;
    if constexpr (MU == 3) {
      const unsigned fl = sNeg[sl];
      negf = (fl & 1u) ? 0x80008000u : 0u;
      negb = (fl & 2u) ? 0x80008000u : 0u;
    }
    dir_mma<S, MU, DAG>(d[i], spf, spf + kMmaHopWords, suf, suf + kMmaLinkHopWords, o, lf, lb, l, negf, negb);
  }
}

template <class S, bool DAG, int EPI>
__global__ void __launch_bounds__(kMmaThreads, 2) dslash_kernel_mma(const DslashArgs a) {
  static_assert(std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value, "16-bit storage only");
  extern __shared__ uint4 smem_mma[];
  unsigned* sA = reinterpret_cast<unsigned*>(smem_mma);
  unsigned* sU = sA + kMmaSpinWords;
  float2* stage = reinterpret_cast<float2*>(smem_mma);  // [row][12][32 sites], stage_idx
  const Geom& g = a.g;
  const int sb = blockIdx.x;
  MmaCtx x;
  x.par = a.c.parity < 0 ? (sb & 1) : a.c.parity;
  x.cb0 = (a.c.parity < 0 ? (sb >> 1) : sb) * kMmaSites;
  x.r0 = blockIdx.y * kMmaRows;
  const int nrhs = a.c.nrhs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  if (a.trace_count && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < nrhs; ++r) n += (a.c.active == nullptr || a.c.active[r] != 0) ? 1 : 0;
    *a.trace_count = n;
  }
  x.amask = 0u;
#pragma unroll 1
  for (int row = 0; row < kMmaRows; ++row) {
    const int r = x.r0 + row;
    if (r < nrhs && (a.c.active == nullptr || a.c.active[r] != 0)) x.amask |= 1u << row;
  }
  x.site_ok = x.cb0 + lane < g.Vh;
  x.s = site_of(g, x.par, x.site_ok ? x.cb0 + lane : x.cb0);
  float d[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int v = 0; v < 4; ++v) d[i][q][v] = 0.0f;
  if (x.amask != 0u) {  // uniform over the block
    unsigned* sNeg = sU + kMmaLinkWords;
    if (warp == 0) {  // hops across the antiperiodic time boundary
      const bool tb = g.antiperiodic && x.site_ok;
      sNeg[lane] = (tb && x.s.c[3] == g.L[3] - 1 ? 1u : 0u) | (tb && x.s.c[3] == 0 ? 2u : 0u);
    }
    const MmaLane l = mma_lane();
    // two buffers: direction mu + 1 is copied while mu is computed
    mma_stage<S, 0>(a, x, sA, sU, 0);
    mma_stage<S, 1>(a, x, sA, sU, 1);
    cp_async_wait<1>();
    __syncthreads();
    mma_compute<S, DAG, 0>(x, l, sA, sU, sNeg, 0, g.Vh, d);
    __syncthreads();
    mma_stage<S, 2>(a, x, sA, sU, 0);
    cp_async_wait<1>();
    __syncthreads();
    mma_compute<S, DAG, 1>(x, l, sA, sU, sNeg, 1, g.Vh, d);
    __syncthreads();
    mma_stage<S, 3>(a, x, sA, sU, 1);
    cp_async_wait<1>();
    __syncthreads();
    mma_compute<S, DAG, 2>(x, l, sA, sU, sNeg, 0, g.Vh, d);
    cp_async_wait<0>();
    __syncthreads();
    mma_compute<S, DAG, 3>(x, l, sA, sU, sNeg, 1, g.Vh, d);
    __syncthreads();  // the sums are staged in the spinor area
    if (tq < 3) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int sl = warp * 4 + i;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          const int e = 3 * sp + tq;
          stage[stage_idx(gq, e, sl)] = make_float2(d[i][sp][0], d[i][sp][1]);
          stage[stage_idx(gq + 8, e, sl)] = make_float2(d[i][sp][2], d[i][sp][3]);
        }
      }
    }
  }
  __syncthreads();
  // epilogue: warp w takes rows w and w + 8; lane = site
  const int cb = x.cb0 + lane;
  const EpiConsts<float> k = epi_consts<float>(a);
#pragma unroll 1
  for (int j = 0; j < kMmaRows / (kMmaThreads / 32); ++j) {
    const int rl = warp + (kMmaThreads / 32) * j;
    const int r = x.r0 + rl;
    double part = 0.0;
    if (((x.amask >> rl) & 1u) && cb < g.Vh) {
      Cx<float> acc[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        const float2 v = stage[stage_idx(rl, e, lane)];
        acc[e] = {v.x, v.y};
      }
      part = dslash_epilogue<S, EPI>(a, k, r, x.par, cb, acc);
    }
    if (EPI != EPI_OUT || a.c.partial != nullptr) {
      const double ps = warp_sum(part);
      if (lane == 0 && r < nrhs) a.c.partial[((size_t)r * 2 + x.par) * a.nwarp + x.cb0 / 32] = ps;
    }
  }
}

// the tensor-core kernels need more than the default 48 KB of shared memory
template <class S>
tm_status_t dslash_mma_prepare() {
  const void* k[6] = {(const void*)dslash_kernel_mma<S, false, EPI_OUT>, (const void*)dslash_kernel_mma<S, false, EPI_CGUPD>,
                      (const void*)dslash_kernel_mma<S, false, EPI_RESID>, (const void*)dslash_kernel_mma<S, true, EPI_OUT>,
                      (const void*)dslash_kernel_mma<S, true, EPI_CGUPD>, (const void*)dslash_kernel_mma<S, true, EPI_RESID>};
  for (const void* f : k)
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem) != cudaSuccess) {
      set_error("dslash: shared memory attribute: %s", cudaGetErrorString(cudaGetLastError()));
      return TM_ERR_CUDA;
    }
  return TM_OK;
}

}  // namespace tml
