/*
 * tmloops — stochastic disconnected fermion loops for twisted-mass Wilson
 * fermions on one GB300 GPU (method of arXiv:1401.6749).
 *
 * C ABI.  Every pointer to a field, a loop array or a gauge field is a DEVICE
 * pointer owned by the caller; the library never frees caller memory.  The
 * library allocates device memory only from its own stream-ordered pool (one
 * per device, see tm_mem_trim): inside an opaque tm_op_t (link copies, solver
 * work vectors) and, for the two-stage reductions of the contraction kernels
 * and the HPE ping-pong fields, scratch taken from and returned to that pool
 * in the caller's stream order.  All calls are asynchronous with respect to the host and
 * ordered on the given stream, except tm_op_create (waits for the link packing)
 * and tm_cg_solve (returns when every right-hand side has converged or hit
 * its iteration limit).  Functions return a tm_status_t; on failure
 * tm_last_error() (thread-local) describes the cause.  Nothing here traps the
 * GPU: argument errors are reported before any launch, and solver failures
 * (no convergence, non-finite residuals) come back as status codes.
 *
 * Lattice and fields
 * ------------------
 * Extents L = {X, Y, Z, T}, every one even and >= 2; V = X*Y*Z*T.  Site
 * x = (x, y, z, t) has lexicographic index  lex = x + X*(y + Y*(z + Z*t))  and
 * parity (x + y + z + t) mod 2.  Direction mu = 0, 1, 2, 3 is x, y, z, t.
 *
 * Canonical (host-facing) layouts, complex numbers as (re, im) pairs of double:
 *   spinor  [nrhs][V (lex)][4 Dirac][3 colour][2]
 *   gauge   [4 mu][V (lex)][3][3][2]         U[mu](x) = link from x to x + mu_hat
 *   loops   local: [nrhs][16 Gamma][T][2]    one-derivative: [nrhs][4 mu][16][T][2]
 *
 * Internal (device compute) spinor layout, produced by tm_spinor_pack or
 * z4_noise and consumed by every kernel: for precision P with element size s,
 * a field is [nrhs][2 parity][24*s/16 chunks][V/2 sites][16 bytes], site index
 * within a parity cb = lex/2, each 16-byte chunk holding consecutive reals of the
 * canonical per-site order.  Bytes per field: tm_spinor_bytes().
 *
 * Dirac basis: DeGrand-Rossi chiral, Euclidean, gamma_5 = g1 g2 g3 g4 =
 * diag(1, 1, -1, -1).  The 16 insertions are Gamma_n = g1^n0 g2^n1 g3^n2 g4^n3
 * with n = n0 + 2 n1 + 4 n2 + 8 n3 (Gamma_0 = 1, Gamma_15 = gamma_5).
 */
#ifndef TMLOOPS_H
#define TMLOOPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL selects the legacy default stream. */
typedef struct CUstream_st *tm_stream_t;

typedef enum {
  TM_OK = 0,
  TM_ERR_ARG = 1,        /* invalid argument (null pointer, bad extent, size) */
  TM_ERR_CUDA = 2,       /* a CUDA runtime call failed */
  TM_ERR_NOCONV = 3,     /* CG reached max_iter before the tolerance */
  TM_ERR_NAN = 4,        /* a residual norm became non-finite */
  TM_ERR_TIMEOUT = 5,    /* a bounded wait gave up */
  TM_ERR_UNSUPPORTED = 6 /* valid but unsupported combination (e.g. 18-real half links) */
} tm_status_t;

typedef enum {
  TM_PREC_F64 = 0,
  TM_PREC_F32 = 1,
  TM_PREC_F16 = 2,  /* IEEE binary16 storage, FP32 arithmetic */
  TM_PREC_BF16 = 3, /* bfloat16 storage, FP32 arithmetic */
  TM_PREC_FF = 4    /* float-float: each real is a pair (hi, lo) of FP32 values
                       (8 bytes) summing to it, about 48 significant bits, FP32
                       exponent range; float-float arithmetic on the FP32 pipes.
                       For the Dslash, the contractions and the layout helpers;
                       not a solver precision (tm_cg_solve returns TM_ERR_ARG). */
} tm_prec_t;

typedef struct { int L[4]; } tm_geom_t;

/* Twisted-mass Wilson operator (Sec. 2.2 and 2.4; kappa normalisation):
 *   M psi(x) = psi(x) + i nu g5 psi(x)
 *            - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ],
 * nu = 2 kappa mu, psi antiperiodic in time when antiperiodic_t != 0.
 * M^dag = g5 M(-mu) g5;  D_W = M at mu = 0 (Eq. 6).                      */
typedef struct {
  int L[4];
  double kappa;
  double mu;
  int antiperiodic_t;
  int recon;  /* 12 or 18: real numbers stored per link in the F32/F16/BF16
                 copies (12 = two rows, third = conj(row0 x row1)); the F64
                 copy always stores 18.  0: per precision, as measured fastest
                 on GB300: 12 for F32 (its Dslash streams more bytes per flop),
                 18 for F16/BF16 (their Dslash is bound by FP32 issue, and the
                 third-row reconstruction costs more than the extra bytes) */
} tm_params_t;

typedef struct tm_op tm_op_t;

/* Create an operator: validates p, copies the FP64 canonical gauge field
 * U_lex ([4][V][3][3][2] doubles, not retained) into internal even/odd link
 * arrays for every precision.  U_lex is device memory, or page-locked host
 * memory (cudaHostAlloc / cudaHostRegister, 16-byte aligned) that the GPU reads
 * in one pass of its SMs over the host link into a staging buffer; other host
 * memory is TM_ERR_ARG.  Blocks until done.                               */
tm_status_t tm_op_create(tm_op_t **op, const tm_params_t *p, const double *U_lex, tm_stream_t s);
tm_status_t tm_op_destroy(tm_op_t *op);
/* A second handle on the same operator: shares the source's link arrays (no
 * copy) but has its own solver work space, so that solves on different host
 * threads and streams can run concurrently.  Destroy clones before their
 * source.  Calls on one handle must not overlap.                          */
tm_status_t tm_op_clone(tm_op_t **out, const tm_op_t *src);

/* Device memory.  Link copies, solver work spaces and contraction scratch come
 * from a stream-ordered pool owned by the library, one per device, that keeps
 * freed memory for its next allocations: creating an operator after
 * destroying one of the same lattice maps no new pages.  tm_op_destroy waits
 * for the device (like cudaFree) before returning its memory to the pool.
 * tm_mem_trim(keep_bytes) waits for the device and releases unused pool
 * memory beyond keep_bytes to the system (and the cached pinned host blocks
 * of the solver's flags); tm_mem_reserved gives the bytes the pool of the
 * current device holds, in use or not.                                     */
tm_status_t tm_mem_trim(size_t keep_bytes);
tm_status_t tm_mem_reserved(size_t *bytes);

/* Bytes of nrhs internal spinor fields of precision prec on geometry g. */
size_t tm_spinor_bytes(const tm_geom_t *g, tm_prec_t prec, int nrhs);

/* Canonical FP64 <-> internal layout (round to nearest even on narrowing). */
tm_status_t tm_spinor_pack(const tm_geom_t *g, void *out, tm_prec_t prec,
                           const double *in_lex, int nrhs, tm_stream_t s);
tm_status_t tm_spinor_unpack(const tm_geom_t *g, double *out_lex, const void *in,
                             tm_prec_t prec, int nrhs, tm_stream_t s);
/* Internal layout precision conversion, out and in must not overlap. */
tm_status_t tm_spinor_convert(const tm_geom_t *g, void *out, tm_prec_t out_prec,
                              const void *in, tm_prec_t in_prec, int nrhs, tm_stream_t s);
/* out = gamma_5 in (internal layout; out may equal in). */
tm_status_t tm_gamma5(const tm_geom_t *g, void *out, const void *in, tm_prec_t prec,
                      int nrhs, tm_stream_t s);

/* out = M in, M^dag in (dagger != 0) or D_W in (mu_zero != 0) for nrhs
 * internal-layout fields of precision prec; FP32 arithmetic for F16/BF16.
 * out and in must not overlap.                                             */
tm_status_t tm_dslash(tm_op_t *op, void *out, const void *in, int nrhs, int dagger,
                      int mu_zero, tm_prec_t prec, tm_stream_t s);
/* out = gamma_5 M in (or gamma_5 M^dag in, gamma_5 D_W in) in one pass: the
 * right field R = gamma_5 D_W s of the generalised one-end trick (Eq. 6),
 * without the separate gamma_5 pass.  Arguments as for tm_dslash.          */
tm_status_t tm_dslash_g5(tm_op_t *op, void *out, const void *in, int nrhs, int dagger,
                         int mu_zero, tm_prec_t prec, tm_stream_t s);

/* System-interleaved 16-bit layout (this library's own; the paper gives no
 * layout).  nrhs F16 or BF16 fields stored as ceil(nrhs / 16) blocks of 16
 * systems: [block][parity][cb][k = 3 spin + colour][slot 0..15], 4 bytes per
 * slot (one complex number, re in the low half), 64 bytes per (site, k) and
 * 768 per site; system j < 8 of a block sits in slot 2p and system j + 8 in
 * slot 2p + 1, p = j in the rows k = 0, 1 (mod 3) and p = j ^ 4 in the rows
 * k = 2 (mod 3).
 * The multi-system Dslash reads it with one 8-byte load per (spin, colour,
 * two systems) and feeds the tensor cores straight from it.
 * tm_spinor_bytes_il: bytes of nrhs systems (0 on a bad geometry).
 * tm_spinor_to_il / tm_spinor_from_il: standard internal layout <-> this one
 *   (a byte permutation: exact; slots of systems >= nrhs are written as
 *   zero); out and in must not overlap.  prec F16 or BF16, else TM_ERR_ARG.
 * tm_dslash_il: out = M in, M^dag in or D_W in (as tm_dslash) on fields in
 *   this layout, each hop a warp-level MMA over 16 systems (FP16/BF16
 *   products, FP32 accumulation), every site's neighbours staged in shared
 *   memory by asynchronous tensor (gather4) and bulk copies (the fields must
 *   be 16-byte aligned, else TM_ERR_ARG; TM_ERR_CUDA if the driver cannot
 *   encode a tensor map).  Needs the 18-real 16-bit link copy (recon 18 or 0:
 *   TM_ERR_UNSUPPORTED for 12).  Results agree with tm_dslash to the 16-bit
 *   tolerance; the bits differ (summation order).  A staging wait that never
 *   completes gives up after about one second and sets a flag of
 *   the operator: tm_op_check(op) waits for the device and returns
 *   TM_ERR_TIMEOUT (clearing the flag) if that happened, tm_cg_solve returns
 *   TM_ERR_TIMEOUT at its next poll.
 * tm_cg_il_enable(1) (default, unless the environment sets TM_CG_IL=0): plain
 *   F16/BF16 solves of tm_cg_solve convert eta to this layout, iterate on it
 *   with tm_dslash_il's kernel and convert x back; 0 keeps them on the
 *   CUDA-core kernel of the standard layout.  Switch between solves only: the
 *   two give different (equally valid) truncated solutions.                */
size_t tm_spinor_bytes_il(const tm_geom_t *g, int nrhs);
tm_status_t tm_spinor_to_il(const tm_geom_t *g, void *out_il, const void *in, tm_prec_t prec, int nrhs,
                            tm_stream_t s);
tm_status_t tm_spinor_from_il(const tm_geom_t *g, void *out, const void *in_il, tm_prec_t prec, int nrhs,
                              tm_stream_t s);
tm_status_t tm_dslash_il(tm_op_t *op, void *out_il, const void *in_il, int nrhs, int dagger, int mu_zero,
                         tm_prec_t prec, tm_stream_t s);
tm_status_t tm_cg_il_enable(int on);
tm_status_t tm_op_check(tm_op_t *op);


/* Z4 noise (Sec. 2, Eqs. 1-2): eta_r(x)_{alpha c} = i^k with k = bits
 * [2(3 alpha + c), 2(3 alpha + c) + 1] of word 0 of Philox4x32-10 applied to
 * counter (lex, r, 0, 0) with key (seed mod 2^32, seed >> 32), for
 * r = first_src .. first_src + nsrc - 1.  Values are exact in every precision.
 * Output: nsrc internal-layout fields of precision prec.                   */
tm_status_t z4_noise(const tm_geom_t *g, void *eta, tm_prec_t prec, uint64_t seed,
                     uint32_t first_src, int nsrc, tm_stream_t s);

/* Time dilution with coherent sources (Sec. 2.3): the same Z4 noise as
 * z4_noise on the time slices t = t0 (mod dt), zero on all others (dt = T: one
 * slice; dt < T: coherent sources on slices dt apart).  The diluted sources
 * t0 = 0 .. dt-1 add up to the undiluted one.  1 <= dt, 0 <= t0 < dt.     */
tm_status_t z4_noise_diluted(const tm_geom_t *g, void *eta, tm_prec_t prec, uint64_t seed,
                             uint32_t first_src, int nsrc, int t0, int dt, tm_stream_t s);

/* z4_noise written straight into the interleaved 16-bit layout (the same
 * bits as z4_noise followed by tm_spinor_to_il): source r = first_src + j
 * is system j of eta_il (tm_spinor_bytes_il(g, nsrc) bytes, 4-byte aligned);
 * the slots of systems >= nsrc in the last block of 16 are written as zero.
 * prec F16 or BF16, else TM_ERR_ARG.                                       */
tm_status_t z4_noise_il(const tm_geom_t *g, void *eta_il, tm_prec_t prec, uint64_t seed,
                        uint32_t first_src, int nsrc, tm_stream_t s);

/* Hopping Parameter Expansion (Sec. 2.4, Eqs. 7-8).  With B = (1 + i nu g5)^-1
 * and H = M - B^-1 (-kappa times the hops of M),
 *   M^-1 = B - B H B + (BH)^2 B - (BH)^3 B + (BH)^4 M^-1.
 * tm_hpe_apply: out = (BH)^order in (nrhs internal fields of precision prec;
 *   out and in must not overlap; uses stream-ordered scratch of one field set).
 * tm_hpe_exact: the exact part of the local loops, Tr_t[Gamma_g (B - BHB +
 *   (BH)^2 B - (BH)^3 B)] for every time slice, written to the HOST array
 *   out[16][T][2]; the odd orders vanish on the diagonal and the rest is gauge
 *   independent when every extent is >= 4 (TM_ERR_UNSUPPORTED otherwise).
 * The HPE estimate of Tr_t[Gamma M^-1] is tm_hpe_exact plus the standard
 * contraction (L = eta, R = (BH)^4 s, TM_LOOP_STD) averaged over sources.   */
tm_status_t tm_hpe_apply(tm_op_t *op, void *out, const void *in, int nrhs, int order,
                         tm_prec_t prec, tm_stream_t s);
tm_status_t tm_hpe_exact(const tm_params_t *p, double *out);

/* Conjugate gradient on the normal equations (Sec. 2.1: "a CG solver"):
 *   M^dag M x = M^dag eta,  x_0 = 0,  so that x = M^{-1} eta = s (Eq. 3);
 * stop when the iterated residual satisfies |r| <= tol |M^dag eta|.
 * TM_CG_PLAIN: every vector in `prec` (the low-precision TSM solves run this
 *   way in F16/BF16 with tol ~ 1e-2, Sec. 2.1; the FP64 baseline in F64).
 * TM_CG_MIXED: x, eta and the true residual in F64; the iteration in
 *   inner_prec; reliable updates (x += y, r = b - M^dag M x in F64) whenever
 *   |r| < delta * max|r| since the last update, and before accepting
 *   convergence.  eta and x are then F64 internal fields.
 * schur = 1: even/odd preconditioning (the paper does not say whether it was
 *   used).  With A = 1 + i nu g5 (the even-even and odd-odd blocks of M),
 *   CG runs on M_hat^dag M_hat x_o = M_hat^dag eta_hat on the odd sites,
 *   M_hat = A - kappa^2 H_oe A^-1 H_eo, eta_hat = eta_o + kappa H_oe A^-1 eta_e,
 *   and s_e = A^-1 (eta_e + kappa H_eo s_o) completes x = M^-1 eta; tol,
 *   rel_res and true_res then refer to this odd-site system.
 * nrhs independent systems are solved together; each has its own scalars and
 * stops on its own.  stats (host array of nrhs, may be NULL) receives per-system
 * results.  Blocks the calling thread until all systems have stopped.
 * Returns TM_ERR_NOCONV if any system hit max_iter, TM_ERR_NAN on non-finite
 * norms.  x and eta must not overlap.
 * graph = 1: the check_every iterations between two host polls (every kernel
 *   of them plus the copy of the convergence flags) are captured once into a
 *   CUDA graph and replayed, one graph launch per poll; the results are
 *   bit-identical to graph = 0 (converged systems are masked on the device
 *   either way).  Launches inside the graph are not traced individually: each
 *   replay is one trace record "cg.graph".  A single-set solve keeps its graph
 *   in the operator and replays it, without capturing, in the next solve whose
 *   launches are the same (same buffers, systems and parameters).
 * ru_prec (MIXED): TM_PREC_F64 (0) computes the true residuals
 *   r = b - M^dag M x of the reliable updates (and the final one) in FP64;
 *   TM_PREC_FF in float-float on the FP32 pipes (about 48-bit significands,
 *   from float-float copies of x and b; x itself still accumulates in FP64).
 *   FF residuals are exact to about 2^-48 cond(M^dag M) |b|, so only solves
 *   conditioned well enough for that to stay far below tol should use them.
 *   Other values: TM_ERR_ARG.                                               */
typedef enum { TM_CG_PLAIN = 0, TM_CG_MIXED = 1 } tm_cg_mode_t;

typedef struct {
  double tol;
  int max_iter;
  tm_cg_mode_t mode;
  tm_prec_t prec;        /* PLAIN: precision of eta, x and work vectors     */
  tm_prec_t inner_prec;  /* MIXED: precision of the inner iteration         */
  double delta;          /* MIXED: reliable-update threshold (e.g. 0.1)     */
  int check_every;       /* host polls the convergence flags every N iterations (>= 1) */
  int true_residual;     /* PLAIN: compute |b - M^dag M x| / |b| at the end */
  int schur;             /* 1: even/odd preconditioned solve (see below), 0: plain M */
  int graph;             /* 1: replay the iterations between polls as one CUDA graph */
  tm_prec_t ru_prec;     /* MIXED: arithmetic of the true residuals, F64 (0) or FF   */
} tm_cg_params_t;

typedef struct {
  int iters;
  int reliable_updates;
  int status;            /* tm_status_t of this system */
  double rel_res;        /* iterated |r| / |b| at exit  */
  double true_res;       /* |b - M^dag M x| / |b| (MIXED, or PLAIN with true_residual), else -1 */
} tm_cg_stats_t;

tm_status_t tm_cg_solve(tm_op_t *op, void *x, const void *eta, int nrhs,
                        const tm_cg_params_t *p, tm_cg_stats_t *stats, tm_stream_t s);

/* tm_cg_solve on fields in the interleaved layout: eta_il and x_il (each
 * 16-byte aligned, tm_spinor_bytes_il(g, nrhs) bytes, not overlapping) hold
 * the sources and receive the solutions.  The solution bits equal those that
 * tm_cg_solve, given the same sources in the standard layout, converts into
 * x.  Only for the solves that run on the interleaved layout (plain
 * F16/BF16, 18-real links, tm_cg_il_enable on): TM_ERR_UNSUPPORTED
 * otherwise.                                                               */
tm_status_t tm_cg_solve_il(tm_op_t *op, void *x_il, const void *eta_il, int nrhs,
                           const tm_cg_params_t *p, tm_cg_stats_t *stats, tm_stream_t s);

/* Several independent batched solves advanced together (an uneven batch:
 * different lattices, kappa, mu and numbers of systems, as in a sweep over
 * volumes and quark masses; each set is the solve tm_cg_solve describes, with
 * the common parameters p).  Set i solves ops[i] on the nrhs[i] systems of the
 * internal fields x[i] / eta[i] and writes stats[i][0 .. nrhs[i]-1] (stats or
 * any stats[i] may be NULL).  The sets run on streams forked from s and joined
 * back into it, so that small lattices share the GPU; with p->graph = 1 the
 * iterations of ALL sets between two polls are one CUDA graph launch.  Every
 * set needs its own operator handle (tm_op_clone shares the links): a handle
 * used twice is TM_ERR_ARG.  Results of each set are bit-identical to
 * tm_cg_solve of that set alone.  Returns the worst status over the sets.
 * This grouping is this library's own (the paper solves one source at a time). */
tm_status_t tm_cg_solve_group(int nsets, tm_op_t *const *ops, void *const *x,
                              const void *const *eta, const int *nrhs,
                              const tm_cg_params_t *p, tm_cg_stats_t *const *stats,
                              tm_stream_t s);

/* Loop contractions (Sec. 2.2; Sec. 1 and Table 2 for the operator classes).
 * For each right-hand side r and time slice t,
 *   local:  out[r][g][t] = sum_{x_t = t} L_r(x)^dag (P Gamma_g) R_r(x)
 *   oneD:   out[r][mu][g][t] = sum_{x_t = t} 1/4 [ Lb(x) G U_mu(x) R(x+mu) - Lb(x) G U_mu(x-mu)^dag R(x-mu)
 *                                - Lb(x+mu) G U_mu(x)^dag R(x) + Lb(x-mu) G U_mu(x-mu) R(x) ]
 *           (symmetric covariant derivative, Lb = L^dag, G = P Gamma_g, antiperiodic hops in t)
 * with P = 1 for TM_LOOP_STD (L = eta, R = s: Tr[X M^-1], Eq. 3) and
 * P = gamma_5 for TM_LOOP_VV (L = R = s, Eq. 5, prefactor -2 i nu) and
 * TM_LOOP_GEN (L = s, R = gamma_5 D_W s, Eq. 6, prefactor 2).  The caller
 * forms L and R; the prefactor is applied by tsm_combine.  left/right are
 * internal-layout fields of precision prec; out is a device array of doubles
 * (layout above).  The two-stage reductions take their scratch from the
 * library's pool: 64 * nrhs * T * ceil(X*Y*Z/2048) doubles (local), a few
 * times that (oneD).  The launch grid limits T to 2 T <= 65535 and nrhs to
 * 65535 (TM_ERR_ARG beyond).                                               */
typedef enum { TM_LOOP_STD = 0, TM_LOOP_VV = 1, TM_LOOP_GEN = 2 } tm_loop_mode_t;

tm_status_t loop_contract_local(const tm_geom_t *g, const void *left, const void *right,
                                tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                                double *out, tm_stream_t s);
tm_status_t loop_contract_oneD(tm_op_t *op, const void *left, const void *right,
                               tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                               double *out, tm_stream_t s);

/* Loop contractions on the interleaved layout (Sec. 2.2, Table 2: the
 * operators of loop_contract_local / loop_contract_oneD above, same modes,
 * prefactor convention and output layout).  left_il / right_il: nrhs F16 or
 * BF16 fields in the interleaved layout (16-byte aligned, else TM_ERR_ARG);
 * right_g5 = 1 contracts gamma_5 right_il instead of right_il (the generalised
 * estimator's R = gamma_5 D_W s from the D_W s that tm_dslash_il writes);
 * out as for the standard contractions.
 * loop_contract_local_il: the products conj(L_ac) R_bc of each site as
 *   mixed-precision FMAs (exact products of the 16-bit numbers, FP32 sums).
 * loop_contract_oneD_il: per site and 16 systems, the link products of all
 *   directions as warp-level MMAs over the systems (FP32 accumulation, rounded
 *   once to the storage format), then the 4 x 4 spin products per system as
 *   MMAs over (colour, re/im) with FP32 sums over the sites; every site's
 *   neighbours staged by bounded tensor and bulk copies as in tm_dslash_il (its
 *   time-outs set the operator's flag: tm_op_check).  Needs the 18-real
 *   16-bit links (recon 18 or 0, else TM_ERR_UNSUPPORTED).
 * Results agree with the standard contractions of the same fields to the
 * 16-bit tolerance; each system's values depend on its own fields only.      */
tm_status_t loop_contract_local_il(const tm_geom_t *g, const void *left_il, const void *right_il,
                                   tm_prec_t prec, int nrhs, tm_loop_mode_t mode, int right_g5,
                                   double *out, tm_stream_t s);
tm_status_t loop_contract_oneD_il(tm_op_t *op, const void *left_il, const void *right_il, tm_prec_t prec,
                                  int nrhs, tm_loop_mode_t mode, int right_g5, double *out, tm_stream_t s);

/* Momentum-projected local loops:
 *   out[r][q][g][t] = sum_{x_t = t} exp(-i p_q . x) L_r(x)^dag (P Gamma_g) R_r(x),
 *   p_q = 2 pi (n_x / X, n_y / Y, n_z / Z),  mom = host array [n_mom][3] of (n_x, n_y, n_z)
 * (the paper computes zero-momentum loops; 1 <= n_mom <= 64, nrhs * n_mom <= 65535).
 * out: device [nrhs][n_mom][16][T][2].                                      */
tm_status_t loop_contract_local_mom(const tm_geom_t *g, const void *left, const void *right,
                                    tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                                    const int *mom, int n_mom, double *out, tm_stream_t s);

/* Same computation and result as loop_contract_local, for callers that cannot
 * allocate device memory: e.g. an application whose own memory manager has
 * reserved the GPU's memory up front, or a tight loop that must not pay for an
 * allocation on every call.  This call allocates nothing (no cudaMalloc,
 * cudaMallocAsync, cudaFree or allocating library routine).  Its reduction
 * scratch is a fixed array of 2^20 doubles (8 MiB) inside the library, which
 * every GPU that loads the library holds until the process exits; sizes that
 * need more, i.e. 64 * nrhs * T * ceil(X*Y*Z/2048) > 2^20 doubles (e.g. more
 * than 16 right-hand sides at 32^3 x 64), are rejected with TM_ERR_ARG before
 * any launch.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array: calls whose
 * kernels may overlap on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.  The paper has no
 * counterpart to this entry point; it exists for the allocation constraint
 * only.  Arguments, layouts and errors as for loop_contract_local.         */
tm_status_t loop_contract_local_noalloc(const tm_geom_t *g, const void *left, const void *right,
                                        tm_prec_t prec, int nrhs, tm_loop_mode_t mode,
                                        double *out, tm_stream_t s);

/* Truncated Solver Method combination (Sec. 2.1, Eq. 4), per component j:
 *   mean_j = (1/N_HP) sum_{i<N_HP} c (l_hp - l_lp_on_hp)_ij + (1/N_LP) sum_i c (l_lp)_ij
 *   err_j^2 = Var_i(c (l_hp - l_lp_on_hp))/N_HP + Var_i(c l_lp)/N_LP,
 * c = scale_re + i scale_im, unbiased variances, separately for re and im;
 * a variance over fewer than two sources is NaN; n_hp = 0 drops the
 * correction.  l_hp, l_lp_on_hp: [n_hp][len][2]; l_lp: [n_lp][len][2];
 * mean, err: [len][2] (err = {err_re, err_im}).  Device pointers; n_lp >= 1. */
tm_status_t tsm_combine(const double *l_hp, const double *l_lp_on_hp, int n_hp,
                        const double *l_lp, int n_lp, size_t len, double scale_re,
                        double scale_im, double *mean, double *err, tm_stream_t s);
/* The same combination (same formula and operation order per component) on
 * HOST arrays, synchronous: for per-source loops gathered on the host or across
 * processes, which are small (kilobytes per source).  Arguments as above. */
tm_status_t tsm_combine_host(const double *l_hp, const double *l_lp_on_hp, int n_hp,
                             const double *l_lp, int n_lp, size_t len, double scale_re,
                             double scale_im, double *mean, double *err);

/* Diagnostics.  tm_last_error: thread-local text of the last failure.
 * tm_launch_count: kernels this library launched so far (all threads).
 * tm_trace_enable(1): bracket every Dslash launch with CUDA events on its
 * stream and record its algorithmic bytes (every array once: per active
 * system the neighbour, centre and epilogue fields of the output sites, per
 * launch the links of all sites); the kernel itself records how many systems
 * were active.  tm_trace_read returns, since the last reset, the launches,
 * summed device milliseconds and summed algorithmic bytes of a kernel class
 * "dslash.<f64|f32|f16|bf16|ff>.<out|cgupd|resid>", "local.<prec>",
 * "oneD.<prec>", "blas.xpay", "z4_noise", "cg.graph" (exact name, or a prefix
 * ending in '*', e.g. "dslash.f16.*"); it synchronises the device.        */
const char *tm_last_error(void);
uint64_t tm_launch_count(void);
void tm_trace_enable(int on);
void tm_trace_reset(void);
tm_status_t tm_trace_read(const char *name, int *launches, double *total_ms, double *total_bytes);
/* The algorithmic flops of the same launches (recorded by the Dslash: per
 * output site and active system 1320 for the hops, plus the centre, twist and
 * epilogue terms; 0 for other classes).                                    */
tm_status_t tm_trace_read_flops(const char *name, double *total_flops);

/* Autotuning of the FP32/FP16/BF16 Dslash launch shape (this library's own;
 * the paper has no counterpart): systems per thread (1, 2, 4; for FP16/BF16
 * also 2 in packed FP32x2 arithmetic) and threads per block (32, 64, 128).  The first launch of each kind - precision, link
 * format, dagger, epilogue, parity set, centre and inverse-twist terms, half
 * volume and number of systems - times every shape on its own arguments
 * (blocking the calling thread once) and the fastest is kept for the process;
 * CG-update launches use the shape of the matching plain launch.  Results
 * never depend on the shape.  Tuning is on unless the environment sets
 * TM_TUNE=0; it is skipped while a CUDA graph is captured and when
 * TM_DSLASH_NR fixes the systems per thread.
 * tm_tune_enable(0/1) switches it at run time, tm_tune_reset forgets every
 * choice, tm_tune_count gives the number of kinds tuned, and tm_tune_get(i,
 * key[9], &nr, &block, &packed) reads entry i: key = {prec, reals per link,
 * dagger, epilogue, parity (-1 both), centre (0 none, 1 copy, 2 twisted),
 * inverse twist, half volume, systems}; packed = 1 for the FP32x2 form.    */
void tm_tune_enable(int on);
/* The FP16/BF16 Dslash with 18-real links on the tensor cores (warp-level
 * MMA: 16 systems per MMA row block, the forward and backward hops of a
 * direction in one m16n8k16 product per output spin, FP32 accumulation)
 * instead of the CUDA-core kernel.  Off unless the environment sets
 * TM_DSLASH_MMA=1; tm_dslash_mma_enable(0/1) switches it for the process
 * (between launches).  Both kernels agree with the FP64 operator to the
 * 16-bit tolerance; their bits differ (another summation order).          */
tm_status_t tm_dslash_mma_enable(int on);
void tm_tune_reset(void);
int tm_tune_count(void);
tm_status_t tm_tune_get(int i, int *key, int *nr, int *block, int *packed);

#ifdef __cplusplus
}
#endif
#endif /* TMLOOPS_H */
