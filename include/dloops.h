/*
 * dloops.h - C ABI of the GB300 (sm_103a) disconnected-loop library.
 *
 * The library computes disconnected quark loops as in "Exact calculation of
 * disconnected loops" (Alexandrou, Christaras, O Cais, Strelchenko, Lattice
 * 2010): repeated inversion of the N_f = 2 Wilson-Dirac matrix
 * M = 1 - kappa*D (Sec. 2) over point sources or diluted complex Z2 noise
 * sources (Sec. 2), followed by the loop contraction
 * L_Gamma(t) = sum_{x in t} Tr[Gamma M^{-1}(x, x)] (Sec. 3, Eq. 2) for local and
 * Gaussian-smeared sinks, and the truncated-solver-method estimate (Sec. 2).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: dims = {Lx, Ly, Lz, T}; every extent even and in [2, 256].  Site
 *   index i = x + Lx*(y + Ly*(z + Lz*t)) (x fastest).  Directions mu = 0..3 are
 *   x, y, z, t.  Space is periodic; the quark fields get the factor t_bc (+1 or
 *   -1) on hops across the time boundary.
 * Operator (the paper fixes no convention; this is the standard Wilson form
 *   with r = 1): (D psi)(x) = sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *   + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)], M = 1 - kappa*D, gamma matrices in
 *   the chiral DeGrand-Rossi basis (g5 = diag(1, 1, -1, -1)).
 * Gauge field (host): complex128 [V][4 mu][3][3], row-major 3x3 (U[a][b] at
 *   a*3+b), each complex as two doubles (re, im).
 * Spinor fields ("canonical", device): complex128 [n_rhs][V][4 spin][3 colour],
 *   i.e. 24 doubles per site, right-hand sides back to back.  Device pointers
 *   are caller-owned memory; the library never frees them and keeps no
 *   reference after the call returns.
 * Gamma basis (every loop output): 16 matrices in the order 1, g1, g2, g3, g4,
 *   g5, g5g1, g5g2, g5g3, g5g4, g1g2, g1g3, g1g4, g2g3, g2g4, g3g4.
 * Loop outputs (host): double [..][16 Gamma][T][2] (re, im), with
 *   L_Gamma(t) = sum_{x in t} eta(x)^dag Gamma phi(x).
 * Streams: every call is stream-ordered on the stream given to dl_create;
 *   calls that return host data synchronise that stream before returning.
 * Errors: every call returns a dl_status.  On error nothing is written to the
 *   host outputs; device outputs may be partially written.  No call aborts the
 *   process or traps on the device; device-side iteration loops are bounded.
 *   There is no CPU fallback: a missing or unusable GPU is DL_ECUDA.
 * Threads: separate contexts may be used from separate host threads, each on
 *   its own stream; one context is not safe for concurrent calls.
 * Environment (read when a call starts):
 *   DLOOPS_SMEAR_FP64=1       smearing in FP64 instead of float-float arithmetic
 *                             (read by dl_create);
 *   DLOOPS_CONTINUE_CYCLES=1  keep the BiCGStab search direction and shadow
 *                             residual across defect-correction cycles instead of
 *                             restarting (measured slower);
 *   DLOOPS_OUTER_DFF=0        defect-correction hops of mixed-precision solves in
 *                             FP64 instead of float-float arithmetic (float-float is
 *                             used only for tol >= 1e-11);
 *   DLOOPS_HOP_ARITH=dff      dl_apply_hop / dl_apply_m in float-float arithmetic.
 */
#ifndef DLOOPS_H
#define DLOOPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dl_status {
    DL_OK = 0,
    DL_EINVAL = 1,          /* bad argument (size, pointer, flag, lattice shape) */
    DL_ENOMEM = 2,          /* device allocation failed */
    DL_ECUDA = 3,           /* a CUDA runtime call failed (message in dl_last_error) */
    DL_NOT_CONVERGED = 4,   /* some right-hand side did not reach the tolerance */
    DL_BREAKDOWN = 5,       /* BiCGStab breakdown (rho, omega or <r0,v> vanished) */
    DL_NAN = 6,             /* a non-finite value appeared in a solve */
    DL_ESTATE = 7           /* call out of order (e.g. solve before load_gauge) */
} dl_status;

/* Precision of the Krylov iteration.  DL_PREC_F64 is a plain double-precision
 * BiCGStab; F32 and BF16 keep spinors and links in that storage type with FP32
 * arithmetic inside a defect-correction loop on FP64 fields (solution
 * accumulation and final result in FP64; the true residual in float-float
 * arithmetic, about 48 significant bits, for tol >= 1e-11, else in FP64).
 * Sec. 2: the paper's inversions use mixed-precision CG/BiCGStab. */
enum { DL_PREC_F64 = 0, DL_PREC_F32 = 1, DL_PREC_BF16 = 2 };

/* Krylov method of the inner solve.  BICGSTAB works on the even-site Schur
 * system Mhat x = bhat directly.  CGNR is conjugate gradient on the normal
 * equations Mhat^dag Mhat x = Mhat^dag bhat.  Sec. 2 names it: single-precision
 * CG to a 1e-6 tolerance for the low-precision solves of the truncated solver
 * method.  Both stop on the residual of Mhat x = bhat itself. */
enum { DL_METHOD_BICGSTAB = 0, DL_METHOD_CGNR = 1 };

/* Dilution bitmask (Sec. 2): spin (x4 inversions), colour (x3), even-odd
 * spatial partition (x2), cubic partition (x8: the vertex class
 * (x&1) + 2(y&1) + 4(z&1) of the elementary 3-cube), time (source on a single
 * timeslice; no extra inversions). */
enum { DL_DIL_SPIN = 1, DL_DIL_COLOUR = 2, DL_DIL_EVENODD = 4, DL_DIL_CUBIC = 8, DL_DIL_TIME = 16 };

/* Sink selection for loop contractions (Sec. 2: local and smeared fields).
 * DL_SUM_T, or-ed into the sink mask of dl_trace_loops, sums each loop over
 * the timeslices on the device (the total sum_x eta^dag Gamma phi). */
enum { DL_SINK_LOCAL = 1, DL_SINK_SMEARED = 2, DL_SUM_T = 4 };

typedef struct dl_ctx dl_ctx;

typedef struct dl_solve_params {
    double tol;          /* stop when ||b - M x|| / ||b|| <= tol (true residual on FP64 fields); > 0 */
    int precision;       /* DL_PREC_* */
    int max_iter;        /* cap on inner Krylov iterations summed over outer cycles */
    int fixed_iters;     /* > 0: run exactly this many inner iterations, one cycle, no
                            tolerance test (a deterministic low-precision map, as the
                            truncated solver method needs); 0: iterate to tol */
    double delta;        /* inner relative residual reduction per outer cycle (mixed
                            precision); <= 0 picks 3e-6 (F32) or 1e-3 (BF16).  A cycle
                            stops earlier once its residual meets the outer tolerance
                            with a margin of 4 */
    int max_outer;       /* cap on defect-correction cycles; <= 0 picks 60 */
    int batch;           /* right-hand sides solved together per launch (1..64, a power
                            of two for F32/BF16 >= 2); <= 0 picks 16 */
    int use_graph;       /* capture the inner iteration in CUDA graphs (1) or launch
                            directly (0) */
    int chunk;           /* inner iterations per graph launch / convergence poll; <= 0: 2 */
    int method;          /* DL_METHOD_*; 0 (BiCGStab) by default */
} dl_solve_params;

typedef struct dl_solve_stats {
    int status;          /* dl_status of this right-hand side */
    int iters;           /* inner Krylov iterations */
    int outer;           /* defect-correction cycles */
    double true_residual;/* ||b - M x|| / ||b||, full lattice, FP64 fields */
} dl_solve_stats;

typedef struct dl_smear {
    double alpha;        /* K = [(1 + alpha H)/(1 + 6 alpha)]^n_iter, H the spatial hop */
    int n_iter;
} dl_smear;

/* Timers accumulated by the context (CUDA events around each Wilson-hop
 * launch when enabled by dl_set_timing). */
typedef struct dl_timing {
    double hop_ms[4];        /* per kind: 0 low-precision plain, 1 low-precision fused
                                (xpay + reductions), 2 FP64 plain, 3 FP64 fused */
    int64_t hop_launches[4];
    double hop_bytes[4];     /* algorithmic bytes of those launches */
    int64_t kernel_launches; /* every kernel this context launched */
} dl_timing;

/* --- context -------------------------------------------------------------- */

/* Create a context for one lattice on the current CUDA device.
 * dims: {Lx, Ly, Lz, T}; t_bc: +1 periodic or -1 antiperiodic in time;
 * cuda_stream: a cudaStream_t (0 = legacy default stream).  *out receives the
 * context, owned by the caller until dl_destroy. */
int dl_create(dl_ctx **out, const int dims[4], int t_bc, void *cuda_stream);
int dl_destroy(dl_ctx *ctx);
/* Message of the last failing call on this thread (static storage). */
const char *dl_last_error(void);
const char *dl_status_string(int status);

/* Copy the gauge field U_mu(x) (Sec. 2: the SESAM links; here any SU(3)
 * field) from host memory (layout above) into the context, which keeps it in
 * even-odd site-major order in FP64, FP32 and BF16.  check_unitarity != 0
 * rejects (DL_EINVAL) links with |U U^dag - 1| > 1e-10. */
int dl_load_gauge(dl_ctx *ctx, const double *host_U, int check_unitarity);

/* Set the hopping parameter kappa of M = 1 - kappa D (Sec. 2: kappa = 0.157). */
int dl_set_kappa(dl_ctx *ctx, double kappa);

/* Clover (Sheikholeslami-Wohlert) improvement, an extension: the paper's
 * inversions use plain Wilson fermions (Sec. 2), which c_sw = 0 (the default)
 * keeps.  With c_sw != 0 the operator becomes M = A - kappa D with the
 * site-local, hermitian, gamma_5-commuting
 *   A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu],
 *   F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag)/(8i),
 * Q_{mu nu}(x) the sum of the four plaquettes of the mu-nu plane that start
 * and end at x, each traversed mu first.  A and its inverse (two 6 x 6 blocks
 * per site in the chiral basis; A in FP64, A^-1 in FP64, FP32 and BF16:
 * 3168 bytes of device memory per site) are built from the FP64 links before the next call that
 * needs them, after any change of links, kappa or c_sw.  dl_apply_m, the
 * solvers and every solve inside the loop estimators then use M; dl_apply_hop
 * is still D alone.  The even-odd solve uses the asymmetric Schur system
 * A_ee^-1 (A_ee - kappa^2 D_eo A_oo^-1 D_oe) with A^-1 applied in the inner
 * hops; the residual and tolerance remain those of b - M x.  BiCGStab only:
 * a solve with DL_METHOD_CGNR fails with DL_EINVAL, and mixed-precision clover
 * solves run their defect-correction steps in FP64.  Errors: DL_EINVAL
 * (non-finite c_sw), DL_ECUDA; an allocation failure (DL_ENOMEM) is reported
 * by the call that builds the blocks. */
int dl_set_clover(dl_ctx *ctx, double c_sw);

/* Enable (1) or disable (0) CUDA-event timing of Wilson-hop launches; read and
 * reset with dl_get_timing. */
int dl_set_timing(dl_ctx *ctx, int enable);
int dl_get_timing(dl_ctx *ctx, dl_timing *out, int reset);

/* --- sources (Sec. 2) ----------------------------------------------------- */

/* Diluted complex Z2 sources.  For noise vectors n = noise_first ..
 * noise_first + n_noise - 1, xi_n(x, alpha, a) = (s_re + i s_im)/sqrt(2) with
 * signs from Philox4x64-10 (key (seed, 0), counter (i >> 2, n, 0, 0); word
 * i & 3 belongs to site i; bits 2c and 2c+1 of that word give the real and
 * imaginary sign of component c = 3 alpha + a; a set bit means -1).  Each noise
 * vector yields K diluted sources P_k xi_n (K from the dilution mask, class
 * index k = ((k_spin*C + k_colour)*E + k_eo)*Q + k_cubic), written to
 * dev_out[(n - noise_first)*K + k] in canonical layout (complex128).  With
 * DL_DIL_TIME only timeslice t0 is kept, or n mod T when t0 < 0.  *n_rhs
 * (may be NULL) receives n_noise*K.  dev_out must hold n_noise*K*V*12 complex
 * values in the storage of `prec`: DL_PREC_F64 complex128, DL_PREC_F32
 * complex64 (two floats), DL_PREC_BF16 two bfloat16 (re, im); the value
 * +-1/sqrt(2) is rounded from FP64 to nearest (through float for BF16).  The
 * solver and the contractions take complex128 fields; the narrower outputs
 * feed callers that keep sources in working precision.  Errors: DL_EINVAL
 * (ranges, dilution bits, t0, precision, NULL output), DL_ECUDA. */
int dl_make_sources(dl_ctx *ctx, uint64_t seed, int64_t noise_first, int n_noise,
                    unsigned dilution, int t0, int prec, void *dev_out, int64_t *n_rhs);

/* Point sources e_s with s = 12*i + 3*alpha + a for s = first .. first + n - 1
 * (Sec. 1-2: the exact all-to-all diagonal needs all 12V of them), n canonical
 * fields in the storage of `prec` (as for dl_make_sources). */
int dl_make_point_sources(dl_ctx *ctx, int64_t first, int n, int prec, void *dev_out);

/* --- solver (Sec. 2) ------------------------------------------------------ */

/* Solve M x_j = b_j for n_rhs right-hand sides (canonical complex128 device
 * buffers; dev_x may not alias dev_b).  Even-odd preconditioned BiCGStab on
 * the Schur complement 1 - kappa^2 D_eo D_oe with the precision and batching of
 * *params (NULL: defaults, tol 1e-10, F32).  stats (host, may be NULL) receives
 * n_rhs entries.  Returns DL_OK if every right-hand side converged, otherwise
 * the first failing status (the solutions are still written). */
int dl_solve(dl_ctx *ctx, const void *dev_b, void *dev_x, int n_rhs,
             const dl_solve_params *params, dl_solve_stats *stats);

/* Solve M^dag x = b, via M^dag = g5 M g5 (gamma5-hermiticity). */
int dl_solve_adjoint(dl_ctx *ctx, const void *dev_b, void *dev_x, int n_rhs,
                     const dl_solve_params *params, dl_solve_stats *stats);

/* --- operators (building blocks, FP64) ------------------------------------ */

/* out = D in (Wilson hopping term, full lattice, FP64), n_rhs fields.  With
 * the environment variable DLOOPS_HOP_ARITH=dff these two operators compute in
 * float-float arithmetic (about 48 significant bits) on the same FP64 fields.
 * Mixed-precision solves use that arithmetic for their defect-correction
 * steps; the variable exposes it for testing. */
int dl_apply_hop(dl_ctx *ctx, const void *dev_in, void *dev_out, int n_rhs);
/* out = D in computed by the inner solver's low-precision Wilson hop (Sec. 2:
 * the mixed-precision inversions): both halves of `in` (canonical complex128)
 * are rounded to the storage type of `precision` (DL_PREC_F32 or DL_PREC_BF16;
 * FP64 -> float -> storage, as the solver rounds its residual), the hop runs
 * on the FP32/BF16 link copies with FP32 arithmetic in the kernel and launch
 * shape the context uses for that precision and width, and the result is
 * widened exactly to complex128 in `out`.  DL_PREC_F64 is dl_apply_hop.  It
 * exposes the reduced-precision operator so that its error against FP64 can
 * be measured.  Errors: DL_EINVAL (precision, sizes, pointers, in == out),
 * DL_ESTATE (no gauge field), DL_ENOMEM, DL_ECUDA. */
int dl_apply_hop_prec(dl_ctx *ctx, int precision, const void *dev_in, void *dev_out, int n_rhs);
/* out = M in = in - kappa D in (with clover: A in - kappa D in, dl_set_clover). */
int dl_apply_m(dl_ctx *ctx, const void *dev_in, void *dev_out, int n_rhs);
/* out = -dM/dkappa in = D in (+ c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu} in with
 * clover, formed as (in - A in)/kappa in FP64): the derivative that the
 * kappa-gradient of a loop needs (Sec. 3's loops as functions of kappa:
 * dM^-1/dkappa = M^-1 (-dM/dkappa) M^-1).  Errors as dl_apply_m, and
 * DL_EINVAL for kappa = 0 with clover. */
int dl_apply_dm_dkappa(dl_ctx *ctx, const void *dev_in, void *dev_out, int n_rhs);
/* out = A in (inverse = 0) or A^-1 in (inverse != 0), site by site in FP64:
 * the clover blocks of dl_set_clover (a copy of in without clover).  Canonical
 * complex128 fields as dl_apply_m.  Errors: DL_EINVAL (sizes, pointers,
 * in == out), DL_ESTATE (no gauge field or kappa), DL_ENOMEM, DL_ECUDA. */
int dl_apply_clover(dl_ctx *ctx, const void *dev_in, void *dev_out, int n_rhs, int inverse);
/* out = K in, Gaussian smearing (Sec. 2), restricted to timeslices
 * [t_lo, t_hi) (other timeslices of out are set to zero). */
int dl_apply_smear(dl_ctx *ctx, const void *dev_in, void *dev_out, int n_rhs,
                   const dl_smear *smear, int t_lo, int t_hi);
/* Per-timeslice spin matrices built from Gamma weights w[j][16][T] (complex,
 * host): mode 0: out(x) (+)= sum_G w[j][G][t(x)] G^dag in(x);
 * mode 1: out(x) (+)= sum_G conj(w[j][G][t(x)]) G in(x).  accumulate = 1 adds
 * to out.  (Used by the loop gradients: the adjoint source and the
 * direct term.) */
int dl_apply_gamma_weights(dl_ctx *ctx, const void *dev_in, void *dev_out, int n_rhs,
                           const double *host_w, int mode, int accumulate);

/* --- loops (Sec. 3, Eq. 2) ------------------------------------------------ */

/* Loop contraction L_Gamma(t) = sum_{x in t} eta(x)^dag Gamma phi(x) for each
 * pair (eta_j, phi_j) and all 16 Gamma (Sec. 3, Eq. 2; FP64 sums).
 * Timeslices: with t_of_rhs == NULL every pair is contracted on [t_lo, t_hi);
 * otherwise (host array of n_rhs entries) pair j only on timeslice t_of_rhs[j]
 * (time-diluted sources; t_lo, t_hi unused).  Other timeslices are zero.
 * sink: DL_SINK_LOCAL and/or DL_SINK_SMEARED; for the smeared sink eta and phi
 * are both smeared by K first (Sec. 2), on the same timeslices; smear must be
 * non-NULL.  group >= 1 must divide n_rhs: the loops of each run of `group`
 * consecutive pairs are summed (for instance the dilution classes of one noise
 * vector; group = 1 gives per-pair loops, group = n_rhs the total).
 * host_out: double [n_rhs/group][n_sinks][16][T][2] (local first); with
 * DL_SUM_T in `sink`, double [n_rhs/group][n_sinks][16][2], each value the sum
 * over the timeslices (fixed order, FP64). */
int dl_trace_loops(dl_ctx *ctx, const void *dev_eta, const void *dev_phi, int n_rhs, int sink,
                   const dl_smear *smear, int t_lo, int t_hi, const int *t_of_rhs, int group,
                   double *host_out);

/* Exact loops (Sec. 1-2: the all-to-all diagonal): solve the point sources
 * s = src_first .. src_first + n_src - 1 and accumulate
 * sum_{x in t} Tr[Gamma M^{-1}(x, x)] restricted to those sources into
 * host_out[n_sinks][16][T][2] (overwritten).  All 12V sources give the exact
 * loop.  Smeared sinks use sum over sources of (K e_s)^dag Gamma K M^{-1} e_s. */
int dl_exact_loops(dl_ctx *ctx, int64_t src_first, int64_t n_src,
                   const dl_solve_params *params, int sink, const dl_smear *smear,
                   double *host_out, dl_solve_stats *stats_sum);

/* Truncated solver method (Sec. 2, after Bali et al.): n_lp noise vectors
 * (indices 0..n_lp-1) solved with *lp, and n_hp further noise vectors
 * (n_lp..n_lp+n_hp-1) solved with both *hp and *lp;
 * mean = <L_lp> + <L_hp - L_lp>, var = s^2_lp/n_lp + s^2_diff/n_hp per Gamma
 * and timeslice, each noise vector summed over its dilution classes, and a
 * timeslice counted only for the noise vectors whose source covers it.
 * mean_out, var_out: host double [n_sinks][16][T][2] (var: real variances of
 * re and im parts).  per_noise_out (may be NULL): host double
 * [n_lp + 2*n_hp][n_sinks][16][T][2]: LP loops, then HP loops, then LP loops on
 * the HP ensemble. */
int dl_tsm_estimate(dl_ctx *ctx, uint64_t seed, int n_lp, int n_hp, unsigned dilution, int t0,
                    const dl_solve_params *lp, const dl_solve_params *hp,
                    int sink, const dl_smear *smear,
                    double *mean_out, double *var_out, double *per_noise_out);

/* Dilution study (Sec. 3, Figs. 3-4): the stochastic error of the loop
 * estimate of one diluted noise vector.  Noise vectors n = 0 .. n_noise-1 of
 * `seed` are diluted by `dilution` (K classes) and solved with *params; each
 * gives the estimate L_n[Gamma][t] = sum over its classes of
 * sum_{x in t} eta^dag Gamma phi (local sink).  With host_exact the exact loops
 * (double [16][T][2], e.g. from dl_exact_loops),
 *   sigma2[Gamma] = mean over n of |L_n[Gamma][t_n] - exact[Gamma][t_n]|^2
 * on the source timeslice t_n (t0, or n mod T when t0 < 0) for DL_DIL_TIME,
 * else the mean over n and all timeslices.  An estimate that costs N_inv
 * inversions then has the error sqrt(sigma2 K / N_inv) (the quantity plotted
 * against the number of inversions per scheme).  host_sigma2: double [16];
 * per_noise_out (may be NULL): double [n_noise][16][T][2].  The per-noise
 * loops and the mean run on the device in a fixed order.  Errors: DL_EINVAL,
 * DL_ESTATE, DL_ENOMEM, DL_ECUDA; the status of the worst solve otherwise. */
int dl_dilution_error(dl_ctx *ctx, uint64_t seed, int n_noise, unsigned dilution, int t0,
                      const dl_solve_params *params, const double *host_exact, double *host_sigma2,
                      double *per_noise_out);

/* --- two-point functions (Sec. 3, Eqs. 1 and 3) --------------------------- */

/* Momentum-projected loops.  Sec. 3 puts the momentum phases inside the
 * operators Gamma(p); with p = 2 pi n / L for integer spatial n (momenta:
 * host int [n_mom][3], 1 <= n_mom <= 256):
 *   L_Gamma(p, t) = sum_{x in t} exp(-i p.x) eta_j(x)^dag Gamma phi_j(x)
 * for the local and/or smeared sink as in dl_trace_loops.  Fields are
 * canonical complex128 device fields (n_rhs of each).  t_of_rhs (host, n_rhs
 * ints, or NULL) restricts pair j to one timeslice; otherwise all T
 * timeslices are used.  Consecutive runs of `group` (1..64, dividing n_rhs)
 * pairs are summed.  host_out: double [n_rhs/group][n_sinks][n_mom][16][T][2].
 * The device work is a per-site spin matrix, its Fourier sum over each
 * timeslice (FP64, fixed order) and the Gamma traces.  Errors: DL_EINVAL for
 * bad arguments, DL_ESTATE without a gauge field for the smeared sink,
 * DL_ENOMEM, DL_ECUDA. */
int dl_trace_loops_mom(dl_ctx *ctx, const void *dev_eta, const void *dev_phi, int n_rhs, int sink,
                       const dl_smear *smear, const int *momenta, int n_mom, const int *t_of_rhs, int group,
                       double *host_out);

/* Connected meson two-point function of a point source at src = {x, y, z, t}
 * (Eq. 1 with the source sum replaced by one point):
 *   C^{BA}(p, t) = - sum_x exp(-i p.(x - y)) Tr[S(y; x) Gamma_B S(x; y) Gamma_A],
 * evaluated as - sum_x exp(-i p.(x - y)) Tr[g5 S(x; y)^dag g5 Gamma_B S(x; y) Gamma_A]
 * through gamma5-hermiticity, with t measured from the source timeslice.
 * dev_prop: the 12 solutions of M phi_j = e_{src, alpha, a} (j = 3 alpha + a),
 * canonical complex128 [12][V][4][3] on the device (from dl_make_point_sources
 * and dl_solve).  host_out: double [n_mom][16 A][16 B][T][2] for all source
 * (A) and sink (B) operators of the Gamma basis.  For A = B = gamma5 (the
 * pion) the value is -sum_x Tr[S^dag S] < 0 in this sign convention.
 * Allocates 4 KiB per lattice site of scratch device memory (kept by the
 * context). */
int dl_meson_correlators(dl_ctx *ctx, const void *dev_prop, const int src[4], const int *momenta, int n_mom,
                         double *host_out);

/* Disconnected two-point function from per-noise loops (Eq. 3, read as the
 * product of two loop traces):
 *   D^{BA}(p, dt) = -(1 / (L^3 T)) sum_t E[L_B(p, t + dt) L_A(-p, t)],
 * with the expectation taken over ordered pairs of distinct noise vectors so
 * that no vector's noise is multiplied with itself.  host_loops: double
 * [n_noise][n_mom][16][T][2] (e.g. from dl_trace_loops_mom with one group per
 * noise vector); host_cover: unsigned char [n_noise][T], 1 where a vector's
 * loop estimates timeslice t (time dilution), or NULL for all; the list of
 * momenta must contain -p for every p.  host_out: double [n_mom][16 A][16 B][T][2]. */
int dl_disconnected(dl_ctx *ctx, const double *host_loops, const unsigned char *host_cover, int n_noise,
                    const int *momenta, int n_mom, double *host_out);

/* --- contraction without allocation --------------------------------------- */

/* The paper has no counterpart to this call.  It exists for callers that
 * cannot call cudaMalloc, so cannot create a dl_ctx: for example, code that
 * runs while a stream is being captured into a CUDA graph, host programs that
 * hand their whole device-memory budget to their own allocator, or plug-ins
 * inside another application's CUDA context.  It computes the local loops
 * L_Gamma(t) = sum_{x in t} eta_j(x)^dag Gamma phi_j(x), the same values as
 * dl_trace_loops with DL_SINK_LOCAL, without any context and without
 * allocating device or host memory.
 *
 * dev_eta, dev_phi: canonical complex128 fields, n_rhs of them, on the current
 * device; dims: {Lx, Ly, Lz, T}, each in [1, 256]; timeslices [t_lo, t_hi).
 * dev_out: device memory for double [n_rhs][16][T][2]; timeslices outside the
 * range are set to zero.  Kernels run on cuda_stream (0 = legacy default
 * stream); the call does not synchronise.
 *
 * Limit: n_rhs * (t_hi - t_lo) <= 16384.  Larger requests return DL_EINVAL with
 * a message (split them into several calls).  Per-block partial sums live in a
 * 4 MiB array of static device storage in the library's device module.  With
 * CUDA's lazy module loading that array comes into being on a device the first
 * time any kernel of the library is used there, and it is held until the
 * process exits.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing); the Gamma table is a
 * compile-time constant.  Make the first call on each device before any stream
 * capture, so that module loading does not happen during a capture.  All calls
 * share the array: calls whose kernels may overlap on the GPU (other streams,
 * other host threads) race on it and must be serialised.
 * Errors: DL_EINVAL for bad arguments or sizes beyond the limit; DL_ECUDA when
 * a CUDA error from earlier work of the calling thread is pending (reported
 * and left in place, not cleared) or when a launch fails. */
int dl_trace_loops_noalloc(const void *dev_eta, const void *dev_phi, int n_rhs, const int dims[4], int t_lo,
                           int t_hi, void *dev_out, void *cuda_stream);

/* --- low-level kernels exposed for measurement ---------------------------- */

/* Apply the even-odd hop to an internal batch of n_rhs random fields in
 * storage precision `precision`, `reps` times, and return the mean kernel time
 * in *ms (CUDA events) and its algorithmic bytes per launch in *bytes.  fused:
 * 0 the plain hop; 1 the BiCGStab hop v = y - kappa^2 D x with <rhat, v>; 2 the
 * hop t = y - kappa^2 D x with its five reductions.  Used to time the Wilson
 * hop alone. */
int dl_bench_hop(dl_ctx *ctx, int precision, int n_rhs, int fused, int reps,
                 double *ms, double *bytes);

/* Autotuner for the Wilson-hop launch shape at storage precision `precision`
 * and batch width n_rhs.  The candidates are: right-hand sides per thread R in
 * {1, 2, 4}, threads per block in {64, 128, 256}, and for FP32/BF16 the
 * kernel kind: 0 direct, 1 cp.async-prefetching, 2 bulk-copy staged, 3 direct
 * with one contiguous range of sites per (widest resident) block, 4 warp-staged
 * (one site per warp with its own ring of bulk copies; only where
 * n_rhs = 32 R, i.e. widths 32 and 64), 5 BF16 on the tensor cores (n_rhs =
 * 32 R), 6 packed FP32 arithmetic; on the paired FP32 layout
 * (DLOOPS_F32_PAIRS=1, even widths) 0, 7 and 8 (packed, uncapped and capped)
 * and 9 (packed, warp-staged; widths 32 and 64); 10 the direct FP32 kernel
 * under a wider register cap (R = 1); 11 warp-staged with two stages per warp
 * (widths 32 R, twice the warps per SM of kind 4).  Each candidate times three classes of
 * hops on random fields: the plain hop (class 0), the fused hop with <rhat, v>
 * (class 1, which also serves the other fused hops) and the fused hop with the
 * five BiCGStab reductions (class 2), in two sweeps over all candidates, and
 * the fastest is kept for each class separately (so they may use different
 * kernels); another kind replaces the direct kernel only when it is more than
 * 2% faster.  force_R / force_block > 0 and force_pf >= 0 restrict the
 * candidates (for all classes).  Solves tune their (precision, batch) on first
 * use.  *R_out, *block_out, *pf_out receive the class-2 choice and *ms_out the
 * time of one plain plus one class-2 hop (each may be NULL).  The call
 * overwrites the context's inner workspace, so make it between solves.
 * Errors: DL_EINVAL (arguments, or a kind the storage layout lacks),
 * DL_ESTATE (no gauge field), DL_ECUDA. */
int dl_tune_hop(dl_ctx *ctx, int precision, int n_rhs, int force_R, int force_block, int force_pf,
                int *R_out, int *block_out, int *pf_out, double *ms_out);
/* The launch shape the context currently uses for one class of Wilson hops
 * (cls: 0 plain, 1 fused, 2 fused with the five BiCGStab reductions; see
 * dl_tune_hop) of width n_rhs in the inner storage for `precision`:
 * right-hand sides per thread, threads per block and kernel kind (outputs may
 * be NULL).  No tuning, no GPU work.  Errors: DL_EINVAL. */
int dl_hop_shape(dl_ctx *ctx, int precision, int n_rhs, int cls, int *R_out, int *block_out, int *kind_out);
/* Set that launch shape explicitly (R in {1, 2, 4}, block in {64, 128, 256},
 * kind as dl_tune_hop; kinds 3-5, 9 and 11 take block 64 and size their own
 * blocks); the width then counts as tuned.  Errors: DL_EINVAL for a shape the
 * precision, width or storage layout does not allow. */
int dl_set_hop_shape(dl_ctx *ctx, int precision, int n_rhs, int cls, int R, int block, int kind);

/* Fused-multiply-add rate of the current device at `precision` (DL_PREC_F64 or
 * DL_PREC_F32), in TFLOP/s (2 flops per FMA), from one launch of independent
 * FMA chains over 8 blocks of 256 threads per SM on `cuda_stream` (NULL: the
 * default stream).  *ms (may be NULL) receives the kernel time.  It is the
 * arithmetic ceiling of the FP64 solve, which on this GPU class is bound by
 * FP64 issue rate rather than by memory.  Allocates and frees a scratch
 * buffer of 8 bytes per thread.  Errors: DL_EINVAL for another precision or a
 * NULL tflops, DL_ENOMEM, DL_ECUDA. */
int dl_bench_fma(int precision, void *cuda_stream, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* DLOOPS_H */
