/*
 * slar.h -- C ABI of the B300 (sm_103a) SLAR + adaptive-weight implicit LoMaC library.
 *
 * Method: "A Mass, Momentum, and Energy Conserving Semi-Lagrangian Adaptive-Rank (SLAR)
 * Method for the Vlasov-Poisson System" (arXiv 2606.29027).  The distribution function is
 * a hierarchical-Tucker (HT) tensor on a cell-centred periodic phase-space grid; each time
 * step advances it with SLAR_VP (Sec. 3.1, Eq. slarvp) and restores mass, momentum and
 * energy with the implicit adaptive-weight LoMaC correction (Sec. 3.2, Eq.
 * LoMaC_update_discrete) solved by JFNK on the BDF3/DIRK3-discretised macroscopic system
 * (Sec. 3.2.3, Eq. BE_nonlinear_system).
 *
 * Conventions shared by every entry point
 *  - Dimension order (x1..x_dx, v1..v_dv), dx = dv in {1, 2}; d = dx + dv in {2, 4}.
 *    Tree: d = 2 root{0,1}; d = 4 root{12{0,1}, 34{2,3}}.
 *  - Indices are 0-based.  Spatial fields are row-major over (x1, .., x_dx), x1 slowest;
 *    a spatial field has NX = prod_{m<dx} N[m] values.
 *  - Pointers documented "device" are plain CUDA device pointers (any allocator); pointers
 *    documented "host" are host memory.  The library never frees caller memory and keeps
 *    no caller pointer after a call returns.
 *  - All device work is enqueued on the stream given to slar_create; calls that return
 *    host values (stats, energies, exported tensors) synchronise that stream.
 *  - One context per stream; a context is not thread-safe.
 *  - Every function returns a slar_status.  On failure the context (if any) keeps a
 *    message retrievable with slar_last_error; no C++ exception crosses the ABI.
 */
#ifndef SLAR_H
#define SLAR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef int slar_status;
enum {
    SLAR_OK = 0,
    SLAR_EINVAL = 1,    /* bad argument, shape or state */
    SLAR_ENOMEM = 2,    /* device allocation failed */
    SLAR_ECUDA = 3,     /* a CUDA call failed (message has the CUDA error string) */
    SLAR_ENOCONV = 4,   /* Newton / GMRES did not reach its tolerance; state is still advanced */
    SLAR_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    SLAR_ERANK = 6,     /* warning: a rank cap was reached before eps was met, in the cross
                           approximation (rank-1 stop test unmet at the cap) or in an HSVD
                           truncation (discarded energy above the threshold at the cap); the
                           call completed and its result is valid (sl_step, slar_advect,
                           ht_truncate, init_ht) */
    SLAR_ENAN = 7       /* non-finite values detected */
};

/* precision of the SL entry evaluation (gathers + transfer-tensor contractions);
   moments, truncation, LoMaC and the Newton solve are always FP64.
   SLAR_FP32_BF16X3: FP32 gathers, transfer-tensor contractions of d = 4 trees on the tensor
   cores (tcgen05, operands split x = hi + lo into BF16, three products hi.hi + hi.lo +
   lo.hi accumulated in FP32; about 2^-16 relative per product), 128 entries per CTA;
   d = 2 trees use the FP32 path.
   SLAR_FP32_BF16X6: as SLAR_FP32_BF16X3 with the operands split x = x1 + x2 + x3 into three
   BF16 pieces and the six products x1.y1 + x1.y2 + x2.y1 + x1.y3 + x3.y1 + x2.y2 (about
   2^-24 relative per product, the FP32 evaluator's accuracy), twice the MMAs of BF16x3. */
enum { SLAR_FP64 = 0, SLAR_FP32 = 1, SLAR_FP32_BF16X3 = 2, SLAR_FP32_BF16X6 = 3 };

/* flags */
enum {
    SLAR_LOMAC = 1,        /* apply the implicit LoMaC correction every step (Sec. 3.2) */
    SLAR_FOOT_EULER = 2,   /* first-order foot (x - v tau, v + E tau) instead of RK3 */
    SLAR_PROFILE = 4,      /* CUDA events at phase boundaries (stats.phase_ms) */
    SLAR_PROFILE_EVAL = 8, /* CUDA events around every entry-evaluator launch (stats.eval_ms);
                              the cross approximation then runs as individual launches
                              instead of its captured CUDA graph */
    SLAR_PRECOND = 16,     /* BDF3 Newton-Krylov solves with a block-circulant right
                              preconditioner: the Jacobian of G (Eq. BE_nonlinear_system) is
                              probed at the initial guess with one impulse per conserved
                              component, its (dv+2) x (dv+2) Fourier-mode blocks are inverted
                              and applied mode by mode (an addition to the paper, whose JFNK is
                              unpreconditioned; the Newton stop test is unchanged).  The blocks
                              are kept over BDF3 steps and probed again at the first BDF3 step,
                              when dt changes, after 8 steps, after a failed solve, or when a
                              solve needed more than 2 GMRES iterations beyond the solve that
                              followed the last probe (stats.pc_built).  After a preconditioned
                              solve that did not converge (stats.fallback) the next 8 BDF3 steps
                              are solved by plain JFNK. */
    SLAR_LEARNED = 32,     /* warm start of the BDF3 solves from the network attached with
                              slar_attach_net: initial guess U* + s_D d(x) (kept only if its
                              residual is not larger than that of U(F*)) and a per-point block
                              B(x) = I + b(x) applied before the block-circulant
                              preconditioner; if the solve does not converge it is repeated by
                              plain JFNK from U(F*).  Implies SLAR_PRECOND. */
    SLAR_NO_AUTOTUNE = 64, /* keep the entry evaluator at 32 entries per CTA instead of the
                              autotuned tile (results then do not depend on timings) */
    SLAR_OWN_STREAM = 128, /* the context creates (and destroys) a private non-blocking stream
                              and ignores the stream argument of slar_create; see slar_stream */
    SLAR_DIRK_ONLY = 256   /* with SLAR_LOMAC: the DIRK3 step (three stages, each one SLAR_VP to
                              the stage time and one JFNK solve) every step, the DIRK coupling
                              of Sec. 3.2.3, instead of BDF3 after the two start-up steps; no
                              step-ratio bound applies */
};

typedef struct slar_config {
    int dx, dv;             /* 1,1 or 2,2 */
    int N[4];               /* points per dimension, 4 <= N <= 128 */
    double lo[4], hi[4];    /* periodic box [lo, hi) per dimension */
    double eps;             /* relative truncation tolerance eps_Base (Sec. 3.1) */
    int rank_cap;           /* maximum HT rank, <= 64 */
    double newton_tol;      /* Newton tolerance on ||G||_inf relative to max(1,||U^n||_inf) */
    double krylov_tol;      /* GMRES relative tolerance */
    int krylov_restart;     /* GMRES restart length, <= 64 */
    int newton_max;         /* Newton iteration cap */
    int krylov_max;         /* Krylov iterations cap per Newton step */
    int precision;          /* SLAR_FP64 or SLAR_FP32 */
    int flags;              /* SLAR_LOMAC | SLAR_FOOT_EULER */
    double delta_floor;     /* positivity floor of the adaptive weight (Supp. B.1) */
    int aca_block;          /* fibres per cross-approximation step: 0 or 1 = partial pivoting
                               (one row and one column fibre per step); 2..8 = block cross
                               approximation: the b rows of largest residual of the latest
                               column are sampled at once, pivots are taken in them in order,
                               their columns are sampled at once (an addition: a rank-level
                               parallel variant of the paper's HTACA).  Replayed pivots always
                               take the one-fibre path (the approximation depends on the pivots
                               only). */
    int interp_order;       /* 0 or 2: the paper's quadratic stencil (Eq.
                               1d_quadratic_interp_weight); 4: quartic centred Lagrange weights
                               on the five-point stencil {j-2, ..., j+2} in the leaf gathers, the
                               field interpolation of the feet and the LoMaC correction (the
                               higher-order option noted after Eq. tp_interp).  Order 4 needs
                               SLAR_FP64 entries and N >= 5 in every dimension. */
} slar_config;

typedef struct slar_stats {
    long long entries;      /* SL entries sampled by the cross approximation this step */
    int ranks[6];           /* HT ranks of F* after truncation: leaves, then r12, r34 */
    int aca_rank[9];        /* cross-approximation rank of each SLAR call this step */
    int n_slar;             /* number of SLAR calls this step (3, or 9 in a DIRK3 step) */
    int newton, krylov;     /* Newton and GMRES iterations this step */
    double residual;        /* final ||G||_inf */
    int converged;          /* 1 if every Newton solve met its tolerance */
    double field_energy;    /* W = 1/2 sum |E|^2 dx^dx of the new state */
    double totals[4];       /* mass, momentum (dv components), energy of U^{n+1} */
    double eval_ms;         /* SLAR_PROFILE_EVAL: summed device time of the evaluator launches */
    double eval_flop;       /* algorithmic flops of the sampled entries this step */
    long long launches;     /* kernels this library launched during the step */
    double phase_ms[6];     /* SLAR_PROFILE: device time of cross approximation, truncation,
                               fields/moments, LoMaC closure, Newton-Krylov, diagnostics */
    int guess_used;         /* SLAR_LEARNED: the network's initial guess was taken */
    int fallback;           /* the preconditioned solve failed and plain JFNK was run */
    int recorded;           /* a training sample was written (slar_set_record) */
    int g_evals;            /* residual evaluations G(U) of the Newton-Krylov solves */
    int eval_tile;          /* entries per CTA of the entry evaluator (autotuned: 16, 32, 64) */
    int rank_capped;        /* cross approximations and truncations of this step that stopped at
                               the rank cap with eps unmet (non-zero: sl_step returns SLAR_ERANK) */
    int pc_built;           /* SLAR_PRECOND / SLAR_LEARNED: the block-circulant preconditioner was
                               probed this step (else the previous one was reused) */
} slar_stats;

/* Host-side view of an HT state for import/export.  Layouts (row-major):
 *   U[mu]  : N[mu] x rank[mu]                       (leaf bases, row = grid index)
 *   B12    : rank[4] x rank[0] x rank[1]  ([p][a][b]) (d = 4)
 *   B34    : rank[5] x rank[2] x rank[3]  ([q][c][e]) (d = 4)
 *   Broot  : d = 2: rank[0] x rank[1];  d = 4: rank[4] x rank[5]
 *   dC     : (dv+2) x NX   separable LoMaC correction coefficients (if has_corr)
 *   qv     : 3 x dv x N[dx]  velocity factors omega, q1, q2 per velocity dimension
 * On export with any array pointer NULL only d, N, rank and has_corr are filled. */
typedef struct slar_ht_view {
    int d;
    int N[4];
    int rank[6];
    double* U[4];
    double* B12;
    double* B34;
    double* Broot;
    int has_corr;
    double* dC;
    double* qv;
} slar_ht_view;

typedef struct slar_ctx slar_ctx;

/* Create a context: validates the grid and tolerances, allocates all device workspaces
 * on the current device.  `stream` is a cudaStream_t (NULL = legacy default stream).
 * Errors: SLAR_EINVAL, SLAR_ENOMEM, SLAR_ECUDA.  *out is NULL on failure. */
slar_status slar_create(const slar_config* cfg, void* stream, slar_ctx** out);

/* Free all device memory of the context (after synchronising its stream). */
slar_status slar_destroy(slar_ctx* ctx);

/* Last error message of the context ("" if none); static storage owned by the context. */
const char* slar_last_error(const slar_ctx* ctx);

/* Initial data (Sec. 4 test problems): F^0 = sum_t prod_mu f_{t,mu}, given as host FP64
 * `factors` of n_terms * (N[0]+..+N[d-1]) values laid out [t][mu][i].  The separable sum
 * is converted to an HT, HSVD-truncated with eps and rank_cap (Supp. B.1), the ion
 * density is set to mean(M0(F^0)) and U^0 = U(F^0).  Resets the step counter.
 * Errors: SLAR_EINVAL (n_terms < 1 or > rank limit); SLAR_ERANK (warning: the truncation
 * met its cap with eps unmet; the state is set). */
slar_status init_ht(slar_ctx* ctx, int n_terms, const double* factors);

/* Autotuning (an addition to the paper): the first SLAR call that meets a new (tree,
 * precision, grid, rank bucket 8/16/32/64) times the entry evaluator with 16, 32 and 64
 * entries per CTA on that call's check-row evaluation and keeps the fastest for the
 * process; SLAR_NO_AUTOTUNE disables it.  The tile changes the summation order of the root
 * contraction only (results agree to rounding). */

/* One full time step of size dt (flowchart of Sec. 3.2.3): SLAR_VP by the third-order
 * RK exponential integrator (Eq. slarvp; three frozen-field SLAR calls), then, with
 * SLAR_LOMAC, the moments of F*, the adaptive weight and basis (Supp. B), the JFNK solve
 * of the macroscopic system (DIRK3 for the first two steps, BDF3 after) and the update
 * F^{n+1} = F* - R(U(F*)) + R(U^{n+1}).  Steps may vary: BDF3 takes the variable-step
 * coefficients of the last three step sizes (Gear; equal steps give 18/11, -9/11, 2/11 and
 * 6/11), and a step longer than 1.4877 times the previous one is rejected after the start-up
 * (see slar_cfl_dt).  `stats` (host, may be NULL) receives the step diagnostics.
 * Errors: SLAR_EINVAL (no state, dt <= 0, step ratio above the bound), SLAR_ENAN (U^n, the Newton residual,
 * the field energy or the totals are not finite; checked before the solve and after the
 * step), SLAR_ENOCONV (Newton or GMRES did not converge within newton_max / krylov_max;
 * with SLAR_PRECOND / SLAR_LEARNED the failed solve was first repeated by plain JFNK,
 * stats.fallback = 1; the state is advanced with the last iterate), SLAR_ERANK (warning,
 * see above; the state is advanced).  SLAR_ENOCONV takes precedence over SLAR_ERANK. */
slar_status sl_step(slar_ctx* ctx, double dt, slar_stats* stats);

/* Adaptive step size for the next sl_step (Sec. 3.2.3: variable-step BDF3 for adaptive time
 * stepping; CFL numbers lambda_i = a_i dt / Delta_i per dimension as in Appendix A):
 *   dt = cfl / max_i(a_i / Delta_i),   a = max |v_m| in x_m, max |E_m| of the state's field in v_m,
 * capped at dt_max and, after the two DIRK3 start-up steps, at 1.4877 times the previous step
 * (the step-ratio bound under which variable-step BDF3 is stable, after the analysis of Li and
 * Liao that Sec. 3.2.3 cites).  dt: host output.  Synchronises the stream.
 * Errors: SLAR_EINVAL (no state, cfl or dt_max not > 0), SLAR_ENAN (non-finite field). */
slar_status slar_cfl_dt(slar_ctx* ctx, double cfl, double dt_max, double* dt);

/* HSVD truncation of the HT part of the state (Supp. B.1): orthogonalise, node Gram
 * matrices from the root down, eigendecomposition, keep per node the smallest rank with
 * discarded energy <= (eps ||F||)^2/(2d-3), capped at rank_cap.  Afterwards column 0 of
 * every leaf is the leading left singular vector of its mode matricisation.
 * Errors: SLAR_EINVAL (eps < 0, rank_cap < 1 or > 64); SLAR_ERANK (warning: the cap bound
 * with eps unmet, result valid). */
slar_status ht_truncate(slar_ctx* ctx, double eps, int rank_cap);

/* Velocity moments of the state (HT + correction) as device FP64 out[n_sel][NX]
 * (Eq. raw moments and the flux moments of Eq. macro_sys_comp).  The full table, in order:
 * M0, M1_1..M1_dv, M2, <v_a v_b f> (a <= b), <|v|^2 v_a f>;  n_mom = 5 (dv = 1) or 9
 * (dv = 2).  `mask` selects groups of it (SLAR_MOM_*; 0 = all); the selected rows are
 * written packed in table order, n_sel = 1 (M0) + dv (M1) + 1 (M2) + (n_mom - dv - 2)
 * (flux) over the selected groups.  Midpoint quadrature in v (Supp. B.1).
 * Errors: SLAR_EINVAL (null pointer, unknown mask bits, no state). */
enum { SLAR_MOM_M0 = 1, SLAR_MOM_M1 = 2, SLAR_MOM_M2 = 4, SLAR_MOM_FLUX = 8, SLAR_MOM_ALL = 15 };
slar_status moments(slar_ctx* ctx, unsigned mask, double* out_dev);

/* Adaptive-weight LoMaC update of the current state treated as F* (Sec. 3.2.2,
 * Supp. B): weight from column 0 of the velocity leaves, weighted Gram-Schmidt, then
 * F <- F - R(U(F)) + R(U_target).  U_target: device FP64 [dv+2][NX] = (n, m_1..m_dv, e).
 * The state's HT must carry no correction yet.  Afterwards U(F) = U_target. */
slar_status lomac_correct(slar_ctx* ctx, const double* U_target_dev);

/* Spectral Poisson solve (Eq. Poisson, Eq. Efromphi): -Lap(phi) = rho, E = -grad(phi),
 * W = 1/2 sum |E|^2 dx^dx.  rho: device [NX]; E: device [dx][NX]; phi: device [NX] or NULL;
 * energy: host scalar or NULL. */
slar_status poisson_field(slar_ctx* ctx, const double* rho_dev, double* E_dev, double* phi_dev,
                          double* energy);

/* Entries of the state (HT + correction) at n grid tuples idx_dev (device int32 [n][d]);
 * out_dev: device FP64 [n].  Evaluated in the context's precision. */
slar_status ht_eval(slar_ctx* ctx, long long n, const int* idx_dev, double* out_dev);

/* The local SL-FD entry evaluator (Sec. 3.1, Eq. SL_basic_formulation, Eq. tp_interp in
 * HT form): for each tuple, the backward foot of the frozen-field characteristic over
 * tau (dx/dt = v, dv/dt = -E(x)), quadratic Lagrange weights per dimension
 * (Eq. 1d_quadratic_interp_weight), gathers of three leaf rows and the contraction up the
 * tree.  E_dev: device FP64 [dx][NX].  Output device FP64 [n]. */
slar_status sl_eval(slar_ctx* ctx, double tau, const double* E_dev, long long n, const int* idx_dev,
                    double* out_dev);

/* One SLAR call (Sec. 3.1): cross approximation of the SL-updated tensor from sampled row
 * and column fibres of the (x | v) matricisation, exact HT embedding, HSVD truncation;
 * the state's HT is replaced by the result (its correction is consumed).  aca_rank and
 * entries (host, may be NULL) receive the cross rank and the number of sampled entries. */
slar_status slar_advect(slar_ctx* ctx, double tau, const double* E_dev, int* aca_rank,
                        long long* entries);

/* Replay mode for the cross approximation: the next SLAR calls take their (row, column)
 * pivots from `pivots` (host int32 [n_calls][kmax][2], -1 ends a call's list) instead of
 * choosing them.  n_calls = 0 switches replay off. */
slar_status slar_set_pivot_replay(slar_ctx* ctx, int n_calls, int kmax, const int* pivots);

/* Copy the HT state (and correction) out to / in from host memory (see slar_ht_view). */
slar_status ht_export(slar_ctx* ctx, slar_ht_view* view);
slar_status ht_import(slar_ctx* ctx, const slar_ht_view* view);

/* Checkpoint and restore of a run (Sec. 3.2.3: everything the next step reads).  The file
 * (host byte order, written by slar_checkpoint at `path`, overwritten if present) holds the
 * FP64 HT factors of F^n and its LoMaC correction, U^n, U^{n-1}, U^{n-2}, the ion density,
 * the step counter (which selects DIRK3 start-up or BDF3), the sizes of the previous two
 * steps (variable-step BDF3), the FP64 eigenbases that the next
 * truncation starts its Jacobi sweeps from, and the parameters of the attached network (if
 * any).  slar_restore loads it into a context created with the same grid and box (else
 * SLAR_EINVAL); the state is FP64 in every precision, so the run may resume in another entry
 * precision.  The network parameters are loaded only if a network of the same size is
 * attached.  A restored FP64 run continues bit for bit like the run that wrote the file
 * (same process: the autotuned evaluator tile is kept per process) with the paper's plain
 * JFNK; with SLAR_PRECOND the block-circulant preconditioner is not saved and the next BDF3
 * step probes it again, so the Newton iterates may differ from the straight run's (the
 * converged U^{n+1} agree to the Newton tolerance).  Both calls synchronise
 * the context stream.  Errors: SLAR_EINVAL (no state, file cannot be opened / read /
 * written, wrong magic or version, mismatch), SLAR_ECUDA. */
slar_status slar_checkpoint(slar_ctx* ctx, const char* path);
slar_status slar_restore(slar_ctx* ctx, const char* path);

/* Conserved variables U^n (device FP64 [dv+2][NX]) and the ion density. */
slar_status slar_get_conserved(slar_ctx* ctx, double* U_dev, double* n_i);
slar_status slar_set_conserved(slar_ctx* ctx, const double* U_dev, double n_i);

/* Allocation-free spectral Poisson solve for callers that cannot allocate device memory:
 * a host framework that owns a fixed, pre-reserved device pool and does not let libraries
 * allocate, or code running where a cudaMalloc is not permitted at that point.  The paper has
 * no counterpart of this entry point; it computes what poisson_field computes, without a
 * context.
 *   dx in {1, 2}; N[m] a power of two <= 128; L[m] > 0 the period of dimension m;
 *   rho_dev: device [NX]; E_dev: device [dx][NX]; phi_dev: device [NX] or NULL;
 *   energy: host scalar or NULL; when non-NULL the call copies the energy back and
 *   synchronises `stream`, with NULL it only enqueues work;
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Scratch (1 MiB of spectra plus twiddle and wavenumber tables) is a set of file-scope
 * static __device__ arrays that every GPU loading the library holds until process exit;
 * this call allocates nothing (no cudaMalloc/cudaFree).  The first call on a device looks
 * up the arrays' device addresses (cudaGetSymbolAddress), so make that first call before
 * any stream capture.  All calls share the arrays: every call rewrites the twiddle and
 * wavenumber tables as well as the spectra, so calls that overlap on the GPU (several
 * streams or threads) race, even when their grids differ.  Returns SLAR_EINVAL for sizes
 * beyond the maximum or bad arguments, SLAR_ECUDA if a CUDA call fails. */
slar_status slar_poisson_field_static(int dx, const int* N, const double* L, const double* rho_dev,
                                      double* E_dev, double* phi_dev, double* energy, void* stream);

/* ---------------------------------------------------------------------------------------
 * Learned JFNK warm start (an addition to the paper's method).  A network of four periodic
 * 3x3 convolutions on the spatial grid, FP32, channels 2m -> H -> H -> H -> m + m*m
 * (m = dv + 2, H <= 32 hidden channels, tanh after the first three layers):
 *   input  x[2m][NX]: the fluctuations of U^n about their means (= -rho, -J, e for the
 *          electron moments of Sec. 2), each divided by its RMS over the grid, then
 *          U* - U^n (U* = U(F*), the moments after SLAR_VP), each divided by its RMS s_D;
 *   output y[m + m*m][NX]: d (guess U* + s_D d) and b, the per-point block B = I + b
 *          (row-major m x m per point).
 * Parameters are one flat FP32 vector: per layer W (Cout, Cin, 3, 3) row-major, then the
 * bias (Cout).  A convolution is the periodic cross-correlation
 *   out[o][i][j] = bias[o] + sum_c sum_{p,q=-1..1} W[o][c][p+1][q+1] in[c][i+p][j+q].
 * Training sample (FP32, written by slar_set_record, n_probes = S >= 1), consecutive:
 *   x[2m][NX] | t[m][NX] = (U^{n+1} - U*) / s_D | v[S][m][NX] | w[S][m][NX]
 * with w_s = J P v_s (J the Jacobian of G and P the block-circulant preconditioner, both
 * at U*; v_0 = -G(U*) scaled to unit RMS per component, v_s>0 random signs from
 * SplitMix64).  Loss per sample, averaged over the batch:
 *   mean_x,c (d - t)^2  +  mean_s,x,c ((B w_s - v_s))^2.
 * ------------------------------------------------------------------------------------- */
typedef struct slar_net slar_net;

/* Number of FP32 parameters of a network for m conserved variables, H hidden channels. */
slar_status slar_net_param_count(int m, int hidden, long long* out);

/* Floats of one training sample on a grid of nx points with n_probes probe pairs. */
slar_status slar_sample_floats(int m, int nx, int n_probes, long long* out);

/* Create a network for grids n0 x n1 (n1 = 1 in one dimension; n0, n1 powers of two
 * <= 128), up to max_batch samples per training step, parameters zero, work on `stream`
 * (cudaStream_t, NULL = legacy default stream).  Errors: SLAR_EINVAL, SLAR_ENOMEM. */
slar_status slar_net_create(int m, int hidden, int n0, int n1, int max_batch, void* stream,
                            slar_net** out);
slar_status slar_net_destroy(slar_net* net);

/* Copy the parameters in (host FP32 [n], n = slar_net_param_count; also resets the Adam
 * moments and step counter) or out (synchronises the stream). */
slar_status slar_net_set_params(slar_net* net, const float* theta_host, long long n);
slar_status slar_net_get_params(slar_net* net, float* theta_host, long long n);

/* Inference: x_dev device FP32 [batch][2m][NX] -> y_dev device FP32 [batch][m + m*m][NX]. */
slar_status slar_net_forward(slar_net* net, const float* x_dev, int batch, float* y_dev);

/* Mean loss over the samples idx_dev[0..batch) (device int32) of the sample array
 * samples_dev (device FP32, sample k at k * slar_sample_floats) and its gradient with
 * respect to the parameters.  loss: host scalar or NULL; grad_dev: device FP32 [n] or
 * NULL.  With a non-NULL loss the call synchronises the stream. */
slar_status slar_net_loss_grad(slar_net* net, const float* samples_dev, int n_probes,
                               const int* idx_dev, int batch, double* loss, float* grad_dev);

/* One Adam step (Kingma and Ba 2015; beta1 0.9, beta2 0.999, epsilon 1e-8, bias-corrected)
 * with learning rate lr on the mean loss of the given samples. */
slar_status slar_net_train_step(slar_net* net, const float* samples_dev, int n_probes,
                                const int* idx_dev, int batch, float lr, double* loss);

/* Use `net` (NULL detaches) for the SLAR_LEARNED warm start of the context; the network's
 * m and grid must match the context.  The context keeps the pointer until detached. */
slar_status slar_attach_net(slar_ctx* ctx, slar_net* net);

/* Write the training sample of the next BDF3 step to sample_dev (device FP32,
 * slar_sample_floats(dv+2, NX, n_probes) floats; NULL cancels).  The random probe signs
 * come from SplitMix64 seeded with `seed` and the step index.  One-shot: call again for
 * the next step.  Recording costs n_probes + dv + 2 extra residual evaluations. */
slar_status slar_set_record(slar_ctx* ctx, float* sample_dev, int n_probes,
                            unsigned long long seed);

/* Measured FMA throughput of the current GPU in TFLOP/s (2 flops per FMA): a kernel of
 * eight independent FMA chains per thread, iters x 128 FMAs each, 8 CTAs of 256 threads per
 * SM, in double (fp64 = 1) or float (fp64 = 0), timed with CUDA events on `stream`
 * (cudaStream_t; synchronised).  The ALU denominators of the entry evaluator's roofline.
 * Errors: SLAR_EINVAL (iters outside [1, 2^24]), SLAR_ECUDA. */
slar_status slar_fma_peak(int fp64, int iters, double* tflops, void* stream);

/* Ensemble step: advance n independent contexts (uneven grids, ranks and tolerances
 * allowed) by one step each, dts[i] for context i, concurrently.  Each context's work stays
 * on its own stream, so the contexts must have pairwise distinct streams; up to `threads`
 * host threads drive them (a context is only ever touched by one thread).  stats: host
 * array of n or NULL.  Returns SLAR_OK, or after every context has finished its step the
 * status of the first context (in index order) that failed. */
slar_status slar_ensemble_step(slar_ctx** ctxs, int n, const double* dts, int threads, slar_stats* stats);

/* Total number of kernels launched by this library in this process (all contexts). */
slar_status slar_launch_count(long long* out);

/* The stream the context works on (the caller's, or its own with SLAR_OWN_STREAM). */
slar_status slar_stream(const slar_ctx* ctx, void** stream);

/* Test hook of the bounded device-side waits (no counterpart in the paper): a kernel waits,
 * with the same bounded poll loop as the tensor-core evaluator's mbarrier waits, for a phase
 * that never completes, and gives up after `polls` polls (1 <= polls <= 2^22) instead of
 * hanging.  status_dev: device int that receives 1 (gave up) or 0.  Work on `stream`
 * (cudaStream_t), synchronised.  Returns SLAR_ETIMEOUT when the wait gave up -- the CUDA
 * context stays usable -- SLAR_EINVAL for a bad argument, SLAR_ECUDA on a CUDA error. */
slar_status slar_wait_probe(long long polls, int* status_dev, void* stream);

/* Number of moments returned by `moments` and the spatial size NX. */
slar_status slar_sizes(const slar_ctx* ctx, int* n_mom, int* nx);

#ifdef __cplusplus
}
#endif
#endif /* SLAR_H */
