/*
 * lqcd.h -- C ABI of the GB300 (sm_103a) Wilson-clover solver library.
 *
 * The library implements the solver hot path of Marinkovic & Schaefer,
 * "Comparison of the mass preconditioned HMC and the DD-HMC algorithm for
 * two-flavour QCD" (Lattice 2010):
 *   - the O(a)-improved Wilson-clover operator D(m) of Eq. 1,
 *   - its even-odd Schur complement Dhat = D_ee - D_eo D_oo^-1 D_oe (Eq. 2),
 *   - the clover term, its inverse and log det (Eq. 1, Eq. 4),
 *   - the Schwarz (SAP) preconditioner and the locally deflated GCR solver
 *     named in Sec. 3-4 (Table 1), and the solution of Dhat psi = eta through
 *     a full-lattice solve (Eq. 5),
 *   - the Hasenbusch operator W(dm) = Q_S + dm and its solves (Eq. 3-4), the
 *     chronological initial guess (Sec. 2) and the DD-HMC block solves by
 *     BiCGstab on Dirichlet blocks (Sec. 3),
 *   - a batched solver for several lattices in one set of launches, and a
 *     learned gauge-equivariant preconditioner usable inside the GCR.
 *
 * Conventions (shared by every entry point):
 *   Lattice   T x L1 x L2 x L3, every extent even; x0 is time and the slowest
 *             coordinate: site = x3 + L3*(x2 + L2*(x1 + L1*x0)).
 *   Parity    a site is even when x0+x1+x2+x3 is even.  A half-lattice
 *             ("even" or "odd") field lists the sites of that parity in
 *             increasing site order (rank r holds site 2r or 2r+1).
 *   Spinor    canonical layout [site][spin 4][colour 3][re,im]; LQCD_F64
 *             uses double, LQCD_F32 and LQCD_F16S float.  nrhs fields are stored one after
 *             the other ([rhs][site]...).
 *   Links     [site][mu 0..3][row 3][col 3][re,im] double, forward links
 *             U_mu(x), SU(3); the gauge field is periodic.
 *   Gamma     chiral basis, gamma5 = g0 g1 g2 g3 = diag(1,1,-1,-1),
 *             g0 = [[0,-1],[-1,0]], gk = [[0,-i s_k],[i s_k,0]] (2x2 blocks).
 *   Operator  D = (4+m0) + c_sw sum_{mu,nu} (i/4) sigma_{mu nu} Fhat_{mu nu}
 *                 - 1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu)
 *                               + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)],
 *             m0 = 1/(2 kappa) - 4, sigma = (i/2)[g_mu, g_nu],
 *             Fhat = (Q - Q^dag)/8 with Q the four plaquette leaves at x.
 *             The fermion field is antiperiodic in time when
 *             geom.antiperiodic_t != 0: hops across x0 = T-1 <-> 0 carry -1.
 *   Pointers  every field pointer is a caller-owned DEVICE buffer (e.g. a
 *             torch tensor); the library copies what it keeps.  All work is
 *             enqueued on the context's stream; calls that return host
 *             scalars synchronise that stream.
 *   Errors    every entry point returns an lqcd_status; nothing aborts, traps
 *             or throws.  lqcd_last_error() gives a one-line reason.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#if defined(__GNUC__)
#define LQCD_API __attribute__((visibility("default")))
#else
#define LQCD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lqcd_ctx lqcd_ctx;

typedef enum {
    LQCD_OK = 0,
    LQCD_ERR_ARG = 1,              /* invalid argument, size or pointer */
    LQCD_ERR_CUDA = 2,             /* a CUDA call failed */
    LQCD_ERR_NOMEM = 3,            /* device allocation failed */
    LQCD_ERR_SINGULAR_CLOVER = 4,  /* |pivot| < 1e-12 max|A| in a 6x6 clover block */
    LQCD_ERR_NOT_CONVERGED = 5,    /* iteration limit reached; best iterate returned */
    LQCD_ERR_BREAKDOWN = 6,        /* zero norm in Gram-Schmidt / MinRes / CG */
    LQCD_ERR_NAN = 7,              /* non-finite residual */
    LQCD_ERR_TIMEOUT = 8,          /* a bounded device-side wait expired */
    LQCD_ERR_STATE = 9             /* call out of order (no gauge field, no clover, no subspace) */
} lqcd_status;

typedef enum {
    LQCD_F64 = 0,   /* double storage and arithmetic */
    LQCD_F32 = 1,   /* float storage and arithmetic, SU(3) links stored as 2 rows */
    LQCD_F16S = 2,  /* half storage with one float scale per site and field, float arithmetic */
    LQCD_BF16 = 3   /* bfloat16 storage, tensor-core products, float accumulation (network only) */
} lqcd_prec;

typedef struct {
    int T, L1, L2, L3;
    int antiperiodic_t;
} lqcd_geom;

/* ------------------------------------------------------------------ context */

/* Create a context for one lattice.  stream: a cudaStream_t (NULL = legacy
 * default stream) on which all work of this context is enqueued.
 * Errors: LQCD_ERR_ARG for odd or non-positive extents or V > 2^31 / 4. */
LQCD_API lqcd_status lqcd_create(const lqcd_geom *geom, void *stream, lqcd_ctx **out);
LQCD_API lqcd_status lqcd_destroy(lqcd_ctx *ctx);
LQCD_API const char *lqcd_last_error(const lqcd_ctx *ctx);
/* Number of kernels this context has launched so far (instrumentation). */
LQCD_API long lqcd_kernel_launches(const lqcd_ctx *ctx);
/* Change the stream used by later calls. */
LQCD_API lqcd_status lqcd_set_stream(lqcd_ctx *ctx, void *stream);

/* Copy the gauge field (canonical layout, FP64, device) into the context and
 * derive its FP32 / FP16 copies.  Invalidates the clover term and any
 * deflation subspace.  (Eq. 1: U enters D through the hops and Fhat.) */
LQCD_API lqcd_status lqcd_set_gauge(lqcd_ctx *ctx, const double *U_dev);

/* Build Fhat from the clover leaves, A(x) = (4+m0) + c_sw (i/4) sum sigma Fhat
 * as two 6x6 Hermitian blocks per site, and invert every block in FP64 by LU
 * with partial pivoting (Eq. 1; the log det enters S_eff in Eq. 4).
 * logdet_ee / logdet_oo (host pointers, may be NULL) receive
 * sum over even / odd sites of log|det A(x)|.
 * Errors: LQCD_ERR_STATE without gauge field, LQCD_ERR_SINGULAR_CLOVER. */
LQCD_API lqcd_status lqcd_clover_invert(lqcd_ctx *ctx, double kappa, double csw, double *logdet_ee,
                               double *logdet_oo);

/* out = A(x) in (inverse = 0) or A(x)^-1 in (inverse = 1) on the sites of one
 * parity; in, out: canonical FP64 half-lattice spinors (Eq. 1 / Eq. 2). */
LQCD_API lqcd_status lqcd_apply_clover(lqcd_ctx *ctx, int parity, int inverse, const double *in_dev,
                              double *out_dev);

/* -------------------------------------------------------------- operators */

/* out = D in on the full lattice (Eq. 1).  in, out: nrhs canonical full
 * spinor fields of precision prec (F64: double; F32 and F16S: float, the
 * F16S operator storing every field in half precision with a per-site scale
 * and computing in float).  in != out. */
LQCD_API lqcd_status lqcd_apply_D(lqcd_ctx *ctx, lqcd_prec prec, const void *in_dev, void *out_dev,
                         int nrhs);

/* out_e = Dhat in_e = A_ee in_e - H_eo A_oo^-1 H_oe in_e (Eq. 2) on even
 * fields; in, out: nrhs canonical even spinor fields of precision prec. */
LQCD_API lqcd_status lqcd_apply_Dhat(lqcd_ctx *ctx, lqcd_prec prec, const void *in_dev, void *out_dev,
                            int nrhs);

/* Native (device-private, resident) layout for repeated applications.
 * A native half-lattice field of precision prec and nrhs right-hand sides is
 * lqcd_native_bytes(ctx, prec, 1, nrhs) bytes (a full field: nsub = 2, the
 * even half first).  Layout, for sites s of one parity, rhs k:
 *   F64:  double2 at [(k*12 + c) * Vh + s], c = 3*spin+colour
 *   F32:  float4  at [(k*6 + q) * Vh + s],  q-th group of 4 reals of the site
 *   F16S: per half field (one parity, one rhs) uint4 (8 halves = 4 complex)
 *         at [q * Vh + s], q = 0..2, then float scale[s]: value = half * scale,
 *         scale = largest |real component| of the site (52 bytes per site).
 *         The F16S operators read FP16 copies of the links and clover term.
 * Pack / unpack convert between canonical and native fields. */
LQCD_API size_t lqcd_native_bytes(const lqcd_ctx *ctx, lqcd_prec prec, int nsub, int nrhs);
LQCD_API lqcd_status lqcd_pack(lqcd_ctx *ctx, lqcd_prec prec, int nsub, const void *canon_dev,
                      void *native_dev, int nrhs);
LQCD_API lqcd_status lqcd_unpack(lqcd_ctx *ctx, lqcd_prec prec, int nsub, const void *native_dev,
                        void *canon_dev, int nrhs);
/* Dhat / D on native fields: the benchmarked kernels, no layout conversion. */
LQCD_API lqcd_status lqcd_apply_Dhat_native(lqcd_ctx *ctx, lqcd_prec prec, const void *in_dev,
                                   void *out_dev, int nrhs);
LQCD_API lqcd_status lqcd_apply_D_native(lqcd_ctx *ctx, lqcd_prec prec, const void *in_dev, void *out_dev,
                                int nrhs);

/* Dhat on native fields exactly as lqcd_apply_Dhat_native (FP64, FP32 or
 * F16S; the same kernels and launch shapes, so the results are bitwise those
 * of lqcd_apply_Dhat_native), except that the
 * odd-site intermediate A_oo^-1 H_oe in_e lives in a fixed device array
 * compiled into the library instead of the context's workspace, so that the
 * call never allocates device memory.  The paper has no counterpart: it is
 * for callers that must not allocate during their own run, e.g. an HMC driver
 * that has handed the rest of the device to its memory pool, or code that
 * cannot afford the device-wide synchronisation an allocation can imply.
 * Limit: native_half_bytes(prec) * nrhs <= LQCD_DHAT_STATIC_SCRATCH_BYTES
 * (32 MiB: one FP32 right-hand side of a 48x24^3 lattice); larger requests,
 * and any precision other than FP64, FP32 and F16S, return LQCD_ERR_ARG
 * before any work.  The array is one per device and per
 * process: calls that overlap in time (other streams, host threads or
 * contexts on the same device) share it and race.  The first call on a device
 * looks up the array's device address (and, for a new shape, the autotuner may
 * time launch shapes); make that first call before any stream capture.
 * Nothing in the array needs to start at zero: every odd site of every
 * right-hand side is written before it is read. */
#define LQCD_DHAT_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
LQCD_API lqcd_status lqcd_apply_Dhat_native_static(lqcd_ctx *ctx, lqcd_prec prec, const void *in_dev,
                                                   void *out_dev, int nrhs);

/* ---------------------------------------------------------------- tuner */

/* Autotuner of launch shapes and kernel forms (the paper has no counterpart;
 * the kernels' results do not depend on the choice).  The first call with a
 * new key -- kernel, mode, precision, number of right-hand sides, lattice
 * extents, GPU name -- times every candidate (stencil: occupancy variant,
 * CTA shape, fields per thread, kernel form; SAP: clover staged in shared
 * memory or read through L1, timed over the sweeps of the first
 * application; batched solver: tile size) with CUDA events on the context's
 * stream, keeps the fastest and appends it to the cache file
 * $LQCD_TUNE_CACHE (default $HOME/.cache/lqcd_tune.json; one line per key:
 * "key": [variant, tx, ty, microseconds, fields per thread, kind]), so later
 * processes skip the search.  Such a first call synchronises the stream and
 * must not be inside a stream capture.  LQCD_TUNE=0 disables the search
 * (defaults are used); LQCD_TUNE_VERBOSE=1 prints every timed candidate on
 * stderr.  lqcd_tune_reset forgets the choices held in memory; the next
 * lookup reads the cache file again.  Always LQCD_OK. */
LQCD_API lqcd_status lqcd_tune_reset(void);

/* -------------------------------------------------------------------- SAP */

typedef struct {
    int bs[4];       /* block extents (even, dividing the lattice); 4,4,4,4 */
    int ncy;         /* Schwarz cycles (each: both block colours) */
    int nmr;         /* MinRes steps per block visit */
    lqcd_prec prec;  /* block-solve precision */
} lqcd_sap_params;

/* psi = M_sap eta: Schwarz alternating procedure on the block colours with
 * even-odd block MinRes (the Schwarz preconditioner of Sec. 3-4).
 * eta, psi: canonical FP64 full spinors.  Errors: LQCD_ERR_ARG for a block
 * shape that does not tile the lattice. */
LQCD_API lqcd_status lqcd_sap(lqcd_ctx *ctx, const lqcd_sap_params *p, const double *eta_dev,
                     double *psi_dev);

/* -------------------------------------------------------------- deflation */

typedef struct {
    int bs[4];        /* deflation block extents; 4,4,4,4 */
    int Ns;           /* subspace vectors per block (<= 32) */
    int ninv;         /* SAP inverse-iteration passes */
    int ncy, nmr;     /* SAP parameters used in the passes */
    lqcd_prec prec;   /* SAP precision used in the passes */
    double coarse_tol;/* relative residual of the little-Dirac solve */
    int coarse_nkv;   /* GCR Krylov length of the little-Dirac solve */
    int coarse_nmx;   /* iteration limit of the little-Dirac solve */
    lqcd_prec coarse_prec; /* arithmetic of the little-Dirac solve: LQCD_F64, or LQCD_F32
                              (operator, block-Jacobi inverse, Krylov vectors and
                              Gram-Schmidt in float; GCR scalars and the sums of the
                              per-CTA partial inner products in FP64).  With LQCD_F32
                              coarse_tol must be >= 1e-6, else LQCD_ERR_ARG */
    lqcd_prec build_sap_prec; /* LQCD_F16S: the inverse-iteration SAP of an FP32 subspace runs in
                                 FP16 with per-site scale (each pass converts the fields to F16S
                                 and back); any other value: the SAP runs in prec */
    int coarse_eo;    /* nonzero: with the FP32 little operator and an even number (>= 2) of
                         blocks in every direction, solve its even-odd (block-colour) Schur
                         complement Dinv_e (A_ee - A_eo A_oo^-1 A_oe) and reconstruct the odd
                         blocks; coarse_tol then applies to the Schur system */
} lqcd_dfl_params;

/* Build the deflation subspace ("locally deflated" solver, Sec. 3-4,
 * Table 1): v_l <- M_sap v_l, normalised, ninv times; block Gram-Schmidt on
 * every block; little Dirac operator A_{(L k),(L' l)} = <phi^L_k, D phi^L'_l>
 * (FP64 arithmetic for an FP64 subspace, FP32 products with FP64 sums over
 * warps for an FP32 one).
 * v0_dev: Ns canonical FP64 full fields (the random start vectors; the
 * caller draws them).  Requires lqcd_clover_invert. */
LQCD_API lqcd_status lqcd_dfl_build(lqcd_ctx *ctx, const lqcd_dfl_params *p, const double *v0_dev);
/* Export: the block-orthonormal fields (Ns canonical FP64 full fields) and
 * the little operator as [nblk][9][Ns][Ns] complex (entry j of block b couples
 * to the neighbour reached by direction j: 0 self, 1+2mu: +mu, 2+2mu: -mu;
 * hops that stay in the block are part of entry 0). */
LQCD_API lqcd_status lqcd_dfl_export(lqcd_ctx *ctx, double *phi_dev, double *A_dev);
/* c = Pi^dag in (in: canonical FP64 full field; c: nblk*Ns complex),
 * out = Pi c, out = A c, and the coarse solve A c = b (plain FP64 GCR). */
LQCD_API lqcd_status lqcd_dfl_project(lqcd_ctx *ctx, const double *in_dev, double *c_dev);
LQCD_API lqcd_status lqcd_dfl_expand(lqcd_ctx *ctx, const double *c_dev, double *out_dev);
LQCD_API lqcd_status lqcd_dfl_little_apply(lqcd_ctx *ctx, const double *c_dev, double *out_dev);
LQCD_API lqcd_status lqcd_dfl_coarse_solve(lqcd_ctx *ctx, const double *b_dev, double *c_dev, int *iters);
/* Counters of the little-Dirac solves since the subspace was built (host
 * pointers; instrumentation).  Errors: LQCD_ERR_STATE without a subspace. */
LQCD_API lqcd_status lqcd_dfl_stats(const lqcd_ctx *ctx, long *coarse_solves, long *coarse_iters);
/* phi = M_dfl rho = M_sap(rho - D Pi A^-1 Pi^dag rho) + Pi A^-1 Pi^dag rho. */
LQCD_API lqcd_status lqcd_dfl_precond(lqcd_ctx *ctx, const lqcd_sap_params *sap, const double *rho_dev,
                             double *phi_dev);

/* ----------------------------------------------------------------- solvers */

typedef enum {
    LQCD_SOLVER_CGNR = 0,     /* even-odd CG on Dhat^dag Dhat (FP64) */
    LQCD_SOLVER_SAP_GCR = 1,  /* flexible GCR, SAP preconditioner */
    LQCD_SOLVER_DFL_SAP_GCR = 2, /* flexible GCR, deflated SAP preconditioner */
    LQCD_SOLVER_NET_GCR = 3,  /* flexible GCR, network preconditioner, SAP where it fails */
    LQCD_SOLVER_DFL_NET_GCR = 4  /* flexible GCR, deflated preconditioner with the network in place of
                                    SAP (N(rho - D Pi A^-1 Pi^dag rho) + Pi A^-1 Pi^dag rho), the
                                    deflated SAP preconditioner where the network's step fails */
} lqcd_solver;

typedef struct {
    lqcd_solver solver;
    int nkv;                 /* GCR Krylov length before restart (<= 64) */
    int nmx;                 /* iteration limit */
    double tol;              /* target true relative residual */
    lqcd_sap_params sap;     /* preconditioner */
    lqcd_prec inner;         /* precision of the preconditioner output and of D phi_k */
    lqcd_prec krylov;        /* GCR Krylov vectors phi_k, chi_k and their Gram-Schmidt: LQCD_F64
                                (0, the default), or LQCD_F32 with inner == LQCD_F32 (native F32
                                fields, products in float, sums in double).  The residual, the
                                solution and the restart residual eta - D psi stay FP64 in both;
                                any other value is LQCD_ERR_ARG */
} lqcd_solver_params;

typedef struct {
    int iters;               /* preconditioned GCR steps (or CG iterations) */
    int restarts;            /* FP64 true-residual recomputations */
    double true_relres;      /* |eta - D psi| / |eta| in FP64 (full system) */
    double relres_dhat;      /* |eta_e - Dhat psi_e| / |eta_e| in FP64 */
    double seconds;          /* wall time of the solve */
    lqcd_status status;
    int net_fallbacks;       /* GCR steps where the network was replaced by SAP */
} lqcd_solve_info;

/* Solve Dhat psi_e = eta_e (Eq. 2) for nrhs even fields to a true relative
 * residual <= tol.  CGNR works on Dhat directly; the GCR solvers solve the
 * full system D chi = (eta_e, 0) and return psi_e = chi_e (Eq. 5), then
 * check the Dhat residual in FP64 and tighten the tolerance when needed.
 * eta_e, psi_e: nrhs canonical FP64 even fields.  info: host array of nrhs
 * entries (may be NULL).  Returns the worst per-RHS status. */
LQCD_API lqcd_status lqcd_solve_dhat(lqcd_ctx *ctx, const lqcd_solver_params *p, const double *eta_dev,
                            double *psi_dev, int nrhs, lqcd_solve_info *info);

/* ------------------------------------------------- learned preconditioner */
/* A gauge-equivariant parallel-transport network N (no counterpart in the
 * paper; it is the learned preconditioner of the benchmark workload):
 *   y_o(x) = sum_i sum_d W_{o,i,d} (T_d y_i)(x),  T_0 = 1,
 *   (T_+mu f)(x) = U_mu(x) f(x+mu),  (T_-mu f)(x) = U_mu(x-mu)^dag f(x-mu),
 * with the antiperiodic sign on hops across the time boundary; W_{o,i,d} is a
 * complex 4x4 spin matrix (identity on colour), d = 0, 1+2mu (+mu), 2+2mu (-mu).
 * Weights (host, complex float interleaved re,im) are laid out layer after
 * layer as W[o][i][d][s][s'].  Activations are stored as act (LQCD_BF16:
 * bfloat16 with tensor-core products and float accumulation; LQCD_F32).
 * The network keeps FP32 master weights; it survives lqcd_set_gauge. */
typedef struct {
    int nlayers;      /* 1..4 */
    int chans[5];     /* chans[0] = chans[nlayers] = 1; every entry 1 or 2 */
    lqcd_prec act;    /* LQCD_BF16 or LQCD_F32 */
} lqcd_net_desc;

LQCD_API lqcd_status lqcd_net_set(lqcd_ctx *ctx, const lqcd_net_desc *desc, const float *W_host);
LQCD_API lqcd_status lqcd_net_get(lqcd_ctx *ctx, float *W_host);
/* out = N(in) for nrhs canonical FP64 full fields (device). */
LQCD_API lqcd_status lqcd_net_apply(lqcd_ctx *ctx, const double *in_dev, double *out_dev, int nrhs);
/* Loss L = (1/nb) sum_b |N(in_b) - t_b|^2 / |t_b|^2 over nb canonical FP64 full
 * fields and its gradient dL/dRe W + i dL/dIm W (host, same layout as W). */
LQCD_API lqcd_status lqcd_net_loss_grad(lqcd_ctx *ctx, const double *in_dev, const double *target_dev, int nb,
                                        double *loss, float *grad_host);

typedef struct {
    int steps;             /* Adam steps */
    int batch;             /* sources per step */
    double lr, beta1, beta2, eps;
    lqcd_sap_params sap;   /* targets t = M_sap(source) */
    int loss;              /* 0: imitation of the SAP correction, (1/nb) sum |N(x) - M_sap x|^2 / |M_sap x|^2;
                              1: the residual of one GCR step with unit coefficient,
                              (1/nb) sum |x - D N(x)|^2 / |x|^2 (no targets needed; its gradient
                              -2 D^dag (x - D N x) / |x|^2 uses D^dag = gamma5 D gamma5) */
} lqcd_net_train_params;
/* Train on (gauge field of ctx, source, M_sap source) pairs: the nsrc sources
 * (canonical FP64 full fields, device; the caller draws them) are paired with
 * their SAP outputs computed here (loss 0); Adam on the selected loss,
 * cycling through the sources in batches.  loss_history (host, may be NULL)
 * receives steps values.  Requires lqcd_clover_invert and lqcd_net_set. */
LQCD_API lqcd_status lqcd_net_train(lqcd_ctx *ctx, const lqcd_net_train_params *p, const double *sources_dev,
                                    int nsrc, double *loss_history);

/* Solve D psi = eta on the full lattice (GCR solvers only); canonical FP64. */
LQCD_API lqcd_status lqcd_solve_D(lqcd_ctx *ctx, const lqcd_solver_params *p, const double *eta_dev,
                         double *psi_dev, int nrhs, lqcd_solve_info *info);

/* As lqcd_solve_dhat (GCR solvers), starting from the guess that psi_dev
 * holds on entry instead of from zero. */
LQCD_API lqcd_status lqcd_solve_dhat_guess(lqcd_ctx *ctx, const lqcd_solver_params *p, const double *eta_dev,
                                           double *psi_dev, int nrhs, lqcd_solve_info *info);

/* ---------------------------------------------- chronological initial guess */
/* Sec. 2: each inversion starts from a prediction built from earlier
 * solutions (the chronological method of Brower et al.).  The context keeps
 * the last nkeep (0..16; 0 drops the store) solutions added; the guess for a
 * source eta is x0 = sum_i c_i x_i with c minimising |eta - Dhat x0|
 * (normal equations in FP64, nearly dependent solutions dropped).  Fields are
 * canonical FP64 even fields (device).  nused (may be NULL) receives the
 * number of stored solutions the guess uses; with none stored x0 = 0. */
LQCD_API lqcd_status lqcd_chrono_reset(lqcd_ctx *ctx, int nkeep);
LQCD_API lqcd_status lqcd_chrono_add(lqcd_ctx *ctx, const double *psi_dev);
LQCD_API lqcd_status lqcd_chrono_guess(lqcd_ctx *ctx, const double *eta_dev, double *x0_dev, int *nused);

/* ------------------------------------------- Hasenbusch mass preconditioning */
/* W(dm) = Q_S + dm (Eq. 3) with Q_S = 1 - Q_ee^-1 Q_eo Q_oo^-1 Q_oe (Eq. 2),
 * Q = gamma5 D; the gamma5 factors cancel, so W(dm) = A_ee^-1 Dhat + dm.
 * out = W(dm) in: nrhs canonical even fields of precision prec (F64 or F32). */
LQCD_API lqcd_status lqcd_apply_W(lqcd_ctx *ctx, lqcd_prec prec, double dm, const void *in_dev, void *out_dev,
                                  int nrhs);
/* Solve W(dm) psi = eta (the pseudofermion solve of Eq. 4) for nrhs canonical
 * FP64 even fields, as Dhat' psi = A_ee eta where Dhat' is the Schur
 * complement of D with its even-site clover blocks scaled by 1 + dm (built
 * for the solve, then the clover term of D is rebuilt).  p->solver: CGNR or
 * SAP-GCR (a deflation subspace or network belongs to D, not to D').
 * info[k].relres_dhat holds the FP64 residual |eta - W psi| / |eta|.
 * dm > -1. */
LQCD_API lqcd_status lqcd_solve_W(lqcd_ctx *ctx, const lqcd_solver_params *p, double dm, const double *eta_dev,
                                  double *psi_dev, int nrhs, lqcd_solve_info *info);

/* ------------------------------------------------------ DD-HMC block solves */
/* Sec. 3: the inversions on the blocks needed for the DD-HMC block force use
 * BiCGstab.  The lattice is cut into Dirichlet blocks of extents bs (even,
 * tiling the lattice; 6,6,12,12 in the paper's 48x24^3 runs): hops whose
 * other end lies in another block are dropped, a block that spans a whole
 * direction keeps the wrapped hop.  Each block's Schur operator
 * Dhat_blk = A_ee - H_eo,blk A_oo^-1 H_oe,blk is an independent system.
 * Blocks are numbered lexicographically in their block coordinates
 * (b = c3 + nb3 (c2 + nb2 (c1 + nb1 c0)), nb = L / bs).  FP64. */
typedef struct {
    int bs[4];    /* block extents */
    double tol;   /* per block: |eta_b - Dhat_blk psi_b| <= tol |eta_b| */
    int nmx;      /* BiCGstab iterations per block at most (>= 0) */
} lqcd_block_params;

/* Number of blocks of extents bs, or -1 if bs does not tile the lattice. */
LQCD_API long lqcd_block_count(const lqcd_ctx *ctx, const int bs[4]);
/* out = Dhat_blk in on every block: one canonical FP64 even field (device). */
LQCD_API lqcd_status lqcd_apply_Dhat_block(lqcd_ctx *ctx, const int bs[4], const double *in_dev, double *out_dev);
/* Solve Dhat_blk psi = eta on every block by BiCGstab from psi = 0 (all
 * blocks in lockstep; a converged block takes no further updates).
 * eta_dev, psi_dev: one canonical FP64 even field each (device).  iters,
 * relres, status: optional host arrays of lqcd_block_count entries receiving
 * each block's steps, recomputed relative residual and status (LQCD_OK,
 * LQCD_ERR_NOT_CONVERGED, LQCD_ERR_BREAKDOWN, LQCD_ERR_NAN).  Returns the
 * first non-OK block status, LQCD_OK when every block converged. */
LQCD_API lqcd_status lqcd_block_solve(lqcd_ctx *ctx, const lqcd_block_params *p, const double *eta_dev,
                                      double *psi_dev, int *iters, double *relres, int *status);

/* ----------------------------------------------- MD forces and leapfrog step */
/* The molecular-dynamics part of the two-flavour HMC (Sec. 2, Eq. 4), FP64.
 * A link moves along U_mu(x) -> exp(eps T_a) U_mu(x), T_a = i lambda_a / 2
 * (Gell-Mann lambda_a); every gradient is dS/d eps written to a caller-owned
 * device array g[site][mu][a] of V x 4 x 8 doubles (lexicographic sites; the
 * MD force is -g).  The context must hold the gauge field and its clover
 * term (lqcd_set_gauge, lqcd_clover_invert); otherwise LQCD_ERR_STATE. */

/* g = Re <Y, (dD/d eps) X> for every link and generator (hop and clover
 * terms of D, Eq. 1); X, Y: canonical full FP64 fields. */
LQCD_API lqcd_status lqcd_force_dD(lqcd_ctx *ctx, const double *X_dev, const double *Y_dev, double *g_dev);
/* g = d log|det A_parity| / d eps = sum over the sites of that parity of
 * Re tr(A^-1 dA) (the clover determinant of Eq. 4: S gets -2 log|det A_oo|). */
LQCD_API lqcd_status lqcd_force_logdet(lqcd_ctx *ctx, int parity, double *g_dev);
/* Wilson gauge action S_g = beta sum_P (1 - Re tr U_P / 3) (host scalar,
 * synchronises) and its gradient. */
LQCD_API lqcd_status lqcd_gauge_action(lqcd_ctx *ctx, double beta, double *S_host);
LQCD_API lqcd_status lqcd_force_gauge(lqcd_ctx *ctx, double beta, double *g_dev);
/* Gradient of the pseudofermion action |Dhat^-1 phi_e|^2 (Eq. 2, 4):
 * -2 Re <y_e, dDhat x_e> with x_e = Dhat^-1 phi_e, y_e = Dhat^-dag x_e, both
 * solved with the given solver parameters (info: host array of 2 entries or
 * NULL); phi_e: canonical FP64 even field.  A solve that does not reach its
 * tolerance returns its status (g is still written). */
LQCD_API lqcd_status lqcd_force_pf(lqcd_ctx *ctx, const lqcd_solver_params *p, const double *phi_e_dev,
                                   double *g_dev, lqcd_solve_info *info);

typedef struct {
    double beta;                 /* Wilson gauge coupling */
    double dt;                   /* leapfrog step size */
    int nsteps;                  /* leapfrog steps */
    lqcd_solver_params solver;   /* the solves of the pseudofermion force */
} lqcd_md_params;

/* Total gradient of S = S_g + |Dhat^-1 phi_e|^2 - 2 log|det A_oo| (the
 * even-odd factorised two-flavour action with the clover term, Eq. 2 and 4)
 * at the context's gauge field; S_host (may be NULL) receives S. */
LQCD_API lqcd_status lqcd_md_gradient(lqcd_ctx *ctx, const lqcd_md_params *p, const double *phi_e_dev,
                                      double *g_dev, double *S_host);
/* nsteps leapfrog steps of size dt (the integrator of Sec. 2):
 *   p -= dt/2 g;  U <- exp(dt P) U (P = sum_a p^a T_a);  p -= dt/2 g.
 * U_dev: canonical links (V x 4 x 3 x 3 complex), which must be the field the
 * context holds on entry; on return U_dev and the context hold the evolved
 * field with its clover term rebuilt (same kappa, c_sw).  p_dev: momenta
 * V x 4 x 8 doubles, updated in place.  The exponential is a Taylor series
 * after scaling and squaring; the links are not re-unitarised.  Synchronises. */
LQCD_API lqcd_status lqcd_md_leapfrog(lqcd_ctx *ctx, const lqcd_md_params *p, double *U_dev, double *p_dev,
                                      const double *phi_e_dev);

/* ------------------------------------------------ batched multi-lattice solve */
/* Several independent lattices (each its own context: gauge field, kappa,
 * clover term) solved together with the SAP-preconditioned flexible GCR of
 * Sec. 3-4, one right-hand side per lattice.  Every phase of a GCR step runs
 * as ONE launch over a work list of (lattice, tile / SAP block / vector chunk)
 * items of all lattices: the SAP block solves (precision sap.prec, F16S or
 * F32), D phi in F32, the FP64 Gram-Schmidt (one cooperative persistent
 * kernel whose grid barriers wait at most wait_timeout_s, then report
 * LQCD_ERR_TIMEOUT), and the FP64 residual restart.  Per-lattice scalars and
 * convergence flags stay on the device; converged lattices drop out of the
 * work lists.  With use_graph the GCR cycle (nkv steps and the solution
 * update) is captured once as a CUDA graph and replayed; the host waits once
 * per cycle.  All contexts must share one SAP block shape; they must not be
 * used by other calls while a batch solve runs. */
typedef struct lqcd_batch lqcd_batch;
typedef struct {
    int nkv;                /* Krylov vectors per cycle, 1..32 */
    int nmx;                /* GCR steps per lattice, at most */
    double tol;             /* relative residual |eta - D psi| / |eta| per lattice */
    lqcd_sap_params sap;    /* preconditioner; prec LQCD_F16S or LQCD_F32 */
    int use_graph;          /* replay the GCR cycle from a captured CUDA graph */
    double wait_timeout_s;  /* limit of each device-side wait */
    int stall_test;         /* test aid: the first grid barrier waits for one CTA too many,
                               so it can only end by its time limit; 0 in normal use */
} lqcd_batch_params;
/* ctxs: n contexts with gauge field and clover term.  stream: the caller's
 * stream, ordered before and after each solve; the batch works on its own. */
LQCD_API lqcd_status lqcd_batch_create(lqcd_ctx *const *ctxs, int n, const lqcd_batch_params *p, void *stream,
                                       lqcd_batch **out);
LQCD_API lqcd_status lqcd_batch_destroy(lqcd_batch *b);
LQCD_API const char *lqcd_batch_last_error(const lqcd_batch *b);
/* Solve Dhat_l psi_l = eta_l (Eq. 2, through Eq. 5) for every lattice l:
 * eta_dev[l], psi_dev[l]: canonical FP64 even fields of lattice l (device).
 * info: n entries.  Returns the worst per-lattice status. */
LQCD_API lqcd_status lqcd_batch_solve_dhat(lqcd_batch *b, const double *const *eta_dev, double *const *psi_dev,
                                           lqcd_solve_info *info);
/* Statistics of the last solve: GCR cycles, cycles replayed from the graph,
 * kernel launches issued by the host. */
LQCD_API lqcd_status lqcd_batch_stats(const lqcd_batch *b, int *cycles, int *graph_replays, long *launches);

#ifdef __cplusplus
}
#endif

#endif
