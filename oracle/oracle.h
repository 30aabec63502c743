/*
 * Plain double-precision CPU oracle for the Wilson-clover solver path of
 * Marinkovic & Schaefer, "Comparison of the mass preconditioned HMC and the
 * DD-HMC algorithm for two-flavour QCD" (Lattice 2010).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the test suite, the package's smoke check and the
 * timed CPU baseline of the benchmark load it.  It shares no source, header,
 * table or helper with the CUDA path.
 *
 * Every routine is written for a reader who checks it against the definitions:
 * one site at a time, full 4x4 Dirac matrices, full 12x12 clover matrices,
 * no spin projection, no blocking, no fused kernels.
 *
 * Conventions (the paper gives Eq. 1 only; these readings are the standard
 * lattice ones):
 *   - lattice T x L1 x L2 x L3, x0 = time is the slowest coordinate,
 *     site = x3 + L3*(x2 + L2*(x1 + L1*x0));
 *   - spinor psi[site][spin 4][colour 3] complex; link U[site][mu][3][3];
 *   - chiral gamma basis, gamma5 = g0 g1 g2 g3 = diag(1,1,-1,-1);
 *   - D = (4+m0) + c_sw sum_{mu,nu} (i/4) sigma_{mu nu} Fhat_{mu nu} + H,
 *     H psi(x) = -1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu)
 *                            + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)],
 *     m0 = 1/(2 kappa) - 4, antiperiodic fermion boundary in time applied as a
 *     sign on the hop (never folded into the links);
 *   - Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag)/8, Q the sum of the four
 *     same-orientation plaquette leaves at x;
 *   - even sites: x0+x1+x2+x3 even; an even (odd) field is indexed by the rank
 *     of the site among the even (odd) sites in lexicographic order.
 *
 * Parity status of each function is recorded beside it ("pinned by" names the
 * independent check in the test suite).
 */
#ifndef LQCD_ORACLE_H
#define LQCD_ORACLE_H

#include <complex.h>

typedef double complex ocplx;

typedef struct oracle {
    int L[4];            /* L[0] = T */
    long V, Vh;
    double bc_t;         /* -1: antiperiodic fermion field in time, +1 periodic */
    double kappa, csw, m0;
    ocplx *U;            /* [V][4][3][3] gauge links (copied) */
    ocplx *A;            /* [V][12][12] clover matrix incl. 4+m0 */
    ocplx *Ainv;         /* [V][12][12] inverse of A */
    double logdet[2];    /* sum over even / odd sites of log|det A(x)| */
    int have_clover;
    int *par;            /* [V] parity */
    long *rank;          /* [V] rank among the sites of the same parity */
    long *site_of[2];    /* [parity][rank] -> site */
    long *fw, *bw;       /* [V][4] neighbour x+mu, x-mu (periodic wrap) */
    int *coord;          /* [V][4] */
    struct or_dfl *dfl;  /* deflation subspace state, NULL until built */
} oracle;

/* status codes (numerically equal to the library's, defined independently) */
#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SINGULAR 4
#define OR_ERR_NOT_CONVERGED 5
#define OR_ERR_BREAKDOWN 6

/* --- lattice and operators (oracle_dirac.c) --- */
oracle *or_create(int T, int L1, int L2, int L3, int antiperiodic_t);
void or_destroy(oracle *o);
void or_set_gauge(oracle *o, const double *U);
int or_set_params(oracle *o, double kappa, double csw);
void or_gamma(int mu, double *g);
void or_fhat_site(const oracle *o, long x, int mu, int nu, double *F);
void or_clover_site(const oracle *o, long x, double *A12);
void or_clover_inv_site(const oracle *o, long x, double *A12);
double or_logdet(const oracle *o, int parity);
void or_hop(const oracle *o, const double *in, double *out);
void or_apply_clover(const oracle *o, int inverse, const double *in, double *out);
void or_apply_D(const oracle *o, const double *in, double *out);
void or_apply_Dhat(const oracle *o, const double *in_e, double *out_e);
/* W(dm) = Q_S + dm, Q_S = 1 - A_ee^-1 H_eo A_oo^-1 H_oe (Eq. 2-3); even fields */
void or_apply_W(const oracle *o, double dm, const double *in_e, double *out_e);
void or_apply_Dhat_dag(const oracle *o, const double *in_e, double *out_e);
void or_apply_gamma5(long n, const double *in, double *out);
void or_dhat_site(const oracle *o, const double *in_e, long xe, double *out12);
void or_d_site(const oracle *o, const double *in, long x, double *out12);
long or_even_rank_to_site(const oracle *o, int parity, long r);
int or_num_threads(void);

/* --- Lie derivatives for the MD forces (Sec. 2, Eq. 4), oracle_dirac.c ---
 * The link U_mu(x) moves along exp(eps T_a) U_mu(x), T_a = i lambda_a / 2.
 * or_dD_apply: out = (dD/d eps) in (full fields).  Arrays g hold [V][4][8]. */
void or_dD_apply(const oracle *o, long x, int mu, int a, const double *in, double *out);
void or_force_dD(const oracle *o, const double *X, const double *Y, double *g);   /* Re <Y, dD X> */
void or_force_logdet(const oracle *o, int parity, double *g);                     /* d log|det A_p| */
/* Wilson gauge action beta sum_P (1 - Re tr U_P / 3) and its gradient */
double or_gauge_action(const oracle *o, double beta);
void or_grad_gauge(const oracle *o, double beta, double *g);

/* --- solvers (oracle_solvers.c) --- */
int or_cgnr(const oracle *o, const double *eta_e, double *psi_e, double tol, int maxit,
            int *iters);
void or_sap(const oracle *o, const int bs[4], int ncy, int nmr, const double *eta,
            double *psi);
void or_sap_block_solve(const oracle *o, const int bs[4], long blk, int nmr,
                        const double *r, double *chi);
/* DD-HMC block solves: Dhat_blk (Dirichlet blocks of extents bs) on even half
 * fields, and BiCGstab on every block to tol (iters / relres per block) */
void or_block_dhat(const oracle *o, const int bs[4], const double *in_e, double *out_e);
int or_block_bicgstab(const oracle *o, const int bs[4], const double *eta_e, double *psi_e, double tol,
                      int maxit, int *iters, double *relres);
int or_gcr(const oracle *o, int precond, const int bs[4], int ncy, int nmr, int nkv, int nmx,
           double tol, const double *eta, double *psi, int *iters, double *relres);

/* --- deflation (oracle_dfl.c) --- */
int or_dfl_build(oracle *o, const int bs[4], int Ns, int ninv, int ncy, int nmr,
                 const double *v0);
void or_dfl_project(const oracle *o, const double *in, double *c);
void or_dfl_expand(const oracle *o, const double *c, double *out);
void or_dfl_little(const oracle *o, double *Amat);
void or_dfl_little_apply(const oracle *o, const double *c, double *out);
int or_dfl_coarse_solve(const oracle *o, const double *b, double *c, double tol, int nkv,
                        int nmx, int *iters);
void or_dfl_precond(const oracle *o, const int bs[4], int ncy, int nmr, double ctol,
                    const double *rho, double *phi);
void or_dfl_subspace(const oracle *o, double *phi);
void or_dfl_free(oracle *o);

/* --- parallel-transport network (oracle_ptc.c) --- */
void or_ptc_transport(const oracle *o, int d, const double *f, double *out);
void or_ptc_forward(const oracle *o, int nl, const int *chans, const double *W, const double *in, double *out,
                    double *acts);
void or_ptc_backward(const oracle *o, int nl, const int *chans, const double *W, const double *acts,
                     const double *gout, double *dW, double *gin);

#endif
