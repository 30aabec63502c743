/*
 * Oracle, part 4: the gauge-equivariant parallel-transport convolution network
 * used as a learned preconditioner next to SAP in the flexible GCR.  The paper
 * has no such network; the definition follows the benchmark workload:
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *   (T_0 f)(x)    = f(x)
 *   (T_+mu f)(x)  = s U_mu(x) f(x+mu)
 *   (T_-mu f)(x)  = s U_mu(x-mu)^dag f(x-mu)
 *   with s = -1 on hops across the antiperiodic time boundary, else +1;
 *   path index d: 0 identity, 1+2mu: +mu, 2+2mu: -mu.
 *   layer:  y_o(x) = sum_i sum_d W_{o,i,d} (T_d y_i)(x),
 *   W_{o,i,d} a complex 4x4 matrix on spin (identity on colour); no bias,
 *   no activation.  Weights are stored layer after layer as
 *   W[o][i][d][s][s'] (complex), fields as [channel][site][spin][colour].
 *
 * Backward, for a real loss L and the "conjugate gradient" g = dL/dRe + i dL/dIm:
 *   dL/dW_{o,i,d}[s][s'] = sum_{x,c} g_o(x)[s][c] conj((T_d y_i)(x)[s'][c])
 *   g_i = sum_{o,d} T_d^dag (W_{o,i,d}^dag g_o),  T_+mu^dag = T_-mu.
 * Pinned by (tests/test_oracle_ptc.py): gauge equivariance; identity weights give
 * the identity; one layer with the Wilson weights reproduces the hop term of D;
 * T_d^dag is the adjoint of T_d; central finite differences of the loss.
 */
#include "oracle_internal.h"

#include <stdlib.h>
#include <string.h>

/* (T_d f)(x) for every site; f, out: [V][4][3] */
void or_ptc_transport(const oracle *o, int d, const double *f_, double *out_)
{
    const ocplx *f = (const ocplx *)f_;
    ocplx *out = (ocplx *)out_;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < o->V; x++) {
        if (d == 0) {
            for (int i = 0; i < 12; i++) out[12 * x + i] = f[12 * x + i];
            continue;
        }
        int mu = (d - 1) / 2, fwd = (d % 2) == 1;
        int x0 = o->coord[4 * x];
        long y = fwd ? o->fw[4 * x + mu] : o->bw[4 * x + mu];
        double s = 1.0;
        if (mu == 0 && ((fwd && x0 == o->L[0] - 1) || (!fwd && x0 == 0))) s = o->bc_t;
        const ocplx *U = o->U + 9 * (4 * (fwd ? x : y) + mu);
        for (int sp = 0; sp < 4; sp++)
            for (int a = 0; a < 3; a++) {
                ocplx acc = 0;
                for (int b = 0; b < 3; b++)
                    acc += (fwd ? U[3 * a + b] : conj(U[3 * b + a])) * f[12 * y + 3 * sp + b];
                out[12 * x + 3 * sp + a] = s * acc;
            }
    }
}

static long layer_weights(int cin, int cout) { return (long)cout * cin * 9 * 16; }

/* one layer: out[o] = sum_i sum_d W[o][i][d] (T_d in[i]) */
static void layer_forward(const oracle *o, int cin, int cout, const ocplx *W, const ocplx *in, ocplx *out)
{
    long n = 12 * o->V;
    ocplx *t = malloc(sizeof(ocplx) * n);
    for (long j = 0; j < n * cout; j++) out[j] = 0;
    for (int i = 0; i < cin; i++)
        for (int d = 0; d < 9; d++) {
            or_ptc_transport(o, d, (const double *)(in + n * i), (double *)t);
            for (int oc = 0; oc < cout; oc++) {
                const ocplx *w = W + ((oc * cin + i) * 9 + d) * 16;
                ocplx *y = out + n * oc;
                for (long x = 0; x < o->V; x++)
                    for (int s = 0; s < 4; s++)
                        for (int c = 0; c < 3; c++) {
                            ocplx acc = 0;
                            for (int sp = 0; sp < 4; sp++) acc += w[4 * s + sp] * t[12 * x + 3 * sp + c];
                            y[12 * x + 3 * s + c] += acc;
                        }
            }
        }
    free(t);
}

/* forward through nl layers; chans[0..nl]; acts (optional) receives every
 * layer's input, layer after layer ([chans[l]] fields each) */
void or_ptc_forward(const oracle *o, int nl, const int *chans, const double *W_, const double *in_, double *out_,
                    double *acts_)
{
    long n = 12 * o->V;
    const ocplx *W = (const ocplx *)W_;
    ocplx *cur = malloc(sizeof(ocplx) * n * chans[0]);
    memcpy(cur, in_, sizeof(ocplx) * n * chans[0]);
    ocplx *acts = (ocplx *)acts_;
    long woff = 0, aoff = 0;
    for (int l = 0; l < nl; l++) {
        if (acts) {
            memcpy(acts + aoff, cur, sizeof(ocplx) * n * chans[l]);
            aoff += n * chans[l];
        }
        ocplx *nxt = malloc(sizeof(ocplx) * n * chans[l + 1]);
        layer_forward(o, chans[l], chans[l + 1], W + woff, cur, nxt);
        woff += layer_weights(chans[l], chans[l + 1]);
        free(cur);
        cur = nxt;
    }
    memcpy(out_, cur, sizeof(ocplx) * n * chans[nl]);
    free(cur);
}

/* backward: g_out (conjugate gradient at the output) -> dW (same layout as W)
 * and, if g_in != NULL, the conjugate gradient at the input */
void or_ptc_backward(const oracle *o, int nl, const int *chans, const double *W_, const double *acts_,
                     const double *gout_, double *dW_, double *gin_)
{
    long n = 12 * o->V;
    const ocplx *W = (const ocplx *)W_;
    const ocplx *acts = (const ocplx *)acts_;
    ocplx *dW = (ocplx *)dW_;
    long wtot = 0, atot = 0;
    for (int l = 0; l < nl; l++) {
        wtot += layer_weights(chans[l], chans[l + 1]);
        atot += n * chans[l];
    }
    ocplx *g = malloc(sizeof(ocplx) * n * chans[nl]);
    memcpy(g, gout_, sizeof(ocplx) * n * chans[nl]);
    ocplx *t = malloc(sizeof(ocplx) * n), *u = malloc(sizeof(ocplx) * n);
    long woff = wtot, aoff = atot;
    for (int l = nl - 1; l >= 0; l--) {
        int cin = chans[l], cout = chans[l + 1];
        woff -= layer_weights(cin, cout);
        aoff -= n * cin;
        const ocplx *y = acts + aoff;
        /* weight gradient */
        for (int i = 0; i < cin; i++)
            for (int d = 0; d < 9; d++) {
                or_ptc_transport(o, d, (const double *)(y + n * i), (double *)t);
                for (int oc = 0; oc < cout; oc++) {
                    ocplx *gw = dW + woff + ((oc * cin + i) * 9 + d) * 16;
                    const ocplx *go = g + n * oc;
                    for (int s = 0; s < 4; s++)
                        for (int sp = 0; sp < 4; sp++) {
                            ocplx acc = 0;
                            for (long x = 0; x < o->V; x++)
                                for (int c = 0; c < 3; c++) acc += go[12 * x + 3 * s + c] * conj(t[12 * x + 3 * sp + c]);
                            gw[4 * s + sp] = acc;
                        }
                }
            }
        /* data gradient g_i = sum_{o,d} T_d^dag (W^dag g_o) */
        ocplx *gi = calloc(n * cin, sizeof(ocplx));
        for (int i = 0; i < cin; i++)
            for (int d = 0; d < 9; d++) {
                for (long j = 0; j < n; j++) u[j] = 0;
                for (int oc = 0; oc < cout; oc++) {
                    const ocplx *w = W + woff + ((oc * cin + i) * 9 + d) * 16;
                    const ocplx *go = g + n * oc;
                    for (long x = 0; x < o->V; x++)
                        for (int sp = 0; sp < 4; sp++)
                            for (int c = 0; c < 3; c++) {
                                ocplx acc = 0;
                                for (int s = 0; s < 4; s++) acc += conj(w[4 * s + sp]) * go[12 * x + 3 * s + c];
                                u[12 * x + 3 * sp + c] += acc;
                            }
                }
                /* T_d^dag = T_{-d}: +mu <-> -mu */
                int dd = d == 0 ? 0 : ((d % 2) ? d + 1 : d - 1);
                or_ptc_transport(o, dd, (const double *)u, (double *)t);
                for (long j = 0; j < n; j++) gi[n * i + j] += t[j];
            }
        free(g);
        g = gi;
    }
    if (gin_) memcpy(gin_, g, sizeof(ocplx) * n * chans[0]);
    free(g);
    free(t);
    free(u);
}
