/*
 * Oracle: block decomposition of the lattice (SAP blocks, deflation blocks)
 * and the Dirichlet block-restricted hop.  TEST INFRASTRUCTURE ONLY.
 *
 * A block is a bs0 x bs1 x bs2 x bs3 sub-lattice starting at multiples of bs;
 * its colour is the sum of its block coordinates mod 2.  The block operator is
 * D_blk = P_blk D P_blk: hops whose other end lies outside the block are
 * dropped (a hop that wraps around the lattice and lands in the same block is
 * kept, so one block covering the lattice gives back the full D).
 */
#include "oracle_internal.h"

#include <stdlib.h>


int ob_make_blocking(const oracle *o, const int bs[4], blocking *B)
{
    long vol = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (bs[mu] <= 0 || bs[mu] % 2 || o->L[mu] % bs[mu]) return OR_ERR_ARG;
        B->bs[mu] = bs[mu];
        B->nb[mu] = o->L[mu] / bs[mu];
        vol *= bs[mu];
    }
    B->vol = vol;
    B->nblk = (long)B->nb[0] * B->nb[1] * B->nb[2] * B->nb[3];
    B->blk_of = malloc(sizeof(long) * o->V);
    B->loc = malloc(sizeof(long) * o->V);
    B->se = malloc(sizeof(long) * B->nblk * (vol / 2));
    B->so = malloc(sizeof(long) * B->nblk * (vol / 2));
    B->colour = malloc(sizeof(int) * B->nblk);
    long *cnt = calloc(2 * B->nblk, sizeof(long));
    for (long b = 0; b < B->nblk; b++) {
        long r = b;
        int c3 = r % B->nb[3];
        r /= B->nb[3];
        int c2 = r % B->nb[2];
        r /= B->nb[2];
        int c1 = r % B->nb[1];
        int c0 = r / B->nb[1];
        B->colour[b] = (c0 + c1 + c2 + c3) % 2;
    }
    for (long x = 0; x < o->V; x++) {
        const int *c = o->coord + 4 * x;
        long b = (c[3] / bs[3]) + B->nb[3] * ((c[2] / bs[2]) + B->nb[2] *
                  ((c[1] / bs[1]) + (long)B->nb[1] * (c[0] / bs[0])));
        B->blk_of[x] = b;
        int p = o->par[x];
        long k = cnt[2 * b + p]++;
        B->loc[x] = k;
        (p ? B->so : B->se)[b * (vol / 2) + k] = x;
    }
    free(cnt);
    return OR_OK;
}

void ob_free_blocking(blocking *B)
{
    free(B->blk_of);
    free(B->loc);
    free(B->se);
    free(B->so);
    free(B->colour);
}

/* gamma table access for the block hop (same definitions as oracle_dirac.c,
 * fetched through the exported accessor) */
ocplx ob_G[4][4][4];
void ob_load_gammas(void)
{
    for (int mu = 0; mu < 4; mu++) or_gamma(mu, (double *)&ob_G[mu][0][0]);
}

void ob_colour_mul(const ocplx *M, int dagger, const ocplx *psi, ocplx *t)
{
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            ocplx acc = 0;
            for (int b = 0; b < 3; b++)
                acc += (dagger ? conj(M[3 * b + a]) : M[3 * a + b]) * psi[3 * s + b];
            t[3 * s + a] = acc;
        }
}

void ob_add_proj(ocplx *res, const ocplx *t, int mu, double sgn, double coef)
{
    for (int s = 0; s < 4; s++)
        for (int c = 0; c < 3; c++) {
            ocplx acc = t[3 * s + c];
            for (int r = 0; r < 4; r++) acc += sgn * ob_G[mu][s][r] * t[3 * r + c];
            res[3 * s + c] += coef * acc;
        }
}

void ob_mat12_vec(const ocplx *M, const ocplx *v, ocplx *r)
{
    for (int i = 0; i < 12; i++) {
        ocplx acc = 0;
        for (int j = 0; j < 12; j++) acc += M[12 * i + j] * v[j];
        r[i] = acc;
    }
}

/* Block-restricted hop (Dirichlet): res = (P_blk H P_blk in)(x) for x in block
 * blk.  The input is a block-local field indexed by B->loc of the opposite
 * parity to x; hops to sites outside the block are dropped. */
void ob_block_hop_site(const oracle *o, const blocking *B, long blk, const ocplx *in_loc,
                           long x, ocplx *res)
{
    for (int i = 0; i < 12; i++) res[i] = 0;
    int x0 = o->coord[4 * x];
    const ocplx *U = o->U;
    for (int mu = 0; mu < 4; mu++) {
        ocplx t[12];
        long y = o->fw[4 * x + mu];
        if (B->blk_of[y] == blk) {
            double sf = (mu == 0 && x0 == o->L[0] - 1) ? o->bc_t : 1.0;
            ob_colour_mul(U + 9 * (4 * x + mu), 0, in_loc + 12 * B->loc[y], t);
            ob_add_proj(res, t, mu, -1.0, -0.5 * sf);
        }
        long z = o->bw[4 * x + mu];
        if (B->blk_of[z] == blk) {
            double sb = (mu == 0 && x0 == 0) ? o->bc_t : 1.0;
            ob_colour_mul(U + 9 * (4 * z + mu), 1, in_loc + 12 * B->loc[z], t);
            ob_add_proj(res, t, mu, +1.0, -0.5 * sb);
        }
    }
}

