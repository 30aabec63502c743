/*
 * Oracle internal declarations shared by the oracle's own source files:
 * the block decomposition used by SAP and by deflation, and the per-site
 * colour / spin helpers of the block-restricted hop.  TEST INFRASTRUCTURE ONLY.
 */
#ifndef LQCD_ORACLE_INTERNAL_H
#define LQCD_ORACLE_INTERNAL_H

#include "oracle.h"

typedef struct {
    int bs[4], nb[4];
    long nblk, vol;   /* number of blocks, sites per block */
    long *blk_of;     /* [V] block of a site */
    long *loc;        /* [V] position of the site in its block's parity list */
    long *se, *so;    /* [nblk][vol/2] even / odd sites of each block, lexicographic */
    int *colour;      /* [nblk] (sum of block coordinates) mod 2 */
} blocking;

extern ocplx ob_G[4][4][4];
int ob_make_blocking(const oracle *o, const int bs[4], blocking *B);
void ob_free_blocking(blocking *B);
void ob_load_gammas(void);
void ob_colour_mul(const ocplx *M, int dagger, const ocplx *psi, ocplx *t);
void ob_add_proj(ocplx *res, const ocplx *t, int mu, double sgn, double coef);
void ob_mat12_vec(const ocplx *M, const ocplx *v, ocplx *r);
void ob_block_hop_site(const oracle *o, const blocking *B, long blk, const ocplx *in_loc,
                       long x, ocplx *res);

#endif
