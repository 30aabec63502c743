// Chronological initial guess (Sec. 2: every inversion of the HMC starts
// from a prediction built from earlier solutions, the method of Brower et
// al.): the context keeps the last nkeep solutions x_i of Dhat x = eta, and a
// new source gets x0 = sum_i c_i x_i with c minimising |eta - Dhat x0| over
// their span.  The small least-squares problem is solved through its normal
// equations G c = d, G_ij = <Dhat x_i, Dhat x_j>, d_i = <Dhat x_i, eta>, by an
// FP64 Cholesky factorisation on the host that drops directions whose pivot
// falls below 1e-12 of the largest diagonal entry (nearly dependent
// solutions).  The device work is nkeep Dhat applications, FP64 dot products
// and one multi-axpy.
#include <cmath>
#include <complex>
#include <vector>

#include "lqcd_internal.cuh"

struct ChronoState {
    int nkeep = 0, count = 0, head = 0;
    double2 *X = nullptr;   // nkeep native FP64 even half fields, slots 0 .. count-1 filled
};

void chrono_free(lqcd_ctx *c)
{
    if (!c || !c->chrono) return;
    cudaFree(c->chrono->X);
    delete c->chrono;
    c->chrono = nullptr;
}

namespace {

using Z = std::complex<double>;

// solve G c = d (G Hermitian positive semi-definite, n x n) by Cholesky,
// dropping directions with a pivot below tol * max diag; returns the kept count
int chol_solve(int n, const std::vector<Z> &G, const std::vector<Z> &d, std::vector<Z> &cout)
{
    double dmax = 0;
    for (int i = 0; i < n; i++) dmax = std::max(dmax, G[i * n + i].real());
    std::vector<Z> L(n * n, 0.0);
    std::vector<char> keep(n, 0);
    int kept = 0;
    for (int j = 0; j < n; j++) {
        Z s = G[j * n + j];
        for (int k = 0; k < j; k++)
            if (keep[k]) s -= L[j * n + k] * std::conj(L[j * n + k]);
        if (!(s.real() > 1e-12 * dmax)) continue;
        keep[j] = 1;
        kept++;
        const double ljj = std::sqrt(s.real());
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            Z t = G[i * n + j];
            for (int k = 0; k < j; k++)
                if (keep[k]) t -= L[i * n + k] * std::conj(L[j * n + k]);
            L[i * n + j] = t / ljj;
        }
    }
    // forward L y = d, backward L^H c = y over the kept indices
    std::vector<Z> y(n, 0.0);
    cout.assign(n, 0.0);
    for (int i = 0; i < n; i++) {
        if (!keep[i]) continue;
        Z t = d[i];
        for (int k = 0; k < i; k++)
            if (keep[k]) t -= L[i * n + k] * y[k];
        y[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        if (!keep[i]) continue;
        Z t = y[i];
        for (int k = i + 1; k < n; k++)
            if (keep[k]) t -= std::conj(L[k * n + i]) * cout[k];
        cout[i] = t / L[i * n + i];
    }
    return kept;
}

}  // namespace

extern "C" {

lqcd_status lqcd_chrono_reset(lqcd_ctx *c, int nkeep)
{
    if (!c || nkeep < 0 || nkeep > 16) return set_err(c, LQCD_ERR_ARG, "nkeep=%d (0..16)", nkeep);
    chrono_free(c);
    if (nkeep == 0) return LQCD_OK;
    ChronoState *s = new ChronoState();
    s->nkeep = nkeep;
    if (cudaMalloc(&s->X, (size_t)nkeep * 12 * c->g.Vh * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return set_err(c, LQCD_ERR_NOMEM, "chronological store");
    }
    c->chrono = s;
    return LQCD_OK;
}

lqcd_status lqcd_chrono_add(lqcd_ctx *c, const double *psi_e)
{
    if (!c || !psi_e) return set_err(c, LQCD_ERR_ARG, "null argument");
    ChronoState *s = c->chrono;
    if (!s) return set_err(c, LQCD_ERR_STATE, "chronological store not set (lqcd_chrono_reset)");
    LQCD_TRY(pack_field(c, LQCD_F64, 1, psi_e, s->X + (size_t)s->head * 12 * c->g.Vh, 1, false));
    s->head = (s->head + 1) % s->nkeep;
    s->count = std::min(s->count + 1, s->nkeep);
    return LQCD_OK;
}

lqcd_status lqcd_chrono_guess(lqcd_ctx *c, const double *eta_e, double *x0_e, int *nused)
{
    if (!c || !eta_e || !x0_e) return set_err(c, LQCD_ERR_ARG, "null argument");
    ChronoState *s = c->chrono;
    if (!s) return set_err(c, LQCD_ERR_STATE, "chronological store not set (lqcd_chrono_reset)");
    if (!c->have_clover) return set_err(c, LQCD_ERR_STATE, "clover term not built");
    const long Vh = c->g.Vh, nh = 12 * Vh, n2 = 24 * Vh;
    const int n = s->count;
    void *buf;
    LQCD_TRY(ws_get(c, WS_HASEN, (size_t)(n + 2) * nh * sizeof(double2), &buf));
    double2 *Y = (double2 *)buf, *e = Y + (size_t)n * nh, *x = e + nh;
    LQCD_TRY(blas_zero(c, nh * sizeof(double2), x));
    int kept = 0;
    if (n > 0) {
        void *tmp;
        LQCD_TRY(ws_get(c, WS_TMP_O, (size_t)n * nh * sizeof(double2), &tmp));
        LQCD_TRY(dirac_dhat(c, LQCD_F64, s->X, Y, tmp, n));
        LQCD_TRY(pack_field(c, LQCD_F64, 1, eta_e, e, 1, false));
        std::vector<Z> G((size_t)n * n), d(n), cf;
        std::vector<double> dots(2 * n);
        for (int j = 0; j < n; j++) {
            LQCD_TRY(blas_dot(c, n2, (const double *)Y, (const double *)(Y + (size_t)j * nh), n, n2, dots.data()));
            for (int i = 0; i < n; i++) G[(size_t)i * n + j] = Z(dots[2 * i], dots[2 * i + 1]);
        }
        LQCD_TRY(blas_dot(c, n2, (const double *)Y, (const double *)e, n, n2, dots.data()));
        for (int i = 0; i < n; i++) d[i] = Z(dots[2 * i], dots[2 * i + 1]);
        kept = chol_solve(n, G, d, cf);
        std::vector<double> coef(2 * n);
        for (int i = 0; i < n; i++) {
            coef[2 * i] = cf[i].real();
            coef[2 * i + 1] = cf[i].imag();
        }
        LQCD_TRY(blas_multi_axpy(c, n2, n, coef.data(), (const double *)s->X, n2, (double *)x, 1.0));
    }
    LQCD_TRY(pack_field(c, LQCD_F64, 1, x0_e, x, 1, true));
    if (nused) *nused = kept;
    return LQCD_OK;
}

}  // extern "C"
