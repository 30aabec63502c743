// Local deflation (placeholder until the subspace kernels land).
#include "lqcd_internal.cuh"

struct DflState {
    int Ns;
};

void dfl_free(lqcd_ctx *c)
{
    delete c->dfl;
    c->dfl = nullptr;
}

lqcd_status dfl_precond_native(lqcd_ctx *c, const lqcd_sap_params *, const double2 *, double2 *)
{
    return set_err(c, LQCD_ERR_STATE, "deflation subspace not built");
}

extern "C" {
lqcd_status lqcd_dfl_build(lqcd_ctx *c, const lqcd_dfl_params *, const double *)
{
    return set_err(c, LQCD_ERR_STATE, "deflation not available");
}
lqcd_status lqcd_dfl_export(lqcd_ctx *c, double *, double *) { return set_err(c, LQCD_ERR_STATE, "no subspace"); }
lqcd_status lqcd_dfl_project(lqcd_ctx *c, const double *, double *) { return set_err(c, LQCD_ERR_STATE, "no subspace"); }
lqcd_status lqcd_dfl_expand(lqcd_ctx *c, const double *, double *) { return set_err(c, LQCD_ERR_STATE, "no subspace"); }
lqcd_status lqcd_dfl_little_apply(lqcd_ctx *c, const double *, double *)
{
    return set_err(c, LQCD_ERR_STATE, "no subspace");
}
lqcd_status lqcd_dfl_coarse_solve(lqcd_ctx *c, const double *, double *, int *)
{
    return set_err(c, LQCD_ERR_STATE, "no subspace");
}
lqcd_status lqcd_dfl_precond(lqcd_ctx *c, const lqcd_sap_params *, const double *, double *)
{
    return set_err(c, LQCD_ERR_STATE, "no subspace");
}
}
