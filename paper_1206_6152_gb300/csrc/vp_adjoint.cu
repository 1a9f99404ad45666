// vp_adjoint.cu -- discrete adjoint of the split step (not in the paper).
#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"

extern "C" {

int vp_adjoint_step(vp_ctx *c, const void *f_start, const double *g_start, double *lambda_f,
                    double *lambda_g)
{
    (void)c; (void)f_start; (void)g_start; (void)lambda_f; (void)lambda_g;
    return VP_ERR_UNSUPPORTED;
}

int vp_field_adjoint(vp_ctx *c, const double *lambda_g, double *lambda_f)
{
    (void)c; (void)lambda_g; (void)lambda_f;
    return VP_ERR_UNSUPPORTED;
}

int vp_functional(vp_ctx *c, int kind, const double *target, double *lambda_f, double *J_out)
{
    (void)c; (void)kind; (void)target; (void)lambda_f; (void)J_out;
    return VP_ERR_UNSUPPORTED;
}

}  // extern "C"
