// Adiabatic preconditioner of Sec. VI (filled in below).
#include "internal.cuh"

namespace hol {
int kpm_setup(hol_ctx* c, cudaStream_t s)
{
    (void)c;
    (void)s;
    return HOL_OK;
}
}  // namespace hol
namespace hol {
int cg_precond(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
               int* iters, double* resid, cudaStream_t s)
{
    (void)c; (void)b; (void)v; (void)n_rhs; (void)o; (void)iters; (void)resid; (void)s;
    return set_error(HOL_EINVAL, "cg_solve: preconditioner not available yet");
}
}  // namespace hol
