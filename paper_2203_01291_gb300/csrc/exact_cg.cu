// Fermion operators with the exact kinetic propagator exp(-dtau K) in place
// of the checkerboard product (a second discretisation of B_tau, Sec. II D):
// the scalar-layout kernels of mvscalar.cuh instantiated with EX = true.
// This file: the CG-step variants (FP64 direction update fused with M,
// FP64 residual b - M^T u, FP32 fused M^T M step); exact.cu: M v and M^T u.
// Every other launch shape is refused for such a context (context.cu), so
// these five calls carry all its operator work.
#include "internal.cuh"
#include "mvscalar.cuh"

namespace hol {

void fp64_cg_geom_exact(const hol_ctx* c, int n_rhs, int* pstride, int* nrun)
{
    switch (c->L) {
#define X(LL)                                                \
    case LL: {                                               \
        const MvGeom g = geom_m_upd64<LL, true>(c, n_rhs);   \
        *pstride = g.pstride;                                \
        *nrun = g.nrun;                                      \
        return;                                              \
    }
        HOL_FOR_EACH_L(X)
#undef X
    }
}

int launch_M_upd64_exact(const hol_ctx* c, const double* r, const double* pold, double* pnew,
                         double* w, int n_rhs, const int* mask, BetaSrc beta,
                         double* norm_part, cudaStream_t s)
{
    switch (c->L) {
#define X(LL) \
    case LL: return run_M_upd64<LL, true>(c, r, pold, pnew, w, n_rhs, mask, beta, norm_part, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_MT_resid64_exact(const hol_ctx* c, const double* u, const double* b, double* out,
                            int n_rhs, const int* mask, cudaStream_t s)
{
    switch (c->L) {
#define X(LL) case LL: return run_MT_resid<LL, true>(c, u, b, out, n_rhs, mask, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_cg_mtm32_exact(const hol_ctx* c, const float* r, const float* pold, float* pnew,
                          float* q, int n_rhs, const int* mask, const double* rr_new,
                          const double* rr_old, int rr_stride, int rr_n, int first,
                          double* pq_part, cudaStream_t s)
{
    switch (c->L) {
#define X(LL)                                                                                \
    case LL:                                                                                 \
        return run_cg_mtm32_scalar<LL, true>(c, r, pold, pnew, q, n_rhs, mask, rr_new, rr_old, \
                                             rr_stride, rr_n, first, pq_part, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

}  // namespace hol
