// Fermion operators with the exact kinetic propagator exp(-dtau K) in place
// of the checkerboard product (a second discretisation of B_tau, Sec. II D):
// the scalar-layout kernels of mvscalar.cuh instantiated with EX = true.
// This file: M v and M^T u; exact_cg.cu: the CG-step variants.
// Every other launch shape is refused for such a context (context.cu), so
// these five calls carry all its operator work (and occ64_warm_exact fills
// the occupancy caches of their FP64 kernels).
#include "internal.cuh"
#include "mvscalar.cuh"

namespace hol {

void occ64_warm_exact(const hol_ctx* c)
{
    switch (c->L) {
#define X(LL) case LL: occ64_warm_l<LL, true>(); return;
        HOL_FOR_EACH_L(X)
#undef X
    }
}

int launch_M_exact(const hol_ctx* c, int prec, const void* v, void* out, int n_rhs,
                   const int* mask, double* norm_part, cudaStream_t s)
{
    switch (c->L) {
#define X(LL) case LL: return run_M<LL, true>(c, prec, v, out, n_rhs, mask, norm_part, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_MT_exact(const hol_ctx* c, int prec, const void* u, void* out, int n_rhs,
                    const int* mask, cudaStream_t s)
{
    switch (c->L) {
#define X(LL) case LL: return run_MT<LL, true>(c, prec, u, out, n_rhs, mask, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

}  // namespace hol
