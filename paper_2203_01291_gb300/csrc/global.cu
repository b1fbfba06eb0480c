// Reflection and swap updates of the phonon field (Sec. IV): a global move
// x -> x' at fixed pseudofermion fields Phi, accepted with the Metropolis
// rule (Eq. (metropolis)) on dS = S(x') - S(x), S = S_B + S_F with
// S_F = (1/2) sum_sigma |A^{-T} Phi_sigma|^2 (Eq. (S_again)).
//
// S_F is evaluated as (1/2) sum_sigma b_sigma . v_sigma with
// b = Lambda^{-T}(x) Phi and M^T M v = b (A = M Lambda), i.e. one batched CG
// solve of the n_pf right-hand sides at the proposed field.
#include <math.h>

#include "internal.cuh"

namespace hol {
namespace {

// xp = the proposed field: site line i reflected, or lines i and j exchanged
__global__ void k_propose(const double* __restrict__ x, double* __restrict__ xp, int N, int T,
                          int kind, int i, int j)
{
    const long n = (long)N * T;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x) {
        const int tau = (int)(k / N), s = (int)(k - (long)tau * N);
        const long row = (long)tau * N;
        double val = x[k];
        if (kind == HOL_REFLECT) {
            if (s == i) val = -val;
        } else if (s == i) {
            val = x[row + j];
        } else if (s == j) {
            val = x[row + i];
        }
        xp[k] = val;
    }
}

// S(x) at fixed Phi into host S_out: set-up, b, solve, S_B and S_F terms.
int action_at(hol_ctx* c, const double* x, const double* Phi, int n_pf, const hol_cg_opts* o,
              double* S_out, cudaStream_t s)
{
    int rc;
    if ((rc = hol_set_field(c, x, s))) return rc;
    if ((rc = launch_lambda(c, false, Phi, c->md_b, n_pf, s))) return rc;   // b = Lambda^{-T} Phi
    if ((rc = cg_solve(c, c->md_b, c->md_v, n_pf, o, nullptr, nullptr, s))) return rc;
    double* terms = c->md_s + 8;
    if ((rc = launch_action_terms(c, x, c->md_b, c->md_v, n_pf, terms, s))) return rc;
    double h[2];
    HOL_CUDA(cudaMemcpyAsync(h, terms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HOL_CUDA(cudaStreamSynchronize(s));
    *S_out = h[0] + h[1];
    if (!isfinite(*S_out)) return set_error(HOL_ENUMERIC, "global_update: non-finite action");
    return HOL_OK;
}

}  // namespace
}  // namespace hol

using namespace hol;

extern "C" int global_update(hol_ctx* c, double* x, const double* Phi, int n_pf, int kind, int i,
                             int j, double u, const hol_cg_opts* o, double* S_cur, int* accepted,
                             double* dS, void* stream)
{
    HOL_TRACE("global_update");
    if (!c || !x || !Phi || !o) return set_error(HOL_EINVAL, "global_update: null argument");
    if (int rc_ = require_aligned("global_update", {x, Phi})) return rc_;
    if (n_pf < 1 || n_pf > c->p.max_rhs)
        return set_error(HOL_EINVAL, "global_update: n_pf=%d outside [1, %d]", n_pf,
                         c->p.max_rhs);
    if (kind != HOL_REFLECT && kind != HOL_SWAP)
        return set_error(HOL_EINVAL, "global_update: bad kind %d", kind);
    if (i < 0 || i >= c->N || (kind == HOL_SWAP && (j < 0 || j >= c->N || j == i)))
        return set_error(HOL_EINVAL, "global_update: bad sites (%d, %d)", i, j);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    double S0;
    if (S_cur != nullptr && isfinite(*S_cur)) {
        S0 = *S_cur;
    } else if ((rc = action_at(c, x, Phi, n_pf, o, &S0, s))) {
        return rc;
    }
    double* xp = c->md_x0;
    k_propose<<<ceil_div(c->n, 256) < 4096 ? ceil_div(c->n, 256) : 4096, 256, 0, s>>>(
        x, xp, c->N, c->T, kind, i, j);
    HOL_CHECK_LAUNCH("k_propose");
    double S1;
    if ((rc = action_at(c, xp, Phi, n_pf, o, &S1, s))) return rc;
    const double d = S1 - S0;
    const int acc = (u < exp(-d)) ? 1 : 0;
    if (acc) {
        HOL_CUDA(cudaMemcpyAsync(x, xp, c->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if ((rc = hol_set_field(c, x, s))) {   // the context describes the kept field
        return rc;
    }
    HOL_CUDA(cudaStreamSynchronize(s));
    if (S_cur) *S_cur = acc ? S1 : S0;
    if (accepted) *accepted = acc;
    if (dS) *dS = d;
    return HOL_OK;
}
