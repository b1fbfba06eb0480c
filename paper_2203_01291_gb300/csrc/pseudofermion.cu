// Pseudofermion sampling and the CG right-hand side (Sec. II D).
//   Phi = A^T R = Lambda^T M^T R                       (Eq. (PhiSample-1))
//   b   = Lambda^{-T} Phi                              (below Eq. (psi_def))
// with Lambda of Eq. (Lambda_def): (Lambda^T w)_{i,tau} = s'_tau
// exp(+dtau alpha x_{i,tau}/2) w_{i,tau-1} and (Lambda^{-T} w)_{i,tau} =
// s'_{tau+1} exp(-dtau alpha x_{i,tau+1}/2) w_{i,tau+1}, where s'_0 = +1 and
// s'_tau = -1 otherwise (tau periodic).
#include "internal.cuh"

namespace hol {
namespace {

// out[k][tau][i] = s'_tau e^{+h x[tau][i]} w[k][tau-1][i]        (LT = true)
// out[k][tau][i] = s'_{tau+1} e^{-h x[tau+1][i]} w[k][tau+1][i]  (LT = false)
template <bool LT>
__global__ void k_lambda(const double* __restrict__ w, const double* __restrict__ x,
                         double* __restrict__ out, int N, int T, int nv, double h)
{
    const long n = (long)N * T;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n * nv;
         k += (long)gridDim.x * blockDim.x) {
        const long vb = (k / n) * n;
        const long e = k - vb;
        const int tau = (int)(e / N), i = (int)(e - (long)tau * N);
        if (LT) {
            const int tm = tau == 0 ? T - 1 : tau - 1;
            const double sg = tau == 0 ? 1.0 : -1.0;
            out[k] = sg * exp(h * x[e]) * w[vb + (long)tm * N + i];
        } else {
            const int tp = tau + 1 == T ? 0 : tau + 1;
            const double sg = tp == 0 ? 1.0 : -1.0;
            out[k] = sg * exp(-h * x[(long)tp * N + i]) * w[vb + (long)tp * N + i];
        }
    }
}

}  // namespace

int launch_lambda(const hol_ctx* c, bool transpose_forward, const double* w, double* out, int nv,
                  cudaStream_t s)
{
    const long tot = c->n * nv;
    int nb = ceil_div(tot, 256);
    if (nb > 8192) nb = 8192;
    const double h = 0.5 * c->p.dtau * c->p.alpha;
    if (transpose_forward)
        k_lambda<true><<<nb, 256, 0, s>>>(w, c->x, out, c->N, c->T, nv, h);
    else
        k_lambda<false><<<nb, 256, 0, s>>>(w, c->x, out, c->N, c->T, nv, h);
    HOL_CHECK_LAUNCH("k_lambda");
    return HOL_OK;
}

}  // namespace hol

using namespace hol;

extern "C" int pseudofermion_phi(hol_ctx* c, const double* R, double* Phi, int n_pf, void* stream)
{
    HOL_TRACE("pseudofermion_phi");
    if (!c || !R || !Phi) return set_error(HOL_EINVAL, "pseudofermion_phi: null argument");
    if (int rc_ = require_aligned("pseudofermion_phi", {R, Phi})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "pseudofermion_phi: hol_set_field not called");
    if (n_pf < 1 || n_pf > c->p.max_rhs)
        return set_error(HOL_EINVAL, "pseudofermion_phi: n_pf=%d outside [1, %d]", n_pf,
                         c->p.max_rhs);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_MT(c, HOL_F64, R, c->v64e, n_pf, nullptr, s);
    if (rc) return rc;
    return launch_lambda(c, true, c->v64e, Phi, n_pf, s);
}

extern "C" int phi_to_rhs(hol_ctx* c, const double* Phi, double* b, int n_pf, void* stream)
{
    HOL_TRACE("phi_to_rhs");
    if (!c || !Phi || !b) return set_error(HOL_EINVAL, "phi_to_rhs: null argument");
    if (int rc_ = require_aligned("phi_to_rhs", {Phi, b})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "phi_to_rhs: hol_set_field not called");
    if (n_pf < 1 || n_pf > c->p.max_rhs)
        return set_error(HOL_EINVAL, "phi_to_rhs: n_pf=%d outside [1, %d]", n_pf, c->p.max_rhs);
    if (Phi == b) return set_error(HOL_EINVAL, "phi_to_rhs: Phi and b must not overlap");
    return launch_lambda(c, false, Phi, b, n_pf, (cudaStream_t)stream);
}
