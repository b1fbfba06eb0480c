// Phonon force dS/dx = dS_B/dx + dS_F/dx (Sec. III A) and S_F (Eq. (Sf_Psi)).
//
// With b = Lambda^{-T} Phi and v = (M^T M)^{-1} b, Eq. (dSF_dx) with
// dA = dM Lambda + M dLambda reduces, for the Holstein B_tau, to one M sweep:
//   dS_F/dx_{i,tau} = dtau alpha s_tau u_{i,tau} y_{i,tau}
//                     - (dtau alpha / 2) b_{i,tau-1} v_{i,tau-1},
//   y_tau = exp(-dtau V_tau) C v_{tau-1},  u_tau = v_tau + s_tau y_tau,
// so the kernel recomputes B_tau v_{tau-1} slice by slice (nothing of M is
// stored) and adds the bosonic stencil of Eq. (dSB_dx). C is the checkerboard
// product or, for a context with the exact propagator, exp(-dtau K).
#include "cb.cuh"
#include "internal.cuh"

namespace hol {
namespace {

struct ForceArgs {
    int T, K, nrun, n_pf;
    int pg;          // pseudofermions per group (blockIdx.y selects the group)
    int groups;      // > 1: each group writes its partial force to Fp[group]
    long n;
    int with_bos;
    double da, dtau, w02;
    double inv_dtau;   // 1 / dtau, so the stencil needs no division
    Kin<double> kin;   // propagator (checkerboard or exact)
};

template <int L, bool EX>
__global__ void __launch_bounds__(32) k_force(const double* __restrict__ v,
                                               const double* __restrict__ b,
                                               const double* __restrict__ x,
                                               const double* __restrict__ ev,
                                               double* __restrict__ F,
                                               double* __restrict__ sf_part, ForceArgs a)
{
    constexpr int N = L * L;
    const LaneGeom<L> geo;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp * LaneGeom<L>::G >= a.nrun) return;
    const int run = warp * LaneGeom<L>::G + geo.g;
    const bool valid = geo.ok && run < a.nrun;
    const int t0 = (run < a.nrun ? run : a.nrun - 1) * a.K;
    const int grp = blockIdx.y;
    const int sp0 = grp * a.pg;
    const int sp1 = (sp0 + a.pg < a.n_pf) ? sp0 + a.pg : a.n_pf;
    const bool bos = a.with_bos && a.groups == 1;   // else added by k_force_sum
    double* Fout = F + (a.groups > 1 ? (long)grp * a.n : 0L);
    double acc = 0.0;
    for (int s = 0; s < a.K; ++s) {
        const int tau = t0 + s;
        const int tm = (tau == 0) ? a.T - 1 : tau - 1;
        const int tp = (tau + 1 == a.T) ? 0 : tau + 1;
        const double sg = (tau == 0) ? 1.0 : -1.0;
        // f accumulates the fermion force over the group divided by dtau alpha:
        // sum_sigma y (y + s_tau v_tau) - b_{tau-1} v_{tau-1} / 2
        double f[L];
#pragma unroll
        for (int iy = 0; iy < L; ++iy) f[iy] = 0.0;
        for (int sp = sp0; sp < sp1; ++sp) {
            const long base = (long)sp * a.n + geo.ix;
            double c[L];
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                const long o = base + (long)tm * N + iy * L;
                const double vv = v[o];
                const double bv = b[o] * vv;
                acc += bv;
                f[iy] = fma(-0.5, bv, f[iy]);
                c[iy] = vv;
            }
            kin_apply<double, L, EX>(c, geo, a.kin);
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                const double y = ev[(long)tau * N + iy * L + geo.ix] * c[iy];
                const double vt = v[base + (long)tau * N + iy * L];
                f[iy] = fma(y, fma(sg, vt, y), f[iy]);
            }
        }
        if (valid) {
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                double fo = a.da * f[iy];
                if (bos) {
                    const long o = iy * L + geo.ix;
                    const double xc = x[(long)tau * N + o];
                    const double lap = x[(long)tp * N + o] - 2.0 * xc + x[(long)tm * N + o];
                    fo += a.dtau * a.w02 * xc - lap * a.inv_dtau;
                }
                Fout[(long)tau * N + iy * L + geo.ix] = fo;
            }
        }
    }
    // per-unit sum of b.v over the slices tau-1 of the run
    __shared__ double red[32];
    const int lane = threadIdx.x & 31;
    red[lane] = valid ? acc : 0.0;
    __syncwarp();
    if (valid && geo.ix == 0) {
        double ssum = 0.0;
        for (int k = 0; k < L; ++k) ssum += red[geo.g * L + k];
        sf_part[grp * a.nrun + run] = ssum;
    }
}

// F = sum over pseudofermion groups of the partial forces (fixed order)
// plus the bosonic force of Eq. (dSB_dx).
__global__ void k_force_sum(const double* __restrict__ Fp, int groups, const double* __restrict__ x,
                            int N, int T, int with_bos, double dtau, double w02,
                            double inv_dtau, double* __restrict__ F)
{
    const long n = (long)N * T;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x) {
        double f = 0.0;
        for (int g = 0; g < groups; ++g) f += Fp[(long)g * n + k];
        if (with_bos) {
            const int tau = (int)(k / N), i = (int)(k - (long)tau * N);
            const int tp = tau + 1 == T ? 0 : tau + 1, tm = tau == 0 ? T - 1 : tau - 1;
            const double xc = x[k];
            const double lap = x[(long)tp * N + i] - 2.0 * xc + x[(long)tm * N + i];
            f += dtau * w02 * xc - lap * inv_dtau;
        }
        F[k] = f;
    }
}

// S_F = (1/2) sum of the unit partials (one warp).
__global__ void k_sf_finish(const double* __restrict__ part, int cnt, double* __restrict__ out)
{
    const double s = warp_sum_array(part, cnt);
    if (threadIdx.x == 0) *out = 0.5 * s;
}

// Partial sums of b . v over all pseudofermions, one per block in a fixed
// order (the action alone, Eq. (Sf_Psi), without the force).
__global__ void k_sf_dot(const double* __restrict__ v, const double* __restrict__ b, long len,
                         double* __restrict__ part)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < len;
         k += (long)gridDim.x * blockDim.x)
        acc = fma(b[k], v[k], acc);
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        acc = warp_sum(acc);
        if (lane == 0) part[blockIdx.x] = acc;
    }
}

// Launch plan of the force kernel. Nothing is reused between the slices of
// a run, so each run is one slice (K = 1) unless the per-run partial sums of
// S_F would not fit the partial-sum bank. The pseudofermions are split into
// groups run by separate blocks until about eight warps per multiprocessor
// are resident; with more than one group the partial forces go to scratch
// and k_force_sum adds them in a fixed order.
struct ForcePlan {
    int K, nrun, groups, pg;
};

ForcePlan force_plan(const hol_ctx* c, int n_pf)
{
    ForcePlan f;
    f.K = (c->T <= c->part_len) ? 1 : c->mv_k;
    f.nrun = c->T / f.K;
    const int G = 32 / c->L;                       // runs per warp
    const long warps = (f.nrun + G - 1) / G;      // warps per group
    const long target = 8L * c->sms;
    long g = (target + warps - 1) / warps;
    if (g > n_pf) g = n_pf;
    if (g * f.nrun > c->part_len) g = c->part_len / f.nrun;
    if (g < 1) g = 1;
    f.pg = n_pf > 0 ? (int)((n_pf + g - 1) / g) : 0;
    f.groups = f.pg > 0 ? (n_pf + f.pg - 1) / f.pg : 1;
    return f;
}

template <int L>
int run_force(hol_ctx* c, const double* v, const double* b, int n_pf, double* F, int with_bos,
              double* sf_part, cudaStream_t s)
{
    const ForcePlan f = force_plan(c, n_pf);
    ForceArgs a;
    a.T = c->T;
    a.K = f.K;
    a.nrun = f.nrun;
    a.n_pf = n_pf;
    a.pg = f.pg;
    a.groups = f.groups;
    a.n = c->n;
    a.with_bos = with_bos;
    a.kin = kin_of<double>(c);
    a.da = c->p.dtau * c->p.alpha;
    a.dtau = c->p.dtau;
    a.w02 = c->p.omega0 * c->p.omega0;
    a.inv_dtau = 1.0 / c->p.dtau;
    const int warps = ceil_div(a.nrun, LaneGeom<L>::G);
    double* Fp = a.groups > 1 ? c->v64a : F;
    if (c->exact)
        k_force<L, true><<<dim3(warps, a.groups), 32, 0, s>>>(v, b, c->x, c->ev64, Fp, sf_part, a);
    else
        k_force<L, false><<<dim3(warps, a.groups), 32, 0, s>>>(v, b, c->x, c->ev64, Fp, sf_part, a);
    HOL_CHECK_LAUNCH("k_force");
    if (a.groups > 1) {
        const int nb = ceil_div(c->n, 256) < 4096 ? ceil_div(c->n, 256) : 4096;
        k_force_sum<<<nb, 256, 0, s>>>(Fp, a.groups, c->x, c->N, c->T, with_bos, a.dtau, a.w02,
                                       a.inv_dtau, F);
        HOL_CHECK_LAUNCH("k_force_sum");
    }
    return HOL_OK;
}

}  // namespace

int launch_force(hol_ctx* c, const double* v, const double* b, int n_pf, double* F, int with_bos,
                 double* S_F, cudaStream_t s)
{
    double* sf_part = c->part + 6 * c->part_len;
    int rc = HOL_EINVAL;
    switch (c->L) {
#define X(LL) case LL: rc = run_force<LL>(c, v, b, n_pf, F, with_bos, sf_part, s); break;
        X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)
#undef X
    default:
        return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
    }
    if (rc) return rc;
    if (S_F != nullptr) {
        const ForcePlan f = force_plan(c, n_pf);
        k_sf_finish<<<1, 32, 0, s>>>(sf_part, f.groups * f.nrun, S_F);
        HOL_CHECK_LAUNCH("k_sf_finish");
    }
    return HOL_OK;
}

}  // namespace hol

using namespace hol;

extern "C" int force(hol_ctx* c, const double* v, const double* b, int n_pf, double* dSdx,
                     int with_bosonic, double* S_F, void* stream)
{
    HOL_TRACE("force");
    if (!c || !v || !b || (!dSdx && !S_F)) return set_error(HOL_EINVAL, "force: null argument");
    if (int rc_ = require_aligned("force", {v, b, dSdx})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "force: hol_set_field not called");
    if (n_pf < 0 || n_pf > c->p.max_rhs)
        return set_error(HOL_EINVAL, "force: n_pf=%d outside [0, %d]", n_pf, c->p.max_rhs);
    if (!dSdx) {   // the action alone
        cudaStream_t s = (cudaStream_t)stream;
        double* part = c->part + 6 * c->part_len;
        const long len = (long)n_pf * c->n;
        long nb = (len + 255) / 256;
        if (nb > 1024) nb = 1024;
        if (nb > c->part_len) nb = c->part_len;
        if (nb < 1) nb = 1;
        k_sf_dot<<<(int)nb, 256, 0, s>>>(v, b, len, part);
        HOL_CHECK_LAUNCH("k_sf_dot");
        k_sf_finish<<<1, 32, 0, s>>>(part, (int)nb, S_F);
        HOL_CHECK_LAUNCH("k_sf_finish");
        return HOL_OK;
    }
    timer_start(c, KT_FORCE, (cudaStream_t)stream);
    int rc = launch_force(c, v, b, n_pf, dSdx, with_bosonic, S_F, (cudaStream_t)stream);
    timer_stop(c, KT_FORCE, (cudaStream_t)stream);
    return rc;
}
