// Fourier-accelerated, time-step-split leapfrog (Sec. III B, Algorithm 1).
//
// Dynamical mass (Sec. III B 1, Eq. (dynamical_M_def)):
//   Mass~_omega = dtau (m_reg^2 + omega0^2 + (4/dtau^2) sin^2(pi omega/T))
//                 / (m_reg^2 + omega0^2),   Mass = F^{-1} Mass~ F along tau,
// (m_reg = inf gives the constant mass dtau). Mass^{-1} p, Mass^{1/2} R and
// p.Mass^{-1}p are applied with one shared-memory kernel per call: forward
// FFT of each site's tau line, multiplication by the table, inverse FFT
// (fft.cuh), with an axpy epilogue so the drift x += dt' Mass^{-1} p is one
// launch.
//
// One trajectory (Algorithm 1): Phi = A^T R (pseudofermion.cu), p = Mass^{1/2}
// R_p, H_i = S_B + |R|^2/2 + p.Mass^{-1}p/2; N_t steps of
//   p -= dt/2 dS_F/dx;  n_t x { p -= dt'/2 dS_B/dx; x += dt' Mass^{-1} p;
//                              p -= dt'/2 dS_B/dx };  p -= dt/2 dS_F/dx
// (the closing and opening fermion half kicks of consecutive steps act at the
// same x and are merged into one force evaluation); H_f with a tight solve;
// Metropolis with the caller's uniform draw.
#include <math.h>

#include "cb.cuh"
#include "fft.cuh"
#include "internal.cuh"

namespace hol {
namespace {

using namespace fft;

// g[k*T + omega]: k = 0 Mass~^{-1}, 1 Mass~^{1/2}, 2 Mass~
__global__ void k_mass_tables(double* __restrict__ g, int T, double dtau, double omega0,
                              double m_reg)
{
    for (int w = threadIdx.x; w < T; w += blockDim.x) {
        double m;
        if (isinf(m_reg)) {
            m = dtau;
        } else {
            const double mr2 = m_reg * m_reg + omega0 * omega0;
            const double s = sinpi((double)w / T);
            m = dtau * (mr2 + 4.0 / (dtau * dtau) * s * s) / mr2;
        }
        g[w] = 1.0 / m;
        g[T + w] = sqrt(m);
        g[2 * T + w] = m;
    }
}

// out = base + coef * (F^{-1} diag(g) F in) along tau for TS sites per block
// (base may be null; out may alias base). g is real and symmetric
// (g[w] = g[T-w]), so the filter maps real lines to real lines and two lines
// share one complex transform: z = x_a + i x_b gives y_a + i y_b.
__global__ void __launch_bounds__(256) k_tau_filter(const double* __restrict__ in, const double* base,
                                                    double* out, double coef,
                                                    const double* __restrict__ g,
                                                    const double2* __restrict__ w2, int T, int N,
                                                    int TS, RadixPlan plan)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TH = TS / 2;
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (long)T * TH;
    const int i0 = blockIdx.x * TS;
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, tau = item / TH;
        const int i = i0 + 2 * c;   // N is even, so i < N implies i + 1 < N
        a[tau * TH + c] = i < N ? make_double2(in[(long)tau * N + i], in[(long)tau * N + i + 1])
                                : make_double2(0.0, 0.0);
    }
    double2* res = fft_tau<double>(a, b, w2, T, TH, plan);
    // conj(g X): the forward transform of it is T times the conjugate of the
    // inverse transform of g X
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, w = item / TH;
        double2 z = res[w * TH + c];
        const double gw = g[w];
        res[w * TH + c] = make_double2(gw * z.x, -gw * z.y);
    }
    double2* oth = (res == a) ? b : a;
    double2* res2 = fft_tau<double>(res, oth, w2, T, TH, plan);
    const double scale = coef / T;
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, tau = item / TH;
        const int i = i0 + 2 * c;
        if (i < N) {
            const long k = (long)tau * N + i;
            const double2 z = res2[tau * TH + c];   // T conj(y_a + i y_b)
            out[k] = (base != nullptr ? base[k] : 0.0) + scale * z.x;
            out[k + 1] = (base != nullptr ? base[k + 1] : 0.0) - scale * z.y;
        }
    }
}

// p -= c * dS_B/dx (Eq. (dSB_dx))
__global__ void k_boson_kick(double* __restrict__ p, const double* __restrict__ x, int N, int T,
                             double c, double dtau, double w02)
{
    const long n = (long)N * T;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x) {
        const int tau = (int)(k / N), i = (int)(k - (long)tau * N);
        const int tp = tau + 1 == T ? 0 : tau + 1, tm = tau == 0 ? T - 1 : tau - 1;
        const double xc = x[k];
        const double lap = x[(long)tp * N + i] - 2.0 * xc + x[(long)tm * N + i];
        p[k] -= c * dtau * (w02 * xc - lap / (dtau * dtau));
    }
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, long n)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x)
        y[k] = fma(a, x[k], y[k]);
}

// y += -(*coef) x: the kick of k_axpy with its coefficient read on the
// device (a captured step graph serves every step of a trajectory)
__global__ void k_axpy_dev(double* __restrict__ y, const double* __restrict__ x,
                           const double* __restrict__ coef, long n)
{
    const double a = -coef[0];
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x)
        y[k] = fma(a, x[k], y[k]);
}

__global__ void k_set1(double* __restrict__ dst, double value) { *dst = value; }

// out[0] = scale * sum_k a[k] b[k] (one block, fixed order)
__global__ void __launch_bounds__(1024) k_dot1(const double* __restrict__ a,
                                               const double* __restrict__ b, long n, double scale,
                                               double* __restrict__ out)
{
    __shared__ double red[32];
    double s = 0.0;
    for (long k = threadIdx.x; k < n; k += blockDim.x) s += a[k] * b[k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        *out = scale * t;
    }
}

// out[0] = S_B(x) (Eq. (S_B)), one block
__global__ void __launch_bounds__(1024) k_sb1(const double* __restrict__ x, int N, int T,
                                              double dtau, double w02, double* __restrict__ out)
{
    __shared__ double red[32];
    const long n = (long)N * T;
    double s = 0.0;
    for (long k = threadIdx.x; k < n; k += blockDim.x) {
        const int tau = (int)(k / N), i = (int)(k - (long)tau * N);
        const int tp = tau + 1 == T ? 0 : tau + 1;
        const double xc = x[k], d = (x[(long)tp * N + i] - xc) / dtau;
        s += w02 * xc * xc + d * d;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        *out = 0.5 * dtau * t;
    }
}

// Sites per tile of the tau filter: 16 on the largest lattice, 4 below it so
// that small lattices still spread over many blocks.
int filter_tile(const hol_ctx* c) { return c->N >= 1024 ? 16 : 4; }

int grid_1d(long n)
{
    long nb = (n + 255) / 256;
    return (int)(nb > 8192 ? 8192 : (nb < 1 ? 1 : nb));
}

int filter(hol_ctx* c, const double* in, const double* base, double* out, double coef, int which,
           cudaStream_t s)
{
    const RadixPlan plan = plan_of(c->T);
    if (plan.n < 0) return set_error(HOL_EINVAL, "leapfrog: Ltau=%d has a prime factor > 7", c->T);
    const int ts = filter_tile(c);
    const size_t sm = 2 * (size_t)c->T * (ts / 2) * sizeof(double2);   // two sites per column
    if (int rc = smem_raise((const void*)k_tau_filter, sm)) return rc;
    k_tau_filter<<<ceil_div(c->N, ts), 256, sm, s>>>(in, base, out, coef,
                                                      c->md_g + which * c->T, c->tw64, c->T,
                                                      c->N, ts, plan);
    HOL_CHECK_LAUNCH("k_tau_filter");
    return HOL_OK;
}

int mass_tables(hol_ctx* c, double m_reg, cudaStream_t s)
{
    k_mass_tables<<<1, 256, 0, s>>>(c->md_g, c->T, c->p.dtau, c->p.omega0, m_reg);
    HOL_CHECK_LAUNCH("k_mass_tables");
    return HOL_OK;
}

int boson_kick(hol_ctx* c, double* p, const double* x, double coef, cudaStream_t s)
{
    k_boson_kick<<<grid_1d(c->n), 256, 0, s>>>(p, x, c->N, c->T, coef, c->p.dtau,
                                              c->p.omega0 * c->p.omega0);
    HOL_CHECK_LAUNCH("k_boson_kick");
    return HOL_OK;
}

// F <- dS_F/dx at x for the fixed Phi (set-up, b = Lambda^{-T} Phi, solve, force)
int fermion_force(hol_ctx* c, const double* x, const double* Phi, int n_pf,
                  const hol_cg_opts* cg, cudaStream_t s)
{
    int rc;
    if ((rc = hol_set_field(c, x, s))) return rc;
    if ((rc = launch_lambda(c, false, Phi, c->md_b, n_pf, s))) return rc;
    // inside a graph capture the solve is device-driven (same result)
    rc = c->capturing ? cg_run_dev(c, c->md_b, c->md_v, n_pf, cg, s)
                      : cg_solve(c, c->md_b, c->md_v, n_pf, cg, nullptr, nullptr, s);
    if (rc) return rc;
    timer_start(c, KT_FORCE, s);
    rc = launch_force(c, c->md_v, c->md_b, n_pf, c->md_F, 0, nullptr, s);
    timer_stop(c, KT_FORCE, s);
    return rc;
}

int check_md(const hol_ctx* c, const hol_md_opts* o, int n_pf)
{
    if (!o) return set_error(HOL_EINVAL, "leapfrog: null options");
    if (!(o->dt > 0.0) || o->n_steps < 0 || o->n_sub < 1)
        return set_error(HOL_EINVAL, "leapfrog: dt > 0, n_steps >= 0, n_sub >= 1 required");
    if (!(o->m_reg >= 0.0)) return set_error(HOL_EINVAL, "leapfrog: m_reg must be >= 0 or inf");
    if (n_pf < 1 || n_pf > c->p.max_rhs)
        return set_error(HOL_EINVAL, "leapfrog: n_pf=%d outside [1, %d]", n_pf, c->p.max_rhs);
    if (plan_of(c->T).n < 0) return set_error(HOL_EINVAL, "leapfrog: Ltau has a prime factor > 7");
    return HOL_OK;
}

int md_run(hol_ctx* c, double* x, double* p, const double* Phi, int n_pf, const hol_md_opts* o,
           cudaStream_t s)
{
    int rc;
    if ((rc = mass_tables(c, o->m_reg, s))) return rc;
    if (o->n_steps == 0) return HOL_OK;
    const double dt = o->dt, dts = o->dt / o->n_sub;
    if ((rc = fermion_force(c, x, Phi, n_pf, &o->cg_force, s))) return rc;
    k_axpy<<<grid_1d(c->n), 256, 0, s>>>(p, c->md_F, -0.5 * dt, c->n);
    HOL_CHECK_LAUNCH("k_axpy");
    for (int t = 0; t < o->n_steps; ++t) {
        for (int k = 0; k < o->n_sub; ++k) {
            if ((rc = boson_kick(c, p, x, 0.5 * dts, s))) return rc;
            if ((rc = filter(c, p, x, x, dts, 0, s))) return rc;   // x += dt' Mass^{-1} p
            if ((rc = boson_kick(c, p, x, 0.5 * dts, s))) return rc;
        }
        if ((rc = fermion_force(c, x, Phi, n_pf, &o->cg_force, s))) return rc;
        const double kick = (t + 1 == o->n_steps) ? 0.5 * dt : dt;
        k_axpy<<<grid_1d(c->n), 256, 0, s>>>(p, c->md_F, -kick, c->n);
        HOL_CHECK_LAUNCH("k_axpy");
    }
    return HOL_OK;
}

}  // namespace

// The three parts of fourier_accel_leapfrog that a captured batch replays
// (graph.cu), with the kernel sequence of fourier_accel_leapfrog / md_run:
// the start (Phi, p, H_i, the first force and half kick), one leapfrog step
// (n_sub bosonic sub-steps, the force, the kick by the device-side
// coefficient md_s[kKickSlot]) and the end (the tight action solve and H_f).
int md_start(hol_ctx* c, double* x, const double* R_pf, const double* R_p, int n_pf,
             const hol_md_opts* o, cudaStream_t s)
{
    int rc;
    const long n = c->n;
    double* sc = c->md_s;
    if ((rc = hol_set_field(c, x, s))) return rc;
    if ((rc = launch_MT(c, HOL_F64, R_pf, c->v64e, n_pf, nullptr, s))) return rc;
    if ((rc = launch_lambda(c, true, c->v64e, c->md_phi, n_pf, s))) return rc;
    if ((rc = mass_tables(c, o->m_reg, s))) return rc;
    if ((rc = filter(c, R_p, nullptr, c->md_p, 1.0, 1, s))) return rc;
    HOL_CUDA(cudaMemcpyAsync(c->md_x0, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const double w02 = c->p.omega0 * c->p.omega0;
    k_sb1<<<1, 1024, 0, s>>>(x, c->N, c->T, c->p.dtau, w02, sc + 0);
    k_dot1<<<1, 1024, 0, s>>>(R_pf, R_pf, (long)n_pf * n, 0.5, sc + 1);
    if ((rc = filter(c, c->md_p, nullptr, c->md_F, 1.0, 0, s))) return rc;
    k_dot1<<<1, 1024, 0, s>>>(c->md_p, c->md_F, n, 0.5, sc + 2);
    HOL_CHECK_LAUNCH("initial energies");
    // md_run up to its first half kick
    if ((rc = mass_tables(c, o->m_reg, s))) return rc;
    if ((rc = fermion_force(c, x, c->md_phi, n_pf, &o->cg_force, s))) return rc;
    k_axpy<<<grid_1d(c->n), 256, 0, s>>>(c->md_p, c->md_F, -0.5 * o->dt, c->n);
    HOL_CHECK_LAUNCH("k_axpy");
    return md_set_kick(c, o->n_steps == 1 ? 0.5 * o->dt : o->dt, s);
}

int md_set_kick(hol_ctx* c, double kick, cudaStream_t s)
{
    k_set1<<<1, 1, 0, s>>>(c->md_s + kKickSlot, kick);
    HOL_CHECK_LAUNCH("k_set1");
    return HOL_OK;
}

int md_step(hol_ctx* c, double* x, int n_pf, const hol_md_opts* o, cudaStream_t s)
{
    int rc;
    const double dts = o->dt / o->n_sub;
    for (int k = 0; k < o->n_sub; ++k) {
        if ((rc = boson_kick(c, c->md_p, x, 0.5 * dts, s))) return rc;
        if ((rc = filter(c, c->md_p, x, x, dts, 0, s))) return rc;
        if ((rc = boson_kick(c, c->md_p, x, 0.5 * dts, s))) return rc;
    }
    if ((rc = fermion_force(c, x, c->md_phi, n_pf, &o->cg_force, s))) return rc;
    k_axpy_dev<<<grid_1d(c->n), 256, 0, s>>>(c->md_p, c->md_F, c->md_s + kKickSlot, c->n);
    HOL_CHECK_LAUNCH("k_axpy_dev");
    return HOL_OK;
}

int md_end(hol_ctx* c, double* x, int n_pf, const hol_md_opts* o, cudaStream_t s)
{
    int rc;
    const long n = c->n;
    double* sc = c->md_s;
    const double w02 = c->p.omega0 * c->p.omega0;
    if ((rc = hol_set_field(c, x, s))) return rc;
    if ((rc = launch_lambda(c, false, c->md_phi, c->md_b, n_pf, s))) return rc;
    rc = c->capturing ? cg_run_dev(c, c->md_b, c->md_v, n_pf, &o->cg_action, s)
                      : cg_solve(c, c->md_b, c->md_v, n_pf, &o->cg_action, nullptr, nullptr, s);
    if (rc) return rc;
    k_sb1<<<1, 1024, 0, s>>>(x, c->N, c->T, c->p.dtau, w02, sc + 3);
    k_dot1<<<1, 1024, 0, s>>>(c->md_b, c->md_v, (long)n_pf * n, 0.5, sc + 4);
    if ((rc = filter(c, c->md_p, nullptr, c->md_F, 1.0, 0, s))) return rc;
    k_dot1<<<1, 1024, 0, s>>>(c->md_p, c->md_F, n, 0.5, sc + 5);
    HOL_CHECK_LAUNCH("final energies");
    return HOL_OK;
}

int md_check(const hol_ctx* c, const hol_md_opts* o, int n_pf) { return check_md(c, o, n_pf); }

int leapfrog_alloc(hol_ctx* c)
{
    const long n = c->n, R = c->p.max_rhs;
    HOL_CUDA(cudaMalloc((void**)&c->md_phi, R * n * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_b, R * n * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_v, R * n * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_F, n * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_p, n * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_x0, n * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_g, 3 * c->T * sizeof(double)));
    HOL_CUDA(cudaMalloc((void**)&c->md_s, 16 * sizeof(double)));
    return HOL_OK;
}

int launch_action_terms(const hol_ctx* c, const double* x, const double* b, const double* v,
                        int n_pf, double* out2, cudaStream_t s)
{
    const double w02 = c->p.omega0 * c->p.omega0;
    k_sb1<<<1, 1024, 0, s>>>(x, c->N, c->T, c->p.dtau, w02, out2);
    HOL_CHECK_LAUNCH("k_sb1");
    k_dot1<<<1, 1024, 0, s>>>(b, v, (long)n_pf * c->n, 0.5, out2 + 1);
    HOL_CHECK_LAUNCH("k_dot1");
    return HOL_OK;
}

}  // namespace hol

using namespace hol;

extern "C" int mass_apply(hol_ctx* c, int which, double m_reg, const double* p, double* out,
                          void* stream)
{
    HOL_TRACE("mass_apply");
    if (!c || !p || !out) return set_error(HOL_EINVAL, "mass_apply: null argument");
    if (int rc_ = require_aligned("mass_apply", {p, out})) return rc_;
    if (which < 0 || which > 2) return set_error(HOL_EINVAL, "mass_apply: bad selector %d", which);
    if (!(m_reg >= 0.0)) return set_error(HOL_EINVAL, "mass_apply: m_reg must be >= 0 or inf");
    if (plan_of(c->T).n < 0) return set_error(HOL_EINVAL, "mass_apply: Ltau has a prime factor > 7");
    if (p == out) return set_error(HOL_EINVAL, "mass_apply: p and out must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = mass_tables(c, m_reg, s);
    if (rc) return rc;
    return filter(c, p, nullptr, out, 1.0, which, s);
}

extern "C" int md_integrate(hol_ctx* c, double* x, double* p, const double* Phi, int n_pf,
                            const hol_md_opts* o, void* stream)
{
    HOL_TRACE("md_integrate");
    if (!c || !x || !p || !Phi) return set_error(HOL_EINVAL, "md_integrate: null argument");
    if (int rc_ = require_aligned("md_integrate", {x, p, Phi})) return rc_;
    int rc = check_md(c, o, n_pf);
    if (rc) return rc;
    return md_run(c, x, p, Phi, n_pf, o, (cudaStream_t)stream);
}

extern "C" int fourier_accel_leapfrog(hol_ctx* c, double* x, const double* R_pf, const double* R_p,
                                      int n_pf, const hol_md_opts* o, double u, int* accepted,
                                      double* dH, double* terms, void* stream)
{
    HOL_TRACE("fourier_accel_leapfrog");
    if (!c || !x || !R_pf || !R_p) return set_error(HOL_EINVAL, "fourier_accel_leapfrog: null argument");
    if (int rc_ = require_aligned("fourier_accel_leapfrog", {x, R_pf, R_p})) return rc_;
    int rc = check_md(c, o, n_pf);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const long n = c->n;
    double* sc = c->md_s;   // [0] S_B_i [1] S_F_i [2] K_i [3] S_B_f [4] S_F_f [5] K_f
    // initial state (Algorithm 1): Phi = A^T(x_i) R, p = Mass^{1/2} R_p
    if ((rc = hol_set_field(c, x, s))) return rc;
    if ((rc = launch_MT(c, HOL_F64, R_pf, c->v64e, n_pf, nullptr, s))) return rc;
    if ((rc = launch_lambda(c, true, c->v64e, c->md_phi, n_pf, s))) return rc;
    if ((rc = mass_tables(c, o->m_reg, s))) return rc;
    if ((rc = filter(c, R_p, nullptr, c->md_p, 1.0, 1, s))) return rc;
    HOL_CUDA(cudaMemcpyAsync(c->md_x0, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    const double w02 = c->p.omega0 * c->p.omega0;
    k_sb1<<<1, 1024, 0, s>>>(x, c->N, c->T, c->p.dtau, w02, sc + 0);
    k_dot1<<<1, 1024, 0, s>>>(R_pf, R_pf, (long)n_pf * n, 0.5, sc + 1);   // S_F(x_i) = |R|^2/2
    if ((rc = filter(c, c->md_p, nullptr, c->md_F, 1.0, 0, s))) return rc;
    k_dot1<<<1, 1024, 0, s>>>(c->md_p, c->md_F, n, 0.5, sc + 2);
    HOL_CHECK_LAUNCH("initial energies");
    // molecular dynamics
    if ((rc = md_run(c, x, c->md_p, c->md_phi, n_pf, o, s))) return rc;
    // final energies with the tight solve
    if ((rc = hol_set_field(c, x, s))) return rc;
    if ((rc = launch_lambda(c, false, c->md_phi, c->md_b, n_pf, s))) return rc;
    if ((rc = cg_solve(c, c->md_b, c->md_v, n_pf, &o->cg_action, nullptr, nullptr, s))) return rc;
    k_sb1<<<1, 1024, 0, s>>>(x, c->N, c->T, c->p.dtau, w02, sc + 3);
    k_dot1<<<1, 1024, 0, s>>>(c->md_b, c->md_v, (long)n_pf * n, 0.5, sc + 4);
    if ((rc = filter(c, c->md_p, nullptr, c->md_F, 1.0, 0, s))) return rc;
    k_dot1<<<1, 1024, 0, s>>>(c->md_p, c->md_F, n, 0.5, sc + 5);
    HOL_CHECK_LAUNCH("final energies");
    double h[6];
    HOL_CUDA(cudaMemcpyAsync(h, sc, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HOL_CUDA(cudaStreamSynchronize(s));
    const double d = (h[3] + h[4] + h[5]) - (h[0] + h[1] + h[2]);
    if (!isfinite(d)) return set_error(HOL_ENUMERIC, "fourier_accel_leapfrog: non-finite dH");
    const int acc = (u < exp(-d)) ? 1 : 0;
    if (!acc) HOL_CUDA(cudaMemcpyAsync(x, c->md_x0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HOL_CUDA(cudaStreamSynchronize(s));
    if (dH) *dH = d;
    if (accepted) *accepted = acc;
    if (terms)
        for (int k = 0; k < 6; ++k) terms[k] = h[k];
    return HOL_OK;
}
