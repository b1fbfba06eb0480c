// Adiabatic preconditioner (Sec. VI, App. C) and preconditioned CG.
//
// P^{-1} v = U^dag Ptilde^{-1} U v (Eq. (P_change_basis)) with
// U_{omega,tau} = exp(-2 pi i tau (omega + 1/2)/T)/sqrt(T) (Eq. (U_omega)) and
// the blocks Mtilde_{omega,omega}^{-1} = (I - e^{-i phi_omega} Bbar)^{-1}
// approximated by the Chebyshev series sum_m c_m T_m(A), A = 2(Bbar -
// bmin)/db - 1 (Eqs. (A_def), (f_A_approx), (Minv_KPM), (alpha_recur)).
// Only omega < T/2 is computed; omega' = T-1-omega is the complex conjugate
// (App. C B), so a real v maps to a real result.
//
// The transpose used by PCG is the exact transpose of the approximation,
// P^{-T} = U^dag diag(sum conj(c_m) T_m(A^T)) U, A^T built from Bbar^T =
// C^T diag(dbar). Because U U^dag = I, the PCG preconditioner
// P^{-1} P^{-T} = U^dag [diag f(A)] [diag f(A)]^dag U is applied with one
// forward transform, both polynomial passes per omega in one kernel, and one
// inverse transform.
//
// Kernels:
//   k_kpm_coeffs  N_P(omega) (Eq. (NP_heuristic), a1 = a2 = 1, floored at 1)
//                 and c_m by Chebyshev-Gauss quadrature with N_Q = 2 N_P
//                 points (Eq. (Cheby-Gauss)), one block per omega.
//   k_tau_fwd     twisted DFT along tau, tiles of TS sites x T slices in
//                 shared memory, Stockham mixed-radix passes (radix 4,2,3,5,7).
//   k_kpm         one block per (omega, rhs); the N-vector lives in shared
//                 memory, the checkerboard colours are applied pair-parallel.
//   k_tau_inv     inverse twisted transform, real output, optional r.z sums.
#include <math.h>
#include <stdlib.h>

#include <vector>

#include "cb.cuh"
#include "fft.cuh"
#include "internal.cuh"

namespace hol {
namespace {

using namespace fft;

// v (real [nr][T][N]) -> vh (complex [nr][T/2][N]) = U v restricted to omega < T/2
template <typename R>
__global__ void __launch_bounds__(256) k_tau_fwd(const R* __restrict__ v,
                                                 typename Cx<R>::T2* __restrict__ vh,
                                                 const typename Cx<R>::T2* __restrict__ w2, int T,
                                                 int N, int TS, RadixPlan plan, R scale)
{
    using C2 = typename Cx<R>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    C2* b = a + (long)T * TS;
    const int rhs = blockIdx.y;
    const int i0 = blockIdx.x * TS;
    const long base = (long)rhs * T * N;
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, tau = item / TS;
        const int i = i0 + c;
        const R x = (i < N) ? v[base + (long)tau * N + i] : R(0);
        const C2 t = tw<R>(w2, tau, T);    // exp(-i pi tau / T)
        a[tau * TS + c] = Cx<R>::mk(x * t.x, x * t.y);
    }
    C2* res = fft_tau<R>(a, b, w2, T, TS, plan);
    const int Th = T / 2;
    const long ob = (long)rhs * Th * N;
    for (int item = threadIdx.x; item < Th * TS; item += blockDim.x) {
        const int c = item % TS, w = item / TS;
        const int i = i0 + c;
        if (i < N) {
            C2 z = res[w * TS + c];
            z.x *= scale;
            z.y *= scale;
            vh[ob + (long)w * N + i] = z;
        }
    }
}

// yh (complex [nr][T/2][N]) -> y (real [nr][T][N]) = U^dag of the conjugate-
// symmetric extension; optional dot partials sum(y * rdot) per (rhs, tile).
template <typename R>
__global__ void __launch_bounds__(256) k_tau_inv(const typename Cx<R>::T2* __restrict__ yh,
                                                 R* __restrict__ y,
                                                 const typename Cx<R>::T2* __restrict__ w2, int T,
                                                 int N, int TS, RadixPlan plan, R scale,
                                                 const R* __restrict__ rdot,
                                                 double* __restrict__ dot_part)
{
    using C2 = typename Cx<R>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    C2* b = a + (long)T * TS;
    const int rhs = blockIdx.y;
    const int i0 = blockIdx.x * TS;
    const int Th = T / 2;
    const long ib = (long)rhs * Th * N;
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, w = item / TS;
        const int i = i0 + c;
        C2 z = Cx<R>::mk(R(0), R(0));
        if (w < Th && i < N) {
            z = yh[ib + (long)w * N + i];
            z.y = -z.y;   // conj
        }
        a[w * TS + c] = z;
    }
    C2* res = fft_tau<R>(a, b, w2, T, TS, plan);
    const long ob = (long)rhs * T * N;
    double acc = 0.0;
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, tau = item / TS;
        const int i = i0 + c;
        if (i < N) {
            const C2 t = tw<R>(w2, tau, T);
            const C2 z = res[tau * TS + c];
            const R val = scale * (t.x * z.x - t.y * z.y);   // 2/sqrt(T) Re(w2 * Y)
            y[ob + (long)tau * N + i] = val;
            if (rdot != nullptr) acc += (double)val * (double)rdot[ob + (long)tau * N + i];
        }
    }
    if (dot_part != nullptr) {
        __shared__ double red[8];
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
            dot_part[(long)rhs * kRedStride + blockIdx.x] = s;
        }
    }
}

// ---------------------------------------------------------------- KPM
struct KpmArgs {
    int L, N, Th, max_np;
    int mode;         // bit 0: apply conj-coefficient series of A^T first; bit 1: then series of A
    double ch, sh;
};

// In-place checkerboard colour (0: x-even, 1: x-odd, 2: y-even, 3: y-odd) on
// a complex vector in shared memory; pairs are processed in parallel.
template <typename C2, typename R>
__device__ __forceinline__ void kpm_colour(C2* v, int colour, int L, R ch, R sh)
{
    const int half = L / 2;
    const int npair = L * half;
    for (int k = threadIdx.x; k < npair; k += blockDim.x) {
        int i, j;
        if (colour < 2) {
            const int iy = k / half, h = k - iy * half;
            const int ix = 2 * h + colour;
            i = ix + L * iy;
            j = (ix + 1 == L ? 0 : ix + 1) + L * iy;
        } else {
            const int ix = k % L, hy = k / L;
            const int iy = 2 * hy + (colour - 2);
            i = ix + L * iy;
            j = ix + L * (iy + 1 == L ? 0 : iy + 1);
        }
        const C2 a = v[i], b = v[j];
        C2 na, nb;
        na.x = fma(ch, a.x, sh * b.x);
        na.y = fma(ch, a.y, sh * b.y);
        nb.x = fma(sh, a.x, ch * b.x);
        nb.y = fma(sh, a.y, ch * b.y);
        v[i] = na;
        v[j] = nb;
    }
    __syncthreads();
}

constexpr int kKpmMaxE = 8;   // elements per thread (N <= 8 * blockDim)

// One polynomial series sum_m c_m T_m(Aop) u with Aop = a Bop + c0,
// Bop = diag(d) C (trans = 0) or C^T diag(d) (trans = 1), coefficients
// conjugated when conjc. u is in `cur` (shared) on entry; the result is left
// in `cur` on exit. prev/acc/old are per-thread register arrays.
template <typename R>
__device__ void kpm_series(typename Cx<R>::T2* cur, const double* __restrict__ dbar,
                           const double2* __restrict__ coef, int np, bool trans, bool conjc,
                           double a, double c0, const KpmArgs& ka)
{
    using C2 = typename Cx<R>::T2;
    const int N = ka.N;
    const R ch = (R)ka.ch, sh = (R)ka.sh;
    C2 prev[kKpmMaxE], acc[kKpmMaxE], old[kKpmMaxE];
    R dd[kKpmMaxE];
    {
        double2 c = coef[0];
        if (conjc) c.y = -c.y;
#pragma unroll
        for (int e = 0; e < kKpmMaxE; ++e) {
            const int i = threadIdx.x + e * blockDim.x;
            if (i < N) {
                const C2 u = cur[i];
                acc[e] = Cx<R>::mk((R)c.x * u.x - (R)c.y * u.y, (R)c.x * u.y + (R)c.y * u.x);
                prev[e] = u;
                dd[e] = (R)dbar[i];
            }
        }
    }
    for (int m = 1; m < np; ++m) {
        // old <- alpha_{m-1} (current), then cur <- Bop * cur
#pragma unroll
        for (int e = 0; e < kKpmMaxE; ++e) {
            const int i = threadIdx.x + e * blockDim.x;
            if (i < N) {
                old[e] = cur[i];
                if (trans) {
                    C2 t = old[e];
                    t.x *= dd[e];
                    t.y *= dd[e];
                    cur[i] = t;
                }
            }
        }
        __syncthreads();
        if (trans) {
            kpm_colour<C2, R>(cur, 3, ka.L, ch, sh);
            kpm_colour<C2, R>(cur, 2, ka.L, ch, sh);
            kpm_colour<C2, R>(cur, 1, ka.L, ch, sh);
            kpm_colour<C2, R>(cur, 0, ka.L, ch, sh);
        } else {
            kpm_colour<C2, R>(cur, 0, ka.L, ch, sh);
            kpm_colour<C2, R>(cur, 1, ka.L, ch, sh);
            kpm_colour<C2, R>(cur, 2, ka.L, ch, sh);
            kpm_colour<C2, R>(cur, 3, ka.L, ch, sh);
        }
        double2 c = coef[m];
        if (conjc) c.y = -c.y;
#pragma unroll
        for (int e = 0; e < kKpmMaxE; ++e) {
            const int i = threadIdx.x + e * blockDim.x;
            if (i < N) {
                C2 bv = cur[i];
                if (!trans) {
                    bv.x *= dd[e];
                    bv.y *= dd[e];
                }
                // A alpha_{m-1} = a Bop alpha + c0 alpha
                C2 av;
                av.x = (R)a * bv.x + (R)c0 * old[e].x;
                av.y = (R)a * bv.y + (R)c0 * old[e].y;
                C2 nx;
                if (m == 1) {
                    nx = av;
                } else {
                    nx.x = R(2) * av.x - prev[e].x;
                    nx.y = R(2) * av.y - prev[e].y;
                }
                acc[e].x += (R)c.x * nx.x - (R)c.y * nx.y;
                acc[e].y += (R)c.x * nx.y + (R)c.y * nx.x;
                // alpha_{m-1} becomes the "two back" term of the next step
                prev[e] = old[e];
                cur[i] = nx;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < kKpmMaxE; ++e) {
        const int i = threadIdx.x + e * blockDim.x;
        if (i < N) cur[i] = acc[e];
    }
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(256) k_kpm(const typename Cx<R>::T2* __restrict__ vin,
                                             typename Cx<R>::T2* __restrict__ vout,
                                             const double* __restrict__ dbar,
                                             const double* __restrict__ scal,
                                             const int* __restrict__ npv,
                                             const double2* __restrict__ coef, int n_rhs,
                                             KpmArgs ka)
{
    using C2 = typename Cx<R>::T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* cur = reinterpret_cast<C2*>(smem_raw);
    // longest series first: omega varies slowest
    const int w = blockIdx.x / n_rhs, rhs = blockIdx.x - w * n_rhs;
    const int N = ka.N;
    const long off = ((long)rhs * ka.Th + w) * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) cur[i] = vin[off + i];
    __syncthreads();
    const double bmin = scal[S_BMIN], bmax = scal[S_BMAX];
    const double db = bmax - bmin;
    const double a = 2.0 / db, c0 = -2.0 * bmin / db - 1.0;
    const int np = npv[w];
    const double2* cw = coef + (long)w * ka.max_np;
    if (ka.mode & 1) kpm_series<R>(cur, dbar, cw, np, true, true, a, c0, ka);
    if (ka.mode & 2) kpm_series<R>(cur, dbar, cw, np, false, false, a, c0, ka);
    for (int i = threadIdx.x; i < N; i += blockDim.x) vout[off + i] = cur[i];
}

// N_P(omega) and c_m(omega), m < N_P, one block per omega < T/2.
__global__ void k_kpm_coeffs(const double* __restrict__ scal, int T, int max_np,
                             int* __restrict__ npv, double2* __restrict__ coef,
                             int* __restrict__ clamped)
{
    const int w = blockIdx.x;
    const double bmin = scal[S_BMIN], bmax = scal[S_BMAX];
    const double db = bmax - bmin;
    const double phi = 2.0 * M_PI / T * (w + 0.5);
    double npd = floor(db * (1.0 / phi + 1.0));
    int np = npd < 1.0 ? 1 : (npd > (double)max_np ? max_np : (int)npd);
    if (threadIdx.x == 0) {
        npv[w] = np;
        if (npd > (double)max_np) atomicExch(clamped, 1);
    }
    const int nq = 2 * np;
    double sp, cp;
    sincos(phi, &sp, &cp);
    for (int m = threadIdx.x; m < np; m += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double th = (q + 0.5) / nq;            // theta / pi
            const double y = cospi(th);
            const double bb = bmin + (y + 1.0) * db * 0.5;
            // f = 1 / (1 - e^{-i phi} bb) = 1 / ((1 - bb cos phi) + i bb sin phi)
            const double re = 1.0 - bb * cp, im = bb * sp;
            const double den = re * re + im * im;
            const double cm = cospi(m * th);
            sr += cm * re / den;
            si += cm * (-im) / den;
        }
        const double qm = (m == 0) ? 2.0 : 1.0;   // q_m / (pi/2)
        const double fac = 2.0 / (qm * nq);       // pi / (q_m N_Q)
        coef[(long)w * max_np + m] = make_double2(fac * sr, fac * si);
    }
}

int tile_sites(int prec) { return prec == HOL_F64 ? 16 : 32; }

size_t fft_smem(const hol_ctx* c, int prec)
{
    const size_t cs = prec == HOL_F64 ? sizeof(double2) : sizeof(float2);
    return 2 * (size_t)c->T * tile_sites(prec) * cs;
}

int kpm_threads(const hol_ctx* c)
{
    int t = c->N / 2;
    t = (t + 31) / 32 * 32;
    if (t < 32) t = 32;
    if (t > 256) t = 256;
    return t;
}

template <typename R>
int set_smem_attr(const void* fn, size_t bytes)
{
    if (bytes > 48 * 1024)
        HOL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return HOL_OK;
}

// fwd transform, KPM (mode), inverse transform (+ optional dot partials)
template <typename R>
int precond_run(hol_ctx* c, const R* v, R* out, int n_rhs, int mode, const R* rdot,
                double* dot_part, cudaStream_t s)
{
    using C2 = typename Cx<R>::T2;
    const int prec = sizeof(R) == 8 ? HOL_F64 : HOL_F32;
    const RadixPlan plan = plan_of(c->T);
    const int TS = tile_sites(prec);
    const size_t sm = fft_smem(c, prec);
    const dim3 gf(ceil_div(c->N, TS), n_rhs);
    const C2* w2 = reinterpret_cast<const C2*>(prec == HOL_F64 ? (const void*)c->tw64
                                                                : (const void*)c->tw32);
    C2* h0 = reinterpret_cast<C2*>(c->cbuf0);
    C2* h1 = reinterpret_cast<C2*>(c->cbuf1);
    int rc;
    if ((rc = set_smem_attr<R>((const void*)k_tau_fwd<R>, sm))) return rc;
    if ((rc = set_smem_attr<R>((const void*)k_tau_inv<R>, sm))) return rc;
    const R isq = (R)(1.0 / sqrt((double)c->T));
    k_tau_fwd<R><<<gf, 256, sm, s>>>(v, h0, w2, c->T, c->N, TS, plan, isq);
    HOL_CHECK_LAUNCH("k_tau_fwd");
    KpmArgs ka;
    ka.L = c->L;
    ka.N = c->N;
    ka.Th = c->T / 2;
    ka.max_np = c->kpm.max_np;
    ka.mode = mode;
    ka.ch = c->ch;
    ka.sh = c->sh;
    const int kt = kpm_threads(c);
    const size_t ks = (size_t)c->N * sizeof(C2);
    if ((rc = set_smem_attr<R>((const void*)k_kpm<R>, ks))) return rc;
    k_kpm<R><<<ka.Th * n_rhs, kt, ks, s>>>(h0, h1, c->dbar, c->scal, c->kpm.np, c->kpm.coef,
                                           n_rhs, ka);
    HOL_CHECK_LAUNCH("k_kpm");
    k_tau_inv<R><<<gf, 256, sm, s>>>(h1, out, w2, c->T, c->N, TS, plan, (R)2 * isq, rdot,
                                     dot_part);
    HOL_CHECK_LAUNCH("k_tau_inv");
    return HOL_OK;
}

}  // namespace

int precond_tiles(const hol_ctx* c, int prec) { return ceil_div(c->N, tile_sites(prec)); }

int precond_check_shape(const hol_ctx* c)
{
    const RadixPlan p = plan_of(c->T);
    if (p.n < 0) return set_error(HOL_EINVAL, "preconditioner: Ltau=%d has a prime factor > 7", c->T);
    if (fft_smem(c, HOL_F64) > 220 * 1024)
        return set_error(HOL_EINVAL, "preconditioner: Ltau=%d too long for one tile", c->T);
    if (c->N > kKpmMaxE * 256) return set_error(HOL_EINVAL, "preconditioner: N too large");
    return HOL_OK;
}

int precond_apply_impl(hol_ctx* c, int prec, const void* v, void* out, int n_rhs, int mode,
                       const void* rdot, double* dot_part, cudaStream_t s)
{
    if (prec == HOL_F64)
        return precond_run<double>(c, (const double*)v, (double*)out, n_rhs, mode,
                                   (const double*)rdot, dot_part, s);
    return precond_run<float>(c, (const float*)v, (float*)out, n_rhs, mode, (const float*)rdot,
                              dot_part, s);
}

// Twiddles w2[k] = exp(-i pi k / T) (long double on the host) and the
// Chebyshev plan buffers; called from hol_create.
int precond_alloc(hol_ctx* c)
{
    const int T = c->T;
    std::vector<double2> h64(2 * T);
    std::vector<float2> h32(2 * T);
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < 2 * T; ++k) {
        const long double a = -pi * (long double)k / (long double)T;
        h64[k] = make_double2((double)cosl(a), (double)sinl(a));
        h32[k] = make_float2((float)cosl(a), (float)sinl(a));
    }
    HOL_CUDA(cudaMalloc((void**)&c->tw64, 2 * T * sizeof(double2)));
    HOL_CUDA(cudaMalloc((void**)&c->tw32, 2 * T * sizeof(float2)));
    HOL_CUDA(cudaMemcpy(c->tw64, h64.data(), 2 * T * sizeof(double2), cudaMemcpyHostToDevice));
    HOL_CUDA(cudaMemcpy(c->tw32, h32.data(), 2 * T * sizeof(float2), cudaMemcpyHostToDevice));
    c->kpm.max_np = 4 * T + 16;
    HOL_CUDA(cudaMalloc((void**)&c->kpm.np, (T / 2) * sizeof(int) + sizeof(int)));
    HOL_CUDA(cudaMalloc((void**)&c->kpm.coef, (long)(T / 2) * c->kpm.max_np * sizeof(double2)));
    HOL_CUDA(cudaMemset(c->kpm.np, 0, (T / 2) * sizeof(int) + sizeof(int)));
    return HOL_OK;
}

int kpm_setup(hol_ctx* c, cudaStream_t s)
{
    k_kpm_coeffs<<<c->T / 2, 128, 0, s>>>(c->scal, c->T, c->kpm.max_np, c->kpm.np, c->kpm.coef,
                                          c->kpm.np + c->T / 2);
    HOL_CHECK_LAUNCH("k_kpm_coeffs");
    return HOL_OK;
}

}  // namespace hol

using namespace hol;

extern "C" int precond_apply(hol_ctx* c, int which, int prec, const void* v, void* out, int n_rhs,
                             void* stream)
{
    if (!c || !v || !out) return set_error(HOL_EINVAL, "precond_apply: null argument");
    if (!c->field_set) return set_error(HOL_EINVAL, "precond_apply: hol_set_field not called");
    if (n_rhs < 1 || n_rhs > c->p.max_rhs)
        return set_error(HOL_EINVAL, "precond_apply: n_rhs=%d outside [1, %d]", n_rhs,
                         c->p.max_rhs);
    if (prec != HOL_F64 && prec != HOL_F32)
        return set_error(HOL_EINVAL, "precond_apply: bad precision %d", prec);
    int mode;
    switch (which) {
    case HOL_PINV: mode = 2; break;
    case HOL_PINVT: mode = 1; break;
    case HOL_PINV_PINVT: mode = 3; break;
    default: return set_error(HOL_EINVAL, "precond_apply: bad selector %d", which);
    }
    int rc = precond_check_shape(c);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    timer_start(c, KT_PRECOND, s);
    rc = precond_apply_impl(c, prec, v, out, n_rhs, mode, nullptr, nullptr, s);
    timer_stop(c, KT_PRECOND, s);
    return rc;
}
