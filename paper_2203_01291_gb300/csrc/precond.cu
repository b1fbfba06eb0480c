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
//   k_kpm_coeffs  N_P(omega) (Eq. (NP_heuristic); a1 = a2 = 1 unless the
//                 launch options say otherwise; floored at 1) and c_m by
//                 Chebyshev-Gauss quadrature with N_Q = 2 N_P points
//                 (Eq. (Cheby-Gauss)), one block per omega.
//   k_tau_fwd     twisted DFT along tau, tiles of TS sites x T slices in
//                 shared memory, Stockham mixed-radix passes (radix 4,2,3,5,7).
//   k_tau_fwd_upd the same with the PCG vector update fused into its loads.
//   k_kpm_reg     FP32, L = 16, 32: one (omega, rhs) problem per block, two
//                 rows and two or four complex columns per lane.
//   k_kpm_lane    FP32, any L: lane = column, rows in registers, the real and
//                 imaginary parts in two lane groups (no barrier per step).
//   k_kpm_band    FP64: the lane layout with the rows in bands over several
//                 warps (one exchange per Bbar apply).
//   k_kpm         one block per (omega, rhs); the N-vector lives in shared
//                 memory, the checkerboard colours are applied pair-parallel
//                 (the exact propagator, and FP64 where no band layout is
//                 built).
//   k_tau_inv     inverse twisted transform, real output, optional r.z sums.
#include <math.h>
#include <stdlib.h>

#include <type_traits>
#include <vector>

#include "cb.cuh"
#include "fft.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace hol {
namespace {

using namespace fft;

// Two adjacent values (sites i, i + 1 with i even, so the pair is aligned to
// its own size) as one vector access.
__device__ __forceinline__ void ld_pair(const float* p, float& a, float& b)
{
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_pair(const double* p, double& a, double& b)
{
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void st_pair(float* p, float a, float b)
{
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(double* p, double a, double b)
{
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
__device__ __forceinline__ void ld_cpair(const float2* p, float2& a, float2& b)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_cpair(const double2* p, double2& a, double2& b)
{
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void st_cpair(float2* p, float2 a, float2 b)
{
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_cpair(double2* p, double2 a, double2 b)
{
    p[0] = a;
    p[1] = b;
}

// The tau transforms act on real site lines, two per complex transform: the
// tile holds TS sites as TS / 2 columns, site 2c in the real and site 2c + 1
// in the imaginary part of column c.
//
// Forward. With t_tau = exp(-i pi tau / T), X[w] = sum_tau t_tau x_tau
// exp(-2 pi i w tau / T) of a real x has X[T-1-w] = conj(X[w]), so from
// Z = X_a + i X_b: X_a = (Z[w] + conj Z[T-1-w]) / 2 and
// X_b = (Z[w] - conj Z[T-1-w]) / (2 i).
//
// v (real [nr][T][N]) -> vh (complex [nr][T/2][N]) = U v restricted to omega < T/2
// TC, TSC > 0: length and tile width (sites) fixed at compile time
// (fft_tau_ct); 0: taken from the arguments (fft_tau).
template <typename R, int TC = 0, int TSC = 0>
__global__ void __launch_bounds__(256) k_tau_fwd(const R* __restrict__ v,
                                                 typename Cx<R>::T2* __restrict__ vh,
                                                 const typename Cx<R>::T2* __restrict__ w2, int T_,
                                                 int N, int TS_, RadixPlan plan, R scale)
{
    pdl_wait();      // the input comes from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    using C2 = typename Cx<R>::T2;
    const int T = TC > 0 ? TC : T_;
    const int TS = TSC > 0 ? TSC : TS_;
    const int TH = TS / 2;                 // transform columns
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    C2* b = a + (long)T * TH;
    const int rhs = blockIdx.y;
    const int i0 = blockIdx.x * TS;
    const long base = (long)rhs * T * N;
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, tau = item / TH;
        const int i = i0 + 2 * c;          // N is even, so i < N implies i + 1 < N
        R xa = R(0), xb = R(0);
        if (i < N) ld_pair(v + base + (long)tau * N + i, xa, xb);
        const C2 t = tw<R>(w2, tau, T);    // exp(-i pi tau / T)
        a[tau * TH + c] = Cx<R>::mk(xa * t.x - xb * t.y, xa * t.y + xb * t.x);
    }
    C2* res;
    if constexpr (TC > 0)
        res = fft_tau_ct<R, TC, TSC / 2, 256>(a, b, w2);
    else
        res = fft_tau<R>(a, b, w2, T, TH, plan);
    const int Th = T / 2;
    const long ob = (long)rhs * Th * N;
    const R hs = R(0.5) * scale;
    for (int item = threadIdx.x; item < Th * TH; item += blockDim.x) {
        const int c = item % TH, w = item / TH;
        const int i = i0 + 2 * c;
        if (i < N) {
            const C2 z = res[w * TH + c];
            const C2 zm = res[(T - 1 - w) * TH + c];
            // X_a = (z + conj zm) / 2,  X_b = (z - conj zm) / (2 i)
            st_cpair(vh + ob + (long)w * N + i, Cx<R>::mk(hs * (z.x + zm.x), hs * (z.y - zm.y)),
                     Cx<R>::mk(hs * (z.y + zm.y), hs * (zm.x - z.x)));
        }
    }
}

// The forward transform with the CG update of the PCG iteration fused into
// its load phase (PcUpd): each element of r is read once, updated
// (r -= alpha q, and the x accumulator by the fold mode's terms), written
// back, summed into this tile's r.r partial and transformed. alpha is formed
// by one warp per block from the partials, as k_cg_update forms it. Masked
// right-hand sides are transformed without an update.
template <typename R>
struct PcUpdK {
    R* x;
    const R* p;
    const R* pp;
    const R* q;
    const int* mask;
    const double* pq_part;
    int pq_stride, pq_n;
    const double* dz_part;
    int dz_n;
    double* rr_out;
    double* alpha_buf;
    int fold;
};

template <typename R, int TC = 0, int TSC = 0>
__global__ void __launch_bounds__(256) k_tau_fwd_upd(R* __restrict__ v,
                                                     typename Cx<R>::T2* __restrict__ vh,
                                                     const typename Cx<R>::T2* __restrict__ w2,
                                                     int T_, int N, int TS_, RadixPlan plan,
                                                     R scale, PcUpdK<R> u)
{
    pdl_wait();      // p, q and the partials come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    using C2 = typename Cx<R>::T2;
    const int T = TC > 0 ? TC : T_;
    const int TS = TSC > 0 ? TSC : TS_;
    const int TH = TS / 2;                 // transform columns
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    C2* b = a + (long)T * TH;
    const int rhs = blockIdx.y;
    const int i0 = blockIdx.x * TS;
    const long base = (long)rhs * T * N;
    const bool act = u.mask == nullptr || u.mask[rhs] != 0;
    __shared__ double s_alpha, s_alpha_prev;
    if (threadIdx.x < 32) {
        double al = 0.0, alp = 0.0;
        if (act) {
            const double pq = warp_sum_array(u.pq_part + (long)rhs * u.pq_stride, u.pq_n);
            const double dz = warp_sum_array(u.dz_part + (long)rhs * kRedStride, u.dz_n);
            al = cg_ratio(dz, pq);
            if (u.fold == 2) alp = u.alpha_buf[rhs];
        }
        if (threadIdx.x == 0) {
            s_alpha = al;
            s_alpha_prev = alp;
        }
    }
    __syncthreads();
    const R al = (R)s_alpha, ap = (R)s_alpha_prev;
    if (act && u.fold == 0 && blockIdx.x == 0 && threadIdx.x == 0) u.alpha_buf[rhs] = s_alpha;
    double acc = 0.0;
    F2 acc2{0.0f, 0.0f};
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, tau = item / TH;
        const int i = i0 + 2 * c;          // N is even, so i < N implies i + 1 < N
        R xa = R(0), xb = R(0);
        if (i < N) {
            const long o = base + (long)tau * N + i;
            ld_pair(v + o, xa, xb);
            if (act) {
                R qa, qb;
                ld_pair(u.q + o, qa, qb);
                if (u.fold != 0) {
                    R ea, eb, pa, pb;
                    ld_pair(u.x + o, ea, eb);
                    ld_pair(u.p + o, pa, pb);
                    if (u.fold == 2) {
                        R qa2, qb2;
                        ld_pair(u.pp + o, qa2, qb2);
                        ea = fma(ap, qa2, ea);
                        eb = fma(ap, qb2, eb);
                    }
                    ea = fma(al, pa, ea);
                    eb = fma(al, pb, eb);
                    st_pair(u.x + o, ea, eb);
                }
                xa = fma(-al, qa, xa);
                xb = fma(-al, qb, xb);
                st_pair(v + o, xa, xb);
                const R part = fma(xa, xa, xb * xb);
                if constexpr (sizeof(R) == 4)
                    acc2 = f2_add(acc2, (float)part);
                else
                    acc += (double)part;
            }
        }
        const C2 t = tw<R>(w2, tau, T);    // exp(-i pi tau / T)
        a[tau * TH + c] = Cx<R>::mk(xa * t.x - xb * t.y, xa * t.y + xb * t.x);
    }
    {
        double sum;
        if constexpr (sizeof(R) == 4)
            sum = block_sum_f2(acc2);
        else
            sum = block_sum(acc);
        if (act && threadIdx.x == 0) u.rr_out[(long)rhs * kRedStride + blockIdx.x] = sum;
    }
    C2* res;
    if constexpr (TC > 0)
        res = fft_tau_ct<R, TC, TSC / 2, 256>(a, b, w2);
    else
        res = fft_tau<R>(a, b, w2, T, TH, plan);
    const int Th = T / 2;
    const long ob = (long)rhs * Th * N;
    const R hs = R(0.5) * scale;
    for (int item = threadIdx.x; item < Th * TH; item += blockDim.x) {
        const int c = item % TH, w = item / TH;
        const int i = i0 + 2 * c;
        if (i < N) {
            const C2 z = res[w * TH + c];
            const C2 zm = res[(T - 1 - w) * TH + c];
            st_cpair(vh + ob + (long)w * N + i, Cx<R>::mk(hs * (z.x + zm.x), hs * (z.y - zm.y)),
                     Cx<R>::mk(hs * (z.y + zm.y), hs * (zm.x - z.x)));
        }
    }
}

// Inverse. y_tau = (2 / sqrt T) Re sum_{w < T/2} Y_w exp(2 pi i (w + 1/2) tau / T)
// is the real inverse of the conjugate-symmetric extension Y_full (Y_w for
// w < T/2, conj Y_{T-1-w} above), so two sites share one transform:
// with Z = Y_full,a + i Y_full,b and F = FFT(conj Z),
// y_a + i y_b = (1 / sqrt T) conj(t_tau F_tau).
// yh (complex [nr][T/2][N]) -> y (real [nr][T][N]); optional dot partials
// sum(y * rdot) per (rhs, tile). `scale` is 2 / sqrt T.
template <typename R, int TC = 0, int TSC = 0>
__global__ void __launch_bounds__(256) k_tau_inv(const typename Cx<R>::T2* __restrict__ yh,
                                                 R* __restrict__ y,
                                                 const typename Cx<R>::T2* __restrict__ w2, int T_,
                                                 int N, int TS_, RadixPlan plan, R scale,
                                                 const R* __restrict__ rdot,
                                                 double* __restrict__ dot_part)
{
    pdl_wait();      // the input comes from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    using C2 = typename Cx<R>::T2;
    const int T = TC > 0 ? TC : T_;
    const int TS = TSC > 0 ? TSC : TS_;
    const int TH = TS / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    C2* b = a + (long)T * TH;
    const int rhs = blockIdx.y;
    const int i0 = blockIdx.x * TS;
    const int Th = T / 2;
    const long ib = (long)rhs * Th * N;
    // one load of (Y_a, Y_b)[w] fills rows w and T-1-w of conj Z
    for (int item = threadIdx.x; item < Th * TH; item += blockDim.x) {
        const int c = item % TH, w = item / TH;
        const int i = i0 + 2 * c;
        C2 lo = Cx<R>::mk(R(0), R(0)), hi = lo;
        if (i < N) {
            C2 ya, yb;
            ld_cpair(yh + ib + (long)w * N + i, ya, yb);
            lo = Cx<R>::mk(ya.x - yb.y, -(ya.y + yb.x));   // conj(Y_a + i Y_b)
            hi = Cx<R>::mk(ya.x + yb.y, ya.y - yb.x);      // conj(conj Y_a + i conj Y_b)
        }
        a[w * TH + c] = lo;
        a[(T - 1 - w) * TH + c] = hi;
    }
    C2* res;
    if constexpr (TC > 0)
        res = fft_tau_ct<R, TC, TSC / 2, 256>(a, b, w2);
    else
        res = fft_tau<R>(a, b, w2, T, TH, plan);
    const long ob = (long)rhs * T * N;
    const R hs = R(0.5) * scale;           // 1 / sqrt T
    double acc = 0.0;
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, tau = item / TH;
        const int i = i0 + 2 * c;
        if (i < N) {
            const C2 t = tw<R>(w2, tau, T);
            const C2 f = res[tau * TH + c];
            const R ya = hs * (t.x * f.x - t.y * f.y);     // Re(t F) / sqrt T
            const R yb = -hs * (t.x * f.y + t.y * f.x);    // -Im(t F) / sqrt T
            const long o = ob + (long)tau * N + i;
            st_pair(y + o, ya, yb);
            if (rdot != nullptr) {
                R ra, rb;
                ld_pair(rdot + o, ra, rb);
                // the pair's two products in R, accumulated in FP64 (one
                // conversion and one FP64 add per pair: the FP64 pipe is scarce)
                acc += (double)fma(ya, ra, yb * rb);
            }
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
    double th;        // tanh(dtau t); dbar carries cosh^4 (see cb.cuh)
    int ex;           // exact propagator exp(-dtau K) instead of the checkerboard
    int D;            // exact: taps kept on each side
    double e[kKinTaps];   // exact: ring factor taps
};

// v <- exp(-dtau K) v = (E (x) E) v on a complex slice in shared memory:
// x direction into tmp, then y direction back into v.
template <typename C2, typename R>
__device__ __forceinline__ void kpm_exact(C2* v, C2* tmp, const KpmArgs& ka)
{
    const int L = ka.L, N = ka.N;
    const R e0 = (R)ka.e[0];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int iy = i / L, ix = i - iy * L, row = iy * L;
        const C2 a = v[i];
        C2 o;
        o.x = e0 * a.x;
        o.y = e0 * a.y;
        for (int d = 1; d <= ka.D; ++d) {
            C2 u = v[row + (ix + d) % L];
            if (2 * d != L) {
                const C2 w = v[row + (ix + L - d) % L];
                u.x += w.x;
                u.y += w.y;
            }
            const R ed = (R)ka.e[d];
            o.x = fma(ed, u.x, o.x);
            o.y = fma(ed, u.y, o.y);
        }
        tmp[i] = o;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int iy = i / L, ix = i - iy * L;
        const C2 a = tmp[i];
        C2 o;
        o.x = e0 * a.x;
        o.y = e0 * a.y;
        for (int d = 1; d <= ka.D; ++d) {
            C2 u = tmp[((iy + d) % L) * L + ix];
            if (2 * d != L) {
                const C2 w = tmp[((iy + L - d) % L) * L + ix];
                u.x += w.x;
                u.y += w.y;
            }
            const R ed = (R)ka.e[d];
            o.x = fma(ed, u.x, o.x);
            o.y = fma(ed, u.y, o.y);
        }
        v[i] = o;
    }
    __syncthreads();
}

// In-place checkerboard colour (0: x-even, 1: x-odd, 2: y-even, 3: y-odd) on
// a complex vector in shared memory; pairs are processed in parallel.
template <typename C2, typename R>
__device__ __forceinline__ void kpm_colour(C2* v, int colour, int L, R th)
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
        na.x = fma(th, b.x, a.x);
        na.y = fma(th, b.y, a.y);
        nb.x = fma(th, a.x, b.x);
        nb.y = fma(th, a.y, b.y);
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
__device__ void kpm_series(typename Cx<R>::T2* cur, typename Cx<R>::T2* tmp,
                           const double* __restrict__ dbar,
                           const double2* __restrict__ coef, int np, bool trans, bool conjc,
                           double a, double c0, const KpmArgs& ka)
{
    using C2 = typename Cx<R>::T2;
    const int N = ka.N;
    const R th = (R)ka.th;
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
        if (ka.ex) {
            kpm_exact<C2, R>(cur, tmp, ka);   // symmetric: same for Bop and its transpose
        } else if (trans) {
            kpm_colour<C2, R>(cur, 3, ka.L, th);
            kpm_colour<C2, R>(cur, 2, ka.L, th);
            kpm_colour<C2, R>(cur, 1, ka.L, th);
            kpm_colour<C2, R>(cur, 0, ka.L, th);
        } else {
            kpm_colour<C2, R>(cur, 0, ka.L, th);
            kpm_colour<C2, R>(cur, 1, ka.L, th);
            kpm_colour<C2, R>(cur, 2, ka.L, th);
            kpm_colour<C2, R>(cur, 3, ka.L, th);
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
    pdl_wait();      // the input comes from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
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
    // exact propagator: a second slice of scratch; then this omega's
    // coefficients in shared memory (read once per Chebyshev step)
    C2* tmp = cur + N;
    double2* cw = reinterpret_cast<double2*>(cur + (ka.ex ? 2 * N : N));
    for (int m = threadIdx.x; m < np; m += blockDim.x) cw[m] = coef[(long)w * ka.max_np + m];
    __syncthreads();
    if (ka.mode & 1) kpm_series<R>(cur, tmp, dbar, cw, np, true, true, a, c0, ka);
    if (ka.mode & 2) kpm_series<R>(cur, tmp, dbar, cw, np, false, false, a, c0, ka);
    for (int i = threadIdx.x; i < N; i += blockDim.x) vout[off + i] = cur[i];
}

// ---------------------------------------------------------------- KPM, registers
// FP32 KPM for L = 16 and 32 with the slice in registers. Lane (j, cx) of
// warp w holds rows 2J, 2J+1 (J = w * PPW + j) and the CPL columns
// CPL cx .. CPL cx + CPL - 1 (CPL = 4 or 2) of the complex N-vector; x-bonds
// and in-warp y-bonds are register pairs or shuffles, the colour-4 bond
// between the last row of one warp and the first row of the next goes through
// shared memory (one barrier per Bbar apply, slots alternate). CPL = 2 spreads
// a problem over twice the warps with half the work per lane on its chain of
// dependent Bbar applies.
template <int CPL>
struct CV {
    float re[CPL], im[CPL];
};

__device__ __forceinline__ void bond2(float& a, float& b, float th)
{
    const float x = a, y = b;
    a = fmaf(th, y, x);
    b = fmaf(th, x, y);
}

template <int L, int CPL>
struct KGeo {
    static constexpr int LR = L / CPL;        // lanes per row segment
    static constexpr int PPW = 32 / LR;       // row pairs per warp
    static constexpr int W = L / (2 * PPW);   // warps per problem
    int lane, w, j, cx, right, left, down, up;
    __device__ __forceinline__ KGeo()
    {
        lane = threadIdx.x & 31;
        w = threadIdx.x >> 5;
        j = lane / LR;
        cx = lane - j * LR;
        right = j * LR + (cx + 1 == LR ? 0 : cx + 1);
        left = j * LR + (cx == 0 ? LR - 1 : cx - 1);
        down = (lane + LR) & 31;
        up = (lane + 32 - LR) & 31;
    }
    __device__ __forceinline__ int row0() const { return 2 * (w * PPW + j); }
};

// colour 1 (x, even ix): column pairs inside the lane
template <int CPL>
__device__ __forceinline__ void kc1(CV<CPL> (&v)[2], float th)
{
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int e = 0; e < CPL; e += 2) {
            bond2(v[r].re[e], v[r].re[e + 1], th);
            bond2(v[r].im[e], v[r].im[e + 1], th);
        }
}
// colour 2 (x, odd ix): inner pairs (1, 2), ..., the last column with the
// right lane's first, the first with the left lane's last
template <int L, int CPL>
__device__ __forceinline__ void kc2(CV<CPL> (&v)[2], const KGeo<L, CPL>& g, float th)
{
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float rxr = __shfl_sync(kFull, v[r].re[0], g.right);
        const float rxi = __shfl_sync(kFull, v[r].im[0], g.right);
        const float lwr = __shfl_sync(kFull, v[r].re[CPL - 1], g.left);
        const float lwi = __shfl_sync(kFull, v[r].im[CPL - 1], g.left);
#pragma unroll
        for (int e = 1; e + 1 < CPL; e += 2) {
            bond2(v[r].re[e], v[r].re[e + 1], th);
            bond2(v[r].im[e], v[r].im[e + 1], th);
        }
        v[r].re[CPL - 1] = fmaf(th, rxr, v[r].re[CPL - 1]);
        v[r].im[CPL - 1] = fmaf(th, rxi, v[r].im[CPL - 1]);
        v[r].re[0] = fmaf(th, lwr, v[r].re[0]);
        v[r].im[0] = fmaf(th, lwi, v[r].im[0]);
    }
}
// colour 3 (y, even iy): rows 2J, 2J+1 of the same lane
template <int CPL>
__device__ __forceinline__ void kc3(CV<CPL> (&v)[2], float th)
{
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
        bond2(v[0].re[e], v[1].re[e], th);
        bond2(v[0].im[e], v[1].im[e], th);
    }
}
// colour 4 (y, odd iy): row 2J+1 with row 2J+2 (next lane group / next warp)
template <int L, int CPL>
__device__ __forceinline__ void kc4(CV<CPL> (&v)[2], const KGeo<L, CPL>& g, float th,
                                    float* xbuf, int par)
{
    CV<CPL> dn, upv;
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
        dn.re[e] = __shfl_sync(kFull, v[0].re[e], g.down);
        dn.im[e] = __shfl_sync(kFull, v[0].im[e], g.down);
        upv.re[e] = __shfl_sync(kFull, v[1].re[e], g.up);
        upv.im[e] = __shfl_sync(kFull, v[1].im[e], g.up);
    }
    if constexpr (KGeo<L, CPL>::W > 1) {
        constexpr int LR = KGeo<L, CPL>::LR;
        constexpr int PPW = KGeo<L, CPL>::PPW;
        constexpr int W = KGeo<L, CPL>::W;
        // slot (par, warp, 0: first row of the warp / 1: last row, cx): CPL
        // real parts then CPL imaginary parts
        auto slot = [&](int wq, int which) {
            return xbuf + ((((par * W + wq) * 2 + which) * LR + g.cx) * 2 * CPL);
        };
        if (g.j == 0) {
            float* sl = slot(g.w, 0);
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
                sl[e] = v[0].re[e];
                sl[CPL + e] = v[0].im[e];
            }
        }
        if (g.j == PPW - 1) {
            float* sl = slot(g.w, 1);
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
                sl[e] = v[1].re[e];
                sl[CPL + e] = v[1].im[e];
            }
        }
        __syncthreads();
        if (g.j == PPW - 1) {
            const float* sl = slot((g.w + 1) % W, 0);
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
                dn.re[e] = sl[e];
                dn.im[e] = sl[CPL + e];
            }
        }
        if (g.j == 0) {
            const float* sl = slot((g.w + W - 1) % W, 1);
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
                upv.re[e] = sl[e];
                upv.im[e] = sl[CPL + e];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
        v[1].re[e] = fmaf(th, dn.re[e], v[1].re[e]);
        v[1].im[e] = fmaf(th, dn.im[e], v[1].im[e]);
        v[0].re[e] = fmaf(th, upv.re[e], v[0].re[e]);
        v[0].im[e] = fmaf(th, upv.im[e], v[0].im[e]);
    }
}

// One block per (omega, rhs) problem (queue null), or a persistent grid of a
// few blocks per multiprocessor taking problems from an atomic queue in the
// order omega = 0, 1, ... (the longest Chebyshev series first, since N_P
// falls with omega): the long series then run on multiprocessors shared with
// few other blocks while the short ones fill the rest. queue[0] is the next
// problem, queue[1] counts finished blocks; the last block resets both for
// the next launch (no block waits for another). Which block runs a problem
// does not change its arithmetic.
template <int L, int CPL>
__global__ void __launch_bounds__(32 * KGeo<L, CPL>::W)
    k_kpm_reg(const float2* __restrict__ vin, float2* __restrict__ vout,
              const double* __restrict__ dbar, const double* __restrict__ scal,
              const int* __restrict__ npv, const double2* __restrict__ coef, int n_rhs, int Th,
              int max_np, int mode, float th, int* __restrict__ queue)
{
    pdl_wait();      // the input comes from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    using G = KGeo<L, CPL>;
    __shared__ float xbuf[G::W > 1 ? 2 * G::W * 2 * G::LR * 2 * CPL : 1];
    __shared__ int s_item;
    const G g;
    const int n_items = n_rhs * Th;
    for (int item = blockIdx.x;;) {
        if (queue != nullptr) {
            __syncthreads();   // the previous problem's shared data is no longer read
            if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
            __syncthreads();
            item = s_item;
            if (item >= n_items) break;
        }
        const int wq = item / n_rhs, rhs = item - wq * n_rhs;
        const long off = ((long)rhs * Th + wq) * L * L;
        const int r0 = g.row0();
        CV<CPL> cur[2];
        float d[2][CPL];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const long e = off + (long)(r0 + r) * L + CPL * g.cx;
#pragma unroll
            for (int q = 0; q < CPL; q += 2) {
                const float4 a = *reinterpret_cast<const float4*>(vin + e + q);
                cur[r].re[q] = a.x;
                cur[r].im[q] = a.y;
                cur[r].re[q + 1] = a.z;
                cur[r].im[q + 1] = a.w;
            }
            const int i = (r0 + r) * L + CPL * g.cx;
#pragma unroll
            for (int q = 0; q < CPL; ++q) d[r][q] = (float)dbar[i + q];
        }
        const double bmin = scal[S_BMIN], bmax = scal[S_BMAX];
        const double db = bmax - bmin;
        const float a = (float)(2.0 / db), c0 = (float)(-2.0 * bmin / db - 1.0);
        const int np = npv[wq];
        // this omega's coefficients, rounded to FP32 once (no conversion on the
        // chain of dependent steps)
        extern __shared__ float2 cw[];
        for (int m = threadIdx.x; m < np; m += blockDim.x) {
            const double2 c = coef[(long)wq * max_np + m];
            cw[m] = make_float2((float)c.x, (float)c.y);
        }
        __syncthreads();
        int par = 0;
        // one series; the direction is a compile-time constant, so the chain
        // of dependent steps carries no branch on it
        auto series = [&](auto trans_c) {
            constexpr bool trans = decltype(trans_c)::value;
            const float sgn = trans ? -1.0f : 1.0f;    // conj coefficients for the transpose
            CV<CPL> acc[2], prev[2];
            {
                const float2 c = cw[0];
                const float cr = c.x, ci = sgn * c.y;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    prev[r] = cur[r];
#pragma unroll
                    for (int e = 0; e < CPL; ++e) {
                        acc[r].re[e] = cr * cur[r].re[e] - ci * cur[r].im[e];
                        acc[r].im[e] = cr * cur[r].im[e] + ci * cur[r].re[e];
                    }
                }
            }
            for (int m = 1; m < np; ++m) {
                CV<CPL> old[2], b[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    old[r] = cur[r];
                    b[r] = cur[r];
                    if constexpr (trans) {
#pragma unroll
                        for (int e = 0; e < CPL; ++e) {
                            b[r].re[e] *= d[r][e];
                            b[r].im[e] *= d[r][e];
                        }
                    }
                }
                if constexpr (trans) {
                    kc4<L, CPL>(b, g, th, xbuf, par);
                    kc3<CPL>(b, th);
                    kc2<L, CPL>(b, g, th);
                    kc1<CPL>(b, th);
                } else {
                    kc1<CPL>(b, th);
                    kc2<L, CPL>(b, g, th);
                    kc3<CPL>(b, th);
                    kc4<L, CPL>(b, g, th, xbuf, par);
                }
                par ^= 1;
                const float2 c = cw[m];
                const float cr = c.x, ci = sgn * c.y;
                // alpha_m = (m == 1 ? 1 : 2) (a B + c0) alpha_{m-1} - (m == 1 ? 0 : alpha_{m-2})
                const float f2 = (m == 1) ? 1.0f : 2.0f;
                const float pm = (m == 1) ? 0.0f : 1.0f;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
#pragma unroll
                    for (int e = 0; e < CPL; ++e) {
                        float br = b[r].re[e], bi = b[r].im[e];
                        if constexpr (!trans) {
                            br *= d[r][e];
                            bi *= d[r][e];
                        }
                        const float xr = f2 * fmaf(a, br, c0 * old[r].re[e]) - pm * prev[r].re[e];
                        const float xi = f2 * fmaf(a, bi, c0 * old[r].im[e]) - pm * prev[r].im[e];
                        cur[r].re[e] = xr;
                        cur[r].im[e] = xi;
                        acc[r].re[e] = fmaf(cr, xr, fmaf(-ci, xi, acc[r].re[e]));
                        acc[r].im[e] = fmaf(cr, xi, fmaf(ci, xr, acc[r].im[e]));
                    }
                    prev[r] = old[r];
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) cur[r] = acc[r];
        };
        if (mode & 1) series(std::true_type{});
        if (mode & 2) series(std::false_type{});
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const long e = off + (long)(r0 + r) * L + CPL * g.cx;
#pragma unroll
            for (int q = 0; q < CPL; q += 2)
                *reinterpret_cast<float4*>(vout + e + q) =
                    make_float4(cur[r].re[q], cur[r].im[q], cur[r].re[q + 1], cur[r].im[q + 1]);
        }
        if (queue == nullptr) break;
    }
    if (queue != nullptr && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
            queue[0] = 0;
            queue[1] = 0;
        }
    }
}

// ---------------------------------------------------------- KPM, lane layout
// FP32 KPM for any even L <= 32 in the scalar register layout of cb.cuh: a
// lane group of L lanes holds one real N-vector (lane = column, registers =
// rows; x-bonds by shuffles, y-bonds on register pairs). Bbar is real, so
// T_m(A) acts on the real and imaginary parts of a problem's complex vector
// independently: lane group 2s + p holds part p (0: real, 1: imaginary) of
// problem s of the block, and the two recurrences meet only in the complex
// coefficient sum. Each group accumulates A_p = sum c_m.re x_p and
// B_p = sum c_m.im x_p; at the end of a series acc.re = A_0 - s B_1 and
// acc.im = A_1 + s B_0 (s = -1 for the conjugate coefficients of the
// transpose), one exchange per series instead of one per step. With
// G = 32 / L >= 2 groups per warp a block is one warp holding G / 2 problems
// (an odd last group shadows and never stores); with G = 1 a block is two
// warps, one per part, exchanging through shared memory. The problems of a
// block share omega (consecutive right-hand sides), so every group runs the
// same N_P(omega) steps and the warp-wide shuffles stay converged.
template <int L>
struct KLane {
    static constexpr int G = 32 / L;                  // lane groups per warp
    static constexpr int PPB = G >= 2 ? G / 2 : 1;    // problems per block
    static constexpr int THREADS = G >= 2 ? 32 : 64;
};

template <typename R, int L>
__global__ void __launch_bounds__(KLane<L>::THREADS)
    k_kpm_lane(const typename Cx<R>::T2* __restrict__ vin, typename Cx<R>::T2* __restrict__ vout,
               const double* __restrict__ dbar, const double* __restrict__ scal,
               const int* __restrict__ npv, const double2* __restrict__ coef, int n_rhs, int Th,
               int max_np, int mode, R th)
{
    using C2 = typename Cx<R>::T2;
    pdl_wait();      // the input comes from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    using K = KLane<L>;
    constexpr int N = L * L;
    const LaneGeom<L> geo;
    // this lane's group within the block: part and problem slot
    const int grp = (K::G >= 2) ? geo.g : (int)(threadIdx.x >> 5);
    const int part = grp & 1, slot = grp >> 1;
    const bool live = geo.ok && slot < K::PPB;
    const int rpb = (n_rhs + K::PPB - 1) / K::PPB;   // blocks per omega
    const int wq = blockIdx.x / rpb;
    const int rhs_raw = (blockIdx.x - wq * rpb) * K::PPB + (slot < K::PPB ? slot : 0);
    const bool own = live && rhs_raw < n_rhs;        // stores its results
    const int rhs = rhs_raw < n_rhs ? rhs_raw : n_rhs - 1;
    const long off = ((long)rhs * Th + wq) * N + geo.ix;
    const R* vin_f = reinterpret_cast<const R*>(vin);
    R t[L], d[L];
#pragma unroll
    for (int iy = 0; iy < L; ++iy) {
        t[iy] = vin_f[2 * (off + iy * L) + part];
        d[iy] = (R)dbar[geo.ix + iy * L];
    }
    const double bmin = scal[S_BMIN], bmax = scal[S_BMAX];
    const double db = bmax - bmin;
    const R a = (R)(2.0 / db), c0 = (R)(-2.0 * bmin / db - 1.0);
    const int np = npv[wq];
    // this omega's coefficients (rounded to R once), then (G = 1) the exchange
    extern __shared__ __align__(16) unsigned char kl_smem[];
    C2* cw = reinterpret_cast<C2*>(kl_smem);
    for (int m = threadIdx.x; m < np; m += blockDim.x) {
        const double2 cm = coef[(long)wq * max_np + m];
        C2 cr;
        cr.x = (R)cm.x;
        cr.y = (R)cm.y;
        cw[m] = cr;
    }
    R* xbuf = reinterpret_cast<R*>(cw + max_np);   // [2][32][L]
    __syncthreads();
    // one series; the direction is a compile-time constant
    auto series = [&](auto trans_c) {
        constexpr bool trans = decltype(trans_c)::value;
        const R sgn = trans ? R(-1) : R(1);   // conj coefficients for the transpose
        R A[L], B[L], prev[L];
        {
            const C2 cm = cw[0];
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                A[iy] = cm.x * t[iy];
                B[iy] = cm.y * t[iy];
                prev[iy] = t[iy];
            }
        }
        for (int m = 1; m < np; ++m) {
            R b[L];
#pragma unroll
            for (int iy = 0; iy < L; ++iy) b[iy] = trans ? t[iy] * d[iy] : t[iy];
            if constexpr (trans)
                cb_apply_t<R, L>(b, geo, th);
            else
                cb_apply<R, L>(b, geo, th);
            const C2 cm = cw[m];
            // alpha_m = (m == 1 ? 1 : 2) (a Bbar + c0) alpha_{m-1} - (m == 1 ? 0 : alpha_{m-2})
            const R f2 = (m == 1) ? R(1) : R(2);
            const R pm = (m == 1) ? R(0) : R(1);
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                const R bv = trans ? b[iy] : b[iy] * d[iy];
                const R x = f2 * fma(a, bv, c0 * t[iy]) - pm * prev[iy];
                prev[iy] = t[iy];
                t[iy] = x;
                A[iy] = fma(cm.x, x, A[iy]);
                B[iy] = fma(cm.y, x, B[iy]);
            }
        }
        // acc.re = A_0 - sgn B_1, acc.im = A_1 + sgn B_0: swap B with the other part
        R Bo[L];
        if constexpr (K::G >= 2) {
            const int lane = threadIdx.x & 31;
            const int src = part == 0 ? lane + L : lane - L;   // the other part's lane
            const int srcc = (src >= 0 && src < 32) ? src : lane;
#pragma unroll
            for (int iy = 0; iy < L; ++iy) Bo[iy] = __shfl_sync(kFull, B[iy], srcc);
        } else {
            const int lane = threadIdx.x & 31;
            // (the previous series' reads of xbuf ended at its third barrier)
#pragma unroll
            for (int iy = 0; iy < L; ++iy) xbuf[(part * 32 + lane) * L + iy] = B[iy];
            __syncthreads();
#pragma unroll
            for (int iy = 0; iy < L; ++iy) Bo[iy] = xbuf[((1 - part) * 32 + lane) * L + iy];
            __syncthreads();
        }
#pragma unroll
        for (int iy = 0; iy < L; ++iy) t[iy] = part == 0 ? A[iy] - sgn * Bo[iy] : A[iy] + sgn * Bo[iy];
    };
    if (mode & 1) series(std::true_type{});
    if (mode & 2) series(std::false_type{});
    if (own) {
        R* vout_f = reinterpret_cast<R*>(vout);
#pragma unroll
        for (int iy = 0; iy < L; ++iy) vout_f[2 * (off + iy * L) + part] = t[iy];
    }
}

// ------------------------------------------------ KPM, banded lane layout
// FP64 KPM in the scalar lane layout with each problem spread over several
// warps: lane = column; the rows are cut into NB bands of RB = L / NB rows
// (RB even, so the even y-bonds stay inside a band); lane group (p, b) holds
// band b of part p (0: real, 1: imaginary). FP64 work is bound by the SM's
// FP64 pipe, which one warp can only use a quarter of (its SMSP's share), so
// a problem's chain of dependent Bbar applies needs its work on several
// warps: 2 NB lane groups over at least four warps. The odd y-bonds across
// band edges are exchanged through shared memory, one barrier per colour-4
// application (two alternating slot sets); the x-bonds are shuffles within
// the lane group; the two parts meet once per series as in k_kpm_lane.
template <int L>
struct KBand {
    // bands per part: RB = L / NB even, 2 NB lane groups over as many warps
    // as that gives. Measured (P^{-1} P^{-T}, 2 rhs, against the
    // shared-memory kernel): L = 8 82 / 215 us, 12 111 / 223, 16 176 / 308
    // (Ltau = 160; 191 with NB = 4), 24 364 / 454, 28 432 / 544, 32 808 /
    // 994 (Ltau = 200; 862 with NB = 8); L = 20 gained nothing (306 / 309)
    // and keeps the shared-memory kernel, as do the sizes not listed
    static constexpr int NB = L == 4 ? 2 : L == 6 ? 3 : L == 8 ? 4 : L == 10 ? 5 : L == 12 ? 6
                            : L == 14 ? 7 : L == 16 ? 8 : L == 18 ? 3 : L == 24 ? 6 : L == 28 ? 7
                            : L == 32 ? 4 : 0;
    static constexpr int RB = NB > 0 ? L / NB : 0;
    static constexpr int G = 32 / L;                           // lane groups per warp
    static constexpr int GROUPS = 2 * NB;
    static constexpr int WARPS = (GROUPS + G - 1) / G;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr bool OK = NB > 0 && RB % 2 == 0;
};

template <int L>
__global__ void __launch_bounds__(KBand<L>::THREADS > 0 ? KBand<L>::THREADS : 32)
    k_kpm_band(const double2* __restrict__ vin, double2* __restrict__ vout,
               const double* __restrict__ dbar, const double* __restrict__ scal,
               const int* __restrict__ npv, const double2* __restrict__ coef, int n_rhs, int Th,
               int max_np, int mode, double th)
{
    pdl_wait();      // the input comes from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    using K = KBand<L>;
    constexpr int N = L * L, RB = K::RB, NB = K::NB;
    const LaneGeom<L> geo;
    const int gi = (int)(threadIdx.x >> 5) * K::G + geo.g;     // lane group of the block
    const bool live = geo.ok && gi < K::GROUPS;
    const int gs = live ? gi : 0;                              // idle groups shadow group 0
    const int part = gs / NB, band = gs - part * NB;
    const int wq = blockIdx.x / n_rhs, rhs = blockIdx.x - wq * n_rhs;
    const long off = ((long)rhs * Th + wq) * N + geo.ix;
    const int row0 = band * RB;
    const double* vin_f = reinterpret_cast<const double*>(vin);
    double t[RB], d[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) {
        t[k] = vin_f[2 * (off + (row0 + k) * L) + part];
        d[k] = dbar[geo.ix + (row0 + k) * L];
    }
    const double bmin = scal[S_BMIN], bmax = scal[S_BMAX];
    const double db = bmax - bmin;
    const double a = 2.0 / db, c0 = -2.0 * bmin / db - 1.0;
    const int np = npv[wq];
    extern __shared__ __align__(16) unsigned char kb_smem[];
    double2* cw = reinterpret_cast<double2*>(kb_smem);
    for (int m = threadIdx.x; m < np; m += blockDim.x) cw[m] = coef[(long)wq * max_np + m];
    // band-edge slots [par][part][band][first / last row][column], then the B exchange
    double* eb = reinterpret_cast<double*>(cw + max_np);
    double* xb = eb + 2 * 2 * NB * 2 * L;                      // [part][band][RB][column]
    __syncthreads();
    auto edge = [&](int par, int p, int b, int which) -> double* {
        return eb + ((((par * 2 + p) * NB + b) * 2 + which) * L);
    };
    int par = 0;
    // colour 4 (odd y-bonds): pairs (1, 2), ..., inside the band; the band's
    // last row with the next band's first, its first with the previous
    // band's last (through shared memory)
    auto colour4 = [&](double (&c)[RB]) {
        if (live) {
            edge(par, part, band, 0)[geo.ix] = c[0];
            edge(par, part, band, 1)[geo.ix] = c[RB - 1];
        }
        __syncthreads();
        const int bn = band + 1 == NB ? 0 : band + 1, bp = band == 0 ? NB - 1 : band - 1;
        const double dn = edge(par, part, bn, 0)[geo.ix];
        const double upv = edge(par, part, bp, 1)[geo.ix];
        par ^= 1;   // the next exchange writes the other slot set
#pragma unroll
        for (int k = 1; k + 1 < RB; k += 2) {
            const double x = c[k], y = c[k + 1];
            c[k] = fma(th, y, x);
            c[k + 1] = fma(th, x, y);
        }
        c[RB - 1] = fma(th, dn, c[RB - 1]);
        c[0] = fma(th, upv, c[0]);
    };
    auto colour3 = [&](double (&c)[RB]) {
#pragma unroll
        for (int k = 0; k < RB; k += 2) {
            const double x = c[k], y = c[k + 1];
            c[k] = fma(th, y, x);
            c[k + 1] = fma(th, x, y);
        }
    };
    auto xbond = [&](double (&c)[RB], int partner) {
#pragma unroll
        for (int k = 0; k < RB; ++k) c[k] = fma(th, __shfl_sync(kFull, c[k], partner), c[k]);
    };
    // one series; the direction is a compile-time constant
    auto series = [&](auto trans_c) {
        constexpr bool trans = decltype(trans_c)::value;
        const double sgn = trans ? -1.0 : 1.0;   // conj coefficients for the transpose
        double A[RB], B[RB], prev[RB];
        {
            const double2 cm = cw[0];
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                A[k] = cm.x * t[k];
                B[k] = cm.y * t[k];
                prev[k] = t[k];
            }
        }
        for (int m = 1; m < np; ++m) {
            double b[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k) b[k] = trans ? t[k] * d[k] : t[k];
            if constexpr (trans) {   // C^T: colour 4 first
                colour4(b);
                colour3(b);
                xbond(b, geo.p2);
                xbond(b, geo.p1);
            } else {
                xbond(b, geo.p1);
                xbond(b, geo.p2);
                colour3(b);
                colour4(b);
            }
            const double2 cm = cw[m];
            const double f2 = (m == 1) ? 1.0 : 2.0;
            const double pm = (m == 1) ? 0.0 : 1.0;
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                const double bv = trans ? b[k] : b[k] * d[k];
                const double x = f2 * fma(a, bv, c0 * t[k]) - pm * prev[k];
                prev[k] = t[k];
                t[k] = x;
                A[k] = fma(cm.x, x, A[k]);
                B[k] = fma(cm.y, x, B[k]);
            }
        }
        // acc.re = A_0 - sgn B_1, acc.im = A_1 + sgn B_0
        if (live)
#pragma unroll
            for (int k = 0; k < RB; ++k) xb[((part * NB + band) * RB + k) * L + geo.ix] = B[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const double bo = xb[(((1 - part) * NB + band) * RB + k) * L + geo.ix];
            t[k] = part == 0 ? A[k] - sgn * bo : A[k] + sgn * bo;
        }
        __syncthreads();   // xb is rewritten by the next series
    };
    if (mode & 1) series(std::true_type{});
    if (mode & 2) series(std::false_type{});
    if (live) {
        double* vout_f = reinterpret_cast<double*>(vout);
#pragma unroll
        for (int k = 0; k < RB; ++k) vout_f[2 * (off + (row0 + k) * L) + part] = t[k];
    }
}

// N_P(omega) and c_m(omega), m < N_P, one block per omega < T/2.
// f(cos theta_n) is evaluated once per quadrature node into shared memory;
// cos(m theta_n) follows from a rotation by m pi / N_Q per node, so the
// coefficient sums cost FMAs only (FP64 throughput is scarce on this part).
__global__ void k_kpm_coeffs(const double* __restrict__ scal, int T, int max_np,
                             int* __restrict__ npv, double2* __restrict__ coef,
                             int* __restrict__ clamped, double a1, double a2)
{
    extern __shared__ double2 fq[];              // [2 max_np]
    const int w = blockIdx.x;
    const double bmin = scal[S_BMIN], bmax = scal[S_BMAX];
    const double db = bmax - bmin;
    const double phi = 2.0 * M_PI / T * (w + 0.5);
    const double npd = floor(db * (a1 / phi + a2));   // Eq. (NP_heuristic)
    const int np = npd < 1.0 ? 1 : (npd > (double)max_np ? max_np : (int)npd);
    if (threadIdx.x == 0) {
        npv[w] = np;
        if (npd > (double)max_np) atomicExch(clamped, 1);
    }
    const int nq = 2 * np;
    double sp, cp;
    sincos(phi, &sp, &cp);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const double y = cospi((q + 0.5) / nq);
        const double bb = bmin + (y + 1.0) * db * 0.5;
        // f = 1 / (1 - e^{-i phi} bb) = 1 / ((1 - bb cos phi) + i bb sin phi)
        const double re = 1.0 - bb * cp, im = bb * sp;
        const double den = re * re + im * im;
        fq[q] = make_double2(re / den, -im / den);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < np; m += blockDim.x) {
        double c, sn, cd, sd;
        sincospi(0.5 * m / nq, &sn, &c);      // angle m theta_0
        sincospi((double)m / nq, &sd, &cd);   // step m pi / N_Q
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double2 f = fq[q];
            sr = fma(c, f.x, sr);
            si = fma(c, f.y, si);
            const double c2 = c * cd - sn * sd;
            sn = fma(sn, cd, c * sd);
            c = c2;
        }
        const double qm = (m == 0) ? 2.0 : 1.0;   // q_m / (pi/2)
        const double fac = 2.0 / (qm * nq);       // pi / (q_m N_Q)
        coef[(long)w * max_np + m] = make_double2(fac * sr, fac * si);
    }
}

// Sites per tau-transform tile: 32 (FP32) / 16 (FP64) on the largest lattice;
// 8 below it, so that a small lattice with few right-hand sides still spreads
// over many blocks (N = 256 and 2 rhs: 64 blocks instead of 16).
constexpr int kSmallTile = 8;
int tile_sites(const hol_ctx* c, int prec)
{
    if (c->N < 1024) return kSmallTile;
    return prec == HOL_F64 ? 16 : 32;
}

size_t fft_smem(const hol_ctx* c, int prec)
{
    const size_t cs = prec == HOL_F64 ? sizeof(double2) : sizeof(float2);
    return 2 * (size_t)c->T * (tile_sites(c, prec) / 2) * cs;   // two sites per column
}

template <typename R, int L>
int run_kpm_lane_l(const hol_ctx* c, const typename Cx<R>::T2* in, typename Cx<R>::T2* out,
                   int n_rhs, int Th, int max_np, int mode, cudaStream_t s)
{
    using K = KLane<L>;
    const size_t sm = (size_t)max_np * sizeof(typename Cx<R>::T2) +
                      (K::G >= 2 ? 0 : (size_t)2 * 32 * L * sizeof(R));
    static std::atomic<int> limit(0);   // raised once per instantiation (not a stream call)
    if ((int)sm > limit.load()) {
        HOL_CUDA(cudaFuncSetAttribute((const void*)k_kpm_lane<R, L>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        limit.store((int)sm);
    }
    const int grid = Th * ((n_rhs + K::PPB - 1) / K::PPB);
    HOL_CUDA(launch_pdl(c, k_kpm_lane<R, L>, grid, K::THREADS, sm, s, in, out, c->dbar, c->scal,
                        c->kpm.np, c->kpm.coef, n_rhs, Th, max_np, mode, (R)c->th));
    HOL_CHECK_LAUNCH("k_kpm_lane");
    return HOL_OK;
}

template <int L>
int run_kpm_band_l(const hol_ctx* c, const double2* in, double2* out, int n_rhs, int Th,
                   int max_np, int mode, cudaStream_t s)
{
    using K = KBand<L>;
    if constexpr (!K::OK) {
        return set_error(HOL_EINVAL, "kpm banded layout: unsupported L=%d", L);
    } else {
        const size_t sm = (size_t)max_np * sizeof(double2) +
                          (size_t)(2 * 2 * K::NB * 2 * L + 2 * L * L) * sizeof(double);
        static std::atomic<int> limit(0);   // raised once per instantiation (not a stream call)
        if ((int)sm > limit.load()) {
            HOL_CUDA(cudaFuncSetAttribute((const void*)k_kpm_band<L>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            limit.store((int)sm);
        }
        HOL_CUDA(launch_pdl(c, k_kpm_band<L>, Th * n_rhs, K::THREADS, sm, s, in, out, c->dbar,
                            c->scal, c->kpm.np, c->kpm.coef, n_rhs, Th, max_np, mode, c->th));
        HOL_CHECK_LAUNCH("k_kpm_band");
        return HOL_OK;
    }
}

// FP64 KPM in the banded lane layout, for the L that KBand covers
bool kpm_band_ok(int L)
{
    switch (L) {
#define X(LL) case LL: return KBand<LL>::OK;
        X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(24) X(28) X(32)
#undef X
    }
    return false;
}

int run_kpm_band(const hol_ctx* c, const double2* in, double2* out, int n_rhs, int Th, int max_np,
                 int mode, cudaStream_t s)
{
    switch (c->L) {
#define X(LL) case LL: return run_kpm_band_l<LL>(c, in, out, n_rhs, Th, max_np, mode, s);
        X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(24) X(28) X(32)
#undef X
    }
    return set_error(HOL_EINVAL, "kpm banded layout: unsupported L=%d", c->L);
}

// KPM in the lane layout: FP32, any even L
template <typename R>
int run_kpm_lane(const hol_ctx* c, const typename Cx<R>::T2* in, typename Cx<R>::T2* out,
                 int n_rhs, int Th, int max_np, int mode, cudaStream_t s)
{
    if constexpr (sizeof(R) == 4) {
        switch (c->L) {
#define X(LL) case LL: return run_kpm_lane_l<R, LL>(c, in, out, n_rhs, Th, max_np, mode, s);
            X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30)
            X(32)
#undef X
        }
    }
    return set_error(HOL_EINVAL, "kpm lane layout: FP32 only (L=%d)", c->L);
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
    return smem_raise(fn, bytes);
}

// fwd transform, KPM (mode), inverse transform (+ optional dot partials);
// with `up`, the CG update of v (in place) is fused into the fwd transform
template <typename R>
int precond_run(hol_ctx* c, const R* v, R* out, int n_rhs, int mode, const R* rdot,
                double* dot_part, cudaStream_t s, const PcUpd* up = nullptr)
{
    using C2 = typename Cx<R>::T2;
    const int prec = sizeof(R) == 8 ? HOL_F64 : HOL_F32;
    const RadixPlan plan = plan_of(c->T);
    const int TS = tile_sites(c, prec);
    const size_t sm = fft_smem(c, prec);
    const dim3 gf(ceil_div(c->N, TS), n_rhs);
    const C2* w2 = reinterpret_cast<const C2*>(prec == HOL_F64 ? (const void*)c->tw64
                                                                : (const void*)c->tw32);
    C2* h0 = reinterpret_cast<C2*>(c->cbuf0);
    C2* h1 = reinterpret_cast<C2*>(c->cbuf1);
    int rc;
    // the configured lengths get transforms specialised at compile time
    constexpr int TSW = sizeof(R) == 8 ? 16 : 32;   // tile_sites on the largest lattice
    using FwdK = void (*)(const R*, C2*, const C2*, int, int, int, RadixPlan, R);
    using FwdU = void (*)(R*, C2*, const C2*, int, int, int, RadixPlan, R, PcUpdK<R>);
    using InvK = void (*)(const C2*, R*, const C2*, int, int, int, RadixPlan, R, const R*, double*);
    FwdK fwd = k_tau_fwd<R>;
    FwdU fwdu = k_tau_fwd_upd<R>;
    InvK inv = k_tau_inv<R>;
#define HOL_TAU_CT(TT)                                    \
    case TT:                                              \
        if (TS == TSW) {                                  \
            fwd = k_tau_fwd<R, TT, TSW>;                  \
            fwdu = k_tau_fwd_upd<R, TT, TSW>;             \
            inv = k_tau_inv<R, TT, TSW>;                  \
        } else if (TS == kSmallTile) {                    \
            fwd = k_tau_fwd<R, TT, kSmallTile>;           \
            fwdu = k_tau_fwd_upd<R, TT, kSmallTile>;      \
            inv = k_tau_inv<R, TT, kSmallTile>;           \
        }                                                 \
        break;
    switch (c->T) {
        HOL_TAU_CT(40)
        HOL_TAU_CT(120)
        HOL_TAU_CT(160)
        HOL_TAU_CT(200)
    default: break;
    }
#undef HOL_TAU_CT
    if ((rc = set_smem_attr<R>(up ? (const void*)fwdu : (const void*)fwd, sm))) return rc;
    if ((rc = set_smem_attr<R>((const void*)inv, sm))) return rc;
    const R isq = (R)(1.0 / sqrt((double)c->T));
    if (up) {
        PcUpdK<R> uk{(R*)up->x, (const R*)up->p, (const R*)up->pprev, (const R*)up->q, up->mask,
                     up->pq_part, up->pq_stride, up->pq_n, up->dz_part, up->dz_n, up->rr_out,
                     up->alpha_buf, up->fold};
        HOL_CUDA(launch_pdl(c, fwdu, gf, 256, sm, s, const_cast<R*>(v), h0, w2, c->T, c->N, TS,
                            plan, isq, uk));
        HOL_CHECK_LAUNCH("k_tau_fwd_upd");
    } else {
        HOL_CUDA(launch_pdl(c, fwd, gf, 256, sm, s, v, h0, w2, c->T, c->N, TS, plan, isq));
        HOL_CHECK_LAUNCH("k_tau_fwd");
    }
    KpmArgs ka;
    ka.L = c->L;
    ka.N = c->N;
    ka.Th = c->T / 2;
    ka.max_np = c->kpm.max_np;
    ka.mode = mode;
    ka.th = c->th;
    ka.ex = c->exact;
    ka.D = c->exact ? (sizeof(R) == 8 ? c->kin_d64 : c->kin_d32) : 0;
    for (int d = 0; d < kKinTaps; ++d) ka.e[d] = c->kin_e[d];
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        if ((c->kpm_reg == 1 || c->kpm_reg == 2) && !c->exact && (c->L == 32 || c->L == 16)) {
            const float th = (float)c->th;
            const size_t csm = (size_t)ka.max_np * sizeof(float2);
            const float2* i2 = reinterpret_cast<const float2*>(h0);
            float2* o2 = reinterpret_cast<float2*>(h1);
            auto run = [&](auto kern, int threads) -> int {
                if (int e = set_smem_attr<R>((const void*)kern, csm)) return e;
                const int items = ka.Th * n_rhs;
                int grid = items;
                int* q = nullptr;
                if (c->kpm_queue > 0 && items > c->kpm_queue * c->sms) {
                    grid = c->kpm_queue * c->sms;   // persistent: problems from the queue
                    q = c->kpm_q;
                }
                HOL_CUDA(launch_pdl(c, kern, grid, threads, csm, s, i2, o2, c->dbar, c->scal,
                                    c->kpm.np, c->kpm.coef, n_rhs, ka.Th, ka.max_np, mode, th,
                                    q));
                return HOL_OK;
            };
            const bool two = c->kpm_reg == 2;   // two columns per lane
            if (c->L == 32)
                rc = two ? run(k_kpm_reg<32, 2>, 32 * KGeo<32, 2>::W)
                         : run(k_kpm_reg<32, 4>, 32 * KGeo<32, 4>::W);
            else
                rc = two ? run(k_kpm_reg<16, 2>, 32 * KGeo<16, 2>::W)
                         : run(k_kpm_reg<16, 4>, 32 * KGeo<16, 4>::W);
            if (rc) return rc;
            HOL_CHECK_LAUNCH("k_kpm_reg");
            done = true;
        } else if (c->kpm_reg == 3 && !c->exact) {
            rc = run_kpm_lane<float>(c, reinterpret_cast<const float2*>(h0),
                                     reinterpret_cast<float2*>(h1), n_rhs, ka.Th, ka.max_np,
                                     mode, s);
            if (rc) return rc;
            done = true;
        }
    } else {
        // FP64: the banded lane layout (each problem over several warps: the
        // one-warp lane layout put a problem's chain of FP64 steps on one
        // SMSP's share of the FP64 pipe and measured slower than the
        // shared-memory kernel, 602 against 325 us on the L = 16,
        // Ltau = 160 trajectory's 2 rhs)
        if (c->kpm_reg != 0 && !c->exact && kpm_band_ok(c->L)) {
            rc = run_kpm_band(c, reinterpret_cast<const double2*>(h0),
                              reinterpret_cast<double2*>(h1), n_rhs, ka.Th, ka.max_np, mode, s);
            if (rc) return rc;
            done = true;
        }
    }
    if (!done) {
        const int kt = kpm_threads(c);
        const size_t ks = ((size_t)c->N * sizeof(C2) * (c->exact ? 2 : 1) + 15) / 16 * 16 +
                          (size_t)ka.max_np * sizeof(double2);
        if ((rc = set_smem_attr<R>((const void*)k_kpm<R>, ks))) return rc;
        HOL_CUDA(launch_pdl(c, k_kpm<R>, ka.Th * n_rhs, kt, ks, s, h0, h1, c->dbar, c->scal,
                            c->kpm.np, c->kpm.coef, n_rhs, ka));
        HOL_CHECK_LAUNCH("k_kpm");
    }
    HOL_CUDA(launch_pdl(c, inv, gf, 256, sm, s, h1, out, w2, c->T, c->N, TS, plan, (R)2 * isq,
                        rdot, dot_part));
    HOL_CHECK_LAUNCH("k_tau_inv");
    return HOL_OK;
}

}  // namespace

int precond_tiles(const hol_ctx* c, int prec) { return ceil_div(c->N, tile_sites(c, prec)); }

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

int precond_apply_upd(hol_ctx* c, int prec, void* r, void* z, int n_rhs, const PcUpd* u,
                      double* dot_part, cudaStream_t s)
{
    if (prec == HOL_F64)
        return precond_run<double>(c, (const double*)r, (double*)z, n_rhs, 3, (const double*)r,
                                   dot_part, s, u);
    return precond_run<float>(c, (const float*)r, (float*)z, n_rhs, 3, (const float*)r, dot_part,
                              s, u);
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
    const size_t sm = 2 * (size_t)c->kpm.max_np * sizeof(double2);
    if (int rc = smem_raise((const void*)k_kpm_coeffs, sm)) return rc;
    k_kpm_coeffs<<<c->T / 2, 128, sm, s>>>(c->scal, c->T, c->kpm.max_np, c->kpm.np, c->kpm.coef,
                                           c->kpm.np + c->T / 2, c->kpm_a1, c->kpm_a2);
    HOL_CHECK_LAUNCH("k_kpm_coeffs");
    return HOL_OK;
}

}  // namespace hol

using namespace hol;

extern "C" int precond_apply(hol_ctx* c, int which, int prec, const void* v, void* out, int n_rhs,
                             void* stream)
{
    HOL_TRACE("precond_apply");
    if (!c || !v || !out) return set_error(HOL_EINVAL, "precond_apply: null argument");
    if (int rc_ = require_aligned("precond_apply", {v, out})) return rc_;
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
