// Stochastic Green's-function measurements with FFT averaging (Sec. V).
//
// For probe vectors xi_n (<xi_i xi_j> = delta_ij, Sec. V B), G xi_n = M^{-1}
// xi_n is obtained from cg_solve on M^T M v = M^T xi_n. The space-time average
// of Eq. (G_avg-1) over the doubled, antiperiodic domain (Eq. (G_def-1)) is
// the circular cross-correlation of a = Q xi and b = Q G xi (Eq. (cross_corr)),
// normalised by 2 N Ltau (the mean over the original N Ltau sites):
//   G_Delta = (1/N_rv) sum_n (a_n star b_n)_Delta / (2 N Ltau).
// Because a and b are antiperiodic in tau with period Ltau, their transform
// over the doubled tau axis is nonzero only at odd frequencies 2 omega + 1,
// which is the twisted length-Ltau transform exp(-i pi (2 omega + 1) tau /
// Ltau) of the preconditioner; real inputs make omega and Ltau-1-omega
// conjugate, so only omega < Ltau/2 is kept, and G_{Delta l + Ltau} =
// -G_{Delta l}. In these terms
//   G_{dl, r} = 2 Re[ sum_{omega < T/2} e^{i pi (2 omega + 1) dl / T}
//               sum_q S_{omega,q} e^{2 pi i q.r / L} ] / ((N T)^2 N_rv),
//   S = sum_n conj(A_n) B_n, A = (twisted tau DFT x spatial DFT) of xi.
// The Wick products of Sec. V C are products of two antiperiodic vectors,
// hence periodic in Ltau: their doubled-domain correlation is twice the
// periodic one, so with plain (untwisted) transforms
//   W_k = IDFT( sum_{n<m} conj(F[p_n,m]) F[q_n,m] ) / (N T npairs),
// averaged over all pairs n < m (Eq. (GG_approx_better)); type 2 factorises
// and uses the prefix sums P_m = sum_{n<m} F[xi_n . G xi_n].
#include <math.h>

#include <vector>

#include "cb.cuh"
#include "fft.cuh"
#include "internal.cuh"

namespace hol {
namespace {

using namespace fft;

constexpr int kMeasTS = 16;

// real [nv][T][N] -> complex [nv][nw][N]: tau DFT of each site line,
// optionally twisted by exp(-i pi tau / T), first nw frequencies kept. Two
// real site lines share one complex transform (TS sites as TS / 2 columns):
// the transform X of a real line has X[w'] = conj X[w] with w' = T-1-w
// (twisted) or (T-w) mod T (plain), so Z = X_a + i X_b gives
// X_a = (Z[w] + conj Z[w']) / 2 and X_b = (Z[w] - conj Z[w']) / (2 i).
__global__ void __launch_bounds__(256) k_m_tau_fwd(const double* __restrict__ in,
                                                   double2* __restrict__ out,
                                                   const double2* __restrict__ w2, int T, int N,
                                                   int TS, RadixPlan plan, int twist, int nw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TH = TS / 2;
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (long)T * TH;
    const int vec = blockIdx.y, i0 = blockIdx.x * TS;
    const long ib = (long)vec * T * N;
    for (int item = threadIdx.x; item < T * TH; item += blockDim.x) {
        const int c = item % TH, tau = item / TH, i = i0 + 2 * c;   // N even: i + 1 < N too
        double xa = 0.0, xb = 0.0;
        if (i < N) {
            xa = in[ib + (long)tau * N + i];
            xb = in[ib + (long)tau * N + i + 1];
        }
        double2 z = make_double2(xa, xb);
        if (twist) {
            const double2 t = w2[tau];
            z = make_double2(xa * t.x - xb * t.y, xa * t.y + xb * t.x);
        }
        a[tau * TH + c] = z;
    }
    double2* res = fft_tau<double>(a, b, w2, T, TH, plan);
    const long ob = (long)vec * nw * N;
    for (int item = threadIdx.x; item < nw * TH; item += blockDim.x) {
        const int c = item % TH, w = item / TH, i = i0 + 2 * c;
        if (i < N) {
            const int wp = twist ? T - 1 - w : (w == 0 ? 0 : T - w);
            const double2 z = res[w * TH + c], zm = res[wp * TH + c];
            out[ob + (long)w * N + i] = make_double2(0.5 * (z.x + zm.x), 0.5 * (z.y - zm.y));
            out[ob + (long)w * N + i + 1] = make_double2(0.5 * (z.y + zm.y), 0.5 * (zm.x - z.x));
        }
    }
}

// In-place 2-D DFT of complex L x L planes [plane][iy][ix] (one block per
// plane): forward exp(-2 pi i q.r / L), or with inverse != 0 the unnormalised
// exp(+2 pi i q.r / L) (conjugate in and out); output times scale.
__global__ void __launch_bounds__(256) k_m_space(double2* __restrict__ planes,
                                                 const double2* __restrict__ w2L, int L,
                                                 RadixPlan plan, int inverse, double scale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + L * L;
    double2* p = planes + (long)blockIdx.x * L * L;
    for (int k = threadIdx.x; k < L * L; k += blockDim.x) {
        double2 z = p[k];
        if (inverse) z.y = -z.y;
        a[k] = z;                                  // a[iy][ix]
    }
    double2* res = fft_tau<double>(a, b, w2L, L, L, plan);   // along iy
    double2* oth = (res == a) ? b : a;
    for (int k = threadIdx.x; k < L * L; k += blockDim.x) {
        const int qy = k / L, ix = k - qy * L;
        oth[ix * L + qy] = res[k];                 // transpose: oth[ix][qy]
    }
    double2* res2 = fft_tau<double>(oth, res, w2L, L, L, plan);   // along ix -> [qx][qy]
    for (int k = threadIdx.x; k < L * L; k += blockDim.x) {
        const int qx = k / L, qy = k - qx * L;
        double2 z = res2[k];
        if (inverse) z.y = -z.y;
        p[qy * L + qx] = make_double2(scale * z.x, scale * z.y);
    }
}

// acc[k] += sum_v conj(A[v][k]) B[v][k]
__global__ void k_m_accum(double2* __restrict__ acc, const double2* __restrict__ A,
                          const double2* __restrict__ B, int nv, long len)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < len;
         k += (long)gridDim.x * blockDim.x) {
        double2 s = acc[k];
        for (int v = 0; v < nv; ++v) {
            const double2 a = A[(long)v * len + k], bb = B[(long)v * len + k];
            s.x += a.x * bb.x + a.y * bb.y;
            s.y += a.x * bb.y - a.y * bb.x;
        }
        acc[k] = s;
    }
}

// in order over v: acc += conj(P) C_v ; P += C_v
__global__ void k_m_prefix(double2* __restrict__ acc, double2* __restrict__ P,
                           const double2* __restrict__ C, int nv, long len)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < len;
         k += (long)gridDim.x * blockDim.x) {
        double2 s = acc[k], pp = P[k];
        for (int v = 0; v < nv; ++v) {
            const double2 c = C[(long)v * len + k];
            s.x += pp.x * c.x + pp.y * c.y;
            s.y += pp.x * c.y - pp.y * c.x;
            pp.x += c.x;
            pp.y += c.y;
        }
        acc[k] = s;
        P[k] = pp;
    }
}

// out[v][k] = x[k] * y[v][k]   (x stride 0) or xs[v][k] * ys[v][k]
__global__ void k_m_prod(double* __restrict__ out, const double* __restrict__ x, long xstride,
                         const double* __restrict__ y, long n, int nv)
{
    const long tot = n * nv;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < tot;
         k += (long)gridDim.x * blockDim.x) {
        const long v = k / n, e = k - v * n;
        out[k] = x[v * xstride + e] * y[k];
    }
}

// complex [T/2][N] (conjugate-symmetric, twisted) -> real [T][N]:
// out = scale * Re(exp(-i pi tau/T) * sum_{w<T/2} conj(in_w) e^{-2 pi i w tau/T})
__global__ void __launch_bounds__(256) k_m_tau_inv_half(const double2* __restrict__ in,
                                                        double* __restrict__ out,
                                                        const double2* __restrict__ w2, int T,
                                                        int N, int TS, RadixPlan plan,
                                                        double scale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (long)T * TS;
    const int i0 = blockIdx.x * TS, Th = T / 2;
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, w = item / TS, i = i0 + c;
        double2 z = make_double2(0.0, 0.0);
        if (w < Th && i < N) {
            z = in[(long)w * N + i];
            z.y = -z.y;
        }
        a[w * TS + c] = z;
    }
    double2* res = fft_tau<double>(a, b, w2, T, TS, plan);
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, tau = item / TS, i = i0 + c;
        if (i < N) {
            const double2 t = w2[tau], z = res[tau * TS + c];
            out[(long)tau * N + i] = scale * (t.x * z.x - t.y * z.y);
        }
    }
}

// complex [T][N] (full, untwisted) -> real [T][N]:
// out = scale * Re(sum_w in_w e^{+2 pi i w tau / T})
__global__ void __launch_bounds__(256) k_m_tau_inv_full(const double2* __restrict__ in,
                                                        double* __restrict__ out,
                                                        const double2* __restrict__ w2, int T,
                                                        int N, int TS, RadixPlan plan,
                                                        double scale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* a = reinterpret_cast<double2*>(smem_raw);
    double2* b = a + (long)T * TS;
    const int i0 = blockIdx.x * TS;
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, w = item / TS, i = i0 + c;
        double2 z = make_double2(0.0, 0.0);
        if (i < N) {
            z = in[(long)w * N + i];
            z.y = -z.y;
        }
        a[w * TS + c] = z;
    }
    double2* res = fft_tau<double>(a, b, w2, T, TS, plan);
    for (int item = threadIdx.x; item < T * TS; item += blockDim.x) {
        const int c = item % TS, tau = item / TS, i = i0 + c;
        if (i < N) out[(long)tau * N + i] = scale * res[tau * TS + c].x;
    }
}

// out[dl][r] = in[dl][r] for dl < T and sign * in[dl - T][r] for dl >= T
__global__ void k_m_fill(const double* __restrict__ in, double* __restrict__ out, long n,
                         double sign)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x) {
        const double v = in[k];
        out[k] = v;
        out[n + k] = sign * v;
    }
}

int g1(long n)
{
    long nb = (n + 255) / 256;
    return (int)(nb > 8192 ? 8192 : (nb < 1 ? 1 : nb));
}

struct Meas {
    hol_ctx* c;
    RadixPlan pt, ps;
    size_t sm_t, sm_s;
    int ts_threads;   // threads of the spatial FFT: a multiple of L
    cudaStream_t s;

    int attrs()
    {
        const void* fns[] = {(const void*)k_m_tau_fwd, (const void*)k_m_tau_inv_half,
                             (const void*)k_m_tau_inv_full};
        for (const void* f : fns)
            if (int rc = smem_raise(f, sm_t)) return rc;
        return HOL_OK;
    }
    // real vectors [nv][T][N] -> spectra [nv][nw][N] (tau then space)
    int spectra(const double* in, double2* out, int nv, int twist, int nw)
    {
        const dim3 g(ceil_div(c->N, kMeasTS), nv);
        k_m_tau_fwd<<<g, 256, sm_t, s>>>(in, out, c->tw64, c->T, c->N, kMeasTS, pt, twist, nw);
        HOL_CHECK_LAUNCH("k_m_tau_fwd");
        k_m_space<<<nv * nw, ts_threads, sm_s, s>>>(out, c->twL64, c->L, ps, 0, 1.0);
        HOL_CHECK_LAUNCH("k_m_space");
        return HOL_OK;
    }
};

}  // namespace

int measure_alloc(hol_ctx* c)
{
    const long TN = c->n;
    HOL_CUDA(cudaMalloc((void**)&c->ms_acc, 5 * TN * sizeof(double2)));
    std::vector<double2> h(2 * c->L);
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int k = 0; k < 2 * c->L; ++k) {
        const long double ang = -pi * (long double)k / (long double)c->L;
        h[k] = make_double2((double)cosl(ang), (double)sinl(ang));
    }
    HOL_CUDA(cudaMalloc((void**)&c->twL64, 2 * c->L * sizeof(double2)));
    HOL_CUDA(cudaMemcpy(c->twL64, h.data(), 2 * c->L * sizeof(double2), cudaMemcpyHostToDevice));
    return HOL_OK;
}

// Shared-memory limits of the measurement kernels for this context's shape,
// raised outside any stream capture.
int measure_prepare(hol_ctx* c)
{
    Meas m;
    m.c = c;
    m.pt = plan_of(c->T);
    m.ps = plan_of(c->L);
    if (m.pt.n < 0 || m.ps.n < 0)
        return set_error(HOL_EINVAL, "stochastic_measure: L=%d and Ltau=%d need prime factors in {2,3,5,7}",
                         c->L, c->T);
    m.sm_t = 2 * (size_t)c->T * kMeasTS * sizeof(double2);
    return m.attrs();
}

int measure_run(hol_ctx* c, const double* xi, int n_rv, const hol_cg_opts* opts, double* Gxi,
                double* G2, double* G4, int four_point, int* iters, cudaStream_t stream);

}  // namespace hol

using namespace hol;

extern "C" int stochastic_measure(hol_ctx* c, const double* xi, int n_rv, const hol_cg_opts* opts,
                                  double* Gxi, double* G2, double* G4, int four_point, int* iters,
                                  void* stream)
{
    HOL_TRACE("stochastic_measure");
    return measure_run(c, xi, n_rv, opts, Gxi, G2, G4, four_point, iters, (cudaStream_t)stream);
}

// The measurement of stochastic_measure; inside a graph capture its probe
// solves are device-driven (cg_run_dev) and no iteration counts are returned.
int hol::measure_run(hol_ctx* c, const double* xi, int n_rv, const hol_cg_opts* opts, double* Gxi,
                     double* G2, double* G4, int four_point, int* iters, cudaStream_t stream)
{
    if (!c || !xi || !opts || !Gxi || !G2) return set_error(HOL_EINVAL, "stochastic_measure: null argument");
    if (int rc_ = require_aligned("stochastic_measure", {xi, Gxi, G2, G4})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "stochastic_measure: hol_set_field not called");
    if (n_rv < 1) return set_error(HOL_EINVAL, "stochastic_measure: n_rv=%d", n_rv);
    if (four_point & ~7) return set_error(HOL_EINVAL, "stochastic_measure: bad four_point mask");
    if (four_point && (!G4 || n_rv < 2))
        return set_error(HOL_EINVAL, "stochastic_measure: four-point products need G4 and n_rv >= 2");
    Meas m;
    m.c = c;
    m.s = (cudaStream_t)stream;
    m.pt = plan_of(c->T);
    m.ps = plan_of(c->L);
    if (m.pt.n < 0 || m.ps.n < 0)
        return set_error(HOL_EINVAL, "stochastic_measure: L=%d and Ltau=%d need prime factors in {2,3,5,7}",
                         c->L, c->T);
    m.sm_t = 2 * (size_t)c->T * kMeasTS * sizeof(double2);
    m.sm_s = 2 * (size_t)c->N * sizeof(double2);
    m.ts_threads = c->L * (256 / c->L);
    int rc = m.attrs();
    if (rc) return rc;
    cudaStream_t s = m.s;
    const long n = c->n, N = c->N;
    const int T = c->T, Th = T / 2;
    const int R = c->p.max_rhs;

    // 1. G xi = (M^T M)^{-1} M^T xi, in chunks of max_rhs
    for (int v0 = 0; v0 < n_rv; v0 += R) {
        const int nv = (n_rv - v0) < R ? (n_rv - v0) : R;
        if ((rc = launch_MT(c, HOL_F64, xi + (long)v0 * n, c->md_b, nv, nullptr, s))) return rc;
        if (c->capturing) {
            if ((rc = cg_run_dev(c, c->md_b, Gxi + (long)v0 * n, nv, opts, s))) return rc;
            continue;
        }
        std::vector<int> it(nv);
        if ((rc = cg_solve(c, c->md_b, Gxi + (long)v0 * n, nv, opts, it.data(), nullptr, s)))
            return rc;
        if (iters)
            for (int k = 0; k < nv; ++k) iters[v0 + k] = it[k];
    }

    double2* S2 = c->ms_acc;              // [T/2][N]
    double2* W = c->ms_acc + n;           // three [T][N] accumulators
    double2* P = c->ms_acc + 4 * n;       // [T][N] type-2 prefix (only T/2.. used as full)
    // the half-spectrum accumulator only needs T/2 planes; the prefix needs T
    double2* A = c->cbuf0;
    double2* B = c->cbuf1;
    const long cap = c->cbuf_len;         // complex elements per buffer
    HOL_CUDA(cudaMemsetAsync(S2, 0, (size_t)Th * N * sizeof(double2), s));
    HOL_CUDA(cudaMemsetAsync(W, 0, (size_t)3 * n * sizeof(double2), s));
    HOL_CUDA(cudaMemsetAsync(P, 0, (size_t)n * sizeof(double2), s));

    // 2. two-point: S += conj(A_n) B_n over twisted half spectra
    {
        const int chunk = (int)(cap / ((long)Th * N));
        for (int v0 = 0; v0 < n_rv; v0 += chunk) {
            const int nv = (n_rv - v0) < chunk ? (n_rv - v0) : chunk;
            if ((rc = m.spectra(xi + (long)v0 * n, A, nv, 1, Th))) return rc;
            if ((rc = m.spectra(Gxi + (long)v0 * n, B, nv, 1, Th))) return rc;
            k_m_accum<<<g1((long)Th * N), 256, 0, s>>>(S2, A, B, nv, (long)Th * N);
            HOL_CHECK_LAUNCH("k_m_accum");
        }
        k_m_space<<<Th, m.ts_threads, m.sm_s, s>>>(S2, c->twL64, c->L, m.ps, 1, 1.0);
        HOL_CHECK_LAUNCH("k_m_space inv");
        double* tmp = c->v64a;
        const double sc = 2.0 / ((double)N * T * (double)N * T * n_rv);
        k_m_tau_inv_half<<<ceil_div(N, kMeasTS), 256, m.sm_t, s>>>(S2, tmp, c->tw64, T, (int)N,
                                                                    kMeasTS, m.pt, sc);
        HOL_CHECK_LAUNCH("k_m_tau_inv_half");
        k_m_fill<<<g1(n), 256, 0, s>>>(tmp, G2, n, -1.0);
        HOL_CHECK_LAUNCH("k_m_fill");
    }
    if (!four_point) return HOL_OK;

    // 3. Wick products (plain transforms, periodic in Ltau), pairs n < m
    const long npairs = (long)n_rv * (n_rv - 1) / 2;
    const int chunk = (int)(cap / n);     // full spectra per buffer
    if (chunk < 1) return set_error(HOL_EINVAL, "stochastic_measure: scratch too small");
    double* pa = c->v64a;                 // real products, up to max_rhs vectors
    double* pb = c->v64b;
    const int pchunk = chunk < R ? chunk : R;
    if (four_point & 2) {   // type 2 by prefix sums: c_n = xi_n . G xi_n
        for (int v0 = 0; v0 < n_rv; v0 += pchunk) {
            const int nv = (n_rv - v0) < pchunk ? (n_rv - v0) : pchunk;
            k_m_prod<<<g1(n * nv), 256, 0, s>>>(pa, xi + (long)v0 * n, n, Gxi + (long)v0 * n, n, nv);
            HOL_CHECK_LAUNCH("k_m_prod");
            if ((rc = m.spectra(pa, A, nv, 0, T))) return rc;
            k_m_prefix<<<g1(n), 256, 0, s>>>(W + n, P, A, nv, n);
            HOL_CHECK_LAUNCH("k_m_prefix");
        }
    }
    if (four_point & 5) {   // types 1 and 3 pair by pair
        for (int a = 0; a + 1 < n_rv; ++a) {
            for (int v0 = a + 1; v0 < n_rv; v0 += pchunk) {
                const int nv = (n_rv - v0) < pchunk ? (n_rv - v0) : pchunk;
                if (four_point & 1) {   // (xi_a . xi_m) star (G xi_a . G xi_m)
                    k_m_prod<<<g1(n * nv), 256, 0, s>>>(pa, xi + (long)a * n, 0, xi + (long)v0 * n, n, nv);
                    k_m_prod<<<g1(n * nv), 256, 0, s>>>(pb, Gxi + (long)a * n, 0, Gxi + (long)v0 * n, n, nv);
                    HOL_CHECK_LAUNCH("k_m_prod");
                    if ((rc = m.spectra(pa, A, nv, 0, T))) return rc;
                    if ((rc = m.spectra(pb, B, nv, 0, T))) return rc;
                    k_m_accum<<<g1(n), 256, 0, s>>>(W, A, B, nv, n);
                    HOL_CHECK_LAUNCH("k_m_accum");
                }
                if (four_point & 4) {   // (xi_a . G xi_m) star (xi_m . G xi_a)
                    k_m_prod<<<g1(n * nv), 256, 0, s>>>(pa, xi + (long)a * n, 0, Gxi + (long)v0 * n, n, nv);
                    k_m_prod<<<g1(n * nv), 256, 0, s>>>(pb, Gxi + (long)a * n, 0, xi + (long)v0 * n, n, nv);
                    HOL_CHECK_LAUNCH("k_m_prod");
                    if ((rc = m.spectra(pa, A, nv, 0, T))) return rc;
                    if ((rc = m.spectra(pb, B, nv, 0, T))) return rc;
                    k_m_accum<<<g1(n), 256, 0, s>>>(W + 2 * n, A, B, nv, n);
                    HOL_CHECK_LAUNCH("k_m_accum");
                }
            }
        }
    }
    const double sc4 = 1.0 / ((double)N * T * (double)N * T * npairs);
    for (int k = 0; k < 3; ++k) {
        double* out = G4 + (long)k * 2 * n;
        if (!(four_point & (1 << k))) {
            HOL_CUDA(cudaMemsetAsync(out, 0, 2 * n * sizeof(double), s));
            continue;
        }
        k_m_space<<<T, m.ts_threads, m.sm_s, s>>>(W + (long)k * n, c->twL64, c->L, m.ps, 1, 1.0);
        HOL_CHECK_LAUNCH("k_m_space inv");
        double* tmp = c->v64a;
        k_m_tau_inv_full<<<ceil_div(N, kMeasTS), 256, m.sm_t, s>>>(W + (long)k * n, tmp, c->tw64, T,
                                                                    (int)N, kMeasTS, m.pt, sc4);
        HOL_CHECK_LAUNCH("k_m_tau_inv_full");
        k_m_fill<<<g1(n), 256, 0, s>>>(tmp, out, n, 1.0);
        HOL_CHECK_LAUNCH("k_m_fill");
    }
    return HOL_OK;
}


// ---------------------------------------------------------------------------
// Observables from the averaged 2-point function and the Wick products
// (Eq. (Scdw) and the pair susceptibility P_s), one block:
//   g0 = G2[0][0][0] (mean G_aa), <n> = 2 (1 - g0),
//   C(r) = 4 (1 - 2 g0 + G4[1][0][r]) + 2 (delta_{r,0} g0 - G4[2][0][r]),
//   S_cdw = sum_r (-1)^(rx+ry) C(r),  P_s = dtau sum_{l < T} sum_r G4[0][l][r].
// Every sum is taken in a fixed order by thread 0 of one warp (the arrays
// hold a few thousand numbers).
// ---------------------------------------------------------------------------
namespace hol {
namespace {
__global__ void k_observables(const double* __restrict__ G2, const double* __restrict__ G4,
                              int L, int T, double dtau, double* __restrict__ C,
                              double* __restrict__ scal)
{
    const int LL = L * L;
    const double g0 = G2[0];
    const double* w0 = G4;                       // type 1 [2T][L][L]
    const double* w1 = G4 + (long)2 * T * LL;    // type 2
    const double* w2 = G4 + (long)4 * T * LL;    // type 3
    for (int r = threadIdx.x; r < LL; r += blockDim.x)
        C[r] = 4.0 * (1.0 - 2.0 * g0 + w1[r]) + 2.0 * ((r == 0 ? g0 : 0.0) - w2[r]);
    __syncthreads();
    if (threadIdx.x == 0) {
        double scdw = 0.0;
        for (int r = 0; r < LL; ++r) {
            const int dx = r % L, dy = r / L;
            scdw += ((dx + dy) & 1) ? -C[r] : C[r];
        }
        double ps = 0.0;
        for (long k = 0; k < (long)T * LL; ++k) ps += w0[k];
        scal[0] = 2.0 * (1.0 - g0);
        scal[1] = scdw;
        scal[2] = dtau * ps;
    }
}
}  // namespace
}  // namespace hol

extern "C" int measure_observables(hol_ctx* c, const double* G2, const double* G4, double* C,
                                   double* out3, void* stream)
{
    HOL_TRACE("measure_observables");
    if (!c || !G2 || !G4 || !C || !out3)
        return set_error(HOL_EINVAL, "measure_observables: null argument");
    if (int rc_ = require_aligned("measure_observables", {G2, G4, C})) return rc_;
    cudaStream_t s = (cudaStream_t)stream;
    double* scal = c->md_s + 12;
    k_observables<<<1, 256, 0, s>>>(G2, G4, c->L, c->T, c->p.dtau, C, scal);
    HOL_CHECK_LAUNCH("k_observables");
    HOL_CUDA(cudaMemcpyAsync(out3, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HOL_CUDA(cudaStreamSynchronize(s));
    return HOL_OK;
}
