// Arnoldi estimate of the spectral bounds of Bbar = exp(-dtau Vbar) C
// (App. C D): m steps of the Arnoldi process from a caller-given start
// vector on Bbar, whose largest Ritz modulus (eigenvalue of the m x m
// Hessenberg matrix, on the host) increased by a margin gives bmax, and on
// Bbar^{-1} = C^{-1} exp(dtau Vbar), whose largest Ritz modulus increased by
// the margin gives 1 / bmin (the paper's way to reach the small end stably).
// The paper runs about twenty steps from a random start with a 5 % margin.
// Optionally installs the bounds in the context (Chebyshev orders and
// coefficients recomputed), in place of the deterministic norm bounds that
// hol_set_field sets.
//
// The process runs in one block: Bbar v is the propagator (checkerboard
// colours or the exact separable taps) on a slice in shared memory followed
// by the diagonal dbar; every dot product is a block reduction in a fixed
// order, so the result is deterministic. Modified Gram-Schmidt applied twice
// per step.
#include <complex>
#include <math.h>
#include <vector>

#include "internal.cuh"

namespace hol {

int kpm_setup(hol_ctx* c, cudaStream_t s);   // precond.cu

namespace {

struct ArnArgs {
    int N, L, m;
    int inv;                  // 0: Bbar, 1: Bbar^{-1}
    int ex, D;                // exact propagator and its taps
    double th;                // checkerboard bond tanh(dtau t) (negated for the inverse)
    double scale;             // inverse checkerboard: (1 - th^2)^-4, else 1
    double e[kKinTaps];       // exact taps (sign-alternated for the inverse)
};

// Fixed-order block sum, the same value in every thread.
__device__ double block_total(double v, double* red)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    __syncthreads();
    return t;
}

// One checkerboard colour (0: x-even, 1: x-odd, 2: y-even, 3: y-odd) on a
// real slice in shared memory, bonds [[1, th], [th, 1]].
__device__ void arn_colour(double* v, int colour, int L, double th)
{
    const int half = L / 2;
    for (int k = threadIdx.x; k < L * half; k += blockDim.x) {
        int i, j;
        if (colour < 2) {
            const int iy = k / half, ix = 2 * (k - iy * half) + colour;
            i = ix + L * iy;
            j = (ix + 1 == L ? 0 : ix + 1) + L * iy;
        } else {
            const int ix = k % L, iy = 2 * (k / L) + (colour - 2);
            i = ix + L * iy;
            j = ix + L * (iy + 1 == L ? 0 : iy + 1);
        }
        const double a = v[i], b = v[j];
        v[i] = fma(th, b, a);
        v[j] = fma(th, a, b);
    }
    __syncthreads();
}

// v <- (E (x) E) v, x direction into tmp, then y back into v.
__device__ void arn_exact(double* v, double* tmp, const ArnArgs& a)
{
    const int L = a.L;
    for (int i = threadIdx.x; i < a.N; i += blockDim.x) {
        const int iy = i / L, ix = i - iy * L, row = iy * L;
        double o = a.e[0] * v[i];
        for (int d = 1; d <= a.D; ++d) {
            double u = v[row + (ix + d) % L];
            if (2 * d != L) u += v[row + (ix + L - d) % L];
            o = fma(a.e[d], u, o);
        }
        tmp[i] = o;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.N; i += blockDim.x) {
        const int iy = i / L, ix = i - iy * L;
        double o = a.e[0] * tmp[i];
        for (int d = 1; d <= a.D; ++d) {
            double u = tmp[((iy + d) % L) * L + ix];
            if (2 * d != L) u += tmp[((iy + L - d) % L) * L + ix];
            o = fma(a.e[d], u, o);
        }
        v[i] = o;
    }
    __syncthreads();
}

// V: [m + 1][N] orthonormal basis; H: [m + 1][m] row-major Hessenberg;
// info[0] = number of completed steps (smaller than m on an invariant
// subspace).
__global__ void __launch_bounds__(256) k_arnoldi(const double* __restrict__ v0,
                                                 const double* __restrict__ dbar, ArnArgs a,
                                                 double* __restrict__ V, double* __restrict__ H,
                                                 int* __restrict__ info)
{
    extern __shared__ double sh[];
    double* w = sh;                 // [N]
    double* tmp = sh + a.N;         // [N] (exact propagator)
    __shared__ double red[32];
    const int N = a.N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += v0[i] * v0[i];
    const double nrm = sqrt(block_total(s, red));
    for (int i = threadIdx.x; i < N; i += blockDim.x) V[i] = v0[i] / nrm;
    for (int k = threadIdx.x; k < (a.m + 1) * a.m; k += blockDim.x) H[k] = 0.0;
    __syncthreads();
    int done = a.m;
    for (int j = 0; j < a.m; ++j) {
        const double* vj = V + (long)j * N;
        for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = vj[i];
        __syncthreads();
        if (a.inv) {   // Bbar^{-1} v = C^{-1} (v / dbar)
            for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] /= dbar[i];
            __syncthreads();
        }
        if (a.ex) {
            arn_exact(w, tmp, a);   // the inverse is exp(-dtau t A) per direction: taps (-1)^d e[d]
        } else if (a.inv) {
            // C^{-1} = C1^{-1} C2^{-1} C3^{-1} C4^{-1}; [[1, th], [th, 1]]^{-1} is
            // [[1, -th], [-th, 1]] / (1 - th^2), and every site is in one bond per colour
            for (int c = 3; c >= 0; --c) arn_colour(w, c, a.L, a.th);
        } else {
            for (int c = 0; c < 4; ++c) arn_colour(w, c, a.L, a.th);   // C4 C3 C2 C1
        }
        double q0 = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            w[i] *= a.inv ? a.scale : dbar[i];
            q0 += w[i] * w[i];
        }
        const double wn0 = sqrt(block_total(q0, red));   // |Bbar v_j| (the barrier is inside)
        // modified Gram-Schmidt, twice (a single pass loses orthogonality as
        // the Ritz values converge); H collects both passes' coefficients
        for (int pass = 0; pass < 2; ++pass)
            for (int k = 0; k <= j; ++k) {
                const double* vk = V + (long)k * N;
                double d = 0.0;
                for (int i = threadIdx.x; i < N; i += blockDim.x) d += vk[i] * w[i];
                const double h = block_total(d, red);
                for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] -= h * vk[i];
                if (threadIdx.x == 0) H[k * a.m + j] += h;
                __syncthreads();
            }
        double q = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) q += w[i] * w[i];
        const double hn = sqrt(block_total(q, red));
        if (threadIdx.x == 0) H[(j + 1) * a.m + j] = hn;
        if (!(hn > 1e-12 * wn0)) {   // invariant subspace (same decision in every thread)
            done = j + 1;
            break;
        }
        double* vn = V + (long)(j + 1) * N;
        for (int i = threadIdx.x; i < N; i += blockDim.x) vn[i] = w[i] / hn;
        __syncthreads();
    }
    if (threadIdx.x == 0) info[0] = done;
}

// Eigenvalues of the n x n upper Hessenberg matrix A (row-major, complex
// copy) by the shifted QR iteration (Wilkinson shift, Givens rotations,
// deflation from the bottom; Golub and Van Loan, Sec. 7.5). Returns false if
// it does not converge.
bool hessenberg_eigenvalues(int n, std::vector<std::complex<double>>& A,
                            std::vector<std::complex<double>>& ev)
{
    using cd = std::complex<double>;
    auto at = [&](int i, int j) -> cd& { return A[(size_t)i * n + j]; };
    ev.assign(n, cd(0.0, 0.0));
    int hi = n - 1, iter = 0;
    const double eps = 1e-15;
    while (hi >= 0) {
        if (hi == 0) {
            ev[0] = at(0, 0);
            break;
        }
        int l = hi;
        while (l > 0) {
            const double sc = std::abs(at(l, l)) + std::abs(at(l - 1, l - 1));
            if (std::abs(at(l, l - 1)) <= eps * (sc > 0.0 ? sc : 1.0)) {
                at(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {   // 1 x 1 block converged
            ev[hi] = at(hi, hi);
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 200 * n) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 closer to its corner
        const cd a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
        const cd mid = 0.5 * (a + d), half = 0.5 * (a - d);
        const cd disc = std::sqrt(half * half + b * c);
        const cd l1 = mid + disc, l2 = mid - disc;
        cd mu = std::abs(l1 - d) <= std::abs(l2 - d) ? l1 : l2;
        if (iter % 11 == 0) mu = d + std::abs(c);   // exceptional shift against cycling
        for (int k = l; k <= hi; ++k) at(k, k) -= mu;
        std::vector<cd> gc(hi - l), gs(hi - l);
        for (int k = l; k < hi; ++k) {   // A - mu I = Q R
            const cd x = at(k, k), y = at(k + 1, k);
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            const cd cc = r > 0.0 ? x / r : cd(1.0), ss = r > 0.0 ? y / r : cd(0.0);
            gc[k - l] = cc;
            gs[k - l] = ss;
            for (int j = k; j <= hi; ++j) {
                const cd u = at(k, j), v = at(k + 1, j);
                at(k, j) = std::conj(cc) * u + std::conj(ss) * v;
                at(k + 1, j) = -ss * u + cc * v;
            }
        }
        for (int k = l; k < hi; ++k) {   // R Q
            const cd cc = gc[k - l], ss = gs[k - l];
            const int top = l;
            const int bot = k + 1 < hi ? k + 2 : hi;
            for (int i = top; i <= bot; ++i) {
                const cd u = at(i, k), v = at(i, k + 1);
                at(i, k) = u * cc + v * ss;
                at(i, k + 1) = -u * std::conj(ss) + v * std::conj(cc);
            }
        }
        for (int k = l; k <= hi; ++k) at(k, k) += mu;
    }
    return true;
}

}  // namespace
}  // namespace hol

using namespace hol;

extern "C" int hol_arnoldi_bounds(hol_ctx* c, const double* v0, int m, double margin, int install,
                                  double* bmin, double* bmax, int* steps, void* stream)
{
    HOL_TRACE("hol_arnoldi_bounds");
    if (!c || !v0) return set_error(HOL_EINVAL, "hol_arnoldi_bounds: null argument");
    if (int rc_ = require_aligned("hol_arnoldi_bounds", {v0})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "hol_arnoldi_bounds: hol_set_field not called");
    if (m < 1 || m > kArnoldiMax || m > c->N)
        return set_error(HOL_EINVAL, "hol_arnoldi_bounds: m=%d outside [1, min(%d, N)]", m,
                         kArnoldiMax);
    if (!(margin >= 0.0 && margin < 1.0))
        return set_error(HOL_EINVAL, "hol_arnoldi_bounds: margin must be in [0, 1)");
    cudaStream_t s = (cudaStream_t)stream;
    double* V = c->arn;
    double* H = c->arn + (size_t)(kArnoldiMax + 1) * c->N;
    int* info = reinterpret_cast<int*>(H + (kArnoldiMax + 1) * kArnoldiMax);
    const size_t sm = 2 * (size_t)c->N * sizeof(double);
    if (int rc = smem_raise((const void*)k_arnoldi, sm)) return rc;
    double top[2] = {0.0, 0.0};   // largest Ritz modulus of Bbar, of Bbar^{-1}
    int done_min = m;
    for (int inv = 0; inv < 2; ++inv) {
        ArnArgs a;
        a.N = c->N;
        a.L = c->L;
        a.m = m;
        a.inv = inv;
        a.ex = c->exact;
        a.D = c->exact ? c->kin_d64 : 0;
        a.th = inv ? -c->th : c->th;
        const double u = 1.0 - c->th * c->th;
        a.scale = (inv && !c->exact) ? 1.0 / (u * u * u * u) : 1.0;
        for (int d = 0; d < kKinTaps; ++d) a.e[d] = (inv && (d & 1)) ? -c->kin_e[d] : c->kin_e[d];
        k_arnoldi<<<1, 256, sm, s>>>(v0, c->dbar, a, V, H, info);
        HOL_CHECK_LAUNCH("k_arnoldi");
        std::vector<double> h((size_t)(m + 1) * m);
        int done = 0;
        HOL_CUDA(cudaMemcpyAsync(h.data(), H, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 s));
        HOL_CUDA(cudaMemcpyAsync(&done, info, sizeof(int), cudaMemcpyDeviceToHost, s));
        HOL_CUDA(cudaStreamSynchronize(s));
        if (done < 1 || done > m)
            return set_error(HOL_ENUMERIC, "hol_arnoldi_bounds: no step done");
        done_min = done < done_min ? done : done_min;
        std::vector<std::complex<double>> A((size_t)done * done), ev;
        for (int i = 0; i < done; ++i)
            for (int j = 0; j < done; ++j) A[(size_t)i * done + j] = h[(size_t)i * m + j];
        if (!hessenberg_eigenvalues(done, A, ev))
            return set_error(HOL_ENUMERIC, "hol_arnoldi_bounds: QR iteration did not converge");
        for (const auto& z : ev) top[inv] = std::abs(z) > top[inv] ? std::abs(z) : top[inv];
    }
    if (!(top[0] > 0.0) || !(top[1] > 0.0) || !isfinite(top[0]) || !isfinite(top[1]))
        return set_error(HOL_ENUMERIC, "hol_arnoldi_bounds: degenerate Ritz values");
    const double b0 = 1.0 / ((1.0 + margin) * top[1]), b1 = (1.0 + margin) * top[0];
    if (bmin) *bmin = b0;
    if (bmax) *bmax = b1;
    if (steps) *steps = done_min;
    if (install) {
        static_assert(S_BMIN == 0 && S_BMAX == 1, "bounds are the first two scalars");
        const double b[2] = {b0, b1};
        HOL_CUDA(cudaMemcpyAsync(c->scal, b, sizeof(b), cudaMemcpyHostToDevice, s));
        if (int rc = kpm_setup(c, s)) return rc;
        HOL_CUDA(cudaStreamSynchronize(s));
    }
    return HOL_OK;
}

extern "C" int hol_get_bounds(hol_ctx* c, double* bmin, double* bmax, void* stream)
{
    HOL_TRACE("hol_get_bounds");
    if (!c || !bmin || !bmax) return set_error(HOL_EINVAL, "hol_get_bounds: null argument");
    if (!c->field_set) return set_error(HOL_EINVAL, "hol_get_bounds: hol_set_field not called");
    cudaStream_t s = (cudaStream_t)stream;
    double b[2];
    HOL_CUDA(cudaMemcpyAsync(b, c->scal, sizeof(b), cudaMemcpyDeviceToHost, s));
    HOL_CUDA(cudaStreamSynchronize(s));
    *bmin = b[S_BMIN];
    *bmax = b[S_BMAX];
    return HOL_OK;
}

extern "C" int hol_hessenberg_eigenvalues(int n, const double* H, double* re, double* im)
{
    HOL_TRACE("hol_hessenberg_eigenvalues");
    if (n < 1 || !H || !re || !im)
        return set_error(HOL_EINVAL, "hol_hessenberg_eigenvalues: bad argument");
    for (int i = 2; i < n; ++i)
        for (int j = 0; j + 1 < i; ++j)
            if (H[(size_t)i * n + j] != 0.0)
                return set_error(HOL_EINVAL, "hol_hessenberg_eigenvalues: not upper Hessenberg");
    std::vector<std::complex<double>> A((size_t)n * n), ev;
    for (size_t k = 0; k < A.size(); ++k) A[k] = H[k];
    if (!hessenberg_eigenvalues(n, A, ev))
        return set_error(HOL_ENUMERIC, "hol_hessenberg_eigenvalues: QR iteration did not converge");
    for (int k = 0; k < n; ++k) {
        re[k] = ev[k].real();
        im[k] = ev[k].imag();
    }
    return HOL_OK;
}

