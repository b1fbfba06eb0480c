// Shared-memory mixed-radix FFT along tau (Stockham passes of radix 4, 2, 3,
// 5, 7) over tiles of TS columns, plus complex helpers. Used by the
// preconditioner (twisted transforms), the Fourier-accelerated leapfrog (mass
// matrix along tau) and the measurements.
#pragma once

#include <cuda_runtime.h>

namespace hol {
namespace fft {

// ---------------------------------------------------------------- complex
template <typename R>
struct Cx;
template <>
struct Cx<float> {
    using T2 = float2;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <>
struct Cx<double> {
    using T2 = double2;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};
template <typename C>
__device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}

struct RadixPlan {
    int n;
    int r[16];
};

// twiddle w2[k] = exp(-i pi k / T), 0 <= k < 2T (every caller's index is in
// range: 2 r k T / (Ns RAD) < 2T and 2 e T / RAD < 2T)
template <typename R>
__device__ __forceinline__ typename Cx<R>::T2 tw(const typename Cx<R>::T2* __restrict__ w2, long k,
                                                 int T)
{
    (void)T;
    return w2[k];
}

template <typename C>
__device__ __forceinline__ C csub(C a, C b)
{
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
// multiply by -i
template <typename C>
__device__ __forceinline__ C cmi(C a)
{
    C r;
    r.x = a.y;
    r.y = -a.x;
    return r;
}

// One Stockham pass of radix RAD over TS columns: in[tau][c] -> out[.][c].
// Butterfly j (0 <= j < T/RAD) with k = j mod Ns reads in[j + r T/RAD],
// scales input r by exp(-2 pi i r k / (Ns RAD)), takes the length-RAD DFT
// and writes out[(j / Ns) Ns RAD + k + q Ns]. blockDim.x must be a multiple
// of TS; (k, j / Ns) are advanced incrementally instead of divided.
template <typename R, int RAD>
__device__ void stockham_pass(const typename Cx<R>::T2* __restrict__ in,
                              typename Cx<R>::T2* __restrict__ out,
                              const typename Cx<R>::T2* __restrict__ w2, int T, int TS, int Ns)
{
    using C2 = typename Cx<R>::T2;
    const int nb = T / RAD;
    const int c = threadIdx.x % TS;
    const int sj = blockDim.x / TS;         // step of j per iteration
    int j = threadIdx.x / TS;
    int k = j % Ns, jb = j / Ns;
    const int sk = sj % Ns, sjb = sj / Ns;
    const int tstep = T / (Ns * RAD);       // twiddle index step per unit of k, halved
    C2 root[RAD];                           // exp(-2 pi i e / RAD)
#pragma unroll
    for (int e = 0; e < RAD; ++e) root[e] = w2[2L * e * (T / RAD)];
    for (; j < nb; j += sj) {
        C2 a[RAD];
        a[0] = in[j * TS + c];
        if (k > 0) {
            const C2 w1 = w2[2L * k * tstep];
            C2 wr = w1;
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                a[r] = cmul(in[(j + r * nb) * TS + c], wr);
                if (r + 1 < RAD) wr = cmul(wr, w1);
            }
        } else {
#pragma unroll
            for (int r = 1; r < RAD; ++r) a[r] = in[(j + r * nb) * TS + c];
        }
        const int ob = jb * Ns * RAD + k;
        if (RAD == 2) {
            out[ob * TS + c] = cadd(a[0], a[1]);
            out[(ob + Ns) * TS + c] = csub(a[0], a[1]);
        } else if (RAD == 4) {
            const C2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
            const C2 s13 = cadd(a[1], a[3]), d13 = cmi(csub(a[1], a[3]));
            out[ob * TS + c] = cadd(s02, s13);
            out[(ob + Ns) * TS + c] = cadd(d02, d13);
            out[(ob + 2 * Ns) * TS + c] = csub(s02, s13);
            out[(ob + 3 * Ns) * TS + c] = csub(d02, d13);
        } else {
#pragma unroll
            for (int q = 0; q < RAD; ++q) {
                C2 s = a[0];
#pragma unroll
                for (int r = 1; r < RAD; ++r) s = cadd(s, cmul(a[r], root[(r * q) % RAD]));
                out[(ob + q * Ns) * TS + c] = s;
            }
        }
        k += sk;
        jb += sjb;
        if (k >= Ns) {
            k -= Ns;
            jb += 1;
        }
    }
}

// Full forward DFT of length T along the first index of buf (TS columns);
// returns the buffer holding the result.
template <typename R>
__device__ typename Cx<R>::T2* fft_tau(typename Cx<R>::T2* a, typename Cx<R>::T2* b,
                                       const typename Cx<R>::T2* __restrict__ w2, int T, int TS,
                                       const RadixPlan& plan)
{
    int Ns = 1;
    for (int s = 0; s < plan.n; ++s) {
        __syncthreads();
        switch (plan.r[s]) {
        case 2: stockham_pass<R, 2>(a, b, w2, T, TS, Ns); break;
        case 3: stockham_pass<R, 3>(a, b, w2, T, TS, Ns); break;
        case 4: stockham_pass<R, 4>(a, b, w2, T, TS, Ns); break;
        case 5: stockham_pass<R, 5>(a, b, w2, T, TS, Ns); break;
        default: stockham_pass<R, 7>(a, b, w2, T, TS, Ns); break;
        }
        Ns *= plan.r[s];
        typename Cx<R>::T2* t = a;
        a = b;
        b = t;
    }
    __syncthreads();
    return a;
}


// ---------------------------------------------------------------------------
// The same transform with the length T, the tile width TS and the block size
// NT known at compile time (the lengths of the configured workloads): the
// plan, the butterfly loops and every index division are resolved by the
// compiler. Same passes and twiddles as fft_tau.
// ---------------------------------------------------------------------------
struct PlanCT {
    int n;
    int r[16];
};

__host__ __device__ constexpr PlanCT plan_ct(int T)
{
    PlanCT p{0, {}};
    int t = T;
    const int rs[5] = {4, 2, 3, 5, 7};
    for (int k = 0; k < 5; ++k)
        while (t % rs[k] == 0 && p.n < 16) {
            p.r[p.n++] = rs[k];
            t /= rs[k];
        }
    if (t != 1) p.n = -1;
    return p;
}

template <typename R, int RAD, int T, int TS, int NT, int Ns>
__device__ __forceinline__ void stockham_pass_ct(const typename Cx<R>::T2* __restrict__ in,
                                                 typename Cx<R>::T2* __restrict__ out,
                                                 const typename Cx<R>::T2* __restrict__ w2)
{
    using C2 = typename Cx<R>::T2;
    static_assert(NT % TS == 0, "block size must be a multiple of the tile width");
    constexpr int nb = T / RAD;
    constexpr int SJ = NT / TS;
    constexpr int tstep = T / (Ns * RAD);
    const int c = threadIdx.x % TS;
    const int j0 = threadIdx.x / TS;
    C2 root[RAD];
#pragma unroll
    for (int e = 0; e < RAD; ++e) root[e] = w2[2 * e * (T / RAD)];
#pragma unroll
    for (int jj = 0; jj < (nb + SJ - 1) / SJ; ++jj) {
        const int j = j0 + jj * SJ;
        if (nb % SJ != 0 && j >= nb) break;
        const int k = j % Ns, jb = j / Ns;
        C2 a[RAD];
        a[0] = in[j * TS + c];
        if (Ns > 1 && k > 0) {
            const C2 w1 = w2[2 * k * tstep];
            C2 wr = w1;
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                a[r] = cmul(in[(j + r * nb) * TS + c], wr);
                if (r + 1 < RAD) wr = cmul(wr, w1);
            }
        } else {
#pragma unroll
            for (int r = 1; r < RAD; ++r) a[r] = in[(j + r * nb) * TS + c];
        }
        const int ob = jb * Ns * RAD + k;
        if constexpr (RAD == 2) {
            out[ob * TS + c] = cadd(a[0], a[1]);
            out[(ob + Ns) * TS + c] = csub(a[0], a[1]);
        } else if constexpr (RAD == 4) {
            const C2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
            const C2 s13 = cadd(a[1], a[3]), d13 = cmi(csub(a[1], a[3]));
            out[ob * TS + c] = cadd(s02, s13);
            out[(ob + Ns) * TS + c] = cadd(d02, d13);
            out[(ob + 2 * Ns) * TS + c] = csub(s02, s13);
            out[(ob + 3 * Ns) * TS + c] = csub(d02, d13);
        } else {
#pragma unroll
            for (int q = 0; q < RAD; ++q) {
                C2 sum = a[0];
#pragma unroll
                for (int r = 1; r < RAD; ++r) sum = cadd(sum, cmul(a[r], root[(r * q) % RAD]));
                out[(ob + q * Ns) * TS + c] = sum;
            }
        }
    }
}

template <typename R, int T, int TS, int NT, int S = 0, int Ns = 1>
__device__ __forceinline__ typename Cx<R>::T2* fft_tau_ct(typename Cx<R>::T2* a,
                                                          typename Cx<R>::T2* b,
                                                          const typename Cx<R>::T2* __restrict__ w2)
{
    constexpr PlanCT P = plan_ct(T);
    static_assert(P.n > 0, "length with a prime factor above 7");
    if constexpr (S < P.n) {
        constexpr int RAD = P.r[S];
        __syncthreads();
        stockham_pass_ct<R, RAD, T, TS, NT, Ns>(a, b, w2);
        return fft_tau_ct<R, T, TS, NT, S + 1, Ns * RAD>(b, a, w2);
    } else {
        __syncthreads();
        return a;
    }
}

// radix plan of a length (host): factors 4 first, then 2, 3, 5, 7; n = -1 if
// another prime factor remains
inline RadixPlan plan_of(int T)
{
    RadixPlan p;
    p.n = 0;
    int t = T;
    const int rs[5] = {4, 2, 3, 5, 7};
    for (int k = 0; k < 5; ++k)
        while (t % rs[k] == 0 && p.n < 16) {
            p.r[p.n++] = rs[k];
            t /= rs[k];
        }
    if (t != 1) p.n = -1;
    return p;
}

}  // namespace fft
}  // namespace hol
