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

// twiddle w2[k] = exp(-i pi k / T), k < 2T
template <typename R>
__device__ __forceinline__ typename Cx<R>::T2 tw(const typename Cx<R>::T2* __restrict__ w2, long k,
                                                 int T)
{
    return w2[k % (2 * T)];
}

// One Stockham pass of radix RAD over TS columns: in[tau][c] -> out[.][c].
template <typename R, int RAD>
__device__ void stockham_pass(const typename Cx<R>::T2* __restrict__ in,
                              typename Cx<R>::T2* __restrict__ out,
                              const typename Cx<R>::T2* __restrict__ w2, int T, int TS, int Ns)
{
    using C2 = typename Cx<R>::T2;
    const int nb = T / RAD;
    for (int item = threadIdx.x; item < nb * TS; item += blockDim.x) {
        const int c = item % TS, j = item / TS;
        const int k = j % Ns;
        C2 a[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            C2 v = in[(j + r * nb) * TS + c];
            if (r > 0 && k > 0) {
                // exp(-2 pi i r k / (Ns RAD)) = w2[2 r k T / (Ns RAD)]
                v = cmul(v, tw<R>(w2, 2L * r * k * (T / (Ns * RAD)), T));
            }
            a[r] = v;
        }
        const int ob = (j / Ns) * Ns * RAD + k;
#pragma unroll
        for (int q = 0; q < RAD; ++q) {
            C2 s = a[0];
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                // exp(-2 pi i r q / RAD) = w2[2 (r q mod RAD) T / RAD]
                const int e = (r * q) % RAD;
                s = e == 0 ? cadd(s, a[r]) : cadd(s, cmul(a[r], tw<R>(w2, 2L * e * (T / RAD), T)));
            }
            out[(ob + q * Ns) * TS + c] = s;
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
