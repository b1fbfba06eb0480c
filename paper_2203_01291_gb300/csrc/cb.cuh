// Register-resident checkerboard propagator for one tau slice of the L x L
// lattice (Sec. II D "minimal split checkerboard", C = C4 C3 C2 C1).
//
// A lane group of L consecutive lanes holds one slice: lane ix holds the
// column x = ix, all L rows iy in registers c[iy]. The x-bonds (colours 1, 2)
// pair neighbouring lanes and are exchanged with one warp shuffle per row;
// the y-bonds (colours 3, 4) pair neighbouring registers of the same lane.
// No shared memory and no barriers are involved.
#pragma once

#include <cuda_runtime.h>

namespace hol {

constexpr unsigned kFull = 0xffffffffu;

// Lane-group geometry for side L: G = floor(32/L) groups per warp. Lanes
// beyond G*L shadow group 0 (same loads and arithmetic, never store).
template <int L>
struct LaneGeom {
    static constexpr int G = 32 / L;
    int g, ix, p1, p2;
    bool ok;
    __device__ __forceinline__ LaneGeom()
    {
        const int lane = threadIdx.x & 31;
        g = lane / L;
        ix = lane - g * L;
        ok = g < G;
        if (!ok) {
            g = 0;
            ix = lane - G * L;
        }
        const int base = g * L;
        p1 = base + (ix ^ 1);                                   // colour 1 partner
        p2 = base + ((ix & 1) ? (ix + 1 == L ? 0 : ix + 1)      // colour 2 partner
                              : (ix == 0 ? L - 1 : ix - 1));
    }
};

// Each bond factor [[cosh, sinh], [sinh, cosh]](dtau t) is applied as
// cosh * [[1, th], [th, 1]] with th = tanh(dtau t); the four factors cosh of
// the four colours are folded into the stored diagonal exp(-dtau V) (times
// cosh^4), so a bond costs one FMA per site.

// Bond [[1, th], [th, 1]] on (own, partner) across lanes.
template <typename R, int L>
__device__ __forceinline__ void cb_xbond(R (&c)[L], int partner, R th)
{
#pragma unroll
    for (int iy = 0; iy < L; ++iy) {
        const R o = __shfl_sync(kFull, c[iy], partner);
        c[iy] = fma(th, o, c[iy]);
    }
}

// Bond on register pairs (iy, iy+1 mod L), iy = P, P+2, ...
template <typename R, int L, int P>
__device__ __forceinline__ void cb_ybond(R (&c)[L], R th)
{
#pragma unroll
    for (int iy = P; iy < L; iy += 2) {
        const int j = (iy + 1) % L;
        const R a = c[iy], b = c[j];
        c[iy] = fma(th, b, a);
        c[j] = fma(th, a, b);
    }
}

// c <- C' c with C' = C4' C3' C2' C1' (colour 1 acts first), C = cosh^4 C'.
template <typename R, int L>
__device__ __forceinline__ void cb_apply(R (&c)[L], const LaneGeom<L>& g, R th)
{
    cb_xbond<R, L>(c, g.p1, th);
    cb_xbond<R, L>(c, g.p2, th);
    cb_ybond<R, L, 0>(c, th);
    cb_ybond<R, L, 1>(c, th);
}

// c <- C'^T c (colour 4 acts first).
template <typename R, int L>
__device__ __forceinline__ void cb_apply_t(R (&c)[L], const LaneGeom<L>& g, R th)
{
    cb_ybond<R, L, 1>(c, th);
    cb_ybond<R, L, 0>(c, th);
    cb_xbond<R, L>(c, g.p2, th);
    cb_xbond<R, L>(c, g.p1, th);
}

// ---------------------------------------------------------------------------
// Exact kinetic propagator exp(-dtau K). On the periodic L x L lattice K is a
// sum of commuting x and y hopping terms, so exp(-dtau K) = E (x) E with E =
// exp(dtau t A) for the adjacency A of a ring of L sites: a symmetric
// circulant, E[i][j] = e[d], d the ring distance of i and j (0..L/2). The
// host computes e[d] from the ring's spectrum 2 cos(2 pi k / L) and keeps the
// taps d <= D beyond which |e[d]| is below the rounding of the precision.
// ---------------------------------------------------------------------------
constexpr int kKinTaps = 17;   // L / 2 + 1 for L <= 32

template <typename R>
struct Kin {
    R th;             // checkerboard bond tanh(dtau t)
    int D;            // exact propagator: taps kept on each side of the centre
    R e[kKinTaps];    // exact propagator: e[0..D]
};

// c <- exp(-dtau K) c for the slice held by a lane group (x along the lanes,
// then y along the registers; E is symmetric, so this is also the transpose).
template <typename R, int L>
__device__ __forceinline__ void kin_exact(R (&c)[L], const LaneGeom<L>& g, const Kin<R>& k)
{
    const int base = g.g * L;
    R o[L];
#pragma unroll
    for (int iy = 0; iy < L; ++iy) o[iy] = k.e[0] * c[iy];
#pragma unroll
    for (int d = 1; d <= L / 2; ++d) {
        if (d <= k.D) {
            const int jp = base + (g.ix + d) % L;
            const int jm = base + (g.ix + L - d) % L;
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                R a = __shfl_sync(kFull, c[iy], jp);
                if (2 * d != L) a += __shfl_sync(kFull, c[iy], jm);
                o[iy] = fma(k.e[d], a, o[iy]);
            }
        }
    }
#pragma unroll
    for (int iy = 0; iy < L; ++iy) c[iy] = k.e[0] * o[iy];
#pragma unroll
    for (int d = 1; d <= L / 2; ++d) {
        if (d <= k.D) {
#pragma unroll
            for (int iy = 0; iy < L; ++iy) {
                R a = o[(iy + d) % L];
                if (2 * d != L) a += o[(iy + L - d) % L];
                c[iy] = fma(k.e[d], a, c[iy]);
            }
        }
    }
}

// c <- C c with the propagator the kernel was instantiated for.
template <typename R, int L, bool EX>
__device__ __forceinline__ void kin_apply(R (&c)[L], const LaneGeom<L>& g, const Kin<R>& k)
{
    if constexpr (EX)
        kin_exact<R, L>(c, g, k);
    else
        cb_apply<R, L>(c, g, k.th);
}

// c <- C^T c.
template <typename R, int L, bool EX>
__device__ __forceinline__ void kin_apply_t(R (&c)[L], const LaneGeom<L>& g, const Kin<R>& k)
{
    if constexpr (EX)
        kin_exact<R, L>(c, g, k);
    else
        cb_apply_t<R, L>(c, g, k.th);
}

// Warp-wide sum of a double, identical result in every lane (fixed order).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sum of a[0..n) by one full warp (lane-strided, then butterfly); every lane
// gets the same bits.
__device__ __forceinline__ double warp_sum_array(const double* __restrict__ a, int n)
{
    double s = 0.0;
    for (int k = (threadIdx.x & 31); k < n; k += 32) s += a[k];
    return warp_sum(s);
}

// Compensated float pair (a double-float): the value hi + lo with lo the
// rounding error of hi, kept by Knuth's TwoSum at every addition, so sums of
// FP32 terms keep about 48 significant bits while running on the FP32 pipes
// (on this GPU an FP64 instruction costs sixty-four times an FP32 one). The
// order of additions is fixed, so results are reproducible bit for bit.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return F2{s, e};
}
// x + y, renormalised so that |lo| stays below half an ulp of hi
__device__ __forceinline__ F2 f2_add(F2 x, F2 y)
{
    const F2 s = f2_two_sum(x.hi, y.hi);
    const float lo = s.lo + (x.lo + y.lo);
    const float hi = s.hi + lo;
    return F2{hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ F2 f2_add(F2 x, float y) { return f2_add(x, F2{y, 0.0f}); }
// Warp-wide sum, identical in every lane (fixed butterfly order).
__device__ __forceinline__ F2 f2_warp_sum(F2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const F2 y{__shfl_xor_sync(kFull, v.hi, o), __shfl_xor_sync(kFull, v.lo, o)};
        v = f2_add(v, y);
    }
    return v;
}
__device__ __forceinline__ double f2_to_double(F2 v) { return (double)v.hi + (double)v.lo; }

// Sum of a[0..n) by one full warp as warp_sum_array (same order, same bits),
// loading through L2 only: for partials written by other blocks of the same
// launch.
__device__ __forceinline__ double warp_sum_array_cg(const double* __restrict__ a, int n)
{
    double s = 0.0;
    for (int k = (threadIdx.x & 31); k < n; k += 32) s += __ldcg(a + k);
    return warp_sum(s);
}

// Sum `acc` over the L lanes of each group and store it for valid units.
template <int L>
__device__ __forceinline__ void group_store_sum(double acc, bool valid, double* __restrict__ dst)
{
    __shared__ double red[32 * 8];   // up to 8 warps per block
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    red[w * 32 + lane] = valid ? acc : 0.0;
    __syncwarp();
    const LaneGeom<L> geo;
    if (valid && geo.ix == 0) {
        double s = 0.0;
        for (int k = 0; k < L; ++k) s += red[w * 32 + geo.g * L + k];
        *dst = s;
    }
}

// The same for a compensated float pair: the sum over each group's L lanes
// (a butterfly when L is a power of two, else one lane summing the group in
// a fixed order), converted to FP64 once for the stored value.
template <int L>
__device__ __forceinline__ void group_store_sum(F2 acc, bool valid, double* __restrict__ dst)
{
    const LaneGeom<L> geo;
    if constexpr ((L & (L - 1)) == 0) {
        if (!valid) acc = F2{0.0f, 0.0f};
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            const F2 y{__shfl_xor_sync(kFull, acc.hi, o), __shfl_xor_sync(kFull, acc.lo, o)};
            acc = f2_add(acc, y);
        }
        if (valid && geo.ix == 0) *dst = f2_to_double(acc);
    } else {
        __shared__ float red_h[32 * 8], red_l[32 * 8];   // up to 8 warps per block
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        red_h[w * 32 + lane] = valid ? acc.hi : 0.0f;
        red_l[w * 32 + lane] = valid ? acc.lo : 0.0f;
        __syncwarp();
        if (valid && geo.ix == 0) {
            F2 t{0.0f, 0.0f};
            for (int k = 0; k < L; ++k) {
                const int j = w * 32 + geo.g * L + k;
                t = f2_add(t, F2{red_h[j], red_l[j]});
            }
            *dst = f2_to_double(t);
        }
    }
}

}  // namespace hol
