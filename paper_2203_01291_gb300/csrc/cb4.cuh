// Vectorised register layout of one tau slice for L divisible by 8.
//
// A group of L lanes holds the slice: lane (cx, rc) of the group holds the
// four columns 4cx..4cx+3 (one float4) of the L/4 rows rc*L/4 ..
// rc*L/4 + L/4 - 1 (cx < L/4, rc < 4). Every global access is a float4 of a
// row, so a slice costs L/4 vector loads per lane instead of L scalar ones.
// Checkerboard colours (C = C4 C3 C2 C1):
//   colour 1, x-bonds (even ix, ix+1): inside the float4;
//   colour 2, x-bonds (odd ix, ix+1):  (.y,.z) inside, (.w, right.x) and
//             (.x, left.w) by two shuffles per row;
//   colour 3, y-bonds (even iy, iy+1): register pairs;
//   colour 4, y-bonds (odd iy, iy+1):  register pairs, plus the chunk edges
//             (last row with the next chunk's first row) by shuffles.
#pragma once

#include "cb.cuh"

namespace hol {

template <int L>
struct Geom4 {
    static_assert(L % 8 == 0, "vector layout needs L divisible by 8");
    static constexpr int LR = L / 4;   // lanes per row segment
    static constexpr int RT = L / 4;   // rows per lane
    static constexpr int G = 32 / L;   // slices per warp
    int g, cx, rc, left, right, down, up;
    bool ok;
    __device__ __forceinline__ Geom4()
    {
        const int lane = threadIdx.x & 31;
        g = lane / L;
        int ls = lane - g * L;
        ok = g < G;
        if (!ok) {
            g = 0;
            ls = lane - G * L;
        }
        cx = ls % LR;
        rc = ls / LR;
        const int b = g * L;
        right = b + rc * LR + (cx + 1 == LR ? 0 : cx + 1);
        left = b + rc * LR + (cx == 0 ? LR - 1 : cx - 1);
        down = b + ((rc + 1) & 3) * LR + cx;
        up = b + ((rc + 3) & 3) * LR + cx;
    }
    // float offset of row k of this lane inside a slice
    __device__ __forceinline__ int off(int k) const { return (rc * RT + k) * L + 4 * cx; }
};

// bond [[1, th], [th, 1]] (cosh folded into the diagonal, see cb.cuh)
__device__ __forceinline__ void bond(float& a, float& b, float th)
{
    const float x = a, y = b;
    a = fmaf(th, y, x);
    b = fmaf(th, x, y);
}

__device__ __forceinline__ float4 shfl4(const float4& v, int src)
{
    float4 r;
    r.x = __shfl_sync(kFull, v.x, src);
    r.y = __shfl_sync(kFull, v.y, src);
    r.z = __shfl_sync(kFull, v.z, src);
    r.w = __shfl_sync(kFull, v.w, src);
    return r;
}

template <int L>
__device__ __forceinline__ void c4_colour1(float4 (&c)[L / 4], float th)
{
#pragma unroll
    for (int k = 0; k < L / 4; ++k) {
        bond(c[k].x, c[k].y, th);
        bond(c[k].z, c[k].w, th);
    }
}

template <int L>
__device__ __forceinline__ void c4_colour2(float4 (&c)[L / 4], const Geom4<L>& g, float th)
{
#pragma unroll
    for (int k = 0; k < L / 4; ++k) {
        const float rx = __shfl_sync(kFull, c[k].x, g.right);
        const float lw = __shfl_sync(kFull, c[k].w, g.left);
        bond(c[k].y, c[k].z, th);
        c[k].w = fmaf(th, rx, c[k].w);
        c[k].x = fmaf(th, lw, c[k].x);
    }
}

template <int L>
__device__ __forceinline__ void c4_colour3(float4 (&c)[L / 4], float th)
{
#pragma unroll
    for (int k = 0; k < L / 4; k += 2) {
        bond(c[k].x, c[k + 1].x, th);
        bond(c[k].y, c[k + 1].y, th);
        bond(c[k].z, c[k + 1].z, th);
        bond(c[k].w, c[k + 1].w, th);
    }
}

template <int L>
__device__ __forceinline__ void c4_colour4(float4 (&c)[L / 4], const Geom4<L>& g, float th)
{
    constexpr int RT = L / 4;
    const float4 dn = shfl4(c[0], g.down);        // partner of my last row
    const float4 upv = shfl4(c[RT - 1], g.up);    // partner of my first row
#pragma unroll
    for (int k = 1; k + 1 < RT; k += 2) {
        bond(c[k].x, c[k + 1].x, th);
        bond(c[k].y, c[k + 1].y, th);
        bond(c[k].z, c[k + 1].z, th);
        bond(c[k].w, c[k + 1].w, th);
    }
    c[RT - 1].x = fmaf(th, dn.x, c[RT - 1].x);
    c[RT - 1].y = fmaf(th, dn.y, c[RT - 1].y);
    c[RT - 1].z = fmaf(th, dn.z, c[RT - 1].z);
    c[RT - 1].w = fmaf(th, dn.w, c[RT - 1].w);
    c[0].x = fmaf(th, upv.x, c[0].x);
    c[0].y = fmaf(th, upv.y, c[0].y);
    c[0].z = fmaf(th, upv.z, c[0].z);
    c[0].w = fmaf(th, upv.w, c[0].w);
}

// c <- C c (colour 1 first)
template <int L>
__device__ __forceinline__ void c4_apply(float4 (&c)[L / 4], const Geom4<L>& g, float th)
{
    c4_colour1<L>(c, th);
    c4_colour2<L>(c, g, th);
    c4_colour3<L>(c, th);
    c4_colour4<L>(c, g, th);
}

// c <- C^T c (colour 4 first)
template <int L>
__device__ __forceinline__ void c4_apply_t(float4 (&c)[L / 4], const Geom4<L>& g, float th)
{
    c4_colour4<L>(c, g, th);
    c4_colour3<L>(c, th);
    c4_colour2<L>(c, g, th);
    c4_colour1<L>(c, th);
}

__device__ __forceinline__ float4 ld4(const float* __restrict__ p, long o)
{
    return *reinterpret_cast<const float4*>(p + o);
}
__device__ __forceinline__ void st4(float* __restrict__ p, long o, const float4& v)
{
    *reinterpret_cast<float4*>(p + o) = v;
}
__device__ __forceinline__ float4 fma4s(float a, const float4& x, const float4& y)
{
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

}  // namespace hol
