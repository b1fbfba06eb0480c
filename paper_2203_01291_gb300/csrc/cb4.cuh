// Vectorised register layout of one tau slice for L divisible by 4 (L >= 8).
//
// A group of L lanes holds the slice: lane (cx, rc) of the group holds the
// four columns 4cx..4cx+3 (one float4) of a chunk of consecutive rows
// (cx < L/4, rc < 4). Every global access is a float4 of a row, so a slice
// costs about L/4 vector loads per lane instead of L scalar ones.
// Chunks: for L % 8 == 0 chunk rc holds the L/4 rows rc*L/4 .. rc*L/4 + L/4 - 1.
// For L % 8 == 4 (L/4 odd) an equal split would start every other chunk on an
// odd row; there the chunks alternate L/4 + 1 and L/4 - 1 rows (12: 4,2,4,2;
// 20: 6,4,6,4; 28: 8,6,8,6), so every chunk starts on an even row and holds an
// even number of rows. A lane keeps RT = L/4 + 1 register rows; a short chunk
// leaves its last two unused (never loaded or stored, and no lattice row
// ever reads them).
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
    static_assert(L % 4 == 0 && L >= 8 && L <= 32, "vector layout needs L % 4 == 0, 8 <= L <= 32");
    static constexpr int LR = L / 4;                  // lanes per row segment
    static constexpr bool kUneven = (L / 4) % 2 == 1;   // chunks of L/4 +- 1 rows
    static constexpr int RT = L / 4 + (kUneven ? 1 : 0);   // register rows per lane
    static constexpr int G = 32 / L;                  // slices per warp
    int g, cx, rc, left, right, down, up;
    bool shortc;   // the chunk holds RT - 2 rows (L % 8 == 4, odd rc; else false)
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
        shortc = kUneven && (rc & 1) != 0;
    }
    // first lattice row of this lane's chunk
    __device__ __forceinline__ int row0() const
    {
        if constexpr (kUneven) return (rc >> 1) * (L / 2) + (rc & 1) * (L / 4 + 1);
        return rc * RT;
    }
    // float offset of register row k of this lane inside a slice
    __device__ __forceinline__ int off(int k) const { return (row0() + k) * L + 4 * cx; }
    // register row k holds a lattice row (always, unless L % 8 == 4)
    __device__ __forceinline__ bool has(int k) const
    {
        if constexpr (kUneven) return k < RT - 2 || !shortc;
        return true;
    }
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
__device__ __forceinline__ void c4_colour1(float4 (&c)[Geom4<L>::RT], float th)
{
#pragma unroll
    for (int k = 0; k < Geom4<L>::RT; ++k) {
        bond(c[k].x, c[k].y, th);
        bond(c[k].z, c[k].w, th);
    }
}

template <int L>
__device__ __forceinline__ void c4_colour2(float4 (&c)[Geom4<L>::RT], const Geom4<L>& g, float th)
{
#pragma unroll
    for (int k = 0; k < Geom4<L>::RT; ++k) {
        const float rx = __shfl_sync(kFull, c[k].x, g.right);
        const float lw = __shfl_sync(kFull, c[k].w, g.left);
        bond(c[k].y, c[k].z, th);
        c[k].w = fmaf(th, rx, c[k].w);
        c[k].x = fmaf(th, lw, c[k].x);
    }
}

template <int L>
__device__ __forceinline__ void c4_colour3(float4 (&c)[Geom4<L>::RT], float th)
{
#pragma unroll
    for (int k = 0; k < Geom4<L>::RT; k += 2) {
        bond(c[k].x, c[k + 1].x, th);
        bond(c[k].y, c[k + 1].y, th);
        bond(c[k].z, c[k + 1].z, th);
        bond(c[k].w, c[k + 1].w, th);
    }
}

__device__ __forceinline__ void fma4_into(float4& a, float th, const float4& b)
{
    a.x = fmaf(th, b.x, a.x);
    a.y = fmaf(th, b.y, a.y);
    a.z = fmaf(th, b.z, a.z);
    a.w = fmaf(th, b.w, a.w);
}

__device__ __forceinline__ float4 sel4(bool p, const float4& a, const float4& b)
{
    return make_float4(p ? a.x : b.x, p ? a.y : b.y, p ? a.z : b.z, p ? a.w : b.w);
}

template <int L>
__device__ __forceinline__ void c4_colour4(float4 (&c)[Geom4<L>::RT], const Geom4<L>& g, float th)
{
    constexpr int RT = Geom4<L>::RT;
    if constexpr (!Geom4<L>::kUneven) {
        const float4 dn = shfl4(c[0], g.down);        // partner of my last row
        const float4 upv = shfl4(c[RT - 1], g.up);    // partner of my first row
#pragma unroll
        for (int k = 1; k + 1 < RT; k += 2) {
            bond(c[k].x, c[k + 1].x, th);
            bond(c[k].y, c[k + 1].y, th);
            bond(c[k].z, c[k + 1].z, th);
            bond(c[k].w, c[k + 1].w, th);
        }
        fma4_into(c[RT - 1], th, dn);
        fma4_into(c[0], th, upv);
    } else {
        // a long chunk's last row is register RT - 1, a short one's RT - 3;
        // the pairs below RT - 3 are interior in both
        const float4 dn = shfl4(c[0], g.down);
        const float4 upv = shfl4(sel4(g.shortc, c[RT - 3], c[RT - 1]), g.up);
#pragma unroll
        for (int k = 1; k + 1 < RT - 3; k += 2) {
            bond(c[k].x, c[k + 1].x, th);
            bond(c[k].y, c[k + 1].y, th);
            bond(c[k].z, c[k + 1].z, th);
            bond(c[k].w, c[k + 1].w, th);
        }
        // rows RT - 3 and RT - 2: a bond in a long chunk; in a short one
        // RT - 3 is the last row and pairs with the next chunk instead
        // (register RT - 2 is unused there)
        const float4 a = c[RT - 3];
        fma4_into(c[RT - 3], th, sel4(g.shortc, dn, c[RT - 2]));
        fma4_into(c[RT - 2], th, a);
        fma4_into(c[RT - 1], th, dn);   // (unused register in a short chunk)
        fma4_into(c[0], th, upv);
    }
}

// c <- C c (colour 1 first)
template <int L>
__device__ __forceinline__ void c4_apply(float4 (&c)[Geom4<L>::RT], const Geom4<L>& g, float th)
{
    c4_colour1<L>(c, th);
    c4_colour2<L>(c, g, th);
    c4_colour3<L>(c, th);
    c4_colour4<L>(c, g, th);
}

// c <- C^T c (colour 4 first)
template <int L>
__device__ __forceinline__ void c4_apply_t(float4 (&c)[Geom4<L>::RT], const Geom4<L>& g, float th)
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
