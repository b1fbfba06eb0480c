// Checkerboard kinetic propagator C = C4 C3 C2 C1 (Sec. II D) on one tau
// slice of an L x L lattice spread over NW warps ("split" float4 layout,
// L = 32): lane (cx, rcl) of warp w of the group holds columns 4cx..4cx+3
// of the RT = L / (4 NW) rows starting at (4 w + rcl) RT. x-bonds are warp
// shuffles, y-bonds inside a lane's rows are register pairs, y-bonds between
// lanes are shuffles inside a warp and a shared-memory exchange between the
// warps of the group (one barrier per odd-y colour, double buffered). Bond
// factors are [[1, th], [th, 1]] with cosh folded into the diagonal, as in
// cb4.cuh.
#pragma once

#include "cb4.cuh"

namespace hol {

template <int L, int NW>
struct GeomS {
    static_assert(L == 32, "split layout: one warp spans a full row set only at L = 32");
    static constexpr int LR = L / 4;          // lanes per row segment
    static constexpr int RT = L / (4 * NW);   // rows per lane
    static_assert(RT >= 2 && RT % 2 == 0, "rows per lane must be even");
    int cx, rcl, rc, w, left, right, down, up;
    __device__ __forceinline__ GeomS()
    {
        const int lane = threadIdx.x & 31;
        w = (threadIdx.x >> 5) % NW;
        cx = lane % LR;
        rcl = lane / LR;
        rc = w * 4 + rcl;
        right = rcl * LR + (cx + 1 == LR ? 0 : cx + 1);
        left = rcl * LR + (cx == 0 ? LR - 1 : cx - 1);
        down = ((rcl + 1) & 3) * LR + cx;
        up = ((rcl + 3) & 3) * LR + cx;
    }
    __device__ __forceinline__ int off(int k) const { return (rc * RT + k) * L + 4 * cx; }
};

// Exchange scratch of one group: [2 buffers][NW warps][first, last row][LR].
template <int L, int NW>
struct SplitX {
    float4 b[2][NW][2][L / 4];
};

template <int RT>
__device__ __forceinline__ void cs_colour1(float4 (&c)[RT], float th)
{
#pragma unroll
    for (int k = 0; k < RT; ++k) {
        bond(c[k].x, c[k].y, th);
        bond(c[k].z, c[k].w, th);
    }
}

template <int L, int NW>
__device__ __forceinline__ void cs_colour2(float4 (&c)[GeomS<L, NW>::RT], const GeomS<L, NW>& g,
                                           float th)
{
#pragma unroll
    for (int k = 0; k < GeomS<L, NW>::RT; ++k) {
        const float rx = __shfl_sync(kFull, c[k].x, g.right);
        const float lw = __shfl_sync(kFull, c[k].w, g.left);
        bond(c[k].y, c[k].z, th);
        c[k].w = fmaf(th, rx, c[k].w);
        c[k].x = fmaf(th, lw, c[k].x);
    }
}

template <int RT>
__device__ __forceinline__ void cs_colour3(float4 (&c)[RT], float th)
{
#pragma unroll
    for (int k = 0; k < RT; k += 2) {
        bond(c[k].x, c[k + 1].x, th);
        bond(c[k].y, c[k + 1].y, th);
        bond(c[k].z, c[k + 1].z, th);
        bond(c[k].w, c[k + 1].w, th);
    }
}

// Odd y-bonds. All threads of the block take part (one barrier when NW > 1).
template <int L, int NW>
__device__ __forceinline__ void cs_colour4(float4 (&c)[GeomS<L, NW>::RT], const GeomS<L, NW>& g,
                                           float th, SplitX<L, NW>& xs, int& par)
{
    constexpr int RT = GeomS<L, NW>::RT;
    float4 dn = shfl4(c[0], g.down);       // partner of my last row
    float4 upv = shfl4(c[RT - 1], g.up);   // partner of my first row
    if constexpr (NW > 1) {
        if (g.rcl == 0) xs.b[par][g.w][0][g.cx] = c[0];
        if (g.rcl == 3) xs.b[par][g.w][1][g.cx] = c[RT - 1];
        __syncthreads();
        if (g.rcl == 3) dn = xs.b[par][g.w + 1 == NW ? 0 : g.w + 1][0][g.cx];
        if (g.rcl == 0) upv = xs.b[par][g.w == 0 ? NW - 1 : g.w - 1][1][g.cx];
        par ^= 1;
    }
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

// c <- C c
template <int L, int NW>
__device__ __forceinline__ void cs_apply(float4 (&c)[GeomS<L, NW>::RT], const GeomS<L, NW>& g,
                                         float th, SplitX<L, NW>& xs, int& par)
{
    cs_colour1<GeomS<L, NW>::RT>(c, th);
    cs_colour2<L, NW>(c, g, th);
    cs_colour3<GeomS<L, NW>::RT>(c, th);
    cs_colour4<L, NW>(c, g, th, xs, par);
}

// c <- C^T c
template <int L, int NW>
__device__ __forceinline__ void cs_apply_t(float4 (&c)[GeomS<L, NW>::RT], const GeomS<L, NW>& g,
                                           float th, SplitX<L, NW>& xs, int& par)
{
    cs_colour4<L, NW>(c, g, th, xs, par);
    cs_colour3<GeomS<L, NW>::RT>(c, th);
    cs_colour2<L, NW>(c, g, th);
    cs_colour1<GeomS<L, NW>::RT>(c, th);
}

}  // namespace hol
