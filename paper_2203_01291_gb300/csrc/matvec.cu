// Fermion-matrix kernels in the float4, split and streaming layouts, the
// merged and fused one-kernel CG iterations, and the launch dispatch of all
// operator kernels (Eq. (M_def), Sec. II D). The scalar-layout kernels are
// in mvscalar.cuh.
#include "cb.cuh"
#include "cb4.cuh"
#include "cbs.cuh"
#include <atomic>

#include "internal.cuh"
#include "mvscalar.cuh"

namespace hol {
namespace {

// ---------------------------------------------------------------------------
// Same fused FP32 CG step in the float4 layout of cb4.cuh (L % 8 == 0).
// ---------------------------------------------------------------------------
// Ask L2 to fetch the 128-byte line of a slice that this lane covers
// (32 lanes x 128 B = one 4 KB slice; smaller slices are covered by fewer
// lanes), so that the later float4 loads of the slice hit L2.
template <int L>
__device__ __forceinline__ void prefetch_slice_l2(const float* base)
{
    constexpr int lines = (L * L * 4 + 127) / 128;
    const int lane = threadIdx.x & 31;
    for (int l = lane; l < lines; l += 32)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(base + l * 32));
}

template <int L>
__global__ void __launch_bounds__(128, 3) k_cg_mtm32_v4(const float* __restrict__ r,
                                                     const float* __restrict__ pold,
                                                     float* __restrict__ pnew,
                                                     float* __restrict__ q,
                                                     const float* __restrict__ ev, MvGeom gm,
                                                     const int* __restrict__ mask,
                                                     const double* __restrict__ rr_new_part,
                                                     const double* __restrict__ rr_old_part,
                                                     int rr_stride, int rr_n, int first,
                                                     double* __restrict__ pq_part, float th)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = L / 4;
    const Geom4<L> geo;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = (warp - rhs * gm.wpr) * Geom4<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N;

    const float bt = cg_beta(gm, rhs, first, rr_new_part, rr_old_part, rr_stride, rr_n);

    // the unit's later slices t0+1 .. t0+K go to L2 while the first ones compute
    if (geo.g == 0 || Geom4<L>::G == 1) {
        for (int s = 1; s <= gm.K; ++s) {
            int tq = t0 + s;
            if (tq >= gm.T) tq -= gm.T;
            prefetch_slice_l2<L>(r + base + (long)tq * N);
            if (!first) prefetch_slice_l2<L>(pold + base + (long)tq * N);
        }
    }
    float4 W[RT], X[RT], P[RT], Y[RT];
    {
        const int tm = (t0 == 0) ? gm.T - 1 : t0 - 1;
        const long o = base + (long)tm * N;
#pragma unroll
        for (int k = 0; k < RT; ++k) Y[k] = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(r, o + geo.off(k)));
        c4_apply<L>(Y, geo, th);
    }
    {
        const long o = base + (long)t0 * N;
        const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(r, o + geo.off(k)));
            if (valid && pnew != nullptr) st4(pnew, o + geo.off(k), pv);
            X[k] = pv;
            float4 d = ld4(ev, (long)t0 * N + geo.off(k));
            W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                               fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
        }
        c4_apply<L>(X, geo, th);
    }
    F2 acc{0.0f, 0.0f};   // compensated float pair (see cb.cuh)
    for (int s = 0; s < gm.K; ++s) {
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
        const long op = base + (long)tp * N;
        const float sgp = (tp == 0) ? 1.0f : -1.0f;
        const bool own = valid && (s + 1 < gm.K) && pnew != nullptr;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = fma4s(bt, ld4(pold, op + geo.off(k)), ld4(r, op + geo.off(k)));
            if (own) st4(pnew, op + geo.off(k), pv);
            P[k] = pv;
            float4 d = ld4(ev, (long)tp * N + geo.off(k));
            d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
            X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                               fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
            Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
        }
        c4_apply<L>(P, geo, th);
        c4_apply_t<L>(Y, geo, th);
        const long o = base + (long)tau * N;
        float part = 0.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            if (valid)
                st4(q, o + geo.off(k), make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y,
                                                   W[k].z + Y[k].z, W[k].w + Y[k].w));
            part = fmaf(W[k].x, W[k].x, part);
            part = fmaf(W[k].y, W[k].y, part);
            part = fmaf(W[k].z, W[k].z, part);
            part = fmaf(W[k].w, W[k].w, part);
            W[k] = X[k];
            X[k] = P[k];
        }
        acc = f2_add(acc, part);
    }
    if (pq_part != nullptr) {
        group_store_sum<L>(acc, valid, pq_part + (long)rhs * gm.pstride + run);
        cg_alpha_epilogue(gm, rhs, pq_part, rr_new_part, rr_stride, rr_n);
    }
}


// ---------------------------------------------------------------------------
// Float4 fused CG step with the r, p_old and expV rows of the next tau
// slice prefetched into a per-lane shared-memory ring by cp.async (16-byte
// async copies, two stages), so the global loads of slice tau+1 are in
// flight while slice tau is computed. Each lane copies and later reads only its own
// slots, so cp.async.wait_group is the only synchronisation needed. Also
// built for L % 8 == 4, where a lane's row chunk may leave its last two
// register rows unused (cb4.cuh): those rows are never copied, stored or
// summed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory"); }

template <int L, int S>
__global__ void __launch_bounds__(128, 3) k_cg_mtm32_v4a(const float* __restrict__ r,
                                                         const float* __restrict__ pold,
                                                         float* __restrict__ pnew,
                                                         float* __restrict__ q,
                                                         const float* __restrict__ ev, MvGeom gm,
                                                         const int* __restrict__ mask,
                                                         const double* __restrict__ rr_new_part,
                                                         const double* __restrict__ rr_old_part,
                                                         int rr_stride, int rr_n, int first,
                                                         double* __restrict__ pq_part, float th)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = Geom4<L>::RT;   // L/4 rows, L/4 + 1 for L % 8 == 4 (see cb4.cuh)
    extern __shared__ __align__(16) float4 ring[];   // [warp][slot][array: r, p_old, expV][RT][32]
    const Geom4<L> geo;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* my = ring + (long)wib * (S * 3 * RT * 32);
    auto slot_ptr = [&](int slot, int arr, int k) -> float4* {
        return my + ((slot * 3 + arr) * RT + k) * 32 + lane;
    };
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = (warp - rhs * gm.wpr) * Geom4<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N;
    // slice sequence: j = 0 -> t0-1 (halo), j = 1.. -> t0, t0+1, ..., t0+K
    auto seq = [&](int j) -> int {
        int t = t0 - 1 + j;
        if (t < 0) t += gm.T;
        if (t >= gm.T) t -= gm.T;
        return t;
    };
    const int last = gm.K + 1;   // index of the last slice in the sequence
    // slice j goes to slot j % S; the copy of slice j + S - 1 is issued just
    // before slice j is waited for (its slot held slice j - 1, already read)
    auto issue = [&](int j) {
        if (j <= last) {
            const int t = seq(j);
            const long o = base + (long)t * N;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                if (!geo.has(k)) continue;   // unused register row (short chunk)
                cp_async16(slot_ptr(j % S, 0, k), r + o + geo.off(k));
                cp_async16(slot_ptr(j % S, 1, k), pold + o + geo.off(k));
                if (j > 0) cp_async16(slot_ptr(j % S, 2, k), ev + (long)t * N + geo.off(k));
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < S - 1; ++j) issue(j);

    const float bt = cg_beta(gm, rhs, first, rr_new_part, rr_old_part, rr_stride, rr_n);

    float4 W[RT], X[RT], P[RT], Y[RT];
    issue(S - 1);
    cp_async_wait<S - 1>();   // slice j = 0 has landed
#pragma unroll
    for (int k = 0; k < RT; ++k) Y[k] = fma4s(bt, *slot_ptr(0, 1, k), *slot_ptr(0, 0, k));
    c4_apply<L>(Y, geo, th);
    issue(S);
    cp_async_wait<S - 1>();   // slice j = 1 (t0)
    {
        const long o = base + (long)t0 * N;
        const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = fma4s(bt, *slot_ptr(1 % S, 1, k), *slot_ptr(1 % S, 0, k));
            if (valid && pnew != nullptr && geo.has(k)) st4(pnew, o + geo.off(k), pv);
            X[k] = pv;
            const float4 d = *slot_ptr(1 % S, 2, k);
            W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                               fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
        }
        c4_apply<L>(X, geo, th);
    }
    F2 acc{0.0f, 0.0f};   // compensated float pair (see cb.cuh)
    for (int s = 0; s < gm.K; ++s) {
        const int j = s + 2;             // slice t0 + 1 + s
        issue(j + S - 1);
        cp_async_wait<S - 1>();
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
        const long op = base + (long)tp * N;
        const float sgp = (tp == 0) ? 1.0f : -1.0f;
        const bool own = valid && (s + 1 < gm.K) && pnew != nullptr;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = fma4s(bt, *slot_ptr(j % S, 1, k), *slot_ptr(j % S, 0, k));
            if (own && geo.has(k)) st4(pnew, op + geo.off(k), pv);
            P[k] = pv;
            float4 d = *slot_ptr(j % S, 2, k);
            d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
            X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                               fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
            Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
        }
        c4_apply<L>(P, geo, th);
        c4_apply_t<L>(Y, geo, th);
        const long o = base + (long)tau * N;
        float part = 0.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            if (valid && geo.has(k))
                st4(q, o + geo.off(k), make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y,
                                                   W[k].z + Y[k].z, W[k].w + Y[k].w));
            if (geo.has(k)) {
                part = fmaf(W[k].x, W[k].x, part);
                part = fmaf(W[k].y, W[k].y, part);
                part = fmaf(W[k].z, W[k].z, part);
                part = fmaf(W[k].w, W[k].w, part);
            }
            W[k] = X[k];
            X[k] = P[k];
        }
        acc = f2_add(acc, part);
    }
    cp_async_wait<0>();
    if (pq_part != nullptr) {
        group_store_sum<L>(acc, valid, pq_part + (long)rhs * gm.pstride + run);
        cg_alpha_epilogue(gm, rhs, pq_part, rr_new_part, rr_stride, rr_n);
    }
}


// ---------------------------------------------------------------------------
// Streaming float4 fused CG step: a resident set of warps walks the units
// (grid stride) and keeps a ring of S slice stages (r and p_old rows of one
// tau slice per stage) in flight with cp.async across unit boundaries, so the
// next unit's slices load while the current one computes. Each lane copies
// and reads only its own ring slots (no barriers).
// ---------------------------------------------------------------------------
template <int L, int S>
__global__ void __launch_bounds__(128, 2) k_cg_mtm32_v4s(const float* __restrict__ r,
                                                        const float* __restrict__ pold,
                                                        float* __restrict__ pnew,
                                                        float* __restrict__ q,
                                                        const float* __restrict__ ev, MvGeom gm,
                                                        const int* __restrict__ mask,
                                                        const double* __restrict__ rr_new_part,
                                                        const double* __restrict__ rr_old_part,
                                                        int rr_stride, int rr_n, int first,
                                                        double* __restrict__ pq_part, float th,
                                                        int total_warps)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = L / 4;
    extern __shared__ __align__(16) float4 ring[];   // [warp][stage][array][RT][32]
    const Geom4<L> geo;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* my = ring + (long)wib * (S * 2 * RT * 32);
    auto slot = [&](int st, int arr, int k) -> float4* {
        return my + ((st * 2 + arr) * RT + k) * 32 + lane;
    };
    const int warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw_units = gm.wpr * gm.n_rhs;              // warp-units in the launch
    const int rounds = (nw_units - warp0 + total_warps - 1) / total_warps;
    const int per = gm.K + 2;                            // slices per unit
    const int npos = rounds * per;
    // position -> (round, slice index j in the unit)
    auto unit_of = [&](int rd, int& rhs, int& run) {
        const int w = warp0 + rd * total_warps;
        rhs = w / gm.wpr;
        run = (w - rhs * gm.wpr) * Geom4<L>::G + geo.g;
    };
    auto issue = [&](int pos) {
        if (pos < npos) {
            const int rd = pos / per, j = pos - rd * per;
            int rhs, run;
            unit_of(rd, rhs, run);
            const bool act = (mask == nullptr || mask[rhs] != 0);
            if (act) {
                const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
                int t = t0 - 1 + j;
                if (t < 0) t += gm.T;
                if (t >= gm.T) t -= gm.T;
                const long o = (long)rhs * gm.T * N + (long)t * N;
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    cp_async16(slot(pos % S, 0, k), r + o + geo.off(k));
                    cp_async16(slot(pos % S, 1, k), (first ? r : pold) + o + geo.off(k));
                }
            }
        }
        cp_async_commit();
    };
    for (int p = 0; p < S - 1; ++p) issue(p);
    int pos = 0;
    for (int rd = 0; rd < rounds; ++rd) {
        int rhs, run;
        unit_of(rd, rhs, run);
        const bool act = (mask == nullptr || mask[rhs] != 0);
        if (!act) {   // the ring still advances over this unit's (empty) stages
            for (int j = 0; j < per; ++j, ++pos) {
                issue(pos + S - 1);
                cp_async_wait<S - 1>();
            }
            continue;
        }
        const bool valid = geo.ok && run < gm.nrun;
        const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
        const long base = (long)rhs * gm.T * N;
        float bt = 0.0f;
        if (!first) {
            const double rn = warp_sum_array(rr_new_part + (long)rhs * rr_stride, rr_n);
            const double ro = warp_sum_array(rr_old_part + (long)rhs * rr_stride, rr_n);
            bt = (float)cg_ratio(rn, ro);
        }
        float4 W[RT], X[RT], P[RT], Y[RT];
        issue(pos + S - 1);
        cp_async_wait<S - 1>();
#pragma unroll
        for (int k = 0; k < RT; ++k)
            Y[k] = fma4s(bt, *slot(pos % S, 1, k), *slot(pos % S, 0, k));
        c4_apply<L>(Y, geo, th);
        ++pos;
        issue(pos + S - 1);
        cp_async_wait<S - 1>();
        {
            const long o = base + (long)t0 * N;
            const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                const float4 pv = fma4s(bt, *slot(pos % S, 1, k), *slot(pos % S, 0, k));
                if (valid && pnew != nullptr) st4(pnew, o + geo.off(k), pv);
                X[k] = pv;
                const float4 d = ld4(ev, (long)t0 * N + geo.off(k));
                W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                                   fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
            }
            c4_apply<L>(X, geo, th);
        }
        ++pos;
        F2 acc{0.0f, 0.0f};   // compensated float pair (see cb.cuh)
        for (int s = 0; s < gm.K; ++s, ++pos) {
            issue(pos + S - 1);
            cp_async_wait<S - 1>();
            const int tau = t0 + s;
            const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
            const long op = base + (long)tp * N;
            const float sgp = (tp == 0) ? 1.0f : -1.0f;
            const bool own = valid && (s + 1 < gm.K) && pnew != nullptr;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                const float4 pv = fma4s(bt, *slot(pos % S, 1, k), *slot(pos % S, 0, k));
                if (own) st4(pnew, op + geo.off(k), pv);
                P[k] = pv;
                float4 d = ld4(ev, (long)tp * N + geo.off(k));
                d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
                X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                                   fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
                Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
            }
            c4_apply<L>(P, geo, th);
            c4_apply_t<L>(Y, geo, th);
            const long o = base + (long)tau * N;
            float part = 0.0f;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                if (valid)
                    st4(q, o + geo.off(k), make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y,
                                                       W[k].z + Y[k].z, W[k].w + Y[k].w));
                part = fmaf(W[k].x, W[k].x, part);
                part = fmaf(W[k].y, W[k].y, part);
                part = fmaf(W[k].z, W[k].z, part);
                part = fmaf(W[k].w, W[k].w, part);
                W[k] = X[k];
                X[k] = P[k];
            }
            acc = f2_add(acc, part);
        }
        if (pq_part != nullptr) group_store_sum<L>(acc, valid, pq_part + (long)rhs * gm.pstride + run);
    }
    cp_async_wait<0>();
}


// ---------------------------------------------------------------------------
// Merged CG iteration (single reduction per iteration, Chronopoulos-Gear
// recurrences): with w = A r and s = A p for A = M^T M,
//   beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//   p = r + beta p_old,  s = w + beta s_old,  x += alpha p,  r' = r - alpha s,
//   w' = A r',  gamma' = r'.r',  delta' = r'.w' = |M r'|^2.
// r' is formed on the fly for the unit's slices and its two tau neighbours,
// so the whole iteration is one pass over the vectors (float4 layout).
// mode 1 (after a reliable update, with s_old = A p_old recomputed):
//   beta = -rho / pi (p re-conjugated against the new r),
//   alpha = gamma / (delta + 2 beta rho + beta^2 pi), rho = r.s_old,
//   pi = p_old.s_old; mode 2 (start): beta = 0, alpha = gamma / delta.
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(128, 3) k_cg_merged(
    const float* __restrict__ r, const float* __restrict__ w, const float* __restrict__ pold,
    const float* __restrict__ sold, float* __restrict__ e, float* __restrict__ pnew,
    float* __restrict__ snew, float* __restrict__ rnew, float* __restrict__ wnew,
    const float* __restrict__ ev, MvGeom gm, const int* __restrict__ mask, MergedScal sc,
    float th)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = L / 4;
    const Geom4<L> geo;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int wr = warp - rhs * gm.wpr;
    const int run = wr * Geom4<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N;

    // scalars: every warp forms them from the same partials in the same order
    const double* si = sc.slot_in + rhs * 4;
    const int mode = (int)si[2];
    const double dl = warp_sum_array(sc.d_in + (long)rhs * gm.pstride, gm.nrun);
    double ga, be, al;
    if (mode == 0) {
        ga = warp_sum_array(sc.g_in + (long)rhs * gm.pstride, gm.nrun);
        be = cg_ratio(ga, si[1]);
        al = cg_ratio(ga, dl - be * cg_ratio(ga, si[0]));
    } else {
        ga = warp_sum_array(sc.gr + (long)rhs * kRedStride, sc.e_n);
        if (mode == 1) {   // p_old re-conjugated against the new r
            const double pi = warp_sum_array(sc.pi + (long)rhs * gm.pstride, gm.nrun);
            const double rho = warp_sum_array(sc.rho + (long)rhs * kRedStride, sc.e_n);
            be = cg_ratio(-rho, pi);
            al = cg_ratio(ga, dl + 2.0 * be * rho + be * be * pi);
        } else {
            be = 0.0;
            al = cg_ratio(ga, dl);
        }
    }
    if (wr == 0 && (threadIdx.x & 31) == 0) {
        sc.slot_out[rhs * 4 + 0] = al;
        sc.slot_out[rhs * 4 + 1] = ga;
        sc.slot_out[rhs * 4 + 2] = 0.0;
    }
    const float a = (float)al, b = (float)be, ap = (float)si[0];
    const bool old = (mode != 2);
    const int fold = sc.fold;

    if (geo.g == 0 || Geom4<L>::G == 1) {
        for (int s = 1; s <= gm.K; ++s) {
            int tq = t0 + s;
            if (tq >= gm.T) tq -= gm.T;
            const long o = base + (long)tq * N;
            prefetch_slice_l2<L>(r + o);
            prefetch_slice_l2<L>(w + o);
            if (old) {
                prefetch_slice_l2<L>(sold + o);
                prefetch_slice_l2<L>(pold + o);
            }
            if (fold) prefetch_slice_l2<L>(e + o);
        }
    }
    // r' of slice t (row k of this lane); own slices also store p, s, r', x
    auto step = [&](long o, bool own, double& gacc) -> float4 {
        const float4 rv = ld4(r, o);
        float4 sv = ld4(w, o);
        if (old) sv = fma4s(b, ld4(sold, o), sv);
        const float4 rn = fma4s(-a, sv, rv);
        if (own) {
            float4 pv = rv, po = make_float4(0.f, 0.f, 0.f, 0.f);
            if (old) {
                po = ld4(pold, o);
                pv = fma4s(b, po, rv);
            }
            st4(pnew, o, pv);
            st4(snew, o, sv);
            st4(rnew, o, rn);
            if (fold) {
                float4 xv = ld4(e, o);
                if (fold == 2) xv = fma4s(ap, po, xv);
                st4(e, o, fma4s(a, pv, xv));
            }
            gacc += (double)(rn.x * rn.x + rn.y * rn.y + rn.z * rn.z + rn.w * rn.w);
        }
        return rn;
    };

    double gacc = 0.0;
    float4 W[RT], X[RT], P[RT], Y[RT];
    {
        const int tm = (t0 == 0) ? gm.T - 1 : t0 - 1;
        const long o = base + (long)tm * N;
#pragma unroll
        for (int k = 0; k < RT; ++k) Y[k] = step(o + geo.off(k), false, gacc);
        c4_apply<L>(Y, geo, th);
    }
    {
        const long o = base + (long)t0 * N;
        const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = step(o + geo.off(k), valid, gacc);
            X[k] = pv;
            const float4 d = ld4(ev, (long)t0 * N + geo.off(k));
            W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                               fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
        }
        c4_apply<L>(X, geo, th);
    }
    double acc = 0.0;
    for (int s = 0; s < gm.K; ++s) {
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
        const long op = base + (long)tp * N;
        const float sgp = (tp == 0) ? 1.0f : -1.0f;
        const bool own = valid && (s + 1 < gm.K);
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = step(op + geo.off(k), own, gacc);
            P[k] = pv;
            float4 d = ld4(ev, (long)tp * N + geo.off(k));
            d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
            X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                               fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
            Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
        }
        c4_apply<L>(P, geo, th);
        c4_apply_t<L>(Y, geo, th);
        const long o = base + (long)tau * N;
        float part = 0.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            if (valid)
                st4(wnew, o + geo.off(k), make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y,
                                                      W[k].z + Y[k].z, W[k].w + Y[k].w));
            part = fmaf(W[k].x, W[k].x, part);
            part = fmaf(W[k].y, W[k].y, part);
            part = fmaf(W[k].z, W[k].z, part);
            part = fmaf(W[k].w, W[k].w, part);
            W[k] = X[k];
            X[k] = P[k];
        }
        acc += (double)part;
    }
    group_store_sum<L>(acc, valid, sc.d_out + (long)rhs * gm.pstride + run);
    __syncwarp();
    group_store_sum<L>(gacc, valid, sc.g_out + (long)rhs * gm.pstride + run);
}


// ---------------------------------------------------------------------------
// Fused FP32 CG step in the split float4 layout of cbs.cuh (L = 32): one
// block of NW warps per unit of K slices, so each lane holds L / (4 NW) rows
// of a slice and the per-slice chain of dependent work is NW times shorter
// than with one warp per slice. Same arithmetic as k_cg_mtm32_v4.
// ---------------------------------------------------------------------------
template <int L, int NW>
__global__ void __launch_bounds__(32 * NW) k_cg_mtm32_split(const float* __restrict__ r,
                                                           const float* __restrict__ pold,
                                                           float* __restrict__ pnew,
                                                           float* __restrict__ q,
                                                           const float* __restrict__ ev,
                                                           MvGeom gm,
                                                           const int* __restrict__ mask,
                                                           const double* __restrict__ rr_new_part,
                                                           const double* __restrict__ rr_old_part,
                                                           int rr_stride, int rr_n, int first,
                                                           double* __restrict__ pq_part, float th)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = GeomS<L, NW>::RT;
    __shared__ SplitX<L, NW> xs;
    __shared__ double red[NW];
    __shared__ float s_bt;
    const GeomS<L, NW> geo;
    const int unit = blockIdx.x;
    const int rhs = unit / gm.nrun;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = unit - rhs * gm.nrun;
    const int t0 = run * gm.K;
    const long base = (long)rhs * gm.T * N;
    int par = 0;

    // the unit's later slices go to L2 while beta is formed
    if (threadIdx.x < 32) {
        for (int s = 1; s <= gm.K; ++s) {
            int tq = t0 + s;
            if (tq >= gm.T) tq -= gm.T;
            prefetch_slice_l2<L>(r + base + (long)tq * N);
            if (!first) prefetch_slice_l2<L>(pold + base + (long)tq * N);
        }
        float bt = 0.0f;
        if (!first) {
            const double rn = warp_sum_array(rr_new_part + (long)rhs * rr_stride, rr_n);
            const double ro = warp_sum_array(rr_old_part + (long)rhs * rr_stride, rr_n);
            bt = (float)cg_ratio(rn, ro);
        }
        if (threadIdx.x == 0) s_bt = bt;
    }
    __syncthreads();
    const float bt = s_bt;

    float4 W[RT], X[RT], P[RT], Y[RT];
    {
        const int tm = (t0 == 0) ? gm.T - 1 : t0 - 1;
        const long o = base + (long)tm * N;
#pragma unroll
        for (int k = 0; k < RT; ++k) Y[k] = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(r, o + geo.off(k)));
        cs_apply<L, NW>(Y, geo, th, xs, par);
    }
    {
        const long o = base + (long)t0 * N;
        const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(r, o + geo.off(k)));
            if (pnew != nullptr) st4(pnew, o + geo.off(k), pv);
            X[k] = pv;
            const float4 d = ld4(ev, (long)t0 * N + geo.off(k));
            W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                               fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
        }
        cs_apply<L, NW>(X, geo, th, xs, par);
    }
    double acc = 0.0;
    for (int s = 0; s < gm.K; ++s) {
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
        const long op = base + (long)tp * N;
        const float sgp = (tp == 0) ? 1.0f : -1.0f;
        const bool own = (s + 1 < gm.K) && pnew != nullptr;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 pv = fma4s(bt, ld4(pold, op + geo.off(k)), ld4(r, op + geo.off(k)));
            if (own) st4(pnew, op + geo.off(k), pv);
            P[k] = pv;
            float4 d = ld4(ev, (long)tp * N + geo.off(k));
            d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
            X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                               fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
            Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
        }
        cs_apply<L, NW>(P, geo, th, xs, par);
        cs_apply_t<L, NW>(Y, geo, th, xs, par);
        const long o = base + (long)tau * N;
        float part = 0.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            st4(q, o + geo.off(k), make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y,
                                               W[k].z + Y[k].z, W[k].w + Y[k].w));
            part = fmaf(W[k].x, W[k].x, part);
            part = fmaf(W[k].y, W[k].y, part);
            part = fmaf(W[k].z, W[k].z, part);
            part = fmaf(W[k].w, W[k].w, part);
            W[k] = X[k];
            X[k] = P[k];
        }
        acc += (double)part;
    }
    if (pq_part != nullptr) {
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += red[w];
            pq_part[(long)rhs * gm.pstride + run] = t;
        }
    }
}


// ---------------------------------------------------------------------------
// Fused CG iteration (float4 layout, cp.async ring of r, q, p, expV, x): the
// vector update of iteration i and the operator of iteration i + 1 in one
// pass. From the unit partials of the previous pass (g = r.r, pq = p.q,
// rq = r.q, qq = q.q, all of iteration i):
//   alpha = g / pq,  g' = |r - alpha q|^2 = g - 2 alpha rq + alpha^2 qq,
//   beta = g' / g,   r' = r - alpha q,  p' = r' + beta p,  x += alpha p,
//   q' = M^T M p',   and the new partials g' (of the stored r'), p'.q',
//   r'.q', q'.q'.
// g' is the exact expansion of |r'|^2, so no conjugacy is assumed; r' is
// formed on the fly for the unit's slices and both tau neighbours.
// ---------------------------------------------------------------------------
struct FusedBanks {
    const double* g;    // unit partials in (stride pstride, nrun per rhs)
    const double* pq;
    const double* rq;
    const double* qq;
    double* g_out;
    double* pq_out;
    double* rq_out;
    double* qq_out;
};

template <int L>
__global__ void __launch_bounds__(128, 2) k_cg_fused(const float* __restrict__ r,
                                                     const float* __restrict__ q,
                                                     const float* __restrict__ pold,
                                                     float* __restrict__ x,
                                                     float* __restrict__ rnew,
                                                     float* __restrict__ pnew,
                                                     float* __restrict__ qnew,
                                                     const float* __restrict__ ev, MvGeom gm,
                                                     const int* __restrict__ mask, FusedBanks bk,
                                                     float th)
{
    pdl_wait();      // inputs come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = L / 4;
    constexpr int S = 2;
    constexpr int NA = 5;   // ring arrays: r, q, p, expV, x
    // [warp][ring: slot][array][RT][32] then [warp][r' of the slice awaiting output][RT][32]
    extern __shared__ __align__(16) float4 ring[];
    const Geom4<L> geo;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* my = ring + (long)wib * ((S * NA + 1) * RT * 32);
    auto slot_ptr = [&](int slot, int arr, int k) -> float4* {
        return my + ((slot * NA + arr) * RT + k) * 32 + lane;
    };
    auto rbuf = [&](int k) -> float4* { return my + ((S * NA) * RT + k) * 32 + lane; };
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = (warp - rhs * gm.wpr) * Geom4<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N;
    auto seq = [&](int j) -> int {
        int t = t0 - 1 + j;
        if (t < 0) t += gm.T;
        if (t >= gm.T) t -= gm.T;
        return t;
    };
    const int last = gm.K + 1;
    auto issue = [&](int j) {
        if (j <= last) {
            const int t = seq(j);
            const long o = base + (long)t * N;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                cp_async16(slot_ptr(j % S, 0, k), r + o + geo.off(k));
                cp_async16(slot_ptr(j % S, 1, k), q + o + geo.off(k));
                cp_async16(slot_ptr(j % S, 2, k), pold + o + geo.off(k));
                if (j > 0) cp_async16(slot_ptr(j % S, 3, k), ev + (long)t * N + geo.off(k));
                if (j > 0 && j <= gm.K) cp_async16(slot_ptr(j % S, 4, k), x + o + geo.off(k));
            }
        }
        cp_async_commit();
    };
    issue(0);

    // scalars of iteration i (every warp forms them from the same partials)
    const long pb = (long)rhs * gm.pstride;
    const double g = warp_sum_array(bk.g + pb, gm.nrun);
    const double pq = warp_sum_array(bk.pq + pb, gm.nrun);
    const double rq = warp_sum_array(bk.rq + pb, gm.nrun);
    const double qq = warp_sum_array(bk.qq + pb, gm.nrun);
    const double ad = cg_ratio(g, pq);
    double gn = g - 2.0 * ad * rq + ad * ad * qq;
    if (!(gn > 0.0)) gn = 0.0;   // roundoff below zero: restart the direction (beta = 0)
    const float a = (float)ad, bt = (float)cg_ratio(gn, g);

    // r' and p' of ring slot `sl` (row k)
    auto rn_of = [&](int sl, int k) -> float4 {
        return fma4s(-a, *slot_ptr(sl, 1, k), *slot_ptr(sl, 0, k));
    };

    F2 gacc{0.0f, 0.0f}, pacc{0.0f, 0.0f}, rqacc{0.0f, 0.0f}, qqacc{0.0f, 0.0f};   // see cb.cuh
    float4 W[RT], X[RT], P[RT], Y[RT];
    issue(1);
    cp_async_wait<1>();   // slice j = 0 (halo t0 - 1)
#pragma unroll
    for (int k = 0; k < RT; ++k) Y[k] = fma4s(bt, *slot_ptr(0, 2, k), rn_of(0, k));
    c4_apply<L>(Y, geo, th);
    issue(2);
    cp_async_wait<1>();   // slice j = 1 (t0)
    {
        const long o = base + (long)t0 * N;
        const float sg = (t0 == 0) ? 1.0f : -1.0f;
        float gp = 0.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 rv = rn_of(1, k);
            const float4 po = *slot_ptr(1, 2, k);
            const float4 pv = fma4s(bt, po, rv);
            if (valid) {
                st4(rnew, o + geo.off(k), rv);
                st4(pnew, o + geo.off(k), pv);
                st4(x, o + geo.off(k), fma4s(a, po, *slot_ptr(1, 4, k)));
            }
            *rbuf(k) = rv;
            gp = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, gp))));
            X[k] = pv;
            const float4 d = *slot_ptr(1, 3, k);
            W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                               fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
        }
        gacc = f2_add(gacc, gp);
        c4_apply<L>(X, geo, th);
    }
    for (int s = 0; s < gm.K; ++s) {
        const int j = s + 2;             // slice t0 + 1 + s
        issue(j + 1);
        cp_async_wait<1>();
        const int sl = j % S;
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
        const long op = base + (long)tp * N;
        const float sgp = (tp == 0) ? 1.0f : -1.0f;
        const bool own = valid && (s + 1 < gm.K);
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 rv = rn_of(sl, k);
            const float4 po = *slot_ptr(sl, 2, k);
            const float4 pv = fma4s(bt, po, rv);
            if (own) {
                st4(rnew, op + geo.off(k), rv);
                st4(pnew, op + geo.off(k), pv);
                st4(x, op + geo.off(k), fma4s(a, po, *slot_ptr(sl, 4, k)));
            }
            P[k] = pv;
            float4 d = *slot_ptr(sl, 3, k);
            d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
            X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                               fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
            Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
        }
        c4_apply<L>(P, geo, th);
        c4_apply_t<L>(Y, geo, th);
        const long o = base + (long)tau * N;
        float pp = 0.0f, rqp = 0.0f, qqp = 0.0f;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 qv = make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y, W[k].z + Y[k].z,
                                          W[k].w + Y[k].w);
            if (valid) st4(qnew, o + geo.off(k), qv);
            const float4 rv = *rbuf(k);   // r' of slice tau
            pp = fmaf(W[k].x, W[k].x, fmaf(W[k].y, W[k].y, fmaf(W[k].z, W[k].z, fmaf(W[k].w, W[k].w, pp))));
            rqp = fmaf(rv.x, qv.x, fmaf(rv.y, qv.y, fmaf(rv.z, qv.z, fmaf(rv.w, qv.w, rqp))));
            qqp = fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, fmaf(qv.z, qv.z, fmaf(qv.w, qv.w, qqp))));
            W[k] = X[k];
            X[k] = P[k];
        }
        pacc = f2_add(pacc, pp);
        rqacc = f2_add(rqacc, rqp);
        qqacc = f2_add(qqacc, qqp);
        if (s + 1 < gm.K) {   // r' of slice tp waits for its output in the next step
            float gp = 0.0f;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                const float4 rv = rn_of(sl, k);
                *rbuf(k) = rv;
                gp = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, gp))));
            }
            gacc = f2_add(gacc, gp);
        }
    }
    cp_async_wait<0>();
    group_store_sum<L>(gacc, valid, bk.g_out + pb + run);
    __syncwarp();
    group_store_sum<L>(pacc, valid, bk.pq_out + pb + run);
    __syncwarp();
    group_store_sum<L>(rqacc, valid, bk.rq_out + pb + run);
    __syncwarp();
    group_store_sum<L>(qqacc, valid, bk.qq_out + pb + run);
}

// Unit partials of r.r, r.q and q.q (same units and layout as the operator
// kernels' partials), for the flagged rhs: one block per (unit, rhs).
__global__ void __launch_bounds__(256) k_unit_dots(const float* __restrict__ r,
                                                   const float* __restrict__ q, MvGeom gm, int N,
                                                   const int* __restrict__ mask,
                                                   double* __restrict__ g_out,
                                                   double* __restrict__ rq_out,
                                                   double* __restrict__ qq_out)
{
    const int run = blockIdx.x, rhs = blockIdx.y;
    if (mask[rhs] == 0) return;
    const long o = (long)rhs * gm.T * N + (long)run * gm.K * N;
    const long len = (long)gm.K * N;
    double gg = 0.0, rqs = 0.0, qqs = 0.0;
    for (long k = threadIdx.x; 4 * k < len; k += blockDim.x) {
        const float4 rv = ld4(r, o + 4 * k);
        const float4 qv = ld4(q, o + 4 * k);
        gg += (double)fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, rv.w * rv.w)));
        rqs += (double)fmaf(rv.x, qv.x, fmaf(rv.y, qv.y, fmaf(rv.z, qv.z, rv.w * qv.w)));
        qqs += (double)fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, fmaf(qv.z, qv.z, qv.w * qv.w)));
    }
    __shared__ double red[3][8];
    gg = warp_sum(gg);
    rqs = warp_sum(rqs);
    qqs = warp_sum(qqs);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = gg;
        red[1][w] = rqs;
        red[2][w] = qqs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            for (int m = 0; m < 3; ++m) t[m] += red[m][i];
        const long pbi = (long)rhs * gm.pstride + run;
        g_out[pbi] = t[0];
        rq_out[pbi] = t[1];
        qq_out[pbi] = t[2];
    }
}


// ---------------------------------------------------------------------------
// The same fused FP32 CG step with the tau chain spread over the warps of a
// block (float4 layout, L = 32): warp w of the block for unit u owns slice
// tau = u K + w alone. The neighbour slices the step needs (C p_{tau-1} for
// w_tau, s D w_{tau+1} for q_tau) come from the adjacent warps through
// shared memory, two barriers per launch, instead of each warp walking a
// chain of K slices with a recomputed halo: K times the warps of the chained
// kernel on the same launch, for one extra C apply per block (the slice
// before the block) and one extra slice load (the slice after it).
// ---------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(256, 2) k_cg_mtm32_tp(const float* __restrict__ r,
                                                        const float* __restrict__ pold,
                                                        float* __restrict__ pnew,
                                                        float* __restrict__ q,
                                                        const float* __restrict__ ev, MvGeom gm,
                                                        const int* __restrict__ mask,
                                                        const double* __restrict__ rr_new_part,
                                                        const double* __restrict__ rr_old_part,
                                                        int rr_stride, int rr_n, int first,
                                                        double* __restrict__ pq_part, float th)
{
    static_assert(L == 32, "one slice per warp needs L = 32");
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    constexpr int RT = L / 4;
    const Geom4<L> geo;
    const int K = gm.K;                          // warps (slices) per block
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rhs = blockIdx.x / gm.nrun;
    if (rhs >= gm.n_rhs) return;                 // whole block: same rhs
    if (mask != nullptr && mask[rhs] == 0) return;
    const int unit = blockIdx.x - rhs * gm.nrun;
    const int t0 = unit * K;
    const int tau = t0 + wi;
    const long base = (long)rhs * gm.T * N;
    // shared: X slot j (0..K) = C p_{t0-1+j}; Z slot j (0..K) = s D w_{t0+j};
    // each slot [RT][32] float4
    extern __shared__ __align__(16) float4 xz[];
    float4* Xs = xz;
    float4* Zs = xz + (long)(K + 1) * RT * 32;
    __shared__ double red[32];
    auto at = [&](float4* a, int j, int k) -> float4* { return a + ((long)j * RT + k) * 32 + lane; };

    const float bt = cg_beta(gm, rhs, first, rr_new_part, rr_old_part, rr_stride, rr_n);
    auto load_p = [&](int t, float4 (&dst)[RT]) {
        const long o = base + (long)t * N;
#pragma unroll
        for (int k = 0; k < RT; ++k) dst[k] = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(r, o + geo.off(k)));
    };
    float4 P[RT], X[RT];
    load_p(tau, P);
    if (pnew != nullptr) {
        const long o = base + (long)tau * N;
#pragma unroll
        for (int k = 0; k < RT; ++k) st4(pnew, o + geo.off(k), P[k]);
    }
#pragma unroll
    for (int k = 0; k < RT; ++k) X[k] = P[k];
    c4_apply<L>(X, geo, th);                     // C p_tau
#pragma unroll
    for (int k = 0; k < RT; ++k) *at(Xs, wi + 1, k) = X[k];
    if (wi == 0) {                               // C p_{t0-1}: the slice before the block
        load_p(t0 == 0 ? gm.T - 1 : t0 - 1, X);
        c4_apply<L>(X, geo, th);
#pragma unroll
        for (int k = 0; k < RT; ++k) *at(Xs, 0, k) = X[k];
    }
    __syncthreads();
    // w_tau = p_tau + s_tau D_tau C p_{tau-1};  Z_tau = s_tau D_tau w_tau
    const float sg = (tau == 0) ? 1.0f : -1.0f;
    float part = 0.0f;
#pragma unroll
    for (int k = 0; k < RT; ++k) {
        const float4 d = ld4(ev, (long)tau * N + geo.off(k));
        const float4 xm = *at(Xs, wi, k);
        P[k].x = fmaf(sg * d.x, xm.x, P[k].x);
        P[k].y = fmaf(sg * d.y, xm.y, P[k].y);
        P[k].z = fmaf(sg * d.z, xm.z, P[k].z);
        P[k].w = fmaf(sg * d.w, xm.w, P[k].w);
        part = fmaf(P[k].x, P[k].x, part);
        part = fmaf(P[k].y, P[k].y, part);
        part = fmaf(P[k].z, P[k].z, part);
        part = fmaf(P[k].w, P[k].w, part);
        *at(Zs, wi, k) = make_float4(sg * d.x * P[k].x, sg * d.y * P[k].y, sg * d.z * P[k].z,
                                     sg * d.w * P[k].w);
    }
    if (wi == K - 1) {                           // Z_{t0+K}: the slice after the block
        const int tp = (t0 + K == gm.T) ? 0 : t0 + K;
        const float sp = (tp == 0) ? 1.0f : -1.0f;
        load_p(tp, X);
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float4 d = ld4(ev, (long)tp * N + geo.off(k));
            const float4 xm = *at(Xs, K, k);     // C p_{t0+K-1}, written by this warp
            float4 wv;
            wv.x = fmaf(sp * d.x, xm.x, X[k].x);
            wv.y = fmaf(sp * d.y, xm.y, X[k].y);
            wv.z = fmaf(sp * d.z, xm.z, X[k].z);
            wv.w = fmaf(sp * d.w, xm.w, X[k].w);
            *at(Zs, K, k) = make_float4(sp * d.x * wv.x, sp * d.y * wv.y, sp * d.z * wv.z,
                                        sp * d.w * wv.w);
        }
    }
    __syncthreads();
    // q_tau = w_tau + C^T Z_{tau+1}
#pragma unroll
    for (int k = 0; k < RT; ++k) X[k] = *at(Zs, wi + 1, k);
    c4_apply_t<L>(X, geo, th);
    {
        const long o = base + (long)tau * N;
#pragma unroll
        for (int k = 0; k < RT; ++k)
            st4(q, o + geo.off(k), make_float4(P[k].x + X[k].x, P[k].y + X[k].y,
                                                P[k].z + X[k].z, P[k].w + X[k].w));
    }
    if (pq_part != nullptr) {                    // |M p|^2 over the block's slices
        const double s = warp_sum((double)part);
        if (lane == 0) red[wi] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int j = 0; j < K; ++j) t += red[j];
            pq_part[(long)rhs * gm.pstride + unit] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// dispatch on L
// ---------------------------------------------------------------------------

template <int L>
int run_cg_mtm32(const hol_ctx* c, const float* r, const float* pold, float* pnew, float* q,
                 int n_rhs, const int* mask, const double* rr_new, const double* rr_old,
                 int rr_stride, int rr_n, int first, double* pq_part, cudaStream_t s,
                 double* alpha_out, int* alpha_done, const double* beta_in)
{
    const MvGeom g = make_geom<L>(c, n_rhs);
    // the layouts whose kernels run cg_alpha_epilogue (scalar, float4, float4
    // with a cp.async ring) form alpha when asked; the others leave it to the
    // update kernel
    MvGeom ga = g;
    if (alpha_out != nullptr) {
        ga.alpha_out = alpha_out;
        ga.alpha_cnt = c->alpha_cnt;
    }
    ga.beta_in = beta_in;   // (the other layouts sum the partials: the same value)
    auto mark = [&]() {
        if (alpha_out != nullptr && alpha_done != nullptr) *alpha_done = 1;
    };
    const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
    if constexpr (L == 32) {
        if (c->mv_vec == 7) {   // one slice per warp, K warps per block
            const int K = c->mv_k;
            if (K > 8) return set_error(HOL_EINVAL, "layout 7 needs slices_per_group <= 8");
            const size_t sm = (size_t)2 * (K + 1) * (L / 4) * 32 * sizeof(float4);
            if (int rc = smem_raise((const void*)k_cg_mtm32_tp<L>, sm)) return rc;
            HOL_CUDA(launch_pdl(c, k_cg_mtm32_tp<L>, g.nrun * g.n_rhs, 32 * K, sm, s, r, pold,
                                pnew, q, c->ev32, g, mask, rr_new, rr_old, rr_stride, rr_n, first,
                                pq_part, (float)c->th));
            HOL_CHECK_LAUNCH("k_cg_mtm32_tp");
            return HOL_OK;
        }
        if (c->mv_vec == 4 || c->mv_vec == 5) {   // split layout, 2 or 4 warps per unit
            const int units = g.nrun * g.n_rhs;
            if (c->mv_vec == 4)
                HOL_CUDA(launch_pdl(c, k_cg_mtm32_split<L, 2>, units, 64, 0, s, r, pold, pnew,
                                    q, c->ev32, g, mask, rr_new, rr_old, rr_stride, rr_n, first,
                                    pq_part, (float)c->th));
            else
                HOL_CUDA(launch_pdl(c, k_cg_mtm32_split<L, 4>, units, 128, 0, s, r, pold, pnew,
                                    q, c->ev32, g, mask, rr_new, rr_old, rr_stride, rr_n, first,
                                    pq_part, (float)c->th));
            HOL_CHECK_LAUNCH("k_cg_mtm32_split");
            return HOL_OK;
        }
    }
    if constexpr (L % 4 == 0 && L >= 8) {   // float4 layout with a cp.async ring (cb4.cuh)
        if (c->mv_vec == 2 || c->mv_vec == 6) {   // cp.async ring of 2 or 3 slices
            const bool deep = c->mv_vec == 6;
            const size_t sm =
                (size_t)c->mv_warps * (deep ? 3 : 2) * 3 * Geom4<L>::RT * 32 * sizeof(float4);
            // raised once per instantiation to the largest size any block shape needs
            // (the static reduction scratch counts against the default limit)
            static std::atomic<int> limit(0);
            if ((int)sm > limit.load()) {
                const int most2 = 4 * 2 * 3 * Geom4<L>::RT * 32 * (int)sizeof(float4);
                const int most3 = 4 * 3 * 3 * Geom4<L>::RT * 32 * (int)sizeof(float4);
                HOL_CUDA(cudaFuncSetAttribute((const void*)k_cg_mtm32_v4a<L, 2>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, most2));
                HOL_CUDA(cudaFuncSetAttribute((const void*)k_cg_mtm32_v4a<L, 3>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, most3));
                limit.store(most3);
            }
            if (deep)
                HOL_CUDA(launch_pdl(c, k_cg_mtm32_v4a<L, 3>, nb, nt, sm, s, r, pold, pnew, q,
                                    c->ev32, ga, mask, rr_new, rr_old, rr_stride, rr_n, first,
                                    pq_part, (float)c->th));
            else
                HOL_CUDA(launch_pdl(c, k_cg_mtm32_v4a<L, 2>, nb, nt, sm, s, r, pold, pnew, q,
                                    c->ev32, ga, mask, rr_new, rr_old, rr_stride, rr_n, first,
                                    pq_part, (float)c->th));
            HOL_CHECK_LAUNCH("k_cg_mtm32_v4a");
            mark();
            return HOL_OK;
        }
    }
    if constexpr (L % 8 == 0) {
        if (c->mv_vec == 3) {
            constexpr int S = 3;
            const int wpb = 4;
            const size_t sm = (size_t)wpb * S * 2 * (L / 4) * 32 * sizeof(float4);
            // resident blocks, queried once per instantiation (one GPU model per process)
            static std::atomic<int> resident(0);
            if (resident.load() == 0) {
                int per_sm = 0, sms = 0;
                // the static reduction scratch counts against the default 48 KB
                // dynamic limit, so the limit is always raised explicitly
                HOL_CUDA(cudaFuncSetAttribute((const void*)k_cg_mtm32_v4s<L, S>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                HOL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per_sm, k_cg_mtm32_v4s<L, S>, 32 * wpb, sm));
                HOL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
                resident.store((per_sm < 1 ? 1 : per_sm) * sms);
            }
            const int need = g.wpr * g.n_rhs;                 // warp-units
            int blocks = resident.load();
            if ((long)blocks * wpb > need) blocks = (need + wpb - 1) / wpb;
            HOL_CUDA(launch_pdl(c, k_cg_mtm32_v4s<L, S>, blocks, 32 * wpb, sm, s, r, pold,
                                pnew, q, c->ev32, g, mask, rr_new, rr_old, rr_stride, rr_n, first,
                                pq_part, (float)c->th, blocks * wpb));
            HOL_CHECK_LAUNCH("k_cg_mtm32_v4s");
            return HOL_OK;
        }
        if (c->mv_vec) {
            HOL_CUDA(launch_pdl(c, k_cg_mtm32_v4<L>, nb, nt, 0, s, r, pold, pnew, q,
                                c->ev32, ga, mask, rr_new, rr_old, rr_stride, rr_n, first, pq_part,
                                (float)c->th));
            HOL_CHECK_LAUNCH("k_cg_mtm32_v4");
            mark();
            return HOL_OK;
        }
    }
    const int rc = run_cg_mtm32_scalar<L, false>(c, r, pold, pnew, q, n_rhs, mask, rr_new, rr_old,
                                                 rr_stride, rr_n, first, pq_part, s,
                                                 ga.alpha_out, beta_in);
    if (rc == HOL_OK) mark();
    return rc;
}


template <int L>
int run_cg_merged(const hol_ctx* c, const float* r, const float* w, const float* pold,
                  const float* sold, float* e, float* pnew, float* snew, float* rnew, float* wnew,
                  int n_rhs, const int* mask, const MergedScal& sc, cudaStream_t s)
{
    if constexpr (L % 8 == 0) {
        const MvGeom g = make_geom<L>(c, n_rhs);
        const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
        HOL_CUDA(launch_pdl(c, k_cg_merged<L>, nb, nt, 0, s, r, w, pold, sold, e, pnew,
                            snew, rnew, wnew, c->ev32, g, mask, sc, (float)c->th));
        HOL_CHECK_LAUNCH("k_cg_merged");
        return HOL_OK;
    } else {
        return set_error(HOL_EINVAL, "merged CG needs L %% 8 == 0 (L=%d)", c->L);
    }
}


template <int L>
int run_cg_fused(const hol_ctx* c, const float* r, const float* q, const float* pold, float* x,
                 float* rnew, float* pnew, float* qnew, int n_rhs, const int* mask,
                 const FusedPartials& fp, cudaStream_t s)
{
    if constexpr (L % 8 == 0) {
        const MvGeom g = make_geom<L>(c, n_rhs);
        const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
        const size_t sm = (size_t)c->mv_warps * (2 * 5 + 1) * (L / 4) * 32 * sizeof(float4);
        static std::atomic<int> limit(0);
        if ((int)sm > limit.load()) {
            const int most = 4 * (2 * 5 + 1) * (L / 4) * 32 * (int)sizeof(float4);
            HOL_CUDA(cudaFuncSetAttribute((const void*)k_cg_fused<L>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, most));
            limit.store(most);
        }
        FusedBanks bk{fp.g, fp.pq, fp.rq, fp.qq, fp.g_out, fp.pq_out, fp.rq_out, fp.qq_out};
        HOL_CUDA(launch_pdl(c, k_cg_fused<L>, nb, nt, sm, s, r, q, pold, x, rnew, pnew, qnew,
                            c->ev32, g, mask, bk, (float)c->th));
        HOL_CHECK_LAUNCH("k_cg_fused");
        return HOL_OK;
    } else {
        return set_error(HOL_EINVAL, "fused CG needs L %% 8 == 0 (L=%d)", c->L);
    }
}

template <int L>
int run_unit_dots(const hol_ctx* c, const float* r, const float* q, int n_rhs, const int* mask,
                  double* g_out, double* rq_out, double* qq_out, cudaStream_t s)
{
    const MvGeom g = make_geom<L>(c, n_rhs);
    k_unit_dots<<<dim3(g.nrun, n_rhs), 256, 0, s>>>(r, q, g, c->N, mask, g_out, rq_out, qq_out);
    HOL_CHECK_LAUNCH("k_unit_dots");
    return HOL_OK;
}

}  // namespace

int launch_cg_fused(const hol_ctx* c, const float* r, const float* q, const float* pold, float* x,
                    float* rnew, float* pnew, float* qnew, int n_rhs, const int* mask,
                    const FusedPartials& fp, cudaStream_t s)
{
    switch (c->L) {
#define X(LL)                                                                               \
    case LL:                                                                                \
        return run_cg_fused<LL>(c, r, q, pold, x, rnew, pnew, qnew, n_rhs, mask, fp, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_unit_dots(const hol_ctx* c, const float* r, const float* q, int n_rhs,
                     const int* mask, double* g_out, double* rq_out, double* qq_out,
                     cudaStream_t s)
{
    switch (c->L) {
#define X(LL)                                                                                \
    case LL:                                                                                 \
        return run_unit_dots<LL>(c, r, q, n_rhs, mask, g_out, rq_out, qq_out, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

namespace {
}  // namespace

int launch_cg_merged(const hol_ctx* c, const float* r, const float* w, const float* pold,
                     const float* sold, float* e, float* pnew, float* snew, float* rnew,
                     float* wnew, int n_rhs, const int* mask, const MergedScal& sc,
                     cudaStream_t s)
{
    switch (c->L) {
#define X(LL)                                                                                  \
    case LL:                                                                                   \
        return run_cg_merged<LL>(c, r, w, pold, sold, e, pnew, snew, rnew, wnew, n_rhs, mask, \
                                 sc, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

namespace {
}  // namespace

int matvec_units(const hol_ctx* c, int n_rhs)
{
    // upper bound of pstride * n_rhs over all L (G >= 1)
    return (c->T / c->mv_k + 31) * n_rhs;
}

int matvec_pstride(const hol_ctx* c)
{
    switch (c->L) {
#define X(LL) case LL: return make_geom<LL>(c, 1).pstride;
        HOL_FOR_EACH_L(X)
#undef X
    }
    return 0;
}

void fp64_cg_geom_exact(const hol_ctx* c, int n_rhs, int* pstride, int* nrun);   // exact_cg.cu

void fp64_cg_geom(const hol_ctx* c, int n_rhs, int* pstride, int* nrun)
{
    *pstride = matvec_pstride(c);
    *nrun = c->T / c->mv_k;
    if (c->exact) {
        fp64_cg_geom_exact(c, n_rhs, pstride, nrun);
        return;
    }
    switch (c->L) {
#define X(LL)                                                 \
    case LL: {                                                \
        const MvGeom g = geom_m_upd64<LL, false>(c, n_rhs);   \
        *pstride = g.pstride;                                 \
        *nrun = g.nrun;                                       \
        return;                                               \
    }
        HOL_FOR_EACH_L(X)
#undef X
    }
}

void occ64_warm(const hol_ctx* c)
{
    switch (c->L) {
#define X(LL) case LL: occ64_warm_l<LL, false>(); return;
        HOL_FOR_EACH_L(X)
#undef X
    }
}

int launch_M(const hol_ctx* c, int prec, const void* v, void* out, int n_rhs, const int* mask,
             double* norm_part, cudaStream_t s)
{
    if (c->exact) return launch_M_exact(c, prec, v, out, n_rhs, mask, norm_part, s);
    switch (c->L) {
#define X(LL) case LL: return run_M<LL, false>(c, prec, v, out, n_rhs, mask, norm_part, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_M_upd64(const hol_ctx* c, const double* r, const double* pold, double* pnew, double* w,
                   int n_rhs, const int* mask, BetaSrc beta, double* norm_part, cudaStream_t s)
{
    if (c->exact)
        return launch_M_upd64_exact(c, r, pold, pnew, w, n_rhs, mask, beta, norm_part, s);
    switch (c->L) {
#define X(LL) case LL: return run_M_upd64<LL, false>(c, r, pold, pnew, w, n_rhs, mask, beta, norm_part, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_MT(const hol_ctx* c, int prec, const void* u, void* out, int n_rhs, const int* mask,
              cudaStream_t s)
{
    if (c->exact) return launch_MT_exact(c, prec, u, out, n_rhs, mask, s);
    switch (c->L) {
#define X(LL) case LL: return run_MT<LL, false>(c, prec, u, out, n_rhs, mask, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_MT_resid64(const hol_ctx* c, const double* u, const double* b, double* out, int n_rhs,
                      const int* mask, cudaStream_t s)
{
    if (c->exact) return launch_MT_resid64_exact(c, u, b, out, n_rhs, mask, s);
    switch (c->L) {
#define X(LL) case LL: return run_MT_resid<LL, false>(c, u, b, out, n_rhs, mask, s);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

int launch_cg_mtm32(const hol_ctx* c, const float* r, const float* pold, float* pnew, float* q,
                    int n_rhs, const int* mask, const double* rr_new, const double* rr_old,
                    int rr_stride, int rr_n, int first, double* pq_part, cudaStream_t s,
                    double* alpha_out, int* alpha_done, const double* beta_in)
{
    if (alpha_done) *alpha_done = 0;
    if (first) beta_in = nullptr;
    if (pq_part == nullptr) alpha_out = nullptr;
    if (c->exact)
        return launch_cg_mtm32_exact(c, r, pold, pnew, q, n_rhs, mask, rr_new, rr_old, rr_stride,
                                     rr_n, first, pq_part, s);
    switch (c->L) {
#define X(LL)                                                                                 \
    case LL:                                                                                  \
        return run_cg_mtm32<LL>(c, r, pold, pnew, q, n_rhs, mask, rr_new, rr_old, rr_stride, \
                                rr_n, first, pq_part, s, alpha_out, alpha_done, beta_in);
        HOL_FOR_EACH_L(X)
#undef X
    }
    return set_error(HOL_EINVAL, "unsupported L=%d", c->L);
}

}  // namespace hol
