// Persistent mixed-precision CG iterations (one cooperative launch per chunk).
//
// For the plain (unpreconditioned) mixed solve with L % 8 == 0 the two
// kernels of a CG iteration are fused into one resident grid that runs a
// chunk of iterations with two grid-wide barriers per iteration:
//   phase A (per unit: one rhs, K tau slices):
//       beta = (r.r)_new / (r.r)_old from the partial sums,
//       p_new = r + beta p_old on the slices t0-1 .. t0+K (halo recomputed),
//       q = M^T M p_new on t0 .. t0+K-1 (float4 register layout, cb4.cuh),
//       p_new and q of the own slices kept in shared memory, p_new stored,
//       partial sums of |M p_new|^2 = p_new . q;
//   grid barrier;
//   phase B: alpha = (r.r)/(p.q); e += alpha p_new, r -= alpha q on the own
//       slices (q never leaves the SM), partial sums of the new r.r;
//   grid barrier.
// Per iteration each vector element is read and written once per array
// (r, p, e) apart from the tau halo, against ten passes for the two-kernel
// form. The host keeps the polls and the FP64 reliable updates between
// chunks (cg.cu). The partial sums use the same banks as the two-kernel form
// (stride kRedStride); the counts of valid entries are passed in because the
// reliable update writes its own (block-layout) partials.
#include <cooperative_groups.h>

#include "cb.cuh"
#include "cb4.cuh"
#include "internal.cuh"

namespace hol {
namespace {

namespace cgrp = cooperative_groups;

struct PersistArgs {
    float* r;
    float* p0;
    float* p1;
    float* e;
    const float* ev;
    const int* mask;
    double* pq;        // [rhs][kRedStride] unit partials of p.q
    double* rr0;       // [rhs][kRedStride] partials of r.r (two banks)
    double* rr1;
    int T, K, nrun, wpr, n_rhs;
    int cur;           // bank with the current r.r at entry
    int cnt_cur;       // valid partials in rr[cur] at entry
    int cnt_old;       // valid partials in rr[1 - cur] at entry
    int pp;            // p buffer holding p_old at entry
    int first;         // first iteration of the solve (beta = 0)
    int nit;           // iterations to run
    float th;
};

template <int L>
__global__ void __launch_bounds__(128, 3) k_cg_persist(PersistArgs a)
{
    constexpr int N = L * L;
    constexpr int RT = L / 4;
    extern __shared__ __align__(16) float4 keep[];   // [warp][2 (p, q)][K][RT][32]
    cgrp::grid_group grid = cgrp::this_grid();
    const Geom4<L> geo;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* myk = keep + (long)wib * (2 * a.K * RT * 32);
    auto kp = [&](int s, int k) -> float4* { return myk + ((0 * a.K + s) * RT + k) * 32 + lane; };
    auto kq = [&](int s, int k) -> float4* { return myk + ((1 * a.K + s) * RT + k) * 32 + lane; };
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / a.wpr;
    const bool work = rhs < a.n_rhs && (a.mask == nullptr || a.mask[rhs] != 0);
    const int rr_ = work ? rhs : 0;
    const int run = (warp - rr_ * a.wpr) * Geom4<L>::G + geo.g;
    const bool valid = work && geo.ok && run < a.nrun;
    const int t0 = (run < a.nrun ? run : a.nrun - 1) * a.K;
    const long base = (long)rr_ * a.T * N;

    int cur = a.cur, pp = a.pp, first = a.first;
    int cnt_cur = a.cnt_cur, cnt_old = a.cnt_old;
    for (int it = 0; it < a.nit; ++it) {
        const float* pold = first ? a.r : (pp ? a.p1 : a.p0);
        float* pnew = pp ? a.p0 : a.p1;
        double* rr_now = cur ? a.rr1 : a.rr0;
        double* rr_nxt = cur ? a.rr0 : a.rr1;
        if (work) {
            // ---------------- phase A
            float bt = 0.0f;
            if (!first) {
                const double rn = warp_sum_array(rr_now + (long)rhs * kRedStride, cnt_cur);
                const double ro = warp_sum_array(rr_nxt + (long)rhs * kRedStride, cnt_old);
                bt = (float)cg_ratio(rn, ro);
            }
            float4 W[RT], X[RT], P[RT], Y[RT];
            {
                const int tm = (t0 == 0) ? a.T - 1 : t0 - 1;
                const long o = base + (long)tm * N;
#pragma unroll
                for (int k = 0; k < RT; ++k)
                    Y[k] = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(a.r, o + geo.off(k)));
                c4_apply<L>(Y, geo, a.th);
            }
            {
                const long o = base + (long)t0 * N;
                const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    const float4 pv = fma4s(bt, ld4(pold, o + geo.off(k)), ld4(a.r, o + geo.off(k)));
                    if (valid) st4(pnew, o + geo.off(k), pv);
                    *kp(0, k) = pv;
                    X[k] = pv;
                    const float4 d = ld4(a.ev, (long)t0 * N + geo.off(k));
                    W[k] = make_float4(fmaf(sg * d.x, Y[k].x, pv.x), fmaf(sg * d.y, Y[k].y, pv.y),
                                       fmaf(sg * d.z, Y[k].z, pv.z), fmaf(sg * d.w, Y[k].w, pv.w));
                }
                c4_apply<L>(X, geo, a.th);
            }
            double acc = 0.0;
            for (int s = 0; s < a.K; ++s) {
                const int tau = t0 + s;
                const int tp = (tau + 1 == a.T) ? 0 : tau + 1;
                const long op = base + (long)tp * N;
                const float sgp = (tp == 0) ? 1.0f : -1.0f;
                const bool own = valid && (s + 1 < a.K);
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    const float4 pv = fma4s(bt, ld4(pold, op + geo.off(k)), ld4(a.r, op + geo.off(k)));
                    if (own) st4(pnew, op + geo.off(k), pv);
                    if (s + 1 < a.K) *kp(s + 1, k) = pv;
                    P[k] = pv;
                    float4 d = ld4(a.ev, (long)tp * N + geo.off(k));
                    d.x *= sgp; d.y *= sgp; d.z *= sgp; d.w *= sgp;
                    X[k] = make_float4(fmaf(d.x, X[k].x, pv.x), fmaf(d.y, X[k].y, pv.y),
                                       fmaf(d.z, X[k].z, pv.z), fmaf(d.w, X[k].w, pv.w));
                    Y[k] = make_float4(d.x * X[k].x, d.y * X[k].y, d.z * X[k].z, d.w * X[k].w);
                }
                c4_apply<L>(P, geo, a.th);
                c4_apply_t<L>(Y, geo, a.th);
                float part = 0.0f;
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    *kq(s, k) = make_float4(W[k].x + Y[k].x, W[k].y + Y[k].y, W[k].z + Y[k].z,
                                            W[k].w + Y[k].w);
                    part = fmaf(W[k].x, W[k].x, part);
                    part = fmaf(W[k].y, W[k].y, part);
                    part = fmaf(W[k].z, W[k].z, part);
                    part = fmaf(W[k].w, W[k].w, part);
                    W[k] = X[k];
                    X[k] = P[k];
                }
                acc += (double)part;
            }
            group_store_sum<L>(acc, valid, a.pq + (long)rhs * kRedStride + run);
        }
        grid.sync();
        if (work) {
            // ---------------- phase B
            const double pqs = warp_sum_array(a.pq + (long)rhs * kRedStride, a.nrun);
            const double rz = warp_sum_array(rr_now + (long)rhs * kRedStride, cnt_cur);
            const float al = (float)cg_ratio(rz, pqs);
            double acc = 0.0;
            for (int s = 0; s < a.K; ++s) {
                const long o = base + (long)(t0 + s) * N;
                float part = 0.0f;
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    float4 ev4 = ld4(a.e, o + geo.off(k));
                    float4 rv4 = ld4(a.r, o + geo.off(k));
                    const float4 p4 = *kp(s, k), q4 = *kq(s, k);
                    ev4 = make_float4(fmaf(al, p4.x, ev4.x), fmaf(al, p4.y, ev4.y),
                                      fmaf(al, p4.z, ev4.z), fmaf(al, p4.w, ev4.w));
                    rv4 = make_float4(fmaf(-al, q4.x, rv4.x), fmaf(-al, q4.y, rv4.y),
                                      fmaf(-al, q4.z, rv4.z), fmaf(-al, q4.w, rv4.w));
                    if (valid) {
                        st4(a.e, o + geo.off(k), ev4);
                        st4(a.r, o + geo.off(k), rv4);
                    }
                    part = fmaf(rv4.x, rv4.x, part);
                    part = fmaf(rv4.y, rv4.y, part);
                    part = fmaf(rv4.z, rv4.z, part);
                    part = fmaf(rv4.w, rv4.w, part);
                }
                acc += (double)part;
            }
            group_store_sum<L>(acc, valid, rr_nxt + (long)rhs * kRedStride + run);
        }
        grid.sync();
        cnt_old = cnt_cur;
        cnt_cur = a.nrun;
        cur = 1 - cur;
        pp = 1 - pp;
        first = 0;
    }
}

template <int L>
int run_persist(const hol_ctx* c, PersistArgs a, int check_only, cudaStream_t s)
{
    const int G = 32 / L;
    a.nrun = c->T / c->mv_k;
    a.K = c->mv_k;
    a.wpr = (a.nrun + G - 1) / G;
    const int warps = a.wpr * a.n_rhs;
    const int wpb = c->mv_warps;
    const int blocks = (warps + wpb - 1) / wpb;
    const size_t sm = (size_t)wpb * 2 * a.K * (L / 4) * 32 * sizeof(float4);
    if (a.nrun > kRedStride) return HOL_EINVAL;
    int smem_max = 0;
    HOL_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (sm + 4096 > (size_t)smem_max) return HOL_EINVAL;   // does not fit: caller falls back
    if (int rc = smem_raise((const void*)k_cg_persist<L>, sm)) return rc;
    int per_sm = 0, sms = 0;
    HOL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persist<L>, 32 * wpb, sm));
    HOL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if ((long)per_sm * sms < blocks) return HOL_EINVAL;   // does not fit: caller falls back
    if (check_only) return HOL_OK;
    void* args[] = {&a};
    HOL_CUDA(cudaLaunchCooperativeKernel((const void*)k_cg_persist<L>, dim3(blocks), dim3(32 * wpb),
                                         args, sm, s));
    count_launch();
    return HOL_OK;
}

}  // namespace

// Run nit fused CG iterations in one cooperative launch; returns HOL_EINVAL
// without launching when the shape is unsupported or the grid cannot be
// resident (check_only: only answer that question).
int launch_cg_persist(const hol_ctx* c, float* r, float* p0, float* p1, float* e, int n_rhs,
                      const int* mask, double* pq, double* rr0, double* rr1, int cur, int cnt_cur,
                      int cnt_old, int pp, int first, int nit, int check_only, cudaStream_t s)
{
    PersistArgs a;
    a.r = r;
    a.p0 = p0;
    a.p1 = p1;
    a.e = e;
    a.ev = c->ev32;
    a.mask = mask;
    a.pq = pq;
    a.rr0 = rr0;
    a.rr1 = rr1;
    a.T = c->T;
    a.n_rhs = n_rhs;
    a.cur = cur;
    a.cnt_cur = cnt_cur;
    a.cnt_old = cnt_old;
    a.pp = pp;
    a.first = first;
    a.nit = nit;
    a.th = (float)c->th;
    switch (c->L) {
    case 8: return run_persist<8>(c, a, check_only, s);
    case 16: return run_persist<16>(c, a, check_only, s);
    case 24: return run_persist<24>(c, a, check_only, s);
    case 32: return run_persist<32>(c, a, check_only, s);
    }
    return HOL_EINVAL;
}

}  // namespace hol
