// Scalar-layout fermion-matrix kernels (Eq. (M_def), Sec. II D): M v, M^T u
// and the fused FP32 M^T M step of the CG iteration, for the checkerboard
// propagator (EX = false) and the exact exp(-dtau K) (EX = true).
//
// Work decomposition. A "unit" is one right-hand side and a run of K
// consecutive tau slices; one lane group (L lanes, see cb.cuh) streams the
// run, holding one slice per register column. A warp holds G = 32/L groups
// that always belong to the same right-hand side (the run index is padded to
// a multiple of G), so per-rhs scalars are warp-uniform. Every global access
// is a row of L consecutive sites (coalesced); the propagator itself never
// leaves registers.
//
// Included by matvec.cu (checkerboard instantiations) and exact.cu (exact
// ones), so each translation unit compiles only its own half.
#pragma once

#include <atomic>

#include "cb.cuh"
#include "internal.cuh"

namespace hol {
namespace {

struct MvGeom {
    int T;              // slices
    int K;              // slices per unit (divides T)
    int nrun;           // T / K
    int wpr;            // warps per right-hand side = ceil(nrun / G)
    int n_rhs;
    int pstride;        // stride of the per-unit partial sums (= wpr * G)
    double* alpha_out;  // CG operator only (nullable): alpha per rhs, formed by the last warp
    int* alpha_cnt;     // warps of each rhs that have finished (reset by the last one)
    const double* beta_in;   // CG operator only (nullable): beta per rhs, formed by the update
};

template <int L>
__host__ MvGeom make_geom(const hol_ctx* c, int n_rhs)
{
    MvGeom g;
    g.T = c->T;
    g.K = c->mv_k;
    g.nrun = c->T / c->mv_k;
    constexpr int G = 32 / L;
    g.wpr = (g.nrun + G - 1) / G;
    g.n_rhs = n_rhs;
    g.pstride = g.wpr * G;
    g.alpha_out = nullptr;
    g.alpha_cnt = nullptr;
    g.beta_in = nullptr;
    return g;
}

// beta of a CG step: 0 on the first, else the value the update kernel formed
// for this rhs (when given), else (r.r)_new / (r.r)_old from the partial rows
// (the same sums, so the same bits either way).
__device__ __forceinline__ float cg_beta(const MvGeom& gm, int rhs, int first,
                                         const double* __restrict__ rr_new_part,
                                         const double* __restrict__ rr_old_part, int rr_stride,
                                         int rr_n)
{
    if (first) return 0.0f;
    if (gm.beta_in != nullptr) return (float)gm.beta_in[rhs];
    const double rn = warp_sum_array(rr_new_part + (long)rhs * rr_stride, rr_n);
    const double ro = warp_sum_array(rr_old_part + (long)rhs * rr_stride, rr_n);
    return (float)cg_ratio(rn, ro);
}

// CG operator epilogue: once every warp of a right-hand side has stored its
// partial sums of p.q, the last warp to finish forms alpha = (r.z) / (p.q)
// of that right-hand side from the partial rows, in the order the update
// kernel would sum them (so the same bits), and resets the count. The update
// kernel then reads one number instead of reducing partials in every block
// (FP64 sums cost sixty-four FP32 operations each on this GPU). The count is
// an atomic; no warp waits for another.
__device__ __forceinline__ void cg_alpha_epilogue(const MvGeom& gm, int rhs,
                                                  const double* __restrict__ pq_part,
                                                  const double* __restrict__ dz_part,
                                                  int dz_stride, int dz_n)
{
    if (gm.alpha_out == nullptr) return;
    __syncwarp();
    __threadfence();
    int prev = 0;
    if ((threadIdx.x & 31) == 0) prev = atomicAdd(gm.alpha_cnt + rhs, 1);
    prev = __shfl_sync(kFull, prev, 0);
    if (prev != gm.wpr - 1) return;
    __threadfence();
    const double pq = warp_sum_array_cg(pq_part + (long)rhs * gm.pstride, gm.nrun);
    const double dz = warp_sum_array_cg(dz_part + (long)rhs * dz_stride, dz_n);
    if ((threadIdx.x & 31) == 0) {
        gm.alpha_out[rhs] = cg_ratio(dz, pq);
        gm.alpha_cnt[rhs] = 0;
    }
}

// -x when neg, else x: a sign-bit flip on the integer pipe (the FP64 pipe,
// 1/64 of the FP32 rate on this part, is not spent on a multiplication by -1)
__device__ __forceinline__ double neg_if(bool neg, double x)
{
    const unsigned long long m = neg ? 0x8000000000000000ULL : 0ULL;
    return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^ m));
}
__device__ __forceinline__ float neg_if(bool neg, float x)
{
    return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000 : 0));
}

// ---------------------------------------------------------------------------
// out = M v. With UPD the loaded vector is p_new = r + beta p_old (the CG
// direction update), whose own slices are also stored to pnew.
// norm_part (used when NORM, else ignored): |out|^2 summed over the unit's
// slices.
// ---------------------------------------------------------------------------
template <typename R, int L, bool UPD, bool EX, bool NORM = true>
__global__ void __launch_bounds__(128) k_M(const R* __restrict__ v, const R* __restrict__ pold,
                                           R* __restrict__ pnew, R* __restrict__ out,
                                           const R* __restrict__ ev, MvGeom gm,
                                           const int* __restrict__ mask, BetaSrc bsrc,
                                           double* __restrict__ norm_part, Kin<R> kin)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    const LaneGeom<L> geo;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = (warp - rhs * gm.wpr) * LaneGeom<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N + geo.ix;
    R bt = R(0);
    if (UPD && !bsrc.first) {
        const double rn = warp_sum_array(bsrc.rn + (long)rhs * bsrc.stride, bsrc.n);
        const double ro = warp_sum_array(bsrc.ro + (long)rhs * bsrc.stride, bsrc.n);
        bt = (R)cg_ratio(rn, ro);
    }

    R a[L], c[L];
    {
        const int tm = (t0 == 0) ? gm.T - 1 : t0 - 1;
        const long o = base + (long)tm * N;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            R val = v[o + iy * L];
            if (UPD) val = fma(bt, pold[o + iy * L], val);
            a[iy] = val;
        }
    }
    double acc = 0.0;
    for (int s = 0; s < gm.K; ++s) {
        const int tau = t0 + s;
        const long o = base + (long)tau * N;
        kin_apply<R, L, EX>(a, geo, kin);
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            R val = v[o + iy * L];
            if (UPD) {
                val = fma(bt, pold[o + iy * L], val);
                if (valid) pnew[o + iy * L] = val;
            }
            c[iy] = val;
        }
        const bool neg = tau != 0;   // s_tau = -1 except at tau = 0
        R part = R(0);
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            const R w = fma(neg_if(neg, ev[(long)tau * N + iy * L + geo.ix]), a[iy], c[iy]);
            if (valid) out[o + iy * L] = w;
            if constexpr (NORM) part = fma(w, w, part);
            a[iy] = c[iy];
        }
        if constexpr (NORM) acc += (double)part;
    }
    if constexpr (NORM) {
        if (norm_part != nullptr)
            group_store_sum<L>(acc, valid, norm_part + (long)rhs * gm.pstride + run);
    }
}

// ---------------------------------------------------------------------------
// out = M^T u (EPI = MT_PLAIN) or, FP64 only, out = b - M^T u (MT_RESID).
// Streams the run downwards: (M^T u)_tau needs u_tau and u_{tau+1}.
// ---------------------------------------------------------------------------
template <typename R, int L, int EPI, bool EX>
__global__ void __launch_bounds__(128) k_MT(const R* __restrict__ u, const R* __restrict__ bvec,
                                            R* __restrict__ out, const R* __restrict__ ev,
                                            MvGeom gm, const int* __restrict__ mask, Kin<R> kin)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    const LaneGeom<L> geo;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = (warp - rhs * gm.wpr) * LaneGeom<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N + geo.ix;

    R a[L], c[L];
    {
        int tp = t0 + gm.K;
        if (tp == gm.T) tp = 0;
        const long o = base + (long)tp * N;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) a[iy] = u[o + iy * L];
    }
    for (int s = gm.K - 1; s >= 0; --s) {
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) a[iy] *= ev[(long)tp * N + iy * L + geo.ix];
        kin_apply_t<R, L, EX>(a, geo, kin);
        const long o = base + (long)tau * N;
        const R sg = (tp == 0) ? R(1) : R(-1);
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            c[iy] = u[o + iy * L];
            R w = fma(sg, a[iy], c[iy]);
            if (EPI == MT_RESID) w = bvec[o + iy * L] - w;
            if (valid) out[o + iy * L] = w;
            a[iy] = c[iy];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 fused CG step: p_new = r + beta p_old, q = M^T M p_new,
// pq_part = |M p_new|^2 = p_new . q per unit. The run needs w = M p on
// [t0, t0+K] and hence p on [t0-1, t0+K]; halo values are recomputed.
// ---------------------------------------------------------------------------
template <int L, bool EX>
__global__ void __launch_bounds__(128) k_cg_mtm32(const float* __restrict__ r,
                                                  const float* __restrict__ pold,
                                                  float* __restrict__ pnew, float* __restrict__ q,
                                                  const float* __restrict__ ev, MvGeom gm,
                                                  const int* __restrict__ mask,
                                                  const double* __restrict__ rr_new_part,
                                                  const double* __restrict__ rr_old_part,
                                                  int rr_stride, int rr_n, int first,
                                                  double* __restrict__ pq_part, Kin<float> kin)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    constexpr int N = L * L;
    const LaneGeom<L> geo;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rhs = warp / gm.wpr;
    if (rhs >= gm.n_rhs) return;
    if (mask != nullptr && mask[rhs] == 0) return;
    const int run = (warp - rhs * gm.wpr) * LaneGeom<L>::G + geo.g;
    const bool valid = geo.ok && run < gm.nrun;
    const int t0 = (run < gm.nrun ? run : gm.nrun - 1) * gm.K;
    const long base = (long)rhs * gm.T * N + geo.ix;

    // beta = (r.r)_new / (r.r)_old, identical bits in every warp of this rhs
    const float bt = cg_beta(gm, rhs, first, rr_new_part, rr_old_part, rr_stride, rr_n);

    float W[L], X[L], P[L], Y[L];
    // Y <- C p_{t0-1}
    {
        const int tm = (t0 == 0) ? gm.T - 1 : t0 - 1;
        const long o = base + (long)tm * N;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) Y[iy] = fmaf(bt, pold[o + iy * L], r[o + iy * L]);
        kin_apply<float, L, EX>(Y, geo, kin);
    }
    // W <- w_{t0} = p_{t0} + s_{t0} D_{t0} C p_{t0-1};  X <- C p_{t0}
    {
        const long o = base + (long)t0 * N;
        const float sg = (t0 == 0) ? 1.0f : -1.0f;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            const float pv = fmaf(bt, pold[o + iy * L], r[o + iy * L]);
            if (valid && pnew != nullptr) pnew[o + iy * L] = pv;
            X[iy] = pv;
            W[iy] = fmaf(sg * ev[(long)t0 * N + iy * L + geo.ix], Y[iy], pv);
        }
        kin_apply<float, L, EX>(X, geo, kin);
    }
    F2 acc{0.0f, 0.0f};   // compensated float pair (see cb.cuh)
    for (int s = 0; s < gm.K; ++s) {
        const int tau = t0 + s;
        const int tp = (tau + 1 == gm.T) ? 0 : tau + 1;
        const long op = base + (long)tp * N;
        const float sgp = (tp == 0) ? 1.0f : -1.0f;
        const bool own = valid && (s + 1 < gm.K) && pnew != nullptr;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            const float pv = fmaf(bt, pold[op + iy * L], r[op + iy * L]);
            if (own) pnew[op + iy * L] = pv;
            P[iy] = pv;
            const float d = sgp * ev[(long)tp * N + iy * L + geo.ix];
            X[iy] = fmaf(d, X[iy], pv);       // w_{tau+1}
            Y[iy] = d * X[iy];
        }
        kin_apply<float, L, EX>(P, geo, kin);     // C p_{tau+1}
        kin_apply_t<float, L, EX>(Y, geo, kin);   // C^T s D w_{tau+1}
        const long o = base + (long)tau * N;
        float part = 0.0f;
#pragma unroll
        for (int iy = 0; iy < L; ++iy) {
            if (valid) q[o + iy * L] = W[iy] + Y[iy];
            part = fmaf(W[iy], W[iy], part);
            W[iy] = X[iy];
            X[iy] = P[iy];
        }
        acc = f2_add(acc, part);
    }
    if (pq_part != nullptr) {
        group_store_sum<L>(acc, valid, pq_part + (long)rhs * gm.pstride + run);
        cg_alpha_epilogue(gm, rhs, pq_part, rr_new_part, rr_stride, rr_n);
    }
}

template <int L>
int blocks_for(const hol_ctx* c, const MvGeom& g)
{
    const long warps = (long)g.wpr * g.n_rhs;
    return ceil_div(warps, c->mv_warps);
}

// Resident blocks per SM of `kern` at wpb warps per block, cached per kernel
// in `cache` (indexed by wpb). The occupancy query is not a stream operation;
// it is made once, before any capture (occ64_warm, from hol_create). The
// caches are process-wide (g_occ64, shared by the translation units that
// instantiate the same kernel).
inline int occ_blocks(const void* kern, int wpb, std::atomic<int> (&cache)[5])
{
    int rb = cache[wpb].load();
    if (rb == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rb, kern, 32 * wpb, 0) != cudaSuccess ||
            rb < 1)
            rb = 1;
        cache[wpb].store(rb);
    }
    return rb;
}

// Geometry of an FP64 operator launch that keeps no per-unit partial sums
// (M without |Mv|^2, M^T, the residual M^T): these kernels are bound by the
// FP64 pipe (1/64 of the FP32 rate on this part) and need every resident
// warp slot filled to hide its latency, while the CG's FP32 shape (few long
// slice runs) suits bandwidth. K is the smallest divisor of T, at most the
// context's K, whose warps fit one resident wave (rb blocks per SM); a halo
// slice is re-read per run, no slice is computed twice, so the results do
// not depend on K.
template <int L>
__host__ MvGeom make_geom64(const hol_ctx* c, int n_rhs, int rb, long max_pstride = 1L << 30)
{
    const long wave = (long)rb * c->mv_warps * c->sms;
    constexpr int G = 32 / L;
    int k = c->mv_k;
    for (int kk = 1; kk < c->mv_k; ++kk) {
        if (c->T % kk) continue;
        const long wpr = (c->T / kk + G - 1) / G;
        if (wpr * G > max_pstride) continue;   // the per-unit partial sums must fit their bank
        if (wpr * n_rhs <= wave) {
            k = kk;
            break;
        }
    }
    MvGeom g = make_geom<L>(c, n_rhs);
    g.K = k;
    g.nrun = c->T / k;
    g.wpr = (g.nrun + G - 1) / G;
    g.pstride = g.wpr * G;
    return g;
}

#define HOL_FOR_EACH_L(X) \
    X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) X(30) X(32)

// warm the occupancy caches of the partial-free FP64 operator kernels
// (make_geom64) for every block size, outside any stream capture
template <int L, bool EX>
void occ64_warm_l()
{
    for (int w : {1, 2, 4}) {
        occ_blocks((const void*)k_M<double, L, false, EX, false>, w, g_occ64[EX][0][L]);
        occ_blocks((const void*)k_MT<double, L, MT_PLAIN, EX>, w, g_occ64[EX][1][L]);
        occ_blocks((const void*)k_MT<double, L, MT_RESID, EX>, w, g_occ64[EX][2][L]);
        occ_blocks((const void*)k_M<double, L, true, EX, true>, w, g_occ64[EX][3][L]);
    }
}

// Geometry of the FP64 CG's M (p = z + beta p_old, w = M p, |w|^2 partials
// per unit): the FP64 grouping of make_geom64, limited so that its partial
// sums fit the bank; the update kernel reads them with this geometry's
// stride and count (fp64_cg_geom).
template <int L, bool EX>
MvGeom geom_m_upd64(const hol_ctx* c, int n_rhs)
{
    const int rb = occ_blocks((const void*)k_M<double, L, true, EX, true>, c->mv_warps,
                              g_occ64[EX][3][L]);
    return make_geom64<L>(c, n_rhs, rb, c->part_len / c->p.max_rhs);
}

template <int L, bool EX>
int run_M(const hol_ctx* c, int prec, const void* v, void* out, int n_rhs, const int* mask,
          double* norm_part, cudaStream_t s)
{
    const MvGeom g = make_geom<L>(c, n_rhs);
    const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
    if (prec == HOL_F64 && norm_part == nullptr) {
        const int rb = occ_blocks((const void*)k_M<double, L, false, EX, false>, c->mv_warps,
                                  g_occ64[EX][0][L]);
        const MvGeom g64 = make_geom64<L>(c, n_rhs, rb);
        HOL_CUDA(launch_pdl(c, k_M<double, L, false, EX, false>, blocks_for<L>(c, g64), nt, 0, s,
                            (const double*)v, nullptr, nullptr, (double*)out, c->ev64, g64, mask,
                            BetaSrc{}, nullptr, kin_of<double>(c)));
    } else if (prec == HOL_F64)
        HOL_CUDA(launch_pdl(c, k_M<double, L, false, EX>, nb, nt, 0, s, (const double*)v,
                            nullptr, nullptr, (double*)out, c->ev64, g, mask, BetaSrc{},
                            norm_part, kin_of<double>(c)));
    else
        HOL_CUDA(launch_pdl(c, k_M<float, L, false, EX>, nb, nt, 0, s, (const float*)v, nullptr,
                            nullptr, (float*)out, c->ev32, g, mask, BetaSrc{}, norm_part,
                            kin_of<float>(c)));
    HOL_CHECK_LAUNCH("k_M");
    return HOL_OK;
}

template <int L, bool EX>
int run_M_upd64(const hol_ctx* c, const double* r, const double* pold, double* pnew, double* w,
                int n_rhs, const int* mask, BetaSrc beta, double* norm_part, cudaStream_t s)
{
    const MvGeom g = geom_m_upd64<L, EX>(c, n_rhs);
    const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
    HOL_CUDA(launch_pdl(c, k_M<double, L, true, EX>, nb, nt, 0, s, r, pold, pnew, w, c->ev64, g,
                        mask, beta, norm_part, kin_of<double>(c)));
    HOL_CHECK_LAUNCH("k_M upd");
    return HOL_OK;
}

template <int L, bool EX>
int run_MT(const hol_ctx* c, int prec, const void* u, void* out, int n_rhs, const int* mask,
           cudaStream_t s)
{
    const MvGeom g = make_geom<L>(c, n_rhs);
    const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
    if (prec == HOL_F64) {
        const int rb = occ_blocks((const void*)k_MT<double, L, MT_PLAIN, EX>, c->mv_warps,
                                  g_occ64[EX][1][L]);
        const MvGeom g64 = make_geom64<L>(c, n_rhs, rb);
        HOL_CUDA(launch_pdl(c, k_MT<double, L, MT_PLAIN, EX>, blocks_for<L>(c, g64), nt, 0, s,
                            (const double*)u, nullptr, (double*)out, c->ev64, g64, mask,
                            kin_of<double>(c)));
    } else
        HOL_CUDA(launch_pdl(c, k_MT<float, L, MT_PLAIN, EX>, nb, nt, 0, s, (const float*)u,
                            nullptr, (float*)out, c->ev32, g, mask, kin_of<float>(c)));
    HOL_CHECK_LAUNCH("k_MT");
    return HOL_OK;
}

template <int L, bool EX>
int run_MT_resid(const hol_ctx* c, const double* u, const double* b, double* out, int n_rhs,
                 const int* mask, cudaStream_t s)
{
    const int rb = occ_blocks((const void*)k_MT<double, L, MT_RESID, EX>, c->mv_warps,
                              g_occ64[EX][2][L]);
    const MvGeom g = make_geom64<L>(c, n_rhs, rb);
    const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
    HOL_CUDA(launch_pdl(c, k_MT<double, L, MT_RESID, EX>, nb, nt, 0, s, u, b, out, c->ev64, g,
                        mask, kin_of<double>(c)));
    HOL_CHECK_LAUNCH("k_MT resid");
    return HOL_OK;
}

// FP32 fused CG step in the scalar layout.
template <int L, bool EX>
int run_cg_mtm32_scalar(const hol_ctx* c, const float* r, const float* pold, float* pnew,
                        float* q, int n_rhs, const int* mask, const double* rr_new,
                        const double* rr_old, int rr_stride, int rr_n, int first,
                        double* pq_part, cudaStream_t s, double* alpha_out = nullptr,
                        const double* beta_in = nullptr)
{
    MvGeom g = make_geom<L>(c, n_rhs);
    if (alpha_out != nullptr && pq_part != nullptr) {   // see cg_alpha_epilogue
        g.alpha_out = alpha_out;
        g.alpha_cnt = c->alpha_cnt;
    }
    g.beta_in = beta_in;
    const int nb = blocks_for<L>(c, g), nt = 32 * c->mv_warps;
    HOL_CUDA(launch_pdl(c, k_cg_mtm32<L, EX>, nb, nt, 0, s, r, pold, pnew, q, c->ev32, g, mask,
                        rr_new, rr_old, rr_stride, rr_n, first, pq_part, kin_of<float>(c)));
    HOL_CHECK_LAUNCH("k_cg_mtm32");
    return HOL_OK;
}

}  // namespace
}  // namespace hol
