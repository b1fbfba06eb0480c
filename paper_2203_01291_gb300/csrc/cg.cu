// Conjugate gradients on M^T M v = b (Eq. (CG)), optionally preconditioned
// with z = P^{-1} P^{-T} r (Eq. (CG_precon)); stopping rule of Sec. VI B on
// the true residual |b - M^T M v| / |b|.
//
// One iteration is
//   1. direction + operator: p_new = z + beta p_old, q = M^T M p_new and the
//      partial sums of p_new . q = |M p_new|^2 (matvec.cu);
//   2. update: alpha = (r.z)/(p.q), x += alpha p, r -= alpha q and the partial
//      sums of the new r.r;
//   3. (preconditioned only) z = P^{-1} P^{-T} r with the partial sums of r.z
//      (precond.cu); without a preconditioner z is r itself. By default the
//      update of step 2 runs inside the forward transform of step 3
//      (k_tau_fwd_upd, option fused_pc_update).
// alpha and beta are recomputed by every consumer from the partial sums in a
// fixed order, so no extra launch or grid barrier sits on the critical path.
// Dot products are summed in FP64 across blocks; inside a block the mixed
// path sums FP32 products as compensated float pairs (cb.cuh, F2).
//
// Mixed precision (opts->prec == HOL_F32): x is an FP32 increment e on top
// of the FP64 solution v; every `reliable_every` iterations, and whenever the
// recursive residual estimate says "converged", e is folded into v and the
// true residual b - M^T M v is recomputed in FP64 (reliable update) and
// replaces r; the search direction is kept but re-conjugated against the new
// residual (beta = -(z, A p) / (p, A p)). Every reported convergence is
// certified by that FP64 residual. The preconditioner of the mixed path runs
// in FP32.
#include <math.h>
#include <string.h>

#include <vector>

#include "cb.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace hol {
namespace {

template <typename R>
struct V4;
template <>
struct V4<float> {
    float v[4];
    __device__ __forceinline__ void ld(const float* p)
    {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ void st(float* p) const
    {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct V4<double> {
    double v[4];
    __device__ __forceinline__ void ld(const double* p)
    {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ void st(double* p) const
    {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
    }
};

// The operands of one float4 element of the update kernel (x, p, p_prev
// only when the x update is folded in).
template <typename R>
struct Ops {
    V4<R> r, q, x, p, pp;
    __device__ __forceinline__ void load(const R* rr, const R* qq, const R* xx, const R* ppv,
                                         const R* ppr, long o, int fold)
    {
        r.ld(rr + o);
        q.ld(qq + o);
        if (fold != 0) {
            x.ld(xx + o);
            p.ld(ppv + o);
            if (fold == 2) pp.ld(ppr + o);
        }
    }
};


// r -= alpha q with the new (r.r) partials; alpha = dz / pq from partials.
// The x update may be deferred by one iteration (FOLD 0 stores alpha for
// the next launch and leaves x alone; FOLD 2 then adds alpha_prev p_prev +
// alpha p), so x is read and written every other iteration; FOLD 1 is the
// plain x += alpha p.
template <typename R, int FOLD>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_cg_update(R* __restrict__ x, R* __restrict__ r,
                                                   const R* __restrict__ p,
                                                   const R* __restrict__ pprev,
                                                   const R* __restrict__ q, long n,
                                                   const int* __restrict__ mask,
                                                   const double* __restrict__ pq_part, int pq_stride,
                                                   int pq_n, const double* __restrict__ dz_part,
                                                   int dz_n, double* __restrict__ rr_out,
                                                   double* __restrict__ alpha_buf,
                                                   const double* __restrict__ alpha_in,
                                                   double* __restrict__ beta_out,
                                                   int* __restrict__ beta_cnt)
{
    pdl_wait();      // p, q and the partials come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    const int rhs = blockIdx.y;
    if (mask != nullptr && mask[rhs] == 0) return;
    const long base = (long)rhs * n;
    const long stride = (long)gridDim.x * blockDim.x;
    // the first element's operands are loaded while alpha is formed
    long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
    Ops<R> cur;
    if (4 * k < n) cur.load(r, q, x, p, pprev, base + 4 * k, FOLD);
    double alpha, alpha_prev = 0.0;
    if (alpha_in != nullptr) {
        // formed once per rhs by the operator's last warp (cg_alpha_epilogue)
        alpha = alpha_in[rhs];
        if (FOLD == 2) alpha_prev = alpha_buf[rhs];
    } else {
        // one warp forms alpha (FP64 sums are slow on this part: doing it
        // in every warp measured slower than the barrier)
        __shared__ double s_alpha, s_alpha_prev;
        if (threadIdx.x < 32) {
            const double pq = warp_sum_array(pq_part + (long)rhs * pq_stride, pq_n);
            const double dz = warp_sum_array(dz_part + (long)rhs * kRedStride, dz_n);
            if (threadIdx.x == 0) {
                s_alpha = cg_ratio(dz, pq);
                if (FOLD == 2) s_alpha_prev = alpha_buf[rhs];
            }
        }
        __syncthreads();
        alpha = s_alpha;
        alpha_prev = s_alpha_prev;
    }
    const R a = (R)alpha;
    R ap = R(0);
    if (FOLD == 2) ap = (R)alpha_prev;
    if (FOLD == 0 && blockIdx.x == 0 && threadIdx.x == 0) alpha_buf[rhs] = alpha;
    // the partial of the new r.r: a compensated float pair in the FP32 path
    // (one FP64 conversion per block), FP64 in the FP64 path
    double acc = 0.0;
    F2 acc2{0.0f, 0.0f};
    // the next element's operands are loaded before the current one is
    // computed (two in flight per thread)
    while (4 * k < n) {
        const long kn = k + stride;
        Ops<R> nxt;
        if (4 * kn < n) nxt.load(r, q, x, p, pprev, base + 4 * kn, FOLD);
        const long o = base + 4 * k;
        if (FOLD != 0) {
            if (FOLD == 2) {
#pragma unroll
                for (int j = 0; j < 4; ++j) cur.x.v[j] = fma(ap, cur.pp.v[j], cur.x.v[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) cur.x.v[j] = fma(a, cur.p.v[j], cur.x.v[j]);
            cur.x.st(x + o);
        }
        R part = R(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cur.r.v[j] = fma(-a, cur.q.v[j], cur.r.v[j]);
            part = fma(cur.r.v[j], cur.r.v[j], part);
        }
        cur.r.st(r + o);
        if constexpr (sizeof(R) == 4)
            acc2 = f2_add(acc2, (float)part);
        else
            acc += (double)part;
        cur = nxt;
        k = kn;
    }
    double s;
    if constexpr (sizeof(R) == 4)
        s = block_sum_f2(acc2);
    else
        s = block_sum(acc);
    if (threadIdx.x == 0) rr_out[(long)rhs * kRedStride + blockIdx.x] = s;
    if (beta_out != nullptr) {
        // the last block of this rhs forms the next beta = (r.r)_new / (r.r)_old
        // from the partial rows, summed as the operator kernel would sum them
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(beta_cnt + rhs, 1) == (int)gridDim.x - 1;
        }
        __syncthreads();
        if (s_last && threadIdx.x < 32) {
            __threadfence();
            const double rn = warp_sum_array_cg(rr_out + (long)rhs * kRedStride, gridDim.x);
            const double ro = warp_sum_array_cg(dz_part + (long)rhs * kRedStride, dz_n);
            if (threadIdx.x == 0) {
                beta_out[rhs] = cg_ratio(rn, ro);
                beta_cnt[rhs] = 0;
            }
        }
    }
}

// Start: r = b (FP64 or rounded to FP32), x = 0; partials of |b|^2 and |r|^2.
template <typename R>
__global__ void __launch_bounds__(256) k_cg_init(const double* __restrict__ b, R* __restrict__ r,
                                                 R* __restrict__ x, long n,
                                                 double* __restrict__ bn_out,
                                                 double* __restrict__ rr_out)
{
    const int rhs = blockIdx.y;
    const long base = (long)rhs * n;
    double ab = 0.0, ar = 0.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x) {
        const double bv = b[base + k];
        const R rv = (R)bv;
        r[base + k] = rv;
        if (x != nullptr) x[base + k] = R(0);
        ab += bv * bv;
        ar += (double)rv * (double)rv;
    }
    double s = block_sum(ab);
    if (threadIdx.x == 0) bn_out[(long)rhs * kRedStride + blockIdx.x] = s;
    __syncthreads();
    s = block_sum(ar);
    if (threadIdx.x == 0) rr_out[(long)rhs * kRedStride + blockIdx.x] = s;
}

// Reliable update, part 1 (mixed only): v += e, e = 0.
__global__ void __launch_bounds__(256) k_fold(double* __restrict__ v, float* __restrict__ e, long n,
                                              const int* __restrict__ mask)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    const int rhs = blockIdx.y;
    if (mask[rhs] == 0) return;
    const long base = (long)rhs * n;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; 4 * k < n;
         k += (long)gridDim.x * blockDim.x) {
        const long o = base + 4 * k;
        V4<double> vv;
        V4<float> ev;
        vv.ld(v + o);
        ev.ld(e + o);
#pragma unroll
        for (int j = 0; j < 4; ++j) vv.v[j] += (double)ev.v[j];
        vv.st(v + o);
        *reinterpret_cast<float4*>(e + o) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Reliable update, part 3: r <- true residual rt (FP64; rounded to FP32 in
// the mixed path); partials of |rt|^2 (true, FP64) and |r|^2 (recursion
// estimate, accumulated in R per group of four).
template <typename R>
__global__ void __launch_bounds__(256) k_recast(const double* rt, R* r, long n,
                                                const int* __restrict__ mask,
                                                double* __restrict__ tr_out,
                                                double* __restrict__ rr_out)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    const int rhs = blockIdx.y;
    if (mask[rhs] == 0) return;
    const long base = (long)rhs * n;
    // |b - M^T M v|^2 in FP64 (the certified true residual); the recast
    // vector's r.r as a compensated float pair in the FP32 path
    double at = 0.0, ar = 0.0;
    F2 ar2{0.0f, 0.0f};
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; 4 * k < n;
         k += (long)gridDim.x * blockDim.x) {
        const long o = base + 4 * k;
        V4<double> tv;
        tv.ld(rt + o);
        V4<R> rv;
        R part = R(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            rv.v[j] = (R)tv.v[j];
            at = fma(tv.v[j], tv.v[j], at);
            part = fma(rv.v[j], rv.v[j], part);
        }
        if ((const void*)r != (const void*)rt) rv.st(r + o);
        if constexpr (sizeof(R) == 4)
            ar2 = f2_add(ar2, (float)part);
        else
            ar += (double)part;
    }
    double s = block_sum(at);
    if (threadIdx.x == 0) tr_out[(long)rhs * kRedStride + blockIdx.x] = s;
    __syncthreads();
    if constexpr (sizeof(R) == 4)
        s = block_sum_f2(ar2);
    else
        s = block_sum(ar);
    if (threadIdx.x == 0) rr_out[(long)rhs * kRedStride + blockIdx.x] = s;
}

// out[rhs] = sum_k bank[rhs*stride + k], k < cnt; one warp per rhs.
__global__ void k_rows(const double* __restrict__ bank, int cnt, int stride, int n_rhs,
                       double* __restrict__ out)
{
    const int rhs = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (rhs >= n_rhs) return;
    const double s = warp_sum_array(bank + (long)rhs * stride, cnt);
    if ((threadIdx.x & 31) == 0) out[rhs] = s;
}

// Block partials of a.b (FP32 vectors, FP64 accumulation) for the flagged rhs.
__global__ void __launch_bounds__(256) k_dot32(const float* __restrict__ a,
                                               const float* __restrict__ b, long n,
                                               const int* __restrict__ mask,
                                               double* __restrict__ out)
{
    const int rhs = blockIdx.y;
    if (mask[rhs] == 0) return;
    const long base = (long)rhs * n;
    double acc = 0.0;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x)
        acc += (double)a[base + k] * (double)b[base + k];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) out[(long)rhs * kRedStride + blockIdx.x] = s;
}

// Merged CG: put the flagged rhs into a start (2) or restart (1) mode.
__global__ void k_set_mode(double* __restrict__ slot, const int* __restrict__ flag, int n_rhs,
                           double mode)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_rhs || flag[k] == 0) return;
    if (mode == 2.0) {   // alpha_prev and gamma_prev are not used; keep them finite
        slot[k * 4 + 0] = 1.0;
        slot[k * 4 + 1] = 1.0;
    }
    slot[k * 4 + 2] = mode;
}


// Restart of the search direction after a reliable update: the kept p is
// re-conjugated against the new residual, beta = -(z, A p) / (p, A p) with
// q = A p. Block partials of (z, q) and (p, q) for the flagged rhs.
template <typename R>
__global__ void __launch_bounds__(256) k_conj_dots(const R* __restrict__ z, const R* __restrict__ p,
                                                   const R* __restrict__ q, long n,
                                                   const int* __restrict__ mask,
                                                   double* __restrict__ zq_out,
                                                   double* __restrict__ pq_out)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    const int rhs = blockIdx.y;
    if (mask[rhs] == 0) return;
    const long base = (long)rhs * n;
    // a group of four in R; the sums as compensated float pairs in the FP32
    // path, FP64 in the FP64 path
    double azq = 0.0, apq = 0.0;
    F2 azq2{0.0f, 0.0f}, apq2{0.0f, 0.0f};
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; 4 * k < n;
         k += (long)gridDim.x * blockDim.x) {
        const long o = base + 4 * k;
        V4<R> zv, pv, qv;
        zv.ld(z + o);
        pv.ld(p + o);
        qv.ld(q + o);
        R szq = R(0), spq = R(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            szq = fma(zv.v[j], qv.v[j], szq);
            spq = fma(pv.v[j], qv.v[j], spq);
        }
        if constexpr (sizeof(R) == 4) {
            azq2 = f2_add(azq2, (float)szq);
            apq2 = f2_add(apq2, (float)spq);
        } else {
            azq += (double)szq;
            apq += (double)spq;
        }
    }
    double t = sizeof(R) == 4 ? block_sum_f2(azq2) : block_sum(azq);
    if (threadIdx.x == 0) zq_out[(long)rhs * kRedStride + blockIdx.x] = t;
    __syncthreads();
    t = sizeof(R) == 4 ? block_sum_f2(apq2) : block_sum(apq);
    if (threadIdx.x == 0) pq_out[(long)rhs * kRedStride + blockIdx.x] = t;
}

// p *= beta = -(z, q) / (p, q) for the flagged rhs (one warp forms beta).
template <typename R>
__global__ void __launch_bounds__(256) k_conj_scale(R* __restrict__ p, long n,
                                                    const int* __restrict__ mask,
                                                    const double* __restrict__ zq_part,
                                                    const double* __restrict__ pq_part, int cnt)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    const int rhs = blockIdx.y;
    if (mask[rhs] == 0) return;
    __shared__ double s_beta;
    if (threadIdx.x < 32) {
        const double zq = warp_sum_array(zq_part + (long)rhs * kRedStride, cnt);
        const double pq = warp_sum_array(pq_part + (long)rhs * kRedStride, cnt);
        if (threadIdx.x == 0) s_beta = cg_ratio(-zq, pq);
    }
    __syncthreads();
    const R bt = (R)s_beta;
    const long base = (long)rhs * n;
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; 4 * k < n;
         k += (long)gridDim.x * blockDim.x) {
        V4<R> pv;
        pv.ld(p + base + 4 * k);
#pragma unroll
        for (int j = 0; j < 4; ++j) pv.v[j] *= bt;
        pv.st(p + base + 4 * k);
    }
}

// dst row = src row (kRedStride partials) for the flagged rhs, so that the
// next beta = sum(src) / sum(dst) is exactly 1.
__global__ void k_copy_rows(const double* __restrict__ src, double* __restrict__ dst,
                            const int* __restrict__ mask, double* __restrict__ beta_out,
                            int beta_n)
{
    pdl_wait();      // inputs may come from the previous kernel of the stream
    const PdlTriggerAtExit pdl_at_exit;
    const int rhs = blockIdx.x;
    if (mask[rhs] == 0) return;
    for (int k = threadIdx.x; k < kRedStride; k += blockDim.x)
        dst[(long)rhs * kRedStride + k] = src[(long)rhs * kRedStride + k];
    if (beta_out != nullptr) {
        // both rows now hold the same partials: the next beta is their ratio,
        // formed as the operator kernel would form it
        __syncthreads();
        if (threadIdx.x < 32) {
            const double v = warp_sum_array(dst + (long)rhs * kRedStride, beta_n);
            if (threadIdx.x == 0) beta_out[rhs] = cg_ratio(v, v);
        }
    }
}


struct Banks {
    double* pq;      // matvec-unit partials of p.q
    double* dz[2];   // alternating partials of r.z (r.r without preconditioner)
    double* tr;      // true residual partials
    double* bn;      // |b|^2 partials
    double* red;     // [max_rhs] reduced per-rhs values
    double* er;      // r.r partials of the preconditioned path
};

Banks banks_of(hol_ctx* c)
{
    Banks b;
    b.pq = c->part;
    b.dz[0] = c->part + 1 * c->part_len;
    b.dz[1] = c->part + 2 * c->part_len;
    b.tr = c->part + 3 * c->part_len;
    b.bn = c->part + 4 * c->part_len;
    b.red = c->part + 5 * c->part_len;
    b.er = c->part + 7 * c->part_len;
    return b;
}

// Reduce bank rows to per-rhs values and copy them to the pinned host buffer.
int rows_to_host(hol_ctx* c, const double* bank, int cnt, int n_rhs, double* host, cudaStream_t s,
                 int stride = kRedStride)
{
    double* red = banks_of(c).red;
    k_rows<<<ceil_div(32L * n_rhs, 256), 256, 0, s>>>(bank, cnt, stride, n_rhs, red);
    HOL_CHECK_LAUNCH("k_rows");
    HOL_CUDA(cudaMemcpyAsync(host, red, n_rhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    HOL_CUDA(cudaStreamSynchronize(s));
    return HOL_OK;
}

// Enqueue per-rhs sums of a bank into a pinned host slot and record `ev`
// when they have landed (the solver keeps the GPU one chunk ahead of these
// reads, see cg_run).
int rows_enqueue(const double* bank, int cnt, int stride, int n_rhs, double* red, double* host,
                 cudaEvent_t ev, cudaStream_t s)
{
    k_rows<<<ceil_div(32L * n_rhs, 256), 256, 0, s>>>(bank, cnt, stride, n_rhs, red);
    HOL_CHECK_LAUNCH("k_rows");
    HOL_CUDA(cudaMemcpyAsync(host, red, n_rhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    HOL_CUDA(cudaEventRecord(ev, s));
    return HOL_OK;
}

struct EventPair {
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int create()
    {
        for (cudaEvent_t& e : ev) HOL_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return HOL_OK;
    }
    ~EventPair()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace

// Blocks per right-hand side of the element-wise CG kernels (256 threads
// each): about four blocks per multiprocessor over all right-hand sides, so
// the update kernel (its two iterations in flight take some 60 registers)
// runs as one resident wave; at least one float4 per thread, at most
// kRedStride blocks (the stride of the partial-sum banks).
int elementwise_blocks(const hol_ctx* c, int n_rhs)
{
    const long v4 = c->n / 4;
    const long most = (v4 + 255) / 256;
    long nb = (4L * c->sms + n_rhs - 1) / (n_rhs > 0 ? n_rhs : 1);
    if (nb > most) nb = most;
    if (nb < 1) nb = 1;
    if (nb > kRedStride) nb = kRedStride;
    return (int)nb;
}

// The CG loop shared by the FP64 and mixed paths, with or without P.
static int cg_run(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
                  int* iters, double* resid, cudaStream_t s)
{
    const bool mixed = (o->prec == HOL_F32);
    const bool pc = o->precond != 0;
    const int prec = mixed ? HOL_F32 : HOL_F64;
    const long n = c->n;
    const int nb2 = elementwise_blocks(c, n_rhs);
    const dim3 g2(nb2, n_rhs);
    const Banks B = banks_of(c);
    const int pstride = matvec_pstride(c);
    const int pq_n = c->T / c->mv_k;
    int pstride64 = 0, pq_n64 = 0;   // the FP64 CG's M keeps its own grouping
    fp64_cg_geom(c, n_rhs, &pstride64, &pq_n64);
    const int dz_n = pc ? precond_tiles(c, prec) : nb2;   // partial count of r.z
    // PCG: the vector update inside the preconditioner's forward transform;
    // the r.r estimate then has one partial per transform tile
    const bool fuse_pc = pc && c->pc_fuse;
    const int est_n = fuse_pc ? dz_n : nb2;
    int* act_d = c->mask;
    int* rel_d = c->mask + c->p.max_rhs;
    int* act_h = c->hflag;
    int* rel_h = c->hflag + c->p.max_rhs;
    double* hb = c->hbuf;
    int rc;
    if (pc && (rc = precond_check_shape(c))) return rc;

    // FP64 path buffers / mixed path buffers
    double* r64 = c->v64a;
    double* p64[2] = {c->v64b, c->v64c};
    double* q64 = c->v64d;
    double* w64 = c->v64e;
    double* z64 = pc ? c->v64f : r64;
    float* r32 = c->v32a;
    float* p32[2] = {c->v32b, c->v32c};
    float* q32 = c->v32d;
    float* e32 = c->v32e;
    float* z32 = pc ? c->v32f : r32;
    double* t64 = c->v64a;   // mixed: M v during a reliable update
    double* rt64 = c->v64b;  // mixed: true residual
    // bank receiving the r.r partials that drive the convergence estimate
    auto est_bank = [&](int cur) { return pc ? B.er : B.dz[cur]; };

    // z = P^{-1} P^{-T} r for every rhs, with the r.z partials in dz[bank]
    auto apply_prec = [&](int bank) -> int {
        timer_start(c, KT_PRECOND, s, (double)n_rhs);
        const int r2 = mixed ? precond_apply_impl(c, HOL_F32, r32, z32, n_rhs, 3, r32, B.dz[bank], s)
                             : precond_apply_impl(c, HOL_F64, r64, z64, n_rhs, 3, r64, B.dz[bank], s);
        timer_stop(c, KT_PRECOND, s);
        return r2;
    };

    HOL_CUDA(cudaMemsetAsync(v, 0, (size_t)n_rhs * n * sizeof(double), s));
    if (mixed)
        k_cg_init<float><<<g2, 256, 0, s>>>(b, r32, e32, n, B.bn, est_bank(0));
    else
        k_cg_init<double><<<g2, 256, 0, s>>>(b, r64, nullptr, n, B.bn, est_bank(0));
    HOL_CHECK_LAUNCH("k_cg_init");
    if (pc && (rc = apply_prec(0))) return rc;
    if ((rc = rows_to_host(c, B.bn, nb2, n_rhs, hb, s))) return rc;
    std::vector<double> bnorm(n_rhs), true_res(n_rhs, 1.0);
    std::vector<int> it(n_rhs, 0), since(n_rhs, 0), done(n_rhs, 0);
    int n_active = 0;
    for (int k = 0; k < n_rhs; ++k) {
        bnorm[k] = sqrt(hb[k]);
        if (!isfinite(bnorm[k])) return set_error(HOL_ENUMERIC, "cg_solve: non-finite |b|");
        if (bnorm[k] == 0.0) {   // v = 0 is exact
            done[k] = 1;
            true_res[k] = 0.0;
            act_h[k] = 0;
        } else {
            act_h[k] = 1;
            ++n_active;
        }
        rel_h[k] = 0;
    }
    HOL_CUDA(cudaMemcpyAsync(act_d, act_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));

    int cur = 0;     // bank holding the current r.z partials
    int pp = 0;      // p buffer holding the current direction
    int first = 1;
    int k_it = 0;
    const int chk = o->check_every > 0 ? o->check_every : 10;
    const int rel_every = (mixed && o->reliable_every > 0) ? o->reliable_every : 1 << 30;
    // valid partial sums in each r.z bank (the fused persistent chunk writes
    // one per unit, the element-wise kernels one per block)
    int cnt[2] = {nb2, nb2};
    const double nd = (double)n;
    // the plain mixed solve runs whole chunks in one cooperative launch when
    // the grid can be resident (persist.cu)
    const bool persistent =
        mixed && !pc && c->persist &&
        launch_cg_persist(c, r32, p32[0], p32[1], e32, n_rhs, act_d, B.pq, B.dz[0], B.dz[1], 0,
                          nb2, nb2, 0, 1, 1, 1, s) == HOL_OK;
    const int nrun = c->T / c->mv_k;
    const long R = c->p.max_rhs;
    EventPair evp;
    if ((rc = evp.create())) return rc;
    int q = 0;              // host slot of the estimate read of this chunk
    bool have_prev = false; // an unexamined estimate of the previous chunk
    while (n_active > 0 && k_it < o->max_iter) {
        int chunk = chk;
        if (chunk > o->max_iter - k_it) chunk = o->max_iter - k_it;
        if (persistent) {
            timer_start(c, KT_OPERATOR, s, (double)chunk * (n_active * nd * 24.0 + nd * 4.0));
            rc = launch_cg_persist(c, r32, p32[0], p32[1], e32, n_rhs, act_d, B.pq, B.dz[0],
                                   B.dz[1], cur, cnt[cur], cnt[1 - cur], pp, first, chunk, 0, s);
            if (rc) return rc;
            timer_stop(c, KT_OPERATOR, s);
            for (int j = 0; j < chunk; ++j) {
                cnt[1 - cur] = nrun;
                cur = 1 - cur;
                pp = 1 - pp;
            }
            first = 0;
        }
        bool pending = false;   // an x update deferred by the previous iteration
        for (int j = 0; j < chunk && !persistent; ++j) {
            double* rr_dst = pc ? B.er : B.dz[1 - cur];
            // x is settled at the end of every chunk (reliable updates read it)
            int fold;
            if (pending) {
                fold = 2;
                pending = false;
            } else if (j == chunk - 1) {
                fold = 1;
            } else {
                fold = 0;
                pending = true;
            }
            const double upd_bytes = fold == 0 ? 12.0 : fold == 1 ? 24.0 : 28.0;   // FP32
            if (mixed) {
                // on the first step beta = 0 and p_old is not yet defined: pass z
                timer_start(c, KT_OPERATOR, s, n_active * nd * 16.0 + nd * 4.0);
                int adone = 0;   // alpha formed by the operator's last warp
                rc = launch_cg_mtm32(c, z32, first ? z32 : p32[pp], p32[1 - pp], q32, n_rhs, act_d,
                                     B.dz[cur], B.dz[1 - cur], kRedStride, dz_n, first, B.pq, s,
                                     (c->handoff & 1) ? c->alpha_now : nullptr, &adone,
                                     (!pc && (c->handoff & 2)) ? c->beta_now : nullptr);
                if (rc) return rc;
                timer_stop(c, KT_OPERATOR, s);
                pp = 1 - pp;
                if (fuse_pc) {   // the update runs inside the preconditioner's forward transform
                    const PcUpd u{e32, p32[pp], p32[1 - pp], q32, act_d, B.pq, pstride, pq_n,
                                  B.dz[cur], dz_n, rr_dst, c->alpha_buf, fold};
                    timer_start(c, KT_PRECOND, s, (double)n_rhs);
                    rc = precond_apply_upd(c, HOL_F32, r32, z32, n_rhs, &u, B.dz[1 - cur], s);
                    timer_stop(c, KT_PRECOND, s);
                    if (rc) return rc;
                    cur = 1 - cur;
                    first = 0;
                    continue;
                }
                timer_start(c, KT_UPDATE, s, n_active * nd * upd_bytes);
                auto* upd = fold == 0 ? k_cg_update<float, 0>
                                      : fold == 1 ? k_cg_update<float, 1> : k_cg_update<float, 2>;
                HOL_CUDA(launch_pdl(c, upd, g2, 256, 0, s, e32, r32, p32[pp], p32[1 - pp], q32, n,
                                    act_d, B.pq, pstride, pq_n, B.dz[cur], dz_n, rr_dst,
                                    c->alpha_buf, adone ? (const double*)c->alpha_now : nullptr,
                                    (!pc && (c->handoff & 2)) ? c->beta_now : nullptr, c->beta_cnt));
            } else {
                BetaSrc bs{B.dz[cur], B.dz[1 - cur], kRedStride, dz_n, first};
                timer_start(c, KT_OPERATOR, s, n_active * nd * 48.0 + nd * 16.0);
                rc = launch_M_upd64(c, z64, first ? z64 : p64[pp], p64[1 - pp], w64, n_rhs, act_d,
                                    bs, B.pq, s);
                if (rc) return rc;
                rc = launch_MT(c, HOL_F64, w64, q64, n_rhs, act_d, s);
                if (rc) return rc;
                timer_stop(c, KT_OPERATOR, s);
                pp = 1 - pp;
                if (fuse_pc) {
                    const PcUpd u{v, p64[pp], p64[1 - pp], q64, act_d, B.pq, pstride64, pq_n64,
                                  B.dz[cur], dz_n, rr_dst, c->alpha_buf, fold};
                    timer_start(c, KT_PRECOND, s, (double)n_rhs);
                    rc = precond_apply_upd(c, HOL_F64, r64, z64, n_rhs, &u, B.dz[1 - cur], s);
                    timer_stop(c, KT_PRECOND, s);
                    if (rc) return rc;
                    cur = 1 - cur;
                    first = 0;
                    continue;
                }
                timer_start(c, KT_UPDATE, s, n_active * nd * 2.0 * upd_bytes);
                auto* upd = fold == 0 ? k_cg_update<double, 0>
                                      : fold == 1 ? k_cg_update<double, 1> : k_cg_update<double, 2>;
                HOL_CUDA(launch_pdl(c, upd, g2, 256, 0, s, v, r64, p64[pp], p64[1 - pp], q64, n,
                                    act_d, B.pq, pstride64, pq_n64, B.dz[cur], dz_n, rr_dst,
                                    c->alpha_buf, (const double*)nullptr, (double*)nullptr,
                                    (int*)nullptr));
            }
            HOL_CHECK_LAUNCH("k_cg_update");
            timer_stop(c, KT_UPDATE, s);
            if (pc && (rc = apply_prec(1 - cur))) return rc;
            cur = 1 - cur;
            first = 0;
        }
        k_it += chunk;
        // The recursive residual of this chunk is read asynchronously. Unless
        // a reliable update is due by count, the next chunk is launched at
        // once and this estimate is examined one chunk later (the GPU never
        // waits for the host); an estimate below tol makes the end of the
        // chunk then in flight a synchronisation point.
        double* est_h = hb + (2 + q) * R;
        if ((rc = rows_enqueue(est_bank(cur), pc ? est_n : cnt[cur], kRedStride, n_rhs,
                               B.red + (1 + q) * R, est_h, evp.ev[q], s)))
            return rc;
        bool sync = k_it >= o->max_iter;
        for (int k = 0; k < n_rhs; ++k) {
            if (!act_h[k]) continue;
            it[k] += chunk;
            since[k] += chunk;
            if (since[k] >= rel_every) sync = true;
        }
        if (!sync && have_prev) {
            HOL_CUDA(cudaEventSynchronize(evp.ev[1 - q]));
            const double* prev = hb + (2 + (1 - q)) * R;
            for (int k = 0; k < n_rhs; ++k) {
                if (!act_h[k]) continue;
                const double est = sqrt(prev[k]) / bnorm[k];
                if (!isfinite(est))
                    return set_error(HOL_ENUMERIC,
                                     "cg_solve: non-finite residual (rhs %d, iter %d)", k,
                                     it[k] - chunk);
                if (est < o->tol) sync = true;
            }
        }
        if (!sync) {
            have_prev = true;
            q = 1 - q;
            continue;
        }
        HOL_CUDA(cudaEventSynchronize(evp.ev[q]));
        have_prev = false;
        int n_rel = 0;
        for (int k = 0; k < n_rhs; ++k) {
            rel_h[k] = 0;
            if (!act_h[k]) continue;
            const double est = sqrt(est_h[k]) / bnorm[k];
            if (!isfinite(est))
                return set_error(HOL_ENUMERIC, "cg_solve: non-finite residual (rhs %d, iter %d)",
                                 k, it[k]);
            if (est < o->tol || since[k] >= rel_every || k_it >= o->max_iter) {
                rel_h[k] = 1;
                ++n_rel;
            }
        }
        if (n_rel == 0) continue;
        if (persistent)   // bank rows of all rhs must keep one partial count
            for (int k = 0; k < n_rhs; ++k) rel_h[k] = act_h[k];
        // reliable update / convergence certification for the flagged rhs
        HOL_CUDA(cudaMemcpyAsync(rel_d, rel_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
        if (mixed) {
            HOL_CUDA(launch_pdl(c, k_fold, g2, 256, 0, s, v, e32, n, rel_d));
            HOL_CHECK_LAUNCH("k_fold");
            if ((rc = launch_M(c, HOL_F64, v, t64, n_rhs, rel_d, nullptr, s))) return rc;
            if ((rc = launch_MT_resid64(c, t64, b, rt64, n_rhs, rel_d, s))) return rc;
            HOL_CUDA(launch_pdl(c, k_recast<float>, g2, 256, 0, s, rt64, r32, n, rel_d, B.tr,
                                est_bank(cur)));
        } else {
            if ((rc = launch_M(c, HOL_F64, v, w64, n_rhs, rel_d, nullptr, s))) return rc;
            if ((rc = launch_MT_resid64(c, w64, b, r64, n_rhs, rel_d, s))) return rc;
            HOL_CUDA(launch_pdl(c, k_recast<double>, g2, 256, 0, s, r64, r64, n, rel_d, B.tr,
                                est_bank(cur)));
        }
        HOL_CHECK_LAUNCH("k_recast");
        if (!pc) cnt[cur] = nb2;   // k_recast wrote block partials into the current bank
        // the new r changes r.z: recompute z (all rhs; the unchanged ones get
        // the same z again)
        if (pc && (rc = apply_prec(cur))) return rc;
        // keep the direction, re-conjugated against the new z:
        // p *= -(z, A p) / (p, A p) and the next beta forced to 1. Keeping
        // p with beta = (r.z)_new / (r.z)_old instead lets the old direction
        // swamp the new residual in FP32 when the recursive residual had
        // drifted far below the true one.
        {
            double* cj0 = c->part + 8 * c->part_len;
            double* cj1 = c->part + 9 * c->part_len;
            if (mixed) {
                if (persistent &&   // the persistent chunk keeps q in shared memory
                    (rc = launch_cg_mtm32(c, p32[pp], p32[pp], nullptr, q32, n_rhs, rel_d, nullptr,
                                          nullptr, 0, 0, 1, nullptr, s)))
                    return rc;
                HOL_CUDA(launch_pdl(c, k_conj_dots<float>, g2, 256, 0, s, z32, p32[pp], q32, n,
                                    rel_d, cj0, cj1));
                HOL_CHECK_LAUNCH("k_conj_dots");
                HOL_CUDA(launch_pdl(c, k_conj_scale<float>, g2, 256, 0, s, p32[pp], n, rel_d, cj0,
                                    cj1, nb2));
            } else {
                HOL_CUDA(launch_pdl(c, k_conj_dots<double>, g2, 256, 0, s, z64, p64[pp], q64, n,
                                    rel_d, cj0, cj1));
                HOL_CHECK_LAUNCH("k_conj_dots");
                HOL_CUDA(launch_pdl(c, k_conj_scale<double>, g2, 256, 0, s, p64[pp], n, rel_d, cj0,
                                    cj1, nb2));
            }
            HOL_CHECK_LAUNCH("k_conj_scale");
            HOL_CUDA(launch_pdl(c, k_copy_rows, n_rhs, 256, 0, s, B.dz[cur], B.dz[1 - cur], rel_d,
                                (mixed && !pc && (c->handoff & 2)) ? c->beta_now : nullptr, dz_n));
            HOL_CHECK_LAUNCH("k_copy_rows");
            cnt[1 - cur] = cnt[cur];
        }
        if ((rc = rows_to_host(c, B.tr, nb2, n_rhs, hb, s))) return rc;
        int changed = 0;
        for (int k = 0; k < n_rhs; ++k) {
            if (!rel_h[k]) continue;
            since[k] = 0;
            true_res[k] = sqrt(hb[k]) / bnorm[k];
            if (!isfinite(true_res[k]))
                return set_error(HOL_ENUMERIC, "cg_solve: non-finite true residual (rhs %d)", k);
            if (true_res[k] < o->tol) {
                done[k] = 1;
                act_h[k] = 0;
                --n_active;
                changed = 1;
            }
        }
        if (changed)
            HOL_CUDA(cudaMemcpyAsync(act_d, act_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    HOL_CUDA(cudaStreamSynchronize(s));
    int all = 1;
    for (int k = 0; k < n_rhs; ++k) {
        if (iters) iters[k] = it[k];
        if (resid) resid[k] = true_res[k];
        all &= done[k];
    }
    if (!all)
        return set_error(HOL_ENOTCONV, "cg_solve: not converged within %d iterations", o->max_iter);
    return HOL_OK;
}


// Mixed plain CG with one fused kernel per iteration (k_cg_fused in
// matvec.cu): the vector update of iteration i and the operator of
// iteration i + 1 share one pass over the vectors, and beta comes from the
// exact expansion |r - alpha q|^2 = r.r - 2 alpha r.q + alpha^2 q.q of
// partials the previous pass accumulated. r, p and q are double buffered by
// iteration parity (neighbouring units read the tau halo); x is updated in
// place every iteration. Polling, reliable updates and certification work as
// in cg_run; a reliable update replaces r by the true residual, builds the
// direction from it and the previous direction (p = r + beta p_prev with
// beta = -(r, A p_prev) / (p_prev, A p_prev)), recomputes q = A p and the
// partials for the flagged rhs.
static int cg_run_fused(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
                        int* iters, double* resid, cudaStream_t s)
{
    const long n = c->n;
    const int nb2 = elementwise_blocks(c, n_rhs);
    const dim3 g2(nb2, n_rhs);
    const Banks B = banks_of(c);
    const int pstride = matvec_pstride(c);
    const int nrun = c->T / c->mv_k;
    int* act_d = c->mask;
    int* rel_d = c->mask + c->p.max_rhs;
    int* act_h = c->hflag;
    int* rel_h = c->hflag + c->p.max_rhs;
    double* hb = c->hbuf;
    const long R = c->p.max_rhs;
    int rc;
    float* Rv[2] = {c->v32a, c->v32g};
    float* Pv[2] = {c->v32b, c->v32c};
    float* Qv[2] = {c->v32d, c->v32h};
    float* X = c->v32e;
    double* t64 = c->v64a;
    double* rt64 = c->v64b;
    auto bank = [&](int k) { return c->part + (long)k * c->part_len; };
    double* GG[2] = {bank(12), bank(13)};
    double* PQ[2] = {bank(14), bank(15)};
    double* RQ[2] = {bank(16), bank(17)};
    double* QQ[2] = {bank(18), bank(19)};
    double* cj0 = bank(8);
    double* cj1 = bank(9);
    const double nd = (double)n;

    HOL_CUDA(cudaMemsetAsync(v, 0, (size_t)n_rhs * n * sizeof(double), s));
    k_cg_init<float><<<g2, 256, 0, s>>>(b, Rv[0], X, n, B.bn, cj1);
    HOL_CHECK_LAUNCH("k_cg_init");
    if ((rc = rows_to_host(c, B.bn, nb2, n_rhs, hb, s))) return rc;
    std::vector<double> bnorm(n_rhs), true_res(n_rhs, 1.0);
    std::vector<int> it(n_rhs, 0), since(n_rhs, 0), done(n_rhs, 0);
    int n_active = 0;
    for (int k = 0; k < n_rhs; ++k) {
        bnorm[k] = sqrt(hb[k]);
        if (!isfinite(bnorm[k])) return set_error(HOL_ENUMERIC, "cg_solve: non-finite |b|");
        act_h[k] = bnorm[k] != 0.0;
        if (!act_h[k]) {   // v = 0 is exact
            done[k] = 1;
            true_res[k] = 0.0;
        }
        n_active += act_h[k];
        rel_h[k] = 0;
    }
    HOL_CUDA(cudaMemcpyAsync(act_d, act_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
    if (n_active > 0) {   // p = r, q = A p and the partials of iteration 0
        if ((rc = launch_cg_mtm32(c, Rv[0], Rv[0], Pv[0], Qv[0], n_rhs, act_d, nullptr, nullptr,
                                  0, 0, 1, PQ[0], s)))
            return rc;
        if ((rc = launch_unit_dots(c, Rv[0], Qv[0], n_rhs, act_d, GG[0], RQ[0], QQ[0], s)))
            return rc;
    }
    const int chk = o->check_every > 0 ? o->check_every : 10;
    const int rel_every = o->reliable_every > 0 ? o->reliable_every : 1 << 30;
    EventPair evp;
    if ((rc = evp.create())) return rc;
    int q = 0;
    bool have_prev = false;
    int a = 0;   // parity of the current r, p, q and partials
    int k_it = 0;
    while (n_active > 0 && k_it < o->max_iter) {
        int chunk = chk;
        if (chunk > o->max_iter - k_it) chunk = o->max_iter - k_it;
        for (int j = 0; j < chunk; ++j) {
            const int z = 1 - a;
            FusedPartials fp{GG[a], PQ[a], RQ[a], QQ[a], GG[z], PQ[z], RQ[z], QQ[z]};
            timer_start(c, KT_OPERATOR, s, n_active * nd * 32.0 + nd * 4.0);
            rc = launch_cg_fused(c, Rv[a], Qv[a], Pv[a], X, Rv[z], Pv[z], Qv[z], n_rhs, act_d, fp,
                                 s);
            if (rc) return rc;
            timer_stop(c, KT_OPERATOR, s);
            a = z;
        }
        k_it += chunk;
        // estimate read one chunk behind, as in cg_run
        double* est_h = hb + (2 + q) * R;
        if ((rc = rows_enqueue(GG[a], nrun, pstride, n_rhs, B.red + (1 + q) * R, est_h, evp.ev[q],
                               s)))
            return rc;
        bool sync = k_it >= o->max_iter;
        for (int k = 0; k < n_rhs; ++k) {
            if (!act_h[k]) continue;
            it[k] += chunk;
            since[k] += chunk;
            if (since[k] >= rel_every) sync = true;
        }
        if (!sync && have_prev) {
            HOL_CUDA(cudaEventSynchronize(evp.ev[1 - q]));
            const double* prev = hb + (2 + (1 - q)) * R;
            for (int k = 0; k < n_rhs; ++k) {
                if (!act_h[k]) continue;
                const double est = sqrt(prev[k]) / bnorm[k];
                if (!isfinite(est))
                    return set_error(HOL_ENUMERIC,
                                     "cg_solve: non-finite residual (rhs %d, iter %d)", k,
                                     it[k] - chunk);
                if (est < o->tol) sync = true;
            }
        }
        if (!sync) {
            have_prev = true;
            q = 1 - q;
            continue;
        }
        HOL_CUDA(cudaEventSynchronize(evp.ev[q]));
        have_prev = false;
        int n_rel = 0;
        for (int k = 0; k < n_rhs; ++k) {
            rel_h[k] = 0;
            if (!act_h[k]) continue;
            const double est = sqrt(est_h[k]) / bnorm[k];
            if (!isfinite(est))
                return set_error(HOL_ENUMERIC, "cg_solve: non-finite residual (rhs %d, iter %d)",
                                 k, it[k]);
            if (est < o->tol || since[k] >= rel_every || k_it >= o->max_iter) {
                rel_h[k] = 1;
                ++n_rel;
            }
        }
        if (n_rel == 0) continue;
        const int z = 1 - a;
        HOL_CUDA(cudaMemcpyAsync(rel_d, rel_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
        HOL_CUDA(launch_pdl(c, k_fold, g2, 256, 0, s, v, X, n, rel_d));
        HOL_CHECK_LAUNCH("k_fold");
        if ((rc = launch_M(c, HOL_F64, v, t64, n_rhs, rel_d, nullptr, s))) return rc;
        if ((rc = launch_MT_resid64(c, t64, b, rt64, n_rhs, rel_d, s))) return rc;
        HOL_CUDA(launch_pdl(c, k_recast<float>, g2, 256, 0, s, rt64, Rv[a], n, rel_d, B.tr, cj1));
        HOL_CHECK_LAUNCH("k_recast");
        // The stored p (parity a) already contains the old r; the direction
        // the last pass stepped along, p_prev with q_prev = A p_prev, is still
        // in parity z. New direction: p = r + beta p_prev with
        // beta = -(r, q_prev) / (p_prev, q_prev) (p_prev is scaled by beta,
        // then p = r + p_prev from identical partial rows), q = A p and its
        // p.q partials, written to parity a; then the r.r, r.q, q.q partials.
        HOL_CUDA(launch_pdl(c, k_conj_dots<float>, g2, 256, 0, s, Rv[a], Pv[z], Qv[z], n, rel_d,
                            cj0, cj1));
        HOL_CHECK_LAUNCH("k_conj_dots");
        HOL_CUDA(launch_pdl(c, k_conj_scale<float>, g2, 256, 0, s, Pv[z], n, rel_d, cj0, cj1, nb2));
        HOL_CHECK_LAUNCH("k_conj_scale");
        if ((rc = launch_cg_mtm32(c, Rv[a], Pv[z], Pv[a], Qv[a], n_rhs, rel_d, B.tr, B.tr,
                                  kRedStride, nb2, 0, PQ[a], s)))
            return rc;
        if ((rc = launch_unit_dots(c, Rv[a], Qv[a], n_rhs, rel_d, GG[a], RQ[a], QQ[a], s)))
            return rc;
        if ((rc = rows_to_host(c, B.tr, nb2, n_rhs, hb, s))) return rc;
        int changed = 0;
        for (int k = 0; k < n_rhs; ++k) {
            if (!rel_h[k]) continue;
            since[k] = 0;
            true_res[k] = sqrt(hb[k]) / bnorm[k];
            if (!isfinite(true_res[k]))
                return set_error(HOL_ENUMERIC, "cg_solve: non-finite true residual (rhs %d)", k);
            if (true_res[k] < o->tol) {
                done[k] = 1;
                act_h[k] = 0;
                --n_active;
                changed = 1;
            }
        }
        if (changed)
            HOL_CUDA(cudaMemcpyAsync(act_d, act_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    HOL_CUDA(cudaStreamSynchronize(s));
    int all = 1;
    for (int k = 0; k < n_rhs; ++k) {
        if (iters) iters[k] = it[k];
        if (resid) resid[k] = true_res[k];
        all &= done[k];
    }
    if (!all)
        return set_error(HOL_ENOTCONV, "cg_solve: not converged within %d iterations", o->max_iter);
    return HOL_OK;
}

// Mixed plain CG with one fused kernel per iteration (k_cg_merged in
// matvec.cu, Chronopoulos-Gear recurrences). The FP32 state per rhs is
// x (the increment e), r, w = A r, p, s = A p; r, w, p, s are double
// buffered by iteration parity because neighbouring units read the tau halo
// of r and w. The x update of an iteration may be deferred to the next one
// (which reads p_old anyway), so x is touched every other iteration; the
// last iteration of every polling chunk settles it. Reliable updates work
// as in cg_run; the restarted rhs get w = A r and s_old = A p_old
// recomputed in FP32 with rho = r.s_old and pi = p_old.s_old, so the kept
// direction is re-conjugated (beta = -rho / pi) and alpha is formed from
// exact inner products (mode 1).
static int cg_run_merged(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
                         int* iters, double* resid, cudaStream_t s)
{
    const long n = c->n;
    const int nb2 = elementwise_blocks(c, n_rhs);
    const dim3 g2(nb2, n_rhs);
    const Banks B = banks_of(c);
    const int pstride = matvec_pstride(c);
    const int nrun = c->T / c->mv_k;
    int* act_d = c->mask;
    int* rel_d = c->mask + c->p.max_rhs;
    int* act_h = c->hflag;
    int* rel_h = c->hflag + c->p.max_rhs;
    double* hb = c->hbuf;
    int rc;
    double* G[2] = {B.dz[0], B.dz[1]};
    double* D[2] = {B.pq, c->part + 11 * c->part_len};
    double* Gr = c->part + 8 * c->part_len;
    double* PI = c->part + 9 * c->part_len;
    double* RHO = c->part + 10 * c->part_len;
    float* e = c->v32e;
    float* R[2] = {c->v32a, c->v32g};
    float* W[2] = {c->v32d, c->v32h};
    float* P[2] = {c->v32b, c->v32c};
    float* S[2] = {c->v32f, c->v32i};
    double* slot[2] = {c->cgs, c->cgs + 4 * c->p.max_rhs};
    double* t64 = c->v64a;
    double* rt64 = c->v64b;
    const double nd = (double)n;

    HOL_CUDA(cudaMemsetAsync(v, 0, (size_t)n_rhs * n * sizeof(double), s));
    k_cg_init<float><<<g2, 256, 0, s>>>(b, R[0], e, n, B.bn, Gr);
    HOL_CHECK_LAUNCH("k_cg_init");
    if ((rc = rows_to_host(c, B.bn, nb2, n_rhs, hb, s))) return rc;
    std::vector<double> bnorm(n_rhs), true_res(n_rhs, 1.0);
    std::vector<int> it(n_rhs, 0), since(n_rhs, 0), done(n_rhs, 0);
    int n_active = 0;
    for (int k = 0; k < n_rhs; ++k) {
        bnorm[k] = sqrt(hb[k]);
        if (!isfinite(bnorm[k])) return set_error(HOL_ENUMERIC, "cg_solve: non-finite |b|");
        act_h[k] = bnorm[k] != 0.0;
        if (!act_h[k]) {   // v = 0 is exact
            done[k] = 1;
            true_res[k] = 0.0;
        }
        n_active += act_h[k];
        rel_h[k] = 0;
    }
    HOL_CUDA(cudaMemcpyAsync(act_d, act_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
    if (n_active > 0) {   // w = A r, delta partials; start mode
        if ((rc = launch_cg_mtm32(c, R[0], R[0], nullptr, W[0], n_rhs, act_d, nullptr, nullptr, 0,
                                  0, 1, D[0], s)))
            return rc;
        k_set_mode<<<ceil_div(n_rhs, 128), 128, 0, s>>>(slot[1], act_d, n_rhs, 2.0);
        HOL_CHECK_LAUNCH("k_set_mode");
    }
    const int chk = o->check_every > 0 ? o->check_every : 10;
    const int rel_every = o->reliable_every > 0 ? o->reliable_every : 1 << 30;
    long i = 0;   // merged iterations so far (parity selects the buffers)
    int k_it = 0;
    while (n_active > 0 && k_it < o->max_iter) {
        int chunk = chk;
        if (chunk > o->max_iter - k_it) chunk = o->max_iter - k_it;
        bool pending = false;
        for (int j = 0; j < chunk; ++j) {
            const int a = (int)(i & 1), z = 1 - a;
            MergedScal sc;
            sc.slot_in = slot[z];
            sc.slot_out = slot[a];
            sc.g_in = G[a];
            sc.d_in = D[a];
            sc.g_out = G[z];
            sc.d_out = D[z];
            sc.gr = Gr;
            sc.rho = RHO;
            sc.e_n = nb2;
            sc.pi = PI;
            if (pending) {
                sc.fold = 2;
                pending = false;
            } else if (j == chunk - 1) {
                sc.fold = 1;
            } else {
                sc.fold = 0;
                pending = true;
            }
            timer_start(c, KT_OPERATOR, s,
                        n_active * nd * (32.0 + (sc.fold ? 8.0 : 0.0)) + nd * 4.0);
            rc = launch_cg_merged(c, R[a], W[a], P[z], S[z], e, P[a], S[a], R[z], W[z], n_rhs,
                                  act_d, sc, s);
            if (rc) return rc;
            timer_stop(c, KT_OPERATOR, s);
            ++i;
        }
        k_it += chunk;
        const int a = (int)(i & 1), z = 1 - a;   // the next iteration's parity
        if ((rc = rows_to_host(c, G[a], nrun, n_rhs, hb, s, pstride))) return rc;
        int n_rel = 0;
        for (int k = 0; k < n_rhs; ++k) {
            rel_h[k] = 0;
            if (!act_h[k]) continue;
            it[k] += chunk;
            since[k] += chunk;
            const double est = sqrt(hb[k]) / bnorm[k];
            if (!isfinite(est))
                return set_error(HOL_ENUMERIC, "cg_solve: non-finite residual (rhs %d, iter %d)",
                                 k, it[k]);
            if (est < o->tol || since[k] >= rel_every || k_it >= o->max_iter) {
                rel_h[k] = 1;
                ++n_rel;
            }
        }
        if (n_rel == 0) continue;
        HOL_CUDA(cudaMemcpyAsync(rel_d, rel_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
        HOL_CUDA(launch_pdl(c, k_fold, g2, 256, 0, s, v, e, n, rel_d));
        HOL_CHECK_LAUNCH("k_fold");
        if ((rc = launch_M(c, HOL_F64, v, t64, n_rhs, rel_d, nullptr, s))) return rc;
        if ((rc = launch_MT_resid64(c, t64, b, rt64, n_rhs, rel_d, s))) return rc;
        HOL_CUDA(launch_pdl(c, k_recast<float>, g2, 256, 0, s, rt64, R[a], n, rel_d, B.tr, Gr));
        HOL_CHECK_LAUNCH("k_recast");
        // w = A r for the new r, s_old = A p_old, rho = r.s_old
        if ((rc = launch_cg_mtm32(c, R[a], R[a], nullptr, W[a], n_rhs, rel_d, nullptr, nullptr, 0,
                                  0, 1, D[a], s)))
            return rc;
        if ((rc = launch_cg_mtm32(c, P[z], P[z], nullptr, S[z], n_rhs, rel_d, nullptr, nullptr, 0,
                                  0, 1, PI, s)))
            return rc;
        k_dot32<<<g2, 256, 0, s>>>(R[a], S[z], n, rel_d, RHO);
        HOL_CHECK_LAUNCH("k_dot32");
        k_set_mode<<<ceil_div(n_rhs, 128), 128, 0, s>>>(slot[z], rel_d, n_rhs, 1.0);
        HOL_CHECK_LAUNCH("k_set_mode");
        if ((rc = rows_to_host(c, B.tr, nb2, n_rhs, hb, s))) return rc;
        int changed = 0;
        for (int k = 0; k < n_rhs; ++k) {
            if (!rel_h[k]) continue;
            since[k] = 0;
            true_res[k] = sqrt(hb[k]) / bnorm[k];
            if (!isfinite(true_res[k]))
                return set_error(HOL_ENUMERIC, "cg_solve: non-finite true residual (rhs %d)", k);
            if (true_res[k] < o->tol) {
                done[k] = 1;
                act_h[k] = 0;
                --n_active;
                changed = 1;
            }
        }
        if (changed)
            HOL_CUDA(cudaMemcpyAsync(act_d, act_h, n_rhs * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    HOL_CUDA(cudaStreamSynchronize(s));
    int all = 1;
    for (int k = 0; k < n_rhs; ++k) {
        if (iters) iters[k] = it[k];
        if (resid) resid[k] = true_res[k];
        all &= done[k];
    }
    if (!all)
        return set_error(HOL_ENOTCONV, "cg_solve: not converged within %d iterations", o->max_iter);
    return HOL_OK;
}


// ---------------------------------------------------------------------------
// Graph-captured CG: the decisions cg_run takes on the host after every chunk
// of check_every iterations (the one-chunk-late look at the recursive
// residual, reliable updates by count and by estimate, certification by the
// FP64 true residual) are taken by one-block kernels on the device instead,
// in the same order and with the same reductions (warp_sum_array of the same
// partial-sum rows), so the kernel sequence and the result are the same as
// cg_run's. The chunk loop is a conditional WHILE node of the graph and the
// reliable update a conditional IF node inside it; nothing waits on the host.
// ---------------------------------------------------------------------------
namespace {

constexpr int kDcgThreads = 1024;

__global__ void __launch_bounds__(kDcgThreads) k_dcg_start(const double* __restrict__ bn, int cnt,
                                                           int n_rhs, int* __restrict__ act,
                                                           int* __restrict__ rel, DcgState d)
{
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        d.g[DCG_KIT] = 0;
        d.g[DCG_HAVE_PREV] = 0;
        d.g[DCG_ERR] = 0;
        d.g[DCG_ERR_RHS] = -1;
        d.g[DCG_LOOPS] = 0;
    }
    __syncthreads();
    for (int k = wid; k < n_rhs; k += kDcgThreads / 32) {
        const double s = warp_sum_array(bn + (long)k * kRedStride, cnt);
        if (lane == 0) {
            const double nb = sqrt(s);
            d.bnorm[k] = nb;
            if (!isfinite(nb)) atomicExch(&d.g[DCG_ERR], HOL_ENUMERIC);
            const int z = nb == 0.0;   // v = 0 is exact
            d.done[k] = z;
            d.tres[k] = z ? 0.0 : 1.0;
            act[k] = z ? 0 : 1;
            rel[k] = 0;
            d.it[k] = 0;
            d.since[k] = 0;
            d.prev[k] = 0.0;
        }
    }
}

// End of a chunk: the iteration counts, then whether this chunk is a
// synchronisation point (a reliable update due by count, the iteration cap,
// or the previous chunk's estimate below tol); if it is, the rhs to update
// are flagged from this chunk's estimate, else the estimate is kept for the
// next chunk. Sets the IF condition of the reliable update.
__global__ void __launch_bounds__(kDcgThreads) k_dcg_decide(const double* __restrict__ est_bank,
                                                            int cnt, int n_rhs, int chunk, double tol,
                                                            int rel_every, int max_iter,
                                                            const int* __restrict__ act,
                                                            int* __restrict__ rel, DcgState d,
                                                            cudaGraphConditionalHandle h_if)
{
    __shared__ int s_sync, s_nrel, s_err;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kit = d.g[DCG_KIT] + chunk;
    const int have_prev = d.g[DCG_HAVE_PREV];
    if (threadIdx.x == 0) {
        s_sync = kit >= max_iter;
        s_nrel = 0;
        s_err = 0;
    }
    __syncthreads();
    for (int k = wid; k < n_rhs; k += kDcgThreads / 32) {
        const double s = warp_sum_array(est_bank + (long)k * kRedStride, cnt);
        if (lane == 0) {
            d.cur[k] = s;
            if (act[k]) {
                d.it[k] += chunk;
                d.since[k] += chunk;
                if (d.since[k] >= rel_every) s_sync = 1;
            }
        }
    }
    __syncthreads();
    if (!s_sync && have_prev) {
        for (int k = threadIdx.x; k < n_rhs; k += kDcgThreads) {
            if (!act[k]) continue;
            const double est = sqrt(d.prev[k]) / d.bnorm[k];
            if (!isfinite(est)) {
                s_err = 1;
                d.g[DCG_ERR_RHS] = k;   // one failing rhs (any); reported only
            } else if (est < tol) {
                s_sync = 1;
            }
        }
    }
    __syncthreads();
    if (s_err) {
        if (threadIdx.x == 0) {
            d.g[DCG_ERR] = HOL_ENUMERIC;
            d.g[DCG_KIT] = kit;
            cudaGraphSetConditional(h_if, 0u);
        }
        return;
    }
    if (!s_sync) {
        for (int k = threadIdx.x; k < n_rhs; k += kDcgThreads) {
            d.prev[k] = d.cur[k];
            rel[k] = 0;
        }
        if (threadIdx.x == 0) {
            d.g[DCG_HAVE_PREV] = 1;
            d.g[DCG_KIT] = kit;
            cudaGraphSetConditional(h_if, 0u);
        }
        return;
    }
    for (int k = threadIdx.x; k < n_rhs; k += kDcgThreads) {
        int flag = 0;
        if (act[k]) {
            const double est = sqrt(d.cur[k]) / d.bnorm[k];
            if (!isfinite(est)) {
                s_err = 1;
            } else if (est < tol || d.since[k] >= rel_every || kit >= max_iter) {
                flag = 1;
                atomicAdd(&s_nrel, 1);
            }
        }
        rel[k] = flag;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.g[DCG_HAVE_PREV] = 0;
        d.g[DCG_KIT] = kit;
        if (s_err) d.g[DCG_ERR] = HOL_ENUMERIC;
        cudaGraphSetConditional(h_if, (s_nrel > 0 && !s_err) ? 1u : 0u);
    }
}

// After a reliable update: the true residual of the flagged rhs; converged
// ones leave the active set.
__global__ void __launch_bounds__(kDcgThreads) k_dcg_finish(const double* __restrict__ tr, int cnt,
                                                            int n_rhs, double tol,
                                                            int* __restrict__ act,
                                                            const int* __restrict__ rel,
                                                            DcgState d)
{
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = wid; k < n_rhs; k += kDcgThreads / 32) {
        if (!rel[k]) continue;
        const double s = warp_sum_array(tr + (long)k * kRedStride, cnt);
        if (lane == 0) {
            d.since[k] = 0;
            const double t = sqrt(s) / d.bnorm[k];
            d.tres[k] = t;
            if (!isfinite(t)) {
                atomicExch(&d.g[DCG_ERR], HOL_ENUMERIC);
            } else if (t < tol) {
                d.done[k] = 1;
                act[k] = 0;
            }
        }
    }
}

// Loop condition: rhs still active, iterations below the cap, no error, and
// a hard bound on the number of chunks (so the loop ends whatever happens).
// When the loop ends unconverged or with an error, the sticky failure flag
// is raised.
__global__ void __launch_bounds__(kDcgThreads) k_dcg_cond(const int* __restrict__ act, int n_rhs,
                                                          int max_iter, int max_loops, DcgState d,
                                                          cudaGraphConditionalHandle h_while)
{
    __shared__ int s_act;
    if (threadIdx.x == 0) s_act = 0;
    __syncthreads();
    int a = 0;
    for (int k = threadIdx.x; k < n_rhs; k += kDcgThreads) a |= act[k];
    if (a) s_act = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int loops = d.g[DCG_LOOPS] + 1;
        d.g[DCG_LOOPS] = loops;
        const int err = d.g[DCG_ERR];
        const int go = s_act && d.g[DCG_KIT] < max_iter && !err && loops <= max_loops;
        if (!go && (s_act || err)) d.g[DCG_STICKY] = err ? err : HOL_ENOTCONV;
        cudaGraphSetConditional(h_while, go ? 1u : 0u);
    }
}

}  // namespace

int cond_handle(cudaStream_t s, cudaGraphConditionalHandle* h)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    HOL_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
    if (st != cudaStreamCaptureStatusActive || !g)
        return set_error(HOL_EINVAL, "graph solve: stream is not capturing");
    HOL_CUDA(cudaGraphConditionalHandleCreate(h, g, 0u, cudaGraphCondAssignDefault));
    return HOL_OK;
}

int cond_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
              cudaGraph_t* body)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    HOL_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edges, &nd));
    if (st != cudaStreamCaptureStatusActive || !g)
        return set_error(HOL_EINVAL, "graph solve: stream is not capturing");
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    HOL_CUDA(cudaGraphAddNode(&node, g, deps, edges, nd, &np));
    *body = np.conditional.phGraph_out[0];
    HOL_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies));
    return HOL_OK;
}

int cg_run_dev(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
               cudaStream_t s)
{
    const bool mixed = (o->prec == HOL_F32);
    const bool pc = o->precond != 0;
    const long n = c->n;
    const int nb2 = elementwise_blocks(c, n_rhs);
    const dim3 g2(nb2, n_rhs);
    const Banks B = banks_of(c);
    const int pstride = matvec_pstride(c);
    const int pq_n = c->T / c->mv_k;
    int pstride64 = 0, pq_n64 = 0;   // the FP64 CG's M keeps its own grouping
    fp64_cg_geom(c, n_rhs, &pstride64, &pq_n64);
    const int dz_n = pc ? precond_tiles(c, mixed ? HOL_F32 : HOL_F64) : nb2;
    const bool fuse_pc = pc && c->pc_fuse;   // as in cg_run
    const int est_n = fuse_pc ? dz_n : nb2;
    int* act_d = c->mask;
    int* rel_d = c->mask + c->p.max_rhs;
    const DcgState d = dcg_state(c);
    const int chk = o->check_every > 0 ? o->check_every : 10;
    const int rel_every = (mixed && o->reliable_every > 0) ? o->reliable_every : 1 << 30;
    int rc;
    if (!c->capturing) return set_error(HOL_EINVAL, "graph solve: context is not being captured");
    if (chk & 1) return set_error(HOL_EINVAL, "graph solve: check_every must be even (%d)", chk);
    if (c->fused || c->merged || c->persist)
        return set_error(HOL_EINVAL, "graph solve: needs the two-kernel CG iteration (fused_cg, "
                                     "merged_cg and persistent_cg off)");
    if (pc && (rc = precond_check_shape(c))) return rc;

    double* r64 = c->v64a;
    double* p64[2] = {c->v64b, c->v64c};
    double* q64 = c->v64d;
    double* w64 = c->v64e;
    double* z64 = pc ? c->v64f : r64;
    float* r32 = c->v32a;
    float* p32[2] = {c->v32b, c->v32c};
    float* q32 = c->v32d;
    float* e32 = c->v32e;
    float* z32 = pc ? c->v32f : r32;
    double* t64 = c->v64a;
    double* rt64 = c->v64b;
    auto est_bank = [&](int cur) { return pc ? B.er : B.dz[cur]; };
    auto apply_prec = [&](int bank, cudaStream_t cs) -> int {
        return mixed ? precond_apply_impl(c, HOL_F32, r32, z32, n_rhs, 3, r32, B.dz[bank], cs)
                     : precond_apply_impl(c, HOL_F64, r64, z64, n_rhs, 3, r64, B.dz[bank], cs);
    };

    HOL_CUDA(cudaMemsetAsync(v, 0, (size_t)n_rhs * n * sizeof(double), s));
    if (mixed)
        k_cg_init<float><<<g2, 256, 0, s>>>(b, r32, e32, n, B.bn, est_bank(0));
    else
        k_cg_init<double><<<g2, 256, 0, s>>>(b, r64, nullptr, n, B.bn, est_bank(0));
    HOL_CHECK_LAUNCH("k_cg_init");
    if (pc && (rc = apply_prec(0, s))) return rc;
    k_dcg_start<<<1, kDcgThreads, 0, s>>>(B.bn, nb2, n_rhs, act_d, rel_d, d);
    HOL_CHECK_LAUNCH("k_dcg_start");

    // One chunk of chk iterations on stream cs, then the decision and the
    // conditional reliable update. chk is even, so the bank and direction
    // parities are back at 0 at every chunk end and the loop body is the same
    // for every chunk.
    auto chunk = [&](cudaStream_t cs, int first) -> int {
        int cur = 0, pp = 0;
        bool pending = false;
        for (int j = 0; j < chk; ++j) {
            double* rr_dst = pc ? B.er : B.dz[1 - cur];
            int fold;
            if (pending) {
                fold = 2;
                pending = false;
            } else if (j == chk - 1) {
                fold = 1;
            } else {
                fold = 0;
                pending = true;
            }
            int r2;
            if (mixed) {
                int adone = 0;
                r2 = launch_cg_mtm32(c, z32, first ? z32 : p32[pp], p32[1 - pp], q32, n_rhs, act_d,
                                     B.dz[cur], B.dz[1 - cur], kRedStride, dz_n, first, B.pq, cs,
                                     (c->handoff & 1) ? c->alpha_now : nullptr, &adone,
                                     (!pc && (c->handoff & 2)) ? c->beta_now : nullptr);
                if (r2) return r2;
                pp = 1 - pp;
                if (fuse_pc) {
                    const PcUpd u{e32, p32[pp], p32[1 - pp], q32, act_d, B.pq, pstride, pq_n,
                                  B.dz[cur], dz_n, rr_dst, c->alpha_buf, fold};
                    if ((r2 = precond_apply_upd(c, HOL_F32, r32, z32, n_rhs, &u, B.dz[1 - cur],
                                                cs)))
                        return r2;
                    cur = 1 - cur;
                    first = 0;
                    continue;
                }
                auto* upd = fold == 0 ? k_cg_update<float, 0>
                                      : fold == 1 ? k_cg_update<float, 1> : k_cg_update<float, 2>;
                HOL_CUDA(launch_pdl(c, upd, g2, 256, 0, cs, e32, r32, p32[pp], p32[1 - pp], q32, n,
                                    act_d, B.pq, pstride, pq_n, B.dz[cur], dz_n, rr_dst,
                                    c->alpha_buf, adone ? (const double*)c->alpha_now : nullptr,
                                    (!pc && (c->handoff & 2)) ? c->beta_now : nullptr, c->beta_cnt));
            } else {
                BetaSrc bs{B.dz[cur], B.dz[1 - cur], kRedStride, dz_n, first};
                r2 = launch_M_upd64(c, z64, first ? z64 : p64[pp], p64[1 - pp], w64, n_rhs, act_d,
                                    bs, B.pq, cs);
                if (r2) return r2;
                r2 = launch_MT(c, HOL_F64, w64, q64, n_rhs, act_d, cs);
                if (r2) return r2;
                pp = 1 - pp;
                if (fuse_pc) {
                    const PcUpd u{v, p64[pp], p64[1 - pp], q64, act_d, B.pq, pstride64, pq_n64,
                                  B.dz[cur], dz_n, rr_dst, c->alpha_buf, fold};
                    if ((r2 = precond_apply_upd(c, HOL_F64, r64, z64, n_rhs, &u, B.dz[1 - cur],
                                                cs)))
                        return r2;
                    cur = 1 - cur;
                    first = 0;
                    continue;
                }
                auto* upd = fold == 0 ? k_cg_update<double, 0>
                                      : fold == 1 ? k_cg_update<double, 1> : k_cg_update<double, 2>;
                HOL_CUDA(launch_pdl(c, upd, g2, 256, 0, cs, v, r64, p64[pp], p64[1 - pp], q64, n,
                                    act_d, B.pq, pstride64, pq_n64, B.dz[cur], dz_n, rr_dst,
                                    c->alpha_buf, (const double*)nullptr, (double*)nullptr,
                                    (int*)nullptr));
            }
            HOL_CHECK_LAUNCH("k_cg_update");
            if (pc && (r2 = apply_prec(1 - cur, cs))) return r2;
            cur = 1 - cur;
            first = 0;
        }
        // cur == 0 and pp == 0 here (chk even)
        cudaGraphConditionalHandle h_if;
        int r2 = cond_handle(cs, &h_if);
        if (r2) return r2;
        k_dcg_decide<<<1, kDcgThreads, 0, cs>>>(est_bank(cur), pc ? est_n : nb2, n_rhs, chk,
                                                o->tol, rel_every, o->max_iter, act_d, rel_d, d,
                                                h_if);
        HOL_CHECK_LAUNCH("k_dcg_decide");
        cudaGraph_t body;
        if ((r2 = cond_node(cs, h_if, cudaGraphCondTypeIf, &body))) return r2;
        cudaStream_t is = c->cap_s[1];
        HOL_CUDA(cudaStreamBeginCaptureToGraph(is, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        r2 = [&]() -> int {
            // reliable update / certification of the flagged rhs (as in cg_run)
            int r3;
            if (mixed) {
                HOL_CUDA(launch_pdl(c, k_fold, g2, 256, 0, is, v, e32, n, rel_d));
                HOL_CHECK_LAUNCH("k_fold");
                if ((r3 = launch_M(c, HOL_F64, v, t64, n_rhs, rel_d, nullptr, is))) return r3;
                if ((r3 = launch_MT_resid64(c, t64, b, rt64, n_rhs, rel_d, is))) return r3;
                HOL_CUDA(launch_pdl(c, k_recast<float>, g2, 256, 0, is, rt64, r32, n, rel_d, B.tr,
                                    est_bank(cur)));
            } else {
                if ((r3 = launch_M(c, HOL_F64, v, w64, n_rhs, rel_d, nullptr, is))) return r3;
                if ((r3 = launch_MT_resid64(c, w64, b, r64, n_rhs, rel_d, is))) return r3;
                HOL_CUDA(launch_pdl(c, k_recast<double>, g2, 256, 0, is, r64, r64, n, rel_d, B.tr,
                                    est_bank(cur)));
            }
            HOL_CHECK_LAUNCH("k_recast");
            if (pc && (r3 = apply_prec(cur, is))) return r3;
            double* cj0 = c->part + 8 * c->part_len;
            double* cj1 = c->part + 9 * c->part_len;
            if (mixed) {
                HOL_CUDA(launch_pdl(c, k_conj_dots<float>, g2, 256, 0, is, z32, p32[pp], q32, n,
                                    rel_d, cj0, cj1));
                HOL_CHECK_LAUNCH("k_conj_dots");
                HOL_CUDA(launch_pdl(c, k_conj_scale<float>, g2, 256, 0, is, p32[pp], n, rel_d, cj0,
                                    cj1, nb2));
            } else {
                HOL_CUDA(launch_pdl(c, k_conj_dots<double>, g2, 256, 0, is, z64, p64[pp], q64, n,
                                    rel_d, cj0, cj1));
                HOL_CHECK_LAUNCH("k_conj_dots");
                HOL_CUDA(launch_pdl(c, k_conj_scale<double>, g2, 256, 0, is, p64[pp], n, rel_d, cj0,
                                    cj1, nb2));
            }
            HOL_CHECK_LAUNCH("k_conj_scale");
            HOL_CUDA(launch_pdl(c, k_copy_rows, n_rhs, 256, 0, is, B.dz[cur], B.dz[1 - cur], rel_d,
                                (mixed && !pc && (c->handoff & 2)) ? c->beta_now : nullptr, dz_n));
            HOL_CHECK_LAUNCH("k_copy_rows");
            k_dcg_finish<<<1, kDcgThreads, 0, is>>>(B.tr, nb2, n_rhs, o->tol, act_d, rel_d, d);
            HOL_CHECK_LAUNCH("k_dcg_finish");
            return HOL_OK;
        }();
        cudaGraph_t done_body = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(is, &done_body);
        if (r2) return r2;
        if (ee != cudaSuccess) return cuda_error(ee, "graph solve: reliable-update body");
        return HOL_OK;
    };

    const int max_loops = (o->max_iter + chk - 1) / chk + 2;
    if ((rc = chunk(s, 1))) return rc;
    cudaGraphConditionalHandle h_while;
    if ((rc = cond_handle(s, &h_while))) return rc;
    k_dcg_cond<<<1, kDcgThreads, 0, s>>>(act_d, n_rhs, o->max_iter, max_loops, d, h_while);
    HOL_CHECK_LAUNCH("k_dcg_cond");
    cudaGraph_t body;
    if ((rc = cond_node(s, h_while, cudaGraphCondTypeWhile, &body))) return rc;
    cudaStream_t ws = c->cap_s[0];
    HOL_CUDA(cudaStreamBeginCaptureToGraph(ws, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    rc = chunk(ws, 0);
    if (!rc) {
        k_dcg_cond<<<1, kDcgThreads, 0, ws>>>(act_d, n_rhs, o->max_iter, max_loops, d, h_while);
        rc = cudaGetLastError() == cudaSuccess ? HOL_OK : set_error(HOL_ECUDA, "k_dcg_cond");
        count_launch();
    }
    cudaGraph_t wb = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(ws, &wb);
    if (rc) return rc;
    if (ee != cudaSuccess) return cuda_error(ee, "graph solve: loop body");
    return HOL_OK;
}

}  // namespace hol

using namespace hol;

extern "C" int cg_solve(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
                        int* iters, double* resid, void* stream)
{
    HOL_TRACE("cg_solve");
    if (!c || !b || !v || !o) return set_error(HOL_EINVAL, "cg_solve: null argument");
    if (int rc_ = require_aligned("cg_solve", {b, v})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "cg_solve: hol_set_field not called");
    if (n_rhs < 1 || n_rhs > c->p.max_rhs)
        return set_error(HOL_EINVAL, "cg_solve: n_rhs=%d outside [1, %d]", n_rhs, c->p.max_rhs);
    if (o->prec != HOL_F64 && o->prec != HOL_F32)
        return set_error(HOL_EINVAL, "cg_solve: bad precision %d", o->prec);
    if (!(o->tol > 0.0) || o->max_iter < 1)
        return set_error(HOL_EINVAL, "cg_solve: tol must be > 0 and max_iter >= 1");
    if (b == v) return set_error(HOL_EINVAL, "cg_solve: b and v must not overlap");
    if (c->fused && o->prec == HOL_F32 && !o->precond)
        return cg_run_fused(c, b, v, n_rhs, o, iters, resid, (cudaStream_t)stream);
    if (c->merged && o->prec == HOL_F32 && !o->precond)
        return cg_run_merged(c, b, v, n_rhs, o, iters, resid, (cudaStream_t)stream);
    return cg_run(c, b, v, n_rhs, o, iters, resid, (cudaStream_t)stream);
}
