// Context life cycle, error reporting, field set-up (Sec. II C) and the
// fermion_matvec entry point.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "cb.cuh"
#include "internal.cuh"

namespace hol {

static thread_local char g_err[512] = "no error";
static unsigned long long g_launches = 0;
std::atomic<int> g_occ64[2][4][33][5];

void count_launch() { __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED); }

// A region is recorded when its running index is a multiple of the stride;
// timer_stop pairs with the timer_start of the same region.
void timer_start(const hol_ctx* c, int k, cudaStream_t s, double units)
{
    KTimer* t = c->timer;
    if (!t || !t->on) return;
    if (t->seen[k] % t->on != 0) return;
    if (t->used[k] >= t->cap) {
        t->dropped[k]++;
        return;
    }
    cudaEventRecord(t->ev[k][2 * t->used[k]], s);
    t->units[k] += units;
}

void timer_stop(const hol_ctx* c, int k, cudaStream_t s)
{
    KTimer* t = c->timer;
    if (!t || !t->on) return;
    const int rec = (t->seen[k] % t->on == 0);
    t->seen[k]++;
    if (!rec || t->used[k] >= t->cap) return;
    cudaEventRecord(t->ev[k][2 * t->used[k] + 1], s);
    t->used[k]++;
}

static void timer_free(KTimer* t)
{
    if (!t) return;
    for (int k = 0; k < KT_COUNT; ++k) {
        if (!t->ev[k]) continue;
        for (int j = 0; j < 2 * t->cap; ++j)
            if (t->ev[k][j]) cudaEventDestroy(t->ev[k][j]);
        free(t->ev[k]);
    }
    free(t);
}

int set_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char* what)
{
    return set_error(e == cudaErrorMemoryAllocation ? HOL_ENOMEM : HOL_ECUDA, "%s: %s (%s)", what,
                     cudaGetErrorString(e), cudaGetErrorName(e));
}

namespace {

// ev = cosh^4 exp(-dtau (alpha x - mu)) in FP64 and FP32 (the cosh factors
// of the four checkerboard colours, see cb.cuh); copy of x.
__global__ void k_expv(const double* __restrict__ x, double* __restrict__ xc,
                       double* __restrict__ ev64, float* __restrict__ ev32, long n, double dtau,
                       double alpha, double mu, double ch4)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x) {
        const double xv = x[k];
        const double e = ch4 * exp(-dtau * (alpha * xv - mu));
        xc[k] = xv;
        ev64[k] = e;
        ev32[k] = (float)e;
    }
}

// dbar_i = (1/T) sum_tau expV[tau][i] (Eq. (expnVbar)); one thread per site.
__global__ void k_dbar(const double* __restrict__ ev, double* __restrict__ dbar, int N, int T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int tau = 0; tau < T; ++tau) s += ev[(long)tau * N + i];
    dbar[i] = s / T;
}

// Norm bounds of the Bbar spectrum: every checkerboard colour has
// eigenvalues exp(+-dtau t), so |Bbar| <= max(dbar) e^{4 dtau |t|} and
// |Bbar^{-1}| <= e^{4 dtau |t|} / min(dbar), dbar of Eq. (expnVbar) (the
// stored dbar carries the factor cosh^4, removed here). One block.
__global__ void k_bounds(const double* __restrict__ dbar, int N, double g4, double ch4,
                         double* __restrict__ scal)
{
    __shared__ double smin[32], smax[32];
    double lo = 1e300, hi = -1e300;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        lo = fmin(lo, dbar[i]);
        hi = fmax(hi, dbar[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(kFull, lo, o));
        hi = fmax(hi, __shfl_xor_sync(kFull, hi, o));
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        smin[w] = lo;
        smax[w] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            lo = fmin(lo, smin[k]);
            hi = fmax(hi, smax[k]);
        }
        scal[S_BMIN] = lo / ch4 / g4;
        scal[S_BMAX] = hi / ch4 * g4;
    }
}

void free_ctx(hol_ctx* c)
{
    if (!c) return;
    void* dev[] = {c->x, c->ev64, c->ev32, c->dbar, c->scal, c->part, c->v64a, c->v64b,
                   c->v64c, c->v64d, c->v64e, c->v32a,
                   c->mask, c->kpm.np, c->kpm.coef, c->cbuf0, c->cbuf1, c->v64f,
                   c->tw64, c->tw32, c->md_phi, c->md_b, c->md_v, c->md_F, c->md_p,
                   c->md_x0, c->md_g, c->md_s, c->ms_acc, c->twL64, c->v32g, c->v32h,
                   c->v32i, c->cgs, c->alpha_buf, c->arn};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (c->dcg) cudaFree(c->dcg);
    if (c->alpha_now) cudaFree(c->alpha_now);
    if (c->alpha_cnt) cudaFree(c->alpha_cnt);
    if (c->beta_now) cudaFree(c->beta_now);
    if (c->beta_cnt) cudaFree(c->beta_cnt);
    if (c->kpm_q) cudaFree(c->kpm_q);
    for (cudaStream_t cs : c->cap_s)
        if (cs) cudaStreamDestroy(cs);
    timer_free(c->timer);
    if (c->hbuf) cudaFreeHost(c->hbuf);
    if (c->hflag) cudaFreeHost(c->hflag);
    free(c);
}

}  // namespace

int kpm_setup(hol_ctx* c, cudaStream_t s);   // precond.cu

}  // namespace hol

using namespace hol;

extern "C" const char* hol_last_error(void) { return g_err; }

namespace hol {
int smem_raise(const void* fn, size_t bytes)
{
    if (bytes <= 32 * 1024) return HOL_OK;
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> limit;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[fn];
    if (bytes <= cur) return HOL_OK;
    HOL_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return HOL_OK;
}
}  // namespace hol

// Modified Bessel function I_n(x) by its power series
// sum_k (x/2)^(2k+n) / (k! (k+n)!) (all terms of one sign, no cancellation).
static double bessel_i(int n, double x)
{
    const double h = 0.5 * x;
    double term = 1.0;
    for (int j = 1; j <= n; ++j) {
        term *= h / j;
        if (term == 0.0) return 0.0;
    }
    double sum = term;
    for (int k = 1; k < 200; ++k) {
        term *= h * h / ((double)k * (double)(k + n));
        sum += term;
        if (fabs(term) <= 1e-20 * fabs(sum)) break;
    }
    return sum;
}

// Taps of the exact one-direction factor E = exp(dtau t A_ring) on a ring of
// L sites: exp(a A_line) has entries I_|i-j|(2a) on the infinite line, and
// the ring sums the images, e[d] = sum_m I_|d + m L|(2 dtau t). Taps whose
// magnitude is below 2^-60 (FP64) or 2^-30 (FP32) of e[0] are dropped: their
// total is far below the rounding of that arithmetic.
static void compute_exact_taps(int L, double dtau, double t, double* e_out, int* d64_out,
                               int* d32_out)
{
    const double x = 2.0 * dtau * t;
    for (int d = 0; d < kKinTaps; ++d) e_out[d] = 0.0;
    for (int d = 0; d <= L / 2; ++d) {
        double e = 0.0;
        for (int m = -64; m <= 64; ++m) {
            const int k = abs(d + m * L);
            if (k > 400) continue;
            e += bessel_i(k, x);
        }
        e_out[d] = e;
    }
    const double e0 = fabs(e_out[0]);
    int d64 = L / 2, d32 = L / 2;
    while (d64 > 0 && fabs(e_out[d64]) <= 0x1p-60 * e0) --d64;
    while (d32 > 0 && fabs(e_out[d32]) <= 0x1p-30 * e0) --d32;
    *d64_out = d64;
    *d32_out = d32;
}

static void exact_taps(hol_ctx* c)
{
    compute_exact_taps(c->L, c->p.dtau, c->p.t, c->kin_e, &c->kin_d64, &c->kin_d32);
}

extern "C" int hol_exact_taps(int L, double dtau, double t, double* e, int* d64, int* d32)
{
    HOL_TRACE("hol_exact_taps");
    if (!e || !d64 || !d32 || L < 4 || L > kMaxL || (L & 1) || !(dtau > 0.0) ||
        !(fabs(dtau * t) <= 4.0))
        return set_error(HOL_EINVAL, "hol_exact_taps: bad argument");
    compute_exact_taps(L, dtau, t, e, d64, d32);
    return HOL_OK;
}

extern "C" int hol_create(const hol_params* p, hol_ctx** out)
{
    HOL_TRACE("hol_create");
    if (!p || !out) return set_error(HOL_EINVAL, "hol_create: null argument");
    *out = nullptr;
    if (p->L < 4 || p->L > kMaxL || (p->L & 1))
        return set_error(HOL_EINVAL, "hol_create: L=%d must be even and in [4, %d]", p->L, kMaxL);
    if (p->Ltau < 2 || (p->Ltau & 1))
        return set_error(HOL_EINVAL, "hol_create: Ltau=%d must be even and >= 2", p->Ltau);
    if (p->max_rhs < 1 || p->max_rhs > 4096)
        return set_error(HOL_EINVAL, "hol_create: max_rhs=%d out of range", p->max_rhs);
    if (!(p->dtau > 0.0) || !isfinite(p->t) || !isfinite(p->mu) || !isfinite(p->alpha) ||
        !isfinite(p->omega0))
        return set_error(HOL_EINVAL, "hol_create: non-finite or non-positive parameter");
    if (p->kinetic != HOL_KINETIC_CHECKERBOARD && p->kinetic != HOL_KINETIC_EXACT)
        return set_error(HOL_EINVAL, "hol_create: kinetic=%d must be %d (checkerboard) or %d "
                                     "(exact)", p->kinetic, HOL_KINETIC_CHECKERBOARD,
                         HOL_KINETIC_EXACT);
    if (p->kinetic == HOL_KINETIC_EXACT && fabs(p->dtau * p->t) > 4.0)
        return set_error(HOL_EINVAL, "hol_create: exact propagator needs |dtau t| <= 4");

    hol_ctx* c = (hol_ctx*)calloc(1, sizeof(hol_ctx));
    if (!c) return set_error(HOL_ENOMEM, "hol_create: host allocation failed");
    c->p = *p;
    c->L = p->L;
    c->N = p->L * p->L;
    c->T = p->Ltau;
    c->n = (long)c->N * c->T;
    c->th = tanh(p->dtau * p->t);
    c->exact = p->kinetic == HOL_KINETIC_EXACT;
    if (c->exact) {
        c->ch4 = 1.0;
        exact_taps(c);
    } else {
        const double ch = cosh(p->dtau * p->t);
        c->ch4 = ch * ch * ch * ch;
    }
    c->mv_k = (c->T % 4 == 0 && c->T >= 8) ? 2 : 1;
    c->mv_warps = 4;
    c->mv_vec = c->exact ? 0 : 1;
    // register KPM: two columns per lane at L = 32 (measured 0.126 against
    // 0.149 ms for P^{-1} P^{-T} on 16 rhs; 47 us against 58 us for the lane
    // layout on 2 rhs at Ltau = 200), the lane layout (one lane per column,
    // real and imaginary parts in two lane groups) for every other L (at
    // L = 16, Ltau = 160, 2 rhs: 25.3 us against 29.0 us for four columns
    // per lane)
    c->kpm_reg = c->exact ? 0 : (c->L == 32 ? 2 : 3);
    c->persist = 0;
    c->merged = 0;
    c->fused = 0;
    c->pdl = 1;
    c->kpm_a1 = 1.0;
    c->kpm_a2 = 1.0;
    c->pc_fuse = 1;   // measured: hmc16 trajectory 3.10 -> 3.25 /s, 48 chains 52.8 -> 54.8 /s
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        free_ctx(c);
        return set_error(HOL_ECUDA, "hol_create: no CUDA device");
    }
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess ||
        c->sms < 1) {
        free_ctx(c);
        return set_error(HOL_ECUDA, "hol_create: multiprocessor count query failed");
    }
    if (c->exact)
        occ64_warm_exact(c);
    else
        occ64_warm(c);

    const long n = c->n, R = p->max_rhs;
    const long pstride = matvec_pstride(c);
    c->part_len = R * (pstride > kRedStride ? pstride : kRedStride);
    c->cbuf_len = R * (long)(c->T / 2) * c->N;   // complex half spectra
    c->kpm.max_np = 0;

#define ALLOC(ptr, bytes)                                                 \
    do {                                                                  \
        cudaError_t e = cudaMalloc((void**)&(ptr), (bytes));              \
        if (e != cudaSuccess) {                                           \
            free_ctx(c);                                                  \
            return cuda_error(e, "hol_create: cudaMalloc " #ptr);         \
        }                                                                 \
    } while (0)
    ALLOC(c->x, n * sizeof(double));
    ALLOC(c->ev64, n * sizeof(double));
    ALLOC(c->ev32, n * sizeof(float));
    ALLOC(c->dbar, c->N * sizeof(double));
    ALLOC(c->scal, S_COUNT * sizeof(double));
    ALLOC(c->part, kBanks * c->part_len * sizeof(double));
    ALLOC(c->v64a, R * n * sizeof(double));
    ALLOC(c->v64b, R * n * sizeof(double));
    ALLOC(c->v64c, R * n * sizeof(double));
    ALLOC(c->v64d, R * n * sizeof(double));
    ALLOC(c->v64e, R * n * sizeof(double));
    // the six FP32 vector sets of the solver are one arena (v32a is its base)
    ALLOC(c->v32a, 6 * R * n * sizeof(float));
    c->v32b = c->v32a + 1 * R * n;
    c->v32c = c->v32a + 2 * R * n;
    c->v32d = c->v32a + 3 * R * n;
    c->v32e = c->v32a + 4 * R * n;
    c->v32f = c->v32a + 5 * R * n;
    ALLOC(c->v64f, R * n * sizeof(double));
    ALLOC(c->mask, 2 * R * sizeof(int));
    ALLOC(c->alpha_buf, R * sizeof(double));
    ALLOC(c->arn, ((size_t)(kArnoldiMax + 1) * c->N + (kArnoldiMax + 1) * kArnoldiMax + 1) *
                      sizeof(double));
    ALLOC(c->dcg, dcg_bytes(R));
    ALLOC(c->alpha_now, R * sizeof(double));
    ALLOC(c->alpha_cnt, R * sizeof(int));
    ALLOC(c->beta_now, R * sizeof(double));
    ALLOC(c->beta_cnt, R * sizeof(int));
    ALLOC(c->kpm_q, 2 * sizeof(int));
    if (cudaMemset(c->alpha_cnt, 0, R * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->beta_cnt, 0, R * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->kpm_q, 0, 2 * sizeof(int)) != cudaSuccess) {
        free_ctx(c);
        return set_error(HOL_ECUDA, "hol_create: memset");
    }
    for (cudaStream_t& cs : c->cap_s)
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            free_ctx(c);
            return set_error(HOL_ECUDA, "hol_create: stream creation failed");
        }
    ALLOC(c->cbuf0, c->cbuf_len * sizeof(double2));
    ALLOC(c->cbuf1, c->cbuf_len * sizeof(double2));
#undef ALLOC
    if (cudaMallocHost((void**)&c->hbuf, 16 * R * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&c->hflag, 4 * R * sizeof(int)) != cudaSuccess) {
        free_ctx(c);
        return set_error(HOL_ENOMEM, "hol_create: pinned host allocation failed");
    }
    {
        int rc = precond_alloc(c);
        if (!rc) rc = leapfrog_alloc(c);
        if (!rc) rc = measure_alloc(c);
        if (rc) {
            free_ctx(c);
            return rc;
        }
    }
    if (cudaMemset(c->scal, 0, S_COUNT * sizeof(double)) != cudaSuccess) {
        free_ctx(c);
        return set_error(HOL_ECUDA, "hol_create: memset");
    }
    *out = c;
    return HOL_OK;
}

extern "C" int hol_destroy(hol_ctx* c)
{
    HOL_TRACE("hol_destroy");
    if (!c) return HOL_OK;
    cudaDeviceSynchronize();
    free_ctx(c);
    return HOL_OK;
}

extern "C" int hol_set_field(hol_ctx* c, const double* x, void* stream)
{
    HOL_TRACE("hol_set_field");
    if (!c || !x) return set_error(HOL_EINVAL, "hol_set_field: null argument");
    if (int rc_ = require_aligned("hol_set_field", {x})) return rc_;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = ceil_div(c->n, 256) < 4096 ? ceil_div(c->n, 256) : 4096;
    k_expv<<<nb, 256, 0, s>>>(x, c->x, c->ev64, c->ev32, c->n, c->p.dtau, c->p.alpha, c->p.mu,
                              c->ch4);
    HOL_CHECK_LAUNCH("k_expv");
    k_dbar<<<ceil_div(c->N, 128), 128, 0, s>>>(c->ev64, c->dbar, c->N, c->T);
    HOL_CHECK_LAUNCH("k_dbar");
    k_bounds<<<1, 256, 0, s>>>(c->dbar, c->N, exp(4.0 * c->p.dtau * fabs(c->p.t)), c->ch4,
                               c->scal);
    HOL_CHECK_LAUNCH("k_bounds");
    int rc = kpm_setup(c, s);
    if (rc) return rc;
    c->field_set = 1;
    return HOL_OK;
}

extern "C" int fermion_matvec(hol_ctx* c, int op, int prec, const void* v, void* out, int n_rhs,
                              void* stream)
{
    HOL_TRACE("fermion_matvec");
    if (!c || !v || !out) return set_error(HOL_EINVAL, "fermion_matvec: null argument");
    if (int rc_ = require_aligned("fermion_matvec", {v, out})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "fermion_matvec: hol_set_field not called");
    if (n_rhs < 1 || n_rhs > c->p.max_rhs)
        return set_error(HOL_EINVAL, "fermion_matvec: n_rhs=%d outside [1, %d]", n_rhs,
                         c->p.max_rhs);
    if (prec != HOL_F64 && prec != HOL_F32)
        return set_error(HOL_EINVAL, "fermion_matvec: bad precision %d", prec);
    if (v == out) return set_error(HOL_EINVAL, "fermion_matvec: v and out must not overlap");
    cudaStream_t s = (cudaStream_t)stream;
    switch (op) {
    case HOL_OP_M:
        return launch_M(c, prec, v, out, n_rhs, nullptr, nullptr, s);
    case HOL_OP_MT:
        return launch_MT(c, prec, v, out, n_rhs, nullptr, s);
    case HOL_OP_MTM:
        if (prec == HOL_F32)
            return launch_cg_mtm32(c, (const float*)v, (const float*)v, nullptr, (float*)out, n_rhs,
                                   nullptr, nullptr, nullptr, 0, 0, 1, nullptr, s);
        else {
            int rc = launch_M(c, HOL_F64, v, c->v64a, n_rhs, nullptr, nullptr, s);
            if (rc) return rc;
            return launch_MT(c, HOL_F64, c->v64a, out, n_rhs, nullptr, s);
        }
    }
    return set_error(HOL_EINVAL, "fermion_matvec: bad op %d", op);
}

extern "C" unsigned long long hol_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

extern "C" int hol_timer_enable(hol_ctx* c, int on)
{
    HOL_TRACE("hol_timer_enable");
    if (!c) return set_error(HOL_EINVAL, "hol_timer_enable: null context");
    if (on && !c->timer) {
        KTimer* t = (KTimer*)calloc(1, sizeof(KTimer));
        if (!t) return set_error(HOL_ENOMEM, "hol_timer_enable: host allocation");
        t->cap = 4096;
        for (int k = 0; k < KT_COUNT; ++k) {
            t->ev[k] = (cudaEvent_t*)calloc(2 * t->cap, sizeof(cudaEvent_t));
            if (!t->ev[k]) {
                timer_free(t);
                return set_error(HOL_ENOMEM, "hol_timer_enable: host allocation");
            }
            for (int j = 0; j < 2 * t->cap; ++j) {
                cudaError_t e = cudaEventCreate(&t->ev[k][j]);
                if (e != cudaSuccess) {
                    timer_free(t);
                    return cuda_error(e, "hol_timer_enable: cudaEventCreate");
                }
            }
        }
        c->timer = t;
    }
    if (c->timer) {
        c->timer->on = on > 0 ? on : 0;
        if (on)
            for (int k = 0; k < KT_COUNT; ++k)
            {
                c->timer->used[k] = c->timer->dropped[k] = c->timer->seen[k] = 0;
                c->timer->units[k] = 0.0;
            }
    }
    return HOL_OK;
}

extern "C" int hol_timer_read(hol_ctx* c, int klass, int* count, double* total_ms,
                              double* units)
{
    HOL_TRACE("hol_timer_read");
    if (!c || !count || !total_ms || klass < 0 || klass >= KT_COUNT)
        return set_error(HOL_EINVAL, "hol_timer_read: bad argument");
    *count = 0;
    *total_ms = 0.0;
    if (units) *units = 0.0;
    KTimer* t = c->timer;
    if (!t) return HOL_OK;
    double tot = 0.0;
    for (int j = 0; j < t->used[klass]; ++j) {
        HOL_CUDA(cudaEventSynchronize(t->ev[klass][2 * j + 1]));
        float ms = 0.0f;
        HOL_CUDA(cudaEventElapsedTime(&ms, t->ev[klass][2 * j], t->ev[klass][2 * j + 1]));
        tot += ms;
    }
    *count = t->used[klass];
    *total_ms = tot;
    if (units) *units = t->units[klass];
    return HOL_OK;
}

// Three more FP32 vector sets and the merged solver's scalar slots, for the
// merged and fused CG loops (allocated once, on first use).
static int alloc_extra_vectors(hol_ctx* c)
{
    if (c->v32g) return HOL_OK;
    const size_t vb = (size_t)c->p.max_rhs * c->n * sizeof(float);
    float** bufs[3] = {&c->v32g, &c->v32h, &c->v32i};
    for (float** b : bufs) {
        const cudaError_t e = cudaMalloc((void**)b, vb);
        if (e != cudaSuccess) return cuda_error(e, "hol_set_option: solver vector sets");
    }
    const cudaError_t e = cudaMalloc((void**)&c->cgs, 8 * c->p.max_rhs * sizeof(double));
    if (e != cudaSuccess) return cuda_error(e, "hol_set_option: solver scalars");
    return HOL_OK;
}

extern "C" int hol_set_option(hol_ctx* c, const char* name, int value)
{
    HOL_TRACE("hol_set_option");
    if (!c || !name) return set_error(HOL_EINVAL, "hol_set_option: null argument");
    auto is = [&](const char* s) { return strcmp(name, s) == 0; };
    if (is("slices_per_group")) {
        if (value < 1 || c->T % value)
            return set_error(HOL_EINVAL, "hol_set_option: slices_per_group must divide Ltau");
        const int old = c->mv_k;
        c->mv_k = value;
        if ((long)matvec_pstride(c) * c->p.max_rhs > c->part_len) {
            c->mv_k = old;
            return set_error(HOL_EINVAL, "hol_set_option: slices_per_group too small");
        }
    } else if (is("warps_per_block")) {
        if (value != 1 && value != 2 && value != 4)
            return set_error(HOL_EINVAL, "hol_set_option: warps_per_block must be 1, 2 or 4");
        c->mv_warps = value;
    } else if (is("layout")) {
        if (value != 0 && c->exact)
            return set_error(HOL_EINVAL, "hol_set_option: the exact propagator runs in layout 0");
        const bool ring = value == 2 || value == 6;   // float4 with a cp.async ring
        if (value < 0 || value > 7 || (ring && (c->L % 4 || c->L < 8)) ||
            (value > 0 && !ring && c->L % 8) ||
            ((value == 4 || value == 5 || value == 7) && c->L != 32))
            return set_error(HOL_EINVAL, "hol_set_option: layout 0..7 (2, 6 need L %% 4 == 0 "
                                         "and L >= 8; 1, 3 L %% 8 == 0; 4, 5, 7 L == 32)");
        c->mv_vec = value;
    } else if (is("kpm_registers")) {
        if (value && c->exact)
            return set_error(HOL_EINVAL, "hol_set_option: kpm_registers is checkerboard only");
        if (value < 0 || value > 3)
            return set_error(HOL_EINVAL, "hol_set_option: kpm_registers must be 0, 1, 2 or 3");
        c->kpm_reg = value;
    } else if (is("persistent_cg")) {
        if (value && c->exact)
            return set_error(HOL_EINVAL, "hol_set_option: persistent_cg is checkerboard only");
        c->persist = value ? 1 : 0;
    } else if (is("pdl")) {
        c->pdl = value ? 1 : 0;
    } else if (is("fused_pc_update")) {
        c->pc_fuse = value ? 1 : 0;
    } else if (is("kpm_a1_percent") || is("kpm_a2_percent")) {
        if (value < 1 || value > 400)
            return set_error(HOL_EINVAL, "hol_set_option: %s must be in [1, 400]", name);
        if (is("kpm_a1_percent"))
            c->kpm_a1 = value / 100.0;
        else
            c->kpm_a2 = value / 100.0;
    } else if (is("kpm_queue")) {
        if (value < 0 || value > 8)
            return set_error(HOL_EINVAL, "hol_set_option: kpm_queue must be 0..8");
        c->kpm_queue = value;
    } else if (is("scalar_handoff")) {
        if (value < 0 || value > 3)
            return set_error(HOL_EINVAL, "hol_set_option: scalar_handoff must be 0..3");
        c->handoff = value;
    } else if (is("merged_cg") || is("fused_cg")) {
        if (value && c->exact)
            return set_error(HOL_EINVAL, "hol_set_option: %s is checkerboard only", name);
        if (value && c->L % 8)
            return set_error(HOL_EINVAL, "hol_set_option: %s needs L %% 8 == 0", name);
        if (value) {
            const int rc = alloc_extra_vectors(c);
            if (rc) return rc;
        }
        if (is("merged_cg"))
            c->merged = value ? 1 : 0;
        else
            c->fused = value ? 1 : 0;
    } else {
        return set_error(HOL_EINVAL, "hol_set_option: unknown option '%s'", name);
    }
    return HOL_OK;
}

extern "C" int hol_get_option(const hol_ctx* c, const char* name, int* value)
{
    HOL_TRACE("hol_get_option");
    if (!c || !name || !value) return set_error(HOL_EINVAL, "hol_get_option: null argument");
    auto is = [&](const char* s) { return strcmp(name, s) == 0; };
    if (is("slices_per_group")) *value = c->mv_k;
    else if (is("warps_per_block")) *value = c->mv_warps;
    else if (is("layout")) *value = c->mv_vec;
    else if (is("kpm_registers")) *value = c->kpm_reg;
    else if (is("persistent_cg")) *value = c->persist;
    else if (is("merged_cg")) *value = c->merged;
    else if (is("fused_cg")) *value = c->fused;
    else if (is("pdl")) *value = c->pdl;
    else if (is("scalar_handoff")) *value = c->handoff;
    else if (is("kpm_queue")) *value = c->kpm_queue;
    else if (is("fused_pc_update")) *value = c->pc_fuse;
    else if (is("kpm_a1_percent")) *value = (int)lround(c->kpm_a1 * 100.0);
    else if (is("kpm_a2_percent")) *value = (int)lround(c->kpm_a2 * 100.0);
    else return set_error(HOL_EINVAL, "hol_get_option: unknown option '%s'", name);
    return HOL_OK;
}
