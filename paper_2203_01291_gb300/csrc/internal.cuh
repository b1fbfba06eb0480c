// Internal declarations of the Holstein GB300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <atomic>
#include <initializer_list>
#include <stdio.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/holstein.h"
#include "cb.cuh"

namespace hol {

// ----------------------------------------------------------------------------
// error reporting
// ----------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

#define HOL_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e__ = (call);                             \
        if (e__ != cudaSuccess) return hol::cuda_error(e__, #call); \
    } while (0)

// Every kernel launch is followed by this check, which also counts it.
#define HOL_CHECK_LAUNCH(what)                                \
    do {                                                      \
        hol::count_launch();                                  \
        cudaError_t e__ = cudaGetLastError();                 \
        if (e__ != cudaSuccess) return hol::cuda_error(e__, what); \
    } while (0)

void count_launch();

// An NVTX range around each C-ABI call, named after it, so that a profiler's
// timeline shows the library's calls (a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define HOL_TRACE(name) const hol::NvtxRange hol_trace_range_(name)

// Raise the dynamic shared-memory limit of kernel `fn` to at least `bytes`
// (a no-op up to 32 KB, which leaves room for static shared memory under the
// default limit). The limit of a kernel only ever grows, under a lock, so
// contexts of different shapes driven from several host threads never lower
// it under one another's launches.
int smem_raise(const void* fn, size_t bytes);

// Device vectors are moved with 8- and 16-byte vector accesses, so every
// device vector argument of the C ABI must be 16-byte aligned (cudaMalloc and
// PyTorch allocations are, and so is a slice of one along the right-hand-side
// axis, N being even). Checked on the host before any launch.
inline int require_aligned(const char* fn, std::initializer_list<const void*> ptrs)
{
    for (const void* q : ptrs)
        if (q != nullptr && (reinterpret_cast<uintptr_t>(q) & 15u) != 0)
            return set_error(HOL_EINVAL, "%s: device vector %p is not 16-byte aligned", fn, q);
    return HOL_OK;
}

// True when the byte ranges [a, a + na) and [b, b + nb) share an address
// (host-side aliasing check of two device arrays of the C ABI).
inline bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return pa < pb + nb && pb < pa + na;
}

// A CG step ratio (alpha or beta) num / den, 0 when it is not finite. On a
// small system the residual can reach exactly zero between two convergence
// polls; the next step then has 0 / 0, and a zero step keeps the solution
// instead of filling it with NaN.
__host__ __device__ __forceinline__ double cg_ratio(double num, double den)
{
    const double q = num / den;
    return isfinite(q) ? q : 0.0;
}

// Programmatic dependent launch. A kernel launched with launch_pdl may be
// scheduled while the previous kernel of its stream is still running; it
// must call pdl_wait() before touching memory that kernel writes (the wait
// returns once that kernel has completed and its writes are visible; it is
// a no-op for a kernel launched normally). pdl_trigger() lets the next
// PDL-launched kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
}
// Triggers the dependent launch when the thread leaves the kernel (at any
// return), i.e. once this block's work is issued.
struct PdlTriggerAtExit {
    __device__ __forceinline__ ~PdlTriggerAtExit() { pdl_trigger(); }
};
// Launch of a CG-iteration kernel, with programmatic dependent launch when
// the context enables it (hol_ctx::pdl).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(const hol_ctx* c, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                       size_t smem, cudaStream_t s, Args&&... args);


// Optional CUDA-event timing of kernel classes (hol_timer_* entry points).
enum TimerClass { KT_OPERATOR = 0, KT_UPDATE = 1, KT_FORCE = 2, KT_PRECOND = 3, KT_OTHER = 4,
                  KT_COUNT = 5 };
struct KTimer {
    int on;                        // record one region in every `on` (0: off)
    int seen[KT_COUNT];            // regions seen per class since enabling
    double units[KT_COUNT];        // summed work units of the recorded regions
    int cap;                       // event pairs per class
    int used[KT_COUNT];
    int dropped[KT_COUNT];
    cudaEvent_t* ev[KT_COUNT];     // 2*cap events per class
};
// Record the start / stop of a timed region of class k on stream s (no-op
// when timing is off or the pool is full).
void timer_start(const hol_ctx* c, int k, cudaStream_t s, double units = 0.0);
void timer_stop(const hol_ctx* c, int k, cudaStream_t s);

// Largest supported lattice side (one lane per column, L values per lane).
constexpr int kMaxL = 32;
// Most Arnoldi steps of hol_arnoldi_bounds.
constexpr int kArnoldiMax = 32;
// Blocks per right-hand side of the element-wise CG kernels (fixed, so the
// partial-sum banks have a fixed stride).
constexpr int kRedStride = 256;
// Number of partial-sum banks in hol_ctx::part.
constexpr int kBanks = 20;

// Device-side scalars kept by a context (FP64).
enum Scalar {
    S_BMIN = 0,   // lower bound of the Bbar spectrum (modulus)
    S_BMAX = 1,   // upper bound
    S_SF = 2,     // scratch for the fermion action
    S_COUNT = 8
};

// Chebyshev plan of the adiabatic preconditioner (set in hol_set_field).
struct KpmPlan {
    int max_np;          // capacity per omega
    int* np;             // [T/2]  polynomial order N_P(omega)
    double2* coef;       // [T/2][max_np] complex c_m(omega)
};

}  // namespace hol

struct hol_ctx {
    hol_params p;
    int L, N, T;
    long n;              // N * T
    int device;
    int sms;             // streaming multiprocessors of the device
    double th;           // tanh(dtau t): checkerboard bond [[1, th], [th, 1]]
    double ch4;          // cosh(dtau t)^4, folded into the stored exp(-dtau V)
                         // (1 with the exact propagator)
    int exact;           // kinetic == HOL_KINETIC_EXACT
    int kin_d64, kin_d32;            // exact propagator: taps kept in FP64 / FP32
    double kin_e[hol::kKinTaps];     // exact propagator: ring factor taps e[0..L/2]

    // field-derived data (hol_set_field)
    double* x;           // [T][N] copy of the field
    double* ev64;        // [T][N] cosh^4 exp(-dtau (alpha x - mu))
    float* ev32;         // [T][N] float copy
    double* dbar;        // [N] tau-average of ev64 (so cosh^4 times Eq. (expnVbar))
    double* scal;        // [S_COUNT] device scalars
    int field_set;

    hol::KpmPlan kpm;

    // solver workspace, sized for max_rhs right-hand sides
    double* part;        // partial sums, 4 banks of part_len doubles
    long part_len;
    double* v64a;        // FP64 vectors [max_rhs][T][N]
    double* v64b;
    double* v64c;
    double* v64d;
    double* v64e;
    float* v32a;         // FP32 vectors [max_rhs][T][N]
    float* v32b;
    float* v32c;
    float* v32d;
    float* v32e;
    int* mask;           // [2*max_rhs] active / reliable-update flags (device)
    double* v64f;
    float* v32f;
    float* v32g;         // merged / fused CG only (allocated when an option needs them)
    float* v32h;
    float* v32i;
    double* cgs;         // merged CG scalars [2][max_rhs][4]: alpha, gamma, mode
    double* alpha_buf;   // CG: alpha of an iteration whose x update is deferred [max_rhs]
    double* arn;         // Arnoldi: basis [kArnoldiMax + 1][N], H [kArnoldiMax + 1][kArnoldiMax],
                         // then one slot for the step count
    double2* tw64;       // [2T] exp(-i pi k / T)
    float2* tw32;
    double* md_phi;      // leapfrog: Phi [max_rhs][T][N]
    double* md_b;        // leapfrog: b = Lambda^{-T} Phi
    double* md_v;        // leapfrog: v = (M^T M)^{-1} b
    double* md_F;        // leapfrog: force / filter scratch [T][N]
    double* md_p;        // leapfrog: momentum [T][N]
    double* md_x0;       // leapfrog: x at the start of a trajectory
    double* md_g;        // leapfrog: mass tables [3][T]
    double* md_s;        // leapfrog: energy terms [16]
    double2* ms_acc;     // measurement accumulators [5][T][N] complex
    double2* twL64;      // [2L] exp(-i pi k / L)
    double2* cbuf0;      // complex half-spectrum buffers [max_rhs][T/2][N]
    double2* cbuf1;
    long cbuf_len;
    double* hbuf;        // pinned host staging (doubles)
    int* hflag;          // pinned host staging (ints)

    hol::KTimer* timer;  // kernel timers (nullptr until enabled)

    // per-shape launch choices
    int mv_k;            // tau slices per lane group in the matvec kernels
    int mv_warps;        // warps per block in the matvec kernels
    int mv_vec;          // use the float4 layout of the fused FP32 M^T M (L % 8 == 0)
    int kpm_reg;         // use the register KPM kernel (FP32, L = 16 or 32)
    int persist;         // use the persistent fused CG kernel when it fits
    int merged;          // mixed plain CG as one merged (Chronopoulos-Gear) kernel per iteration
    int fused;           // mixed plain CG with the vector update fused into the operator
    int pdl;             // programmatic dependent launch of the CG kernels

    // graph-captured (device-driven) solves: device-side decision state and
    // the side streams that capture the bodies of conditional graph nodes
    double* dcg;         // hol::DcgState storage (see dcg_state)
    cudaStream_t cap_s[3];
    int capturing;       // set while the context's work is being captured

    // alpha of the current mixed CG iteration per rhs, formed by the last warp
    // of the operator kernel (cg_alpha_epilogue), and that kernel's per-rhs
    // count of finished warps (zero between launches)
    double* alpha_now;
    int* alpha_cnt;
    // beta of the next plain mixed CG iteration per rhs, formed by the last
    // block of the update kernel, and that kernel's per-rhs block count
    double* beta_now;
    int* beta_cnt;
    int handoff;         // launch option "scalar_handoff": bit 0 alpha_now, bit 1 beta_now in use
    int kpm_queue;       // launch option "kpm_queue": persistent register-KPM grid of this many
                         // blocks per multiprocessor (0: one block per problem)
    int* kpm_q;          // its work queue [2] (next problem, finished blocks; zero between launches)
    double kpm_a1, kpm_a2;   // constants of the Chebyshev order heuristic (1, 1 by default)
    int pc_fuse;             // PCG: vector update fused into the preconditioner's transform
};

namespace hol {
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(const hol_ctx* c, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                       size_t smem, cudaStream_t s, Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = c->pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
}  // namespace hol

namespace hol {

// fermion operator kernels (matvec.cu) -----------------------------------------
enum MtEpilogue { MT_PLAIN = 0, MT_RESID = 1 };

// out = M v (double or float per prec). norm_part (nullable): per-unit
// sums of |out|^2 at stride matvec_pstride(c) per right-hand side.
// Resident blocks per SM of the FP64 operator kernels that take their own
// slice grouping, by [exact propagator][M, M^T, residual M^T, the FP64 CG's
// M][L][warps per block] (0: not yet queried); filled by occ64_warm at
// context creation.
extern std::atomic<int> g_occ64[2][4][33][5];
void occ64_warm(const hol_ctx* c);         // matvec.cu (checkerboard)
void occ64_warm_exact(const hol_ctx* c);   // exact.cu
// PCG: the CG vector update (r -= alpha q with alpha = (r.z) / (p.q) from
// the partials, the deferred x update of k_cg_update's FOLD modes, the
// partials of the new r.r) fused into the forward tau transform of the
// preconditioner application that follows it (precond_apply_upd).
struct PcUpd {
    void* x;               // solution accumulator (FP32 e or FP64 x)
    const void* p;         // this iteration's direction
    const void* pprev;     // the previous one (fold 2)
    const void* q;         // A p
    const int* mask;       // active right-hand sides
    const double* pq_part; // p.q unit partials
    int pq_stride, pq_n;
    const double* dz_part; // r.z partials (kRedStride per rhs)
    int dz_n;
    double* rr_out;        // new r.r partials, one per transform tile
    double* alpha_buf;     // alpha of the previous iteration (fold 0 writes, 2 reads)
    int fold;              // 0, 1 or 2 as k_cg_update's FOLD
};
// z = P^{-1} P^{-T} r after r has been updated in place as `u` says; dot_part
// receives the r.z partials (precond_tiles per rhs). prec HOL_F32 or HOL_F64.
int precond_apply_upd(hol_ctx* c, int prec, void* r, void* z, int n_rhs, const PcUpd* u,
                      double* dot_part, cudaStream_t s);

// Stride and count of the |Mp|^2 unit partials that the FP64 CG's M// Stride and count of the |Mp|^2 unit partials that the FP64 CG's M
// (launch_M_upd64) writes for n_rhs right-hand sides.
void fp64_cg_geom(const hol_ctx* c, int n_rhs, int* pstride, int* nrun);

int launch_M(const hol_ctx* c, int prec, const void* v, void* out, int n_rhs,
             const int* mask, double* norm_part, cudaStream_t s);
// Where the CG beta = rr_new / rr_old of each right-hand side comes from:
// partial sums at rn[rhs*stride + k] and ro[rhs*stride + k], k < n.
struct BetaSrc {
    const double* rn;
    const double* ro;
    int stride;
    int n;
    int first;   // nonzero: beta = 0
};
// FP64 CG direction update fused with M: pnew = r + beta pold, w = M pnew.
int launch_M_upd64(const hol_ctx* c, const double* r, const double* pold, double* pnew,
                   double* w, int n_rhs, const int* mask, BetaSrc beta,
                   double* norm_part, cudaStream_t s);
// out = M^T u.
int launch_MT(const hol_ctx* c, int prec, const void* u, void* out, int n_rhs,
              const int* mask, cudaStream_t s);
// FP64: out = b - M^T u.
int launch_MT_resid64(const hol_ctx* c, const double* u, const double* b, double* out,
                      int n_rhs, const int* mask, cudaStream_t s);
// FP32 fused CG step: pnew = r + beta pold (beta from the partial sums
// rr_new / rr_old, 0 when first), q = M^T M pnew, pq_part = |M pnew|^2.
// pnew and pq_part may be null.
int launch_cg_mtm32(const hol_ctx* c, const float* r, const float* pold, float* pnew,
                    float* q, int n_rhs, const int* mask, const double* rr_new,
                    const double* rr_old, int rr_stride, int rr_n, int first,
                    double* pq_part, cudaStream_t s,
                    double* alpha_out = nullptr, int* alpha_done = nullptr,
                    const double* beta_in = nullptr);
// The same five operators with the exact propagator exp(-dtau K) (exact.cu;
// scalar layout only). The launch_* calls above forward to these when the
// context was created with HOL_KINETIC_EXACT.
int launch_M_exact(const hol_ctx* c, int prec, const void* v, void* out, int n_rhs,
                   const int* mask, double* norm_part, cudaStream_t s);
int launch_M_upd64_exact(const hol_ctx* c, const double* r, const double* pold, double* pnew,
                         double* w, int n_rhs, const int* mask, BetaSrc beta,
                         double* norm_part, cudaStream_t s);
int launch_MT_exact(const hol_ctx* c, int prec, const void* u, void* out, int n_rhs,
                    const int* mask, cudaStream_t s);
int launch_MT_resid64_exact(const hol_ctx* c, const double* u, const double* b, double* out,
                            int n_rhs, const int* mask, cudaStream_t s);
int launch_cg_mtm32_exact(const hol_ctx* c, const float* r, const float* pold, float* pnew,
                          float* q, int n_rhs, const int* mask, const double* rr_new,
                          const double* rr_old, int rr_stride, int rr_n, int first,
                          double* pq_part, cudaStream_t s);
// Device-side state of a graph-captured CG solve (one context): per right-hand
// side its |b|, the previous and the current chunk's residual sums, the true
// residual, iteration and since-last-reliable-update counts and the converged
// flag; plus solve-wide counters g[DCG_*] (DCG_STICKY collects failures of
// every solve since it was last cleared).
enum DcgSlot { DCG_KIT = 0, DCG_HAVE_PREV = 1, DCG_ERR = 2, DCG_ERR_RHS = 3, DCG_LOOPS = 4,
               DCG_STICKY = 5, DCG_COUNT = 8 };
struct DcgState {
    double* bnorm;
    double* prev;
    double* cur;
    double* tres;
    int* it;
    int* since;
    int* done;
    int* g;
};
inline size_t dcg_bytes(long R)
{
    return (size_t)(4 * R) * sizeof(double) + (size_t)(3 * R + DCG_COUNT) * sizeof(int);
}
inline DcgState dcg_state(const hol_ctx* c)
{
    const long R = c->p.max_rhs;
    DcgState d;
    d.bnorm = c->dcg;
    d.prev = c->dcg + R;
    d.cur = c->dcg + 2 * R;
    d.tres = c->dcg + 3 * R;
    int* ib = reinterpret_cast<int*>(c->dcg + 4 * R);
    d.it = ib;
    d.since = ib + R;
    d.done = ib + 2 * R;
    d.g = ib + 3 * R;
    return d;
}
// Graph-capturable CG: the solve of cg_solve (the same kernels and the same
// decisions, so bitwise the same result) with every decision taken on the
// device: the chunk loop is a WHILE node and the reliable update an IF node.
// `s` must be capturing in thread-local mode, inside a CaptureScope; needs an
// even check_every and the default two-kernel iteration. Per-rhs results stay
// in dcg_state(c) and v.
int cg_run_dev(hol_ctx* c, const double* b, double* v, int n_rhs, const hol_cg_opts* o,
               cudaStream_t s);
// Conditional nodes in a capturing stream: cond_handle creates a handle in the
// graph being captured on s (capture the kernel that sets it next);
// cond_node appends the node after the stream's current dependencies, makes
// it the new dependency and returns its (first) body graph.
int cond_handle(cudaStream_t s, cudaGraphConditionalHandle* h);
int cond_node(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
              cudaGraph_t* body);
// While a context's work is captured: no programmatic launches and no timer
// events (neither may sit in a conditional body), and solves device-driven.
struct CaptureScope {
    hol_ctx* c;
    int pdl;
    KTimer* timer;
    explicit CaptureScope(hol_ctx* ctx) : c(ctx), pdl(ctx->pdl), timer(ctx->timer)
    {
        c->pdl = 0;
        c->timer = nullptr;
        c->capturing = 1;
    }
    ~CaptureScope()
    {
        c->pdl = pdl;
        c->timer = timer;
        c->capturing = 0;
    }
    CaptureScope(const CaptureScope&) = delete;
    CaptureScope& operator=(const CaptureScope&) = delete;
};
// Propagator parameters of a context for kernels computing in R.
template <typename R>
inline Kin<R> kin_of(const hol_ctx* c)
{
    Kin<R> k;
    k.th = (R)c->th;
    k.D = c->exact ? (sizeof(R) == 8 ? c->kin_d64 : c->kin_d32) : 0;
    for (int d = 0; d < kKinTaps; ++d) k.e[d] = (R)c->kin_e[d];
    return k;
}
// Persistent fused CG chunk (persist.cu); HOL_EINVAL without launching when
// unsupported (L % 8 != 0) or when the cooperative grid cannot be resident.
int launch_cg_persist(const hol_ctx* c, float* r, float* p0, float* p1, float* e, int n_rhs,
                      const int* mask, double* pq, double* rr0, double* rr1, int cur, int cnt_cur,
                      int cnt_old, int pp, int first, int nit, int check_only, cudaStream_t s);
// Scalars of one merged (single-reduction) CG iteration; see cg.cu.
struct MergedScal {
    const double* slot_in;   // [rhs*4 + {alpha_prev, gamma_prev, mode}]
    double* slot_out;        // alpha, gamma of this iteration, mode 0
    const double* g_in;      // unit partials of gamma = r.r (mode 0)
    const double* d_in;      // unit partials of delta = r.(M^T M r)
    double* g_out;           // unit partials of the next gamma, delta
    double* d_out;
    const double* gr;        // block partials of gamma after a (re)start (modes 1, 2)
    const double* rho;       // block partials of r.s_old (mode 1)
    int e_n;                 // block partial count of gr and rho
    const double* pi;        // unit partials of p_old.(M^T M p_old) (mode 1)
    int fold;                // 0: defer the x update, 1: x += a p, 2: x += a_prev p_old + a p
};
// One merged CG iteration (float4 layout, L % 8 == 0).
int launch_cg_merged(const hol_ctx* c, const float* r, const float* w, const float* pold,
                     const float* sold, float* e, float* pnew, float* snew, float* rnew,
                     float* wnew, int n_rhs, const int* mask, const MergedScal& sc,
                     cudaStream_t s);
// Unit partials of the fused CG iteration (layout of matvec_pstride / nrun).
struct FusedPartials {
    const double* g;    // r.r, p.q, r.q, q.q of the current iteration
    const double* pq;
    const double* rq;
    const double* qq;
    double* g_out;      // the same for the next iteration
    double* pq_out;
    double* rq_out;
    double* qq_out;
};
// One fused CG iteration (vector update + next operator; float4 layout).
int launch_cg_fused(const hol_ctx* c, const float* r, const float* q, const float* pold, float* x,
                    float* rnew, float* pnew, float* qnew, int n_rhs, const int* mask,
                    const FusedPartials& fp, cudaStream_t s);
// Unit partials of r.r, r.q, q.q for the flagged rhs.
int launch_unit_dots(const hol_ctx* c, const float* r, const float* q, int n_rhs,
                     const int* mask, double* g_out, double* rq_out, double* qq_out,
                     cudaStream_t s);
int matvec_pstride(const hol_ctx* c);          // per-rhs stride of unit partials
int matvec_units(const hol_ctx* c, int n_rhs); // upper bound of units per call

// Lambda^T (transpose_forward) or Lambda^{-T} applied to nv vectors.
int launch_lambda(const hol_ctx* c, bool transpose_forward, const double* w, double* out,
                  int nv, cudaStream_t s);
int launch_force(hol_ctx* c, const double* v, const double* b, int n_pf, double* F,
                 int with_bos, double* S_F, cudaStream_t s);
// out2[0] = S_B(x), out2[1] = (1/2) sum b . v over n_pf vectors (leapfrog.cu).
int launch_action_terms(const hol_ctx* c, const double* x, const double* b, const double* v,
                        int n_pf, double* out2, cudaStream_t s);
int elementwise_blocks(const hol_ctx* c, int n_rhs);

// preconditioner (precond.cu). mode bit 0: P^{-T} part, bit 1: P^{-1} part
// (both: P^{-1} P^{-T}). rdot/dot_part (nullable): partial sums of out . rdot
// per (rhs, tile) at stride kRedStride, precond_tiles(c, prec) per rhs.
int precond_alloc(hol_ctx* c);
int leapfrog_alloc(hol_ctx* c);
// Parts of one HMC trajectory (leapfrog.cu) replayed by the captured batch
// (graph.cu): md_start (Phi, p, the initial energies in md_s[0..2], the first
// force and half kick, the kick coefficient for the next step), md_step (one
// leapfrog step ending with the kick by md_s[kKickSlot]), md_set_kick, md_end
// (tight action solve, final energies in md_s[3..5]); md_check validates the
// options as fourier_accel_leapfrog does.
constexpr int kKickSlot = 12;
int md_start(hol_ctx* c, double* x, const double* R_pf, const double* R_p, int n_pf,
             const hol_md_opts* o, cudaStream_t s);
int md_set_kick(hol_ctx* c, double kick, cudaStream_t s);
int md_step(hol_ctx* c, double* x, int n_pf, const hol_md_opts* o, cudaStream_t s);
int md_end(hol_ctx* c, double* x, int n_pf, const hol_md_opts* o, cudaStream_t s);
int md_check(const hol_ctx* c, const hol_md_opts* o, int n_pf);
// The measurement of stochastic_measure on stream s (measure.cu): inside a
// graph capture its solves are device-driven and `iters` must be null;
// measure_prepare raises the kernels' shared-memory limits beforehand.
int measure_run(hol_ctx* c, const double* xi, int n_rv, const hol_cg_opts* opts, double* Gxi,
                double* G2, double* G4, int four_point, int* iters, cudaStream_t s);
int measure_prepare(hol_ctx* c);
int measure_alloc(hol_ctx* c);
int precond_check_shape(const hol_ctx* c);
int precond_tiles(const hol_ctx* c, int prec);
int precond_apply_impl(hol_ctx* c, int prec, const void* v, void* out, int n_rhs, int mode,
                       const void* rdot, double* dot_part, cudaStream_t s);

// helpers ----------------------------------------------------------------------
inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace hol
