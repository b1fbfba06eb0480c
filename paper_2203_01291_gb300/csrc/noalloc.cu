// Allocation-free variant of the FP64 fermion operator.
//
// Some callers cannot call cudaMalloc: their device memory is owned entirely
// by another allocator (a framework's caching allocator, or a fixed budget
// reserved at start-up), or they must not trigger the device-wide
// synchronisation that cudaMalloc and cudaFree can imply. For them
// fermion_matvec_static computes M v, M^T v or M^T M v in FP64 without a
// context: its scratch (the exp(-dtau V) table and, for M^T M, the
// intermediate M v) lives in one file-scope __device__ array of fixed size,
// present on every GPU that loads this library until the process exits.
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace hol {
namespace {

constexpr long kStaticDoubles = 1L << 20;   // 8 MiB of FP64 scratch per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

std::mutex g_static_mu;
double* g_static_addr[kMaxDevices];

// Device address of g_static_scratch on the current device. In host code the
// symbol itself is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int static_scratch(double** out)
{
    int dev = -1;
    HOL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(HOL_EINVAL, "fermion_matvec_static: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (g_static_addr[dev] == nullptr) {
        void* p = nullptr;
        HOL_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_addr[dev] = (double*)p;
    }
    *out = g_static_addr[dev];
    return HOL_OK;
}

// cosh^4 exp(-dtau (alpha x - mu)): the diagonal with the cosh factors of
// the checkerboard colours folded in, as the operator kernels expect
__global__ void k_expv_static(const double* __restrict__ x, double* __restrict__ ev, long n,
                              double dtau, double alpha, double mu, double ch4)
{
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
         k += (long)gridDim.x * blockDim.x)
        ev[k] = ch4 * exp(-dtau * (alpha * x[k] - mu));
}

}  // namespace
}  // namespace hol

using namespace hol;

extern "C" int fermion_matvec_static(const hol_params* p, const double* x, int op, const double* v,
                                     double* out, int n_rhs, void* stream)
{
    HOL_TRACE("fermion_matvec_static");
    if (!p || !x || !v || !out) return set_error(HOL_EINVAL, "fermion_matvec_static: null argument");
    if (int rc_ = require_aligned("fermion_matvec_static", {x, v, out})) return rc_;
    if (p->L < 4 || p->L > kMaxL || (p->L & 1) || p->Ltau < 2 || (p->Ltau & 1))
        return set_error(HOL_EINVAL, "fermion_matvec_static: unsupported L=%d Ltau=%d", p->L,
                         p->Ltau);
    if (op != HOL_OP_M && op != HOL_OP_MT && op != HOL_OP_MTM)
        return set_error(HOL_EINVAL, "fermion_matvec_static: bad op %d", op);
    if (n_rhs < 1) return set_error(HOL_EINVAL, "fermion_matvec_static: n_rhs=%d", n_rhs);
    if (!(p->dtau > 0.0) || !isfinite(p->t) || !isfinite(p->mu) || !isfinite(p->alpha))
        return set_error(HOL_EINVAL, "fermion_matvec_static: dtau must be > 0 and t, mu, alpha "
                                     "finite");
    if (p->kinetic != HOL_KINETIC_CHECKERBOARD)
        return set_error(HOL_EINVAL, "fermion_matvec_static: checkerboard propagator only");
    const long n = (long)p->L * p->L * p->Ltau;
    const size_t vbytes = (size_t)n_rhs * (size_t)n * sizeof(double);
    if (ranges_overlap(v, vbytes, out, vbytes))
        return set_error(HOL_EINVAL, "fermion_matvec_static: v and out must not overlap");
    const long need = n + (op == HOL_OP_MTM ? (long)n_rhs * n : 0);
    if (need > kStaticDoubles)
        return set_error(HOL_EINVAL,
                         "fermion_matvec_static: needs %ld doubles of scratch, the static "
                         "maximum is %ld (N*Ltau, plus n_rhs*N*Ltau for M^T M)",
                         need, kStaticDoubles);
    double* scratch = nullptr;
    int rc = static_scratch(&scratch);
    if (rc) return rc;

    // a context on the stack that points at the static scratch
    hol_ctx c = {};
    c.p = *p;
    c.L = p->L;
    c.N = p->L * p->L;
    c.T = p->Ltau;
    c.n = n;
    c.th = tanh(p->dtau * p->t);
    const double ch = cosh(p->dtau * p->t);
    c.ch4 = ch * ch * ch * ch;
    c.mv_k = (c.T % 4 == 0 && c.T >= 8) ? 2 : 1;
    c.mv_warps = 4;
    c.ev64 = scratch;
    cudaStream_t s = (cudaStream_t)stream;
    int nb = (int)((n + 255) / 256);
    if (nb > 4096) nb = 4096;
    k_expv_static<<<nb, 256, 0, s>>>(x, scratch, n, p->dtau, p->alpha, p->mu, c.ch4);
    HOL_CHECK_LAUNCH("k_expv_static");
    switch (op) {
    case HOL_OP_M:
        return launch_M(&c, HOL_F64, v, out, n_rhs, nullptr, nullptr, s);
    case HOL_OP_MT:
        return launch_MT(&c, HOL_F64, v, out, n_rhs, nullptr, s);
    default:
        rc = launch_M(&c, HOL_F64, v, scratch + n, n_rhs, nullptr, nullptr, s);
        if (rc) return rc;
        return launch_MT(&c, HOL_F64, scratch + n, out, n_rhs, nullptr, s);
    }
}
