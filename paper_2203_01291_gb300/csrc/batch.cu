// Batched independent chains (host-side scheduler).
//
// Chains of different lattice sizes cannot share one kernel launch without
// padding every chain to the largest shape; instead each chain keeps its own
// context and runs on its own CUDA stream, and a pool of host threads drives
// the chains concurrently so that the GPU interleaves their kernels. Every
// chain's solver synchronises only its own stream (cg_solve polls), so one
// slow chain never stalls the others. Results are per chain and identical to
// running the chains one by one (each chain's arithmetic is unchanged).
#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

using namespace hol;

namespace {

template <typename F>
int run_pool(int n, int n_threads, F&& work)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n) n_threads = n;
    std::atomic<int> next(0);
    std::atomic<int> first_err(0);
    std::mutex mu;
    std::string msg;
    int bad = -1;
    int device = 0;
    cudaGetDevice(&device);
    auto body = [&]() {
        cudaSetDevice(device);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            int z = 0;
            first_err.compare_exchange_strong(z, HOL_ECUDA);
            return;
        }
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= n) break;
            const int rc = work(k, s);
            if (rc) {
                int z = 0;
                if (first_err.compare_exchange_strong(z, rc)) {
                    std::lock_guard<std::mutex> lock(mu);
                    msg = hol_last_error();   // the worker thread's message
                    bad = k;
                }
            }
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < n_threads; ++t) pool.emplace_back(body);
    for (auto& th : pool) th.join();
    const int rc = first_err.load();
    if (rc) return set_error(rc, "chain %d: %s", bad, msg.c_str());
    return HOL_OK;
}

}  // namespace

extern "C" int hmc_batch(hol_ctx* const* ctxs, int n_chains, double* const* x,
                         const double* const* R_pf, const double* const* R_p, int n_pf,
                         const hol_md_opts* opts, const double* u, int* accepted, double* dH,
                         int n_threads)
{
    HOL_TRACE("hmc_batch");
    if (!ctxs || !x || !R_pf || !R_p || !opts || !u || n_chains < 1)
        return set_error(HOL_EINVAL, "hmc_batch: bad argument");
    for (int k = 0; k < n_chains; ++k)
        if (!ctxs[k] || !x[k] || !R_pf[k] || !R_p[k])
            return set_error(HOL_EINVAL, "hmc_batch: null entry for chain %d", k);
    return run_pool(n_chains, n_threads, [&](int k, cudaStream_t s) {
        int acc = 0;
        double d = 0.0;
        const int rc = fourier_accel_leapfrog(ctxs[k], x[k], R_pf[k], R_p[k], n_pf, opts, u[k], &acc,
                                              &d, nullptr, (void*)s);
        if (accepted) accepted[k] = acc;
        if (dH) dH[k] = d;
        return rc;
    });
}

extern "C" int measure_batch(hol_ctx* const* ctxs, int n_chains, const double* const* xi, int n_rv,
                             const hol_cg_opts* opts, double* const* Gxi, double* const* G2,
                             double* const* G4, int four_point, int n_threads)
{
    HOL_TRACE("measure_batch");
    if (!ctxs || !xi || !opts || !Gxi || !G2 || n_chains < 1)
        return set_error(HOL_EINVAL, "measure_batch: bad argument");
    return run_pool(n_chains, n_threads, [&](int k, cudaStream_t s) {
        return stochastic_measure(ctxs[k], xi[k], n_rv, opts, Gxi[k], G2[k],
                                  G4 ? G4[k] : nullptr, four_point, nullptr, (void*)s);
    });
}
