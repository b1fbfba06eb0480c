// Solves and batched HMC trajectories as CUDA graphs with device-side control.
//
// cg_solve_graph captures one cg_solve (cg_run_dev in cg.cu: the chunk loop
// a conditional WHILE node, the reliable update a conditional IF node, every
// decision on the device) and launches it once: no host round trip inside the
// solve. hmc_batch_graph runs one HMC trajectory (Algorithm 1) for many
// independent chains, possibly of different lattice sizes: all chains' start
// (pseudofermions, momenta, initial energies, first force), one leapfrog step
// and the end (the tight action solve, final energies) are each captured once
// into one graph over all chains (each chain on its own forked stream inside
// the capture), and the step graph is launched N_t times. The host only reads
// the energies at the end for the Metropolis decisions. Each chain computes
// exactly what fourier_accel_leapfrog computes for it (same kernels, same
// decisions, bitwise the same numbers). measure_batch_graph captures every
// chain's stochastic measurement (probe solves and FFT accumulation) into one
// graph the same way.
#include <math.h>

#include <vector>

#include "internal.cuh"

namespace hol {
namespace {

struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    ~Graph()
    {
        if (e) cudaGraphExecDestroy(e);
        if (g) cudaGraphDestroy(g);
    }
};

struct Streams {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> e;
    ~Streams()
    {
        for (cudaStream_t x : s)
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
    int create(int ns, int ne)
    {
        s.assign(ns, nullptr);
        e.assign(ne, nullptr);
        for (cudaStream_t& x : s) HOL_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        for (cudaEvent_t& x : e) HOL_CUDA(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        return HOL_OK;
    }
};

// Capture body() on s (thread-local mode) into g and instantiate it. The
// capture is always ended, also when body() fails.
template <class F>
int capture(cudaStream_t s, Graph& g, F&& body)
{
    HOL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int rc = body();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "graph capture");
    g.g = graph;
    HOL_CUDA(cudaGraphInstantiate(&g.e, graph, 0));
    return HOL_OK;
}

// Capture per-chain work on forked streams: origin -> fork -> each chain on
// a stream -> join back into origin. With width w < n, chain k runs on
// stream k % w after the chains before it on that stream (at most w chains
// in flight; their working sets then share L2 with fewer others). Every
// forked stream is joined, also after a failure, so the capture can always
// be ended.
template <class F>
int fork_join(cudaStream_t origin, Streams& st, int n, F&& work, int width = 0)
{
    const int w = (width > 0 && width < n) ? width : n;
    HOL_CUDA(cudaEventRecord(st.e[0], origin));
    for (int j = 0; j < w; ++j) HOL_CUDA(cudaStreamWaitEvent(st.s[j], st.e[0], 0));
    int first_rc = HOL_OK;
    for (int k = 0; k < n; ++k)
        if (first_rc == HOL_OK) first_rc = work(k, st.s[k % w]);
    for (int j = 0; j < w; ++j) {
        HOL_CUDA(cudaEventRecord(st.e[1 + j], st.s[j]));
        HOL_CUDA(cudaStreamWaitEvent(origin, st.e[1 + j], 0));
    }
    return first_rc;
}

int check_graph_solver(const hol_ctx* c, const hol_cg_opts* o, const char* fn)
{
    const int chk = o->check_every > 0 ? o->check_every : 10;
    if (chk & 1) return set_error(HOL_EINVAL, "%s: check_every must be even (%d)", fn, chk);
    if (c->fused || c->merged || c->persist)
        return set_error(HOL_EINVAL, "%s: needs the two-kernel CG iteration (fused_cg, "
                                     "merged_cg and persistent_cg off)", fn);
    if (o->prec != HOL_F64 && o->prec != HOL_F32)
        return set_error(HOL_EINVAL, "%s: bad precision %d", fn, o->prec);
    if (!(o->tol > 0.0) || o->max_iter < 1)
        return set_error(HOL_EINVAL, "%s: tol must be > 0 and max_iter >= 1", fn);
    return HOL_OK;
}

}  // namespace
}  // namespace hol

using namespace hol;

extern "C" int cg_solve_graph(hol_ctx* c, const double* b, double* v, int n_rhs,
                              const hol_cg_opts* o, int* iters, double* resid, void* stream)
{
    HOL_TRACE("cg_solve_graph");
    if (!c || !b || !v || !o) return set_error(HOL_EINVAL, "cg_solve_graph: null argument");
    if (int rc_ = require_aligned("cg_solve_graph", {b, v})) return rc_;
    if (!c->field_set) return set_error(HOL_EINVAL, "cg_solve_graph: hol_set_field not called");
    if (n_rhs < 1 || n_rhs > c->p.max_rhs)
        return set_error(HOL_EINVAL, "cg_solve_graph: n_rhs=%d outside [1, %d]", n_rhs,
                         c->p.max_rhs);
    if (int rc_ = check_graph_solver(c, o, "cg_solve_graph")) return rc_;
    if (b == v) return set_error(HOL_EINVAL, "cg_solve_graph: b and v must not overlap");
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t os = c->cap_s[2];
    Streams st;
    if (int rc_ = st.create(0, 2)) return rc_;
    HOL_CUDA(cudaEventRecord(st.e[0], user));
    HOL_CUDA(cudaStreamWaitEvent(os, st.e[0], 0));
    const DcgState d = dcg_state(c);
    HOL_CUDA(cudaMemsetAsync(d.g, 0, DCG_COUNT * sizeof(int), os));
    Graph g;
    int rc;
    {
        CaptureScope scope(c);
        rc = capture(os, g, [&]() { return cg_run_dev(c, b, v, n_rhs, o, os); });
    }
    if (rc) return rc;
    HOL_CUDA(cudaGraphLaunch(g.e, os));
    std::vector<int> ih(3 * n_rhs + DCG_COUNT);
    std::vector<double> th(n_rhs);
    HOL_CUDA(cudaMemcpyAsync(ih.data(), d.it, n_rhs * sizeof(int), cudaMemcpyDeviceToHost, os));
    HOL_CUDA(cudaMemcpyAsync(ih.data() + n_rhs, d.done, n_rhs * sizeof(int),
                             cudaMemcpyDeviceToHost, os));
    HOL_CUDA(cudaMemcpyAsync(ih.data() + 3 * n_rhs, d.g, DCG_COUNT * sizeof(int),
                             cudaMemcpyDeviceToHost, os));
    HOL_CUDA(cudaMemcpyAsync(th.data(), d.tres, n_rhs * sizeof(double), cudaMemcpyDeviceToHost,
                             os));
    HOL_CUDA(cudaStreamSynchronize(os));
    HOL_CUDA(cudaEventRecord(st.e[1], os));
    HOL_CUDA(cudaStreamWaitEvent(user, st.e[1], 0));
    int all = 1;
    for (int k = 0; k < n_rhs; ++k) {
        if (iters) iters[k] = ih[k];
        if (resid) resid[k] = th[k];
        all &= ih[n_rhs + k];
    }
    const int* gs = ih.data() + 3 * n_rhs;
    if (gs[DCG_ERR])
        return set_error(HOL_ENUMERIC, "cg_solve_graph: non-finite residual (rhs %d)",
                         gs[DCG_ERR_RHS]);
    if (!all)
        return set_error(HOL_ENOTCONV, "cg_solve_graph: not converged within %d iterations",
                         o->max_iter);
    return HOL_OK;
}

extern "C" int hmc_batch_graph(hol_ctx* const* ctxs, int n_chains, double* const* x,
                               const double* const* R_pf, const double* const* R_p, int n_pf,
                               const hol_md_opts* o, const double* u, int* accepted, double* dH,
                               void* stream)
{
    HOL_TRACE("hmc_batch_graph");
    if (!ctxs || !x || !R_pf || !R_p || !o || !u || n_chains < 1)
        return set_error(HOL_EINVAL, "hmc_batch_graph: null argument or no chains");
    if (o->n_steps < 1) return set_error(HOL_EINVAL, "hmc_batch_graph: n_steps >= 1 required");
    for (int k = 0; k < n_chains; ++k) {
        hol_ctx* c = ctxs[k];
        if (!c || !x[k] || !R_pf[k] || !R_p[k])
            return set_error(HOL_EINVAL, "hmc_batch_graph: null argument (chain %d)", k);
        if (int rc_ = require_aligned("hmc_batch_graph", {x[k], R_pf[k], R_p[k]})) return rc_;
        if (int rc_ = md_check(c, o, n_pf)) return rc_;
        if (int rc_ = check_graph_solver(c, &o->cg_force, "hmc_batch_graph")) return rc_;
        if (int rc_ = check_graph_solver(c, &o->cg_action, "hmc_batch_graph")) return rc_;
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c)
                return set_error(HOL_EINVAL, "hmc_batch_graph: context of chain %d repeated", k);
    }
    cudaStream_t user = (cudaStream_t)stream;
    Streams st;
    if (int rc_ = st.create(n_chains + 1, n_chains + 2)) return rc_;
    cudaStream_t os = st.s[n_chains];
    HOL_CUDA(cudaEventRecord(st.e[n_chains + 1], user));
    HOL_CUDA(cudaStreamWaitEvent(os, st.e[n_chains + 1], 0));
    for (int k = 0; k < n_chains; ++k)
        HOL_CUDA(cudaMemsetAsync(dcg_state(ctxs[k]).g, 0, DCG_COUNT * sizeof(int), os));

    Graph g_start, g_step, g_end;
    int rc;
    {
        std::vector<CaptureScope*> scopes;
        for (int k = 0; k < n_chains; ++k) scopes.push_back(new CaptureScope(ctxs[k]));
        rc = capture(os, g_start, [&]() {
            return fork_join(os, st, n_chains, [&](int k, cudaStream_t sk) {
                return md_start(ctxs[k], x[k], R_pf[k], R_p[k], n_pf, o, sk);
            });
        });
        if (!rc)
            rc = capture(os, g_step, [&]() {
                return fork_join(os, st, n_chains, [&](int k, cudaStream_t sk) {
                    return md_step(ctxs[k], x[k], n_pf, o, sk);
                });
            });
        if (!rc)
            rc = capture(os, g_end, [&]() {
                return fork_join(os, st, n_chains, [&](int k, cudaStream_t sk) {
                    return md_end(ctxs[k], x[k], n_pf, o, sk);
                });
            });
        for (CaptureScope* p : scopes) delete p;
    }
    if (rc) return rc;

    HOL_CUDA(cudaGraphLaunch(g_start.e, os));
    for (int t = 0; t < o->n_steps; ++t) {
        if (t + 1 == o->n_steps && o->n_steps > 1)   // the closing half kick
            for (int k = 0; k < n_chains; ++k)
                if ((rc = md_set_kick(ctxs[k], 0.5 * o->dt, os))) return rc;
        HOL_CUDA(cudaGraphLaunch(g_step.e, os));
    }
    HOL_CUDA(cudaGraphLaunch(g_end.e, os));

    std::vector<double> h(6 * (size_t)n_chains);
    std::vector<int> gs(DCG_COUNT * (size_t)n_chains);
    for (int k = 0; k < n_chains; ++k) {
        HOL_CUDA(cudaMemcpyAsync(h.data() + 6 * k, ctxs[k]->md_s, 6 * sizeof(double),
                                 cudaMemcpyDeviceToHost, os));
        HOL_CUDA(cudaMemcpyAsync(gs.data() + DCG_COUNT * k, dcg_state(ctxs[k]).g,
                                 DCG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, os));
    }
    HOL_CUDA(cudaStreamSynchronize(os));
    int bad = HOL_OK, bad_k = -1;
    for (int k = 0; k < n_chains && bad == HOL_OK; ++k)
        if (gs[DCG_COUNT * k + DCG_STICKY]) {
            bad = gs[DCG_COUNT * k + DCG_STICKY];
            bad_k = k;
        }
    if (bad != HOL_OK) {
        HOL_CUDA(cudaEventRecord(st.e[0], os));
        HOL_CUDA(cudaStreamWaitEvent(user, st.e[0], 0));
        return set_error(bad, "hmc_batch_graph: a solve of chain %d %s", bad_k,
                         bad == HOL_ENUMERIC ? "met a non-finite residual" : "did not converge");
    }
    for (int k = 0; k < n_chains; ++k) {
        const double* hk = h.data() + 6 * k;
        const double d = (hk[3] + hk[4] + hk[5]) - (hk[0] + hk[1] + hk[2]);
        if (!isfinite(d)) return set_error(HOL_ENUMERIC, "hmc_batch_graph: non-finite dH (chain %d)", k);
        const int acc = (u[k] < exp(-d)) ? 1 : 0;
        if (!acc)
            HOL_CUDA(cudaMemcpyAsync(x[k], ctxs[k]->md_x0, ctxs[k]->n * sizeof(double),
                                     cudaMemcpyDeviceToDevice, os));
        if (accepted) accepted[k] = acc;
        if (dH) dH[k] = d;
    }
    HOL_CUDA(cudaStreamSynchronize(os));
    HOL_CUDA(cudaEventRecord(st.e[0], os));
    HOL_CUDA(cudaStreamWaitEvent(user, st.e[0], 0));
    return HOL_OK;
}

extern "C" int measure_batch_graph(hol_ctx* const* ctxs, int n_chains, const double* const* xi,
                                   int n_rv, const hol_cg_opts* opts, double* const* Gxi,
                                   double* const* G2, double* const* G4, int four_point,
                                   int concurrency, void* stream)
{
    HOL_TRACE("measure_batch_graph");
    if (!ctxs || !xi || !opts || !Gxi || !G2 || n_chains < 1)
        return set_error(HOL_EINVAL, "measure_batch_graph: null argument or no chains");
    if (four_point && !G4)
        return set_error(HOL_EINVAL, "measure_batch_graph: four-point products need G4");
    if (concurrency < 0)
        return set_error(HOL_EINVAL, "measure_batch_graph: concurrency must be >= 0");
    for (int k = 0; k < n_chains; ++k) {
        hol_ctx* c = ctxs[k];
        if (!c || !xi[k] || !Gxi[k] || !G2[k] || (four_point && !G4[k]))
            return set_error(HOL_EINVAL, "measure_batch_graph: null argument (chain %d)", k);
        if (int rc_ = check_graph_solver(c, opts, "measure_batch_graph")) return rc_;
        if (int rc_ = measure_prepare(c)) return rc_;
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == c)
                return set_error(HOL_EINVAL, "measure_batch_graph: context of chain %d repeated",
                                 k);
    }
    cudaStream_t user = (cudaStream_t)stream;
    Streams st;
    if (int rc_ = st.create(n_chains + 1, n_chains + 2)) return rc_;
    cudaStream_t os = st.s[n_chains];
    HOL_CUDA(cudaEventRecord(st.e[n_chains + 1], user));
    HOL_CUDA(cudaStreamWaitEvent(os, st.e[n_chains + 1], 0));
    for (int k = 0; k < n_chains; ++k)
        HOL_CUDA(cudaMemsetAsync(dcg_state(ctxs[k]).g, 0, DCG_COUNT * sizeof(int), os));
    Graph g;
    int rc;
    {
        std::vector<CaptureScope*> scopes;
        for (int k = 0; k < n_chains; ++k) scopes.push_back(new CaptureScope(ctxs[k]));
        rc = capture(os, g, [&]() {
            return fork_join(
                os, st, n_chains,
                [&](int k, cudaStream_t sk) {
                    return measure_run(ctxs[k], xi[k], n_rv, opts, Gxi[k], G2[k],
                                       four_point ? G4[k] : nullptr, four_point, nullptr, sk);
                },
                concurrency);
        });
        for (CaptureScope* p : scopes) delete p;
    }
    if (rc) return rc;
    HOL_CUDA(cudaGraphLaunch(g.e, os));
    std::vector<int> gs(DCG_COUNT * (size_t)n_chains);
    for (int k = 0; k < n_chains; ++k)
        HOL_CUDA(cudaMemcpyAsync(gs.data() + DCG_COUNT * k, dcg_state(ctxs[k]).g,
                                 DCG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, os));
    HOL_CUDA(cudaStreamSynchronize(os));
    HOL_CUDA(cudaEventRecord(st.e[0], os));
    HOL_CUDA(cudaStreamWaitEvent(user, st.e[0], 0));
    for (int k = 0; k < n_chains; ++k) {
        const int bad = gs[DCG_COUNT * k + DCG_STICKY];
        if (bad)
            return set_error(bad, "measure_batch_graph: a probe solve of chain %d %s", k,
                             bad == HOL_ENUMERIC ? "met a non-finite residual" : "did not converge");
    }
    return HOL_OK;
}
