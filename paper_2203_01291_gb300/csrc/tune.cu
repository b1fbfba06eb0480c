// Launch-shape autotuner for the CG iteration kernels.
//
// Candidates: K (tau slices streamed per lane group) among the divisors
// {1, 2, 4, 5, 8, 10} of Ltau, 1, 2 or 4 warps per block, for L = 32 the
// float4 layout with one slice per warp and K warps per block (7, K <= 8),
// the split float4 layout with 4 or 2 warps per slice (5, 4), and for L % 8 == 0
// the float4 layout with a cp.async ring of three slices (6), the streaming
// float4 kernel with a cp.async ring across units (3), the float4 layout
// with a two-slice cp.async ring (2), without (1), or the scalar register
// layout (0); for L % 8 == 4 (uneven row chunks, cb4.cuh) the two ring
// kernels (6, 2) or the scalar layout. The split and streaming kernels fix their own block shapes, so
// they are timed once per K. With the fused or merged CG on, that iteration
// kernel is timed instead, over K and warps (its layout is fixed). Each
// candidate is timed with CUDA events on the caller's stream (2 warm-up and
// 10 timed launches on the context's scratch vectors) and the fastest is
// kept in the context for every later call. Candidates whose per-unit
// partial sums would not fit the context's partial-sum bank are skipped. A
// context with the exact propagator has the scalar layout only.
#include <cuda_runtime.h>

#include "internal.cuh"

using namespace hol;

extern "C" int hol_tune(hol_ctx* c, int n_rhs, int* best_k, int* best_warps, int* best_vec,
                        double* best_ms, void* stream)
{
    HOL_TRACE("hol_tune");
    if (!c) return set_error(HOL_EINVAL, "hol_tune: null context");
    if (!c->field_set) return set_error(HOL_EINVAL, "hol_tune: hol_set_field not called");
    if (n_rhs < 1 || n_rhs > c->p.max_rhs)
        return set_error(HOL_EINVAL, "hol_tune: n_rhs=%d outside [1, %d]", n_rhs, c->p.max_rhs);
    cudaStream_t s = (cudaStream_t)stream;
    HOL_CUDA(cudaMemsetAsync(c->v32a, 0, (size_t)n_rhs * c->n * sizeof(float), s));
    cudaEvent_t e0, e1;
    HOL_CUDA(cudaEventCreate(&e0));
    HOL_CUDA(cudaEventCreate(&e1));
    const int ks[6] = {1, 2, 4, 5, 8, 10};
    const int ws[3] = {1, 2, 4};
    const int old_k = c->mv_k, old_w = c->mv_warps, old_v = c->mv_vec;
    int bk = old_k, bw = old_w, bv = old_v;
    double bms = 1e30;
    int rc = HOL_OK;
    // with the merged CG on, the merged iteration kernel is what the solver
    // launches: time it (its layout is fixed, so only K and warps vary)
    const bool fused = c->fused != 0;
    const bool merged = c->merged != 0 || fused;
    MergedScal sc;
    FusedPartials fp{c->part, c->part + c->part_len, c->part + 2 * c->part_len,
                     c->part + 3 * c->part_len, c->part + 4 * c->part_len,
                     c->part + 5 * c->part_len, c->part + 6 * c->part_len,
                     c->part + 7 * c->part_len};
    if (merged) {
        HOL_CUDA(cudaMemsetAsync(c->part, 0, kBanks * c->part_len * sizeof(double), s));
        HOL_CUDA(cudaMemsetAsync(c->cgs, 0, 8 * c->p.max_rhs * sizeof(double), s));
        sc.slot_in = c->cgs;
        sc.slot_out = c->cgs + 4 * c->p.max_rhs;
        sc.g_in = c->part;
        sc.d_in = c->part + c->part_len;
        sc.g_out = c->part + 2 * c->part_len;
        sc.d_out = c->part + 3 * c->part_len;
        sc.gr = c->part + 4 * c->part_len;
        sc.rho = c->part + 5 * c->part_len;
        sc.e_n = 1;
        sc.pi = c->part + 6 * c->part_len;
        sc.fold = 0;
    }
    auto launch = [&](int r) -> int {
        if (!merged)
            return launch_cg_mtm32(c, c->v32a, c->v32a, nullptr, c->v32b, n_rhs, nullptr, nullptr,
                                   nullptr, 0, 0, 1, nullptr, s);
        if (fused)
            return launch_cg_fused(c, c->v32a, c->v32b, c->v32c, c->v32e, c->v32f, c->v32g,
                                   c->v32h, n_rhs, nullptr, fp, s);
        sc.fold = (r & 1) ? 2 : 0;
        return launch_cg_merged(c, c->v32a, c->v32b, c->v32c, c->v32d, c->v32e, c->v32f, c->v32g,
                                c->v32h, c->v32i, n_rhs, nullptr, sc, s);
    };
    if (merged) {   // inputs of the merged kernel: zero vectors
        float* bufs[4] = {c->v32b, c->v32c, c->v32d, c->v32e};
        for (float* b : bufs)
            HOL_CUDA(cudaMemsetAsync(b, 0, (size_t)n_rhs * c->n * sizeof(float), s));
    }
    int vecs[8], nvec = 0;
    if (merged) {
        vecs[nvec++] = c->mv_vec;
    } else {
        if (c->L % 8 == 0 && !c->exact) {   // the exact propagator runs in layout 0 only
            vecs[nvec++] = 6;
            if (c->L == 32) {
                vecs[nvec++] = 7;
                vecs[nvec++] = 5;
                vecs[nvec++] = 4;
            }
            vecs[nvec++] = 3;
            vecs[nvec++] = 2;
            vecs[nvec++] = 1;
        } else if (c->L % 4 == 0 && c->L >= 8 && !c->exact) {   // L % 8 == 4: the ring kernels
            vecs[nvec++] = 6;
            vecs[nvec++] = 2;
        }
        vecs[nvec++] = 0;
    }
    for (int vi = 0; vi < nvec && !rc; ++vi) {
        const int vec = vecs[vi];
        for (int ki = 0; ki < 6 && !rc; ++ki) {
            const int k = ks[ki];
            if (c->T % k) continue;
            c->mv_k = k;
            if ((long)matvec_pstride(c) * c->p.max_rhs > c->part_len) continue;
            for (int wi = 0; wi < 3 && !rc; ++wi) {
                if (vec >= 3 && vec <= 5 && wi > 0 && !merged) break;   // fixed block shapes
                if (vec == 7 && (wi > 0 || k > 8)) break;   // K warps per block, K <= 8
                c->mv_warps = ws[wi];
                c->mv_vec = vec;
                for (int r = 0; r < 2 && !rc; ++r) rc = launch(r);
                if (rc) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < 10 && !rc; ++r) rc = launch(r);
                cudaEventRecord(e1, s);
                if (rc) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = set_error(HOL_ECUDA, "hol_tune: event synchronise failed");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / 10.0 < bms) {
                    bms = ms / 10.0;
                    bk = k;
                    bw = ws[wi];
                    bv = vec;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        c->mv_k = old_k;
        c->mv_warps = old_w;
        c->mv_vec = old_v;
        return rc;
    }
    c->mv_k = bk;
    c->mv_warps = bw;
    c->mv_vec = bv;
    if (best_k) *best_k = bk;
    if (best_warps) *best_warps = bw;
    if (best_vec) *best_vec = bv;
    if (best_ms) *best_ms = bms;
    return HOL_OK;
}
