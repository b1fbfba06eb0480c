/*
 * Matrix-free FP64 oracle for the Holstein HMC hot path -- TEST
 * INFRASTRUCTURE ONLY (parity checks at sizes the dense oracle cannot hold,
 * and the timed CPU baseline). Plain C99 + OpenMP, no vector intrinsics.
 *
 * Written from the paper's definitions, independently of the CUDA library:
 *   M (Eq. (M_def)): (M v)_tau = v_tau + s_tau B_tau v_{tau-1}, s_0 = +1,
 *                    s_tau = -1 for tau >= 1, tau-1 taken mod Ltau;
 *   B_tau = exp(-dtau V_tau) exp(-dtau K) (Eq. (B_def)), exp(-dtau K) the
 *   checkerboard product C4 C3 C2 C1 of two-site bond factors
 *   [[cosh, sinh], [sinh, cosh]](dtau t) over four bond colours (x-even,
 *   x-odd, y-even, y-odd), or (kinetic = 1) exp(-dtau K) itself;
 *   M^T is the transpose of that matrix, (M^T u)_tau = u_tau +
 *   s_{tau+1} C^T D_{tau+1} u_{tau+1}, C^T = C1 C2 C3 C4;
 *   CG on M^T M v = b (Eq. (CG)), stopped on |b - M^T M v| / |b| (Sec. VI B);
 *   the fermion force (Eq. (dSF_dx)) with dA = dM Lambda + M dLambda written
 *   out for the Holstein B_tau: dS_F/dx_{i,tau} = dtau alpha s_tau u_{i,tau}
 *   y_{i,tau} - (dtau alpha / 2) b_{i,tau-1} v_{i,tau-1}, u = M v,
 *   y_tau = D_tau C v_{tau-1}; this equals the dense definition in
 *   oracle/dense.py (checked by the tests);
 *   the bosonic force (Eq. (dSB_dx)).
 *
 * Layout: v[tau][i], i = ix + L*iy.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int L, T;
    double dtau, t, mu, alpha, omega0;
    int kinetic;   /* 0: checkerboard C4 C3 C2 C1; 1: exact exp(-dtau K) */
} orc_model;

static int idx(int ix, int iy, int L) { return ((ix + L) % L) + L * ((iy + L) % L); }

/* one bond colour (0: x-even, 1: x-odd, 2: y-even, 3: y-odd) applied in place */
static void bond_colour(const orc_model* m, int colour, double* v)
{
    const int L = m->L;
    const double ch = cosh(m->dtau * m->t), sh = sinh(m->dtau * m->t);
    for (int iy = 0; iy < L; ++iy)
        for (int ix = 0; ix < L; ++ix) {
            int i, j;
            if (colour < 2) {
                if ((ix & 1) != colour) continue;
                i = idx(ix, iy, L); j = idx(ix + 1, iy, L);
            } else {
                if ((iy & 1) != colour - 2) continue;
                i = idx(ix, iy, L); j = idx(ix, iy + 1, L);
            }
            double a = v[i], b = v[j];
            v[i] = ch * a + sh * b;
            v[j] = sh * a + ch * b;
        }
}

/* v <- exp(-dtau K) v exactly. K = -t (nearest-neighbour hopping) on the
 * periodic lattice is the sum of commuting x and y parts, so exp(-dtau K) is
 * E (x) E with E = exp(dtau t A) for the adjacency A of a ring of L sites;
 * E[i][j] = e[(i - j) mod L] with e[d] = (1/L) sum_k exp(2 dtau t
 * cos(2 pi k / L)) cos(2 pi k d / L), from the ring's Fourier modes. */
static void exact_kinetic(const orc_model* m, double* v)
{
    const int L = m->L, N = L * L;
    const double pi = acos(-1.0);
    double* e = (double*)malloc(sizeof(double) * L);
    double* tmp = (double*)malloc(sizeof(double) * N);
    for (int d = 0; d < L; ++d) {
        double s = 0.0;
        for (int k = 0; k < L; ++k)
            s += exp(2.0 * m->dtau * m->t * cos(2.0 * pi * k / L)) * cos(2.0 * pi * k * d / L);
        e[d] = s / L;
    }
    for (int iy = 0; iy < L; ++iy)          /* x direction */
        for (int ix = 0; ix < L; ++ix) {
            double s = 0.0;
            for (int jx = 0; jx < L; ++jx) s += e[(ix - jx + L) % L] * v[jx + L * iy];
            tmp[ix + L * iy] = s;
        }
    for (int iy = 0; iy < L; ++iy)          /* y direction */
        for (int ix = 0; ix < L; ++ix) {
            double s = 0.0;
            for (int jy = 0; jy < L; ++jy) s += e[(iy - jy + L) % L] * tmp[ix + L * jy];
            v[ix + L * iy] = s;
        }
    free(tmp);
    free(e);
}

/* v <- C v (C = C4 C3 C2 C1, so C1 acts first) or v <- C^T v; with the exact
 * propagator (symmetric) both are exp(-dtau K) v */
void orc_kinetic(const orc_model* m, double* v, int transpose)
{
    if (m->kinetic == 1) {
        exact_kinetic(m, v);
        return;
    }
    if (!transpose)
        for (int c = 0; c < 4; ++c) bond_colour(m, c, v);
    else
        for (int c = 3; c >= 0; --c) bond_colour(m, c, v);
}

void orc_expV(const orc_model* m, const double* x, double* d)
{
    const long n = (long)m->T * m->L * m->L;
    for (long k = 0; k < n; ++k) d[k] = exp(-m->dtau * (m->alpha * x[k] - m->mu));
}

void orc_M(const orc_model* m, const double* d, const double* v, double* out)
{
    const int N = m->L * m->L, T = m->T;
#pragma omp parallel
    {
        double* w = (double*)malloc(sizeof(double) * N);
#pragma omp for schedule(static)
        for (int tau = 0; tau < T; ++tau) {
            int tm = (tau + T - 1) % T;
            double s = (tau == 0) ? 1.0 : -1.0;
            memcpy(w, v + (long)tm * N, sizeof(double) * N);
            orc_kinetic(m, w, 0);
            for (int i = 0; i < N; ++i)
                out[(long)tau * N + i] = v[(long)tau * N + i] + s * d[(long)tau * N + i] * w[i];
        }
        free(w);
    }
}

void orc_MT(const orc_model* m, const double* d, const double* u, double* out)
{
    const int N = m->L * m->L, T = m->T;
#pragma omp parallel
    {
        double* w = (double*)malloc(sizeof(double) * N);
#pragma omp for schedule(static)
        for (int tau = 0; tau < T; ++tau) {
            int tp = (tau + 1) % T;
            double s = (tp == 0) ? 1.0 : -1.0;
            for (int i = 0; i < N; ++i) w[i] = d[(long)tp * N + i] * u[(long)tp * N + i];
            orc_kinetic(m, w, 1);
            for (int i = 0; i < N; ++i)
                out[(long)tau * N + i] = u[(long)tau * N + i] + s * w[i];
        }
        free(w);
    }
}

static double dot(const double* a, const double* b, long n)
{
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* out = M^T M v, tmp: n doubles */
void orc_MTM(const orc_model* m, const double* d, const double* v, double* out, double* tmp)
{
    orc_M(m, d, v, tmp);
    orc_MT(m, d, tmp, out);
}

/* Textbook CG on M^T M v = b from v = 0. Stops when the TRUE relative residual
 * |b - M^T M v| / |b| < tol (checked each iteration, as Sec. VI B defines it).
 * Returns iterations, or -1 if max_iter was reached. */
int orc_cg(const orc_model* m, const double* x, const double* b, double* v,
           double tol, int max_iter, double* resid_out)
{
    const long n = (long)m->T * m->L * m->L;
    double* d = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    double* tmp = (double*)malloc(sizeof(double) * n);
    orc_expV(m, x, d);
    for (long k = 0; k < n; ++k) { v[k] = 0.0; r[k] = b[k]; p[k] = b[k]; }
    double rr = dot(r, r, n), nb = sqrt(dot(b, b, n));
    int it, done = -1;
    double res = 1.0;
    for (it = 1; it <= max_iter; ++it) {
        orc_MTM(m, d, p, q, tmp);
        double a = rr / dot(p, q, n);
        for (long k = 0; k < n; ++k) { v[k] += a * p[k]; r[k] -= a * q[k]; }
        double rr_new = dot(r, r, n);
        if (sqrt(rr_new) / nb < tol) {
            /* confirm with the true residual */
            orc_MTM(m, d, v, q, tmp);
            for (long k = 0; k < n; ++k) tmp[k] = b[k] - q[k];
            res = sqrt(dot(tmp, tmp, n)) / nb;
            if (res < tol) { done = it; break; }
        }
        double beta = rr_new / rr;
        rr = rr_new;
        for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
    }
    if (done < 0) {
        orc_MTM(m, d, v, q, tmp);
        for (long k = 0; k < n; ++k) tmp[k] = b[k] - q[k];
        res = sqrt(dot(tmp, tmp, n)) / nb;
    }
    if (resid_out) *resid_out = res;
    free(d); free(r); free(p); free(q); free(tmp);
    return done;
}

/* F[tau][i] += dS_F/dx_{i,tau} for one pseudofermion, given v = (M^T M)^{-1} b. */
void orc_force_fermion(const orc_model* m, const double* x, const double* v,
                       const double* b, double* F)
{
    const int N = m->L * m->L, T = m->T;
    const long n = (long)T * N;
    const double da = m->dtau * m->alpha;
    double* d = (double*)malloc(sizeof(double) * n);
    orc_expV(m, x, d);
#pragma omp parallel
    {
        double* w = (double*)malloc(sizeof(double) * N);
#pragma omp for schedule(static)
        for (int tau = 0; tau < T; ++tau) {
            int tm = (tau + T - 1) % T;
            double s = (tau == 0) ? 1.0 : -1.0;
            memcpy(w, v + (long)tm * N, sizeof(double) * N);
            orc_kinetic(m, w, 0);
            for (int i = 0; i < N; ++i) {
                double y = d[(long)tau * N + i] * w[i];
                double u = v[(long)tau * N + i] + s * y;
                F[(long)tau * N + i] += da * s * u * y
                                        - 0.5 * da * b[(long)tm * N + i] * v[(long)tm * N + i];
            }
        }
        free(w);
    }
    free(d);
}

/* F[tau][i] += dS_B/dx_{i,tau} (Eq. (dSB_dx)) */
void orc_force_boson(const orc_model* m, const double* x, double* F)
{
    const int N = m->L * m->L, T = m->T;
    for (int tau = 0; tau < T; ++tau) {
        int tp = (tau + 1) % T, tm = (tau + T - 1) % T;
        for (int i = 0; i < N; ++i) {
            double xc = x[(long)tau * N + i];
            double lap = x[(long)tp * N + i] - 2.0 * xc + x[(long)tm * N + i];
            F[(long)tau * N + i] += m->dtau * (m->omega0 * m->omega0 * xc - lap / (m->dtau * m->dtau));
        }
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
