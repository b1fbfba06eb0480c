/*
 * holstein.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * hybrid Monte Carlo for the Holstein model (Cohen-Stead, Bradley, Miles,
 * Batrouni, Scalettar, Barros, "Fast and scalable quantum Monte Carlo
 * simulations of electron-phonon models").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Lattice: periodic L x L square lattice, N = L*L sites, site index
 *   i = ix + L*iy, nearest-neighbour hopping t (Sec. II B). L must be even,
 *   4 <= L <= 32. Imaginary time has T = Ltau slices (Sec. II C), T even.
 * - Space-time vectors are real arrays laid out [rhs][tau][i] (tau-slice
 *   contiguous), length n = N*T per right-hand side.
 * - All array arguments are DEVICE pointers unless the comment says "host".
 *   The caller allocates and owns them; the library never frees them.
 * - Device vector arguments are read and written with 8- and 16-byte vector
 *   accesses and must be 16-byte aligned (cudaMalloc and PyTorch allocations
 *   are, and so is a slice of one along the right-hand-side axis, since N is
 *   even); a misaligned one is refused with HOL_EINVAL before any launch.
 * - The context owns its scratch memory (allocated in hol_create, released in
 *   hol_destroy) and is bound to the CUDA device current at hol_create.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls enqueue work on that stream; calls that return host-side results
 *   (cg_solve statistics, dH) synchronise that stream before returning.
 * - Every call returns 0 (HOL_OK) or a negative HOL_E* code; no exception or
 *   abort crosses the ABI. hol_last_error() describes the last failure on the
 *   calling thread.
 * - Precision: HOL_F64 arrays are double; HOL_F32 arrays are float.
 */
#ifndef HOLSTEIN_H
#define HOLSTEIN_H

#ifdef __cplusplus
extern "C" {
#endif

#define HOL_OK        0
#define HOL_EINVAL   -1   /* bad argument (size, null pointer, unsupported shape) */
#define HOL_ENOTCONV -2   /* CG did not reach the tolerance within max_iter     */
#define HOL_ENUMERIC -3   /* NaN / Inf met in a reduction                        */
#define HOL_ETIMEOUT -4   /* reserved: a bounded device-side wait gave up (no
                             call of this version waits on the device)          */
#define HOL_ECUDA    -5   /* a CUDA runtime call failed                          */
#define HOL_ENOMEM   -6   /* device allocation failed                            */

/* operator selector for fermion_matvec */
#define HOL_OP_M   0      /* out = M v                                          */
#define HOL_OP_MT  1      /* out = M^T v                                        */
#define HOL_OP_MTM 2      /* out = M^T M v                                      */

/* precision selector */
#define HOL_F64 0
#define HOL_F32 1

/* preconditioner selector for precond_apply */
#define HOL_PINV        0   /* out = P^{-1} v                                  */
#define HOL_PINVT       1   /* out = P^{-T} v                                  */
#define HOL_PINV_PINVT  2   /* out = P^{-1} P^{-T} v (the PCG preconditioner)  */

/*
 * kinetic propagator C ~ exp(-dtau K) inside B_tau = exp(-dtau V_tau) C
 * (Sec. II D). CHECKERBOARD: the split product C4 C3 C2 C1 of two-site bond
 * factors (colours 1, 2: x-bonds from even / odd x; 3, 4: y-bonds from even /
 * odd y), the paper's discretisation. EXACT: exp(-dtau K) itself, applied as
 * E (x) E with E = exp(dtau t A_ring) the exact factor of one lattice
 * direction (a symmetric circulant whose taps are kept down to the rounding
 * of the arithmetic). An EXACT context runs its operators in the scalar
 * register layout only: hol_set_option refuses the other layouts and the
 * one-kernel CG variants for it, and fermion_matvec_static refuses EXACT.
 */
#define HOL_KINETIC_CHECKERBOARD 0
#define HOL_KINETIC_EXACT        1

/*
 * The taps of the exact one-direction factor E = exp(dtau t A_ring) on a ring
 * of L sites that HOL_KINETIC_EXACT applies (host code, no GPU needed):
 * e[d], d = 0 .. L/2, the entry of E for ring distance d (HOST array of 17
 * doubles; entries past L/2 are zero), summed over the periodic images from
 * the power series of the modified Bessel functions I_k(2 dtau t). d64 / d32
 * (host): the largest d kept by the FP64 / FP32 kernels (|e[d]| above 2^-60
 * / 2^-30 of e[0]). HOL_EINVAL for an unsupported L, dtau <= 0 or
 * |dtau t| > 4.
 */
int hol_exact_taps(int L, double dtau, double t, double* e, int* d64, int* d32);

typedef struct hol_params {
    int L;            /* linear lattice size (even, 4..32)                      */
    int Ltau;         /* number of imaginary-time slices T = beta / dtau (even) */
    double dtau;      /* imaginary-time step                                    */
    double t;         /* nearest-neighbour hopping                              */
    double mu;        /* chemical potential                                     */
    double alpha;     /* electron-phonon coupling                               */
    double omega0;    /* phonon frequency (phonon mass is 1)                    */
    int max_rhs;      /* largest n_rhs any later call will pass (>= 1)          */
    int kinetic;      /* HOL_KINETIC_CHECKERBOARD (0) or HOL_KINETIC_EXACT (1)  */
} hol_params;

typedef struct hol_ctx hol_ctx;

/* Create a context for one lattice shape and set of couplings. Allocates the
 * context's scratch on the current device. Returns HOL_EINVAL for an
 * unsupported shape, HOL_ENOMEM if the scratch does not fit. */
int hol_create(const hol_params* p, hol_ctx** out);

/* Release the context and its scratch (no counterpart in the paper). Waits
 * for the device to finish the context's work first. NULL is accepted. */
int hol_destroy(hol_ctx* ctx);

/* Message describing the last error on the calling thread (thread-local
 * static storage, valid until that thread's next failing call; no
 * counterpart in the paper). */
const char* hol_last_error(void);

/*
 * Set the phonon field x[tau][i] (FP64, device) the operators act on
 * (Sec. II C, Eqs. (B_def), (V_K_def)): computes
 *   expV[tau][i] = exp(-dtau (alpha x[tau][i] - mu))     (FP64 and FP32 copies)
 *   dbar[i]      = (1/T) sum_tau expV[tau][i]             (Eq. (expnVbar))
 *   the spectral bounds of Bbar = diag(dbar) exp(-dtau K) (App. C D; the
 *   deterministic norm bound min/max(dbar) * exp(-/+ 4 dtau |t|)),
 *   and the Chebyshev plan of the preconditioner (Eqs. (NP_heuristic),
 *   (Cheby-Gauss)). x is copied; the caller may reuse its buffer at once.
 */
int hol_set_field(hol_ctx* ctx, const double* x, void* stream);

/*
 * Apply the space-time fermion matrix of Eq. (M_def) to n_rhs vectors:
 *   (M v)_tau   = v_tau + s_tau B_tau v_{tau-1},  s_0 = +1, s_{tau>0} = -1,
 *   (M^T u)_tau = u_tau + s_{tau+1} B_{tau+1}^T u_{tau+1},
 * with B_tau = exp(-dtau V_tau) C (Eq. (B_def)) and C the checkerboard
 * product C4 C3 C2 C1 of Sec. II D (colours: x-bonds from even ix, x-bonds
 * from odd ix, y-bonds from even iy, y-bonds from odd iy; each bond the
 * two-site factor [[cosh, sinh], [sinh, cosh]](dtau t)); tau-1, tau+1 mod T.
 * op: HOL_OP_M, HOL_OP_MT or HOL_OP_MTM. prec: HOL_F64 (v, out double) or
 * HOL_F32 (float). v and out: [n_rhs][T][N], must not overlap.
 * Requires hol_set_field. 1 <= n_rhs <= max_rhs.
 */
int fermion_matvec(hol_ctx* ctx, int op, int prec, const void* v, void* out,
                   int n_rhs, void* stream);

typedef struct hol_cg_opts {
    double tol;          /* stop when |b - M^T M v| / |b| < tol (Sec. VI B)    */
    int max_iter;        /* iteration cap per right-hand side                  */
    int precond;         /* 0: plain CG; 1: adiabatic preconditioner (Sec. VI) */
    int prec;            /* HOL_F64: all FP64. HOL_F32: FP32 matvecs and
                            iterations, FP64 dot products, FP64 solution and
                            true-residual (reliable) updates                   */
    int reliable_every;  /* HOL_F32: iterations between FP64 residual updates  */
    int check_every;     /* iterations between host convergence polls          */
} hol_cg_opts;

/*
 * Solve (M^T M) v = b (Eq. (CG)) for n_rhs right-hand sides by conjugate
 * gradients from v = 0 (so v is a deterministic function of x and b), with
 * the preconditioner z = P^{-1} P^{-T} r when opts->precond (Eq. (CG_precon)).
 * b, v: FP64 [n_rhs][T][N] (device). Convergence of every right-hand side is
 * certified with an FP64 true residual |b - M^T M v| / |b| < tol. With
 * opts->prec HOL_F32 the iterations run in FP32 (FP64 dot products) and
 * every reliable_every iterations, and whenever the recursive residual
 * estimate falls below tol, the FP32 increment is folded into the FP64 v and
 * the residual is replaced by the FP64 true residual; the search direction
 * is then re-conjugated against it, beta = -(z, A p) / (p, A p). The
 * iteration kernels are chosen by the context's launch options (see
 * hol_set_option: two kernels per iteration by default, fused_cg /
 * merged_cg for one).
 * iters, resid: HOST arrays of n_rhs entries (nullable) receiving the
 * iterations and the final true relative residual of each right-hand side.
 * Returns HOL_ENOTCONV if some right-hand side did not converge (v then holds
 * the last iterate). Synchronises `stream`.
 */
int cg_solve(hol_ctx* ctx, const double* b, double* v, int n_rhs,
             const hol_cg_opts* opts, int* iters, double* resid, void* stream);

/*
 * Phonon force of Sec. III A: dS/dx[tau][i] (FP64, device, [T][N]) for the
 * action S = S_B + S_F with S_F = (1/2) sum_sigma Phi_sigma^T (A^T A)^{-1}
 * Phi_sigma, A = M Lambda (Eqs. (S_F), (dSF_dx)). Inputs are the solved
 * pairs (v_sigma, b_sigma), b = Lambda^{-T} Phi, v = (M^T M)^{-1} b, for
 * n_pf pseudofermions ([n_pf][T][N], FP64). With dA = dM Lambda + M dLambda
 * for the Holstein B_tau the fermion part is, per pseudofermion,
 *   dS_F/dx_{i,tau} = dtau alpha s_tau u_{i,tau} y_{i,tau}
 *                     - (dtau alpha / 2) b_{i,tau-1} v_{i,tau-1},
 *   u = M v, y_tau = exp(-dtau V_tau) C v_{tau-1}.
 * with_bosonic != 0 adds dS_B/dx of Eq. (dSB_dx) for the field of the last
 * hol_set_field. S_F (device, nullable, one double) receives
 * (1/2) sum_sigma b_sigma . v_sigma (Eq. (Sf_Psi)). dSdx is overwritten.
 * With dSdx null (and S_F not null) only the action S_F is computed: no
 * force, no B_tau sweep. HOL_EINVAL when both are null.
 */
int force(hol_ctx* ctx, const double* v, const double* b, int n_pf,
          double* dSdx, int with_bosonic, double* S_F, void* stream);

/*
 * Adiabatic preconditioner of Sec. VI A (Eq. (P_def)): P is M with every B_tau
 * replaced by Bbar = diag(dbar) C (Eqs. (Bbar), (expnVbar)). It is applied as
 * P^{-1} v = U^dag Ptilde^{-1} U v (Eq. (P_change_basis)), U the twisted DFT
 * along tau of Eq. (U_omega), each block (I - e^{-i phi_omega} Bbar)^{-1}
 * replaced by its Chebyshev series sum_{m<N_P} c_m T_m(A),
 * A = 2 (Bbar - bmin)/(bmax - bmin) - 1 (App. C, Eqs. (A_def), (Minv_KPM),
 * (alpha_recur)), N_P(omega) = max(1, floor((bmax-bmin)(a1/phi_omega + a2)))
 * (Eq. (NP_heuristic); a1 = a2 = 1 unless the launch options kpm_a1_percent /
 * kpm_a2_percent say otherwise), c_m by Chebyshev-Gauss quadrature
 * with 2 N_P points (Eq. (Cheby-Gauss)); bmin, bmax are the norm bounds set by
 * hol_set_field. HOL_PINVT applies the exact transpose of that approximation,
 * U^dag diag(sum conj(c_m) T_m(A^T)) U. which: HOL_PINV, HOL_PINVT or
 * HOL_PINV_PINVT. prec: HOL_F64 (double) or HOL_F32 (float) for v and out,
 * [n_rhs][T][N], real, must not overlap. Requires Ltau with prime factors in
 * {2, 3, 5, 7} and Ltau <= 400.
 */
int precond_apply(hol_ctx* ctx, int which, int prec, const void* v, void* out,
                  int n_rhs, void* stream);

/*
 * Pseudofermion draw (Sec. II D, Eq. (PhiSample-1)): Phi = A^T R with
 * A = M Lambda, for the field of the last hol_set_field. R, Phi: FP64
 * [n_pf][T][N] (device); R holds standard-normal draws supplied by the caller.
 * Uses context scratch; R and Phi must not overlap.
 */
int pseudofermion_phi(hol_ctx* ctx, const double* R, double* Phi, int n_pf, void* stream);

/*
 * CG right-hand side b = Lambda^{-T} Phi (Sec. II D, below Eq. (psi_def)),
 * Lambda of Eq. (Lambda_def) at the field of the last hol_set_field:
 *   b_{i,tau} = s'_{tau+1} exp(-dtau alpha x_{i,tau+1} / 2) Phi_{i,tau+1},
 *   s'_0 = +1, s'_{tau>0} = -1, tau+1 mod T.
 * Phi, b: FP64 [n_pf][T][N] (device), must not overlap.
 */
int phi_to_rhs(hol_ctx* ctx, const double* Phi, double* b, int n_pf, void* stream);

/*
 * Fourier-accelerated molecular dynamics (Sec. III B, Algorithm 1).
 * The dynamical mass is Mass = F^{-1} Mass~ F along tau (Eq. (dynamical_M_def))
 * with Mass~_omega = dtau (m_reg^2 + omega0^2 + (4/dtau^2) sin^2(pi omega/T))
 * / (m_reg^2 + omega0^2); m_reg = INFINITY gives the constant mass dtau.
 */
typedef struct hol_md_opts {
    double dt;               /* fermionic time step Delta t                          */
    int n_steps;             /* N_t fermionic steps per trajectory                   */
    int n_sub;               /* n_t bosonic sub-steps of Delta t / n_t per step      */
    double m_reg;            /* Fourier-acceleration regulator (>= 0 or INFINITY)   */
    hol_cg_opts cg_force;    /* solves for the forces inside the trajectory          */
    hol_cg_opts cg_action;   /* solve for S_F at the end of a trajectory             */
} hol_md_opts;

/*
 * out = Mass^{-1} p (which = 0), Mass^{1/2} p (1) or Mass p (2) for one
 * [T][N] FP64 field (device); p and out must not overlap. Each site's tau
 * line is transformed with a mixed-radix FFT (Ltau with prime factors in
 * {2, 3, 5, 7}).
 */
int mass_apply(hol_ctx* ctx, int which, double m_reg, const double* p, double* out,
               void* stream);

/*
 * Integrate n_steps steps of the split leapfrog of Algorithm 1 from (x, p)
 * in place (x, p: FP64 [T][N], device), at fixed pseudofermions Phi (FP64
 * [n_pf][T][N]). Each step: p -= dt/2 dS_F/dx; n_sub times { p -= dt'/2
 * dS_B/dx; x += dt' Mass^{-1} p; p -= dt'/2 dS_B/dx }; p -= dt/2 dS_F/dx,
 * dt' = dt/n_sub, dS_F/dx from cg_solve with opts->cg_force and the force of
 * `force`; the closing and opening half kicks of consecutive steps are one
 * force evaluation. Leaves the field of the last force set in the context.
 */
int md_integrate(hol_ctx* ctx, double* x, double* p, const double* Phi, int n_pf,
                 const hol_md_opts* opts, void* stream);

/*
 * One HMC update (Algorithm 1): Phi = A^T(x) R_pf (R_pf: [n_pf][T][N]
 * standard-normal draws), p = Mass^{1/2} R_p (R_p: [T][N] draws), H_i =
 * S_B + |R_pf|^2/2 + p.Mass^{-1}p/2, md_integrate, H_f = S_B + S_F + kinetic
 * energy with S_F from cg_solve(opts->cg_action), and the Metropolis test
 * u < exp(-(H_f - H_i)) with the caller's uniform draw u (Eq. (metropolis)).
 * x (device, in/out) holds the accepted field on return. accepted, dH (host,
 * nullable) receive the decision and H_f - H_i; terms (host, nullable, 6
 * doubles) receive S_B, S_F, kinetic energy at the start and at the end.
 * Synchronises `stream`.
 */
int fourier_accel_leapfrog(hol_ctx* ctx, double* x, const double* R_pf, const double* R_p,
                           int n_pf, const hol_md_opts* opts, double u, int* accepted,
                           double* dH, double* terms, void* stream);

/*
 * Observables of one measurement (Eq. (Scdw) and the pair susceptibility P_s
 * of Sec. II), contracted from the outputs of stochastic_measure run with
 * four_point = 7: G2 (device, [2T][L][L]) and G4 (device, [3][2T][L][L]).
 * Spins are independent and see the same field, so by Wick's theorem per
 * spin, with g0 = G2[0][0][0] the averaged G_aa:
 *   density <n> = 2 (1 - g0);
 *   C(r) = (1/(N T)) sum <n_{i+r} n_i> (equal time) = 4 (1 - 2 g0 + G4[1][0][r])
 *          + 2 (delta_{r,0} g0 - G4[2][0][r]), written to C (device, [L][L],
 *          indexed [dy][dx]);
 *   S_cdw = sum_r (-1)^(rx+ry) C(r);
 *   P_s = dtau sum_{l < T} sum_r G4[0][l][r] (the tau integral as a sum over
 *         slices of the averaged G^2).
 * out3 (host, 3 doubles): density, S_cdw, P_s. Synchronises `stream`.
 */
int measure_observables(hol_ctx* ctx, const double* G2, const double* G4, double* C,
                        double* out3, void* stream);

/*
 * Reflection and swap updates (Sec. IV): one Metropolis move of the phonon
 * field at fixed pseudofermion fields. kind HOL_REFLECT proposes
 * x_{i,tau} -> -x_{i,tau} at every tau of site i; HOL_SWAP exchanges the
 * lines of sites i and j (j != i; the paper uses neighbours, any pair is
 * accepted here). The action is S = S_B + (1/2) sum_sigma |A^{-T} Phi_sigma|^2
 * (Eq. (S_again)), evaluated with b = Lambda^{-T} Phi and one cg_solve(opts)
 * of the n_pf right-hand sides M^T M v = b (the paper uses a tight tolerance,
 * 1e-10, for such action differences, Sec. VI B). The move is accepted when
 * u < exp(-(S(x') - S(x))) (Eq. (metropolis)) with the caller's uniform draw u.
 * x (device, [T][N], in/out) holds the kept field on return, and the
 * context's field is set to it. Phi: device [n_pf][T][N], unchanged.
 * S_cur (host, nullable, in/out): the action at x; when null or not finite on
 * entry it is computed (one more solve); on return it holds the action of the
 * kept field, so a sequence of moves needs one solve each. accepted, dS (host,
 * nullable): the decision and S(x') - S(x). Uses the context scratch (the
 * leapfrog buffers); synchronises `stream`. Errors: HOL_EINVAL (bad kind,
 * sites or n_pf), HOL_ENOTCONV from the solve, HOL_ENUMERIC.
 */
#define HOL_REFLECT 0
#define HOL_SWAP    1
int global_update(hol_ctx* ctx, double* x, const double* Phi, int n_pf, int kind, int i, int j,
                  double u, const hol_cg_opts* opts, double* S_cur, int* accepted, double* dS,
                  void* stream);

/*
 * Stochastic Green's-function measurement with FFT averaging (Sec. V).
 * xi: n_rv probe vectors [n_rv][T][N] (FP64, device; e.g. Z2 draws, so that
 * <xi_i xi_j> = delta_ij, Eq. (Hutch_approx)). Gxi (device, caller-owned,
 * [n_rv][T][N]) receives G xi = M^{-1} xi, solved as M^T M v = M^T xi with
 * cg_solve(opts) in batches of max_rhs. G2 (device, [2T][L][L], indexed
 * [dl][dy][dx]) receives the space-time averaged Green function of
 * Eqs. (G_avg-1), (G_def-1), (cross_corr), averaged over the probes
 * (Eq. (G_approx_better)) and normalised as the mean over the original
 * N*T sites (circular sum over the doubled domain / (2 N T)); G2[dl+T] =
 * -G2[dl]. four_point (bit mask, 0 = none) selects the pair-averaged Wick
 * products of Sec. V C (Eq. (GG_approx_better)), written to G4 (device,
 * [3][2T][L][L], same normalisation, averaged over the n_rv (n_rv-1)/2 pairs
 * n < m): bit 0 (xi_n . xi_m) star (Gxi_n . Gxi_m), bit 1 (xi_n . Gxi_n) star
 * (xi_m . Gxi_m) (prefix sums, cost linear in n_rv), bit 2 (xi_n . Gxi_m) star
 * (xi_m . Gxi_n) (bits 0 and 2 cost one pair of transforms per pair); needs
 * n_rv >= 2 and max_rhs >= 2. iters (host, nullable, n_rv) receives CG
 * iterations. L and Ltau need prime factors in {2, 3, 5, 7}. Uses the context
 * scratch; synchronises `stream` (through cg_solve).
 */
int stochastic_measure(hol_ctx* ctx, const double* xi, int n_rv, const hol_cg_opts* opts,
                       double* Gxi, double* G2, double* G4, int four_point, int* iters,
                       void* stream);

/*
 * Independent chains of possibly different lattice sizes, each with its own
 * context (created by the caller), driven concurrently: a pool of n_threads
 * host threads, each with its own CUDA stream, takes the chains in order.
 * hmc_batch runs one fourier_accel_leapfrog (Algorithm 1) per chain with
 * x[k], R_pf[k] ([n_pf][T_k][N_k]), R_p[k], the uniform u[k] (host array);
 * accepted, dH (host arrays of n_chains, nullable) receive the results.
 * measure_batch runs stochastic_measure per chain (field already set) with
 * n_rv probes xi[k] into Gxi[k], G2[k] and, if G4 is not null, G4[k].
 * Chains never share device buffers; the result of each chain is the same as
 * a separate call. Returns the first failing chain's error. Synchronises all
 * the streams it used.
 */
int hmc_batch(hol_ctx* const* ctxs, int n_chains, double* const* x, const double* const* R_pf,
              const double* const* R_p, int n_pf, const hol_md_opts* opts, const double* u,
              int* accepted, double* dH, int n_threads);
int measure_batch(hol_ctx* const* ctxs, int n_chains, const double* const* xi, int n_rv,
                  const hol_cg_opts* opts, double* const* Gxi, double* const* G2,
                  double* const* G4, int four_point, int n_threads);

/*
 * Graph-launched solve and batched trajectories (no counterpart in the paper:
 * the paper's solver and HMC driver are host loops).
 *
 * cg_solve_graph: the solve of cg_solve -- the same kernels, the same
 * decisions, so bitwise the same v, iterations and residuals -- with every
 * decision of its loop taken on the device: the loop over chunks of
 * check_every iterations is a conditional WHILE node of a CUDA graph, the
 * reliable update (and the certification by the FP64 true residual) a
 * conditional IF node inside it; the host launches the graph once and waits
 * for it. Requires an even check_every and the two-kernel CG iteration
 * (options fused_cg, merged_cg and persistent_cg off), else HOL_EINVAL. The
 * loop runs whole chunks: with max_iter not a multiple of check_every it can
 * run up to check_every - 1 iterations past max_iter before HOL_ENOTCONV; the
 * number of chunks is bounded by max_iter / check_every + 2 in every case (no
 * device-side wait exists that could hang). Arguments and results as
 * cg_solve; uses the context's scratch and internal streams; synchronises
 * `stream`.
 *
 * hmc_batch_graph: one HMC trajectory (Algorithm 1, as fourier_accel_leapfrog)
 * for each of n_chains independent chains with their own contexts (any mix
 * of lattice sizes; no context repeated). The start of all chains, one
 * leapfrog step of all chains and the end of all chains are each captured
 * once into one CUDA graph (each chain on its own branch, its solves
 * graph-driven as in cg_solve_graph); the step graph is launched n_steps
 * times; the host reads the energies at the end and takes the Metropolis
 * decisions with u[k] (host array). x[k], R_pf[k] ([n_pf][T_k][N_k]), R_p[k]
 * as in fourier_accel_leapfrog; accepted, dH (host arrays of n_chains,
 * nullable). Each chain's result is bitwise the one fourier_accel_leapfrog
 * gives it. Both solver option sets need what cg_solve_graph needs. On a
 * failed solve (HOL_ENOTCONV or HOL_ENUMERIC, naming the chain) the fields of
 * all chains are left at the end of the trajectory. Synchronises `stream`.
 */
int cg_solve_graph(hol_ctx* ctx, const double* b, double* v, int n_rhs, const hol_cg_opts* opts,
                   int* iters, double* resid, void* stream);
/*
 * measure_batch_graph: stochastic_measure (Sec. V) for each of n_chains
 * independent chains (own contexts, fields already set, no context
 * repeated), all captured into one CUDA graph (each chain a branch, its probe
 * solves graph-driven as in cg_solve_graph) and launched once. Arguments per
 * chain as stochastic_measure (xi[k], Gxi[k]: [n_rv][T_k][N_k]; G2[k]; G4[k]
 * when four_point != 0); no iteration counts. opts needs what cg_solve_graph
 * needs. concurrency: at most this many chains in flight (chain k follows
 * chain k - concurrency; 0 = all chains at once). Each chain's G2 / G4 / Gxi
 * are bitwise those of stochastic_measure, whatever the concurrency.
 * HOL_ENOTCONV or HOL_ENUMERIC names the first failing chain; concurrency
 * < 0 is HOL_EINVAL. Synchronises `stream`.
 */
int measure_batch_graph(hol_ctx* const* ctxs, int n_chains, const double* const* xi, int n_rv,
                        const hol_cg_opts* opts, double* const* Gxi, double* const* G2,
                        double* const* G4, int four_point, int concurrency, void* stream);
int hmc_batch_graph(hol_ctx* const* ctxs, int n_chains, double* const* x,
                    const double* const* R_pf, const double* const* R_p, int n_pf,
                    const hol_md_opts* opts, const double* u, int* accepted, double* dH,
                    void* stream);

/*
 * Allocation-free FP64 fermion operator (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc: code whose device memory is owned
 * entirely by another allocator (a framework's caching allocator, or a budget
 * fixed at start-up), and code that must not trigger the device-wide
 * synchronisation that cudaMalloc / cudaFree can imply. It needs no context:
 * out = M v, M^T v or M^T M v (op = HOL_OP_M, HOL_OP_MT, HOL_OP_MTM; the
 * operator and kernels of fermion_matvec with HOL_F64 in a checkerboard
 * context) for the field x and the couplings in p (p->max_rhs and p->omega0
 * are ignored). Only the checkerboard propagator is supported: p->kinetic must
 * be HOL_KINETIC_CHECKERBOARD, else HOL_EINVAL. The couplings are checked as
 * hol_create checks them (dtau > 0; t, mu and alpha finite). x: FP64 [T][N];
 * v, out: FP64 [n_rhs][T][N], device; their address ranges must not overlap.
 *
 * Scratch: one file-scope device array of 2^20 doubles (8 MiB) that every GPU
 * loading this library holds until the process exits. A call needs N*T
 * doubles of it (the exp(-dtau V) table) plus n_rhs*N*T more for HOL_OP_MTM
 * (the intermediate M v); larger requests return HOL_EINVAL. Nothing in it
 * has to start at zero: every call writes what it reads. The first call on a
 * device (with that device current) looks up the array's device address and
 * caches it; make that first call before any stream capture. Every call
 * shares the one array, so calls whose work overlaps on the GPU (different
 * streams, or different host threads on one device) race: serialise them.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).
 */
int fermion_matvec_static(const hol_params* p, const double* x, int op, const double* v,
                          double* out, int n_rhs, void* stream);

/*
 * Arnoldi estimate of the spectral bounds of Bbar = exp(-dtau Vbar) C (App. C
 * D): m steps (1 <= m <= 32, m <= N) of the Arnoldi process (modified
 * Gram-Schmidt applied twice per step, FP64) for the field of the last
 * hol_set_field, from the start vector v0 (device, N doubles, any nonzero
 * vector; the paper starts from a random one), on Bbar and on
 * Bbar^{-1} = C^{-1} exp(dtau Vbar); Ritz values are the eigenvalues of the
 * Hessenberg matrices (shifted QR on the host). bmax = (1 + margin) times the
 * largest Ritz modulus of Bbar, bmin = 1 / ((1 + margin) times the largest
 * Ritz modulus of Bbar^{-1}) (host outputs, nullable; the paper uses about
 * twenty steps and a 5 % margin; margin in [0, 1)). steps (host, nullable)
 * receives the fewer of the two runs' steps (fewer than m when an invariant
 * subspace is found).
 * install != 0 replaces the context's bounds (the deterministic norm bounds
 * hol_set_field computes) by these and recomputes the Chebyshev orders N_P
 * and coefficients, for every later precond_apply and preconditioned
 * cg_solve until the next hol_set_field. Returns HOL_ENUMERIC if the QR
 * iteration fails. Synchronises `stream`.
 */
int hol_arnoldi_bounds(hol_ctx* ctx, const double* v0, int m, double margin, int install,
                       double* bmin, double* bmax, int* steps, void* stream);

/* Eigenvalues of an n x n real upper Hessenberg matrix H (HOST, row-major;
 * entries below the first subdiagonal must be zero) by the shifted QR
 * iteration hol_arnoldi_bounds uses for its Ritz values (host code, no GPU
 * needed). re, im: HOST arrays of n, in no particular order. HOL_EINVAL for a
 * bad argument or a matrix that is not Hessenberg, HOL_ENUMERIC if the
 * iteration does not converge. */
int hol_hessenberg_eigenvalues(int n, const double* H, double* re, double* im);

/* The spectral bounds of Bbar (App. C D) the preconditioner currently uses
 * (host outputs): the deterministic norm bounds of hol_set_field, or those
 * installed by hol_arnoldi_bounds. HOL_EINVAL before hol_set_field or for a
 * null argument. Synchronises `stream`. */
int hol_get_bounds(hol_ctx* ctx, double* bmin, double* bmax, void* stream);

/*
 * Launch-shape autotuner (no counterpart in the paper). Times the fused FP32
 * M^T M kernel of the CG iteration for n_rhs right-hand sides over its launch
 * candidates (tau slices per lane group, warps per block, vector or scalar
 * register layout) with CUDA events on `stream`, and keeps the fastest in the
 * context for all later calls (results are unchanged up to rounding; every
 * candidate computes the same operator). Host outputs (nullable): the chosen
 * slices per group, warps per block, layout (the "layout"
 * values of hol_set_option), and its time in ms. A context with the exact
 * propagator (HOL_KINETIC_EXACT) tunes the scalar layout 0 only.
 * Requires hol_set_field; overwrites context scratch; synchronises `stream`.
 */
int hol_tune(hol_ctx* ctx, int n_rhs, int* best_k, int* best_warps, int* best_vec,
             double* best_ms, void* stream);

/*
 * Runtime launch options of a context (no counterpart in the paper; results
 * are the same up to rounding whichever is chosen):
 *   "slices_per_group"  tau slices streamed per lane group (divides Ltau)
 *   "warps_per_block"   1, 2 or 4 for the operator kernels
 *   "layout"            0 scalar, 1 float4, 2 float4 with a two-slice cp.async
 *                       ring, 6 the same with a three-slice ring (2 and 6
 *                       need L % 4 == 0, L >= 8; for L % 8 == 4 the row
 *                       chunks of a lane alternate L/4 + 1 and L/4 - 1
 *                       rows), 3 streaming float4 with a cp.async ring
 *                       across units (1 and 3 need L % 8 == 0), 4 / 5 split
 *                       float4 with each slice
 *                       spread over 2 / 4 warps (L == 32), 7 float4 with one
 *                       slice per warp and slices_per_group (<= 8) warps per
 *                       block exchanging the tau neighbours in shared memory
 *                       (L == 32)
 *   "kpm_registers"     FP32 KPM with the slice in registers: 0 off
 *                       (shared-memory kernel), 1 four columns per lane
 *                       (L = 16 or 32), 2 two columns per lane (L = 16 or
 *                       32: twice the warps per problem, half the work per
 *                       lane on the chain of Bbar applies), 3 the lane
 *                       layout (any L: one lane per column, the rows in
 *                       registers, the real and imaginary parts in two lane
 *                       groups). 1 and 2 fall back to the shared-memory
 *                       kernel for other L. Default 2 at L = 32, 3
 *                       otherwise. The FP64 KPM uses the banded lane layout
 *                       (rows in bands over several warps) where it is
 *                       built (L = 4-18 even, 24, 28, 32) unless this is 0,
 *                       else the shared-memory kernel
 *   "persistent_cg"     plain mixed CG chunks in one cooperative launch (0/1)
 *   "pdl"               programmatic dependent launch of the CG iteration
 *                       kernels: each may be scheduled while its predecessor
 *                       finishes and waits on the device for its results
 *                       (0/1, default 1)
 *   "fused_cg"          plain mixed CG (cg_solve with prec HOL_F32 and no
 *                       preconditioner) with one kernel per iteration: the
 *                       vector update of an iteration is done inside the next
 *                       operator pass and beta comes from the exact expansion
 *                       |r - alpha q|^2 = r.r - 2 alpha r.q + alpha^2 q.q
 *                       (the CG of Eq. (CG), rearranged). Needs L % 8 == 0;
 *                       allocates three more FP32 vector sets of max_rhs
 *                       N Ltau on first use. Default 0: the two-kernel
 *                       iteration (operator, then update), measured as fast
 *                       at the benchmark size (0/1)
 *   "scalar_handoff"    mixed CG (two-kernel iteration): bit 0 set, alpha is
 *                       formed once per right-hand side by the last warp of
 *                       the operator kernel to finish (layouts 0, 1, 2, 6) and
 *                       read by the update kernel; bit 1 set (plain CG), beta
 *                       is formed by the last block of the update kernel and
 *                       read by the operator. Default 0: every block and warp
 *                       forms them from the partial sums (measured faster:
 *                       the last-block step lengthens the producer's tail).
 *                       The values are the same either way (0..3)
 *   "kpm_a1_percent",   100 a1 and 100 a2 of the Chebyshev order N_P(omega) =
 *   "kpm_a2_percent"    max(1, floor((bmax - bmin)(a1 / phi_omega + a2)))
 *                       (Eq. (NP_heuristic)); the paper's a1 = a2 = 1 (100) by
 *                       default; smaller values shorten the series (a cheaper,
 *                       less exact P^{-1}). 1..400; takes effect at the next
 *                       hol_set_field or installed Arnoldi bounds
 *   "fused_pc_update"   preconditioned CG (both precisions): the vector update
 *                       of each iteration (r -= alpha q, the deferred x
 *                       update, the r.r partials) runs inside the forward
 *                       tau transform of the preconditioner applied to the
 *                       new r, one kernel and one pass over r fewer per
 *                       iteration (0/1, default 1). The iteration is the
 *                       same up to the grouping of the r.r partials
 *   "kpm_queue"         FP32 register KPM (kpm_registers 1 or 2): 0 one block
 *                       per (omega, rhs) problem; k in 1..8 a persistent grid
 *                       of k blocks per multiprocessor taking the problems
 *                       from a queue, longest Chebyshev series first (used
 *                       when there are more problems than blocks)
 *   "merged_cg"         with fused_cg 0: plain mixed CG as one kernel per
 *                       iteration with single-reduction Chronopoulos-Gear
 *                       recurrences (L % 8 == 0; allocates the same three
 *                       vector sets on first use) (0/1)
 * Every solver variant certifies convergence by the FP64 true residual;
 * iteration counts may differ by a few percent between them.
 * A context with the exact propagator (HOL_KINETIC_EXACT) keeps layout 0 and
 * refuses any other layout and kpm_registers, persistent_cg, fused_cg and
 * merged_cg set to 1 (those kernels are checkerboard only).
 * Returns HOL_EINVAL for an unknown name or a value out of range (HOL_ECUDA
 * when an allocation fails).
 */
int hol_set_option(hol_ctx* ctx, const char* name, int value);

/* Current value of a launch option of hol_set_option into *value (written on
 * success only; no counterpart in the paper). Returns HOL_EINVAL for a null
 * argument or an unknown name. */
int hol_get_option(const hol_ctx* ctx, const char* name, int* value);

/*
 * Instrumentation (no counterpart in the paper; used by the benchmark).
 * hol_launch_count: number of kernels this library has launched in the
 * process so far. hol_timer_enable(ctx, k) with k >= 1 starts recording CUDA
 * events around one in every k kernel regions of each class below, on the
 * stream each call is given (it resets the counts; 0 stops recording). hol_timer_read returns, for one
 * class, how many regions were recorded and their summed device time in ms
 * (it waits for the recorded events) and (nullable) the summed work units of
 * those regions (for the CG classes: right-hand sides still iterating).
 * Classes: 0 CG operator (fused M^T M),
 * 1 CG vector update, 2 force, 3 preconditioner, 4 other.
 */
unsigned long long hol_launch_count(void);
/* Measured FMA throughput of the current GPU in GFLOP/s (prec HOL_F64 or
 * HOL_F32; 2 flops per FMA): the ALU roofline of the FP64 path (no
 * counterpart in the paper). gflops: host output. Synchronises `stream`. */
int hol_fma_peak(int prec, double* gflops, void* stream);
int hol_timer_enable(hol_ctx* ctx, int on);
int hol_timer_read(hol_ctx* ctx, int klass, int* count, double* total_ms, double* units);

#ifdef __cplusplus
}
#endif
#endif /* HOLSTEIN_H */
