/*
 * leastaction.h -- C ABI of the GB300 least-action propagator.
 *
 * The library propagates psi(x, t) under H = T + V0(x) + E(t) x_axis by the
 * least-action principle (Walters, "An efficient parallel method for relaxing to
 * the minimum action wavefunction", Sec. I): in each time step [t0, t0+dt]
 *     phi(x, t) = sum_{p,n} C_pn chi_p(x) P_n(tau),  tau = 2 (t - t0)/dt - 1,
 * with Legendre time functions P_0..P_K, the initial condition phi(t0) = psi(t0)
 * imposed exactly (C_p0 eliminated), and the remaining K coefficients per point
 * the solution of the stationarity condition (Eq. stationaryphase)
 *     M c = f.
 * M c = f is not solved directly: the coefficients are relaxed by minimising the
 * residual norm N = r^dagger W r of the action residual r = f - M c
 * (Eqs. actionresidual, residnorm) over small spacetime subvolumes of all K time
 * functions of a block of grid points, non-interacting subvolumes in parallel
 * (Sec. II), inside a multigrid V-cycle with Galerkin coarse operators
 * (Sec. III, Eqs. residual_rough and correction_fine).
 *
 * Spatial basis: uniform finite-difference grid, x_k = (k - (n-1)/2) h per axis,
 * Dirichlet walls one spacing beyond the outermost points, T = -1/2 Laplacian
 * (second-order 3/5/7-point stencil in 1/2/3 D), mass 1.
 *
 * Memory layout of every complex array: interleaved double2 (re, im).
 *   psi, V0:          point index p = (z*ny + y)*nx + x (x fastest).
 *   coefficients c:   index p*K + (n-1), n = 1..K (point-major, time function fastest).
 * A pointer argument may be host or device memory unless stated otherwise; the
 * library detects which (cudaPointerGetAttributes) and copies host data through
 * the context's stream.  Device pointers must stay valid until the call returns.
 *
 * Threading and streams: a context is used by one host thread at a time; all
 * work is ordered on the CUDA stream given to la_init (0 = legacy default
 * stream).  Calls that return numbers to the host synchronise that stream.
 *
 * Errors: every call returns la_status; no exception crosses the ABI; the text
 * of the last error of a context is available from la_last_error.  After
 * LA_ECUDA or LA_ETIMEOUT the context should be finalised.  Calls that run the
 * relaxation (la_step, la_step_batch, la_solve_step, la_relax_colour, la_backward)
 * return LA_ECUDA when a subvolume matrix was singular or not positive definite
 * and LA_ETIMEOUT when a staged copy did not arrive within its bounded wait.
 */
#ifndef LEASTACTION_H_
#define LEASTACTION_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LA_OK = 0,
  LA_EINVAL = 1,    /* invalid argument or configuration */
  LA_ENOMEM = 2,    /* device allocation failed */
  LA_ECUDA = 3,     /* CUDA runtime error */
  LA_ENOTCONV = 4,  /* max_cycles reached before rel <= tol (the state is still advanced) */
  LA_ESTATE = 5,    /* call out of order (e.g. la_step before la_set_hamiltonian) */
  LA_ETIMEOUT = 6   /* a kernel's bounded wait for a staged copy gave up (the kernel returned; the
                       device stays usable, the step's result is not valid) */
} la_status;

typedef struct la_ctx la_ctx;

/* Problem and relaxation configuration. */
typedef struct {
  int dim;              /* 1, 2 or 3 */
  int n[3];             /* grid points per axis (x, y, z); unused axes must be 1 */
  double h[3];          /* grid spacing per axis */
  int nt;               /* K: free Legendre time functions per point, 1..8 */
  double dt;            /* time step */
  int sub[3];           /* subvolume extent in points per axis (>= 2 on used axes); the last
                           subvolume on an axis may be shorter (ragged tail) */
  int levels;           /* multigrid levels, >= 1; every level but the coarsest must have an even
                           number of points per used axis */
  int nu1, nu2;         /* pre/post sweeps per level in a V(nu1, nu2) cycle; one level: nu1+nu2 sweeps */
  int coarse_sweeps;    /* sweeps on the coarsest level (levels > 1) */
  int max_cycles;       /* cycles per time step, >= 1 */
  double tol;           /* stop when N(c)/N(0) <= tol; tol <= 0 runs exactly max_cycles */
  int weight;           /* residual-norm weight W: 0 = (O x U)^{-1} (default), 1 = O x U, 2 = identity */
  int precision;        /* 0 = FP64 throughout; 1 = mixed: complex64 factors and V-cycle, FP64
                           residual, action and refinement update */
  int laser_axis;       /* axis of the dipole coupling E(t) x_axis */
  int ckpt_every;       /* > 0: la_step keeps psi every ckpt_every steps for la_backward; 0: no recording */
  int coarse_sub[3];    /* subvolume extent on the Galerkin levels (>= 2 on used axes); 0 = same as sub */
  int trial;            /* trial function of each la_step step, which the relaxation corrects (Sec. IV,
                           Eq. leastaction_correction): 0 = c = 0; 1..3 = extrapolation, polynomial of
                           degree trial-1 in the step index, of the last `trial` converged coefficient
                           vectors of the same propagation */
  int coarse_cycle;     /* 0: V(nu1, nu2) on every level but the coarsest; 1: V(coarse_nu1, coarse_nu2) on
                           the Galerkin levels above the coarsest (the finest keeps nu1, nu2) */
  int coarse_nu1, coarse_nu2;
  int cache_factors;    /* nonzero: la_backward keeps the subvolume factors of a recomputed segment
                           (ckpt_every steps x all levels) in device memory and reuses them for the
                           adjoint relaxation instead of factorising every step again; without the
                           memory for it the factors are recomputed as usual */
  int local_form;       /* local problem of a subvolume U (Sec. II): 0 = least squares, minimise N over
                           c_U (exact block Gauss-Seidel on M^dagger W M, 2^dim colours, never raises N;
                           default); 1 = the paper's square Dirichlet form M_UU delta_U = (f - M c)_U,
                           two-colour checkerboard, LU with partial pivoting; N may rise and the
                           iteration may diverge.  1 requires precision 0, levels 1, sub >= 1 and at
                           most 96 unknowns per subvolume; la_backward rejects it (LA_EINVAL) */
  int factor_group;     /* CTA packing of the shared-memory subvolume factorisations (up to 128 unknowns):
                           0 = several small matrices per CTA on levels of 512 or more subvolumes (8 up to
                           32 unknowns, 2 up to 64; complex64: 4 up to 32, 2 up to 48), chosen by size;
                           1 = one matrix per CTA on every level */
} la_config;

/* Laser field E(t) = sum_k amp[k] * env_k(t) * sin(omega[k] t), env_k = exp(-((t - t_center[k])/sigma[k])^2)
   for sigma[k] > 0, else 1.  Host arrays of length ncomp; ncomp = 0 means no field. */
typedef struct {
  int ncomp;
  const double* amp;
  const double* omega;
  const double* t_center;
  const double* sigma;
} la_pulse;

typedef struct {
  int cycles;           /* V-cycles run in the step */
  int fine_sweeps;      /* fine-level sweeps (every colour once) run in the step */
  double action;        /* N of the final iterate */
  double rel_action;    /* N / N(0) */
} la_step_stats;

/* Allocate a context for one grid and configuration; validates the configuration.
   cuda_stream: a cudaStream_t (0 = default stream).  Errors: LA_EINVAL, LA_ENOMEM, LA_ECUDA. */
la_status la_init(const la_config* cfg, void* cuda_stream, la_ctx** out);

/* Static potential V0 (real, one double per grid point, host or device) and the laser pulse
   (host struct and arrays, copied).  Builds the Galerkin coarse operators of every level
   (Sec. III, P A P^T) for the static part; the per-step time-matrix factors are combined later.
   Errors: LA_EINVAL (null V0, ncomp < 0), LA_ECUDA. */
la_status la_set_hamiltonian(la_ctx* ctx, const double* V0, const la_pulse* pulse);

/* Propagate psi (complex128[Np], host or device, in: psi(t0), out: psi(t0 + nsteps dt)) by nsteps
   least-action steps starting at time t0.  per_step (host, nullable) receives nsteps records.
   Each step: time matrices (Sec. IV Legendre overlaps, Gauss-Legendre quadrature of E(t)), subvolume
   factorisation on every level, V-cycles until N/N(0) <= tol, then psi(t0+dt) = phi(tau = 1).
   N(0) = f^dagger W f is the action of c = 0 in every case.  With cfg.trial > 0 the relaxation of a
   step starts from c extrapolated from the preceding steps' converged coefficients (1, 2 or 3 of
   them: constant, linear, quadratic in the step index) when that trial has a smaller action than
   c = 0, else from c = 0.  The history is kept across calls whose t0 continues the previous call,
   and cleared at every checkpoint (ckpt_every > 0), by la_set_hamiltonian and by la_backward, so
   the recomputation in la_backward repeats the forward iterates exactly.
   Returns LA_ENOTCONV if some step hit max_cycles or its action became non-finite (psi is still
   advanced). */
la_status la_step(la_ctx* ctx, void* psi, int nsteps, double t0, la_step_stats* per_step);

/* Many independent propagations stepped together (each context its own grid, potential, pulse and
   configuration).  psis[i] (complex128[Np_i], host or device) is advanced by nsteps steps from time
   t0s[i].  Every context works on its own internal stream for the whole call, and every step of every
   context is enqueued without waiting for the GPU: time matrices, factorisations, the starting iterate
   (the extrapolated trial when its action is below N(0), else c = 0, decided on the device), one launch
   of the context's relaxation graph -- a conditional loop that runs V-cycles until the action computed on
   the device meets the stopping rule (N/N(0) <= tol, max_cycles, or a non-finite action) -- and the step
   advance.  The contexts' streams run concurrently and the host synchronises once, after the last step.
   stats (host, nullable): nctx * nsteps records, context-major.  Returns LA_ENOTCONV if some step of
   some context hit max_cycles or its action became non-finite (whatever that context's tol).
   Errors: LA_EINVAL (null or repeated context), LA_ESTATE, LA_ENOMEM, LA_ECUDA (also a subvolume matrix
   that was not positive definite in any step, reported after the call's last step). */
la_status la_step_batch(la_ctx* const* ctxs, int nctx, void* const* psis, int nsteps, const double* t0s,
                        la_step_stats* stats);

/* N and N/N(0) (Eq. residnorm) of the final iterate of the last time step; synchronises. */
la_status la_action(la_ctx* ctx, double* action, double* rel_action);

/* Discrete adjoint of the last la_step call (which must have run with ckpt_every > 0).
   Input dJ_dpsiT (complex128[Np], host or device): the conjugate Wirtinger derivative dJ/dpsi_T^* of a
   real objective J of the final state.  Output grad_amp (host, ncomp doubles, nullable): dJ/da_j for
   the pulse amplitudes; dJ_dpsi0 (complex128[Np], host or device, nullable): dJ/dpsi_0^*.
   Per step, backwards (segments of ckpt_every steps are recomputed from their checkpoint):
   mu = M^{-dagger} B^T lambda is obtained by relaxing G z = B^T lambda with the step's factors
   (G = M^dagger W M is Hermitian, so the adjoint is a second relaxation; with cfg.trial > 0 it starts
   from the extrapolation of the preceding backward steps' z when that has the smaller residual), mu = W M z;
   dJ/da_j += 2 Re mu^dagger (dF/da_j psi_k - dM/da_j c_k); lambda += F_k^T mu (Sec. I, stationarity
   and the initial-condition multipliers define M and F).  Errors: LA_ESTATE, LA_EINVAL, LA_ECUDA. */
la_status la_backward(la_ctx* ctx, const void* dJ_dpsiT, double* grad_amp, void* dJ_dpsi0);

/* One step's coefficients without advancing: relax M c = f for initial state psi0 (complex128[Np])
   at time t0 and write c (complex128[Np*K]).  ncycles > 0 runs exactly that many cycles;
   ncycles == 0 runs until tol or max_cycles.  Used to compare iterates with a reference. */
la_status la_solve_step(la_ctx* ctx, const void* psi0, double t0, int ncycles, void* c_out,
                        la_step_stats* stats);

/* Action residual r = f - M c (Eq. actionresidual, complex128[Np*K]) of trial coefficients c for
   initial state psi0 at time t0, and its norm N = r^dagger W r.  r_out may be null. */
la_status la_residual(la_ctx* ctx, const void* psi0, double t0, const void* c, void* r_out,
                      double* action);

/* One relaxation pass of a single colour on the finest level (Sec. II): every subvolume of
   that colour is replaced by the minimiser of N over its coefficients, the others fixed
   (local_form 1: by the solution of its square Dirichlet problem).  c (complex128[Np*K]) is read
   and overwritten.  colour in [0, 2^dim) (local_form 1: the two checkerboard colours 0, 1). */
la_status la_relax_colour(la_ctx* ctx, const void* psi0, double t0, int colour, void* c);

/* Per-step time matrices at t0 (row-major K x K unless noted), for inspection:
   out[0..K*K)    U_b  = (dt/2) int b_m b_n            out[K*K..2K*K)  Q_b = int b_m b_n'
   out[2K*K..3K*K) E_b  = (dt/2) int b_m b_n E(t)      out[3K*K..3K*K+K) U_b0 = (dt/2) int b_m P_0
   out[3K*K+K..3K*K+2K) E_b0                              out[.. +K*K) W_t (time part of W)
   with b_n = P_n - (-1)^n P_0.  out is a host array of 4*K*K + 2*K doubles. */
la_status la_time_matrices(la_ctx* ctx, double t0, double* out);

/* Kernel timing for roofline reporting.  While enabled, the library records CUDA events on its
   stream around every finest-level factorisation launch, every finest-level sweep (the launches of
   all colours together), every finest-level action-residual stencil launch (S1: r = f - M c,
   inside the V-cycle and for the action norm) and every finest-level restriction and prolongation,
   and counts all of its kernel launches.  Algorithmic flops: factorisation
   (4/3) n^3 per subvolume (complex Cholesky of the n = |U| K unknowns); sweep 8 n^2 per subvolume
   (the two triangular solves; the residual stencil is not counted).  Where the finest-level factor
   has 16 x 16 blocks that vanish identically (subvolumes of more than 128 unknowns: G_UU couples only
   points at most two grid steps apart, and the factor keeps that envelope), both counts cover only the
   blocks of the band: the block-banded Cholesky and the solves over the band's blocks.  Algorithmic
   bytes of the residual stencil: c in, r out, f in where present (K complex each per point) and V0 in. */
typedef struct {
  long long launches;     /* kernels launched by the library since enabling */
  int n_factor;           /* finest-level factorisation launches */
  double ms_factor;       /* their summed device time */
  double flops_factor;    /* algorithmic flops per factorisation launch */
  int n_sweep;            /* finest-level sweeps (all colours) */
  double ms_sweep;
  double flops_sweep;     /* algorithmic flops of one full sweep (all colours) */
  int n_resid;            /* finest-level residual stencil launches in FP64 */
  double ms_resid;        /* their summed device time */
  double bytes_resid;     /* their summed algorithmic bytes */
  int n_resid32;          /* the same for the complex64 residual stencil (mixed-precision V-cycle) */
  double ms_resid32;
  double bytes_resid32;
  int n_restrict;         /* finest-level restriction launches (Sec. III, residual to level 1) */
  double ms_restrict;
  double bytes_restrict;  /* algorithmic bytes: the fine normal residual in, level 1's right-hand side out */
  int n_prolong;          /* level 1 -> finest prolongation-and-correction launches (Eq. correction_fine) */
  double ms_prolong;
  double bytes_prolong;   /* algorithmic bytes: level 1's correction in, the fine correction read and written */
} la_profile;
/* enable != 0 resets the counters and starts recording; 0 stops.  Errors: LA_EINVAL. */
la_status la_profile_enable(la_ctx* ctx, int enable);
/* Totals since enabling; synchronises the stream. */
la_status la_profile_read(la_ctx* ctx, la_profile* out);

/* Measured FMA throughput of the current device (no paper counterpart: the denominators of the FP64- and
   FP32-pipe rooflines that the benchmark reports).  Each thread of one full wave of resident CTAs (256
   threads each) on every SM runs 8 independent fused multiply-add chains, one launch per precision after a shorter warm-up launch, timed
   with CUDA events on cuda_stream (about 20 ms each); flops count 2 per FMA.  Outputs are host pointers:
   fp64_tflops, fp32_tflops (TFLOP/s) and sm_count (the device's multiprocessors).  Synchronises
   cuda_stream.  Errors: LA_EINVAL (null pointer), LA_ECUDA. */
la_status la_fma_peaks(double* fp64_tflops, double* fp32_tflops, int* sm_count, void* cuda_stream);

/* Residual norm without device allocation.  The paper has no counterpart to this entry point; it
   exists for callers that may not call cudaMalloc (code running inside a framework that owns all
   device memory through its own pool, or a process whose device memory budget is already spent).
   Computes N = r^dagger W r of trial coefficients c (complex128[Np*K]) for initial state psi0
   (complex128[Np]) at time t0, exactly as la_residual does, but with no context and no allocation:
   V0, psi0 and c must be device (or managed) pointers, else LA_EINVAL; *action is a host double.
   Scratch (per-step time matrices, per-block partial sums, the result) lives in one static device
   array of about 140 KB that every GPU loading the library keeps until exit; grids of more than
   LA_NOALLOC_MAX_POINTS points are rejected with LA_EINVAL.  All calls share that array and
   overwrite it completely, so calls that overlap on the GPU race and must be serialised by the
   caller.  The first call in a CUDA context (normally a device's primary context) looks up the
   array's address with that device current and keeps it for that context.  Under lazy module loading (the CUDA default) that first call may also load the
   library's module, which takes device memory for its code and the array: a process that must not
   allocate at all sets CUDA_MODULE_LOADING=EAGER or makes one call early.
   Synchronises cuda_stream.  Errors: LA_EINVAL (message in la_last_error(NULL)), LA_ECUDA. */
#define LA_NOALLOC_MAX_POINTS (1 << 22)
la_status la_action_noalloc(const la_config* cfg, const double* V0, const la_pulse* pulse, const void* psi0,
                            double t0, const void* c, double* action, void* cuda_stream);

/* Convergence maps of one relaxation step in the paper's Legendre-element basis (Secs. IV-V, the
   plane-wave experiment).  An element is the box y, tau in [-1, 1] with Legendre functions P_i(y),
   i < nx, and P_n(tau), n < nt, obeying the dimensionless least-action rows of
   Eq. leastaction_dimensionless with (kappa, nu).  The trial function exp(i (k x + w t)) on
   x, t in [-1, 1] is projected onto one element (method 0) or onto two elements [-1, 0], [0, 1]
   continuously at x = 0 (methods 1, 2), and relaxed once: method 0 relaxes the element, method 1
   both elements at once, method 2 corrects on the parent element through the Legendre transfers
   (Eqs. residual_rough, correction_fine) and then relaxes each element alone.  A relaxation solves
   the correction rows (Eq. leastaction_correction) with the correction held at zero at t0, at the
   ends of the relaxed volume and continuous inside it, the conditions entering through Lagrange
   multipliers. */
typedef struct {
  int method;           /* 0, 1 or 2 as above */
  int nx, nt;           /* Legendre functions per element in space and in time, 2..8 */
  double kappa, nu;     /* parameters of the dimensionless rows */
} la_lfa_case;

/* For every case c and grid point (w[a], k[b]):
     out[((c * 2 + 0) * nw + a) * nk + b] = log10(N_after / N_before),  N = r^H (O x U) r (Eq. residnorm)
     out[((c * 2 + 1) * nw + a) * nk + b] = log10(|S_after| / |S_before|),  S = the element action
   cases: host array of ncases; k, w: host arrays of nk wavenumbers and nw frequencies; out: device or
   host array of ncases * 2 * nw * nk doubles.  Per case the relaxation step, a linear map, is built on
   the host (dense algebra on at most 128 coefficients) and the maps are evaluated on the GPU on
   cuda_stream; synchronises before returning.  Errors: LA_EINVAL (bad case or grid, or a singular
   relaxation system; message in la_last_error(NULL)), LA_ENOMEM, LA_ECUDA. */
la_status la_lfa_maps(const la_lfa_case* cases, int ncases, const double* k, int nk, const double* w, int nw,
                      void* out, void* cuda_stream);

/* Self-test of the bounded waits (no context): one CTA waits on an mbarrier that nothing completes,
   polling at most `polls` times as the TMA-staged kernels do, and on giving up sets flag 4 (the value
   4) of a status word, which is written to *status_out (host).  The wait ends by itself; the device
   stays usable.
   Synchronises cuda_stream.  Errors: LA_EINVAL (polls < 1 or null status_out), LA_ENOMEM, LA_ECUDA. */
la_status la_wait_selftest(int polls, int* status_out, void* cuda_stream);

/* Waits for the context's stream, then releases everything the context owns (device workspace,
   factor store, checkpoints, captured graphs, events, pinned read-back buffer) and the context
   itself; ctx is invalid afterwards.  Caller-owned buffers are untouched.  Errors: LA_EINVAL (null). */
la_status la_finalize(la_ctx* ctx);
/* Message of the last error of ctx; with ctx = NULL, of the last call on this host thread that had no
   context (la_init, la_action_noalloc, la_lfa_maps).  The string stays valid until
   the next call that records an error on the same context or thread. */
const char* la_last_error(const la_ctx* ctx);
/* Library name, version and target architecture (static string). */
const char* la_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LEASTACTION_H_ */
