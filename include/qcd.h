/*
 * qcd.h -- C ABI of libqcd: the even-odd preconditioned clover-Wilson Dirac
 * operator, its CG solve and the fermion force, on one NVIDIA GB300 (sm_103a).
 *
 * Source of the method.  Shi, Kindratenko and Gottlieb, "Cell processor
 * implementation of a MILC lattice QCD application", Sec. 1: the application is
 * MILC 7.4's clover_dynamical -- dynamical clover-improved Wilson fermions in
 * the hybrid-molecular-dynamics R algorithm (su3_rmd).  Its compute loops
 * iterate over the 4-D lattice reading data at a site and at its neighbours
 * (Sec. 3); the paper prints no formula, so the operator is the standard one:
 *
 *   (M psi)(x) = A(x) psi(x) - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
 *                                           + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *   A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),  sigma = (i/2)[g_mu, g_nu]
 *   F_{mu nu} = traceless part of (Q_{mu nu} - Q_{mu nu}^dag) / (8i), Q = sum of 4 leaves
 *   Mhat = A_ee - kappa^2 D_eo A_oo^-1 D_oe   (even sites),  Mhat^dag = g5 Mhat g5
 *
 * DeGrand-Rossi gamma basis (g5 = diag(1,1,-1,-1)); directions mu = 0..3 are
 * x, y, z, t; periodic in x, y, z; the time boundary factor t_bc multiplies
 * U_t on the last time slice in the hopping term only.
 *
 * Canonical layouts (all complex numbers are interleaved (re, im) doubles):
 *   gauge  U[t][z][y][x][mu][3][3]           complex128, V*4*9 complex
 *   spinor on even sites [nrhs][V/2][spin 4][colour 3], complex128
 *          (even sites = (x+y+z+t) even, in increasing lexicographic index
 *          x + X (y + Y (z + Z t)); odd-site fields likewise)
 *   force  F[t][z][y][x][mu][3][3]           complex128
 *
 * Ownership and ordering.  Every pointer argument is owned by the caller and
 * the library never frees it.  Unless stated otherwise pointers are device
 * pointers on the device that was current at qcd_create.  All work is ordered
 * on the CUDA stream given to qcd_create.  qcd_load_gauge, qcd_clover_build,
 * qcd_cg_solve and qcd_fermion_force synchronise that stream before returning
 * (they report device-side status); qcd_dslash returns after enqueueing.
 * A call that takes a context makes the context's device current while it runs
 * and restores the caller's current device before it returns.  Each call is an
 * NVTX range named after it (visible to Nsight tools; free without one).
 *
 * Errors.  Every call returns a qcd_status; on failure qcd_last_error() gives a
 * message for the calling thread.  No C++ exception crosses the ABI.  Argument
 * errors are detected on the host before any launch.
 */
#ifndef QCD_H
#define QCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qcd_ctx qcd_ctx;

typedef enum {
  QCD_OK = 0,
  QCD_ERR_ARG = 1,           /* bad argument (null pointer, odd extent, unknown op, ...) */
  QCD_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  QCD_ERR_NOMEM = 3,         /* device allocation failed */
  QCD_ERR_STATE = 4,         /* call out of order (no gauge field, no clover term) */
  QCD_ERR_NOT_POSDEF = 5,    /* a clover block is not positive definite */
  QCD_ERR_NOT_CONVERGED = 6, /* CG hit max_iter; best x and stats are still written */
  QCD_ERR_NAN = 7,           /* non-finite input or a non-finite reduction */
  QCD_ERR_TIMEOUT = 8,       /* a bounded device-side wait (grid barrier of the persistent CG kernel) gave up */
  QCD_ERR_COMM = 9           /* a halo-exchange or sum callback of a t-slab call reported a failure */
} qcd_status;

/* qcd_load_gauge flags */
#define QCD_GAUGE_RECON12 1 /* store the FP32/FP16 link copies as rows 0,1 only (needs SU(3) links) */

/* qcd_dslash ops (precision = compute/storage precision of the operation) */
#define QCD_OP_DSLASH_EO 0  /* out_e = D_eo in_o   (dagger: out_e = (D_oe)^dag in_o) */
#define QCD_OP_DSLASH_OE 1  /* out_o = D_oe in_e   (dagger: out_o = (D_eo)^dag in_e) */
#define QCD_OP_MHAT 2       /* out_e = Mhat in_e   (dagger: Mhat^dag) */
#define QCD_OP_MDAGM 3      /* out_e = Mhat^dag Mhat in_e */
#define QCD_OP_CLOVER 4     /* out_e = A_ee in_e */
#define QCD_OP_CLOVER_INV 5 /* out_o = A_oo^-1 in_o */

/* precisions */
#define QCD_PREC_DOUBLE 64
#define QCD_PREC_SINGLE 32
#define QCD_PREC_HALF 16 /* FP16 spinors with one FP32 scale per site, FP32 arithmetic */

typedef struct {
  double tol;            /* target true relative residual |b - Mhat^dag Mhat x| / |b| (e.g. 1e-8) */
  int max_iter;          /* cap on CG iterations per right-hand side */
  int inner_prec;        /* 64: plain FP64 CG; 32 / 16: mixed precision with FP64 reliable updates */
  int reliable_every;    /* mixed: reliable update at least every this many iterations (e.g. 50) */
  double reliable_delta; /* mixed: reliable update once |r| < delta * |r at the last update| (e.g. 0.1) */
  int use_x0;            /* 1: x holds the initial guess; 0: start from x = 0 */
} qcd_solver_params;

typedef struct {
  int iters;              /* CG iterations */
  int reliable_updates;   /* FP64 residual replacements (including the final check) */
  double true_rel_resid;  /* |b - Mhat^dag Mhat x| / |b| recomputed in FP64 at exit */
  double b_dot_x;         /* Re <b, x>: the action S = phi^dag (Mhat^dag Mhat)^-1 phi when b = phi */
  double seconds;         /* wall time of the call (whole batch) */
} qcd_solver_stats;

/* qcd_fermion_force flags */
#define QCD_FORCE_INPUT_IS_SOLUTION 1 /* phi_or_x holds X = (Mhat^dag Mhat)^-1 phi: no solve */
#define QCD_FORCE_GRADIENT 2          /* write G = dS/dRe U + i dS/dIm U instead of the Lie-algebra force */
#define QCD_FORCE_CLOVER_DET 4        /* add the force of S_det = -2 sum_{x odd} log det A(x) */
#define QCD_FORCE_ACCUMULATE 8        /* qcd_gauge_force: add to F instead of overwriting it */
#define QCD_R_STEP_DEFER_CLOVER 16    /* qcd_r_step: leave the clover term of the new links unbuilt */

/*
 * Create a context for a lattice of extents dims = {X, Y, Z, T}; all must be
 * even and >= 2 and V = XYZT must satisfy 8 V < 2^31.  t_bc is +1 (periodic) or
 * -1 (antiperiodic) in time.  cuda_stream is a cudaStream_t (NULL: the legacy
 * default stream).  The context owns its device buffers (packed links, clover
 * term, solver work vectors), allocated on the device current at this call.
 * Returns QCD_ERR_ARG for bad extents, QCD_ERR_CUDA if no device is usable.
 */
qcd_status qcd_create(qcd_ctx** ctx, const int dims[4], double t_bc, void* cuda_stream);

/* Release every buffer the context owns.  NULL is accepted. */
qcd_status qcd_destroy(qcd_ctx* ctx);

/*
 * Load gauge links U in the canonical layout (V*4*9 complex128).  on_device = 1:
 * U is a device pointer; 0: a host pointer (copied).  Packs them into the
 * per-parity structure-of-arrays copies in FP64, FP32 and FP16 (the paper pads
 * MILC's su3_matrix for the Cell's DMA, Sec. 3; this layout needs no padding).
 * flags: QCD_GAUGE_RECON12.  Invalidates a previously built clover term.
 * Returns QCD_ERR_NAN if U holds a non-finite value.
 */
qcd_status qcd_load_gauge(qcd_ctx* ctx, const double* U, int on_device, int flags);

/*
 * Build the clover term A (both parities) from the loaded links and invert it
 * on every site in FP64 (Cholesky of each 6x6 chiral block); keeps FP64 and FP32
 * copies.  Returns QCD_ERR_STATE without links, QCD_ERR_NOT_POSDEF if a block
 * is not positive definite.
 */
qcd_status qcd_clover_build(qcd_ctx* ctx, double kappa, double csw);

/*
 * Apply one operator (QCD_OP_*) to nrhs canonical fields (V/2 sites each):
 * in and out are device complex128 arrays [nrhs][V/2][4][3] on the parities the
 * op names; they must not overlap.  precision (64/32/16) selects the internal
 * storage and arithmetic; the result is returned in FP64.  nrhs >= 1.
 * Returns QCD_ERR_STATE if the op needs links/clover that are not loaded.
 */
qcd_status qcd_dslash(qcd_ctx* ctx, double* out, const double* in, int op, int dagger, int precision, int nrhs);

/*
 * Solve Mhat^dag Mhat x = b for nrhs right-hand sides (device complex128
 * [nrhs][V/2][4][3]; x is read as the initial guess when params->use_x0).
 * inner_prec 64 runs plain FP64 CG; 32 or 16 runs the inner iteration in that
 * precision with FP64 reliable updates (x accumulated in FP64, the residual
 * recomputed in FP64 every reliable_every iterations or when |r| falls by
 * reliable_delta).  Every RHS stops when its true FP64 relative residual is
 * <= tol.  stats (may be NULL) receives nrhs entries.
 * Returns QCD_ERR_NOT_CONVERGED (x and stats written) at max_iter,
 * QCD_ERR_NAN on a non-finite reduction, QCD_ERR_STATE without a clover term.
 */
qcd_status qcd_cg_solve(qcd_ctx* ctx, double* x, const double* b, int nrhs, const qcd_solver_params* params,
                        qcd_solver_stats* stats);

/*
 * Fermion force of S = sum_i phi_i^dag (Mhat^dag Mhat)^-1 phi_i, summed over the
 * nrhs pseudofermions.  phi_or_x: device complex128 [nrhs][V/2][4][3], either
 * phi (a solve with params is run first; stats as in qcd_cg_solve, may be NULL)
 * or, with QCD_FORCE_INPUT_IS_SOLUTION, the solutions X.  F: device complex128
 * [t][z][y][x][mu][3][3]; by default the traceless anti-Hermitian force
 * F_mu(x) = sum_a i T_a dS/d eps_a for U_mu(x) -> exp(i eps_a T_a) U_mu(x)
 * (T_a = lambda_a/2), including the clover-term derivative; with
 * QCD_FORCE_GRADIENT the Wirtinger gradient G = dS/dRe U + i dS/dIm U.
 * Error behaviour as qcd_cg_solve.
 */
qcd_status qcd_fermion_force(qcd_ctx* ctx, double* F, const double* phi_or_x, int nrhs, int flags,
                             const qcd_solver_params* params, qcd_solver_stats* stats);
/*
 * With QCD_FORCE_CLOVER_DET the force (or gradient) of the clover determinant term of the even-odd
 * preconditioned two-flavour action is added: det M = det A_oo det Mhat, so the action carries
 * S_det = -2 log det A_oo = -2 sum_{x odd} log det A(x) besides the pseudofermion term (the form of
 * the clover_dynamical application the paper ports, Sec. 1).  Its derivative enters through the
 * clover leaves like the pseudofermion's clover term.  With this flag nrhs may be 0 (phi_or_x may
 * then be NULL): F is the determinant term alone.
 */

/*
 * log det of the clover term from the Cholesky factors of the last qcd_clover_build, summed over
 * the sites of each parity (both 6x6 chiral blocks): out[0] = sum_{x even} log det A(x),
 * out[1] = sum_{x odd} log det A(x); S_det = -2 out[1].  out: host array of 2.  Synchronises.
 * Returns QCD_ERR_STATE without a clover term.
 */
qcd_status qcd_clover_logdet(qcd_ctx* ctx, double out[2]);

/*
 * The full-lattice system M (x_e, x_o) = (b_e, b_o), M = [[A_ee, -kappa D_eo], [-kappa D_oe, A_oo]]
 * (even sites first), reduces to the even-site system Mhat x_e = b_e + kappa D_eo A_oo^-1 b_o and
 * the odd half x_o = A_oo^-1 (b_o + kappa D_oe x_e).  Both steps in FP64 on device complex128 fields
 * [nrhs][V/2][4][3]; b_o may be NULL (zero).  Outputs must not overlap inputs.
 * qcd_prepare_source: bhat_e = b_e + kappa D_eo A_oo^-1 b_o.
 * qcd_reconstruct_odd: x_o = A_oo^-1 (b_o + kappa D_oe x_e).
 * (Mhat x_e = bhat_e is solved as Mhat^dag Mhat x_e = Mhat^dag bhat_e with qcd_dslash and
 * qcd_cg_solve.)  Return QCD_ERR_STATE without a clover term.
 */
qcd_status qcd_prepare_source(qcd_ctx* ctx, double* bhat_e, const double* b_e, const double* b_o, int nrhs);
qcd_status qcd_reconstruct_odd(qcd_ctx* ctx, double* x_o, const double* x_e, const double* b_o, int nrhs);

/*
 * Molecular dynamics of the hybrid R algorithm the paper's application runs (Sec. 1, su3_rmd), with
 * the standard conventions: Wilson gauge action S_g = beta sum_x sum_{mu<nu} (1 - Re tr P_{mu nu}/3);
 * momenta P_mu(x) traceless anti-Hermitian (device complex128 [t][z][y][x][mu][3][3], like the
 * links), kinetic energy K = -sum tr P^2; equations of motion dU/dtau = P U, dP/dtau = -F with F
 * the Lie-algebra force of qcd_fermion_force's convention.
 *
 * qcd_gauge_force: F (or with QCD_FORCE_GRADIENT G) of S_g for the loaded links; with
 *   QCD_FORCE_ACCUMULATE added to F.
 * qcd_plaquette: *mean = < Re tr P_{mu nu}(x) / 3 > over sites and the six planes of the loaded links
 *   (S_g = 6 V beta (1 - mean)).  Synchronises.
 * qcd_kinetic_energy: *K = -sum tr P^2 = sum |P_ij|^2.  Synchronises.
 * qcd_update_links: U <- exp(eps P) U on every link (the exponential by scaling and squaring of a
 *   Taylor series, to rounding), then reunitarised (rows 0, 1 Gram-Schmidt, row 2 = conj(row 0 x
 *   row 1)).  Touches only U: the context's packed links are not reloaded.
 * qcd_r_step: one two-flavour R-algorithm step on U and P in place, for nrhs pseudofermion noise
 *   fields eta (device [nrhs][V/2][4][3], complex Gaussian drawn by the caller):
 *     U' = exp(eps/2 P) U;  phi = Mhat(U')^dag eta;  P -= eps (F_g + F_f(phi) [+ F_det]);
 *     U = exp(eps/2 P) U'
 *   (the noisy pseudofermion is drawn at the half step: the R algorithm's time shift
 *   eps (1 - N_f/2)/2 vanishes for the two flavours Mhat^dag Mhat describes).  kappa and c_sw are
 *   those of the last qcd_clover_build; flags: QCD_FORCE_CLOVER_DET adds the determinant term.
 *   params/stats as in qcd_fermion_force.  On return the context holds U's packed links and clover
 *   term; with QCD_R_STEP_DEFER_CLOVER the clover term is left unbuilt (operators return
 *   QCD_ERR_STATE until qcd_clover_build; another qcd_r_step needs no rebuild), which saves one
 *   clover build per step of a trajectory.  Synchronises.
 * All return QCD_ERR_STATE without loaded links (qcd_r_step: without a clover term).
 */
qcd_status qcd_gauge_force(qcd_ctx* ctx, double* F, double beta, int flags);
qcd_status qcd_plaquette(qcd_ctx* ctx, double* mean);
qcd_status qcd_kinetic_energy(qcd_ctx* ctx, const double* P, double* K);
qcd_status qcd_update_links(qcd_ctx* ctx, double* U, const double* P, double eps);
qcd_status qcd_r_step(qcd_ctx* ctx, double* U, double* P, const double* eta, int nrhs, double eps, double beta,
                      int flags, const qcd_solver_params* params, qcd_solver_stats* stats);

/*
 * Measurements per trajectory.
 * qcd_polyakov: out[0] + i out[1] = < tr prod_{t=0}^{T-1} U_t(xvec, t) / 3 > over the spatial sites of
 *   the loaded links (plain links: the antiperiodic sign belongs to the fermions).  Synchronises.
 * qcd_pbp: the stochastic psi-bar psi estimate out[r] = Re eta_r^dag M^-1 eta_r / (2V) for nrhs noise
 *   vectors eta_r = (eta_e, eta_o) (device [nrhs][V/2][4][3] each, complex Gaussian with unit
 *   variance per real drawn by the caller, so that it estimates Re Tr M^-1 / V): M^-1 eta through
 *   qcd_prepare_source, the CG of qcd_cg_solve on Mhat^dag Mhat x_e = Mhat^dag bhat_e (params,
 *   stats as there) and qcd_reconstruct_odd.  out: host array of nrhs.  Synchronises.
 */
qcd_status qcd_polyakov(qcd_ctx* ctx, double out[2]);
qcd_status qcd_pbp(qcd_ctx* ctx, const double* eta_e, const double* eta_o, int nrhs, double* out,
                   const qcd_solver_params* params, qcd_solver_stats* stats);

/*
 * Per-kernel timing with CUDA events on the context's stream.  enable = 1 resets
 * the counters and starts recording an event pair around every launch of the
 * tracked kernels (hopping kernels by epilogue, BLAS updates); 0 stops.
 */
qcd_status qcd_profile(qcd_ctx* ctx, int enable);

typedef struct {
  char name[40];         /* kernel class */
  int launches;
  double total_ms;       /* sum of event-measured durations */
  double bytes;          /* algorithmic bytes summed over the launches */
  double flops;          /* conventional flops summed over the launches */
} qcd_kernel_stat;

/* Copy up to max_entries kernel classes with at least one launch since the last
 * qcd_profile(ctx, 1) into out, then a "launches_total" entry (synchronises the stream). */
qcd_status qcd_profile_read(qcd_ctx* ctx, qcd_kernel_stat* out, int max_entries, int* n_entries);

/*
 * qcd_mhat_static -- out = Mhat in (dagger = 1: Mhat^dag in) in FP64 for one
 * even-site field, allocating no device memory.  The paper has no counterpart:
 * this entry exists for callers that cannot call cudaMalloc, such as a host
 * application whose memory pool already holds the GPU's free memory, or a
 * latency-sensitive loop that cannot take the device-wide synchronisation that
 * cudaMalloc / cudaFree may cause.  (qcd_dslash, by contrast, allocates its work
 * buffers on first use.)
 *
 * in, out: device complex128 [V/2][4][3] (canonical layout), not overlapping.
 * Work space is one file-scope device array of QCD_STATIC_SCRATCH_BYTES that every
 * GPU loading the library holds until exit; lattices needing more than
 * 3 * 192 * V/2 bytes of it are rejected with QCD_ERR_ARG before any launch.  The
 * first call on a device looks up the array's device address for that device
 * (make it before any stream capture) and keeps it for the life of the process,
 * which assumes that the device's primary context is not reset (cudaDeviceReset)
 * while the library is loaded.  All calls share the array, which keeps
 * the last call's contents (each call writes everything it reads); calls whose
 * work overlaps on the GPU race on it.  Needs qcd_load_gauge and
 * qcd_clover_build (QCD_ERR_STATE otherwise).  Enqueued on the context's stream;
 * returns without synchronising.
 */
#define QCD_STATIC_SCRATCH_BYTES (24u << 20)
qcd_status qcd_mhat_static(qcd_ctx* ctx, double* out, const double* in, int dagger);

/*
 * Failure-path self-test of the bounded grid barrier used by the persistent single-RHS CG kernel:
 * launches a two-block cooperative kernel in which one block never reaches the barrier, so the
 * other block's wait runs out (after about a second) and sets the context's error word.  Returns
 * QCD_ERR_TIMEOUT when the wait gave up as intended (QCD_OK would mean it did not); the context
 * stays usable.  Synchronises the context's stream.
 */
qcd_status qcd_selftest_barrier_timeout(qcd_ctx* ctx);

/*
 * Index checks of the debug build.  libqcd_debug.so (built with QCD_DEBUG=1 by
 * `python -m paper_0910_0262_gb300.build --debug`) checks, in every kernel, the indices handed to the
 * field accessors: the site (0 <= h < V/2, a face index against its face), the RHS (>= 0), the link's
 * parity and direction, the clover block.  A failed check records a bit in a device word of the
 * kernel's translation unit and skips the access (a load returns zeros, a store writes nothing), so
 * an indexing fault is reported instead of reading or writing out of range.
 * qcd_debug_violations: *violations = the OR of the bits recorded since the previous call
 * (QCD_DBG_SPINOR, QCD_DBG_LINK, QCD_DBG_CLOVER, QCD_DBG_HALO; ~0u if a word could not be read),
 * which it clears.  The words belong to the process on the context's device, not to the context: the
 * kernels of every context on that device record into them; *is_debug (may be null) = 1 in the debug build, 0 in the release build, whose
 * checks are compiled away (*violations is then 0).  Synchronises the context's stream.
 * qcd_selftest_debug_index: launches one thread that loads the FP64 spinor at site index V/2 (one
 * past the last site) from a scratch buffer of 13 V/2 complex doubles it allocates and frees, so
 * that the load stays inside the buffer even where it is not checked; the debug build records
 * QCD_DBG_SPINOR for it.  Synchronises the context's stream.
 */
#define QCD_DBG_SPINOR 1u
#define QCD_DBG_LINK 2u
#define QCD_DBG_CLOVER 4u
#define QCD_DBG_HALO 8u
qcd_status qcd_debug_violations(qcd_ctx* ctx, unsigned* violations, int* is_debug);
qcd_status qcd_selftest_debug_index(qcd_ctx* ctx);

/*
 * Host-only self-test of the multiply-and-shift division by a lattice extent that the kernels use
 * to turn a site index into coordinates (the same expression, evaluated on the host): checks every
 * even extent 2..1024 against integer division on the numerators 0..65535, near each multiple of
 * the extent up to 2^31 - 1, and on pseudo-random numerators.  Returns the number of mismatches
 * (0 on success); needs no GPU and no context.
 */
long long qcd_selftest_fastdiv(void);

/*
 * Host-only self-test of the order in which the staged FP32 multi-RHS hopping kernel takes its
 * 32-site blocks (chunks of time slices, plane by plane; the same function, evaluated on the host):
 * checks that it is a permutation of the blocks for every lattice with even extents X, Y, Z in 2..16
 * and T in 2..34, and for 32^3 x 64, 32^3 x 60, 48^3 x 96, 16^4 and 8 x 8 x 16 x 16.  Returns the
 * number of lattices where it is not (0 on success); needs no GPU and no context.
 */
long long qcd_selftest_site_order(void);

/*
 * Time decomposition over several GPUs (one process per GPU).  The paper runs its application as MPI
 * processes that each hold part of the lattice and exchange boundary data between kernels (Sec. 4);
 * here the global lattice X x Y x Z x T is cut into slabs of consecutive time slices, one per rank.
 * A hopping pass needs, at the sites of its first and last local slice, the spinors one slice beyond
 * the slab; only their spin projections enter the time hops, so each pass exchanges six complex
 * numbers per face site (X Y Z / 2 sites of the input's parity) in each direction, and every CG
 * reduction is summed over the ranks.  Both are done by the caller's callbacks (NCCL, MPI, or copies
 * between contexts of one process), so the library itself holds no communicator.
 *
 * qcd_create_slab: a context for the slab t_offset <= t < t_offset + t_local of the global lattice
 *   dims = {X, Y, Z, T} (t_offset and t_local even, t_local >= 2, t_offset + t_local <= T); fields of
 *   the slab are the global even/odd-site fields restricted to its time slices, in the canonical
 *   order of a lattice X x Y x Z x t_local (a contiguous range of the global field: half indices
 *   t_offset XYZ/2 .. (t_offset + t_local) XYZ/2).  t_bc applies at global time T-1.
 * qcd_load_gauge on a slab context takes the links of global times t_offset-2 .. t_offset+t_local+1
 *   (taken mod T), [t_local+4][Z][Y][X][4][3][3] complex128: the slab and two slices on each side,
 *   which the clover term of its boundary slices needs.  qcd_clover_build, qcd_clover_logdet (the
 *   slab's sites only) and qcd_profile work as on any context.  qcd_dslash and qcd_cg_solve need
 *   t_local = T (a slab that is the whole lattice); the force, molecular-dynamics, measurement and
 *   allocation-free calls are not available on slab contexts (QCD_ERR_STATE).
 * qcd_slab_halo_bytes: bytes each of the four halo buffers needs for nrhs fields at precision.
 * qcd_slab_dslash: qcd_dslash's operators on the slab's fields (DSLASH_EO/OE: one exchange; MHAT:
 *   two; MDAGM: four; CLOVER, CLOVER_INV: none).
 * qcd_slab_cg_solve: qcd_cg_solve on the slab decomposition, every rank calling it with its slab of
 *   x and b: the same iteration (FP64, or FP32 / FP16 inner with FP64 reliable updates), each hopping
 *   pass preceded by an exchange and each reduction summed through comm->allreduce; stats as in
 *   qcd_cg_solve (true residual of the whole lattice).  The callbacks are called from the calling
 *   thread; a rank's call returns after its stream is synchronised.
 *
 * qcd_slab_comm: send_lo/send_hi/recv_lo/recv_hi are device buffers of at least qcd_slab_halo_bytes
 * bytes, owned by the caller.  exchange(user, bytes) is called after the library has enqueued, on the
 * context's stream, the kernels that fill the first `bytes` of send_lo and send_hi; before kernels the
 * library enqueues after it returns, recv_hi must hold the slab above's send_lo faces and recv_lo the
 * slab below's send_hi faces (neighbours taken periodically in t; a single slab of the whole lattice is
 * its own neighbour), in that stream's order: copied there, or with recv_lo / recv_hi pointed at those
 * buffers by the callback.  The library reads the four pointers from *comm at every pass (send_lo and
 * send_hi before it packs, recv_lo and recv_hi after exchange returns), so the callback may rewrite
 * them, for example to alternate between buffer sets; the struct passed to a call must then be the
 * one the callback rewrites.  allreduce(user, values, n) replaces n doubles in device memory by their
 * sums over the ranks, likewise in stream order.  A nonzero return from either makes the call fail
 * with QCD_ERR_COMM.
 */
typedef int (*qcd_halo_exchange_fn)(void* user, size_t bytes);
typedef int (*qcd_allreduce_fn)(void* user, double* values, int n);
typedef struct {
  void* send_lo;
  void* send_hi;
  void* recv_lo;
  void* recv_hi;
  qcd_halo_exchange_fn exchange;
  qcd_allreduce_fn allreduce;
  void* user;
} qcd_slab_comm;

qcd_status qcd_create_slab(qcd_ctx** ctx, const int dims[4], int t_offset, int t_local, double t_bc,
                           void* cuda_stream);
qcd_status qcd_slab_halo_bytes(const qcd_ctx* ctx, int precision, int nrhs, size_t* bytes);
qcd_status qcd_slab_dslash(qcd_ctx* ctx, double* out, const double* in, int op, int dagger, int precision, int nrhs,
                           const qcd_slab_comm* comm);
qcd_status qcd_slab_cg_solve(qcd_ctx* ctx, double* x, const double* b, int nrhs, const qcd_solver_params* params,
                             qcd_solver_stats* stats, const qcd_slab_comm* comm);

/*
 * In-process slab group: the exchanges and sums for n slabs (1 <= n <= 16) of one lattice held by one
 * process on one GPU, each slab's qcd_slab_* calls made from a host thread of its own.
 * qcd_local_group_create: an empty group of n ranks.  qcd_local_group_join(grp, rank, ctx, comm):
 * rank `rank` is the slab context ctx (rank r's slab lies above rank r-1's, periodically; every rank's
 * context on the same device, else QCD_ERR_ARG); the group allocates the rank's two sets of send
 * buffers (qcd_slab_halo_bytes for FP64 and 8 RHS each) on ctx's device and fills *comm with them and
 * with the group's callbacks.  Every later qcd_slab_* call of ctx takes that same struct, which the
 * exchanges rewrite: the receive pointers name the neighbours' send buffers of the pass (read in
 * place), and the send pointers alternate between the two sets.  Every rank joins before any rank
 * calls; a call that finds a rank missing waits for it at the group's host barrier for up to two
 * minutes, then fails with QCD_ERR_COMM, as do all later calls of the group.  The callbacks do not
 * wait for the GPU: a rank records a CUDA event on its context's stream when its faces or partial
 * sums are ready, the ranks meet once per exchange or sum at a host barrier to publish them, and the
 * halo kernels and the sums (in rank order, the same bits on every rank) wait for them on the reading
 * rank's stream.  qcd_local_group_abort releases every rank waiting at the group's barrier and makes
 * this and every later call of the group fail with QCD_ERR_COMM (for a rank that will not come); a
 * rank whose callback fails before the barrier breaks the group the same way.
 * qcd_local_group_destroy frees the buffers and the group (after the last call).
 */
typedef struct qcd_local_group qcd_local_group;
qcd_status qcd_local_group_create(qcd_local_group** grp, int n);
qcd_status qcd_local_group_join(qcd_local_group* grp, int rank, qcd_ctx* ctx, qcd_slab_comm* comm);
qcd_status qcd_local_group_abort(qcd_local_group* grp);
qcd_status qcd_local_group_destroy(qcd_local_group* grp);

/*
 * Device-limit probes for the kernels' rooflines (the paper has no counterpart; it quotes the Cell's
 * peak rates, Sec. 2, and measures its DMA bandwidths, Sec. 3).  Both run on the current device,
 * ordered on cuda_stream (NULL: the legacy default stream), allocate their own buffers and
 * synchronise.  qcd_probe_fma_peak: the FMA throughput in TFLOP/s (2 flops per FMA) of a kernel
 * running 8 independent FMA chains per thread on every SM, in precision 64 or 32.
 * qcd_probe_copy_bandwidth: the bandwidth in GB/s (bytes read + written) of a copy between two
 * buffers of `bytes` each (a multiple of 16), timed over `reps` launches after one untimed launch;
 * buffers of at most 64 MiB are copied 32 times per launch (an L2-resident copy), larger ones once.
 */
qcd_status qcd_probe_fma_peak(int precision, void* cuda_stream, double* tflops);
qcd_status qcd_probe_copy_bandwidth(size_t bytes, int reps, void* cuda_stream, double* gbs);

/* Message describing the last failed call on this thread ("" if none). */
const char* qcd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QCD_H */
