/*
 * lgt.h -- C ABI of liblgt.so, the sm_103a (B300) implementation of the HMC hot
 * path of "Lattice Gauge Theory via LLVM-Level Automatic Differentiation"
 * (arXiv:2602.20516): the SU(3) plaquette gauge action and the two-flavour
 * Wilson pseudofermion action S_f = phi^+ (D^+D)^{-1} phi (Eq. S3.1), their
 * molecular-dynamics forces (Eq. 9 / Eq. S2.8 with the fermion variation of
 * Eq. S3.12), conjugate gradient on D^+D (Eq. S3.4), the left link update
 * U <- exp(i eps P) U (Eq. 6 / Eq. S2.1), the momentum update (Eq. S2.2) and
 * HMC trajectories.
 *
 * Conventions (the paper prints none of them; one reading each):
 *   - site s = x0 + L0*(x1 + L1*(x2 + L2*x3)); mu = 3 is time; every extent
 *     must be even; parity = (x0+x1+x2+x3) mod 2, even = 0.
 *   - T^a = lambda^a / 2; momenta P = sum_a pi_a T^a are Hermitian and
 *     traceless; a force F_a is d/de S(exp(i e T^a) U_mu(x)) at e = 0, and the
 *     MD kick is pi_a <- pi_a - eps F_a.
 *   - D = 1 - kappa H with
 *     (H psi)(x) = sum_mu [ b (1 - g_mu) U_mu(x) psi(x+mu) + b (1 + g_mu) U_mu(x-mu)^+ psi(x-mu) ],
 *     b = -1 on hops that wrap in time (antiperiodic fermions), chiral gammas
 *     g_k = [[0,-i s_k],[i s_k,0]] (mu = k-1 < 3), g_4 = [[0,1],[1,0]] (mu = 3).
 *   - Even-odd: Dhat = 1 - kappa^2 H_eo H_oe on even sites, Dhat^+ = g5 Dhat g5.
 *   - S_G = beta sum_{x, mu<nu} (1 - Re tr U_munu(x) / 3), plus the rectangle term of
 *     the improved actions when lgt_action_params.c1 != 0.
 *   - a real-component gradient ("G form", Eq. S2.11) is dS/dReU + i dS/dImU.
 *
 * Device layouts (all buffers below are DEVICE pointers owned by the caller;
 * Vh = V/2; "half field" = one parity):
 *   canonical links   complex128 [V][4][3][3]   (interleaved re,im doubles)
 *   canonical spinor  complex128 [V][4][3]      (spin, colour)
 *   canonical momenta double [V][4][8]
 *   FP64 spinor field double2 [parity][12][Vh]  component k = 3*spin + colour;
 *                     a half field is the [12][Vh] block of one parity
 *   FP32 spinor field float4  [parity][6][Vh]   float4 k holds components 2k, 2k+1
 *   DF64 spinor field float4  [parity][12][Vh]  component k as (re.hi, re.lo, im.hi, im.lo)
 *   momenta / forces  double2 [parity][4 mu][4][Vh]  double2 k holds pi_{2k}, pi_{2k+1}
 *   G-form gradient   double2 [parity][4 mu][9][Vh]  entry 3*row + col
 * The handle stores the gauge field as FP64 double2 [parity][4][9][Vh] plus an
 * FP32 two-row (12-real) copy float4 [parity][4][3][Vh] derived from it.
 *
 * Errors: every function returns an lgt_status; nothing aborts, traps or prints.
 * lgt_last_error() returns a thread-local message for the last failure.
 * Streams: all work is enqueued on the handle's stream (lgt_set_stream); calls
 * that return host scalars synchronise that stream before returning.
 * Thread safety: one handle must not be used by two threads at once.
 */
#ifndef LGT_H
#define LGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LGT_OK = 0,
    LGT_EINVAL = 1,   /* bad argument (odd extent, null pointer, unknown enum) */
    LGT_ENOMEM = 2,   /* allocation failed or over the memory budget */
    LGT_ENOCONV = 3,  /* solver hit max_iter; stats hold the last true residual */
    LGT_ENAN = 4,     /* a non-finite residual, action or energy was produced */
    LGT_ECUDA = 5,    /* a CUDA runtime call or launch failed */
    LGT_EKERNEL = 6   /* a kernel reported an internal error through its status word */
} lgt_status;

/* precision.  LGT_DF64 (double-float: a value is an unevaluated pair of FP32 numbers,
 * about 48 significant bits) is a field layout and operator arithmetic of
 * lgt_pack_spinor / lgt_unpack_spinor / lgt_dslash (LGT_OP_HOP only): float4
 * [parity][12][Vh], each float4 = (re.hi, re.lo, im.hi, im.lo), the bytes of FP64. */
enum { LGT_FP64 = 0, LGT_MIXED = 1, LGT_FP32 = 2, LGT_DF64 = 3 };
enum { LGT_EVEN = 0, LGT_ODD = 1, LGT_FULL = 2 };         /* parity selector */
/* operators of lgt_dslash */
enum { LGT_OP_HOP = 0,       /* out_p = H_{p,1-p} in_{1-p}, p = out_parity (EVEN|ODD) */
       LGT_OP_D = 1,         /* out = D in on the full lattice */
       LGT_OP_DHAT = 2,      /* out_e = Dhat in_e */
       LGT_OP_DHAT_NORMAL = 3 /* out_e = Dhat^+ Dhat in_e (dagger ignored) */ };
/* integrators: leapfrog (PQP), Omelyan 2MN, Sexton-Weingarten nested leapfrog (the
 * multiple time-scale integrator of Sec. III B: fermion force on the outer scale,
 * n_inner gauge-force leapfrog steps per outer step) */
enum { LGT_LEAPFROG = 0, LGT_OMELYAN2MN = 1, LGT_SEXTON_WEINGARTEN = 2 };
enum { LGT_FORCE_LIE = 0, LGT_GRAD_G = 1 };
enum { LGT_UPDATE_U = 0, LGT_UPDATE_P = 1 };
/* deepest stout chain in front of the Wilson operator */
#define LGT_MAX_STOUT 16
/* force arithmetic of the mixed-precision path (lgt_action_params.force_arith) */
enum { LGT_ARITH_FP64 = 0, LGT_ARITH_FP32 = 1, LGT_ARITH_DF64 = 2 };

typedef struct lgt_lattice *lgt_lattice_t;

/* Device-memory allocator.  alloc returns a device pointer (NULL on failure)
 * usable on `stream`; free releases it.  A NULL allocator makes the library
 * use cudaMalloc / cudaFree. */
typedef struct {
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, void *stream);
    void *ctx;
} lgt_allocator;

typedef struct {
    double beta;      /* gauge coupling of S_G; 0 drops S_G */
    double kappa;     /* hopping parameter of D */
    int fermions;     /* 1: include S_f, 0: pure gauge */
    int even_odd;     /* 1: S_f = phi_e^+ (Dhat^+Dhat)^{-1} phi_e; 0: full lattice */
    int n_stout;      /* stout levels in front of D (0 .. LGT_MAX_STOUT); S_G sees thin links */
    double rho;       /* stout parameter */
    int stout_recompute; /* storage of the smeared levels for the adjoint (every choice
                            gives the same gradient, bit for bit):
                            0: keep every level (n fields);
                            1: keep only the top level, recompute each level's input from
                               the thin links (2 fields, n(n-1)/2 extra smearing steps);
                            c >= 2: keep every c-th level as a checkpoint and recompute
                               each segment once from it (about n/c + c fields, fewer
                               than n extra smearing steps) */
    int force_arith;     /* arithmetic of Lie-form forces when the solver is LGT_MIXED
                            (with LGT_FP64 solves every force kernel is FP64):
                            LGT_ARITH_FP64 (0, default) FP64;
                            LGT_ARITH_FP32 FP32 accumulated in FP64 (about 1e-7 relative;
                              moves an MD trajectory's Delta H by ~1e-4);
                            LGT_ARITH_DF64 double-float: products carried as pairs of FP32
                              numbers (about 48 bits, ~1e-13 relative), accumulated in FP64 */
    double c1;           /* rectangle weight of the gauge action (not printed in the paper; an
                            improved discretisation of Sec. IV): S_G = beta sum_x [c0 sum_{mu<nu}
                            (1 - Re tr P/3) + c1 sum_{mu!=nu} (1 - Re tr R/3)], c0 = 1 - 8 c1,
                            R the 2 x 1 loop with its long side along mu.  0: Wilson action;
                            -1/12 tree-level Symanzik, -0.331 Iwasaki, -1.4088 DBW2.  With
                            c1 != 0 the LGT_ARITH_DF64 gauge force uses FP64 arithmetic. */
    double csw;          /* clover coefficient (not printed in the paper; a further discretisation
                            of Sec. IV): D = 1 - kappa H + A, A(x) = -kappa csw sum_{mu<nu}
                            sigma_munu F_munu(x), sigma_munu = (i/2)[g_mu, g_nu], F_munu =
                            (Q_munu - Q_munu^+)/(8i) with Q_munu the four plaquettes (leaves) of
                            the mu-nu plane at x.  With even_odd = 1, M = 1 + A and
                            Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe (M_oo^{-1} by Cholesky of the
                            two 6x6 chiral blocks per odd site), and S_f = phi_e^+ (Dhat^+
                            Dhat)^{-1} phi_e - 2 ln det M_oo (det D = det M_oo det Dhat); its force
                            adds the insertion of M_oo^{-1} to the clover force.  1 + A must be
                            positive definite on the odd sites (else LGT_ENAN).  The clover
                            force is FP64 arithmetic; chronological guesses are not used. */
} lgt_action_params;

typedef struct {
    int precision;    /* LGT_FP64 or LGT_MIXED (FP32 inner CG, FP64 reliable updates; a
                         breakdown of the FP32 recursion, <p,Ap> <= 0 from FP32 rounding near a
                         nearly singular operator, restarts it from the FP64 residual, and
                         two reliable updates that each fail to halve the residual hand the
                         rest of the solve to FP64 CG) */
    double tol;       /* stop when |b - A x| / |b| <= tol (true residual, FP64) */
    int max_iter;     /* iteration cap -> LGT_ENOCONV */
    double delta;     /* mixed: reliable update when |r| < delta * max|r| since the last one */
    int check_every;  /* iterations enqueued between host checks (0 -> default 16) */
    int chrono;       /* even-odd solves: 0 starts from x = 0; N = 1..LGT_MAX_RHS starts
                         from the combination of the handle's last N solutions of the same
                         operator (same kappa) that minimises the A-norm of the error
                         (chronological inverter, Brower et al., Nucl. Phys. B484 (1997)
                         353), each converged solve being recorded; the FP64 residual of
                         the guess is the first reliable update.  The history is cleared
                         by lgt_chrono_reset and at the start of lgt_hmc_trajectory. */
} lgt_solver_params;

typedef struct {
    int iters;               /* CG iterations (inner iterations for the mixed solver) */
    int reliable_updates;    /* FP64 residual replacements */
    double true_rel_residual;
    double seconds;          /* host wall time of the call */
    /* how the mixed solver got there (all 0 for a clean mixed solve; summed where
     * stats of several solves are accumulated): */
    int breakdowns;          /* FP32 recursions restarted from the FP64 residual after a
                                non-finite or non-positive <p, A p> */
    int diverged;            /* FP32 cycles dropped because their recursion residual grew
                                1e3-fold (in |r|^2) above the true residual they started from */
    int handovers;           /* solves whose FP32 iterations stopped reducing the true residual
                                (two reliable updates in a row short of halving it) and that
                                were finished by CG in FP64 */
    int fp64_iters;          /* iterations of CG in FP64 (every iteration of an LGT_FP64 solve;
                                the iterations after a hand-over in a mixed solve) */
    int restarts;            /* solves from a chronological guess redone from x = 0 */
} lgt_solve_stats;

typedef struct {
    int integrator;          /* LGT_LEAPFROG (PQP) or LGT_OMELYAN2MN */
    int n_steps;
    double tau;
    lgt_solver_params md_solver;      /* solves inside force evaluations */
    lgt_solver_params action_solver;  /* solve of the final action */
    int n_inner;                      /* LGT_SEXTON_WEINGARTEN: gauge steps per outer step */
} lgt_hmc_params;

typedef struct {
    double dH, Sg_old, Sg_new, Sf_old, Sf_new, K_old, K_new, plaquette;
    int accepted;
    int force_evals;
    lgt_solve_stats total;   /* summed over every solve of the trajectory */
} lgt_hmc_result;

/* ------------------------------------------------------------------ library */
/* Thread-local text of the last error (never NULL). */
const char *lgt_last_error(void);
/* ABI version (major*100 + minor). */
int lgt_version(void);

/* ------------------------------------------------------------------ lattice */
/* Create a lattice of extents dims[0..3] (all even, >= 2) on the current CUDA
 * device.  Allocates the gauge field and workspace through `alloc` (NULL:
 * cudaMalloc).  `stream` is a cudaStream_t (NULL: legacy default stream).
 * Gauge field starts as the unit field. */
int lgt_create_lattice(const int dims[4], const lgt_allocator *alloc, void *stream,
                       lgt_lattice_t *out);
/* Free everything the handle allocated.  NULL is accepted. */
int lgt_destroy_lattice(lgt_lattice_t lat);
int lgt_set_stream(lgt_lattice_t lat, void *stream);
/* V and the bytes of device memory the handle holds. */
int lgt_lattice_info(lgt_lattice_t lat, int64_t *volume, size_t *device_bytes);
/* Bytes of one field in the device layout: kind 0 spinor (parity LGT_EVEN/ODD
 * = half field, LGT_FULL = both), 1 momenta, 2 G-form gradient; precision
 * LGT_FP64 or LGT_FP32 (spinors only). */
int lgt_field_bytes(lgt_lattice_t lat, int kind, int parity, int precision, size_t *bytes);

/* ------------------------------------------------------------------ gauge field */
/* Copy a canonical link field (device, complex128 [V][4][3][3]) into the
 * handle; derives the FP32 two-row copy.  Links are used as given. */
int lgt_set_links(lgt_lattice_t lat, const double *links_canonical);
int lgt_get_links(lgt_lattice_t lat, double *links_canonical);
/* U_mu(x) = exp(i alpha sum_a h_a T^a), h_a ~ N(0,1) from Philox-4x32-10
 * (key = seed, counter = (4 s + mu, pair, 0, 3)), Box-Muller on 53-bit uniforms. */
int lgt_random_links(lgt_lattice_t lat, uint64_t seed, double alpha);
/* Gram-Schmidt rows 1, 2 and row 3 = conj(row1 x row2) on every link. */
int lgt_reunitarise(lgt_lattice_t lat);
/* <P> = sum_{x,mu<nu} Re tr U_munu / (3 * 6 V) (host result). */
int lgt_plaquette(lgt_lattice_t lat, double *plaq);
/* <R> = sum_{x,mu!=nu} Re tr R_munu / (3 * 12 V), R the 2 x 1 rectangle with its long
 * side along mu (host result). */
int lgt_rectangle(lgt_lattice_t lat, double *rect);

/* Mean plaquette, as lgt_plaquette, of a canonical link field (device,
 * complex128 [V][4][3][3], extents dims[0..3], all even) without allocating any
 * device memory and without a lattice handle.  The paper has no counterpart:
 * this entry point is for callers that cannot allocate device memory when they
 * need the number (inside another framework's memory pool or budget, allocator-
 * free runtimes, hooks between someone else's launches).  The result (one double)
 * is written to plaq_dev, a device pointer, in stream order on `stream`; the call
 * does not synchronise.  Scratch is a fixed file-scope device array, so
 * V > 8,388,608 sites is rejected with LGT_EINVAL.  The first call on each device
 * looks up that array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls share the array: calls whose
 * kernels overlap on the GPU race and must be serialised by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
int lgt_plaquette_noalloc(const double *links_canonical, const int dims[4], double *plaq_dev,
                          void *stream);

/* ------------------------------------------------------------------ layouts */
/* canonical spinor (device, complex128 [V][4][3]) <-> device field of the given
 * parity (LGT_EVEN/ODD: only that parity's sites) and precision. */
int lgt_pack_spinor(lgt_lattice_t lat, const double *canonical, void *field, int parity,
                    int precision);
int lgt_unpack_spinor(lgt_lattice_t lat, const void *field, double *canonical, int parity,
                      int precision);
/* canonical momenta / forces (device, double [V][4][8]) <-> device layout */
int lgt_pack_momenta(lgt_lattice_t lat, const double *canonical, double *mom);
int lgt_unpack_momenta(lgt_lattice_t lat, const double *mom, double *canonical);
/* canonical gradient (device, complex128 [V][4][3][3]) <-> G-form layout */
int lgt_pack_links_field(lgt_lattice_t lat, const double *canonical, double *field);
int lgt_unpack_links_field(lgt_lattice_t lat, const double *field, double *canonical);

/* ------------------------------------------------------------------ operators */
/* Attach the clover term with coefficient csw (see lgt_action_params.csw) for hopping
 * parameter kappa, built from the handle's current links, to the operators that act
 * on them directly: lgt_dslash (LGT_OP_D, and LGT_OP_DHAT / LGT_OP_DHAT_NORMAL as the
 * even-odd clover Dhat) and lgt_cg_solve (use the same kappa there).  csw = 0 detaches
 * it.  It is not refreshed when the links change (LGT_ENAN if 1 + A is not positive
 * definite on some odd site).
 * lgt_action, lgt_force, lgt_md_update and lgt_hmc_trajectory take the clover term
 * from lgt_action_params.csw instead.  Synchronous. */
int lgt_set_clover(lgt_lattice_t lat, double csw, double kappa);

/* Apply a Wilson-Dirac operator (Sec. III: "Wilson-Dirac operator"; D of
 * Eq. S3.1) to `in`, writing `out` (distinct buffers, device layout of
 * `precision`, LGT_FP64 or LGT_FP32; LGT_DF64 for LGT_OP_HOP only: the hop in
 * double-float arithmetic on a double-float copy of the links, the operator the
 * mixed solver forms its true residuals with).  op/out_parity as in the LGT_OP_*
 * enum; dagger != 0 applies the adjoint (H^+ = g5 H g5).  Asynchronous. */
int lgt_dslash(lgt_lattice_t lat, const void *in, void *out, int op, int out_parity,
               int dagger, double kappa, int precision);

/* Sweep order of the even-odd CG kernels (not in the paper; a B300 design choice):
 * alternate = 1 (the default) makes every hop and vector-update launch of a CG
 * iteration walk the sites in the direction opposite to the launch before it, so it
 * starts on the sites whose links and fields the previous launch left in L2; 0 walks
 * every launch forward.  The order of the sites only: results are bitwise the same. */
int lgt_set_sweep_order(lgt_lattice_t lat, int alternate);

/* Operand staging of the FP32 one-parity hops (the Wilson hop of Eq. S2.1 on one
 * parity, and the CG launches built from it).  mode bit 0: each block of 128 output
 * sites first copies its links (the forward U_mu(x) and backward U_mu(x - mu), 8 per
 * site) into shared memory with bulk copies; bit 1: likewise its input spinors with
 * the neighbour halos (the rows below and above, and the same rows of the planes
 * z -+ 1 and t -+ 1); 0 (the default) reads every operand through L1/L2.  Applies when
 * L0 / 2 divides 128 and 128 / (L0 / 2) divides L1; other lattices keep mode 0.  The
 * arithmetic is unchanged: results are bitwise those of mode 0.  Not in the paper.
 * Returns LGT_EINVAL for a mode outside 0..3. */
int lgt_set_hop_staging(lgt_lattice_t lat, int mode);

/* *applies = 1 when staging applies to this lattice's extents; *timeouts = the number
 * of staged blocks, since the library was loaded, whose wait for their copies gave up
 * after 0.5 s (such a block stores NaN, which the solvers report). */
int lgt_hop_staging_status(lgt_lattice_t lat, int *applies, unsigned *timeouts);


/* Solve A x = b, A = Dhat^+ Dhat on even sites (even_odd = 1; b, x FP64 half
 * fields) or A = D^+ D (even_odd = 0; full FP64 fields), by CG from x = 0
 * (Eq. S3.4: the solve is not differentiated).  Synchronous. */
int lgt_cg_solve(lgt_lattice_t lat, const double *b, double *x, double kappa, int even_odd,
                 const lgt_solver_params *sp, lgt_solve_stats *stats);

/* Forget the solutions kept for chronological initial guesses (lgt_solver_params.chrono),
 * e.g. when the pseudofermion source changes.  Not in the paper. */
int lgt_chrono_reset(lgt_lattice_t lat);

/* Several right-hand sides on the handle's links (not in the paper: the solve of
 * Eq. S3.4 repeated for nrhs sources, as a serving or multi-source workload needs).
 * Solves A_k x_k = b_k, A_k = Dhat_k^+ Dhat_k on even sites with kappa[k], for
 * k < nrhs <= LGT_MAX_RHS; b[k], x[k] are host arrays of device pointers to FP64
 * even half fields (distinct; x[k] aliases nothing), stats (NULL or nrhs entries).
 * LGT_MIXED: every FP32 operator application covers all running systems with one
 * load of each link (the hop moves 8 links + nrhs spinor pairs per site instead of
 * nrhs times 8 links + 1 pair); each system keeps its own scalars, stop test and
 * FP64 reliable updates, so its solution and counts equal those of lgt_cg_solve
 * alone.  LGT_FP64: the systems are solved one after another (the FP64 hop is
 * bound by FP64 arithmetic, which sharing link loads does not reduce).  The first
 * failing system's status is returned after all systems finished.  Synchronous. */
#define LGT_MAX_RHS 4
int lgt_cg_solve_multi(lgt_lattice_t lat, int nrhs, const double *const *b, double *const *x,
                       const double *kappa, const lgt_solver_params *sp, lgt_solve_stats *stats);
/* out_k = H_{p,1-p} in_k (dagger: H^+) for k < nrhs FP32 half fields (host arrays of
 * device pointers), with one load of each FP32 link for all of them; the result of
 * each equals lgt_dslash(LGT_OP_HOP, LGT_FP32) on that field.  Asynchronous. */
int lgt_hop_multi(lgt_lattice_t lat, int nrhs, const void *const *in, void *const *out, int out_parity,
                  int dagger);

/* ------------------------------------------------------------------ actions */
/* S_G (beta from ap) and S_f = phi^+ A^{-1} phi evaluated as 2 Re(phi^+ chi) - |M chi|^2
 * (A chi = phi), phi an FP64 device field (even half for even_odd, else full).
 * Either output pointer may be NULL.  Synchronous. */
int lgt_action(lgt_lattice_t lat, const lgt_action_params *ap, const double *phi,
               const lgt_solver_params *sp, double *S_g, double *S_f, lgt_solve_stats *stats);
/* Kinetic energy 1/2 sum pi_a^2 of a momentum field (device layout). */
int lgt_kinetic_energy(lgt_lattice_t lat, const double *mom, double *K);

/* ------------------------------------------------------------------ forces */
/* F = dS_G + dS_f (Eq. S2.8; fermion part from Eq. S3.12 with chi = A^{-1} phi,
 * eta = M chi).  form LGT_FORCE_LIE writes Lie components in the momentum
 * layout; LGT_GRAD_G writes the real-component gradient G in the G-form layout.
 * With ap->n_stout > 0 the actions are evaluated on the smeared field and the
 * force is taken back through the smearing (adjoint of each level).
 * Synchronous (returns after the solve). */
int lgt_force(lgt_lattice_t lat, const lgt_action_params *ap, const double *phi,
              const lgt_solver_params *sp, double *F_out, int form, lgt_solve_stats *stats);

/* Lie components F_a = Re tr(G^+ i T^a U) (the projection of Eq. 9 applied to a
 * real-component gradient G, Eq. S2.11) on the handle's links: G in the G-form
 * layout, F in the momentum layout (both device).  Asynchronous. */
int lgt_grad_to_lie(lgt_lattice_t lat, const double *G_field, double *F_mom);

/* ------------------------------------------------------------------ stout smearing */
/* n_levels of stout smearing (Morningstar-Peardon, the "smear" steps of Fig. 1)
 * of the handle's gauge field, written in canonical layout to out_canonical
 * (device, complex128 [V][4][3][3]); recompute selects the storage of the levels
 * as lgt_action_params.stout_recompute.  Synchronous. */
int lgt_stout_smear(lgt_lattice_t lat, double rho, int n_levels, int recompute, double *out_canonical);
/* Adjoint of that smearing (the reverse recursion of Eq. 3 through each level):
 * given the real-component gradient (Eq. S2.11) w.r.t. the top level, write the
 * gradient w.r.t. the handle's thin links (both canonical, device).  recompute as
 * lgt_action_params.stout_recompute (0 stored, 1 recomputed from the thin links,
 * c >= 2 checkpoints every c levels); the result does not depend on it.  Synchronous. */
int lgt_stout_backward(lgt_lattice_t lat, double rho, int n_levels, int recompute,
                       const double *G_top_canonical, double *G_thin_canonical);

/* ------------------------------------------------------------------ molecular dynamics */
/* which = LGT_UPDATE_U: U <- exp(i eps P) U (Eq. S2.1), P from mom.  With sp->precision =
 * LGT_MIXED and ap->force_arith = LGT_ARITH_DF64 (ap, sp non-NULL) and a double-float copy
 * of the current links at hand (left by a force evaluation on them), the update runs in
 * double-float arithmetic (~1e-14 relative); otherwise in FP64.
 * which = LGT_UPDATE_P: mom <- mom - eps F(U) (Eq. S2.2), F as in lgt_force. */
int lgt_md_update(lgt_lattice_t lat, double *mom, double eps, int which,
                  const lgt_action_params *ap, const double *phi, const lgt_solver_params *sp,
                  lgt_solve_stats *stats);
/* pi_a ~ N(0,1) (Philox counter (4 s + mu, pair, traj, 1)). */
int lgt_gaussian_momenta(lgt_lattice_t lat, double *mom, uint64_t seed, uint32_t traj);
/* complex Gaussian spinor, Re, Im ~ N(0, 1/2), on the sites of `parity`
 * (counter (s, component, traj, field)); field = 2 is the HMC heatbath xi. */
int lgt_gaussian_spinor(lgt_lattice_t lat, double *field, uint64_t seed, uint32_t traj,
                        uint32_t field_id, int parity);
/* Checkpoint of an HMC chain (not in the paper): its state is the FP64 links, the seed
 * and the index of the next trajectory (every random number is drawn by Philox from
 * seed, trajectory and site, so there is no generator state); a chain resumed from a
 * checkpoint repeats the next trajectory bitwise.  File (little-endian): 7 header words
 * of 64 bits (magic "LGTCKPT1"; version 1; dims[0] | dims[1] << 32; dims[2] | dims[3]
 * << 32; seed; next trajectory; payload bytes), the canonical links (complex128
 * [V][4][3][3]), and the FNV-1a hash (basis 0xcbf29ce484222325, prime 0x100000001b3)
 * of header and payload taken over 64-bit words.  load checks magic, version, the
 * handle's dims, the length and the hash (LGT_EINVAL on any mismatch, the handle's
 * links untouched), then sets the links (FP64 and the FP32 copy); seed and next_traj
 * may be NULL.  Both synchronous; the handle keeps one link field of staging memory. */
int lgt_save_checkpoint(lgt_lattice_t lat, const char *path, uint64_t seed, uint64_t next_traj);
int lgt_load_checkpoint(lgt_lattice_t lat, const char *path, uint64_t *seed, uint64_t *next_traj);

/* One HMC trajectory (Sec. III B): momentum and pseudofermion heatbaths
 * (phi = M^+ xi), integration, Metropolis with u from Philox (counter
 * (0,0,traj,4)), U restored on reject, then reunitarisation.  Synchronous. */
int lgt_hmc_trajectory(lgt_lattice_t lat, const lgt_action_params *ap,
                       const lgt_hmc_params *hp, uint64_t seed, uint32_t traj,
                       lgt_hmc_result *res);

/* ------------------------------------------------------------------ serving */
/* A request server over a pool of resident gauge fields of different volumes.
 * Requests (Dirac solves and force evaluations) are queued by lgt_server_submit
 * and advanced by lgt_server_step: each step admits queued requests in arrival
 * order while active slots and the HBM budget allow, runs `batch_iters` CG
 * iterations of every running request with batched launches (one launch per CG
 * kernel step covers all running requests of a precision, whatever their
 * volume), forms the true residual of requests whose stop condition fired (mixed
 * requests: a reliable update), and finishes converged requests.  The true residual
 * is formed with the FP64 hop, or, for a mixed request on a gauge field that has a
 * double-float copy, with the double-float hop (as the mixed lgt_cg_solve); such a
 * force request's forces are then taken in double-float arithmetic as well.
 * lgt_server_add_gauge makes the double-float copy (as many bytes as the FP64 links)
 * when the gauge fields added so far, with their copies, stay within half the budget.  A request's arithmetic does not
 * depend on the other requests: its result is the same alone and in any mix.  Timestamps are host steady-clock seconds
 * (lgt_clock).  Memory of requests, gauge fields and descriptors is allocated
 * through `alloc` (NULL: cudaMalloc) and counted against hbm_budget_bytes. */
typedef struct lgt_server *lgt_server_t;
enum { LGT_REQ_SOLVE = 0,   /* x = D^{-1} b, b Gaussian from source_seed, by even-odd CGNE:
                               Dhat^+Dhat x_e = Dhat^+(b_e + kappa H_eo b_o), x_o = b_o + kappa H_oe x_e */
       LGT_REQ_FORCE = 1 }; /* F = dS_G + dS_f (even-odd S_f, phi_e Gaussian from source_seed), Lie form */
typedef struct {
    int gauge_id;        /* from lgt_server_add_gauge */
    int kind;            /* LGT_REQ_SOLVE or LGT_REQ_FORCE */
    int precision;       /* LGT_FP64 or LGT_MIXED */
    double kappa, beta;  /* beta only for force requests (0 drops S_G) */
    double tol;          /* true relative residual of the normal equations */
    int max_iter;
    uint64_t source_seed;
    int keep_result;     /* 1: keep the result on the device until lgt_server_result */
} lgt_request;
typedef struct {
    uint64_t id;
    int status;          /* LGT_OK, LGT_ENOCONV, LGT_ENAN, LGT_ENOMEM (cannot fit the budget) */
    int iters, reliable_updates;
    double true_rel_residual;
    double t_submit, t_admit, t_done;
} lgt_completion;

/* delta: reliable-update threshold of mixed requests (<= 0: 1e-3). */
int lgt_server_create(const lgt_allocator *alloc, size_t hbm_budget_bytes, int max_active, int batch_iters,
                      double delta, void *stream, lgt_server_t *out);
int lgt_server_destroy(lgt_server_t srv);
/* Add a resident gauge field exp(i alpha H) (Philox seed, as lgt_random_links). */
int lgt_server_add_gauge(lgt_server_t srv, const int dims[4], uint64_t seed, double alpha, int *gauge_id);
/* Canonical copy (device, complex128 [V][4][3][3]) of a resident gauge field. */
int lgt_server_get_links(lgt_server_t srv, int gauge_id, double *links_canonical);
/* Queue a request (non-blocking); returns its id. */
int lgt_server_submit(lgt_server_t srv, const lgt_request *req, uint64_t *id);
/* One scheduling step (see above); synchronises the server's stream. */
int lgt_server_step(lgt_server_t srv, int *n_active, int *n_queued);
/* Completions since the last poll (at most max); *n gets the count. */
int lgt_server_poll(lgt_server_t srv, lgt_completion *out, int max, int *n);
/* Copy a kept result to out_dev (solve: FP64 full spinor field [2][12][Vh];
 * force: momentum layout) and release it; out_dev NULL only releases it. */
int lgt_server_result(lgt_server_t srv, uint64_t id, double *out_dev, size_t bytes);
int lgt_server_info(lgt_server_t srv, size_t *used_bytes, size_t *budget_bytes, int *n_active, int *n_queued);
/* Host steady clock in seconds (the clock of the completion timestamps). */
double lgt_clock(void);

/* ------------------------------------------------------------------ diagnostics */
/* Peak FP64 FMA throughput of this device (dependent FMA chains), in FLOP/s. */
int lgt_measure_fp64_peak(double *flops, double *seconds);
/* CUDA-event timing of the Wilson hop launches: start arms up to max_launches
 * event pairs (recorded on the launching stream around each hop launch of any
 * handle); stop waits for them and fills ms[LGT_TIMING_KINDS] / n[LGT_TIMING_KINDS]
 * with the summed durations (ms) and counts per kind = 5 * arithmetic + epilogue
 * (arithmetic 0 FP32, 1 FP64, 2 double-float; epilogue 0 hop, 1 xpay, 2 xpay + norm,
 * 3 fused CG residual update, 4 true residual).  Launches
 * shorter than min_ms are only counted (n_short): inside a CG batch, hops enqueued
 * after the solver stopped return at entry and do no work.  Process-wide; not
 * thread safe. */
#define LGT_TIMING_KINDS 15
int lgt_kernel_timing_start(int max_launches);
/* Record only every `every`-th hop launch (>= 1; 1, the default, records all).  Each
 * recorded pair adds a small gap to the stream; sampling keeps the timed region close
 * to its untimed speed while every kind of hop is still measured many times. */
int lgt_kernel_timing_sample(int every);
int lgt_kernel_timing_stop(double min_ms, double *ms, int64_t *n, int64_t *n_short);
/* Kernel launches the library enqueued on this thread since the last reset. */
int64_t lgt_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif
