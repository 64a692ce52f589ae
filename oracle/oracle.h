/*
 * oracle.h -- plain FP64 CPU oracle for the HMC hot path of
 * "Lattice Gauge Theory via LLVM-Level Automatic Differentiation"
 * (arXiv:2602.20516).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA path is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is double precision, written for readability, not speed: site
 * loops are parallelised with OpenMP and nothing else is reordered.
 *
 * Canonical layout (host arrays, full lattice):
 *   site s   = x0 + L0*(x1 + L1*(x2 + L2*x3)), mu = 3 is time
 *   links    U[(s*4+mu)*9 + 3*r + c]       complex double, row-major 3x3
 *   spinor   psi[(s*4+spin)*3 + colour]     complex double
 *   momenta  mom[(s*4+mu)*8 + a]            double, Pi = sum_a mom_a T^a
 *   forces   F[(s*4+mu)*8 + a]              double, F_a = d/de S(e^{ieT^a}U)
 *   gradient G[(s*4+mu)*9 + 3*r + c]        complex double, dS/dReU + i dS/dImU
 *
 * Conventions that the paper does not print are fixed here (one reading each):
 *   T^a = lambda^a/2 (Gell-Mann); Wilson-Dirac D = 1 - kappa*H with r = 1,
 *   fermions antiperiodic in time, chiral gamma basis (see ora_gamma);
 *   S_G = beta * sum_{x,mu<nu} (1 - Re tr U_munu / 3);
 *   left update U <- exp(i eps Pi) U with Pi Hermitian traceless (Eq. S2.1).
 *
 * Parity: every function is "parity pinned" by the not-gpu tests unless its
 * comment says "parity unpinned".
 */
#ifndef LGT_ORACLE_H
#define LGT_ORACLE_H

#include <stdint.h>
#include <complex.h>

typedef double complex ocplx;

/* ---------------- geometry ---------------- */
long ora_volume(const int d[4]);
int  ora_parity(const int d[4], long s);

/* ---------------- Philox-4x32-10 (Salmon et al., SC'11) ---------------- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* one pair of standard normals from counter (c0,c1,c2,c3) under key(seed) */
void ora_gauss_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                    double g[2]);
double ora_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3);

/* ---------------- small matrices ---------------- */
void ora_gamma(int mu, ocplx g[16]);     /* mu = 0..3, 4 -> gamma5, row-major 4x4 */
void ora_gellmann_T(int a, ocplx t[9]);  /* T^a = lambda^a / 2, a = 0..7 */
/* general n x n complex exponential by scaling-and-squaring of the Taylor series */
void ora_expm(int n, const ocplx *A, ocplx *out);

/* ---------------- seeded fields ---------------- */
/* U_mu(x) = exp(i alpha sum_a h_a T^a), h_a ~ N(0,1) from Philox (field id 3) */
void ora_random_links(const int d[4], uint64_t seed, double alpha, ocplx *U);
/* pi_a ~ N(0,1) per link (field id 1, trajectory counter traj) */
void ora_gaussian_momenta(const int d[4], uint64_t seed, uint32_t traj, double *mom);
/* complex Gaussian spinor with Re, Im ~ N(0, 1/2) on sites of parity mask
 * (mask bit 0 even, bit 1 odd; other sites set to 0); field id given */
void ora_gaussian_spinor(const int d[4], uint64_t seed, uint32_t traj, uint32_t field,
                         int parity_mask, ocplx *psi);

/* ---------------- Wilson-Dirac operator ---------------- */
/* out(x) = sum_mu [ b (1 + sf g_mu) U_mu(x) in(x+mu) + b (1 + sb g_mu) U_mu(x-mu)^+ in(x-mu) ]
 * for every site x whose parity bit is in out_mask (others untouched);
 * H: sf=-1, sb=+1.  H^+: sf=+1, sb=-1.  b = -1 across the time boundary. */
void ora_hop(const int d[4], const ocplx *U, const ocplx *in, ocplx *out,
             int out_mask, int dagger);
/* full-lattice D = 1 - kappa H, and D^+ = 1 - kappa H^+ (written out directly) */
void ora_dirac(const int d[4], const ocplx *U, double kappa, const ocplx *in, ocplx *out,
               int dagger);
/* even-odd Schur operator on even sites: Dhat = 1 - kappa^2 H_eo H_oe (dagger:
 * Dhat^+ = 1 - kappa^2 (H^+)_eo (H^+)_oe).  Odd sites of out are set to 0. */
void ora_dhat(const int d[4], const ocplx *U, double kappa, const ocplx *in, ocplx *out,
              int dagger);

/* ---------------- solver ---------------- */
/* CG on A x = b, A = D^+D (eo = 0, full lattice) or Dhat^+ Dhat (eo = 1, even sites).
 * x starts from 0.  Stops when the true residual |b - A x| / |b| <= tol.
 * Returns the iteration count (negative if max_iter was reached); *true_res gets
 * the final true relative residual. */
int ora_cg(const int d[4], const ocplx *U, double kappa, int eo, const ocplx *b, ocplx *x,
           double tol, int max_iter, double *true_res);

/* ---------------- actions ---------------- */
double ora_plaquette_sum(const int d[4], const ocplx *U);   /* sum_{x,mu<nu} Re tr U_munu / 3 */
double ora_gauge_action(const int d[4], const ocplx *U, double beta);
/* S_F = 2 Re(phi^+ chi) - |M chi|^2 with A chi = phi, M = D or Dhat (eo). */
double ora_pf_action(const int d[4], const ocplx *U, double kappa, int eo, const ocplx *phi,
                     double tol, int max_iter, int *iters);
double ora_momentum_energy(const int d[4], const double *mom);    /* 1/2 sum pi_a^2 */

/* ---------------- forces (Lie components F_a, accumulated: F += coef * dS) ------- */
void ora_gauge_force(const int d[4], const ocplx *U, double beta, double coef, double *F);
/* fermion force of delta S = -2 Re[Y^+ dD X] for given full-lattice X, Y */
void ora_fermion_force_xy(const int d[4], const ocplx *U, double kappa, const ocplx *X,
                          const ocplx *Y, double coef, double *F);
/* solves and assembles the pseudofermion force (full lattice or even-odd) */
int ora_pf_force(const int d[4], const ocplx *U, double kappa, int eo, const ocplx *phi,
                 double tol, int max_iter, double coef, double *F);
/* Lie components of a real-component gradient G: F_a = Re tr(G^+ i T^a U) */
void ora_grad_to_force(const int d[4], const ocplx *U, const ocplx *G, double *F);
/* real-component gradients G = dS/dReU + i dS/dImU of S_G and of S_F */
void ora_gauge_action_grad(const int d[4], const ocplx *U, double beta, ocplx *G);
int ora_pf_action_grad(const int d[4], const ocplx *U, double kappa, int eo,
                       const ocplx *phi, double tol, int max_iter, ocplx *G);

/* rectangle-improved gauge action (c0 = 1 - 8 c1; c1 = 0 is the Wilson action):
 * S_G = beta sum_x [c0 sum_{mu<nu}(1 - Re tr P/3) + c1 sum_{mu!=nu}(1 - Re tr R/3)] */
double ora_rectangle_sum(const int d[4], const ocplx *U);   /* sum_{x,mu!=nu} Re tr R_munu / 3 */
double ora_gauge_action_imp(const int d[4], const ocplx *U, double beta, double c1);
void ora_gauge_force_imp(const int d[4], const ocplx *U, double beta, double c1, double coef, double *F);
void ora_gauge_action_grad_imp(const int d[4], const ocplx *U, double beta, double c1, ocplx *G);

/* clover (Sheikholeslami-Wohlert) term, full lattice (below: even-odd form):
 * D_sw = 1 - kappa H + A, A(x) = -kappa c_sw sum_{mu<nu} sigma_munu F_munu(x),
 * sigma_munu = (i/2)[g_mu, g_nu], F_munu = (Q_munu - Q_munu^+)/(8i), Q the four leaves */
void ora_clover_field_strength(const int d[4], const ocplx *U, int mu, int nu, ocplx *F);   /* [V][3][3] */
void ora_clover_term(const int d[4], const ocplx *U, double kappa, double csw, ocplx *A);   /* [V][12][12] */
void ora_dirac_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *in, ocplx *out,
                  int dagger);
int ora_cg_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *b, ocplx *x, double tol,
              int max_iter, double *true_res);
double ora_pf_action_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi, double tol,
                        int max_iter, int *iters);
int ora_pf_action_grad_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi,
                          double tol, int max_iter, ocplx *G);
int ora_pf_force_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi, double tol,
                    int max_iter, double coef, double *F);
/* even-odd form: Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe (M = 1 + A) on even half fields
 * (canonical full fields, odd sites ignored / zero), the sum over odd sites of ln det M,
 * CG on Dhat^+ Dhat, S_f = phi_e^+ (Dhat^+ Dhat)^{-1} phi_e - 2 ln det M_oo, its
 * real-component gradient and its force */
void ora_dhat_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *in, ocplx *out,
                 int dagger);
double ora_clover_logdet_odd(const int d[4], const ocplx *U, double kappa, double csw);
int ora_cg_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *b, ocplx *x, double tol,
                 int max_iter, double *true_res);
double ora_pf_action_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi,
                           double tol, int max_iter, int *iters);
int ora_pf_action_grad_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi,
                             double tol, int max_iter, ocplx *G);
int ora_pf_force_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi, double tol,
                       int max_iter, double coef, double *F);

/* ---------------- link update ---------------- */
/* U <- exp(i eps Pi) U for every link (Eq. S2.1), Pi = sum_a mom_a T^a */
void ora_update_links(const int d[4], ocplx *U, const double *mom, double eps);
/* mom <- mom - eps * F (Eq. S2.2) */
void ora_kick(const int d[4], double *mom, const double *F, double eps);
/* Gram-Schmidt rows 1,2, row 3 = conj(row1 x row2) */
void ora_reunitarise(const int d[4], ocplx *U);

/* ---------------- stout smearing ---------------- */
/* one level: U' = exp(iQ) U, Q from Omega = C U^+, C = rho * sum of staples */
void ora_stout_forward(const int d[4], const ocplx *U, double rho, ocplx *Uout);
/* adjoint of one level: Gin = G(U) from Gout = G(U'); exp adjoint by the
 * block-triangular (Van Loan) identity, staple adjoints written out. */
void ora_stout_backward(const int d[4], const ocplx *U, double rho, const ocplx *Gout,
                        ocplx *Gin);

/* ---------------- HMC ---------------- */
typedef struct {
    double beta, kappa;
    int eo;              /* 0: full-lattice pseudofermion, 1: even-odd */
    int fermions;        /* 0: pure gauge */
    int integrator;      /* 0: leapfrog (PQP), 1: Omelyan 2MN, 2: Sexton-Weingarten */
    int n_steps;
    double tau;
    double tol_md, tol_action;
    int max_iter;
    int n_inner;         /* Sexton-Weingarten: gauge-force steps per outer step */
    int n_stout;         /* stout levels in front of the Wilson operator (S_G: thin links) */
    double rho;
    double c1;           /* rectangle coefficient of the gauge action (0: Wilson) */
    double csw;          /* clover coefficient of the pseudofermion operator (full lattice or even-odd) */
} ora_hmc_params;

/* parts of the MD force: 0 all, 1 gauge only, 2 fermion only */
int ora_md_force_part(const int d[4], const ocplx *U, const ora_hmc_params *p, const ocplx *phi,
                      int part, double *F);
/* H = K + S_G + S_f(smeared links) for given momenta and phi (S_f by the variational form) */
double ora_hamiltonian(const int d[4], const ocplx *U, const double *mom, const ocplx *phi,
                       const ora_hmc_params *p);

typedef struct {
    double dH, Sg_old, Sg_new, Sf_old, Sf_new, K_old, K_new, plaquette;
    int accepted, cg_iters, force_evals;
} ora_hmc_result;

/* total MD force F = dS_G + dS_F (coef = 1) */
int ora_md_force(const int d[4], const ocplx *U, const ora_hmc_params *p, const ocplx *phi,
                 double *F);
/* integrate (U, mom) over tau with the chosen integrator; phi fixed */
int ora_md_integrate(const int d[4], ocplx *U, double *mom, const ocplx *phi,
                     const ora_hmc_params *p);
/* one trajectory: heatbaths (counters traj), integrate, Metropolis, reunitarise */
int ora_hmc_trajectory(const int d[4], ocplx *U, const ora_hmc_params *p, uint64_t seed,
                       uint32_t traj, ora_hmc_result *res);

#endif
