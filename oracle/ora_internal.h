/* ora_internal.h -- helpers shared by the oracle's own source files only. */
#ifndef LGT_ORA_INTERNAL_H
#define LGT_ORA_INTERNAL_H
#include "oracle.h"

/* Philox counter word 3: which field a random number belongs to */
enum { ORA_FIELD_MOMENTA = 1, ORA_FIELD_XI = 2, ORA_FIELD_LINKS = 3, ORA_FIELD_METROPOLIS = 4,
       ORA_FIELD_SOURCE = 5 };

void ora_coords(const int d[4], long s, int x[4]);
long ora_index(const int d[4], const int x[4]);
long ora_neighbour(const int d[4], long s, int mu, int dir);
double ora_fermion_bc(const int d[4], long s, int mu, int dir);

void su3_mul(const ocplx *A, const ocplx *B, ocplx *C);
void su3_dag(const ocplx *A, ocplx *B);
void su3_from_coeffs(const double *h, ocplx *H);
void su3_expi(const ocplx *H, double eps, ocplx *out);

/* Dirac operator, CG, action and force vectors with an optional clover term C
 * ([V][12][12], NULL: Wilson); the public entry points pass NULL */
void ora_dirac_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, const ocplx *in,
                 ocplx *out, int dagger);
int ora_cg_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, int eo, const ocplx *b, ocplx *x,
             double tol, int max_iter, double *true_res);
double ora_pf_action_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, int eo, const ocplx *phi,
                       double tol, int max_iter, int *iters);
int ora_force_vectors_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, int eo,
                        const ocplx *phi, double tol, int max_iter, ocplx *X, ocplx *Y);
/* Dhat with the clover term C (NULL: Wilson) and Minv = (1 + C)^{-1} on odd sites */
void ora_dhat_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, const ocplx *Minv,
                const ocplx *in, ocplx *out, int dagger);
/* (1 + C(x))^{-1} on odd sites x into Minv ([V][12][12], even sites untouched); returns
 * the sum over odd sites of ln det (1 + C(x)) */
double ora_clover_inverse_odd(const int d[4], const ocplx *C, ocplx *Minv);
/* real-component gradient of the hopping part of S_f from X, Y (written to G) */
void ora_fermion_grad_xy(const int d[4], double kappa, const ocplx *X, const ocplx *Y, ocplx *G);

/* inner products over sites whose parity bit is in mask */
ocplx ora_dot(const int d[4], const ocplx *a, const ocplx *b, int mask);
double ora_norm2(const int d[4], const ocplx *a, int mask);

#endif
