/*
 * ora_dirac.c -- Wilson-Dirac operator, even-odd Schur operator, CG, the
 * pseudofermion action S_f = phi^+ (D^+D)^{-1} phi (Eq. S3.1) and its force
 * from delta S_f = -2 Re[eta^+ (delta D) chi] (Eq. S3.12).
 * Test infrastructure only (see oracle.h).
 */
#include "oracle.h"
#include "ora_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Hopping term, written as the 4x4 spin matrix (1 + s gamma_mu) times the 3x3
 * colour matrix, summed over the 8 neighbours.
 *   out(x) = sum_mu [ b (1 + sf g_mu) U_mu(x) in(x+mu) + b (1 + sb g_mu) U_mu(x-mu)^+ in(x-mu) ]
 * ------------------------------------------------------------------------- */
static void hop_site(const int d[4], const ocplx *U, const ocplx *in, long x, int sf, int sb,
                     const ocplx gam[4][16], ocplx out[12])
{
    for (int i = 0; i < 12; ++i) out[i] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            long y = ora_neighbour(d, x, mu, dir);
            double b = ora_fermion_bc(d, x, mu, dir);
            double s = (dir > 0) ? sf : sb;
            ocplx M[9];
            if (dir > 0) memcpy(M, &U[(x * 4 + mu) * 9], sizeof M);
            else su3_dag(&U[(y * 4 + mu) * 9], M);
            /* colour: Mpsi[spin][c] = sum_c' M[c][c'] in(y)[spin][c'] */
            ocplx Mpsi[12];
            for (int sp = 0; sp < 4; ++sp)
                for (int c = 0; c < 3; ++c) {
                    ocplx acc = 0;
                    for (int k = 0; k < 3; ++k) acc += M[c * 3 + k] * in[y * 12 + sp * 3 + k];
                    Mpsi[sp * 3 + c] = acc;
                }
            /* spin: (1 + s gamma_mu) */
            for (int a = 0; a < 4; ++a)
                for (int c = 0; c < 3; ++c) {
                    ocplx acc = Mpsi[a * 3 + c];
                    for (int bsp = 0; bsp < 4; ++bsp)
                        acc += s * gam[mu][a * 4 + bsp] * Mpsi[bsp * 3 + c];
                    out[a * 3 + c] += b * acc;
                }
        }
    }
}

void ora_hop(const int d[4], const ocplx *U, const ocplx *in, ocplx *out, int out_mask,
             int dagger)
{
    ocplx gam[4][16];
    for (int mu = 0; mu < 4; ++mu) ora_gamma(mu, gam[mu]);
    int sf = dagger ? +1 : -1;
    int sb = -sf;
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        if (!(out_mask & (1 << ora_parity(d, x)))) continue;
        hop_site(d, U, in, x, sf, sb, gam, &out[x * 12]);
    }
}

/* D = 1 - kappa H (+ A when a clover term A, [V][12][12], is given; A is Hermitian,
 * so D^+ = 1 - kappa H^+ + A) */
void ora_dirac_c(const int d[4], const ocplx *U, double kappa, const ocplx *A, const ocplx *in,
                 ocplx *out, int dagger)
{
    long V = ora_volume(d);
    ora_hop(d, U, in, out, 3, dagger);
    for (long i = 0; i < V * 12; ++i) out[i] = in[i] - kappa * out[i];
    if (!A) return;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int i = 0; i < 12; ++i) {
            ocplx acc = 0;
            for (int j = 0; j < 12; ++j) acc += A[(x * 12 + i) * 12 + j] * in[x * 12 + j];
            out[x * 12 + i] += acc;
        }
}

void ora_dirac(const int d[4], const ocplx *U, double kappa, const ocplx *in, ocplx *out,
               int dagger)
{
    ora_dirac_c(d, U, kappa, NULL, in, out, dagger);
}

/* out[x] = Ms[x] in[x] on the sites of parity p, Ms a [V][12][12] field of site matrices */
static void site_apply(const int d[4], const ocplx *Ms, int p, const ocplx *in, ocplx *out)
{
    long V = ora_volume(d);
    for (long x = 0; x < V; ++x) {
        if (ora_parity(d, x) != p) continue;
        for (int i = 0; i < 12; ++i) {
            ocplx acc = 0;
            for (int j = 0; j < 12; ++j) acc += Ms[(x * 12 + i) * 12 + j] * in[x * 12 + j];
            out[x * 12 + i] = acc;
        }
    }
}

/* Schur complement on even sites of D = [[M_ee, -kappa H_eo], [-kappa H_oe, M_oo]]:
 *   Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe,
 * M = 1 without a clover term (C = NULL), M = 1 + C with one (Minv = M^{-1} on odd
 * sites).  M is Hermitian, so the adjoint swaps H for H^+ only. */
void ora_dhat_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, const ocplx *Minv,
                const ocplx *in, ocplx *out, int dagger)
{
    long V = ora_volume(d);
    ocplx *t = calloc(V * 12, sizeof(ocplx));
    ocplx *u = calloc(V * 12, sizeof(ocplx));
    ocplx *m = NULL;
    ora_hop(d, U, in, t, 2, dagger);   /* odd sites from even in */
    if (C) {
        ocplx *t2 = calloc(V * 12, sizeof(ocplx));
        site_apply(d, Minv, 1, t, t2);
        free(t);
        t = t2;
        m = calloc(V * 12, sizeof(ocplx));
        site_apply(d, C, 0, in, m);    /* A_ee in */
    }
    ora_hop(d, U, t, u, 1, dagger);    /* even sites from odd t */
    for (long x = 0; x < V; ++x) {
        int even = (ora_parity(d, x) == 0);
        for (int i = 0; i < 12; ++i)
            out[x * 12 + i] = even ? in[x * 12 + i] + (m ? m[x * 12 + i] : 0) - kappa * kappa * u[x * 12 + i] : 0;
    }
    free(t);
    free(u);
    free(m);
}

void ora_dhat(const int d[4], const ocplx *U, double kappa, const ocplx *in, ocplx *out,
              int dagger)
{
    ora_dhat_c(d, U, kappa, NULL, NULL, in, out, dagger);
}

ocplx ora_dot(const int d[4], const ocplx *a, const ocplx *b, int mask)
{
    long V = ora_volume(d);
    ocplx acc = 0;
    for (long x = 0; x < V; ++x) {
        if (!(mask & (1 << ora_parity(d, x)))) continue;
        for (int i = 0; i < 12; ++i) acc += conj(a[x * 12 + i]) * b[x * 12 + i];
    }
    return acc;
}

double ora_norm2(const int d[4], const ocplx *a, int mask)
{
    return creal(ora_dot(d, a, a, mask));
}

/* A = M^+ M with M = D (full, with clover term C if given) or Dhat (even sites; with
 * C, Minv = (1 + C)^{-1} on odd sites) */
static void apply_A(const int d[4], const ocplx *U, double kappa, const ocplx *C, const ocplx *Minv, int eo,
                    const ocplx *in, ocplx *out, ocplx *tmp)
{
    if (eo) {
        ora_dhat_c(d, U, kappa, C, Minv, in, tmp, 0);
        ora_dhat_c(d, U, kappa, C, Minv, tmp, out, 1);
    } else {
        ora_dirac_c(d, U, kappa, C, in, tmp, 0);
        ora_dirac_c(d, U, kappa, C, tmp, out, 1);
    }
}

/* ---------------------------------------------------------------------------
 * Conjugate gradient (Hestenes-Stiefel), zero initial guess.  The linear solve
 * of Eq. S3.4 is not differentiated; only its solution enters the force.
 * When the recursive residual passes tol the true residual is formed; if it is
 * still above tol the recursion restarts from it.
 * ------------------------------------------------------------------------- */
int ora_cg_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, int eo, const ocplx *b, ocplx *x,
             double tol, int max_iter, double *true_res)
{
    long n = ora_volume(d) * 12;
    int mask = eo ? 1 : 3;
    ocplx *r = malloc(n * sizeof(ocplx));
    ocplx *p = malloc(n * sizeof(ocplx));
    ocplx *Ap = malloc(n * sizeof(ocplx));
    ocplx *tmp = malloc(n * sizeof(ocplx));
    ocplx *Minv = NULL;
    if (eo && C) {
        Minv = calloc(n * 12, sizeof(ocplx));
        ora_clover_inverse_odd(d, C, Minv);
    }
    double bb = ora_norm2(d, b, mask);
    for (long i = 0; i < n; ++i) { x[i] = 0; r[i] = b[i]; p[i] = b[i]; }
    double rr = bb;
    int k = 0, converged = 0;
    double res = (bb > 0) ? 1.0 : 0.0;
    if (bb == 0) converged = 1;
    while (!converged && k < max_iter) {
        apply_A(d, U, kappa, C, Minv, eo, p, Ap, tmp);
        double pAp = creal(ora_dot(d, p, Ap, mask));
        double alpha = rr / pAp;
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
        double rr_new = ora_norm2(d, r, mask);
        ++k;
        if (rr_new <= tol * tol * bb) {
            apply_A(d, U, kappa, C, Minv, eo, x, Ap, tmp);
            for (long i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
            rr_new = ora_norm2(d, r, mask);
            res = sqrt(rr_new / bb);
            if (res <= tol) { converged = 1; break; }
        }
        double beta = rr_new / rr;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    if (!converged) {
        apply_A(d, U, kappa, C, Minv, eo, x, Ap, tmp);
        for (long i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
        res = sqrt(ora_norm2(d, r, mask) / bb);
    }
    if (true_res) *true_res = res;
    free(r); free(p); free(Ap); free(tmp); free(Minv);
    return converged ? k : -k;
}

int ora_cg(const int d[4], const ocplx *U, double kappa, int eo, const ocplx *b, ocplx *x,
           double tol, int max_iter, double *true_res)
{
    return ora_cg_c(d, U, kappa, NULL, eo, b, x, tol, max_iter, true_res);
}

/* S_f = phi^+ A^{-1} phi evaluated as 2 Re(phi^+ chi) - |M chi|^2, which equals it
 * at the exact chi and deviates only quadratically in the solver error. */
double ora_pf_action_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, int eo, const ocplx *phi,
                       double tol, int max_iter, int *iters)
{
    long n = ora_volume(d) * 12;
    int mask = eo ? 1 : 3;
    ocplx *chi = malloc(n * sizeof(ocplx));
    ocplx *eta = malloc(n * sizeof(ocplx));
    double res;
    int it = ora_cg_c(d, U, kappa, C, eo, phi, chi, tol, max_iter, &res);
    if (iters) *iters = it;
    double S_det = 0.0;
    if (eo && C) {
        /* det(D^+ D) = det(M_oo)^2 det(Dhat^+ Dhat): the odd-site clover determinant is
         * part of the even-odd action, -2 ln det M_oo */
        ocplx *Minv = calloc(n * 12, sizeof(ocplx));
        S_det = -2.0 * ora_clover_inverse_odd(d, C, Minv);
        ora_dhat_c(d, U, kappa, C, Minv, chi, eta, 0);
        free(Minv);
    } else if (eo) {
        ora_dhat(d, U, kappa, chi, eta, 0);
    } else {
        ora_dirac_c(d, U, kappa, C, chi, eta, 0);
    }
    double S = 2 * creal(ora_dot(d, phi, chi, mask)) - ora_norm2(d, eta, mask) + S_det;
    free(chi);
    free(eta);
    return S;
}

double ora_pf_action(const int d[4], const ocplx *U, double kappa, int eo, const ocplx *phi,
                     double tol, int max_iter, int *iters)
{
    return ora_pf_action_c(d, U, kappa, NULL, eo, phi, tol, max_iter, iters);
}

/* ---------------------------------------------------------------------------
 * Fermion force from Eq. S3.12 with chi -> X, eta -> Y.  Writing out the two
 * places where U_mu(x) enters Y^+ H X,
 *   P1 = b sum_s [(1 - g_mu) X(x+mu)]_s Y(x)_s^+ ,
 *   P2 = b sum_s X(x)_s [(1 + g_mu) Y(x+mu)]_s^+ ,
 *   W  = U P1 - P2 U^+ ,    d_a S_f = -2 kappa Im tr(T^a W),
 * and the real-component gradient G = 2 kappa (P1^+ + P2).
 * ------------------------------------------------------------------------- */
static void outer_terms(const int d[4], const ocplx *X, const ocplx *Y, long x, int mu,
                        const ocplx gam[16], ocplx P1[9], ocplx P2[9])
{
    long y = ora_neighbour(d, x, mu, +1);
    double b = ora_fermion_bc(d, x, mu, +1);
    ocplx PX[12], PY[12];   /* (1 - g) X(x+mu), (1 + g) Y(x+mu) */
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) {
            ocplx ax = X[y * 12 + a * 3 + c], ay = Y[y * 12 + a * 3 + c];
            for (int s = 0; s < 4; ++s) {
                ax -= gam[a * 4 + s] * X[y * 12 + s * 3 + c];
                ay += gam[a * 4 + s] * Y[y * 12 + s * 3 + c];
            }
            PX[a * 3 + c] = ax;
            PY[a * 3 + c] = ay;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            ocplx s1 = 0, s2 = 0;
            for (int s = 0; s < 4; ++s) {
                s1 += PX[s * 3 + i] * conj(Y[x * 12 + s * 3 + j]);
                s2 += X[x * 12 + s * 3 + i] * conj(PY[s * 3 + j]);
            }
            P1[i * 3 + j] = b * s1;
            P2[i * 3 + j] = b * s2;
        }
}

void ora_fermion_force_xy(const int d[4], const ocplx *U, double kappa, const ocplx *X,
                          const ocplx *Y, double coef, double *F)
{
    ocplx gam[4][16];
    for (int mu = 0; mu < 4; ++mu) ora_gamma(mu, gam[mu]);
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx P1[9], P2[9], A[9], B[9], Ud[9], W[9], T[9];
            const ocplx *Uxm = &U[(x * 4 + mu) * 9];
            outer_terms(d, X, Y, x, mu, gam[mu], P1, P2);
            su3_mul(Uxm, P1, A);
            su3_dag(Uxm, Ud);
            su3_mul(P2, Ud, B);
            for (int i = 0; i < 9; ++i) W[i] = A[i] - B[i];
            for (int a = 0; a < 8; ++a) {
                ora_gellmann_T(a, T);
                ocplx tr = 0;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) tr += T[i * 3 + k] * W[k * 3 + i];
                F[(x * 4 + mu) * 8 + a] += coef * (-2.0 * kappa * cimag(tr));
            }
        }
}

void ora_fermion_grad_xy(const int d[4], double kappa, const ocplx *X, const ocplx *Y, ocplx *G)
{
    ocplx gam[4][16];
    for (int mu = 0; mu < 4; ++mu) ora_gamma(mu, gam[mu]);
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx P1[9], P2[9], P1d[9];
            outer_terms(d, X, Y, x, mu, gam[mu], P1, P2);
            su3_dag(P1, P1d);
            for (int i = 0; i < 9; ++i) G[(x * 4 + mu) * 9 + i] = 2.0 * kappa * (P1d[i] + P2[i]);
        }
}

/* X and Y of the force: full lattice X = chi, Y = D chi; even-odd
 * X = (chi_e, kappa M_oo^{-1} H_oe chi_e), Y = (eta_e, kappa M_oo^{-1} (H^+)_oe eta_e),
 * eta_e = Dhat chi_e (M_oo = 1 without a clover term), from
 *   eta_e^+ (delta Dhat) chi_e = Y^+ (-kappa delta H + delta A) X
 * (delta Dhat = delta A_ee - kappa^2 delta H_eo M^{-1} H_oe - kappa^2 H_eo M^{-1} delta H_oe
 *  + kappa^2 H_eo M^{-1} delta A_oo M^{-1} H_oe, the last term being Y_o^+ delta A_oo X_o). */
int ora_force_vectors_c(const int d[4], const ocplx *U, double kappa, const ocplx *C, int eo,
                        const ocplx *phi, double tol, int max_iter, ocplx *X, ocplx *Y)
{
    long n = ora_volume(d) * 12;
    double res;
    int it = ora_cg_c(d, U, kappa, C, eo, phi, X, tol, max_iter, &res);
    if (!eo) {
        ora_dirac_c(d, U, kappa, C, X, Y, 0);
        return it;
    }
    ocplx *Minv = NULL;
    if (C) {
        Minv = calloc(n * 12, sizeof(ocplx));
        ora_clover_inverse_odd(d, C, Minv);
    }
    ora_dhat_c(d, U, kappa, C, Minv, X, Y, 0);   /* eta_e on even sites, 0 on odd */
    ocplx *t = calloc(n, sizeof(ocplx));
    ocplx *t2 = calloc(n, sizeof(ocplx));
    for (int which = 0; which < 2; ++which) {
        ocplx *F = which ? Y : X;
        memset(t, 0, n * sizeof(ocplx));
        ora_hop(d, U, F, t, 2, which);
        if (C) site_apply(d, Minv, 1, t, t2);
        for (long x = 0; x < ora_volume(d); ++x)
            if (ora_parity(d, x) == 1)
                for (int i = 0; i < 12; ++i) F[x * 12 + i] = kappa * (C ? t2 : t)[x * 12 + i];
    }
    free(t);
    free(t2);
    free(Minv);
    return it;
}

int ora_pf_force(const int d[4], const ocplx *U, double kappa, int eo, const ocplx *phi,
                 double tol, int max_iter, double coef, double *F)
{
    long n = ora_volume(d) * 12;
    ocplx *X = calloc(n, sizeof(ocplx));
    ocplx *Y = calloc(n, sizeof(ocplx));
    int it = ora_force_vectors_c(d, U, kappa, NULL, eo, phi, tol, max_iter, X, Y);
    ora_fermion_force_xy(d, U, kappa, X, Y, coef, F);
    free(X);
    free(Y);
    return it;
}

int ora_pf_action_grad(const int d[4], const ocplx *U, double kappa, int eo,
                       const ocplx *phi, double tol, int max_iter, ocplx *G)
{
    long n = ora_volume(d) * 12;
    ocplx *X = calloc(n, sizeof(ocplx));
    ocplx *Y = calloc(n, sizeof(ocplx));
    int it = ora_force_vectors_c(d, U, kappa, NULL, eo, phi, tol, max_iter, X, Y);
    ora_fermion_grad_xy(d, kappa, X, Y, G);
    free(X);
    free(Y);
    return it;
}

/* F_a = d/de S(e^{ieT^a}U) = Re tr(G^+ i T^a U) for a real-component gradient G */
void ora_grad_to_force(const int d[4], const ocplx *U, const ocplx *G, double *F)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < 4 * V; ++l) {
        ocplx T[9], TU[9], Gd[9];
        su3_dag(&G[l * 9], Gd);
        for (int a = 0; a < 8; ++a) {
            ora_gellmann_T(a, T);
            su3_mul(T, &U[l * 9], TU);
            ocplx tr = 0;
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) tr += Gd[i * 3 + k] * I * TU[k * 3 + i];
            F[l * 8 + a] = creal(tr);
        }
    }
}
