/*
 * ora_clover.c -- the clover (Sheikholeslami-Wohlert) term of the Wilson-Dirac
 * operator, named by the paper as a further discretisation (Sec. IV) without a
 * formula.  Reading (one of the standard conventions):
 *   D_sw = 1 - kappa H + A,   A(x) = -kappa c_sw sum_{mu<nu} sigma_munu (x) F_munu(x),
 *   sigma_munu = (i/2) [g_mu, g_nu],   F_munu(x) = (Q_munu(x) - Q_munu(x)^+) / (8 i),
 *   Q_munu(x) = the four plaquettes ("leaves") of the mu-nu plane at x, each
 *   traversed mu before nu and starting and ending at x.
 * A is Hermitian, so D_sw^+ = 1 - kappa H^+ + A and gamma_5 D_sw gamma_5 = D_sw^+.
 * The full-lattice and the even-odd pseudofermion actions are covered (the even-odd
 * one with the odd-site determinant, see below).
 *
 * Force: with chi = (D^+D)^{-1} phi and eta = D chi, delta S_f = -2 Re eta^+ (delta D) chi,
 * whose clover part is 2 kappa c_sw Re sum_{x,mu<nu} tr(delta F_munu Lambda_munu) with
 * Lambda_munu(x) = sum_{s,s'} (sigma_munu)_{s s'} chi_{s'}(x) eta_s(x)^+ (a 3x3 colour
 * matrix); with Xi = Lambda + Lambda^+ this is sum Re tr(M delta Q_munu), M = -i kappa
 * c_sw Xi / 4.  The real-component gradient of Re tr(M L_1 ... L_4) with respect to
 * the link W of factor L_k is N^+ (L_k = W) or N (L_k = W^+), N = L_{k+1}..L_4 M L_1..L_{k-1};
 * it is scattered here leaf by leaf (the library gathers it link by link).
 * Test infrastructure only (see oracle.h).
 */
#include "oracle.h"
#include "ora_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const ocplx *link_at(const ocplx *U, long s, int mu) { return &U[(s * 4 + mu) * 9]; }

/* the four leaves of the (mu, nu) plane as steps from x: +d forward along U_d(y),
 * -d backward along U_d(y - d)^+ (d = direction + 1) */
static void leaf_steps(int mu, int nu, int leaf, int steps[4])
{
    const int m = mu + 1, n = nu + 1;
    const int L[4][4] = {{m, n, -m, -n}, {n, -m, -n, m}, {-m, -n, m, n}, {-n, m, n, -m}};
    memcpy(steps, L[leaf], sizeof(int) * 4);
}

/* factor k of a leaf: link index (site*4 + dir) and whether it enters as W^+ */
static void leaf_links(const int d[4], long x, const int steps[4], long link[4], int dag[4])
{
    long y = x;
    for (int k = 0; k < 4; ++k) {
        const int dir = abs(steps[k]) - 1;
        if (steps[k] > 0) {
            link[k] = y * 4 + dir;
            dag[k] = 0;
            y = ora_neighbour(d, y, dir, +1);
        } else {
            y = ora_neighbour(d, y, dir, -1);
            link[k] = y * 4 + dir;
            dag[k] = 1;
        }
    }
}

static void factor(const ocplx *U, long link, int dag, ocplx out[9])
{
    if (dag) su3_dag(&U[link * 9], out);
    else memcpy(out, &U[link * 9], sizeof(ocplx) * 9);
}

/* F_munu(x), Hermitian */
static void field_strength(const int d[4], const ocplx *U, long x, int mu, int nu, ocplx F[9])
{
    ocplx Q[9] = {0};
    for (int leaf = 0; leaf < 4; ++leaf) {
        int steps[4], dag[4];
        long link[4];
        leaf_steps(mu, nu, leaf, steps);
        leaf_links(d, x, steps, link, dag);
        ocplx acc[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, f[9], t[9];
        for (int k = 0; k < 4; ++k) {
            factor(U, link[k], dag[k], f);
            su3_mul(acc, f, t);
            memcpy(acc, t, sizeof acc);
        }
        for (int i = 0; i < 9; ++i) Q[i] += acc[i];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i * 3 + j] = (Q[i * 3 + j] - conj(Q[j * 3 + i])) / (8.0 * I);
}

void ora_clover_field_strength(const int d[4], const ocplx *U, int mu, int nu, ocplx *F)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) field_strength(d, U, x, mu, nu, &F[x * 9]);
}

/* sigma_munu = (i/2)(g_mu g_nu - g_nu g_mu), 4 x 4 */
static void sigma(int mu, int nu, ocplx s[16])
{
    ocplx gm[16], gn[16];
    ora_gamma(mu, gm);
    ora_gamma(nu, gn);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            ocplx acc = 0;
            for (int c = 0; c < 4; ++c) acc += gm[a * 4 + c] * gn[c * 4 + b] - gn[a * 4 + c] * gm[c * 4 + b];
            s[a * 4 + b] = 0.5 * I * acc;
        }
}

void ora_clover_term(const int d[4], const ocplx *U, double kappa, double csw, ocplx *A)
{
    long V = ora_volume(d);
    ocplx sg[6][16];
    int pm[6], pn[6], np = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) { sigma(mu, nu, sg[np]); pm[np] = mu; pn[np] = nu; ++np; }
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        ocplx *Ax = &A[x * 144];
        for (int i = 0; i < 144; ++i) Ax[i] = 0;
        for (int p = 0; p < 6; ++p) {
            ocplx F[9];
            field_strength(d, U, x, pm[p], pn[p], F);
            for (int s = 0; s < 4; ++s)
                for (int a = 0; a < 3; ++a)
                    for (int t = 0; t < 4; ++t)
                        for (int b = 0; b < 3; ++b)
                            Ax[(s * 3 + a) * 12 + t * 3 + b] += -kappa * csw * sg[p][s * 4 + t] * F[a * 3 + b];
        }
    }
}

/* inverse of a 12x12 complex matrix by Gauss-Jordan elimination with partial pivoting;
 * returns ln |det| (the sum of ln |pivot|) */
static double inv12(const ocplx *Min, ocplx *Mout)
{
    ocplx a[12][24];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 24; ++j) a[i][j] = j < 12 ? Min[i * 12 + j] : (j - 12 == i ? 1.0 : 0.0);
    double logdet = 0.0;
    for (int c = 0; c < 12; ++c) {
        int piv = c;
        for (int r = c + 1; r < 12; ++r)
            if (cabs(a[r][c]) > cabs(a[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 24; ++j) { ocplx t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t; }
        const ocplx pv = a[c][c];
        logdet += log(cabs(pv));
        for (int j = 0; j < 24; ++j) a[c][j] /= pv;
        for (int r = 0; r < 12; ++r) {
            if (r == c) continue;
            const ocplx f = a[r][c];
            if (f == 0) continue;
            for (int j = 0; j < 24; ++j) a[r][j] -= f * a[c][j];
        }
    }
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) Mout[i * 12 + j] = a[i][12 + j];
    return logdet;
}

/* M = 1 + C is Hermitian positive definite for the couplings used (det M > 0, so ln det
 * M = ln |det M|) */
double ora_clover_inverse_odd(const int d[4], const ocplx *C, ocplx *Minv)
{
    long V = ora_volume(d);
    double sum = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sum)
    for (long x = 0; x < V; ++x) {
        if (ora_parity(d, x) != 1) continue;
        ocplx M[144];
        for (int i = 0; i < 144; ++i) M[i] = C[x * 144 + i] + ((i / 12 == i % 12) ? 1.0 : 0.0);
        sum += inv12(M, &Minv[x * 144]);
    }
    return sum;
}

static ocplx *clover_or_null(const int d[4], const ocplx *U, double kappa, double csw)
{
    if (csw == 0.0) return NULL;
    ocplx *A = malloc(sizeof(ocplx) * 144 * ora_volume(d));
    ora_clover_term(d, U, kappa, csw, A);
    return A;
}

void ora_dirac_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *in, ocplx *out,
                  int dagger)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    ora_dirac_c(d, U, kappa, A, in, out, dagger);
    free(A);
}

int ora_cg_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *b, ocplx *x, double tol,
              int max_iter, double *true_res)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    int it = ora_cg_c(d, U, kappa, A, 0, b, x, tol, max_iter, true_res);
    free(A);
    return it;
}

double ora_pf_action_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi, double tol,
                        int max_iter, int *iters)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    double S = ora_pf_action_c(d, U, kappa, A, 0, phi, tol, max_iter, iters);
    free(A);
    return S;
}

/* clover part of the real-component gradient, added to G (serial scatter).  With Minv
 * (even-odd action) the gradient of -2 ln det M_oo is added on odd sites: its variation
 * -2 tr(M^{-1} delta A) has the same form as -2 Re eta^+ delta A chi with the spin-colour
 * matrix chi eta^+ replaced by M^{-1}, so it enters Lambda as
 * sum_{s,t} sigma_{st} (M^{-1})_{(t a),(s b)}. */
static void clover_grad_add(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *X,
                            const ocplx *Y, const ocplx *Minv, ocplx *G)
{
    long V = ora_volume(d);
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                ocplx sg[16], Lam[9] = {0}, M[9];
                sigma(mu, nu, sg);
                /* Lambda_ab = sum_{s,s'} sigma_{s s'} X_{s' a} conj(Y_{s b}) */
                for (int s = 0; s < 4; ++s)
                    for (int t = 0; t < 4; ++t) {
                        if (sg[s * 4 + t] == 0) continue;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                Lam[a * 3 + b] += sg[s * 4 + t] * X[x * 12 + t * 3 + a] * conj(Y[x * 12 + s * 3 + b]);
                                if (Minv && ora_parity(d, x) == 1)
                                    Lam[a * 3 + b] += sg[s * 4 + t] * Minv[x * 144 + (t * 3 + a) * 12 + s * 3 + b];
                            }
                    }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        M[a * 3 + b] = -I * kappa * csw / 4.0 * (Lam[a * 3 + b] + conj(Lam[b * 3 + a]));
                for (int leaf = 0; leaf < 4; ++leaf) {
                    int steps[4], dag[4];
                    long link[4];
                    leaf_steps(mu, nu, leaf, steps);
                    leaf_links(d, x, steps, link, dag);
                    ocplx f[4][9];
                    for (int k = 0; k < 4; ++k) factor(U, link[k], dag[k], f[k]);
                    for (int k = 0; k < 4; ++k) {
                        /* N = L_{k+1} .. L_4 M L_1 .. L_{k-1} */
                        ocplx N[9], t[9];
                        memcpy(N, (ocplx[9]){1, 0, 0, 0, 1, 0, 0, 0, 1}, sizeof N);
                        for (int j = k + 1; j < 4; ++j) { su3_mul(N, f[j], t); memcpy(N, t, sizeof N); }
                        su3_mul(N, M, t);
                        memcpy(N, t, sizeof N);
                        for (int j = 0; j < k; ++j) { su3_mul(N, f[j], t); memcpy(N, t, sizeof N); }
                        ocplx *g = &G[link[k] * 9];
                        if (dag[k]) {
                            for (int i = 0; i < 9; ++i) g[i] += N[i];
                        } else {
                            for (int i = 0; i < 3; ++i)
                                for (int j = 0; j < 3; ++j) g[i * 3 + j] += conj(N[j * 3 + i]);
                        }
                    }
                }
            }
}

int ora_pf_action_grad_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi,
                          double tol, int max_iter, ocplx *G)
{
    long n = ora_volume(d) * 12;
    ocplx *A = clover_or_null(d, U, kappa, csw);
    ocplx *X = calloc(n, sizeof(ocplx));
    ocplx *Y = calloc(n, sizeof(ocplx));
    int it = ora_force_vectors_c(d, U, kappa, A, 0, phi, tol, max_iter, X, Y);
    ora_fermion_grad_xy(d, kappa, X, Y, G);
    if (csw != 0.0) clover_grad_add(d, U, kappa, csw, X, Y, NULL, G);
    free(A);
    free(X);
    free(Y);
    return it;
}

/* ---- even-odd preconditioned clover operator:
 *   Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe,  M = 1 + A,
 *   S_f = phi_e^+ (Dhat^+ Dhat)^{-1} phi_e - 2 ln det M_oo
 * (det D = det M_oo det Dhat, so det(D^+ D) = det(M_oo)^2 det(Dhat^+ Dhat)). */
void ora_dhat_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *in, ocplx *out,
                 int dagger)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    ocplx *Minv = NULL;
    if (A) {
        Minv = calloc(144 * ora_volume(d), sizeof(ocplx));
        ora_clover_inverse_odd(d, A, Minv);
    }
    ora_dhat_c(d, U, kappa, A, Minv, in, out, dagger);
    free(A);
    free(Minv);
}

double ora_clover_logdet_odd(const int d[4], const ocplx *U, double kappa, double csw)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    if (!A) return 0.0;
    ocplx *Minv = calloc(144 * ora_volume(d), sizeof(ocplx));
    double s = ora_clover_inverse_odd(d, A, Minv);
    free(A);
    free(Minv);
    return s;
}

int ora_cg_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *b, ocplx *x, double tol,
                 int max_iter, double *true_res)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    int it = ora_cg_c(d, U, kappa, A, 1, b, x, tol, max_iter, true_res);
    free(A);
    return it;
}

double ora_pf_action_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi,
                           double tol, int max_iter, int *iters)
{
    ocplx *A = clover_or_null(d, U, kappa, csw);
    double S = ora_pf_action_c(d, U, kappa, A, 1, phi, tol, max_iter, iters);
    free(A);
    return S;
}

int ora_pf_action_grad_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi,
                             double tol, int max_iter, ocplx *G)
{
    long n = ora_volume(d) * 12;
    ocplx *A = clover_or_null(d, U, kappa, csw);
    ocplx *X = calloc(n, sizeof(ocplx));
    ocplx *Y = calloc(n, sizeof(ocplx));
    int it = ora_force_vectors_c(d, U, kappa, A, 1, phi, tol, max_iter, X, Y);
    ora_fermion_grad_xy(d, kappa, X, Y, G);
    if (A) {
        ocplx *Minv = calloc(n * 12, sizeof(ocplx));
        ora_clover_inverse_odd(d, A, Minv);
        clover_grad_add(d, U, kappa, csw, X, Y, Minv, G);
        free(Minv);
    }
    free(A);
    free(X);
    free(Y);
    return it;
}

int ora_pf_force_sw_eo(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi, double tol,
                       int max_iter, double coef, double *F)
{
    long V = ora_volume(d);
    ocplx *G = calloc(36 * V, sizeof(ocplx));
    double *Fl = calloc(32 * V, sizeof(double));
    int it = ora_pf_action_grad_sw_eo(d, U, kappa, csw, phi, tol, max_iter, G);
    ora_grad_to_force(d, U, G, Fl);
    for (long i = 0; i < 32 * V; ++i) F[i] += coef * Fl[i];
    free(G);
    free(Fl);
    return it;
}

int ora_pf_force_sw(const int d[4], const ocplx *U, double kappa, double csw, const ocplx *phi, double tol,
                    int max_iter, double coef, double *F)
{
    long V = ora_volume(d);
    ocplx *G = calloc(36 * V, sizeof(ocplx));
    double *Fl = calloc(32 * V, sizeof(double));
    int it = ora_pf_action_grad_sw(d, U, kappa, csw, phi, tol, max_iter, G);
    ora_grad_to_force(d, U, G, Fl);
    for (long i = 0; i < 32 * V; ++i) F[i] += coef * Fl[i];
    free(G);
    free(Fl);
    return it;
}
