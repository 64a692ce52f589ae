/*
 * ora_gauge.c -- Wilson plaquette action, its force and gradient, the left
 * link update of Eq. 6 / Eq. S2.1, reunitarisation, and one level of stout
 * smearing with its adjoint (the reverse step of Eq. 3 applied to the smearing
 * map).  Test infrastructure only (see oracle.h).
 */
#include "oracle.h"
#include "ora_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static const ocplx *link_at(const ocplx *U, long s, int mu) { return &U[(s * 4 + mu) * 9]; }

static double retrace(const ocplx *A) { return creal(A[0] + A[4] + A[8]); }

static void mul3(const ocplx *A, const ocplx *B, const ocplx *C, ocplx *out)
{
    ocplx t[9];
    su3_mul(A, B, t);
    su3_mul(t, C, out);
}

/* Re tr U_munu(x) with U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
static double plaquette_retr(const int d[4], const ocplx *U, long x, int mu, int nu)
{
    long xm = ora_neighbour(d, x, mu, +1), xn = ora_neighbour(d, x, nu, +1);
    ocplx a[9], b[9], c[9], d1[9], d2[9];
    su3_mul(link_at(U, x, mu), link_at(U, xm, nu), a);
    su3_dag(link_at(U, xn, mu), d1);
    su3_dag(link_at(U, x, nu), d2);
    su3_mul(a, d1, b);
    su3_mul(b, d2, c);
    return retrace(c);
}

double ora_plaquette_sum(const int d[4], const ocplx *U)
{
    long V = ora_volume(d);
    double *site = malloc(V * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        double acc = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) acc += plaquette_retr(d, U, x, mu, nu) / 3.0;
        site[x] = acc;
    }
    double sum = 0;
    for (long x = 0; x < V; ++x) sum += site[x];
    free(site);
    return sum;
}

double ora_gauge_action(const int d[4], const ocplx *U, double beta)
{
    return beta * (6.0 * ora_volume(d) - ora_plaquette_sum(d, U));
}

double ora_momentum_energy(const int d[4], const double *mom)
{
    long n = ora_volume(d) * 32;
    double s = 0;
    for (long i = 0; i < n; ++i) s += mom[i] * mom[i];
    return 0.5 * s;
}

/* staple sum V_mu(x): the plaquettes through U_mu(x) are Re tr(U_mu(x) V_mu(x)) */
static void staple(const int d[4], const ocplx *U, long x, int mu, ocplx Vs[9])
{
    for (int i = 0; i < 9; ++i) Vs[i] = 0;
    long xpm = ora_neighbour(d, x, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        long xpn = ora_neighbour(d, x, nu, +1);
        long xmn = ora_neighbour(d, x, nu, -1);
        long xpm_mn = ora_neighbour(d, xpm, nu, -1);
        ocplx a[9], b[9], c[9], t[9];
        /* U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
        su3_dag(link_at(U, xpn, mu), b);
        su3_dag(link_at(U, x, nu), c);
        mul3(link_at(U, xpm, nu), b, c, t);
        for (int i = 0; i < 9; ++i) Vs[i] += t[i];
        /* U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) */
        su3_dag(link_at(U, xpm_mn, nu), a);
        su3_dag(link_at(U, xmn, mu), b);
        mul3(a, b, link_at(U, xmn, nu), t);
        for (int i = 0; i < 9; ++i) Vs[i] += t[i];
    }
}

/* d_a S_G = (beta/3) Im tr(T^a U V), from delta Re tr(UV) = Re tr(i e T^a U V) */
void ora_gauge_force(const int d[4], const ocplx *U, double beta, double coef, double *F)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx Vs[9], UV[9], T[9];
            staple(d, U, x, mu, Vs);
            su3_mul(link_at(U, x, mu), Vs, UV);
            for (int a = 0; a < 8; ++a) {
                ora_gellmann_T(a, T);
                ocplx tr = 0;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) tr += T[i * 3 + k] * UV[k * 3 + i];
                F[(x * 4 + mu) * 8 + a] += coef * (beta / 3.0) * cimag(tr);
            }
        }
}

/* G = dS/dReU + i dS/dImU = -(beta/3) V^+, since delta S_G = -(beta/3) Re tr(V dU) */
void ora_gauge_action_grad(const int d[4], const ocplx *U, double beta, ocplx *G)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx Vs[9], Vd[9];
            staple(d, U, x, mu, Vs);
            su3_dag(Vs, Vd);
            for (int i = 0; i < 9; ++i) G[(x * 4 + mu) * 9 + i] = -(beta / 3.0) * Vd[i];
        }
}

/* ---------------- rectangle-improved gauge action ----------------
 * S_G = beta sum_x [ c0 sum_{mu<nu} (1 - Re tr P_munu(x)/3) + c1 sum_{mu!=nu} (1 - Re tr R_munu(x)/3) ],
 * c0 = 1 - 8 c1, R_munu the 2 x 1 loop with the long side along mu.  Loops are
 * written as step lists: +(mu+1) steps forward along mu with U_mu(y), -(mu+1) steps
 * back with U_mu(y-mu)^+.  The force on U_mu(x) uses every loop through that link
 * rotated to start with it: Re tr(U_mu(x) S), S the product along the rest. */
static void path_product(const int d[4], const ocplx *U, long y, const int *steps, int n, ocplx out[9])
{
    ocplx acc[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t[9], m[9];
    for (int k = 0; k < n; ++k) {
        const int mu = abs(steps[k]) - 1;
        if (steps[k] > 0) {
            su3_mul(acc, link_at(U, y, mu), t);
            y = ora_neighbour(d, y, mu, +1);
        } else {
            y = ora_neighbour(d, y, mu, -1);
            su3_dag(link_at(U, y, mu), m);
            su3_mul(acc, m, t);
        }
        memcpy(acc, t, sizeof acc);
    }
    memcpy(out, acc, sizeof acc);
}

double ora_rectangle_sum(const int d[4], const ocplx *U)
{
    long V = ora_volume(d);
    double *site = malloc(V * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        double acc = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                const int m = mu + 1, n = nu + 1;
                const int loop[6] = {m, m, n, -m, -m, -n};
                ocplx R[9];
                path_product(d, U, x, loop, 6, R);
                acc += retrace(R) / 3.0;
            }
        site[x] = acc;
    }
    double sum = 0;
    for (long x = 0; x < V; ++x) sum += site[x];
    free(site);
    return sum;
}

double ora_gauge_action_imp(const int d[4], const ocplx *U, double beta, double c1)
{
    if (c1 == 0.0) return ora_gauge_action(d, U, beta);
    const double V = (double)ora_volume(d);
    return beta * ((1.0 - 8.0 * c1) * (6.0 * V - ora_plaquette_sum(d, U)) +
                   c1 * (12.0 * V - ora_rectangle_sum(d, U)));
}

/* c0 (plaquette staples) + c1 (rectangle staples) through U_mu(x) */
static void staple_imp(const int d[4], const ocplx *U, long x, int mu, double c1, ocplx Vs[9])
{
    staple(d, U, x, mu, Vs);
    if (c1 == 0.0) return;
    const double c0 = 1.0 - 8.0 * c1;
    for (int i = 0; i < 9; ++i) Vs[i] *= c0;
    const long xp = ora_neighbour(d, x, mu, +1);
    const int m = mu + 1;
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const int n = nu + 1;
        /* the six rectangles through U_mu(x), each starting with the step +mu from x */
        const int loops[6][6] = {
            {m, m, n, -m, -m, -n},  {m, n, -m, -m, -n, m},   /* long side mu, above */
            {m, m, -n, -m, -m, n},  {m, -n, -m, -m, n, m},   /* long side mu, below */
            {m, n, n, -m, -n, -n},  {m, -n, -n, -m, n, n},   /* long side nu */
        };
        for (int k = 0; k < 6; ++k) {
            ocplx S[9];
            path_product(d, U, xp, loops[k] + 1, 5, S);
            for (int i = 0; i < 9; ++i) Vs[i] += c1 * S[i];
        }
    }
}

void ora_gauge_force_imp(const int d[4], const ocplx *U, double beta, double c1, double coef, double *F)
{
    if (c1 == 0.0) { ora_gauge_force(d, U, beta, coef, F); return; }
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx Vs[9], UV[9], T[9];
            staple_imp(d, U, x, mu, c1, Vs);
            su3_mul(link_at(U, x, mu), Vs, UV);
            for (int a = 0; a < 8; ++a) {
                ora_gellmann_T(a, T);
                ocplx tr = 0;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) tr += T[i * 3 + k] * UV[k * 3 + i];
                F[(x * 4 + mu) * 8 + a] += coef * (beta / 3.0) * cimag(tr);
            }
        }
}

void ora_gauge_action_grad_imp(const int d[4], const ocplx *U, double beta, double c1, ocplx *G)
{
    if (c1 == 0.0) { ora_gauge_action_grad(d, U, beta, G); return; }
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx Vs[9], Vd[9];
            staple_imp(d, U, x, mu, c1, Vs);
            su3_dag(Vs, Vd);
            for (int i = 0; i < 9; ++i) G[(x * 4 + mu) * 9 + i] = -(beta / 3.0) * Vd[i];
        }
}

void ora_update_links(const int d[4], ocplx *U, const double *mom, double eps)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < 4 * V; ++l) {
        ocplx P[9], E[9], out[9];
        su3_from_coeffs(&mom[l * 8], P);
        su3_expi(P, eps, E);
        su3_mul(E, &U[l * 9], out);
        memcpy(&U[l * 9], out, sizeof out);
    }
}

void ora_kick(const int d[4], double *mom, const double *F, double eps)
{
    long n = ora_volume(d) * 32;
    for (long i = 0; i < n; ++i) mom[i] -= eps * F[i];
}

void ora_reunitarise(const int d[4], ocplx *U)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < 4 * V; ++l) {
        ocplx *u = &U[l * 9];
        double n1 = 0;
        for (int k = 0; k < 3; ++k) n1 += creal(u[k] * conj(u[k]));
        n1 = sqrt(n1);
        for (int k = 0; k < 3; ++k) u[k] /= n1;
        ocplx ip = 0;
        for (int k = 0; k < 3; ++k) ip += conj(u[k]) * u[3 + k];
        for (int k = 0; k < 3; ++k) u[3 + k] -= ip * u[k];
        double n2 = 0;
        for (int k = 0; k < 3; ++k) n2 += creal(u[3 + k] * conj(u[3 + k]));
        n2 = sqrt(n2);
        for (int k = 0; k < 3; ++k) u[3 + k] /= n2;
        u[6] = conj(u[1] * u[5] - u[2] * u[4]);
        u[7] = conj(u[2] * u[3] - u[0] * u[5]);
        u[8] = conj(u[0] * u[4] - u[1] * u[3]);
    }
}

/* ---------------------------------------------------------------------------
 * Stout smearing (Morningstar & Peardon 2004, cited for the smearing of
 * Fig. 1):  C_mu(x) = rho sum_{nu != mu} [U_nu(x) U_mu(x+nu) U_nu(x+mu)^+
 *                                        + U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu)],
 * Omega = C U^+, X = i Q = traceless anti-Hermitian part of Omega (the
 * projection of Eq. 9), U' = exp(X) U.
 * ------------------------------------------------------------------------- */
static void stout_C(const int d[4], const ocplx *U, double rho, long x, int mu, ocplx C[9])
{
    for (int i = 0; i < 9; ++i) C[i] = 0;
    long xpm = ora_neighbour(d, x, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        long xpn = ora_neighbour(d, x, nu, +1);
        long xmn = ora_neighbour(d, x, nu, -1);
        long xmn_pm = ora_neighbour(d, xmn, mu, +1);
        ocplx a[9], c[9], t[9];
        su3_dag(link_at(U, xpm, nu), c);
        mul3(link_at(U, x, nu), link_at(U, xpn, mu), c, t);
        for (int i = 0; i < 9; ++i) C[i] += rho * t[i];
        su3_dag(link_at(U, xmn, nu), a);
        mul3(a, link_at(U, xmn, mu), link_at(U, xmn_pm, nu), t);
        for (int i = 0; i < 9; ++i) C[i] += rho * t[i];
    }
}

/* projection of Eq. 9: P[A] = (A - A^+)/2 - tr(A - A^+)/(2N) */
static void proj_ta(const ocplx *A, ocplx *out)
{
    ocplx tr = 0;
    for (int i = 0; i < 3; ++i) tr += A[i * 4] - conj(A[i * 4]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            out[i * 3 + j] = 0.5 * (A[i * 3 + j] - conj(A[j * 3 + i])) - (i == j ? tr / 6.0 : 0);
}

static void stout_link(const int d[4], const ocplx *U, double rho, long x, int mu, ocplx C[9],
                       ocplx X[9], ocplx E[9])
{
    ocplx Ud[9], Om[9];
    stout_C(d, U, rho, x, mu, C);
    su3_dag(link_at(U, x, mu), Ud);
    su3_mul(C, Ud, Om);
    proj_ta(Om, X);
    ora_expm(3, X, E);
}

void ora_stout_forward(const int d[4], const ocplx *U, double rho, ocplx *Uout)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            ocplx C[9], X[9], E[9];
            stout_link(d, U, rho, x, mu, C, X, E);
            su3_mul(E, link_at(U, x, mu), &Uout[(x * 4 + mu) * 9]);
        }
}

/* Adjoint of one stout level.  With <A,B> = Re tr(A^+ B), a gradient G of L
 * w.r.t. M means delta L = <G, delta M>.  Going backwards:
 *   U' = E U          -> G_E = G' U^+,  G_U += E^+ G'
 *   E = exp(X)        -> G_X = L_{X^+}(G_E), the adjoint Frechet derivative, taken
 *                        from exp([[X^+, G_E], [0, X^+]]) (top-right block)
 *   X = P[Omega]      -> G_Omega = P[G_X]   (P is an orthogonal projection)
 *   Omega = C U^+     -> G_C = G_Omega U,  G_U += G_Omega^+ C
 *   C = rho sum ABC   -> product rule on each staple, with G_{W^+} = (G_W)^+.   */
void ora_stout_backward(const int d[4], const ocplx *U, double rho, const ocplx *Gout,
                        ocplx *Gin)
{
    long V = ora_volume(d);
    ocplx *GC = malloc(sizeof(ocplx) * 9 * 4 * V);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            long l = x * 4 + mu;
            ocplx C[9], X[9], E[9], Ud[9], Ed[9], GE[9], GX[9], GO[9], GOd[9], t1[9], t2[9];
            ocplx M[36], EM[36];
            stout_link(d, U, rho, x, mu, C, X, E);
            su3_dag(link_at(U, x, mu), Ud);
            su3_dag(E, Ed);
            su3_mul(&Gout[l * 9], Ud, GE);
            for (int i = 0; i < 36; ++i) M[i] = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    M[i * 6 + j] = conj(X[j * 3 + i]);
                    M[(i + 3) * 6 + (j + 3)] = conj(X[j * 3 + i]);
                    M[i * 6 + (j + 3)] = GE[i * 3 + j];
                }
            ora_expm(6, M, EM);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) GX[i * 3 + j] = EM[i * 6 + (j + 3)];
            proj_ta(GX, GO);
            su3_mul(GO, link_at(U, x, mu), &GC[l * 9]);
            su3_mul(Ed, &Gout[l * 9], t1);
            su3_dag(GO, GOd);
            su3_mul(GOd, C, t2);
            for (int i = 0; i < 9; ++i) Gin[l * 9 + i] = t1[i] + t2[i];
        }
    /* staple adjoints, scattered serially */
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            const ocplx *G = &GC[(x * 4 + mu) * 9];
            ocplx Gd[9];
            su3_dag(G, Gd);
            long xpm = ora_neighbour(d, x, mu, +1);
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                long xpn = ora_neighbour(d, x, nu, +1);
                long xmn = ora_neighbour(d, x, nu, -1);
                long xmn_pm = ora_neighbour(d, xmn, mu, +1);
                ocplx A[9], B[9], Cc[9], BC[9], AB[9], BCd[9], ABd[9], Ad[9], Ccd[9], t[9], t2[9];
                /* staple 1: A = U_nu(x), B = U_mu(x+nu), C = U_nu(x+mu)^+ */
                memcpy(A, link_at(U, x, nu), sizeof A);
                memcpy(B, link_at(U, xpn, mu), sizeof B);
                su3_dag(link_at(U, xpm, nu), Cc);
                su3_mul(B, Cc, BC);
                su3_mul(A, B, AB);
                su3_dag(BC, BCd);
                su3_mul(G, BCd, t);                              /* G_A = G (BC)^+ */
                for (int i = 0; i < 9; ++i) Gin[(x * 4 + nu) * 9 + i] += rho * t[i];
                su3_dag(A, Ad);
                su3_dag(Cc, Ccd);
                mul3(Ad, G, Ccd, t);                             /* G_B = A^+ G C^+ */
                for (int i = 0; i < 9; ++i) Gin[(xpn * 4 + mu) * 9 + i] += rho * t[i];
                su3_mul(Gd, AB, t);                              /* G_W = (AB)^+ G)^+ */
                for (int i = 0; i < 9; ++i) Gin[(xpm * 4 + nu) * 9 + i] += rho * t[i];
                /* staple 2: A = U_nu(x-nu)^+, B = U_mu(x-nu), C = U_nu(x-nu+mu) */
                su3_dag(link_at(U, xmn, nu), A);
                memcpy(B, link_at(U, xmn, mu), sizeof B);
                memcpy(Cc, link_at(U, xmn_pm, nu), sizeof Cc);
                su3_mul(B, Cc, BC);
                su3_mul(A, B, AB);
                su3_mul(BC, Gd, t);                              /* G_W = (G (BC)^+)^+ */
                for (int i = 0; i < 9; ++i) Gin[(xmn * 4 + nu) * 9 + i] += rho * t[i];
                su3_dag(A, Ad);
                su3_dag(Cc, Ccd);
                mul3(Ad, G, Ccd, t);                             /* G_B = A^+ G C^+ */
                for (int i = 0; i < 9; ++i) Gin[(xmn * 4 + mu) * 9 + i] += rho * t[i];
                su3_dag(AB, ABd);
                su3_mul(ABd, G, t2);                             /* G_C = (AB)^+ G */
                for (int i = 0; i < 9; ++i) Gin[(xmn_pm * 4 + nu) * 9 + i] += rho * t2[i];
            }
        }
    free(GC);
}
