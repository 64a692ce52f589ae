/*
 * ora_hmc.c -- molecular dynamics and one HMC trajectory with the left update
 * of Eq. S2.1 / S2.2: leapfrog (PQP), Omelyan 2MN, or a Sexton-Weingarten
 * nested leapfrog (gauge force on the inner time scale), Metropolis on Delta H.
 * The pseudofermion operator may carry the clover term (csw; full lattice or even-odd,
 * the even-odd action with its -2 ln det M_oo).
 * With stout smearing the pseudofermion action sees the smeared links and its
 * force is taken back through every level (the reverse recursion of Eq. 3);
 * the gauge action sees the thin links.
 * Test infrastructure only (see oracle.h).
 */
#include "oracle.h"
#include "ora_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* levels[0] = U, levels[k] = stout(levels[k-1]); caller frees levels[1..n] */
static ocplx **smear_levels(const int d[4], const ocplx *U, int n, double rho)
{
    long V = ora_volume(d);
    ocplx **lv = malloc(sizeof(ocplx *) * (n + 1));
    lv[0] = (ocplx *)U;
    for (int k = 1; k <= n; ++k) {
        lv[k] = malloc(sizeof(ocplx) * 36 * V);
        ora_stout_forward(d, lv[k - 1], rho, lv[k]);
    }
    return lv;
}

static void free_levels(ocplx **lv, int n)
{
    for (int k = 1; k <= n; ++k) free(lv[k]);
    free(lv);
}

int ora_md_force_part(const int d[4], const ocplx *U, const ora_hmc_params *p, const ocplx *phi,
                      int part, double *F)
{
    long V = ora_volume(d);
    memset(F, 0, V * 32 * sizeof(double));
    if (part != 2 && p->beta != 0.0) ora_gauge_force_imp(d, U, p->beta, p->c1, 1.0, F);
    if (part == 1 || !p->fermions) return 0;
    int it;
    if (p->n_stout == 0 && p->csw == 0.0) {
        it = ora_pf_force(d, U, p->kappa, p->eo, phi, p->tol_md, p->max_iter, 1.0, F);
    } else if (p->n_stout == 0) {
        it = p->eo ? ora_pf_force_sw_eo(d, U, p->kappa, p->csw, phi, p->tol_md, p->max_iter, 1.0, F)
                   : ora_pf_force_sw(d, U, p->kappa, p->csw, phi, p->tol_md, p->max_iter, 1.0, F);
    } else {
        ocplx **lv = smear_levels(d, U, p->n_stout, p->rho);
        ocplx *G = malloc(sizeof(ocplx) * 36 * V);
        ocplx *G2 = malloc(sizeof(ocplx) * 36 * V);
        double *Ff = malloc(sizeof(double) * 32 * V);
        if (p->csw == 0.0)
            it = ora_pf_action_grad(d, lv[p->n_stout], p->kappa, p->eo, phi, p->tol_md, p->max_iter, G);
        else if (p->eo)
            it = ora_pf_action_grad_sw_eo(d, lv[p->n_stout], p->kappa, p->csw, phi, p->tol_md, p->max_iter, G);
        else
            it = ora_pf_action_grad_sw(d, lv[p->n_stout], p->kappa, p->csw, phi, p->tol_md, p->max_iter, G);
        for (int k = p->n_stout; k >= 1; --k) {
            ora_stout_backward(d, lv[k - 1], p->rho, G, G2);
            ocplx *t = G; G = G2; G2 = t;
        }
        ora_grad_to_force(d, U, G, Ff);
        for (long i = 0; i < V * 32; ++i) F[i] += Ff[i];
        free(G); free(G2); free(Ff);
        free_levels(lv, p->n_stout);
    }
    return it < 0 ? -it : it;
}

int ora_md_force(const int d[4], const ocplx *U, const ora_hmc_params *p, const ocplx *phi,
                 double *F)
{
    return ora_md_force_part(d, U, p, phi, 0, F);
}

static double pf_action_smeared(const int d[4], const ocplx *U, const ora_hmc_params *p,
                                const ocplx *phi, int *it)
{
    ocplx **lv = smear_levels(d, U, p->n_stout, p->rho);
    double S = (p->csw == 0.0)
                   ? ora_pf_action(d, lv[p->n_stout], p->kappa, p->eo, phi, p->tol_action, p->max_iter, it)
               : p->eo ? ora_pf_action_sw_eo(d, lv[p->n_stout], p->kappa, p->csw, phi, p->tol_action, p->max_iter, it)
                       : ora_pf_action_sw(d, lv[p->n_stout], p->kappa, p->csw, phi, p->tol_action, p->max_iter, it);
    free_levels(lv, p->n_stout);
    return S;
}

double ora_hamiltonian(const int d[4], const ocplx *U, const double *mom, const ocplx *phi,
                       const ora_hmc_params *p)
{
    int it;
    double H = ora_momentum_energy(d, mom) + ora_gauge_action_imp(d, U, p->beta, p->c1);
    if (p->fermions) H += pf_action_smeared(d, U, p, phi, &it);
    return H;
}

static int kick(const int d[4], const ocplx *U, double *mom, const ocplx *phi,
                const ora_hmc_params *p, double eps, int part, double *F, int *evals)
{
    int it = ora_md_force_part(d, U, p, phi, part, F);
    ora_kick(d, mom, F, eps);
    ++*evals;
    return it;
}

static int integrate(const int d[4], ocplx *U, double *mom, const ocplx *phi,
                     const ora_hmc_params *p, int *evals)
{
    long n = ora_volume(d) * 32;
    double *F = malloc(n * sizeof(double));
    double eps = p->tau / p->n_steps;
    int iters = 0;
    if (p->integrator == 0) {
        iters += kick(d, U, mom, phi, p, 0.5 * eps, 0, F, evals);
        for (int i = 0; i < p->n_steps; ++i) {
            ora_update_links(d, U, mom, eps);
            iters += kick(d, U, mom, phi, p, (i + 1 < p->n_steps) ? eps : 0.5 * eps, 0, F, evals);
        }
    } else if (p->integrator == 1) {
        // the second-order minimum-norm (2MN) position-velocity-position integrator of
        // Omelyan, Mryglod and Folk, Comput. Phys. Commun. 151 (2003) 272, Eq. (31):
        // lambda = 0.1931833275037836 minimises the norm of its leading error term
        const double lam = 0.1931833275037836;
        iters += kick(d, U, mom, phi, p, lam * eps, 0, F, evals);
        for (int i = 0; i < p->n_steps; ++i) {
            ora_update_links(d, U, mom, 0.5 * eps);
            iters += kick(d, U, mom, phi, p, (1.0 - 2.0 * lam) * eps, 0, F, evals);
            ora_update_links(d, U, mom, 0.5 * eps);
            iters += kick(d, U, mom, phi, p, (i + 1 < p->n_steps) ? 2.0 * lam * eps : lam * eps,
                          0, F, evals);
        }
    } else {
        /* Sexton-Weingarten: outer leapfrog with the fermion force; every outer
         * step runs n_inner leapfrog steps of the gauge force */
        const int m = p->n_inner > 0 ? p->n_inner : 1;
        const double ein = eps / m;
        iters += kick(d, U, mom, phi, p, 0.5 * eps, 2, F, evals);
        for (int i = 0; i < p->n_steps; ++i) {
            kick(d, U, mom, phi, p, 0.5 * ein, 1, F, evals);
            for (int j = 0; j < m; ++j) {
                ora_update_links(d, U, mom, ein);
                kick(d, U, mom, phi, p, (j + 1 < m) ? ein : 0.5 * ein, 1, F, evals);
            }
            iters += kick(d, U, mom, phi, p, (i + 1 < p->n_steps) ? eps : 0.5 * eps, 2, F, evals);
        }
    }
    free(F);
    return iters;
}

int ora_md_integrate(const int d[4], ocplx *U, double *mom, const ocplx *phi,
                     const ora_hmc_params *p)
{
    int evals = 0;
    return integrate(d, U, mom, phi, p, &evals);
}

int ora_hmc_trajectory(const int d[4], ocplx *U, const ora_hmc_params *p, uint64_t seed,
                       uint32_t traj, ora_hmc_result *res)
{
    long V = ora_volume(d);
    double *mom = malloc(V * 32 * sizeof(double));
    ocplx *U0 = malloc(V * 36 * sizeof(ocplx));
    ocplx *xi = calloc(V * 12, sizeof(ocplx));
    ocplx *phi = calloc(V * 12, sizeof(ocplx));
    memcpy(U0, U, V * 36 * sizeof(ocplx));
    memset(res, 0, sizeof *res);

    ora_gaussian_momenta(d, seed, traj, mom);
    res->K_old = ora_momentum_energy(d, mom);
    res->Sg_old = ora_gauge_action_imp(d, U, p->beta, p->c1);
    if (p->fermions) {
        int mask = p->eo ? 1 : 3;
        ora_gaussian_spinor(d, seed, traj, ORA_FIELD_XI, mask, xi);
        /* phi = M^+ xi on the links the pseudofermion action sees: S_f(old) = xi^+ xi */
        ocplx **lv = smear_levels(d, U, p->n_stout, p->rho);
        if (p->eo) ora_dhat_sw(d, lv[p->n_stout], p->kappa, p->csw, xi, phi, 1);
        else ora_dirac_sw(d, lv[p->n_stout], p->kappa, p->csw, xi, phi, 1);
        res->Sf_old = ora_norm2(d, xi, mask);
        /* the even-odd clover action also holds -2 ln det M_oo */
        if (p->eo && p->csw != 0.0) res->Sf_old -= 2.0 * ora_clover_logdet_odd(d, lv[p->n_stout], p->kappa, p->csw);
        free_levels(lv, p->n_stout);
    }
    int evals = 0;
    res->cg_iters = integrate(d, U, mom, phi, p, &evals);
    res->force_evals = evals;
    res->K_new = ora_momentum_energy(d, mom);
    res->Sg_new = ora_gauge_action_imp(d, U, p->beta, p->c1);
    if (p->fermions) {
        int it = 0;
        res->Sf_new = pf_action_smeared(d, U, p, phi, &it);
        res->cg_iters += it < 0 ? -it : it;
    }
    res->dH = (res->K_new + res->Sg_new + res->Sf_new) - (res->K_old + res->Sg_old + res->Sf_old);
    double u = ora_uniform(seed, 0, 0, traj, ORA_FIELD_METROPOLIS);
    res->accepted = (u < exp(-res->dH));
    if (!res->accepted) memcpy(U, U0, V * 36 * sizeof(ocplx));
    ora_reunitarise(d, U);
    res->plaquette = ora_plaquette_sum(d, U) / (6.0 * V);
    free(mom); free(U0); free(xi); free(phi);
    return 0;
}
