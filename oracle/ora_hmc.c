/*
 * ora_hmc.c -- molecular dynamics and one HMC trajectory with the left update
 * of Eq. S2.1 / S2.2, leapfrog (PQP) or Omelyan 2MN, Metropolis on Delta H.
 * Test infrastructure only (see oracle.h).
 */
#include "oracle.h"
#include "ora_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

int ora_md_force(const int d[4], const ocplx *U, const ora_hmc_params *p, const ocplx *phi,
                 double *F)
{
    long n = ora_volume(d) * 32;
    memset(F, 0, n * sizeof(double));
    ora_gauge_force(d, U, p->beta, 1.0, F);
    if (!p->fermions) return 0;
    int it = ora_pf_force(d, U, p->kappa, p->eo, phi, p->tol_md, p->max_iter, 1.0, F);
    return it < 0 ? -it : it;
}

static int kick(const int d[4], const ocplx *U, double *mom, const ocplx *phi,
                const ora_hmc_params *p, double eps, double *F, int *evals)
{
    int it = ora_md_force(d, U, p, phi, F);
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
        iters += kick(d, U, mom, phi, p, 0.5 * eps, F, evals);
        for (int i = 0; i < p->n_steps; ++i) {
            ora_update_links(d, U, mom, eps);
            iters += kick(d, U, mom, phi, p, (i + 1 < p->n_steps) ? eps : 0.5 * eps, F, evals);
        }
    } else {
        const double lam = 0.1931833275037836;
        iters += kick(d, U, mom, phi, p, lam * eps, F, evals);
        for (int i = 0; i < p->n_steps; ++i) {
            ora_update_links(d, U, mom, 0.5 * eps);
            iters += kick(d, U, mom, phi, p, (1.0 - 2.0 * lam) * eps, F, evals);
            ora_update_links(d, U, mom, 0.5 * eps);
            iters += kick(d, U, mom, phi, p, (i + 1 < p->n_steps) ? 2.0 * lam * eps : lam * eps,
                          F, evals);
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
    res->Sg_old = ora_gauge_action(d, U, p->beta);
    if (p->fermions) {
        int mask = p->eo ? 1 : 3;
        ora_gaussian_spinor(d, seed, traj, ORA_FIELD_XI, mask, xi);
        /* phi = M^+ xi, so S_f(old) = xi^+ xi exactly */
        if (p->eo) ora_dhat(d, U, p->kappa, xi, phi, 1);
        else ora_dirac(d, U, p->kappa, xi, phi, 1);
        res->Sf_old = ora_norm2(d, xi, mask);
    }
    int evals = 0;
    res->cg_iters = integrate(d, U, mom, phi, p, &evals);
    res->force_evals = evals;
    res->K_new = ora_momentum_energy(d, mom);
    res->Sg_new = ora_gauge_action(d, U, p->beta);
    if (p->fermions) {
        int it = 0;
        res->Sf_new = ora_pf_action(d, U, p->kappa, p->eo, phi, p->tol_action, p->max_iter, &it);
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
