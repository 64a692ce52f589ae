/*
 * ora_core.c -- geometry, counter-based random numbers, small matrices, seeded
 * fields.  Test infrastructure only (see oracle.h).
 */
#include "oracle.h"
#include "ora_internal.h"
#include <math.h>
#include <string.h>
#include <stdlib.h>

long ora_volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

void ora_coords(const int d[4], long s, int x[4])
{
    x[0] = (int)(s % d[0]); s /= d[0];
    x[1] = (int)(s % d[1]); s /= d[1];
    x[2] = (int)(s % d[2]); s /= d[2];
    x[3] = (int)s;
}

long ora_index(const int d[4], const int x[4])
{
    return x[0] + (long)d[0] * (x[1] + (long)d[1] * (x[2] + (long)d[2] * x[3]));
}

int ora_parity(const int d[4], long s)
{
    int x[4];
    ora_coords(d, s, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* neighbour of s one step along mu in direction dir (+1 / -1), periodic */
long ora_neighbour(const int d[4], long s, int mu, int dir)
{
    int x[4];
    ora_coords(d, s, x);
    x[mu] = (x[mu] + dir + d[mu]) % d[mu];
    return ora_index(d, x);
}

/* fermion boundary factor of the hop s -> s + dir*mu: -1 when it wraps in time */
double ora_fermion_bc(const int d[4], long s, int mu, int dir)
{
    int x[4];
    if (mu != 3) return 1.0;
    ora_coords(d, s, x);
    if (dir > 0 && x[3] == d[3] - 1) return -1.0;
    if (dir < 0 && x[3] == 0) return -1.0;
    return 1.0;
}

/* ---------------------------------------------------------------------------
 * Philox-4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 * (hi,lo) = M*c products on words 0 and 2 with a Weyl-sequence key schedule.
 * ------------------------------------------------------------------------- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in the open interval (0,1) from two 32-bit words */
static double u53(uint32_t a, uint32_t b)
{
    double hi = (double)(a >> 5);   /* 27 bits */
    double lo = (double)(b >> 6);   /* 26 bits */
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0;
}

static void philox_seeded(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    ora_philox4x32_10(ctr, key, out);
}

/* Box-Muller transform of the two uniforms of one Philox block */
void ora_gauss_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                    double g[2])
{
    uint32_t o[4];
    philox_seeded(seed, c0, c1, c2, c3, o);
    double v1 = u53(o[0], o[1]);
    double v2 = u53(o[2], o[3]);
    double r = sqrt(-2.0 * log(v1));
    double ang = 2.0 * M_PI * v2;
    g[0] = r * cos(ang);
    g[1] = r * sin(ang);
}

double ora_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    uint32_t o[4];
    philox_seeded(seed, c0, c1, c2, c3, o);
    return u53(o[0], o[1]);
}

/* ---------------------------------------------------------------------------
 * gamma matrices, chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]] for
 * k = 1,2,3 (mu = 0,1,2), gamma_4 = [[0, 1], [1, 0]] (mu = 3),
 * gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
 * ------------------------------------------------------------------------- */
static void pauli(int k, ocplx s[4])
{
    memset(s, 0, 4 * sizeof(ocplx));
    if (k == 1) { s[1] = 1; s[2] = 1; }
    if (k == 2) { s[1] = -I; s[2] = I; }
    if (k == 3) { s[0] = 1; s[3] = -1; }
}

static void matmul_n(int n, const ocplx *A, const ocplx *B, ocplx *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            ocplx acc = 0;
            for (int k = 0; k < n; ++k) acc += A[i * n + k] * B[k * n + j];
            C[i * n + j] = acc;
        }
}

void ora_gamma(int mu, ocplx g[16])
{
    memset(g, 0, 16 * sizeof(ocplx));
    if (mu >= 0 && mu <= 2) {
        ocplx s[4];
        pauli(mu + 1, s);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                g[i * 4 + (j + 2)] = -I * s[i * 2 + j];
                g[(i + 2) * 4 + j] = I * s[i * 2 + j];
            }
    } else if (mu == 3) {
        for (int i = 0; i < 2; ++i) {
            g[i * 4 + (i + 2)] = 1;
            g[(i + 2) * 4 + i] = 1;
        }
    } else {
        ocplx a[16], b[16], t[16];
        ora_gamma(0, a);
        ora_gamma(1, b);
        matmul_n(4, a, b, t);
        ora_gamma(2, a);
        matmul_n(4, t, a, b);
        ora_gamma(3, a);
        matmul_n(4, b, a, g);
    }
}

void ora_gellmann_T(int a, ocplx t[9])
{
    memset(t, 0, 9 * sizeof(ocplx));
    switch (a) {
    case 0: t[1] = 1; t[3] = 1; break;
    case 1: t[1] = -I; t[3] = I; break;
    case 2: t[0] = 1; t[4] = -1; break;
    case 3: t[2] = 1; t[6] = 1; break;
    case 4: t[2] = -I; t[6] = I; break;
    case 5: t[5] = 1; t[7] = 1; break;
    case 6: t[5] = -I; t[7] = I; break;
    case 7: t[0] = 1 / sqrt(3.0); t[4] = 1 / sqrt(3.0); t[8] = -2 / sqrt(3.0); break;
    }
    for (int i = 0; i < 9; ++i) t[i] *= 0.5;
}

/* ---------------------------------------------------------------------------
 * exp(A) for a general complex n x n matrix: halve A until its 1-norm is at
 * most 1/2, sum the Taylor series to 30 terms, square back.
 * ------------------------------------------------------------------------- */
void ora_expm(int n, const ocplx *A, ocplx *out)
{
    ocplx *X = malloc(sizeof(ocplx) * n * n);
    ocplx *term = malloc(sizeof(ocplx) * n * n);
    ocplx *tmp = malloc(sizeof(ocplx) * n * n);
    double norm = 0;
    for (int j = 0; j < n; ++j) {
        double col = 0;
        for (int i = 0; i < n; ++i) col += cabs(A[i * n + j]);
        if (col > norm) norm = col;
    }
    int squarings = 0;
    double scale = 1.0;
    while (norm * scale > 0.5) { scale *= 0.5; ++squarings; }
    for (int i = 0; i < n * n; ++i) X[i] = A[i] * scale;
    for (int i = 0; i < n * n; ++i) { out[i] = 0; term[i] = 0; }
    for (int i = 0; i < n; ++i) { out[i * n + i] = 1; term[i * n + i] = 1; }
    for (int k = 1; k <= 30; ++k) {
        matmul_n(n, term, X, tmp);
        for (int i = 0; i < n * n; ++i) { term[i] = tmp[i] / k; out[i] += term[i]; }
    }
    for (int s = 0; s < squarings; ++s) {
        matmul_n(n, out, out, tmp);
        memcpy(out, tmp, sizeof(ocplx) * n * n);
    }
    free(X); free(term); free(tmp);
}

/* ---------------------------------------------------------------------------
 * 3x3 helpers
 * ------------------------------------------------------------------------- */
void su3_mul(const ocplx *A, const ocplx *B, ocplx *C) { matmul_n(3, A, B, C); }

void su3_dag(const ocplx *A, ocplx *B)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[i * 3 + j] = conj(A[j * 3 + i]);
}

/* H = sum_a h_a T^a */
void su3_from_coeffs(const double *h, ocplx *H)
{
    ocplx t[9];
    for (int i = 0; i < 9; ++i) H[i] = 0;
    for (int a = 0; a < 8; ++a) {
        ora_gellmann_T(a, t);
        for (int i = 0; i < 9; ++i) H[i] += h[a] * t[i];
    }
}

/* exp(i eps H) for a 3x3 matrix H */
void su3_expi(const ocplx *H, double eps, ocplx *out)
{
    ocplx A[9];
    for (int i = 0; i < 9; ++i) A[i] = I * eps * H[i];
    ora_expm(3, A, out);
}

/* ---------------------------------------------------------------------------
 * seeded fields.  Counter layout (c0, c1, c2, c3) = (element, block, traj, field):
 * element = 4*s + mu for link fields and s for spinor fields, block = index of
 * the Gaussian pair within the element.
 * ------------------------------------------------------------------------- */
void ora_random_links(const int d[4], uint64_t seed, double alpha, ocplx *U)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < 4 * V; ++l) {
        double h[8];
        for (int j = 0; j < 4; ++j) ora_gauss_pair(seed, (uint32_t)l, j, 0, ORA_FIELD_LINKS, &h[2 * j]);
        ocplx H[9];
        su3_from_coeffs(h, H);
        su3_expi(H, alpha, &U[l * 9]);
    }
}

void ora_gaussian_momenta(const int d[4], uint64_t seed, uint32_t traj, double *mom)
{
    long V = ora_volume(d);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < 4 * V; ++l)
        for (int j = 0; j < 4; ++j)
            ora_gauss_pair(seed, (uint32_t)l, j, traj, ORA_FIELD_MOMENTA, &mom[l * 8 + 2 * j]);
}

void ora_gaussian_spinor(const int d[4], uint64_t seed, uint32_t traj, uint32_t field,
                         int parity_mask, ocplx *psi)
{
    long V = ora_volume(d);
    const double s = sqrt(0.5);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        int p = ora_parity(d, x);
        for (int j = 0; j < 12; ++j) {
            if (parity_mask & (1 << p)) {
                double g[2];
                ora_gauss_pair(seed, (uint32_t)x, j, traj, field, g);
                psi[x * 12 + j] = s * g[0] + I * s * g[1];
            } else {
                psi[x * 12 + j] = 0;
            }
        }
    }
}
