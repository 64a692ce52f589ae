// lgt_stout.cu -- stout smearing (Morningstar & Peardon 2004, the smearing of
// Fig. 1) and its adjoint, the reverse step of Eq. 3 for the map U -> U'.
//
//   C_mu(x) = rho sum_{nu != mu} [U_nu(x) U_mu(x+nu) U_nu(x+mu)^+ + U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu)]
//   Omega = C U^+,  Q = -i P[Omega] (Hermitian traceless, P of Eq. 9),  U' = exp(iQ) U.
//
// Adjoint (gradients in the real-component convention of Eq. S2.11; <A,B> = Re tr A^+B):
//   G_E = G' U^+;  G_Q = traceless Hermitian part of the adjoint of d exp(iQ) applied to G_E,
//   taken from the Cayley-Hamilton form exp(iQ) = f0 + f1 Q + f2 Q^2 with the
//   derivatives of f_j with respect to c0 = det Q and c1 = tr Q^2 / 2 (written out
//   from the chain rule through the eigenvalue parameters u, w), or from the
//   power series when c1 is small;  G_Omega = i G_Q;  G_C = G_Omega U;
//   G_U = E^+ G' + G_Omega^+ C + (staple adjoints of every C that contains U).
// The staple adjoints are gathered per link (18 terms), so no atomics are needed
// and the result is deterministic.
#include "lgt_internal.h"
#include "lgt_su3.cuh"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

__device__ __forceinline__ dmat stout_C(const double2* U, const Geom& g, const int x[4], int mu, double rho) {
    dmat C = zero3<double>();
    int xp[4] = {x[0], x[1], x[2], x[3]};
    shift(g, xp, mu, +1);
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int xpn[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xpn, nu, +1);
        int xmn[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xmn, nu, -1);
        int xmnp[4] = {xmn[0], xmn[1], xmn[2], xmn[3]};
        shift(g, xmnp, mu, +1);
        add_to(C, mul_nd(mul(link_at(U, g, x, nu), link_at(U, g, xpn, mu)), link_at(U, g, xp, nu)));
        add_to(C, mul(mul_dn(link_at(U, g, xmn, nu), link_at(U, g, xmn, mu)), link_at(U, g, xmnp, nu)));
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C.e[a][b] = rho * C.e[a][b];
    return C;
}

// Q = -i P[C U^+]
__device__ __forceinline__ dmat stout_Q(const dmat& C, const dmat& U) {
    dmat Om = mul_nd(C, U);
    dmat Q;
    dcx tr = {0, 0};
    for (int a = 0; a < 3; ++a) tr = tr + (Om.e[a][a] - conj(Om.e[a][a]));
    tr = (1.0 / 3.0) * tr;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            dcx A = 0.5 * (Om.e[a][b] - conj(Om.e[b][a]));
            if (a == b) A = A - 0.5 * tr;
            Q.e[a][b] = times_mi(A);
        }
    return Q;
}

__global__ void __launch_bounds__(NT) stout_forward_kernel(const double2* Uin, double2* Uout, Geom g, double rho) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    eo_coords(g, p, i, x);
    dmat Um = load_link(Uin, g.Vh, p, mu, i);
    dmat C = stout_C(Uin, g, x, mu, rho);
    dmat E = expiQ(stout_Q(C, Um));
    store_link(Uout, g.Vh, p, mu, i, mul(E, Um));
}

// G_Q (full, before projection) for exp(iQ) with Q small: sum_k conj(i^k)/k! sum_m Q^m G Q^(k-1-m)
__device__ dmat expi_adjoint_series(const dmat& Q, const dmat& G) {
    dmat S = G, P = Q, M = zero3<double>();
    double fact = 1.0;
    for (int k = 1; k <= 12; ++k) {
        fact *= k;
        // conj(i^k): k mod 4 = 1 -> -i, 2 -> -1, 3 -> i, 0 -> 1
        dcx c = (k % 4 == 1) ? dcx{0, -1} : (k % 4 == 2) ? dcx{-1, 0} : (k % 4 == 3) ? dcx{0, 1} : dcx{1, 0};
        c = (1.0 / fact) * c;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M.e[a][b] = cmad(M.e[a][b], c, S.e[a][b]);
        // S_{k+1} = Q S_k + G Q^k,  P = Q^(k+1)
        dmat S2 = mul(Q, S);
        add_to(S2, mul(G, P));
        S = S2;
        P = mul(Q, P);
    }
    return M;
}

// pass 1: per-link adjoint of the exponential and of Omega = C U^+
__global__ void __launch_bounds__(NT) stout_bwd_local_kernel(const double2* Uin, const double2* Gout, double2* Gin,
                                                             double2* GC, Geom g, double rho) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    eo_coords(g, p, i, x);
    dmat Um = load_link(Uin, g.Vh, p, mu, i);
    dmat C = stout_C(Uin, g, x, mu, rho);
    dmat Q = stout_Q(C, Um);
    dmat Go = load_link(Gout, g.Vh, p, mu, i);
    dmat Gb = mul_nd(Go, Um);   // G_E
    dmat Q2 = mul(Q, Q);
    double c1 = 0.5 * retrace(Q2);
    dmat E, M;
    if (c1 < 1e-3) {
        E = expiQ(Q);
        M = expi_adjoint_series(Q, Gb);
    } else {
        double c0 = retrace(mul(Q, Q2)) / 3.0;
        const bool neg = c0 < 0;
        if (neg) c0 = -c0;
        double c0max = 2.0 * (c1 / 3.0) * sqrt(c1 / 3.0);
        double theta = acos(fmin(c0 / c0max, 1.0));
        double st, ct;
        sincos(theta / 3.0, &st, &ct);
        double sq = sqrt(c1);
        double u = sq * (1.0 / 1.7320508075688772935) * ct, w = sq * st;
        double u2 = u * u, w2 = w * w;
        double sw, cw;
        sincos(w, &sw, &cw);
        double xi0, xi1;
        if (fabs(w) < 0.05) {
            xi0 = 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0));
            xi1 = -1.0 / 3.0 + w2 / 30.0 * (1.0 - w2 / 28.0 * (1.0 - w2 / 54.0));
        } else {
            xi0 = sw / w;
            xi1 = cw / w2 - sw / (w2 * w);
        }
        double s2u, c2u, su, cu;
        sincos(2.0 * u, &s2u, &c2u);
        sincos(u, &su, &cu);
        dcx e2 = {c2u, s2u}, em = {cu, -su};
        const dcx I1 = {0, 1};
        dcx h[3], r1[3], r2[3];
        h[0] = (u2 - w2) * e2 + em * dcx{8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0};
        h[1] = (2.0 * u) * e2 - em * dcx{2.0 * u * cw, -(3.0 * u2 - w2) * xi0};
        h[2] = e2 - em * dcx{cw, 3.0 * u * xi0};
        // r1_j = d h_j / du,  r2_j = (1/w) d h_j / dw
        r1[0] = 2.0 * (dcx{u, u2 - w2} * e2) +
                2.0 * (em * (dcx{8.0 * u * cw, -4.0 * u2 * cw} +
                             I1 * (xi0 * dcx{9.0 * u2 + w2, -u * (3.0 * u2 + w2)})));
        r1[1] = 2.0 * (dcx{1.0, 2.0 * u} * e2) +
                em * (dcx{-2.0 * cw, 2.0 * u * cw} + I1 * (xi0 * dcx{6.0 * u, w2 - 3.0 * u2}));
        r1[2] = 2.0 * (I1 * e2) + I1 * (em * dcx{cw - 3.0 * xi0, 3.0 * u * xi0});
        r2[0] = -2.0 * e2 + (2.0 * u) * (I1 * (em * dcx{cw + xi0 + 3.0 * u2 * xi1, 4.0 * u * xi0}));
        r2[1] = dcx{0, -1} * (em * dcx{cw + xi0 - 3.0 * u2 * xi1, 2.0 * u * xi0});
        r2[2] = em * dcx{xi0, -3.0 * u * xi1};
        double D = 9.0 * u2 - w2;
        double iD = 1.0 / D, iD2 = 0.5 / (D * D);
        dcx f[3], b1[3], b2[3];
        for (int j = 0; j < 3; ++j) {
            f[j] = iD * h[j];
            b1[j] = iD2 * ((2.0 * u) * r1[j] + (3.0 * u2 - w2) * r2[j] - (2.0 * (15.0 * u2 + w2)) * f[j]);
            b2[j] = iD2 * (r1[j] - (3.0 * u) * r2[j] - (24.0 * u) * f[j]);
        }
        if (neg) {
            f[0] = conj(f[0]); f[1] = -conj(f[1]); f[2] = conj(f[2]);
            b1[0] = conj(b1[0]); b1[1] = -conj(b1[1]); b1[2] = conj(b1[2]);
            b2[0] = -conj(b2[0]); b2[1] = conj(b2[1]); b2[2] = -conj(b2[2]);
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                dcx v = cmad(f[1] * Q.e[a][b], f[2], Q2.e[a][b]);
                E.e[a][b] = (a == b) ? v + f[0] : v;
            }
        // t_j = tr(G_E^+ Q^j)
        dcx t0 = {0, 0}, t1 = {0, 0}, t2 = {0, 0};
        for (int a = 0; a < 3; ++a) {
            t0 = t0 + conj(Gb.e[a][a]);
            for (int b = 0; b < 3; ++b) {
                t1 = cmadc(t1, Gb.e[b][a], Q.e[b][a]);
                t2 = cmadc(t2, Gb.e[b][a], Q2.e[b][a]);
            }
        }
        double r0 = (b2[0] * t0).r + (b2[1] * t1).r + (b2[2] * t2).r;
        double rr1 = (b1[0] * t0).r + (b1[1] * t1).r + (b1[2] * t2).r;
        dmat GQ = mul(Gb, Q);
        add_to(GQ, mul(Q, Gb));
        dcx cf1 = conj(f[1]), cf2 = conj(f[2]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                dcx v = r0 * Q2.e[a][b] + rr1 * Q.e[a][b];
                v = cmad(v, cf1, Gb.e[a][b]);
                v = cmad(v, cf2, GQ.e[a][b]);
                M.e[a][b] = v;
            }
    }
    // G_Q = traceless Hermitian part of M;  G_Omega = i G_Q
    dmat GO;
    double trh = (M.e[0][0].r + M.e[1][1].r + M.e[2][2].r) / 3.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            dcx hq = 0.5 * (M.e[a][b] + conj(M.e[b][a]));
            if (a == b) hq.r -= trh;
            GO.e[a][b] = times_i(hq);
        }
    store_link(GC, g.Vh, p, mu, i, mul(GO, Um));
    dmat local = mul_dn(E, Go);
    add_to(local, mul_dn(GO, C));
    store_link(Gin, g.Vh, p, mu, i, local);
}

// pass 2: gather the staple adjoints of every C that contains U_mu(x)
__global__ void __launch_bounds__(NT) stout_bwd_gather_kernel(const double2* U, const double2* GC, double2* Gin,
                                                              Geom g, double rho) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    eo_coords(g, p, i, x);
    dmat acc = zero3<double>();
    int xpm[4] = {x[0], x[1], x[2], x[3]};
    shift(g, xpm, mu, +1);
#pragma unroll 1
    for (int a = 0; a < 4; ++a) {
        if (a == mu) continue;
        int xma[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xma, a, -1);
        int xmapm[4] = {xma[0], xma[1], xma[2], xma[3]};
        shift(g, xmapm, mu, +1);
        int xpa[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xpa, a, +1);
        // middle factor of staple 1 of C_mu(x-a): U_a(x-a)^+ G_C(x-a,mu) U_a(x-a+mu)
        add_to(acc, mul(mul_dn(link_at(U, g, xma, a), link_at(GC, g, xma, mu)), link_at(U, g, xmapm, a)));
        // middle factor of staple 2 of C_mu(x+a): U_a(x) G_C(x+a,mu) U_a(x+mu)^+
        add_to(acc, mul_nd(mul(link_at(U, g, x, a), link_at(GC, g, xpa, mu)), link_at(U, g, xpm, a)));
        const int n = a;
        int xmn[4] = {xma[0], xma[1], xma[2], xma[3]};     // x - n
        int xpn[4] = {xpa[0], xpa[1], xpa[2], xpa[3]};     // x + n
        int xmnpm[4] = {xmapm[0], xmapm[1], xmapm[2], xmapm[3]};  // x - n + mu
        // first factor of staple 1 of C_n(x): G_C(x,n) U_mu(x+n) U_n(x+mu)^+
        add_to(acc, mul_nd(mul(link_at(GC, g, x, n), link_at(U, g, xpn, mu)), link_at(U, g, xpm, n)));
        // conjugated third factor of staple 1 of C_n(x-n): G_C(x-n,n)^+ U_mu(x-n) U_n(x-n+mu)
        add_to(acc, mul(mul_dn(link_at(GC, g, xmn, n), link_at(U, g, xmn, mu)), link_at(U, g, xmnpm, n)));
        // conjugated first factor of staple 2 of C_n(x+mu): U_n(x) U_mu(x+n) G_C(x+mu,n)^+
        add_to(acc, mul_nd(mul(link_at(U, g, x, n), link_at(U, g, xpn, mu)), link_at(GC, g, xpm, n)));
        // third factor of staple 2 of C_n(x+mu-n): U_n(x-n)^+ U_mu(x-n) G_C(x+mu-n,n)
        add_to(acc, mul(mul_dn(link_at(U, g, xmn, n), link_at(U, g, xmn, mu)), link_at(GC, g, xmnpm, n)));
    }
    dmat G = load_link(Gin, g.Vh, p, mu, i);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G.e[a][b] = G.e[a][b] + rho * acc.e[a][b];
    store_link(Gin, g.Vh, p, mu, i, G);
}

cudaError_t stout_forward(const double2* Uin, double2* Uout, const Geom& g, double rho, cudaStream_t st) {
    stout_forward_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Uin, Uout, g, rho);
    count_launch();
    return cudaGetLastError();
}

cudaError_t stout_backward(const double2* Uin, const double2* Gout, double2* Gin, double2* scratch, const Geom& g,
                           double rho, cudaStream_t st) {
    stout_bwd_local_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Uin, Gout, Gin, scratch, g, rho);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stout_bwd_gather_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Uin, scratch, Gin, g, rho);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
