// lgt_force_df.cu -- Lie-form MD forces in double-float arithmetic (lgt_df64.cuh):
// the staple force of the Wilson gauge action (Eq. 9 applied to S_G) and the
// Wilson pseudofermion force (Eq. S3.12), with the same formulas as the FP64
// kernels of lgt_gauge.cu / lgt_force.cu, products of link matrices and spinor
// outer products carried as FP32 pairs (about 48 significant bits), the eight Lie
// components converted to FP64 and accumulated into FP64 momenta.
//
// Inputs are double-float copies made per force evaluation from the FP64 fields
// (links: float4 [parity][4][9][Vh]; spinors: float4 [parity][12][Vh], each
// float4 = (re.hi, re.lo, im.hi, im.lo)): 144 B per link and 192 B per site, the
// same bytes as FP64.
#include "lgt_internal.h"
#include "lgt_df64.cuh"
#include "lgt_spin.cuh"
#include "lgt_su3.cuh"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

// ---------------------------------------------------------------- conversions
__global__ void __launch_bounds__(NT) links_to_df_kernel(float4* Udf, const double2* U, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    store_link_df(Udf, g.Vh, p, mu, i, load_link(U, g.Vh, p, mu, i));
}
cudaError_t links_to_df(float4* Udf, const double2* U, const Geom& g, cudaStream_t st) {
    links_to_df_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Udf, U, g);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) spinor_to_df_kernel(float4* y, const double2* x, long ne) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const double2 v = __ldg(x + e);
    const df r = df_from(v.x), im = df_from(v.y);
    y[e] = make_float4(r.h, r.l, im.h, im.l);
}
// one full FP64 spinor field [2][12][Vh] -> double-float
cudaError_t spinor_to_df(float4* y, const double2* x, const Geom& g, cudaStream_t st) {
    const long ne = 24L * g.Vh;   // [2][12][Vh] double2 entries
    spinor_to_df_kernel<<<grid_for(ne), NT, 0, st>>>(y, x, ne);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gauge force
// V_mu(x) = sum_nu [U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)],
// d_a S_G = (beta/6) Im tr(lambda^a U V);  out = keep*out + coef * d S_G
__global__ void __launch_bounds__(NT) gauge_force_df_kernel(const float4* U, Geom g, double beta, double coef,
                                                            int keep, double2* out) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    eo_coords(g, p, i, x);
    int xp[4] = {x[0], x[1], x[2], x[3]};
    shift(g, xp, mu, +1);
    dfmat V = df_zero3();
    // six staples through one loop body (the conjugations taken at load time):
    //   upper  U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+,  lower  U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
        const int nu = (k >> 1) + ((k >> 1) >= mu);
        const bool lower = k & 1;
        int a[4] = {xp[0], xp[1], xp[2], xp[3]};   // x + mu (-nu)
        int b[4] = {x[0], x[1], x[2], x[3]};       // x +- nu
        if (lower) shift(g, a, nu, -1);
        shift(g, b, nu, lower ? -1 : +1);
        dfmat T;
        df_mul_rows(T, link_df_op(U, g, a, nu, lower), link_df_op(U, g, b, mu, true), false);
        df_mul_rows(V, T, lower ? link_df_op(U, g, b, nu, false) : link_df_op(U, g, x, nu, true), true);
    }
    const dfmat M = df_mul<false, false>(load_link_df(U, g.Vh, p, mu, i), V);
    double c[8], f[8];
    lie_im_tr_df(M, c);
    if (keep) load_mom(out, g.Vh, p, mu, i, f);
    const double s = coef * beta / 6.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) + s * c[a];
    store_mom(out, g.Vh, p, mu, i, f);
}
cudaError_t gauge_force_df(const float4* Udf, const Geom& g, double beta, double coef, int keep, double2* out,
                           cudaStream_t st) {
    gauge_force_df_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Udf, g, beta, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fermion force
// W = U P1 - P2 U^+ from the projected rows (as w_matrix of lgt_force.cu):
//   U P1 = sum_j (U h_j(X(x+mu))) k_j(Y(x))^+,  P2 U^+ = sum_j h_j(X(x)) (U k_j(Y(x+mu)))^+
template <int MU>
__device__ __forceinline__ void w_matrix_df(const dfmat& U, const dfc (&Xx)[4][3], const dfc (&Yx)[4][3],
                                            const dfc (&Xy)[4][3], const dfc (&Yy)[4][3], dfmat& W) {
    dfc h[2][3], k[2][3], m[2][3], h2[2][3], m2[2][3];
    project<MU, -1>(Xy, h);
    project<MU, -1>(Yx, k);
    project<MU, +1>(Xx, h2);
    {
        dfc k2[2][3];
        project<MU, +1>(Yy, k2);
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dacc re = dacc0(), im = dacc0(), re2 = dacc0(), im2 = dacc0();
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    cacc_mul<false, false>(re, im, U.e[a][b], h[j][b]);
                    cacc_mul<false, false>(re2, im2, U.e[a][b], k2[j][b]);
                }
                m[j][a] = {dacc_get(re), dacc_get(im)};
                m2[j][a] = {dacc_get(re2), dacc_get(im2)};
            }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dacc re = dacc0(), im = dacc0();
            cacc_mul<false, true>(re, im, m[0][a], k[0][c]);
            cacc_mul<false, true>(re, im, m[1][a], k[1][c]);
            cacc_mul<false, true>(re, im, -h2[0][a], m2[0][c]);
            cacc_mul<false, true>(re, im, -h2[1][a], m2[1][c]);
            W.e[a][c] = {dacc_get(re), dacc_get(im)};
        }
}

__global__ void __launch_bounds__(NT) fermion_force_df_kernel(const float4* U, const float4* X, const float4* Y,
                                                              Geom g, double kappa, double coef, int keep,
                                                              double2* out) {
    const long t = (long)blockIdx.x * NT + threadIdx.x;
    if (t >= 8L * g.Vh) return;
    const int mu = (int)(t / (2 * g.Vh));
    const int rem = (int)(t - (long)mu * 2 * g.Vh);
    const int p = rem >= g.Vh, i = rem - p * g.Vh;
    int x[4];
    const int lex = eo_coords(g, p, i, x);
    const int j = nb_lex(g, lex, x, mu, +1) >> 1;
    const double b = (mu == 3 && x[3] == g.L[3] - 1) ? -1.0 : 1.0;
    const size_t hf = (size_t)12 * g.Vh;
    const SpinorDF Xx = load_spinor_df(X + p * hf, g.Vh, i), Yx = load_spinor_df(Y + p * hf, g.Vh, i);
    const SpinorDF Xy = load_spinor_df(X + (1 - p) * hf, g.Vh, j), Yy = load_spinor_df(Y + (1 - p) * hf, g.Vh, j);
    const dfmat Um = load_link_df(U, g.Vh, p, mu, i);
    dfmat W;
    switch (mu) {
    case 0: w_matrix_df<0>(Um, Xx.c, Yx.c, Xy.c, Yy.c, W); break;
    case 1: w_matrix_df<1>(Um, Xx.c, Yx.c, Xy.c, Yy.c, W); break;
    case 2: w_matrix_df<2>(Um, Xx.c, Yx.c, Xy.c, Yy.c, W); break;
    default: w_matrix_df<3>(Um, Xx.c, Yx.c, Xy.c, Yy.c, W); break;
    }
    double cl[8], f[8];
    lie_im_tr_df(W, cl);
    if (keep) load_mom(out, g.Vh, p, mu, i, f);
    const double s = -coef * kappa * b;
#pragma unroll
    for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) + s * cl[a];
    store_mom(out, g.Vh, p, mu, i, f);
}
cudaError_t fermion_force_df(const float4* Udf, const float4* Xdf, const float4* Ydf, const Geom& g, double kappa,
                             double coef, int keep, double2* out, cudaStream_t st) {
    fermion_force_df_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Udf, Xdf, Ydf, g, kappa, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
