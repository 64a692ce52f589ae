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
        const dfmat T = df_mul<false, false>(link_df_op(U, g, a, nu, lower), link_df_op(U, g, b, mu, true));
        df_mul_acc<false, false>(V, T, lower ? link_df_op(U, g, b, nu, false) : link_df_op(U, g, x, nu, true));
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

// ---------------------------------------------------------------- link update
// U <- exp(i eps P) U in double-float arithmetic: the exponential by the Cayley-Hamilton
// recursion of lgt_su3.cuh (expiQ_h: Q^3 = c1 Q + c0, Q scaled so that c1 <= 3/16, 12 or
// 14 series terms, squarings on the coefficients), every real carried as an FP32 pair.
// The link is read from its double-float copy (the one the force evaluation before the
// update made) and the updated link is written as FP64, as the FP32 two-row copy and
// as the double-float copy: the FP64-pipe work is the conversions (~80 per link) in
// place of ~340 FP64 instructions.
__device__ __forceinline__ df dfm(df a, df b) {   // a b
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_renorm(p, e);
}
__host__ __device__ constexpr df df_const(double x) { return df{(float)x, (float)(x - (double)(float)x)}; }
__device__ __forceinline__ df df_scale(df a, float s) { return {a.h * s, a.l * s}; }   // s a power of 2
__device__ __forceinline__ dfc dfcm(const dfc& a, const dfc& b) {   // a b
    dacc re = dacc0(), im = dacc0();
    cacc_mul<false, false>(re, im, a, b);
    return {dacc_get(re), dacc_get(im)};
}
__device__ __forceinline__ dfc dfcm_cb(const dfc& a, const dfc& b) {   // a conj(b)
    dacc re = dacc0(), im = dacc0();
    cacc_mul<false, true>(re, im, a, b);
    return {dacc_get(re), dacc_get(im)};
}
__device__ __forceinline__ dfc dfc_conj(const dfc& a) { return {a.r, df_neg(a.i)}; }
__device__ __forceinline__ dfc dfc_real(const dfc& a, df s) { return {dfm(a.r, s), dfm(a.i, s)}; }   // s a

template <int N>
__device__ __forceinline__ void ch_term_df(df c0, df c1, df& a, df& b, df& d, df (&acc)[3], bool neg) {
    constexpr df inv = df_const(1.0 / N);
    const df na = dfm(dfm(c0, inv), d);
    const df nb = dfm(df_add(dfm(c1, d), a), inv);
    const df nd = dfm(b, inv);
    a = na; b = nb; d = nd;
    acc[0] = neg ? df_sub(acc[0], a) : df_add(acc[0], a);
    acc[1] = neg ? df_sub(acc[1], b) : df_add(acc[1], b);
    acc[2] = neg ? df_sub(acc[2], d) : df_add(acc[2], d);
}

__global__ void __launch_bounds__(NT) update_links_df_kernel(float4* Udf, double2* U, float4* U12,
                                                             const double2* mom, double eps, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    double pv[8];
    load_mom(mom, g.Vh, p, mu, i, pv);
    df q[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) q[a] = df_from(eps * pv[a]);
    // Q = sum_a q_a T^a: diagonal and upper triangle
    constexpr df is3 = df_const(0.57735026918962576451);
    const df t7 = dfm(q[7], is3);
    const df d0 = df_scale(df_add(q[2], t7), 0.5f), d1 = df_scale(df_sub(t7, q[2]), 0.5f);
    const df d2 = df_neg(t7);
    const dfc o01 = {df_scale(q[0], 0.5f), df_scale(df_neg(q[1]), 0.5f)};
    const dfc o02 = {df_scale(q[3], 0.5f), df_scale(df_neg(q[4]), 0.5f)};
    const dfc o12 = {df_scale(q[5], 0.5f), df_scale(df_neg(q[6]), 0.5f)};
    // Q^2 (Hermitian)
    auto n2 = [](const dfc& z) { return df_add(dfm(z.r, z.r), dfm(z.i, z.i)); };
    const df n01 = n2(o01), n02 = n2(o02), n12 = n2(o12);
    const df s00 = df_add(dfm(d0, d0), df_add(n01, n02));
    const df s11 = df_add(dfm(d1, d1), df_add(n01, n12));
    const df s22 = df_add(dfm(d2, d2), df_add(n02, n12));
    const dfc s01 = dfc_real(o01, df_add(d0, d1)) + dfcm_cb(o02, o12);   // (d0 + d1) q01 + q02 conj(q12)
    const dfc s02 = dfc_real(o02, df_add(d0, d2)) + dfcm(o01, o12);      // (d0 + d2) q02 + q01 q12
    const dfc s12 = dfc_real(o12, df_add(d1, d2)) + dfcm(dfc_conj(o01), o02);   // (d1 + d2) q12 + conj(q01) q02
    df c1 = df_scale(df_add(s00, df_add(s11, s22)), 0.5f);
    // det Q = d0 d1 d2 + 2 Re(q01 q12 conj(q02)) - d0 |q12|^2 - d1 |q02|^2 - d2 |q01|^2
    const dfc t = dfcm(o01, o12);
    df c0 = dfm(dfm(d0, d1), d2);
    c0 = df_add(c0, df_scale(df_add(dfm(t.r, o02.r), dfm(t.i, o02.i)), 2.0f));
    c0 = df_sub(c0, df_add(dfm(d0, n12), df_add(dfm(d1, n02), dfm(d2, n01))));
    int s = 0;
    while (c1.h > 0.1875f && s < 64) { c1 = df_scale(c1, 0.25f); c0 = df_scale(c0, 0.125f); ++s; }
    const df one = {1.f, 0.f}, zero = {0.f, 0.f};
    df fr[3] = {one, zero, zero}, fi[3] = {zero, zero, zero};
    df a = one, b = zero, d = zero;
    ch_term_df<1>(c0, c1, a, b, d, fi, false);
    ch_term_df<2>(c0, c1, a, b, d, fr, true);
    ch_term_df<3>(c0, c1, a, b, d, fi, true);
    ch_term_df<4>(c0, c1, a, b, d, fr, false);
    ch_term_df<5>(c0, c1, a, b, d, fi, false);
    ch_term_df<6>(c0, c1, a, b, d, fr, true);
    ch_term_df<7>(c0, c1, a, b, d, fi, true);
    ch_term_df<8>(c0, c1, a, b, d, fr, false);
    ch_term_df<9>(c0, c1, a, b, d, fi, false);
    ch_term_df<10>(c0, c1, a, b, d, fr, true);
    ch_term_df<11>(c0, c1, a, b, d, fi, true);
    ch_term_df<12>(c0, c1, a, b, d, fr, false);
    if (c1.h > 0.046875f) {   // r > 1/4: two more terms
        ch_term_df<13>(c0, c1, a, b, d, fi, false);
        ch_term_df<14>(c0, c1, a, b, d, fr, true);
    }
    dfc f0 = {fr[0], fi[0]}, f1 = {fr[1], fi[1]}, f2 = {fr[2], fi[2]};
    for (; s > 0; --s) {
        const dfc f12 = dfcm(f1, f2), f22 = dfcm(f2, f2);
        const dfc g0 = dfcm(f0, f0) + dfc_real(f12, df_scale(c0, 2.0f));
        const dfc g1 = dfc{df_scale(dfcm(f0, f1).r, 2.0f), df_scale(dfcm(f0, f1).i, 2.0f)} +
                       dfc_real(f12, df_scale(c1, 2.0f)) + dfc_real(f22, c0);
        const dfc g2 = dfcm(f1, f1) + dfc{df_scale(dfcm(f0, f2).r, 2.0f), df_scale(dfcm(f0, f2).i, 2.0f)} +
                       dfc_real(f22, c1);
        f0 = g0;
        f1 = {df_scale(g1.r, 0.5f), df_scale(g1.i, 0.5f)};
        f2 = {df_scale(g2.r, 0.25f), df_scale(g2.i, 0.25f)};
        c1 = df_scale(c1, 4.0f); c0 = df_scale(c0, 8.0f);
    }
    // E = f0 + f1 Q + f2 Q^2
    dfmat E;
    const df dd[3] = {d0, d1, d2}, ss[3] = {s00, s11, s22};
#pragma unroll
    for (int k = 0; k < 3; ++k) E.e[k][k] = f0 + dfc_real(f1, dd[k]) + dfc_real(f2, ss[k]);
    E.e[0][1] = dfcm(f1, o01) + dfcm(f2, s01);
    E.e[0][2] = dfcm(f1, o02) + dfcm(f2, s02);
    E.e[1][2] = dfcm(f1, o12) + dfcm(f2, s12);
    E.e[1][0] = dfcm(f1, dfc_conj(o01)) + dfcm(f2, dfc_conj(s01));
    E.e[2][0] = dfcm(f1, dfc_conj(o02)) + dfcm(f2, dfc_conj(s02));
    E.e[2][1] = dfcm(f1, dfc_conj(o12)) + dfcm(f2, dfc_conj(s12));
    const dfmat m = df_mul<false, false>(E, load_link_df(Udf, g.Vh, p, mu, i));
    float4* bdf = Udf + (size_t)((p * 4 + mu) * 9) * g.Vh + i;
    double2* b64 = U + (size_t)((p * 4 + mu) * 9) * g.Vh + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const dfc& v = m.e[k / 3][k % 3];
        bdf[(size_t)k * g.Vh] = make_float4(v.r.h, v.r.l, v.i.h, v.i.l);
        b64[(size_t)k * g.Vh] = make_double2(df_to(v.r), df_to(v.i));
    }
    // the FP32 two-row copy: the rounded FP64 value is the pair's high word
    float4* b12 = U12 + (size_t)((p * 4 + mu) * 3) * g.Vh + i;
    b12[0] = make_float4(m.e[0][0].r.h, m.e[0][0].i.h, m.e[0][1].r.h, m.e[0][1].i.h);
    b12[g.Vh] = make_float4(m.e[0][2].r.h, m.e[0][2].i.h, m.e[1][0].r.h, m.e[1][0].i.h);
    b12[2 * (size_t)g.Vh] = make_float4(m.e[1][1].r.h, m.e[1][1].i.h, m.e[1][2].r.h, m.e[1][2].i.h);
}
cudaError_t update_links_df(float4* Udf, double2* U, float4* U12, const double2* mom, double eps, const Geom& g,
                            cudaStream_t st) {
    update_links_df_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Udf, U, U12, mom, eps, g);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
