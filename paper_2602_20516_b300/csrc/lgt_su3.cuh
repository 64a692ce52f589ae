// lgt_su3.cuh -- SU(3) functions shared by the gauge-field kernels: the
// exponential of i times a Hermitian traceless matrix and reunitarisation.
#pragma once
#include "lgt_common.cuh"

namespace lgt {

// thread -> (mu, parity, i) for 4 V links
__device__ __forceinline__ bool link_index(const Geom& g, int& mu, int& p, int& i) {
    const long t = (long)blockIdx.x * NT + threadIdx.x;
    if (t >= 8L * g.Vh) return false;
    mu = (int)(t / (2 * g.Vh));
    int rem = (int)(t - (long)mu * 2 * g.Vh);
    p = rem >= g.Vh;
    i = rem - p * g.Vh;
    return true;
}

// coordinates and lexicographic index of an arbitrary site
__device__ __forceinline__ int lex_of(const Geom& g, const int x[4]) {
    return x[0] + g.stride[1] * x[1] + g.stride[2] * x[2] + g.stride[3] * x[3];
}
__device__ __forceinline__ dmat link_at(const double2* U, const Geom& g, const int x[4], int mu) {
    int lex = lex_of(g, x);
    int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    return load_link(U, g.Vh, par, mu, lex >> 1);
}
__device__ __forceinline__ void shift(const Geom& g, int x[4], int mu, int dir) {
    x[mu] += dir;
    if (x[mu] == g.L[mu]) x[mu] = 0;
    if (x[mu] < 0) x[mu] = g.L[mu] - 1;
}


// ---------------------------------------------------------------- exp(iQ)
// exp(iQ) for Hermitian traceless Q, without trigonometric functions.
// Cayley-Hamilton: Q^3 = c1 Q + c0 with c1 = tr(Q^2)/2, c0 = det Q, so every power
// reduces to Q^n / n! = a_n + b_n Q + d_n Q^2 with real coefficients obeying
//   (a, b, d)_{n+1} = (c0 d_n, a_n + c1 d_n, b_n) / (n + 1),
// and exp(iQ) = f0 + f1 Q + f2 Q^2 with f = sum_n i^n (a, b, d)_n.  The spectral
// radius obeys r^2 <= 4 c1 / 3; Q is first scaled by 2^-s so that r <= 1/2, the
// series is cut after 12 terms (r <= 1/4) or 14 terms (r <= 1/2), remainder
// below 3e-17, and the s squarings are done on the coefficients:
//   (f0 + f1 q + f2 q^2)^2 = (f0^2 + 2 c0 f1 f2) + (2 f0 f1 + 2 c1 f1 f2 + c0 f2^2) q
//                            + (f1^2 + 2 f0 f2 + c1 f2^2) q^2.
// Every lane of a warp runs the same instruction sequence unless its r needs the
// longer series or a squaring.  Q is read from its diagonal and upper triangle.
struct HermQ {
    double d[3];   // diagonal (real)
    dcx o01, o02, o12;   // upper triangle
};
__device__ __forceinline__ HermQ herm_parts(const dmat& Q) {
    return HermQ{{Q.e[0][0].r, Q.e[1][1].r, Q.e[2][2].r}, Q.e[0][1], Q.e[0][2], Q.e[1][2]};
}
// P = sum_a p_a T^a from its Lie components
__device__ __forceinline__ HermQ herm_parts_lie(const double p[8]) {
    const double is3 = 0.57735026918962576451;
    HermQ h;
    h.d[0] = 0.5 * (p[2] + p[7] * is3);
    h.d[1] = 0.5 * (-p[2] + p[7] * is3);
    h.d[2] = -p[7] * is3;
    h.o01 = {0.5 * p[0], -0.5 * p[1]};
    h.o02 = {0.5 * p[3], -0.5 * p[4]};
    h.o12 = {0.5 * p[5], -0.5 * p[6]};
    return h;
}
__device__ __forceinline__ double norm2d(dcx a) { return fma(a.r, a.r, a.i * a.i); }
// one step of the coefficient recursion, accumulated with sign sg into acc
template <int N1>
__device__ __forceinline__ void ch_term(double c0, double c1, double& a, double& b, double& d, double (&acc)[3],
                                        double sg) {
    constexpr double inv = 1.0 / N1;
    const double na = (c0 * inv) * d;
    const double nb = fma(c1, d, a) * inv;
    const double nd = b * inv;
    a = na; b = nb; d = nd;
    acc[0] = fma(sg, a, acc[0]);
    acc[1] = fma(sg, b, acc[1]);
    acc[2] = fma(sg, d, acc[2]);
}
__device__ __forceinline__ dmat expiQ_h(const HermQ& h) {
    // Q^2 (Hermitian): diagonal and upper triangle
    const double n01 = norm2d(h.o01), n02 = norm2d(h.o02), n12 = norm2d(h.o12);
    const double s00 = fma(h.d[0], h.d[0], n01 + n02);
    const double s11 = fma(h.d[1], h.d[1], n01 + n12);
    const double s22 = fma(h.d[2], h.d[2], n02 + n12);
    // (Q^2)_01 = (d0 + d1) q01 + q02 conj(q12), etc.
    dcx s01 = (h.d[0] + h.d[1]) * h.o01;
    s01 = cmad_cb(s01, h.o02, h.o12);
    dcx s02 = (h.d[0] + h.d[2]) * h.o02;
    s02 = cmad(s02, h.o01, h.o12);
    dcx s12 = (h.d[1] + h.d[2]) * h.o12;
    s12 = cmadc(s12, h.o01, h.o02);
    double c1 = 0.5 * (s00 + s11 + s22);
    // det Q = d0 d1 d2 + 2 Re(q01 q12 conj(q02)) - d0 |q12|^2 - d1 |q02|^2 - d2 |q01|^2
    const dcx t = h.o01 * h.o12;
    double c0 = h.d[0] * h.d[1] * h.d[2];
    c0 = fma(2.0, fma(t.r, h.o02.r, t.i * h.o02.i), c0);
    c0 = fma(-h.d[0], n12, c0);
    c0 = fma(-h.d[1], n02, c0);
    c0 = fma(-h.d[2], n01, c0);
    // scale so that r^2 <= 4 c1' / 3 <= 1/4, i.e. c1' <= 3/16
    // (bounded: a non-finite Q leaves the loop after 64 halvings and yields NaN)
    int s = 0;
    while (c1 > 0.1875 && s < 64) { c1 *= 0.25; c0 *= 0.125; ++s; }
    // series: real parts from even n, imaginary parts from odd n
    double fr[3] = {1.0, 0.0, 0.0}, fi[3] = {0.0, 0.0, 0.0};
    double a = 1.0, b = 0.0, d = 0.0;
    ch_term<1>(c0, c1, a, b, d, fi, 1.0);
    ch_term<2>(c0, c1, a, b, d, fr, -1.0);
    ch_term<3>(c0, c1, a, b, d, fi, -1.0);
    ch_term<4>(c0, c1, a, b, d, fr, 1.0);
    ch_term<5>(c0, c1, a, b, d, fi, 1.0);
    ch_term<6>(c0, c1, a, b, d, fr, -1.0);
    ch_term<7>(c0, c1, a, b, d, fi, -1.0);
    ch_term<8>(c0, c1, a, b, d, fr, 1.0);
    ch_term<9>(c0, c1, a, b, d, fi, 1.0);
    ch_term<10>(c0, c1, a, b, d, fr, -1.0);
    ch_term<11>(c0, c1, a, b, d, fi, -1.0);
    ch_term<12>(c0, c1, a, b, d, fr, 1.0);
    if (c1 > 0.046875) {   // r > 1/4: two more terms
        ch_term<13>(c0, c1, a, b, d, fi, 1.0);
        ch_term<14>(c0, c1, a, b, d, fr, -1.0);
    }
    dcx f0 = {fr[0], fi[0]}, f1 = {fr[1], fi[1]}, f2 = {fr[2], fi[2]};
    for (; s > 0; --s) {
        const dcx f12 = f1 * f2, f22 = f2 * f2;
        const dcx g0 = cmad(f0 * f0, dcx{2.0 * c0, 0.0}, f12);
        dcx g1 = 2.0 * (f0 * f1);
        g1 = cmad(g1, dcx{2.0 * c1, 0.0}, f12);
        g1 = cmad(g1, dcx{c0, 0.0}, f22);
        dcx g2 = f1 * f1;
        g2 = cmad(g2, dcx{2.0, 0.0}, f0 * f2);
        g2 = cmad(g2, dcx{c1, 0.0}, f22);
        // re-express in the basis of 2q
        f0 = g0; f1 = 0.5 * g1; f2 = 0.25 * g2;
        c1 *= 4.0; c0 *= 8.0;
    }
    // E = f0 + f1 Q + f2 Q^2
    dmat E;
    E.e[0][0] = dcx{fma(f1.r, h.d[0], fma(f2.r, s00, f0.r)), fma(f1.i, h.d[0], fma(f2.i, s00, f0.i))};
    E.e[1][1] = dcx{fma(f1.r, h.d[1], fma(f2.r, s11, f0.r)), fma(f1.i, h.d[1], fma(f2.i, s11, f0.i))};
    E.e[2][2] = dcx{fma(f1.r, h.d[2], fma(f2.r, s22, f0.r)), fma(f1.i, h.d[2], fma(f2.i, s22, f0.i))};
    E.e[0][1] = cmad(f1 * h.o01, f2, s01);
    E.e[0][2] = cmad(f1 * h.o02, f2, s02);
    E.e[1][2] = cmad(f1 * h.o12, f2, s12);
    E.e[1][0] = cmad(f1 * conj(h.o01), f2, conj(s01));
    E.e[2][0] = cmad(f1 * conj(h.o02), f2, conj(s02));
    E.e[2][1] = cmad(f1 * conj(h.o12), f2, conj(s12));
    return E;
}
__device__ __forceinline__ dmat expiQ(const dmat& Q) { return expiQ_h(herm_parts(Q)); }

__device__ __forceinline__ dmat reunit(const dmat& m) {
    dmat u = m;
    double n1 = rsqrt(norm2(u.e[0][0]) + norm2(u.e[0][1]) + norm2(u.e[0][2]));
    for (int k = 0; k < 3; ++k) u.e[0][k] = n1 * u.e[0][k];
    dcx ip = {0, 0};
    for (int k = 0; k < 3; ++k) ip = cmadc(ip, u.e[0][k], u.e[1][k]);
    for (int k = 0; k < 3; ++k) u.e[1][k] = u.e[1][k] - ip * u.e[0][k];
    double n2 = rsqrt(norm2(u.e[1][0]) + norm2(u.e[1][1]) + norm2(u.e[1][2]));
    for (int k = 0; k < 3; ++k) u.e[1][k] = n2 * u.e[1][k];
    u.e[2][0] = conj(u.e[0][1] * u.e[1][2] - u.e[0][2] * u.e[1][1]);
    u.e[2][1] = conj(u.e[0][2] * u.e[1][0] - u.e[0][0] * u.e[1][2]);
    u.e[2][2] = conj(u.e[0][0] * u.e[1][1] - u.e[0][1] * u.e[1][0]);
    return u;
}

}  // namespace lgt
