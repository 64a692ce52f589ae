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
// exp(iQ) for Hermitian traceless Q.  With c0 = det Q, c1 = tr(Q^2)/2, the
// Cayley-Hamilton coefficients f_j give exp(iQ) = f0 + f1 Q + f2 Q^2; c0 < 0 is
// mapped to c0 > 0 by f_j(-c0) = (-1)^j conj(f_j(c0)).  Small Q uses the Taylor
// series, where the closed form loses digits to cancellation.
__device__ __forceinline__ dmat expiQ(const dmat& Q) {
    dmat Q2 = mul(Q, Q);
    double c1 = 0.5 * retrace(Q2);
    dmat R;
    if (c1 < 1e-3) {
        // Horner: 1 + iQ (1 + iQ/2 (1 + iQ/3 (...)))
        R = zero3<double>();
        for (int a = 0; a < 3; ++a) R.e[a][a] = {1.0, 0.0};
        for (int k = 12; k >= 1; --k) {
            dmat T = mul(Q, R);
            double s = 1.0 / k;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) R.e[a][b] = {-s * T.e[a][b].i, s * T.e[a][b].r};
            for (int a = 0; a < 3; ++a) R.e[a][a].r += 1.0;
        }
        return R;
    }
    // c0 = det Q = tr(Q^3) / 3: only the trace of Q Q^2 is needed
    double c0 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) c0 = fma(Q.e[a][b].r, Q2.e[b][a].r, fma(-Q.e[a][b].i, Q2.e[b][a].i, c0));
    c0 *= (1.0 / 3.0);
    const bool neg = c0 < 0;
    if (neg) c0 = -c0;
    const double c1_3 = c1 * (1.0 / 3.0);
    double c0max = 2.0 * c1_3 * sqrt(c1_3);
    double ratio = fmin(c0 / c0max, 1.0);
    double theta = acos(ratio);
    double sq = sqrt(c1);
    double st, ct;
    sincos(theta * (1.0 / 3.0), &st, &ct);
    double u = sq * (1.0 / 1.7320508075688772935) * ct;
    double w = sq * st;
    double u2 = u * u, w2 = w * w;
    double sw, cw;
    sincos(w, &sw, &cw);
    double xi0 = (fabs(w) < 0.05) ? 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)) : sw / w;
    double su, cu;
    sincos(u, &su, &cu);
    // e^{2iu} from e^{iu} by the double-angle identities
    double c2u = fma(cu, cu, -su * su), s2u = 2.0 * su * cu;
    dcx e2iu = {c2u, s2u};
    dcx emiu = {cu, -su};
    dcx h0 = (u2 - w2) * e2iu + emiu * dcx{8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0};
    dcx h1 = (2.0 * u) * e2iu - emiu * dcx{2.0 * u * cw, -(3.0 * u2 - w2) * xi0};
    dcx h2 = e2iu - emiu * dcx{cw, 3.0 * u * xi0};
    double den = 1.0 / (9.0 * u2 - w2);
    dcx f0 = den * h0, f1 = den * h1, f2 = den * h2;
    if (neg) { f0 = conj(f0); f1 = -conj(f1); f2 = conj(f2); }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            dcx v = f1 * Q.e[a][b];
            v = cmad(v, f2, Q2.e[a][b]);
            if (a == b) v = v + f0;
            R.e[a][b] = v;
        }
    return R;
}

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
