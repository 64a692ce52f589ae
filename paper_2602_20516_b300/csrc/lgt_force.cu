// lgt_force.cu -- Wilson pseudofermion force on sm_103a.
//
// delta S_f = -2 Re[Y^+ (delta D) X] (Eq. S3.12, with chi -> X and eta -> Y; for
// the even-odd action X = (chi_e, kappa H_oe chi_e), Y = (eta_e, kappa (H^+)_oe eta_e)).
// U_mu(x) enters Y^+ H X twice, giving the two colour matrices
//   P1 = b sum_s [(1 - g_mu) X(x+mu)]_s Y(x)_s^+ ,  P2 = b sum_s X(x)_s [(1 + g_mu) Y(x+mu)]_s^+ .
// Because (1 -+ g)/2 is a Hermitian projector of rank 2, each sum is two outer
// products of projected colour vectors: sum_s (P X)_s (Y_s)^+ = sum_j h_j(X) h_j(Y)^+.
// Lie form:  W = U P1 - P2 U^+,  F_a = -2 kappa Im tr(T^a W)  (= i kappa P[W], Eq. 9),
//            with U P1 and P2 U^+ formed from the projected rows (see w_matrix);
// G form:    G = dS/dReU + i dS/dImU = 2 kappa (P1^+ + P2)      (Eq. S2.11).
// One thread per link; X(x), Y(x) are re-read per direction through L1/L2.
// The FP64 kernel serves the FP64 path and the G form; the mixed-precision MD path
// uses FP32 arithmetic (FP32 X, Y and two-row links) accumulated into FP64 momenta.
#include "lgt_internal.h"
#include "lgt_spin.cuh"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

template <int MU, typename R>
__device__ __forceinline__ void outer_terms(const cx<R> (&Xx)[4][3], const cx<R> (&Yx)[4][3],
                                            const cx<R> (&Xy)[4][3], const cx<R> (&Yy)[4][3], R b, mat3<R>& P1,
                                            mat3<R>& P2) {
    cx<R> h[2][3], k[2][3];
    project<MU, -1>(Xy, h);
    project<MU, -1>(Yx, k);
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            cx<R> s = {0, 0};
            s = cmad_cb(s, h[0][a], k[0][c]);
            s = cmad_cb(s, h[1][a], k[1][c]);
            P1.e[a][c] = b * s;
        }
    project<MU, +1>(Xx, h);
    project<MU, +1>(Yy, k);
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            cx<R> s = {0, 0};
            s = cmad_cb(s, h[0][a], k[0][c]);
            s = cmad_cb(s, h[1][a], k[1][c]);
            P2.e[a][c] = b * s;
        }
}

template <typename R>
__device__ __forceinline__ void outer_dispatch(int mu, const cx<R> (&Xx)[4][3], const cx<R> (&Yx)[4][3],
                                               const cx<R> (&Xy)[4][3], const cx<R> (&Yy)[4][3], R b,
                                               mat3<R>& P1, mat3<R>& P2) {
    switch (mu) {
    case 0: outer_terms<0, R>(Xx, Yx, Xy, Yy, b, P1, P2); break;
    case 1: outer_terms<1, R>(Xx, Yx, Xy, Yy, b, P1, P2); break;
    case 2: outer_terms<2, R>(Xx, Yx, Xy, Yy, b, P1, P2); break;
    default: outer_terms<3, R>(Xx, Yx, Xy, Yy, b, P1, P2); break;
    }
}

// W = U P1 - P2 U^+ without forming P1, P2: with h_j, k_j the projected rows,
//   U P1 = b sum_j (U h_j(X(x+mu))) k_j(Y(x))^+,   P2 U^+ = b sum_j h_j(X(x)) (U k_j(Y(x+mu)))^+
// (four colour mat-vecs and four outer products instead of two outer products and two
// 3x3 products); the boundary sign b is applied by the caller.
template <int MU, typename R>
__device__ __forceinline__ void w_matrix(const mat3<R>& U, const cx<R> (&Xx)[4][3], const cx<R> (&Yx)[4][3],
                                         const cx<R> (&Xy)[4][3], const cx<R> (&Yy)[4][3], mat3<R>& W) {
    cx<R> h[2][3], k[2][3], m[2][3];
    project<MU, -1>(Xy, h);
    project<MU, -1>(Yx, k);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> v = U.e[a][0] * h[j][0];
            v = cmad(v, U.e[a][1], h[j][1]);
            m[j][a] = cmad(v, U.e[a][2], h[j][2]);
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<R> v = {0, 0};
            v = cmad_cb(v, m[0][a], k[0][c]);
            W.e[a][c] = cmad_cb(v, m[1][a], k[1][c]);
        }
    project<MU, +1>(Xx, h);
    project<MU, +1>(Yy, k);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> v = U.e[a][0] * k[j][0];
            v = cmad(v, U.e[a][1], k[j][1]);
            m[j][a] = cmad(v, U.e[a][2], k[j][2]);
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx<R> v = W.e[a][c];
            v = cmad_cb(v, -h[0][a], m[0][c]);
            W.e[a][c] = cmad_cb(v, -h[1][a], m[1][c]);
        }
}

template <typename R>
__device__ __forceinline__ void w_dispatch(int mu, const mat3<R>& U, const cx<R> (&Xx)[4][3],
                                           const cx<R> (&Yx)[4][3], const cx<R> (&Xy)[4][3],
                                           const cx<R> (&Yy)[4][3], mat3<R>& W) {
    switch (mu) {
    case 0: w_matrix<0, R>(U, Xx, Yx, Xy, Yy, W); break;
    case 1: w_matrix<1, R>(U, Xx, Yx, Xy, Yy, W); break;
    case 2: w_matrix<2, R>(U, Xx, Yx, Xy, Yy, W); break;
    default: w_matrix<3, R>(U, Xx, Yx, Xy, Yy, W); break;
    }
}

template <int FORM>
__global__ void __launch_bounds__(NT) fermion_force_kernel(const double2* U, const double2* X, const double2* Y,
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
    SpinorD Xx = load_spinor(X + p * hf, g.Vh, i), Yx = load_spinor(Y + p * hf, g.Vh, i);
    SpinorD Xy = load_spinor(X + (1 - p) * hf, g.Vh, j), Yy = load_spinor(Y + (1 - p) * hf, g.Vh, j);
    if (FORM == 0) {
        dmat W;
        w_dispatch<double>(mu, load_link(U, g.Vh, p, mu, i), Xx.c, Yx.c, Xy.c, Yy.c, W);
        double cl[8], f[8];
        lie_im_tr(W, cl);
        if (keep) load_mom(out, g.Vh, p, mu, i, f);
        const double s = -coef * kappa * b;
        for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) + s * cl[a];
        store_mom(out, g.Vh, p, mu, i, f);
    } else {
        dmat P1, P2;
        outer_dispatch<double>(mu, Xx.c, Yx.c, Xy.c, Yy.c, b, P1, P2);
        dmat G;
        if (keep) G = load_link(out, g.Vh, p, mu, i);
        const double s = 2.0 * kappa * coef;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                dcx v = s * (conj(P1.e[c][a]) + P2.e[a][c]);
                G.e[a][c] = keep ? G.e[a][c] + v : v;
            }
        store_link(out, g.Vh, p, mu, i, G);
    }
}

// FP32 arithmetic (X, Y: float4 [2][6][Vh]; links: two-row FP32), FP64 accumulation
__global__ void __launch_bounds__(NT) fermion_force_fp32_kernel(const float4* U12, const float4* X, const float4* Y,
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
    const float b = (mu == 3 && x[3] == g.L[3] - 1) ? -1.f : 1.f;
    const size_t hf = (size_t)6 * g.Vh;
    SpinorF Xx = load_spinor(X + p * hf, g.Vh, i), Yx = load_spinor(Y + p * hf, g.Vh, i);
    SpinorF Xy = load_spinor(X + (1 - p) * hf, g.Vh, j), Yy = load_spinor(Y + (1 - p) * hf, g.Vh, j);
    mat3<float> W;
    w_dispatch<float>(mu, load_link12(U12, g.Vh, p, mu, i), Xx.c, Yx.c, Xy.c, Yy.c, W);
    float cl[8];
    lie_im_tr(W, cl);
    double f[8];
    if (keep) load_mom(out, g.Vh, p, mu, i, f);
    const double s = -coef * kappa * (double)b;
    for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) + s * (double)cl[a];
    store_mom(out, g.Vh, p, mu, i, f);
}

cudaError_t fermion_force(const double2* U, const double2* X, const double2* Y, const Geom& g, double kappa,
                          double coef, int keep, int form, double2* out, cudaStream_t st) {
    if (form == 0) fermion_force_kernel<0><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, X, Y, g, kappa, coef, keep, out);
    else fermion_force_kernel<1><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, X, Y, g, kappa, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t fermion_force_fp32(const float4* U12, const float4* X, const float4* Y, const Geom& g, double kappa,
                               double coef, int keep, double2* out, cudaStream_t st) {
    fermion_force_fp32_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(U12, X, Y, g, kappa, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
