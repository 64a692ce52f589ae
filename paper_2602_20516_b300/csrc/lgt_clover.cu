// lgt_clover.cu -- the clover (Sheikholeslami-Wohlert) term of the Wilson-Dirac
// operator for the full-lattice pseudofermion action (a further discretisation the
// paper names in Sec. IV without a formula):
//   D_sw = 1 - kappa H + A,  A(x) = -kappa c_sw sum_{mu<nu} sigma_munu F_munu(x),
//   sigma_munu = (i/2)[g_mu, g_nu],  F_munu = (Q_munu - Q_munu^+) / (8i),
// Q_munu(x) the four plaquettes of the mu-nu plane at x, each traversed mu before
// nu from x.  In the chiral basis sigma_munu commutes with g5 = diag(1,1,-1,-1), so
// 1 + A is two 6x6 blocks per site (spins 0,1 and spins 2,3, colour fastest).
//
// Force: the clover part of delta S_f = -2 Re eta^+ (delta D) chi is
// sum_{x,mu<nu} Re tr(M_munu(x) delta Q_munu(x)) with M = -i kappa c_sw (Lambda +
// Lambda^+) / 4, Lambda_munu(x) = sum_{s,s'} (sigma_munu)_{s s'} chi_{s'}(x) eta_s(x)^+.
// Its real-component gradient for U_m(y) gathers, for every plane (m, n), the two
// plaquettes through the link and the insertion of M at each of their four
// corners: with the rest of the plaquette after the link A1 A2 A3,
//   G += (A1 A2 A3 M_0 + M_1 A1 A2 A3 + A1 M_2 A2 A3 + A1 A2 M_3 A3)^+ ,
// M_j the insertion at corner j with the sign of the plaquette's orientation
// relative to mu -> nu (mu < nu).
#include "lgt_df64.cuh"
#include "lgt_internal.h"
#include "lgt_clover.cuh"
#include "lgt_su3.cuh"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

// F_munu(x) (Hermitian) from the four leaves at x
__device__ __forceinline__ dmat field_strength(const double2* U, const Geom& g, const int x[4], int mu, int nu) {
    int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
    shift(g, xm, mu, -1);
    shift(g, xn, nu, -1);
    int xp_mu[4] = {x[0], x[1], x[2], x[3]}, xp_nu[4] = {x[0], x[1], x[2], x[3]};
    shift(g, xp_mu, mu, +1);
    shift(g, xp_nu, nu, +1);
    int xnm[4] = {xp_nu[0], xp_nu[1], xp_nu[2], xp_nu[3]};   // x + nu - mu
    shift(g, xnm, mu, -1);
    int xmn[4] = {xm[0], xm[1], xm[2], xm[3]};                // x - mu - nu
    shift(g, xmn, nu, -1);
    int xmp[4] = {xn[0], xn[1], xn[2], xn[3]};                // x - nu + mu
    shift(g, xmp, mu, +1);
    const dmat Umu = link_at(U, g, x, mu), Unu = link_at(U, g, x, nu);
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    dmat Q = mul_nd(mul_nd(mul(Umu, link_at(U, g, xp_mu, nu)), link_at(U, g, xp_nu, mu)), Unu);
    // leaf 2: U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    add_to(Q, mul(mul_nd(mul_nd(Unu, link_at(U, g, xnm, mu)), link_at(U, g, xm, nu)), link_at(U, g, xm, mu)));
    // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    add_to(Q, mul(mul(mul_dn(link_at(U, g, xm, mu), dag(link_at(U, g, xmn, nu))), link_at(U, g, xmn, mu)),
                  link_at(U, g, xn, nu)));
    // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    add_to(Q, mul_nd(mul(mul_dn(link_at(U, g, xn, nu), link_at(U, g, xn, mu)), link_at(U, g, xmp, nu)), Umu));
    dmat F;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const dcx z = Q.e[a][b] - conj(Q.e[b][a]);
            F.e[a][b] = {z.i * 0.125, -z.r * 0.125};   // z / (8i)
        }
    return F;
}

// plane p = (mu, nu), mu < nu, in the order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
__constant__ int PLANE_MU[6] = {0, 0, 0, 1, 1, 2};
__constant__ int PLANE_NU[6] = {1, 2, 3, 2, 3, 3};

// 1 + A as double2 [parity][72][Vh] (entry 36 c + 6 i + j of chiral block c) and the
// Hermitian-packed FP32 copy float4 [parity][18][Vh] (lgt_clover.cuh)
__global__ void __launch_bounds__(NT) clover_field_kernel(const double2* U, Geom g, CloverSigma S, double coef,
                                                          double2* C64, float4* C32) {
    const int t = blockIdx.x * NT + threadIdx.x;
    if (t >= 2 * g.Vh) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    int x[4];
    eo_coords(g, p, i, x);
    dcx B[2][6][6];
    for (int c = 0; c < 2; ++c)
        for (int r = 0; r < 6; ++r)
            for (int q = 0; q < 6; ++q) B[c][r][q] = {r == q ? 1.0 : 0.0, 0.0};
#pragma unroll 1
    for (int pl = 0; pl < 6; ++pl) {
        const dmat F = field_strength(U, g, x, PLANE_MU[pl], PLANE_NU[pl]);
        for (int c = 0; c < 2; ++c)
            for (int s = 0; s < 2; ++s)
                for (int u = 0; u < 2; ++u) {
                    const double2 sg = S.s[pl][c][s][u];
                    if (sg.x == 0.0 && sg.y == 0.0) continue;
                    const dcx w = coef * dcx{sg.x, sg.y};
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) B[c][3 * s + a][3 * u + b] = cmad(B[c][3 * s + a][3 * u + b], w, F.e[a][b]);
                }
    }
    double2* o64 = C64 + (size_t)p * 72 * g.Vh + i;
    float4* o32 = C32 + (size_t)p * 18 * g.Vh + i;
    for (int k = 0; k < 72; ++k) {
        const dcx v = B[k / 36][(k % 36) / 6][k % 6];
        o64[(size_t)k * g.Vh] = make_double2(v.r, v.i);
    }
    clover_store_f32(o32, g.Vh, 0, B[0]);
    clover_store_f32(o32, g.Vh, 1, B[1]);
}

cudaError_t clover_field(const double2* U, const Geom& g, const CloverSigma& S, double kappa, double csw,
                         double2* C64, float4* C32, cudaStream_t st) {
    clover_field_kernel<<<grid_for(2L * g.Vh), NT, 0, st>>>(U, g, S, -kappa * csw, C64, C32);
    count_launch();
    return cudaGetLastError();
}

// The same field from the double-float link copy, in two passes.  Pass 1 forms
// F_munu of the six planes in double-float arithmetic (the products of the leaves,
// ~94k FP32 instructions per site against ~8k FP64 FMAs, which are FP64 bound on this
// part), converts it to FP64 and stores it (double2 [parity][6 planes][9][Vh]).  Pass 2
// sums one chiral block per thread with the sigma coefficients into 1 + A.  In one
// pass the two 6 x 6 FP64 blocks of a site (144 doubles) lived in local memory.  Each
// leaf is the closed path of four steps from x (a step +d takes U_d(z), a step -d
// takes U_d(z - d)^+); one loop body over planes, leaves and steps keeps the code
// within the instruction cache.
// steps of the four leaves in terms of (mu, nu): +1 = +mu, +2 = +nu, -1 = -mu, -2 = -nu
__constant__ int LEAF_STEP[4][4] = {{1, 2, -1, -2}, {2, -1, -2, 1}, {-1, -2, 1, 2}, {-2, 1, 2, -1}};

__global__ void __launch_bounds__(NT) clover_leaves_df_kernel(const float4* U, Geom g, double2* Fout) {
    const int t = blockIdx.x * NT + threadIdx.x;
    if (t >= 2 * g.Vh) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    int x[4];
    eo_coords(g, p, i, x);
    double2* o = Fout + (size_t)p * 54 * g.Vh + i;
#pragma unroll 1
    for (int pl = 0; pl < 6; ++pl) {
        const int mu = PLANE_MU[pl], nu = PLANE_NU[pl];
        dfmat Q = df_zero3();
#pragma unroll 1
        for (int lf = 0; lf < 4; ++lf) {
            int z[4] = {x[0], x[1], x[2], x[3]};
            dfmat P;
#pragma unroll 1
            for (int st = 0; st < 4; ++st) {
                const int code = LEAF_STEP[lf][st];
                const int d = (code == 1 || code == -1) ? mu : nu;
                dfmat Lk;
                if (code > 0) {
                    Lk = link_df_op(U, g, z, d, false);
                    shift(g, z, d, +1);
                } else {
                    shift(g, z, d, -1);
                    Lk = link_df_op(U, g, z, d, true);
                }
                if (st == 0) P = Lk;
                else P = df_mul<false, false>(P, Lk);
            }
            df_add_to(Q, P);
        }
        // F = (Q - Q^+) / (8 i), in FP64
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double zr = df_to(Q.e[a][b].r) - df_to(Q.e[b][a].r);
                const double zi = df_to(Q.e[a][b].i) + df_to(Q.e[b][a].i);
                o[(size_t)(9 * pl + 3 * a + b) * g.Vh] = make_double2(zi * 0.125, -zr * 0.125);
            }
    }
}

// chiral block c of 1 + A at every site of both parities: thread t = (c, parity, site)
__global__ void __launch_bounds__(NT) clover_assemble_kernel(const double2* F, Geom g, CloverSigma S, double coef,
                                                             double2* C64, float4* C32) {
    const long t = (long)blockIdx.x * NT + threadIdx.x;
    if (t >= 4L * g.Vh) return;
    const int c = t >= 2L * g.Vh;
    const int rest = (int)(t - (long)c * 2 * g.Vh);
    const int p = rest >= g.Vh, i = rest - p * g.Vh;
    const double2* f = F + (size_t)p * 54 * g.Vh + i;
    dcx B[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int q = 0; q < 6; ++q) B[r][q] = {r == q ? 1.0 : 0.0, 0.0};
#pragma unroll 1
    for (int pl = 0; pl < 6; ++pl) {
        dcx Fp[3][3];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double2 z = __ldg(f + (size_t)(9 * pl + k) * g.Vh);
            Fp[k / 3][k % 3] = {z.x, z.y};
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const double2 sg = S.s[pl][c][s][u];
                if (sg.x == 0.0 && sg.y == 0.0) continue;
                const dcx w = coef * dcx{sg.x, sg.y};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) B[3 * s + a][3 * u + b] = cmad(B[3 * s + a][3 * u + b], w, Fp[a][b]);
            }
    }
    double2* o64 = C64 + (size_t)p * 72 * g.Vh + (size_t)(36 * c) * g.Vh + i;
#pragma unroll
    for (int k = 0; k < 36; ++k) o64[(size_t)k * g.Vh] = make_double2(B[k / 6][k % 6].r, B[k / 6][k % 6].i);
    clover_store_f32(C32 + (size_t)p * 18 * g.Vh + i, g.Vh, c, B);
}

cudaError_t clover_field_df(const float4* Udf, const Geom& g, const CloverSigma& S, double kappa, double csw,
                            double2* Fscratch, double2* C64, float4* C32, cudaStream_t st) {
    clover_leaves_df_kernel<<<grid_for(2L * g.Vh), NT, 0, st>>>(Udf, g, Fscratch);
    count_launch();
    clover_assemble_kernel<<<grid_for(4L * g.Vh), NT, 0, st>>>(Fscratch, g, S, -kappa * csw, C64, C32);
    count_launch();
    return cudaGetLastError();
}

// out = (1 + A) in on the sites of `parity` (0, 1 or 2 = both), spinor layout of the
// precision; out may not alias in
template <typename R> struct CloverIO;
template <> struct CloverIO<double> {
    static __device__ __forceinline__ void load(const void* f, int Vh, int i, dcx (&v)[12]) {
        const double2* b = (const double2*)f + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) { const double2 z = __ldg(b + (size_t)k * Vh); v[k] = {z.x, z.y}; }
    }
    static __device__ __forceinline__ void store(void* f, int Vh, int i, const dcx (&v)[12]) {
        double2* b = (double2*)f + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) b[(size_t)k * Vh] = make_double2(v[k].r, v[k].i);
    }
};
template <> struct CloverIO<float> {
    static __device__ __forceinline__ void load(const void* f, int Vh, int i, fcx (&v)[12]) {
        const float4* b = (const float4*)f + i;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 z = __ldg(b + (size_t)k * Vh);
            v[2 * k] = {z.x, z.y};
            v[2 * k + 1] = {z.z, z.w};
        }
    }
    static __device__ __forceinline__ void store(void* f, int Vh, int i, const fcx (&v)[12]) {
        float4* b = (float4*)f + i;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            b[(size_t)k * Vh] = make_float4(v[2 * k].r, v[2 * k].i, v[2 * k + 1].r, v[2 * k + 1].i);
    }
};

// chiral block c (6 x 6, row-major) of the clover field at half-field site i
template <typename R> struct CloverBlock;
template <> struct CloverBlock<double> {
    static __device__ __forceinline__ void load(const void* C, int Vh, int i, int c, dcx (&M)[6][6]) {
        const double2* b = (const double2*)C + (size_t)(36 * c) * Vh + i;
#pragma unroll
        for (int k = 0; k < 36; ++k) {
            const double2 z = __ldg(b + (size_t)k * Vh);
            M[k / 6][k % 6] = {z.x, z.y};
        }
    }
};

template <typename R>
__global__ void __launch_bounds__(NT) clover_apply_kernel(const void* C, const void* in, void* out, Geom g,
                                                          int parity, size_t cstride, size_t fstride) {
    const int t = blockIdx.x * NT + threadIdx.x;
    const int n = parity == 2 ? 2 * g.Vh : g.Vh;
    if (t >= n) return;
    const int p = parity == 2 ? (t >= g.Vh) : parity, i = parity == 2 ? t - p * g.Vh : t;
    const char* Cp = (const char*)C + p * cstride;
    const size_t fo = parity == 2 ? p * fstride : 0;
    // arithmetic in the field's precision (FP64 FMAs issue at 1/64 of the FP32 rate)
    cx<R> v[12], w[12];
    CloverIO<R>::load((const char*)in + fo, g.Vh, i, v);
    if constexpr (sizeof(R) == 4) {
        clover_mul_f32((const float4*)Cp, g.Vh, i, v, w);   // Hermitian-packed FP32 blocks
    } else {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            cx<R> M[6][6];
            CloverBlock<R>::load(Cp, g.Vh, i, c, M);
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                cx<R> s = {0, 0};
#pragma unroll
                for (int q = 0; q < 6; ++q) s = cmad(s, M[r][q], v[6 * c + q]);
                w[6 * c + r] = s;
            }
        }
    }
    CloverIO<R>::store((char*)out + fo, g.Vh, i, w);
}

cudaError_t clover_apply(const void* C, const void* in, void* out, const Geom& g, int parity, bool fp64,
                         cudaStream_t st) {
    const int n = parity == 2 ? 2 * g.Vh : g.Vh;
    if (fp64)
        clover_apply_kernel<double><<<grid_for(n), NT, 0, st>>>(C, in, out, g, parity, (size_t)72 * g.Vh * 16,
                                                                 (size_t)12 * g.Vh * 16);
    else
        clover_apply_kernel<float><<<grid_for(n), NT, 0, st>>>(C, in, out, g, parity, (size_t)18 * g.Vh * 16,
                                                                (size_t)6 * g.Vh * 16);
    count_launch();
    return cudaGetLastError();
}

// M_munu(x) = -i (kappa c_sw / 4) (Lambda + Lambda^+), Lambda_ab = sum_{s,t} sigma_{st} X_{t a} conj(Y_{s b}),
// for X, Y full FP64 fields; M as double2 [parity][6 planes][9][Vh]
__global__ void __launch_bounds__(NT) clover_insertion_kernel(const double2* X, const double2* Y, Geom g,
                                                              CloverSigma S, double c, double2* Mout) {
    const int t = blockIdx.x * NT + threadIdx.x;
    if (t >= 2 * g.Vh) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    const SpinorD Xs = load_spinor(X + (size_t)p * 12 * g.Vh, g.Vh, i);
    const SpinorD Ys = load_spinor(Y + (size_t)p * 12 * g.Vh, g.Vh, i);
    double2* o = Mout + (size_t)p * 54 * g.Vh + i;
#pragma unroll 1
    for (int pl = 0; pl < 6; ++pl) {
        dmat Lam = zero3<double>();
        for (int cb = 0; cb < 2; ++cb)
            for (int s = 0; s < 2; ++s)
                for (int u = 0; u < 2; ++u) {
                    const double2 sg = S.s[pl][cb][s][u];
                    if (sg.x == 0.0 && sg.y == 0.0) continue;
                    const dcx w = {sg.x, sg.y};
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            Lam.e[a][b] = cmad(Lam.e[a][b], w, Xs.c[2 * cb + u][a] * conj(Ys.c[2 * cb + s][b]));
                }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const dcx h = Lam.e[a][b] + conj(Lam.e[b][a]);
                o[(size_t)(pl * 9 + 3 * a + b) * g.Vh] = make_double2(c * h.i, -c * h.r);   // -i c h
            }
    }
}

cudaError_t clover_insertion(const double2* X, const double2* Y, const Geom& g, const CloverSigma& S, double kappa,
                             double csw, double2* M, cudaStream_t st) {
    clover_insertion_kernel<<<grid_for(2L * g.Vh), NT, 0, st>>>(X, Y, g, S, 0.25 * kappa * csw, M);
    count_launch();
    return cudaGetLastError();
}

__device__ __forceinline__ dmat insertion_at(const double2* M, const Geom& g, const int x[4], int pl, double sgn) {
    const int lex = lex_of(g, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const double2* b = M + (size_t)par * 54 * g.Vh + (lex >> 1);
    dmat m;
    for (int k = 0; k < 9; ++k) {
        const double2 z = __ldg(b + (size_t)(pl * 9 + k) * g.Vh);
        m.e[k / 3][k % 3] = {sgn * z.x, sgn * z.y};
    }
    return m;
}
__device__ __forceinline__ int plane_of(int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
}

// real-component gradient of the clover part for every link; form 0 writes Lie
// components out = keep*out + coef*F_a (F_a = -Im tr(lambda^a U G^+) / 2), form 1
// G-form out = keep*out + coef*G
template <int FORM>
__global__ void __launch_bounds__(NT) clover_force_kernel(const double2* U, const double2* M, Geom g, double coef,
                                                          int keep, double2* out) {
    int m, p, i;
    if (!link_index(g, m, p, i)) return;
    int y[4];
    eo_coords(g, p, i, y);
    dmat Gsum = zero3<double>();   // sum of the N (before the final ^+)
    int ym[4] = {y[0], y[1], y[2], y[3]};
    shift(g, ym, m, +1);
#pragma unroll 1
    for (int n = 0; n < 4; ++n) {
        if (n == m) continue;
        const int pl = plane_of(m, n);
        const double s = m < n ? 1.0 : -1.0;
        // plaquette above: corners y, y+m, y+m+n, y+n; A1 = U_n(y+m), A2 = U_m(y+n)^+, A3 = U_n(y)^+
        {
            int c2[4] = {ym[0], ym[1], ym[2], ym[3]};
            shift(g, c2, n, +1);
            int c3[4] = {y[0], y[1], y[2], y[3]};
            shift(g, c3, n, +1);
            const dmat A1 = link_at(U, g, ym, n);
            const dmat A2 = dag(link_at(U, g, c3, m));
            const dmat A3 = dag(link_at(U, g, y, n));
            const dmat P12 = mul(A1, A2), P23 = mul(A2, A3), P123 = mul(P12, A3);
            add_to(Gsum, mul(P123, insertion_at(M, g, y, pl, s)));
            add_to(Gsum, mul(insertion_at(M, g, ym, pl, s), P123));
            add_to(Gsum, mul(A1, mul(insertion_at(M, g, c2, pl, s), P23)));
            add_to(Gsum, mul(mul(P12, insertion_at(M, g, c3, pl, s)), A3));
        }
        // plaquette below: corners y, y+m, y+m-n, y-n; B1 = U_n(y+m-n)^+, B2 = U_m(y-n)^+, B3 = U_n(y-n)
        {
            int c2[4] = {ym[0], ym[1], ym[2], ym[3]};
            shift(g, c2, n, -1);
            int c3[4] = {y[0], y[1], y[2], y[3]};
            shift(g, c3, n, -1);
            const dmat B1 = dag(link_at(U, g, c2, n));
            const dmat B2 = dag(link_at(U, g, c3, m));
            const dmat B3 = link_at(U, g, c3, n);
            const dmat P12 = mul(B1, B2), P23 = mul(B2, B3), P123 = mul(P12, B3);
            add_to(Gsum, mul(P123, insertion_at(M, g, y, pl, -s)));
            add_to(Gsum, mul(insertion_at(M, g, ym, pl, -s), P123));
            add_to(Gsum, mul(B1, mul(insertion_at(M, g, c2, pl, -s), P23)));
            add_to(Gsum, mul(mul(P12, insertion_at(M, g, c3, pl, -s)), B3));
        }
    }
    if (FORM == 0) {
        // U G^+ with G = Gsum^+  ->  U Gsum
        const dmat UG = mul(load_link(U, g.Vh, p, m, i), Gsum);
        double c[8], f[8];
        lie_im_tr(UG, c);
        if (keep) load_mom(out, g.Vh, p, m, i, f);
        for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) - 0.5 * coef * c[a];
        store_mom(out, g.Vh, p, m, i, f);
    } else {
        dmat Go;
        if (keep) Go = load_link(out, g.Vh, p, m, i);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const dcx v = coef * conj(Gsum.e[b][a]);
                Go.e[a][b] = keep ? Go.e[a][b] + v : v;
            }
        store_link(out, g.Vh, p, m, i, Go);
    }
}

// The same gather in double-float arithmetic (Lie form): links from their double-float
// copy and the insertions from theirs (converted once per force evaluation: split on
// load they cost ~1,300 FP64-pipe operations per link), products as in the gauge
// force's double-float kernel, FP64 only in the final Lie components.
//
// The six plaquettes through U_m(y) run through one loop body.  Per plaquette the
// three other links in path order are L1 = U_n(y1)^(+), L2 = U_m(y2)^+, L3 = U_n(y3)^(+)
// (above: y1 = y+m, y2 = y3 + n... as written below; below: the mirror image, the
// conjugations taken at load time) with the insertions M0..M3 at the corners y, y+m and
// the two corners of the far side.  Its contribution, before the final ^+, is
//   L1 L2 L3 M0 + M1 L1 L2 L3 + L1 M2 L2 L3 + L1 L2 M3 L3
//     = M1 (L1 X) + L1 (L2 (M3 L3) + X M0 + M2 X),  X = L2 L3,
// eight products of 3 x 3 double-float matrices.
__device__ __forceinline__ dfmat insertion_dff_at(const float4* M, const Geom& g, const int x[4], int pl, bool neg) {
    const int lex = lex_of(g, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    const float4* b = M + (size_t)par * 54 * g.Vh + (lex >> 1);
    dfmat m;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float4 z = __ldg(b + (size_t)(pl * 9 + k) * g.Vh);
        m.e[k / 3][k % 3] = neg ? dfc{{-z.x, -z.y}, {-z.z, -z.w}} : dfc{{z.x, z.y}, {z.z, z.w}};
    }
    return m;
}
__global__ void __launch_bounds__(NT) clover_force_df_kernel(const float4* U, const float4* M, Geom g, double coef,
                                                             int keep, double2* out) {
    int m, p, i;
    if (!link_index(g, m, p, i)) return;
    int y[4];
    eo_coords(g, p, i, y);
    dfmat Gsum = df_zero3();
    int ym[4] = {y[0], y[1], y[2], y[3]};
    shift(g, ym, m, +1);
#pragma unroll 1
    for (int k = 0; k < 6; ++k) {
        const int n = (k >> 1) + ((k >> 1) >= m);   // the three directions other than m
        const bool below = k & 1;
        const int pl = plane_of(m, n);
        const bool neg = (m < n) == below;            // insertion sign: +s above, -s below
        // far corners: c2 = y + m -/+ n, c3 = y -/+ n
        int c2[4] = {ym[0], ym[1], ym[2], ym[3]};
        shift(g, c2, n, below ? -1 : +1);
        int c3[4] = {y[0], y[1], y[2], y[3]};
        shift(g, c3, n, below ? -1 : +1);
        // above: L1 = U_n(y+m), L3 = U_n(y)^+;  below: L1 = U_n(y+m-n)^+, L3 = U_n(y-n)
        const dfmat L2 = link_df_op(U, g, c3, m, true);
        const dfmat L3 = below ? link_df_op(U, g, c3, n, false) : link_df_op(U, g, y, n, true);
        dfmat X, Y, T;
        df_mul_rows(X, L2, L3, false);
        df_mul_rows(T, insertion_dff_at(M, g, c3, pl, neg), L3, false);
        df_mul_rows(Y, L2, T, false);
        df_mul_rows(Y, X, insertion_dff_at(M, g, y, pl, neg), true);
        df_mul_rows(Y, insertion_dff_at(M, g, c2, pl, neg), X, true);
        const dfmat L1 = below ? link_df_op(U, g, c2, n, true) : link_df_op(U, g, ym, n, false);
        df_mul_rows(T, L1, X, false);
        df_mul_rows(Gsum, insertion_dff_at(M, g, ym, pl, neg), T, true);
        df_mul_rows(Gsum, L1, Y, true);
    }
    const dfmat UG = df_mul<false, false>(load_link_df(U, g.Vh, p, m, i), Gsum);
    double c[8], f[8];
    lie_im_tr_df(UG, c);
    if (keep) load_mom(out, g.Vh, p, m, i, f);
#pragma unroll
    for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) - 0.5 * coef * c[a];
    store_mom(out, g.Vh, p, m, i, f);
}

cudaError_t clover_force_df(const float4* Udf, const float4* M, const Geom& g, double coef, int keep, double2* out,
                            cudaStream_t st) {
    clover_force_df_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(Udf, M, g, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t clover_force(const double2* U, const double2* M, const Geom& g, double coef, int keep, int form,
                         double2* out, cudaStream_t st) {
    if (form == 0) clover_force_kernel<0><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, M, g, coef, keep, out);
    else clover_force_kernel<1><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, M, g, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- even-odd form
// M = 1 + A on the sites of one parity: its inverse, block by block (Cholesky of the
// Hermitian positive definite 6x6 chiral block, M = L L^+, M^{-1} = L^{-+} L^{-1}), in
// the layout of the clover field, and ln det M = 2 sum ln L_ii summed over the sites
// (fixed-order reduction into the scalars' slot).
__global__ void __launch_bounds__(NT) clover_invert_kernel(const double2* C64, Geom g, int parity, double2* I64,
                                                           float4* I32, RedArgs R, int slot) {
    // every loop is unrolled, so the triangular factors are indexed at compile time and
    // stay in registers (with runtime loop indices they lived in local memory)
    const int i = blockIdx.x * NT + threadIdx.x;
    double logdet = 0.0;
    if (i < g.Vh) {
        const double2* cb = C64 + (size_t)parity * 72 * g.Vh + i;
        double2* o64 = I64 + (size_t)parity * 72 * g.Vh + i;
        float4* o32 = I32 + (size_t)parity * 18 * g.Vh + i;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            dcx L[6][6];   // lower triangle used
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
                for (int q = 0; q <= r; ++q) {
                    const double2 z = __ldg(cb + (size_t)(36 * c + 6 * r + q) * g.Vh);
                    L[r][q] = {z.x, z.y};
                }
            // Cholesky, lower triangle in place (the diagonal real and positive)
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                double dj = L[j][j].r;
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    if (k < j) dj -= L[j][k].r * L[j][k].r + L[j][k].i * L[j][k].i;
                dj = sqrt(dj);
                logdet += 2.0 * log(dj);
                L[j][j] = {dj, 0.0};
                const double inv = 1.0 / dj;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    if (r <= j) continue;
                    dcx s = L[r][j];
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        if (k < j) s = s - L[r][k] * conj(L[j][k]);
                    L[r][j] = inv * s;
                }
            }
            // W = L^{-1} (lower triangular), column by column
            dcx W[6][6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                W[q][q] = {1.0 / L[q][q].r, 0.0};
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    if (r <= q) continue;
                    dcx s = {0, 0};
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        if (k >= q && k < r) s = s + L[r][k] * W[k][q];
                    W[r][q] = (-1.0 / L[r][r].r) * s;
                }
            }
            // M^{-1} = W^+ W, and its FP32 copy Hermitian-packed (lgt_clover.cuh layout)
            float f[36];
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    dcx s = {0, 0};
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        if (k >= r && k >= q) s = cmadc(s, W[k][r], W[k][q]);
                    o64[(size_t)(36 * c + 6 * r + q) * g.Vh] = make_double2(s.r, s.i);
                    if (r == q) {
                        f[r] = (float)s.r;
                    } else if (r < q) {
                        f[clover_upper_index(r, q)] = (float)s.r;
                        f[clover_upper_index(r, q) + 1] = (float)s.i;
                    }
                }
#pragma unroll
            for (int k = 0; k < 9; ++k)
                o32[(size_t)(9 * c + k) * g.Vh] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
        }
    }
    const double b = block_sum(logdet);
    grid_reduce(b, R.partials, R.counter, R.s, RED_STORE, slot);
}

cudaError_t clover_invert(const double2* C64, const Geom& g, int parity, double2* I64, float4* I32, const RedArgs& R,
                          int slot, cudaStream_t st) {
    if (parity != 0 && parity != 1) return cudaErrorInvalidValue;
    if (grid_for(g.Vh) > R.capacity) return cudaErrorInvalidValue;
    clover_invert_kernel<<<grid_for(g.Vh), NT, 0, st>>>(C64, g, parity, I64, I32, R, slot);
    count_launch();
    return cudaGetLastError();
}

// The determinant term -2 ln det M of one parity: its variation -2 tr(M^{-1} delta A)
// has the form of -2 Re eta^+ delta A chi with chi eta^+ replaced by M^{-1}, so
//   Lambda_ab += sum_{s,t} sigma_{st} (M^{-1})_{(t a),(s b)}
// and M_munu += -i (kappa c_sw / 4) (Lambda + Lambda^+) on the sites of that parity.
__global__ void __launch_bounds__(NT) clover_det_insertion_kernel(const double2* I64, Geom g, int parity,
                                                                  CloverSigma S, double c, double2* Mout) {
    const int i = blockIdx.x * NT + threadIdx.x;
    if (i >= g.Vh) return;
    const double2* ib = I64 + (size_t)parity * 72 * g.Vh + i;
    double2* o = Mout + (size_t)parity * 54 * g.Vh + i;
#pragma unroll 1
    for (int pl = 0; pl < 6; ++pl) {
        dmat Lam = zero3<double>();
        for (int cb = 0; cb < 2; ++cb)
            for (int s = 0; s < 2; ++s)
                for (int u = 0; u < 2; ++u) {
                    const double2 sg = S.s[pl][cb][s][u];
                    if (sg.x == 0.0 && sg.y == 0.0) continue;
                    const dcx w = {sg.x, sg.y};
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) {
                            const double2 z = __ldg(ib + (size_t)(36 * cb + 6 * (3 * u + a) + 3 * s + b) * g.Vh);
                            Lam.e[a][b] = cmad(Lam.e[a][b], w, dcx{z.x, z.y});
                        }
                }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const dcx h = Lam.e[a][b] + conj(Lam.e[b][a]);
                double2 v = o[(size_t)(pl * 9 + 3 * a + b) * g.Vh];
                v.x += c * h.i;   // -i c h
                v.y -= c * h.r;
                o[(size_t)(pl * 9 + 3 * a + b) * g.Vh] = v;
            }
    }
}

cudaError_t clover_det_insertion(const double2* I64, const Geom& g, int parity, const CloverSigma& S, double kappa,
                                 double csw, double2* M, cudaStream_t st) {
    if (parity != 0 && parity != 1) return cudaErrorInvalidValue;
    clover_det_insertion_kernel<<<grid_for(g.Vh), NT, 0, st>>>(I64, g, parity, S, 0.25 * kappa * csw, M);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
