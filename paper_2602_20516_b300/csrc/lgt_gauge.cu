// lgt_gauge.cu -- gauge-field kernels: layout conversion, seeded fields,
// exp(iQ) (Cayley-Hamilton form of Morningstar & Peardon 2004), the Wilson
// plaquette action, the staple force (Eq. 9 applied to S_G), the left link
// update of Eq. S2.1 and the momentum heatbath / kinetic energy.
//
// The staple force and action also take the rectangle term of the improved
// gauge actions (weight c1, plaquette weight c0 = 1 - 8 c1).
// Link kernels run one thread per link with the site index fastest, so the
// SoA loads of a warp are contiguous.  The FP64 staple force and the exponential
// are FP64-ALU bound on this part; they are written for FMA throughput.
#include "lgt_internal.h"
#include "lgt_su3.cuh"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

// ---------------------------------------------------------------- layouts
template <bool WITH12>
__global__ void __launch_bounds__(NT) pack_links_kernel(double2* U, float4* U12, const double2* canon, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    int lex = eo_coords(g, p, i, x);
    const double2* c = canon + ((size_t)lex * 4 + mu) * 9;
    dmat m;
    for (int k = 0; k < 9; ++k) { double2 v = c[k]; m.e[k / 3][k % 3] = {v.x, v.y}; }
    store_link(U, g.Vh, p, mu, i, m);
    if (WITH12) store_link12(U12, g.Vh, p, mu, i, m);
}
__global__ void __launch_bounds__(NT) unpack_links_kernel(double2* canon, const double2* U, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    int lex = eo_coords(g, p, i, x);
    dmat m = load_link(U, g.Vh, p, mu, i);
    double2* c = canon + ((size_t)lex * 4 + mu) * 9;
    for (int k = 0; k < 9; ++k) c[k] = make_double2(m.e[k / 3][k % 3].r, m.e[k / 3][k % 3].i);
}

cudaError_t gauge_pack_links(double2* U, float4* U12, const double2* canon, const Geom& g, cudaStream_t st) {
    pack_links_kernel<true><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, U12, canon, g);
    count_launch();
    return cudaGetLastError();
}
cudaError_t gauge_pack_field(double2* F, const double2* canon, const Geom& g, cudaStream_t st) {
    pack_links_kernel<false><<<grid_for(8L * g.Vh), NT, 0, st>>>(F, nullptr, canon, g);
    count_launch();
    return cudaGetLastError();
}
cudaError_t gauge_unpack_links(double* canon, const double2* U, const Geom& g, cudaStream_t st) {
    unpack_links_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>((double2*)canon, U, g);
    count_launch();
    return cudaGetLastError();
}
cudaError_t gauge_unpack_field(double* canon, const double2* F, const Geom& g, cudaStream_t st) {
    return gauge_unpack_links(canon, F, g, st);
}

__global__ void __launch_bounds__(NT) make12_kernel(float4* U12, const double2* U, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    store_link12(U12, g.Vh, p, mu, i, load_link(U, g.Vh, p, mu, i));
}
cudaError_t gauge_make12(float4* U12, const double2* U, const Geom& g, cudaStream_t st) {
    make12_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(U12, U, g);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) unit_kernel(double2* U, float4* U12, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    dmat m = zero3<double>();
    for (int a = 0; a < 3; ++a) m.e[a][a] = {1.0, 0.0};
    store_link(U, g.Vh, p, mu, i, m);
    store_link12(U12, g.Vh, p, mu, i, m);
}
cudaError_t gauge_unit(double2* U, float4* U12, const Geom& g, cudaStream_t st) {
    unit_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(U, U12, g);
    count_launch();
    return cudaGetLastError();
}

// U = exp(i alpha sum_a h_a T^a), h from Philox counter (4 s + mu, j, 0, FIELD_LINKS)
__global__ void __launch_bounds__(NT) random_links_kernel(double2* U, float4* U12, Geom g, uint64_t seed,
                                                          double alpha) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    int lex = eo_coords(g, p, i, x);
    double h[8];
    for (int j = 0; j < 4; ++j) gauss_pair(seed, (uint32_t)(4 * lex + mu), j, 0, FIELD_LINKS, h[2 * j], h[2 * j + 1]);
    for (int a = 0; a < 8; ++a) h[a] *= alpha;
    dmat m = expiQ_h(herm_parts_lie(h));
    store_link(U, g.Vh, p, mu, i, m);
    store_link12(U12, g.Vh, p, mu, i, m);
}
cudaError_t gauge_random(double2* U, float4* U12, const Geom& g, uint64_t seed, double alpha, cudaStream_t st) {
    random_links_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(U, U12, g, seed, alpha);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) reunit_kernel(double2* U, float4* U12, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    dmat m = reunit(load_link(U, g.Vh, p, mu, i));
    store_link(U, g.Vh, p, mu, i, m);
    store_link12(U12, g.Vh, p, mu, i, m);
}
cudaError_t gauge_reunitarise(double2* U, float4* U12, const Geom& g, cudaStream_t st) {
    reunit_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(U, U12, g);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- plaquette
__global__ void __launch_bounds__(NT) plaquette_kernel(const double2* U, Geom g, RedArgs R, int slot) {
    const int t = blockIdx.x * NT + threadIdx.x;
    double acc = 0.0;
    if (t < 2 * g.Vh) {
        const int p = t >= g.Vh, i = t - p * g.Vh;
        int x[4];
        eo_coords(g, p, i, x);
        for (int mu = 0; mu < 4; ++mu) {
            dmat Umu = load_link(U, g.Vh, p, mu, i);
            int xm[4] = {x[0], x[1], x[2], x[3]};
            shift(g, xm, mu, +1);
            for (int nu = mu + 1; nu < 4; ++nu) {
                int xn[4] = {x[0], x[1], x[2], x[3]};
                shift(g, xn, nu, +1);
                dmat a = mul(Umu, link_at(U, g, xm, nu));
                dmat b = mul_nd(a, link_at(U, g, xn, mu));
                dmat c = mul_nd(b, load_link(U, g.Vh, p, nu, i));
                acc += retrace(c);
            }
        }
        acc *= (1.0 / 3.0);
    }
    double bs = block_sum(acc);
    grid_reduce(bs, R.partials, R.counter, R.s, RED_STORE, slot);
}
cudaError_t gauge_plaquette(const double2* U, const Geom& g, const RedArgs& R, int slot, cudaStream_t st) {
    if (grid_for(2L * g.Vh) > R.capacity) return cudaErrorInvalidValue;   // partials too small
    plaquette_kernel<<<grid_for(2L * g.Vh), NT, 0, st>>>(U, g, R, slot);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- staple force
// V_mu(x) = sum_nu [U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)]
// d_a S_G = (beta/3) Im tr(T^a U V) = (beta/6) Im tr(lambda^a U V);  G = -(beta/3) V^+
// link loads by precision: FP64 18-real links or FP32 two-row links
template <typename R> struct GLink;
template <> struct GLink<double> {
    static __device__ __forceinline__ dmat at(const void* U, const Geom& g, const int x[4], int mu) {
        return link_at((const double2*)U, g, x, mu);
    }
};
template <> struct GLink<float> {
    static __device__ __forceinline__ mat3<float> at(const void* U, const Geom& g, const int x[4], int mu) {
        int lex = lex_of(g, x);
        return load_link12((const float4*)U, g.Vh, (x[0] + x[1] + x[2] + x[3]) & 1, mu, lex >> 1);
    }
};

template <typename R>
__device__ __forceinline__ mat3<R> staple_sum(const void* U, const Geom& g, const int x[4], int mu) {
    mat3<R> V = zero3<R>();
    int xp[4] = {x[0], x[1], x[2], x[3]};
    shift(g, xp, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int xpn[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xpn, nu, +1);
        int xmn[4] = {x[0], x[1], x[2], x[3]};
        shift(g, xmn, nu, -1);
        int xpmn[4] = {xp[0], xp[1], xp[2], xp[3]};
        shift(g, xpmn, nu, -1);
        mat3<R> Unx = GLink<R>::at(U, g, x, nu);
        mat3<R> a = mul_nd(GLink<R>::at(U, g, xp, nu), GLink<R>::at(U, g, xpn, mu));
        add_to(V, mul_nd(a, Unx));
        mat3<R> b = mul_dn(GLink<R>::at(U, g, xpmn, nu), dag(GLink<R>::at(U, g, xmn, mu)));
        add_to(V, mul(b, GLink<R>::at(U, g, xmn, nu)));
    }
    return V;
}

// ---------------------------------------------------------------- rectangle staples
// The rectangle-improved action adds c1 sum_{x, mu != nu} (1 - Re tr R_munu(x) / 3),
// R_munu the 2 x 1 loop with its long side along mu (plaquette weight c0 = 1 - 8 c1).
// The six rectangles per nu through U_mu(x), each walked from x + mu after the step
// along U_mu(x): a step +d moves along U_d(y), a step -d moves back with U_d(y-d)^+.
__constant__ signed char RECT_WALKS[6][5] = {
    {'m', 'n', 'M', 'M', 'N'},   // long side mu above, U_mu(x) first
    {'n', 'M', 'M', 'N', 'm'},   // long side mu above, U_mu(x) second
    {'m', 'N', 'M', 'M', 'n'},   // long side mu below, U_mu(x) first
    {'N', 'M', 'M', 'n', 'm'},   // long side mu below, U_mu(x) second
    {'n', 'n', 'M', 'N', 'N'},   // long side nu, above
    {'N', 'N', 'M', 'n', 'n'},   // long side nu, below
};
template <typename R>
__device__ __forceinline__ mat3<R> walk5(const void* U, const Geom& g, const int x0[4], int mu, int nu,
                                         const signed char* w) {
    int y[4] = {x0[0], x0[1], x0[2], x0[3]};
    shift(g, y, mu, +1);
    mat3<R> acc;
#pragma unroll 1
    for (int k = 0; k < 5; ++k) {
        const char c = w[k];
        const int d = (c == 'm' || c == 'M') ? mu : nu;
        mat3<R> L;
        if (c == 'm' || c == 'n') {
            L = GLink<R>::at(U, g, y, d);
            shift(g, y, d, +1);
            acc = (k == 0) ? L : mul(acc, L);
        } else {
            shift(g, y, d, -1);
            L = GLink<R>::at(U, g, y, d);
            acc = (k == 0) ? dag(L) : mul_nd(acc, L);
        }
    }
    return acc;
}
// V_mu(x) = c0 (plaquette staples) + c1 (rectangle staples)
template <typename R>
__device__ __forceinline__ mat3<R> staple_sum_imp(const void* U, const Geom& g, const int x[4], int mu, double c1) {
    mat3<R> V = staple_sum<R>(U, g, x, mu);
    if (c1 == 0.0) return V;
    const R c0 = (R)(1.0 - 8.0 * c1), r1 = (R)c1;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) V.e[a][b] = c0 * V.e[a][b];
#pragma unroll 1
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
#pragma unroll 1
        for (int k = 0; k < 6; ++k) {
            const mat3<R> S = walk5<R>(U, g, x, mu, nu, RECT_WALKS[k]);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) V.e[a][b] = V.e[a][b] + r1 * S.e[a][b];
        }
    }
    return V;
}

// Lie form: out = keep*out + coef*(beta/6) Im tr(lambda^a U V), accumulated in FP64
// whatever the arithmetic precision R of the staples.
template <typename R>
__global__ void __launch_bounds__(NT) gauge_force_lie_kernel(const void* U, Geom g, double beta, double c1,
                                                             double coef, int keep, double2* out) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    eo_coords(g, p, i, x);
    mat3<R> V = staple_sum_imp<R>(U, g, x, mu, c1);
    mat3<R> M = mul(GLink<R>::at(U, g, x, mu), V);
    R c[8];
    lie_im_tr(M, c);
    double f[8];
    if (keep) load_mom(out, g.Vh, p, mu, i, f);
    const double s = coef * beta / 6.0;
    for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) + s * (double)c[a];
    store_mom(out, g.Vh, p, mu, i, f);
}

template <int FORM>
__global__ void __launch_bounds__(NT) gauge_force_kernel(const double2* U, Geom g, double beta, double c1,
                                                         double coef, int keep, double2* out) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    eo_coords(g, p, i, x);
    dmat V = staple_sum_imp<double>(U, g, x, mu, c1);
    if (FORM == 0) {
        dmat M = mul(load_link(U, g.Vh, p, mu, i), V);
        double c[8];
        lie_im_tr(M, c);
        double f[8];
        if (keep) load_mom(out, g.Vh, p, mu, i, f);
        const double s = coef * beta / 6.0;
        for (int a = 0; a < 8; ++a) f[a] = (keep ? f[a] : 0.0) + s * c[a];
        store_mom(out, g.Vh, p, mu, i, f);
    } else {
        const double s = -coef * beta / 3.0;
        dmat G;
        if (keep) G = load_link(out, g.Vh, p, mu, i);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                dcx v = s * conj(V.e[b][a]);
                G.e[a][b] = keep ? G.e[a][b] + v : v;
            }
        store_link(out, g.Vh, p, mu, i, G);
    }
}
cudaError_t gauge_force(const double2* U, const Geom& g, double beta, double c1, double coef, int keep, int form,
                        double2* out, cudaStream_t st) {
    if (form == 0) gauge_force_kernel<0><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, g, beta, c1, coef, keep, out);
    else gauge_force_kernel<1><<<grid_for(8L * g.Vh), NT, 0, st>>>(U, g, beta, c1, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}
cudaError_t gauge_force_fp32(const float4* U12, const Geom& g, double beta, double c1, double coef, int keep,
                             double2* out, cudaStream_t st) {
    gauge_force_lie_kernel<float><<<grid_for(8L * g.Vh), NT, 0, st>>>(U12, g, beta, c1, coef, keep, out);
    count_launch();
    return cudaGetLastError();
}

// sum over x and ordered mu != nu of Re tr R_munu(x) / 3: the loop from x is the link
// U_mu(x) followed by the walk of the first rectangle (long side mu, above)
__global__ void __launch_bounds__(NT) rectangle_kernel(const double2* U, Geom g, RedArgs R, int slot) {
    const int t = blockIdx.x * NT + threadIdx.x;
    double acc = 0.0;
    if (t < 2 * g.Vh) {
        const int p = t >= g.Vh, i = t - p * g.Vh;
        int x[4];
        eo_coords(g, p, i, x);
#pragma unroll 1
        for (int mu = 0; mu < 4; ++mu) {
            const dmat Umu = load_link(U, g.Vh, p, mu, i);
#pragma unroll 1
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                const dmat S = walk5<double>(U, g, x, mu, nu, RECT_WALKS[0]);
                // Re tr(U S) from the diagonal of the product
                double tr = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        tr = fma(Umu.e[a][b].r, S.e[b][a].r, fma(-Umu.e[a][b].i, S.e[b][a].i, tr));
                acc += tr;
            }
        }
        acc *= (1.0 / 3.0);
    }
    double bs = block_sum(acc);
    grid_reduce(bs, R.partials, R.counter, R.s, RED_STORE, slot);
}
cudaError_t gauge_rectangles(const double2* U, const Geom& g, const RedArgs& R, int slot, cudaStream_t st) {
    if (grid_for(2L * g.Vh) > R.capacity) return cudaErrorInvalidValue;
    rectangle_kernel<<<grid_for(2L * g.Vh), NT, 0, st>>>(U, g, R, slot);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- link update
__global__ void __launch_bounds__(NT) update_links_kernel(double2* U, float4* U12, const double2* mom, double eps,
                                                          Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    double pi[8];
    load_mom(mom, g.Vh, p, mu, i, pi);
    for (int a = 0; a < 8; ++a) pi[a] *= eps;
    dmat E = expiQ_h(herm_parts_lie(pi));
    dmat m = mul(E, load_link(U, g.Vh, p, mu, i));
    store_link(U, g.Vh, p, mu, i, m);
    store_link12(U12, g.Vh, p, mu, i, m);
}
cudaError_t gauge_update_links(double2* U, float4* U12, const double2* mom, double eps, const Geom& g,
                               cudaStream_t st) {
    update_links_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(U, U12, mom, eps, g);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- momenta
__global__ void __launch_bounds__(NT) momenta_kernel(double2* mom, Geom g, uint64_t seed, uint32_t traj) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    int lex = eo_coords(g, p, i, x);
    double v[8];
    for (int j = 0; j < 4; ++j) gauss_pair(seed, (uint32_t)(4 * lex + mu), j, traj, FIELD_MOMENTA, v[2 * j], v[2 * j + 1]);
    store_mom(mom, g.Vh, p, mu, i, v);
}
cudaError_t gauge_momenta_heatbath(double2* mom, const Geom& g, uint64_t seed, uint32_t traj, cudaStream_t st) {
    momenta_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(mom, g, seed, traj);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) kinetic_kernel(const double2* mom, Geom g, RedArgs R, int slot) {
    int mu, p, i;
    double acc = 0.0;
    if (link_index(g, mu, p, i)) {
        double v[8];
        load_mom(mom, g.Vh, p, mu, i, v);
        for (int a = 0; a < 8; ++a) acc += v[a] * v[a];
        acc *= 0.5;
    }
    double bs = block_sum(acc);
    grid_reduce(bs, R.partials, R.counter, R.s, RED_STORE, slot);
}
cudaError_t gauge_kinetic(const double2* mom, const Geom& g, const RedArgs& R, int slot, cudaStream_t st) {
    if (grid_for(8L * g.Vh) > R.capacity) return cudaErrorInvalidValue;   // one partial per block of links
    kinetic_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(mom, g, R, slot);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) kick_kernel(double2* mom, const double2* F, double eps, long ne) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    double2 m = mom[e], f = __ldg(F + e);
    m.x = fma(-eps, f.x, m.x);
    m.y = fma(-eps, f.y, m.y);
    mom[e] = m;
}
cudaError_t gauge_kick(double2* mom, const double2* F, double eps, const Geom& g, cudaStream_t st) {
    long ne = 32L * g.Vh;
    kick_kernel<<<grid_for(ne), NT, 0, st>>>(mom, F, eps, ne);
    count_launch();
    return cudaGetLastError();
}

// F_a = Re tr(G^+ i T^a U) = -(1/2) Im tr(lambda^a U G^+)
__global__ void __launch_bounds__(NT) grad_to_lie_kernel(double2* F, const double2* G, const double2* U, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    dmat M = mul_nd(load_link(U, g.Vh, p, mu, i), load_link(G, g.Vh, p, mu, i));
    double c[8];
    lie_im_tr(M, c);
    for (int a = 0; a < 8; ++a) c[a] *= -0.5;
    store_mom(F, g.Vh, p, mu, i, c);
}
cudaError_t grad_to_lie(double2* F, const double2* G, const double2* U, const Geom& g, cudaStream_t st) {
    grad_to_lie_kernel<<<grid_for(8L * g.Vh), NT, 0, st>>>(F, G, U, g);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- spinors
// complex Gaussian, Re/Im ~ N(0,1/2), counter (s, component, traj, field)
__global__ void __launch_bounds__(NT) spinor_gauss_kernel(double2* f, Geom g, int parity, uint64_t seed,
                                                          uint32_t traj, uint32_t field) {
    const int t = blockIdx.x * NT + threadIdx.x;
    const int n = parity == 2 ? 2 * g.Vh : g.Vh;
    if (t >= n) return;
    int p, i;
    if (parity == 2) { p = t >= g.Vh; i = t - p * g.Vh; }
    else { p = parity; i = t; }
    int x[4];
    int lex = eo_coords(g, p, i, x);
    double2* b = f + (parity == 2 ? (size_t)p * 12 * g.Vh : 0) + i;
    const double s = 0.70710678118654752440;
    for (int k = 0; k < 12; ++k) {
        double g0, g1;
        gauss_pair(seed, (uint32_t)lex, k, traj, field, g0, g1);
        b[(size_t)k * g.Vh] = make_double2(s * g0, s * g1);
    }
}
cudaError_t spinor_gaussian(double2* f, const Geom& g, int parity, uint64_t seed, uint32_t traj, uint32_t field,
                            cudaStream_t st) {
    spinor_gauss_kernel<<<grid_for(parity == 2 ? 2L * g.Vh : (long)g.Vh), NT, 0, st>>>(f, g, parity, seed, traj,
                                                                                       field);
    count_launch();
    return cudaGetLastError();
}

template <bool PACK, bool FP64>
__global__ void __launch_bounds__(NT) spinor_layout_kernel(void* field, double2* canon, Geom g, int parity) {
    const int t = blockIdx.x * NT + threadIdx.x;
    const int n = parity == 2 ? 2 * g.Vh : g.Vh;
    if (t >= n) return;
    int p, i;
    if (parity == 2) { p = t >= g.Vh; i = t - p * g.Vh; }
    else { p = parity; i = t; }
    int x[4];
    int lex = eo_coords(g, p, i, x);
    double2* c = canon + (size_t)lex * 12;
    const size_t off = parity == 2 ? (size_t)p * (FP64 ? 12 : 6) * g.Vh : 0;
    if (FP64) {
        double2* b = (double2*)field + off + i;
        for (int k = 0; k < 12; ++k) {
            if (PACK) b[(size_t)k * g.Vh] = c[k];
            else c[k] = b[(size_t)k * g.Vh];
        }
    } else {
        float4* b = (float4*)field + off + i;
        for (int k = 0; k < 6; ++k) {
            if (PACK) {
                double2 u = c[2 * k], v = c[2 * k + 1];
                b[(size_t)k * g.Vh] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
            } else {
                float4 f4 = b[(size_t)k * g.Vh];
                c[2 * k] = make_double2(f4.x, f4.y);
                c[2 * k + 1] = make_double2(f4.z, f4.w);
            }
        }
    }
}
cudaError_t spinor_pack(void* field, const double2* canon, const Geom& g, int parity, bool fp64, cudaStream_t st) {
    int grid = grid_for(parity == 2 ? 2L * g.Vh : (long)g.Vh);
    if (fp64) spinor_layout_kernel<true, true><<<grid, NT, 0, st>>>(field, (double2*)canon, g, parity);
    else spinor_layout_kernel<true, false><<<grid, NT, 0, st>>>(field, (double2*)canon, g, parity);
    count_launch();
    return cudaGetLastError();
}
cudaError_t spinor_unpack(double2* canon, const void* field, const Geom& g, int parity, bool fp64, cudaStream_t st) {
    int grid = grid_for(parity == 2 ? 2L * g.Vh : (long)g.Vh);
    if (fp64) spinor_layout_kernel<false, true><<<grid, NT, 0, st>>>((void*)field, canon, g, parity);
    else spinor_layout_kernel<false, false><<<grid, NT, 0, st>>>((void*)field, canon, g, parity);
    count_launch();
    return cudaGetLastError();
}

template <bool PACK>
__global__ void __launch_bounds__(NT) mom_layout_kernel(double2* mom, double* canon, Geom g) {
    int mu, p, i;
    if (!link_index(g, mu, p, i)) return;
    int x[4];
    int lex = eo_coords(g, p, i, x);
    double* c = canon + ((size_t)lex * 4 + mu) * 8;
    double v[8];
    if (PACK) {
        for (int a = 0; a < 8; ++a) v[a] = c[a];
        store_mom(mom, g.Vh, p, mu, i, v);
    } else {
        load_mom(mom, g.Vh, p, mu, i, v);
        for (int a = 0; a < 8; ++a) c[a] = v[a];
    }
}
cudaError_t mom_pack(double2* mom, const double* canon, const Geom& g, cudaStream_t st) {
    mom_layout_kernel<true><<<grid_for(8L * g.Vh), NT, 0, st>>>(mom, (double*)canon, g);
    count_launch();
    return cudaGetLastError();
}
cudaError_t mom_unpack(double* canon, const double2* mom, const Geom& g, cudaStream_t st) {
    mom_layout_kernel<false><<<grid_for(8L * g.Vh), NT, 0, st>>>((double2*)mom, canon, g);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
