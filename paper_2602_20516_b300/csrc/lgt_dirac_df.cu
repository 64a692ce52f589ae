// lgt_dirac_df.cu -- the even-odd Wilson hopping term H (and H^+) in double-float
// arithmetic (lgt_df64.cuh: a value is an unevaluated pair of FP32 numbers, about 48
// significant bits).
//
// It serves the true residual b - A x of the mixed-precision CG (the reliable
// updates and the final check): on this part an FP64 FMA issues at 1/64 of the FP32
// rate, and the FP64 hop (864 FP64 instructions per site) runs FP64-ALU bound at
// about 17 times the time of the FP32 hop.  The same operator in FP32 pairs is
// accurate to ~1e-14 relative, far below the solver tolerances it is used with
// (the residual it forms differs from the FP64 one by ~1e-14 |b|).
//
// Layout: links float4 [parity][4][9][Vh] and spinor half fields float4 [12][Vh],
// each float4 = (re.hi, re.lo, im.hi, im.lo): the bytes of FP64.  One thread per
// output site; per neighbour the spinor is projected with (1 -/+ g_mu) in
// double-float, multiplied by U or U^+ with compensated dot products, and added into
// the output.  Epilogues: EPI_HOP (a H in), EPI_XPAY (y + a H in), both stored as
// double-float, and EPI_RESID (b - (y + a H in) with b and the result in FP64 and
// |result|^2 reduced in FP64).
#include "lgt_internal.h"
#include "lgt_df64.cuh"
#include "lgt_spin.cuh"
#include "lgt_clover.cuh"

namespace lgt {

// The kernel's arithmetic per neighbour (~1,500 FP32 instructions) is written once
// and driven by runtime direction parameters: unrolled over the 8 directions the
// code is ~12,000 instructions per thread and the warps stall on instruction fetch.

// v * c for c in {0: 1, 1: i, 2: -1, 3: -i}
__device__ __forceinline__ dfc times_phase(const dfc& v, int c) {
    const bool sw = c & 1;
    dfc w = {sw ? v.i : v.r, sw ? v.r : v.i};
    const bool nr = (c == 1) || (c == 2), ni = c >= 2;
    if (nr) w.r = df_neg(w.r);
    if (ni) w.i = df_neg(w.i);
    return w;
}

// Spin structure of (1 + S g_mu) in the chiral basis of lgt_spin.cuh, per (mu, S):
//   projection     h0 = psi0 + c0 psi[k0],  h1 = psi1 + c1 psi[k1]
//   reconstruction out0 += uh0, out1 += uh1, out2 += d2 uh[m2], out3 += d3 uh[m3]
// phases coded as in times_phase; k1 = 5 - k0, m3 = 1 - m2.
struct SpinDir { int k0, c0, c1, m2, d2, d3; };
__device__ __forceinline__ SpinDir spin_dir(int mu, bool neg) {
    // (k0, c0, c1, m2, d2, d3) for S < 0 (neg) and S > 0
    switch (mu) {
    case 0: return neg ? SpinDir{3, 1, 1, 1, 3, 3} : SpinDir{3, 3, 3, 1, 1, 1};
    case 1: return neg ? SpinDir{3, 0, 2, 1, 2, 0} : SpinDir{3, 2, 0, 1, 0, 2};
    case 2: return neg ? SpinDir{2, 1, 3, 0, 3, 1} : SpinDir{2, 3, 1, 0, 1, 3};
    default: return neg ? SpinDir{2, 2, 2, 0, 2, 2} : SpinDir{2, 0, 0, 0, 0, 0};
    }
}

__device__ __forceinline__ int sel4(const int (&v)[4], int mu) {
    return mu == 0 ? v[0] : mu == 1 ? v[1] : mu == 2 ? v[2] : v[3];
}

// out += (1 + S g_mu) W psi(y), W = U_mu(x) (forward, S = SF) or U_mu(x-mu)^+
// (backward, S = -SF), for direction d = 2 mu + (backward)
__device__ __forceinline__ void hop_dir_df(const float4* U, const float4* in, const Geom& g, int p, int lex,
                                           const int (&x)[4], int i, int d, int SF, dfc (&out)[4][3]) {
    const int Vh = g.Vh;
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    const int xm = sel4(x, mu), Lm = sel4(g.L, mu), sm = sel4(g.stride, mu);
    int ylex;
    if (fwd) ylex = (xm == Lm - 1) ? lex - (Lm - 1) * sm : lex + sm;
    else ylex = (xm == 0) ? lex + (Lm - 1) * sm : lex - sm;
    const int j = ylex >> 1;
    const bool wrap_t = mu == 3 && (fwd ? xm == Lm - 1 : xm == 0);   // antiperiodic sign
    const SpinDir sd = spin_dir(mu, (fwd ? SF : -SF) < 0);
    dfc h[2][3];
    {
        const SpinorDF s = load_spinor_df(in, Vh, j);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const dfc a0 = sd.k0 == 3 ? s.c[3][c] : s.c[2][c];
            const dfc a1 = sd.k0 == 3 ? s.c[2][c] : s.c[3][c];
            h[0][c] = s.c[0][c] + times_phase(a0, sd.c0);
            h[1][c] = s.c[1][c] + times_phase(a1, sd.c1);
            if (wrap_t) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
        }
    }
    // W in registers: U_mu(x) as stored, or U_mu(x-mu)^+ by reading entry (b, a) into
    // slot (a, b) and conjugating
    dfmat W;
    {
        const float4* base = U + (size_t)(((fwd ? p : 1 - p) * 4 + mu) * 9) * Vh + (fwd ? i : j);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float4 v = __ldg(base + (size_t)(fwd ? 3 * a + b : 3 * b + a) * Vh);
                W.e[a][b] = {{v.x, v.y}, fwd ? df{v.z, v.w} : df{-v.z, -v.w}};
            }
    }
    dfc uh[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dacc re = dacc0(), im = dacc0();
#pragma unroll
            for (int b = 0; b < 3; ++b) cacc_mul<false, false>(re, im, W.e[a][b], h[r][b]);
            uh[r][a] = {dacc_get(re), dacc_get(im)};
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        out[0][c] = out[0][c] + uh[0][c];
        out[1][c] = out[1][c] + uh[1][c];
        out[2][c] = out[2][c] + times_phase(sd.m2 == 1 ? uh[1][c] : uh[0][c], sd.d2);
        out[3][c] = out[3][c] + times_phase(sd.m2 == 1 ? uh[0][c] : uh[1][c], sd.d3);
    }
}

// w = B v for the double-float clover blocks of site i: Cp = the parity's [36][Vh] block
// of a Hermitian-packed double-float field (the FP32 packed layout of lgt_clover.cuh,
// real k of block c as the pair (hi, lo) in float4 18 c + k / 2)
__device__ __forceinline__ void clover_mul_df(const float4* __restrict__ Cp, int Vh, int i, const dfc (&v)[4][3],
                                              dfc (&w)[4][3]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        df f[36];
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const float4 z = __ldg(Cp + (size_t)(18 * c + k) * Vh + i);
            f[2 * k] = {z.x, z.y};
            f[2 * k + 1] = {z.z, z.w};
        }
#pragma unroll 1
        for (int r = 0; r < 6; ++r) {
            dacc re = dacc0(), im = dacc0();
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const dfc vq = v[(6 * c + q) / 3][(6 * c + q) % 3];
                dfc z;
                if (q == r) z = {f[r], {0.f, 0.f}};
                else {
                    const int o = r < q ? clover_upper_index(r, q) : clover_upper_index(q, r);
                    z = {f[o], r < q ? f[o + 1] : df_neg(f[o + 1])};
                }
                cacc_mul<false, false>(re, im, z, vq);
            }
            w[(6 * c + r) / 3][(6 * c + r) % 3] = {dacc_get(re), dacc_get(im)};
        }
    }
}

// y + a v in double-float (y may be zero)
__device__ __forceinline__ df axpy_df(df a, df v, df y) {
    dacc r = {y.h, y.l};
    dacc_mul(r, a, v);
    return dacc_get(r);
}

// CLV = 1: the output of EPI_HOP is multiplied by the output site's clover block (HopArgs.clov,
// double-float packed); CLV = 2: y is multiplied by it before EPI_XPAY / EPI_RESID
template <bool DAG, int EPI, int CLV = 0>
__global__ void __launch_bounds__(NT) hop_df_kernel(HopArgs A) {
    const int n = (A.parity == 2) ? 2 * A.g.Vh : A.g.Vh;
    const int t = blockIdx.x * NT + threadIdx.x;
    double red = 0.0;
    if (t < n) {
        int p, i;
        if (A.parity == 2) { p = t >= A.g.Vh; i = t - p * A.g.Vh; }
        else { p = A.parity; i = t; }
        int x[4];
        const int lex = eo_coords(A.g, p, i, x);
        dfc out[4][3];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) out[s][c] = {{0.f, 0.f}, {0.f, 0.f}};
        const float4* U = (const float4*)A.U;
        const float4* in = (const float4*)A.in[1 - p];
        constexpr int SF = DAG ? +1 : -1;
#pragma unroll 1
        for (int d = 0; d < 8; ++d) hop_dir_df(U, in, A.g, p, lex, x, i, d, SF, out);
        const df a = df_from(A.a);
        const int Vh = A.g.Vh;
        SpinorDF o;
        const float4* Cp = (const float4*)A.clov + (size_t)p * 36 * Vh;
        if (EPI == EPI_HOP) {
            const df z = {0.f, 0.f};
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.c[s][c] = {axpy_df(a, out[s][c].r, z), axpy_df(a, out[s][c].i, z)};
            if constexpr (CLV == 1) {
                const SpinorDF t = o;
                clover_mul_df(Cp, Vh, i, t.c, o.c);
            }
        } else {
            SpinorDF yv = load_spinor_df((const float4*)A.y[p], Vh, i);
            if constexpr (CLV == 2) {
                const SpinorDF t = yv;
                clover_mul_df(Cp, Vh, i, t.c, yv.c);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    o.c[s][c] = {axpy_df(a, out[s][c].r, yv.c[s][c].r), axpy_df(a, out[s][c].i, yv.c[s][c].i)};
        }
        if (EPI == EPI_RESID) {
            // b - o in FP64; |.|^2 of the site in FP32 (it only steers the solver)
            const double2* b = (const double2*)A.pv[p];
            double2* res = (double2*)A.out[p];
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double2 bv = __ldg(b + (size_t)k * Vh + i);
                const dfc& v = o.c[k / 3][k % 3];
                const double2 r = make_double2(bv.x - df_to(v.r), bv.y - df_to(v.i));
                res[(size_t)k * Vh + i] = r;
                const float rx = (float)r.x, ry = (float)r.y;
                acc = fmaf(rx, rx, fmaf(ry, ry, acc));
            }
            red = (double)acc;
        } else {
            store_spinor_df((float4*)A.out[p], Vh, i, o);
        }
    }
    if (EPI == EPI_RESID) grid_reduce(block_sum(red), A.partials, A.counter, A.s, A.red_op, A.red_slot);
}

template <bool DAG>
static cudaError_t launch_df_epi(const HopArgs& A, int epi, cudaStream_t st) {
    const int n = (A.parity == 2) ? 2 * A.g.Vh : A.g.Vh;
    const int grid = (n + NT - 1) / NT;
    if (epi == EPI_RESID && (!A.partials || !A.s || grid > A.red_capacity)) return cudaErrorInvalidValue;
    if (A.clov) {   // even-odd clover: one parity only
        if (A.parity == 2) return cudaErrorInvalidValue;
        switch (epi) {
        case EPI_HOP: hop_df_kernel<DAG, EPI_HOP, 1><<<grid, NT, 0, st>>>(A); break;
        case EPI_XPAY: hop_df_kernel<DAG, EPI_XPAY, 2><<<grid, NT, 0, st>>>(A); break;
        case EPI_RESID: hop_df_kernel<DAG, EPI_RESID, 2><<<grid, NT, 0, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        count_launch();
        return cudaGetLastError();
    }
    switch (epi) {
    case EPI_HOP: hop_df_kernel<DAG, EPI_HOP><<<grid, NT, 0, st>>>(A); break;
    case EPI_XPAY: hop_df_kernel<DAG, EPI_XPAY><<<grid, NT, 0, st>>>(A); break;
    case EPI_RESID: hop_df_kernel<DAG, EPI_RESID><<<grid, NT, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hop_df(const HopArgs& A, bool dagger, int epi, cudaStream_t st) {
    return dagger ? launch_df_epi<true>(A, epi, st) : launch_df_epi<false>(A, epi, st);
}

// ---------------------------------------------------------------- conversions
// Hermitian-packed double-float copy of the clover blocks of one parity (from the FP64
// field [parity][72][Vh], full blocks): float4 [parity][36][Vh]
__global__ void __launch_bounds__(NT) clover_pack_df_kernel(const double2* C64, Geom g, int parity, float4* Cdf) {
    const int i = blockIdx.x * NT + threadIdx.x;
    if (i >= g.Vh) return;
    const double2* b = C64 + (size_t)parity * 72 * g.Vh + i;
    float4* o = Cdf + (size_t)parity * 36 * g.Vh + i;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        double f[36];
        for (int r = 0; r < 6; ++r) f[r] = __ldg(b + (size_t)(36 * c + 7 * r) * g.Vh).x;
        for (int r = 0; r < 6; ++r)
            for (int q = r + 1; q < 6; ++q) {
                const double2 z = __ldg(b + (size_t)(36 * c + 6 * r + q) * g.Vh);
                f[clover_upper_index(r, q)] = z.x;
                f[clover_upper_index(r, q) + 1] = z.y;
            }
        for (int k = 0; k < 18; ++k) {
            const df a = df_from(f[2 * k]), e = df_from(f[2 * k + 1]);
            o[(size_t)(18 * c + k) * g.Vh] = make_float4(a.h, a.l, e.h, e.l);
        }
    }
}
cudaError_t clover_pack_df(const double2* C64, const Geom& g, int parity, float4* Cdf, cudaStream_t st) {
    if (parity != 0 && parity != 1) return cudaErrorInvalidValue;
    clover_pack_df_kernel<<<(g.Vh + NT - 1) / NT, NT, 0, st>>>(C64, g, parity, Cdf);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) f64_to_df_kernel(float4* y, const double2* x, long ne) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const double2 v = __ldg(x + e);
    const df r = df_from(v.x), im = df_from(v.y);
    y[e] = make_float4(r.h, r.l, im.h, im.l);
}
__global__ void __launch_bounds__(NT) df_to_f64_kernel(double2* y, const float4* x, long ne) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const float4 v = __ldg(x + e);
    y[e] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
// ne complex entries (a half spinor field has 12 Vh)
cudaError_t complex_to_df(float4* y, const double2* x, long ne, cudaStream_t st) {
    if (ne <= 0) return cudaSuccess;
    f64_to_df_kernel<<<(int)((ne + NT - 1) / NT), NT, 0, st>>>(y, x, ne);
    count_launch();
    return cudaGetLastError();
}
cudaError_t complex_from_df(double2* y, const float4* x, long ne, cudaStream_t st) {
    if (ne <= 0) return cudaSuccess;
    df_to_f64_kernel<<<(int)((ne + NT - 1) / NT), NT, 0, st>>>(y, x, ne);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
