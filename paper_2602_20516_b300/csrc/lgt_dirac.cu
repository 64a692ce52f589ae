// lgt_dirac.cu -- even-odd Wilson hopping term H (and H^+ = g5 H g5) on sm_103a.
//
// One thread per output site.  For each of the 8 neighbours the 4-spinor is
// projected to a 2-spinor with (1 -/+ g_mu), multiplied by U or U^+ (3x3 colour),
// and reconstructed into the accumulator; the antiperiodic time sign multiplies
// the projected spinor.  FP64 links are 18 reals (9 x double2, one 128-bit load
// each); FP32 links are the first two rows (3 x float4) with row 3 rebuilt as
// conj(row1 x row2).  Spinor components of one parity are contiguous per
// component (site-major SoA), so every load and store is a coalesced 128-bit access.
//
// Epilogues fuse the CG vector work into the last hop of an operator
// application: xpay (y + a H in), its squared norm, and the CG residual update
// r -= alpha A p with |r|^2, or the true residual b - A x.
#include "lgt_internal.h"
#include "lgt_spin.cuh"
#include "lgt_clover.cuh"

namespace lgt {

template <typename R> struct Prec;
template <> struct Prec<double> {
    using T = double2;
    using S = SpinorD;
    static __device__ __forceinline__ mat3<double> link(const void* U, int Vh, int p, int mu, int i) {
        return load_link((const double2*)U, Vh, p, mu, i);
    }
};
template <> struct Prec<float> {
    using T = float4;
    using S = SpinorF;
    static __device__ __forceinline__ mat3<float> link(const void* U, int Vh, int p, int mu, int i) {
        return load_link12((const float4*)U, Vh, p, mu, i);
    }
};

// colour multiply of both half-spinor rows by M or M^+
template <bool DAGM, typename R>
__device__ __forceinline__ void mult(const mat3<R>& M, const cx<R> (&h)[2][3], cx<R> (&uh)[2][3]) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cx<R> s = {0, 0};
#pragma unroll
            for (int b = 0; b < 3; ++b) s = DAGM ? cmadc(s, M.e[b][a], h[j][b]) : cmad(s, M.e[a][b], h[j][b]);
            uh[j][a] = s;
        }
}

// Input half field of a hop, read through the read-only path: load(j) is the spinor
// of half-field site j.
template <typename R> struct PlainIn {
    const typename Prec<R>::T* f;
    int Vh;
    __device__ __forceinline__ typename Prec<R>::S load(int j) const { return load_spinor(f, Vh, j); }
};
template <int MU, int SF, int SB, typename R, typename IN>
__device__ __forceinline__ void hop_dir(const void* U, const Geom& g, const IN& in, int p, int lex,
                                        const int (&x)[4], int i, cx<R> (&out)[4][3]) {
    using P = Prec<R>;
    const int Vh = g.Vh;
    // forward: b (1 + SF g) U_mu(x) psi(x+mu)
    {
        int j = nb_lex(g, lex, x, MU, +1) >> 1;
        typename P::S s = in.load(j);
        cx<R> h[2][3], uh[2][3];
        project<MU, SF>(s.c, h);
        if (MU == 3 && x[3] == g.L[3] - 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
        }
        mat3<R> M = P::link(U, Vh, p, MU, i);
        mult<false>(M, h, uh);
        accumulate<MU, SF>(out, uh);
    }
    // backward: b (1 + SB g) U_mu(x-mu)^+ psi(x-mu)
    {
        int j = nb_lex(g, lex, x, MU, -1) >> 1;
        typename P::S s = in.load(j);
        cx<R> h[2][3], uh[2][3];
        project<MU, SB>(s.c, h);
        if (MU == 3 && x[3] == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
        }
        mat3<R> M = P::link(U, Vh, 1 - p, MU, j);
        mult<true>(M, h, uh);
        accumulate<MU, SB>(out, uh);
    }
}

// squared norm of one site's spinor in the field's own precision (the cross-site
// accumulation is FP64); FP64 arithmetic here would cost 24 FP64 FMAs per site,
// far more than the FP32 hop's own arithmetic on this part
template <typename R> __device__ __forceinline__ double sq(const cx<R> (&v)[4][3]) {
    R acc = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc = fma(v[a][c].r, v[a][c].r, fma(v[a][c].i, v[a][c].i, acc));
    return (double)acc;
}

// the 8 hops into output site (p, i) at coordinates x, lexicographic index lex
template <typename R, bool DAG, typename IN>
__device__ __forceinline__ void hop_accum(const void* U, const Geom& g, const IN& in, int p, int lex,
                                          const int (&x)[4], int i, cx<R> (&out)[4][3]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) out[a][c] = {0, 0};
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    hop_dir<0, SF, SB, R>(U, g, in, p, lex, x, i, out);
    hop_dir<1, SF, SB, R>(U, g, in, p, lex, x, i, out);
    hop_dir<2, SF, SB, R>(U, g, in, p, lex, x, i, out);
    hop_dir<3, SF, SB, R>(U, g, in, p, lex, x, i, out);
}

// w = B v for the clover blocks of output site i (FP32, Hermitian-packed field of parity p)
__device__ __forceinline__ void clover_site(const HopArgs& A, int p, int i, SpinorF& v) {
    fcx a[12], b[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) a[k] = v.c[k / 3][k % 3];
    clover_mul_f32((const float4*)A.clov + (size_t)p * 18 * A.g.Vh, A.g.Vh, i, a, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) v.c[k / 3][k % 3] = b[k];
}
__device__ __forceinline__ void clover_site(const HopArgs&, int, int, SpinorD&) {}

// The work of one output site t (t < n): accumulate the 8 hops, apply the epilogue
// and return this site's contribution to the epilogue's reduction.  CLV (FP32 only):
// 1 applies the output site's clover block to the result of EPI_HOP, 2 applies it to
// y in EPI_XPAY_NORM / EPI_CG (HopArgs.clov).
template <typename R, bool DAG, int EPI, int CLV = 0>
__device__ __forceinline__ double hop_site(const HopArgs& A, int t) {
    using P = Prec<R>;
    using T = typename P::T;
    double red = 0.0;
    int p, i;
    if (A.parity == 2) { p = t >= A.g.Vh; i = t - p * A.g.Vh; }
    else { p = A.parity; i = t; }
    int x[4];
    int lex = eo_coords(A.g, p, i, x);
    cx<R> out[4][3];
    hop_accum<R, DAG>(A.U, A.g, PlainIn<R>{(const T*)A.in[1 - p], A.g.Vh}, p, lex, x, i, out);
    const R a = (R)A.a;
    const int Vh = A.g.Vh;
    if (EPI == EPI_HOP) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) out[s][c] = a * out[s][c];
        typename P::S o;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.c[s][c] = out[s][c];
        if constexpr (CLV == 1) clover_site(A, p, i, o);
        store_spinor((T*)A.out[p], Vh, i, o);
    } else {
        typename P::S yv = load_spinor((const T*)A.y[p], Vh, i);
        if constexpr (CLV == 2) clover_site(A, p, i, yv);
        typename P::S o;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o.c[s][c].r = fma(a, out[s][c].r, yv.c[s][c].r);
                o.c[s][c].i = fma(a, out[s][c].i, yv.c[s][c].i);
            }
        if (EPI == EPI_XPAY || EPI == EPI_XPAY_NORM) {
            store_spinor((T*)A.out[p], Vh, i, o);
            if (EPI == EPI_XPAY_NORM) red = sq<R>(o.c);
        } else if (EPI == EPI_CG) {
            // o = A p at this site: r -= alpha A p, red = |r|^2 (x += alpha p is left to
            // the p update, which reads p anyway)
            const R alpha = (R)A.s->alpha;
            typename P::S rv = load_spinor((const T*)A.r[p], Vh, i);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rv.c[s][c].r = fma(-alpha, o.c[s][c].r, rv.c[s][c].r);
                    rv.c[s][c].i = fma(-alpha, o.c[s][c].i, rv.c[s][c].i);
                }
            store_spinor((T*)A.r[p], Vh, i, rv);
            red = sq<R>(rv.c);
        } else {  // EPI_RESID: out = b - A x, b in pv
            typename P::S bv = load_spinor((const T*)A.pv[p], Vh, i);
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.c[s][c] = bv.c[s][c] - o.c[s][c];
            store_spinor((T*)A.out[p], Vh, i, o);
            red = sq<R>(o.c);
        }
    }
    return red;
}

template <typename R, bool DAG, int EPI, int CLV = 0>
__device__ __forceinline__ void hop_body(const HopArgs& A, int blk, int nblk, bool first) {
    if (A.skip && A.s->done >= 1) return;
    if (A.fin_n > 0 && first) {   // finish the deferred reduction of an earlier launch
        const double acc = ordered_sum(A.partials, A.fin_n);
        if (threadIdx.x == 0) apply_reduce_op(A.s, A.fin_op, A.red_slot, acc);
    }
    const int n = (A.parity == 2) ? 2 * A.g.Vh : A.g.Vh;
    const int t = blk * NT + threadIdx.x;
    const double red = (t < n) ? hop_site<R, DAG, EPI, CLV>(A, t) : 0.0;
    if (EPI == EPI_XPAY_NORM || EPI == EPI_CG || EPI == EPI_RESID) {
        double b = block_sum(red);
        if (A.defer) {
            if (threadIdx.x == 0) A.partials[blk] = b;
        } else {
            grid_reduce(b, A.partials, A.counter, A.s, A.red_op, A.red_slot, blk, nblk);
        }
    }
}

// Resident blocks per SM requested from the register allocator for the FP32 hop
// (the FP64 hop keeps its registers: it is FP64-ALU bound, not latency bound).
#ifndef LGT_HOP32_MIN_BLOCKS
#define LGT_HOP32_MIN_BLOCKS 4
#endif
#ifndef LGT_HOP32_EPI_MIN_BLOCKS
#define LGT_HOP32_EPI_MIN_BLOCKS 4
#endif
#ifndef LGT_HOP64_MIN_BLOCKS
#define LGT_HOP64_MIN_BLOCKS 1
#endif
template <typename R, int EPI> constexpr int hop_min_blocks() {
    return sizeof(R) == 4 ? (EPI == EPI_HOP ? LGT_HOP32_MIN_BLOCKS : LGT_HOP32_EPI_MIN_BLOCKS) : LGT_HOP64_MIN_BLOCKS;
}

template <typename R, bool DAG, int EPI, int CLV = 0>
__global__ void __launch_bounds__(NT, (hop_min_blocks<R, EPI>())) hop_kernel(HopArgs A) {
    hop_body<R, DAG, EPI, CLV>(A, A.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x, gridDim.x, blockIdx.x == 0);
}

// Many independent problems (lattices of any size) in one launch: block b runs
// block b - first of the descriptor whose range [first, first + nblk) holds b.
template <typename R, bool DAG, int EPI>
__global__ void __launch_bounds__(NT) hop_batch_kernel(const BatchHop* __restrict__ d, int n) {
    int lo = 0, hi = n - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].first <= b) lo = mid;
        else hi = mid - 1;
    }
    const BatchHop& e = d[lo];
    hop_body<R, DAG, EPI>(e.a, b - e.first, e.nblk, false);
}

template <typename R, bool DAG>
static cudaError_t launch_batch_epi(const BatchHop* d, int n, int total_blocks, int epi, cudaStream_t st) {
    switch (epi) {
    case EPI_HOP: hop_batch_kernel<R, DAG, EPI_HOP><<<total_blocks, NT, 0, st>>>(d, n); break;
    case EPI_XPAY: hop_batch_kernel<R, DAG, EPI_XPAY><<<total_blocks, NT, 0, st>>>(d, n); break;
    case EPI_XPAY_NORM: hop_batch_kernel<R, DAG, EPI_XPAY_NORM><<<total_blocks, NT, 0, st>>>(d, n); break;
    case EPI_CG: hop_batch_kernel<R, DAG, EPI_CG><<<total_blocks, NT, 0, st>>>(d, n); break;
    case EPI_RESID: hop_batch_kernel<R, DAG, EPI_RESID><<<total_blocks, NT, 0, st>>>(d, n); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hop_batch(const BatchHop* d, int n, int total_blocks, bool fp64, bool dagger, int epi,
                             cudaStream_t st) {
    if (n <= 0 || total_blocks <= 0) return cudaSuccess;
    if (fp64) return dagger ? launch_batch_epi<double, true>(d, n, total_blocks, epi, st)
                            : launch_batch_epi<double, false>(d, n, total_blocks, epi, st);
    return dagger ? launch_batch_epi<float, true>(d, n, total_blocks, epi, st)
                  : launch_batch_epi<float, false>(d, n, total_blocks, epi, st);
}

template <typename R, bool DAG>
static cudaError_t launch_epi(const HopArgs& A, int epi, cudaStream_t st) {
    const int n = (A.parity == 2) ? 2 * A.g.Vh : A.g.Vh;
    const int grid = (n + NT - 1) / NT;
    const bool reduces = epi == EPI_XPAY_NORM || epi == EPI_CG || epi == EPI_RESID;
    if (reduces && (!A.partials || grid > A.red_capacity)) return cudaErrorInvalidValue;
    if (A.fin_n > 0 && (!A.partials || !A.s || A.fin_n > A.red_capacity)) return cudaErrorInvalidValue;
    if (A.clov) {   // the fused even-odd clover variants (FP32, one parity)
        if (sizeof(R) != 4 || A.parity == 2) return cudaErrorInvalidValue;
        switch (epi) {
        case EPI_HOP: hop_kernel<R, DAG, EPI_HOP, 1><<<grid, NT, 0, st>>>(A); break;
        case EPI_XPAY_NORM: hop_kernel<R, DAG, EPI_XPAY_NORM, 2><<<grid, NT, 0, st>>>(A); break;
        case EPI_CG: hop_kernel<R, DAG, EPI_CG, 2><<<grid, NT, 0, st>>>(A); break;
        default: return cudaErrorInvalidValue;
        }
        count_launch();
        return cudaGetLastError();
    }
    switch (epi) {
    case EPI_HOP: hop_kernel<R, DAG, EPI_HOP><<<grid, NT, 0, st>>>(A); break;
    case EPI_XPAY: hop_kernel<R, DAG, EPI_XPAY><<<grid, NT, 0, st>>>(A); break;
    case EPI_XPAY_NORM: hop_kernel<R, DAG, EPI_XPAY_NORM><<<grid, NT, 0, st>>>(A); break;
    case EPI_CG: hop_kernel<R, DAG, EPI_CG><<<grid, NT, 0, st>>>(A); break;
    case EPI_RESID: hop_kernel<R, DAG, EPI_RESID><<<grid, NT, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hop(const HopArgs& A, bool fp64, bool dagger, int epi, cudaStream_t st) {
    if (fp64) return dagger ? launch_epi<double, true>(A, epi, st) : launch_epi<double, false>(A, epi, st);
    return dagger ? launch_epi<float, true>(A, epi, st) : launch_epi<float, false>(A, epi, st);
}

// ---------------------------------------------------------------- several right-hand sides
// One thread per output site for K systems: each link is loaded once per site and
// direction and applied to the K input spinors, so a launch moves 8 links + K (in +
// out) spinors per site instead of K times 8 links + 1 pair.  The K slots are
// computed in straight-line code (the host packs only running systems, so every
// slot holds valid fields) and the loads of all directions and systems can be in
// flight together; a system whose scalars say done is masked at its stores and its
// reduction.  Per system the arithmetic is that of hop_site (same direction order,
// same epilogue) and the reduction is block_sum / grid_reduce over the same 128
// sites per block, so a system's result does not depend on the others in the launch.
template <int MU, int SF, int SB, typename R, int K>
__device__ __forceinline__ void hop_dir_multi(const HopArgsM& A, int p, int lex, const int (&x)[4], int i,
                                              cx<R> (&out)[K][4][3]) {
    using P = Prec<R>;
    const int Vh = A.g.Vh;
    {
        const int j = nb_lex(A.g, lex, x, MU, +1) >> 1;
        const mat3<R> M = P::link(A.U, Vh, p, MU, i);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            typename P::S s = load_spinor((const typename P::T*)A.in[k], Vh, j);
            cx<R> h[2][3], uh[2][3];
            project<MU, SF>(s.c, h);
            if (MU == 3 && x[3] == A.g.L[3] - 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
            }
            mult<false>(M, h, uh);
            accumulate<MU, SF>(out[k], uh);
        }
    }
    {
        const int j = nb_lex(A.g, lex, x, MU, -1) >> 1;
        const mat3<R> M = P::link(A.U, Vh, 1 - p, MU, j);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            typename P::S s = load_spinor((const typename P::T*)A.in[k], Vh, j);
            cx<R> h[2][3], uh[2][3];
            project<MU, SB>(s.c, h);
            if (MU == 3 && x[3] == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
            }
            mult<true>(M, h, uh);
            accumulate<MU, SB>(out[k], uh);
        }
    }
}

template <typename R, bool DAG, int EPI, int K>
__global__ void __launch_bounds__(NT, (K == 1 ? 4 : (K == 2 ? 3 : 2))) hop_multi_kernel(HopArgsM A) {
    using P = Prec<R>;
    using T = typename P::T;
    bool act[K];
    bool any = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        act[k] = !(A.skip && A.s[k]->done >= 1);
        any = any || act[k];
    }
    if (!any) return;
    if (A.fin_n > 0 && blockIdx.x == 0) {   // finish the deferred reductions of an earlier launch
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!act[k]) continue;
            const double acc = ordered_sum(A.partials[k], A.fin_n);
            if (threadIdx.x == 0) apply_reduce_op(A.s[k], A.fin_op, 0, acc);
        }
    }
    const int t = blockIdx.x * NT + threadIdx.x;
    double red[K];
#pragma unroll
    for (int k = 0; k < K; ++k) red[k] = 0.0;
    if (t < A.g.Vh) {
        const int p = A.parity, i = t;
        int x[4];
        const int lex = eo_coords(A.g, p, i, x);
        cx<R> out[K][4][3];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) out[k][a][c] = {0, 0};
        constexpr int SF = DAG ? +1 : -1;
        constexpr int SB = -SF;
        hop_dir_multi<0, SF, SB, R, K>(A, p, lex, x, i, out);
        hop_dir_multi<1, SF, SB, R, K>(A, p, lex, x, i, out);
        hop_dir_multi<2, SF, SB, R, K>(A, p, lex, x, i, out);
        hop_dir_multi<3, SF, SB, R, K>(A, p, lex, x, i, out);
        const int Vh = A.g.Vh;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!act[k]) continue;
            const R a = (R)A.a[k];
            if (EPI == EPI_HOP) {
                typename P::S o;
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) o.c[s][c] = a * out[k][s][c];
                store_spinor((T*)A.out[k], Vh, i, o);
            } else {
                const typename P::S yv = load_spinor((const T*)A.y[k], Vh, i);
                typename P::S o;
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o.c[s][c].r = fma(a, out[k][s][c].r, yv.c[s][c].r);
                        o.c[s][c].i = fma(a, out[k][s][c].i, yv.c[s][c].i);
                    }
                if (EPI == EPI_XPAY || EPI == EPI_XPAY_NORM) {
                    store_spinor((T*)A.out[k], Vh, i, o);
                    if (EPI == EPI_XPAY_NORM) red[k] = sq<R>(o.c);
                } else {  // EPI_CG
                    const R alpha = (R)A.s[k]->alpha;
                    typename P::S rv = load_spinor((const T*)A.r[k], Vh, i);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            rv.c[s][c].r = fma(-alpha, o.c[s][c].r, rv.c[s][c].r);
                            rv.c[s][c].i = fma(-alpha, o.c[s][c].i, rv.c[s][c].i);
                        }
                    store_spinor((T*)A.r[k], Vh, i, rv);
                    red[k] = sq<R>(rv.c);
                }
            }
        }
    }
    if (EPI == EPI_XPAY_NORM || EPI == EPI_CG) {
        // the last-block reductions of the K systems with one fence and K atomics in
        // flight together (the partials and their summation order are grid_reduce's)
        double b[K];
#pragma unroll
        for (int k = 0; k < K; ++k) b[k] = act[k] ? block_sum(red[k]) : 0.0;   // act: the same in every block
        if (A.defer) {
            if (threadIdx.x == 0)
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (act[k]) A.partials[k][blockIdx.x] = b[k];
            return;
        }
        __shared__ bool last[K];
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (act[k]) A.partials[k][blockIdx.x] = b[k];
            __threadfence();
            unsigned prev[K];
#pragma unroll
            for (int k = 0; k < K; ++k) prev[k] = act[k] ? atomicAdd(A.counter[k], 1u) : 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) last[k] = act[k] && prev[k] == gridDim.x - 1;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (!last[k]) continue;
            __threadfence();
            const double acc = ordered_sum(A.partials[k], gridDim.x);
            if (threadIdx.x == 0) {
                *A.counter[k] = 0u;
                apply_reduce_op(A.s[k], A.red_op, 0, acc);
            }
        }
    }
}

template <bool DAG, int K>
static cudaError_t launch_multi_epi(const HopArgsM& A, int epi, cudaStream_t st) {
    const int grid = (A.g.Vh + NT - 1) / NT;
    switch (epi) {
    case EPI_HOP: hop_multi_kernel<float, DAG, EPI_HOP, K><<<grid, NT, 0, st>>>(A); break;
    case EPI_XPAY: hop_multi_kernel<float, DAG, EPI_XPAY, K><<<grid, NT, 0, st>>>(A); break;
    case EPI_XPAY_NORM: hop_multi_kernel<float, DAG, EPI_XPAY_NORM, K><<<grid, NT, 0, st>>>(A); break;
    case EPI_CG: hop_multi_kernel<float, DAG, EPI_CG, K><<<grid, NT, 0, st>>>(A); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}
template <bool DAG>
static cudaError_t launch_multi_k(const HopArgsM& A, int epi, cudaStream_t st) {
    switch (A.nrhs) {
    case 1: return launch_multi_epi<DAG, 1>(A, epi, st);
    case 2: return launch_multi_epi<DAG, 2>(A, epi, st);
    case 3: return launch_multi_epi<DAG, 3>(A, epi, st);
    default: return launch_multi_epi<DAG, 4>(A, epi, st);
    }
}

// FP32 only: the FP64 hop is bound by FP64 arithmetic, which sharing link loads
// does not reduce (and K FP64 accumulators exceed the register file)
cudaError_t launch_hop_multi(const HopArgsM& A, bool fp64, bool dagger, int epi, cudaStream_t st) {
    if (fp64 || A.nrhs < 1 || A.nrhs > KMAX_RHS || (A.parity != 0 && A.parity != 1)) return cudaErrorInvalidValue;
    for (int k = 0; k < A.nrhs; ++k)
        if (!A.in[k]) return cudaErrorInvalidValue;
    const bool reduces = epi == EPI_XPAY_NORM || epi == EPI_CG;
    if (reduces && (A.g.Vh + NT - 1) / NT > A.red_capacity) return cudaErrorInvalidValue;
    if (A.fin_n > A.red_capacity) return cudaErrorInvalidValue;
    return dagger ? launch_multi_k<true>(A, epi, st) : launch_multi_k<false>(A, epi, st);
}

int hop_grid(const Geom& g, int parity) {
    const int n = (parity == 2) ? 2 * g.Vh : g.Vh;
    return (n + NT - 1) / NT;
}

}  // namespace lgt
