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

// Input half field of a hop, read through the read-only path: load<MU, D>(j) is the
// spinor of half-field site j, the neighbour of the output site in direction D mu.
template <typename R> struct PlainIn {
    const typename Prec<R>::T* f;
    int Vh;
    template <int MU, int D>
    __device__ __forceinline__ typename Prec<R>::S load(int j) const { return load_spinor(f, Vh, j); }
};
// Links read through the read-only path: link<MU, D>(q, site) is U_mu(site) of parity q
// (site = the output site for D = +1, its neighbour j for D = -1).
template <typename R> struct PlainLinks {
    const void* U;
    int Vh;
    template <int MU, int D>
    __device__ __forceinline__ mat3<R> link(int q, int site) const { return Prec<R>::link(U, Vh, q, MU, site); }
};
template <int MU, int SF, int SB, typename R, typename IN, typename LK>
__device__ __forceinline__ void hop_dir(const Geom& g, const IN& in, const LK& lk, int p, int lex,
                                        const int (&x)[4], int i, cx<R> (&out)[4][3]) {
    using P = Prec<R>;
    // forward: b (1 + SF g) U_mu(x) psi(x+mu)
    {
        int j = nb_lex(g, lex, x, MU, +1) >> 1;
        typename P::S s = in.template load<MU, +1>(j);
        cx<R> h[2][3], uh[2][3];
        project<MU, SF>(s.c, h);
        if (MU == 3 && x[3] == g.L[3] - 1) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
        }
        mat3<R> M = lk.template link<MU, +1>(p, i);
        mult<false>(M, h, uh);
        accumulate<MU, SF>(out, uh);
    }
    // backward: b (1 + SB g) U_mu(x-mu)^+ psi(x-mu)
    {
        int j = nb_lex(g, lex, x, MU, -1) >> 1;
        typename P::S s = in.template load<MU, -1>(j);
        cx<R> h[2][3], uh[2][3];
        project<MU, SB>(s.c, h);
        if (MU == 3 && x[3] == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) { h[0][c] = -h[0][c]; h[1][c] = -h[1][c]; }
        }
        mat3<R> M = lk.template link<MU, -1>(1 - p, j);
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
template <typename R, bool DAG, typename IN, typename LK>
__device__ __forceinline__ void hop_accum(const Geom& g, const IN& in, const LK& lk, int p, int lex,
                                          const int (&x)[4], int i, cx<R> (&out)[4][3]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) out[a][c] = {0, 0};
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    hop_dir<0, SF, SB, R>(g, in, lk, p, lex, x, i, out);
    hop_dir<1, SF, SB, R>(g, in, lk, p, lex, x, i, out);
    hop_dir<2, SF, SB, R>(g, in, lk, p, lex, x, i, out);
    hop_dir<3, SF, SB, R>(g, in, lk, p, lex, x, i, out);
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

// The work of output site (p, i): accumulate the 8 hops (input spinors from `in`,
// links from `lk`), apply the epilogue and return this site's contribution to the
// epilogue's reduction.  CLV (FP32 only): 1 applies the output site's clover block to
// the result of EPI_HOP, 2 applies it to y in EPI_XPAY_NORM / EPI_CG (HopArgs.clov).
template <typename R, bool DAG, int EPI, int CLV, typename IN, typename LK>
__device__ __forceinline__ double hop_site_io(const HopArgs& A, int p, int i, const IN& in, const LK& lk) {
    using P = Prec<R>;
    using T = typename P::T;
    double red = 0.0;
    int x[4];
    int lex = eo_coords(A.g, p, i, x);
    cx<R> out[4][3];
    hop_accum<R, DAG>(A.g, in, lk, p, lex, x, i, out);
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

// output site t (t < n) of a launch over parity A.parity (2: both, t >= Vh odd)
template <typename R, bool DAG, int EPI, int CLV = 0>
__device__ __forceinline__ double hop_site(const HopArgs& A, int t) {
    int p, i;
    if (A.parity == 2) { p = t >= A.g.Vh; i = t - p * A.g.Vh; }
    else { p = A.parity; i = t; }
    return hop_site_io<R, DAG, EPI, CLV>(A, p, i, PlainIn<R>{(const typename Prec<R>::T*)A.in[1 - p], A.g.Vh},
                                         PlainLinks<R>{A.U, A.g.Vh});
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

// ---------------------------------------------------------------- staged FP32 hop
// The NT output sites of a block are R = NT / hr whole half-rows (hr = L0 / 2 sites of
// one parity) of one (z, t) plane.  Before any arithmetic, warp 0 issues bulk copies
// (cp.async.bulk, completion counted in bytes on one mbarrier) of the block's operands
// into shared memory:
//  * spinors (stage bit 1): the input half field on the block's rows, on the half-row
//    below and the one above them (y neighbours; x neighbours stay in the row), and on
//    the same rows of the planes z -+ 1 and t -+ 1: 5 NT + 2 hr sites, 6 float4 each;
//  * links (stage bit 0): U_mu at the output sites (forward hops) and at the neighbours
//    x - mu (backward hops; for mu = 0 these are the block's own rows of the other
//    parity): 8 NT links of 3 float4.
// Every operand is then read from shared memory.  The arithmetic per site is
// hop_site_io's, so the results are bitwise those of hop_kernel.
//
// Spinor slots per component (NSP = 5 NT + 2 hr): [0, hr) the half-row below,
// [hr, hr + NT) the block's rows, [hr + NT, 2 hr + NT) the half-row above, then the
// rows of z - 1, z + 1, t - 1, t + 1 (NT each).  Link slots: [2 mu + backward][3][NT].

__device__ unsigned g_stage_timeouts;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\tselp.u32 %0, 1, 0, P;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait for phase `parity` of the barrier; gives up after 0.5 s or 2^22 attempts
__device__ __noinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && global_ns() - t0 > 500000000ull) return false;
    }
    return false;
}

// input spinors from the staged slots; (l, r, h) = the output site's index in the
// block, its row in the block and its place in the row
struct SmemIn {
    const float4* sp;
    int NSP, hr, l, r, h, i0;
    template <int MU, int D> __device__ __forceinline__ SpinorF load(int j) const {
        int idx;
        if (MU == 0) idx = hr + (j - i0);
        else if (MU == 1) idx = hr + (r + D) * hr + h;
        else if (MU == 2) idx = 2 * hr + (D > 0 ? 2 : 1) * NT + l;
        else idx = 2 * hr + (D > 0 ? 4 : 3) * NT + l;
        SpinorF s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = sp[k * NSP + idx];
            const int c0 = 2 * k, c1 = 2 * k + 1;
            s.c[c0 / 3][c0 % 3] = {v.x, v.y};
            s.c[c1 / 3][c1 % 3] = {v.z, v.w};
        }
        return s;
    }
};
struct SmemLinks {
    const float4* lk;
    int l, i0;
    template <int MU, int D> __device__ __forceinline__ mat3<float> link(int, int site) const {
        const int slot = 2 * MU + (D < 0);
        const int idx = (MU == 0 && D < 0) ? site - i0 : l;
        const float4* b = lk + slot * 3 * NT + idx;
        return link12_from(b[0], b[NT], b[2 * NT]);
    }
};

template <int ST> constexpr int stage_min_blocks() { return ST == 3 ? 2 : (ST == 2 ? 3 : 4); }

template <bool DAG, int EPI, int CLV, int ST>
__global__ void __launch_bounds__(NT, (stage_min_blocks<ST>())) hop_staged_kernel(HopArgs A, int hr) {
    extern __shared__ __align__(16) float4 stage_smem[];
    __shared__ __align__(8) unsigned long long bar;
    if (A.skip && A.s->done >= 1) return;
    const int blk = A.reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int p = A.parity, Vh = A.g.Vh;
    const int R = NT / hr, NSP = 5 * NT + 2 * hr;
    const int i0 = blk * NT;
    float4* sp = stage_smem;                               // [6][NSP] with bit 1
    float4* lk = stage_smem + ((ST & 2) ? 6 * NSP : 0);    // [8][3][NT] with bit 0
    const uint32_t bar_a = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(bar_a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int L1 = A.g.L[1], L2 = A.g.L[2], L3 = A.g.L[3];
        const int PS = hr * L1;   // sites of one parity in an x-y plane
        const int plane = i0 / PS, off = i0 - plane * PS;
        const int z = plane % L2, t = plane / L2, y0 = off / hr;
        const int base = plane * PS;
        const int ym = base + ((y0 - 1 + L1) % L1) * hr, yp = base + ((y0 + R) % L1) * hr;
        const int zm = (t * L2 + (z - 1 + L2) % L2) * PS + off, zp = (t * L2 + (z + 1) % L2) * PS + off;
        const int tm = (((t - 1 + L3) % L3) * L2 + z) * PS + off, tp = (((t + 1) % L3) * L2 + z) * PS + off;
        if (threadIdx.x == 0)
            mbar_expect_tx(bar_a, (uint32_t)(((ST & 2) ? 6 * NSP : 0) + ((ST & 1) ? 24 * NT : 0)) * 16u);
        __syncwarp();
        if (ST & 2) {
            const float4* in = (const float4*)A.in[1 - p];
            for (int c = threadIdx.x; c < 42; c += 32) {
                const int k = c / 7, part = c % 7;
                int src, dst, n = NT;
                switch (part) {
                case 0: src = i0; dst = hr; break;
                case 1: src = ym; dst = 0; n = hr; break;
                case 2: src = yp; dst = hr + NT; n = hr; break;
                case 3: src = zm; dst = 2 * hr + NT; break;
                case 4: src = zp; dst = 2 * hr + 2 * NT; break;
                case 5: src = tm; dst = 2 * hr + 3 * NT; break;
                default: src = tp; dst = 2 * hr + 4 * NT; break;
                }
                bulk_to_smem(smem_u32(sp + k * NSP + dst), in + (size_t)k * Vh + src, (uint32_t)n * 16u, bar_a);
            }
        }
        if (ST & 1) {
            const float4* U = (const float4*)A.U;
            for (int c = threadIdx.x; c < 27; c += 32) {
                int q = 1 - p, mu, k, src, slot, dst = 0, n = NT;
                if (c < 12) { q = p; mu = c / 3; k = c % 3; src = i0; slot = 2 * mu; }
                else if (c < 15) { mu = 0; k = c - 12; src = i0; slot = 1; }
                else if (c < 18) { mu = 1; k = c - 15; src = i0; slot = 3; dst = hr; n = NT - hr; }
                else if (c < 21) { mu = 1; k = c - 18; src = ym; slot = 3; n = hr; }
                else if (c < 24) { mu = 2; k = c - 21; src = zm; slot = 5; }
                else { mu = 3; k = c - 24; src = tm; slot = 7; }
                if (n > 0)
                    bulk_to_smem(smem_u32(lk + (slot * 3 + k) * NT + dst), U + (size_t)((q * 4 + mu) * 3 + k) * Vh + src,
                                 (uint32_t)n * 16u, bar_a);
            }
        }
    }
    if (A.fin_n > 0 && blockIdx.x == 0) {   // finish the deferred reduction of an earlier launch
        const double acc = ordered_sum(A.partials, A.fin_n);
        if (threadIdx.x == 0) apply_reduce_op(A.s, A.fin_op, A.red_slot, acc);
    }
    bool ok = __syncthreads_and(mbar_wait_bounded(bar_a, 0));
    if (!ok) {
        // the copies did not complete in time: count it, wait (bounded) for the copies
        // still in flight into this block's shared memory, and store NaN
        if (threadIdx.x == 0) atomicAdd(&g_stage_timeouts, 1u);
        mbar_wait_bounded(bar_a, 0);
    }
    const int l = threadIdx.x, i = i0 + l;
    double red;
    if (ok) {
        const int r = l / hr, h = l - r * hr;
        const SmemIn si{sp, NSP, hr, l, r, h, i0};
        const SmemLinks sl{lk, l, i0};
        if constexpr (ST == 3) red = hop_site_io<float, DAG, EPI, CLV>(A, p, i, si, sl);
        else if constexpr (ST == 2) red = hop_site_io<float, DAG, EPI, CLV>(A, p, i, si, PlainLinks<float>{A.U, Vh});
        else red = hop_site_io<float, DAG, EPI, CLV>(A, p, i, PlainIn<float>{(const float4*)A.in[1 - p], Vh}, sl);
    } else {
        SpinorF o;
        const float qnan = __int_as_float(0x7fffffff);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.c[s][c] = {qnan, qnan};
        store_spinor((float4*)(EPI == EPI_CG ? A.r[p] : A.out[p]), Vh, i, o);
        red = (double)qnan;
    }
    if (EPI == EPI_XPAY_NORM || EPI == EPI_CG || EPI == EPI_RESID) {
        const double b = block_sum(red);
        if (A.defer) {
            if (threadIdx.x == 0) A.partials[blk] = b;
        } else {
            grid_reduce(b, A.partials, A.counter, A.s, A.red_op, A.red_slot, blk, gridDim.x);
        }
    }
}

int hop_stage_hr(const Geom& g) {
    const int hr = g.L[0] / 2;
    if (hr < 1 || NT % hr != 0 || g.L[1] % (NT / hr) != 0 || g.Vh % NT != 0) return 0;
    return hr;
}

unsigned hop_stage_timeouts() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_stage_timeouts, sizeof v) != cudaSuccess) return ~0u;
    return v;
}

template <bool DAG, int EPI, int CLV, int ST>
static cudaError_t launch_staged_st(const HopArgs& A, int hr, cudaStream_t st) {
    const size_t bytes = (size_t)(((ST & 2) ? 6 * (5 * NT + 2 * hr) : 0) + ((ST & 1) ? 24 * NT : 0)) * 16;
    // dynamic shared memory this instantiation may use, per device (the attribute is
    // a property of the function on each device)
    constexpr int kDevices = 64;
    static size_t allowed[kDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices || bytes > allowed[dev]) {
        e = cudaFuncSetAttribute(hop_staged_kernel<DAG, EPI, CLV, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kDevices) allowed[dev] = bytes;
    }
    hop_staged_kernel<DAG, EPI, CLV, ST><<<A.g.Vh / NT, NT, bytes, st>>>(A, hr);
    count_launch();
    return cudaGetLastError();
}
template <bool DAG, int EPI, int CLV>
static cudaError_t launch_staged_mode(const HopArgs& A, int hr, cudaStream_t st) {
    switch (A.stage & 3) {
    case 1: return launch_staged_st<DAG, EPI, CLV, 1>(A, hr, st);
    case 2: return launch_staged_st<DAG, EPI, CLV, 2>(A, hr, st);
    default: return launch_staged_st<DAG, EPI, CLV, 3>(A, hr, st);
    }
}
// the staged variant of an FP32 one-parity launch; cudaErrorNotSupported when it has none
template <bool DAG>
static cudaError_t launch_staged(const HopArgs& A, int epi, int hr, cudaStream_t st) {
    if (A.clov) {
        switch (epi) {
        case EPI_HOP: return launch_staged_mode<DAG, EPI_HOP, 1>(A, hr, st);
        case EPI_XPAY_NORM: return launch_staged_mode<DAG, EPI_XPAY_NORM, 2>(A, hr, st);
        case EPI_CG: return launch_staged_mode<DAG, EPI_CG, 2>(A, hr, st);
        default: return cudaErrorNotSupported;
        }
    }
    switch (epi) {
    case EPI_HOP: return launch_staged_mode<DAG, EPI_HOP, 0>(A, hr, st);
    case EPI_XPAY: return launch_staged_mode<DAG, EPI_XPAY, 0>(A, hr, st);
    case EPI_XPAY_NORM: return launch_staged_mode<DAG, EPI_XPAY_NORM, 0>(A, hr, st);
    case EPI_CG: return launch_staged_mode<DAG, EPI_CG, 0>(A, hr, st);
    default: return cudaErrorNotSupported;
    }
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
    if (sizeof(R) == 4 && (A.stage & 3) && A.parity != 2) {
        const int hr = hop_stage_hr(A.g);
        if (hr > 0) {
            cudaError_t e = launch_staged<DAG>(A, epi, hr, st);
            if (e != cudaErrorNotSupported) return e;
        }
    }
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
