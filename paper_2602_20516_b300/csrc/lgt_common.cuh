// lgt_common.cuh -- device-side building blocks of liblgt: complex and SU(3)
// arithmetic, even-odd geometry, Philox-4x32-10, deterministic reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lgt {

constexpr int NT = 128;   // threads per block of the site kernels

// ---------------------------------------------------------------- complex
template <typename R> struct cx { R r, i; };
using dcx = cx<double>;
using fcx = cx<float>;

template <typename R> __device__ __forceinline__ cx<R> mk(R a, R b) { return {a, b}; }
template <typename R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.r + b.r, a.i + b.i}; }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.r - b.r, a.i - b.i}; }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.r, -a.i}; }
template <typename R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return {fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r)};
}
template <typename R> __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.r, s * a.i}; }
template <typename R> __device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.r, -a.i}; }
// acc + a*b
template <typename R> __device__ __forceinline__ cx<R> cmad(cx<R> acc, cx<R> a, cx<R> b) {
    acc.r = fma(a.r, b.r, acc.r); acc.r = fma(-a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i); acc.i = fma(a.i, b.r, acc.i);
    return acc;
}
// acc + conj(a)*b
template <typename R> __device__ __forceinline__ cx<R> cmadc(cx<R> acc, cx<R> a, cx<R> b) {
    acc.r = fma(a.r, b.r, acc.r); acc.r = fma(a.i, b.i, acc.r);
    acc.i = fma(a.r, b.i, acc.i); acc.i = fma(-a.i, b.r, acc.i);
    return acc;
}
// acc + a*conj(b)
template <typename R> __device__ __forceinline__ cx<R> cmad_cb(cx<R> acc, cx<R> a, cx<R> b) {
    acc.r = fma(a.r, b.r, acc.r); acc.r = fma(a.i, b.i, acc.r);
    acc.i = fma(a.i, b.r, acc.i); acc.i = fma(-a.r, b.i, acc.i);
    return acc;
}
template <typename R> __device__ __forceinline__ cx<R> times_i(cx<R> a) { return {-a.i, a.r}; }
template <typename R> __device__ __forceinline__ cx<R> times_mi(cx<R> a) { return {a.i, -a.r}; }
template <typename R> __device__ __forceinline__ R norm2(cx<R> a) { return a.r * a.r + a.i * a.i; }

// ---------------------------------------------------------------- 3x3 matrices
template <typename R> struct mat3 { cx<R> e[3][3]; };
using dmat = mat3<double>;

template <typename R> __device__ __forceinline__ mat3<R> mul(const mat3<R>& a, const mat3<R>& b) {
    mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<R> s = a.e[i][0] * b.e[0][j];
            s = cmad(s, a.e[i][1], b.e[1][j]);
            s = cmad(s, a.e[i][2], b.e[2][j]);
            c.e[i][j] = s;
        }
    return c;
}
// a * b^+
template <typename R> __device__ __forceinline__ mat3<R> mul_nd(const mat3<R>& a, const mat3<R>& b) {
    mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<R> s = {0, 0};
            s = cmad_cb(s, a.e[i][0], b.e[j][0]);
            s = cmad_cb(s, a.e[i][1], b.e[j][1]);
            s = cmad_cb(s, a.e[i][2], b.e[j][2]);
            c.e[i][j] = s;
        }
    return c;
}
// a^+ * b
template <typename R> __device__ __forceinline__ mat3<R> mul_dn(const mat3<R>& a, const mat3<R>& b) {
    mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<R> s = {0, 0};
            s = cmadc(s, a.e[0][i], b.e[0][j]);
            s = cmadc(s, a.e[1][i], b.e[1][j]);
            s = cmadc(s, a.e[2][i], b.e[2][j]);
            c.e[i][j] = s;
        }
    return c;
}
template <typename R> __device__ __forceinline__ mat3<R> dag(const mat3<R>& a) {
    mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.e[i][j] = conj(a.e[j][i]);
    return c;
}
template <typename R> __device__ __forceinline__ void add_to(mat3<R>& a, const mat3<R>& b) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.e[i][j] = a.e[i][j] + b.e[i][j];
}
template <typename R> __device__ __forceinline__ mat3<R> zero3() {
    mat3<R> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.e[i][j] = {0, 0};
    return c;
}
template <typename R> __device__ __forceinline__ R retrace(const mat3<R>& a) {
    return a.e[0][0].r + a.e[1][1].r + a.e[2][2].r;
}

// Lie components of M: c_a = Im tr(lambda^a M) = 2 Im tr(T^a M), a = 0..7.
template <typename R>
__device__ __forceinline__ void lie_im_tr(const mat3<R>& M, R c[8]) {
    const R is3 = (R)0.57735026918962576451;  // 1/sqrt(3)
    c[0] = M.e[0][1].i + M.e[1][0].i;
    c[1] = M.e[0][1].r - M.e[1][0].r;
    c[2] = M.e[0][0].i - M.e[1][1].i;
    c[3] = M.e[0][2].i + M.e[2][0].i;
    c[4] = M.e[0][2].r - M.e[2][0].r;
    c[5] = M.e[1][2].i + M.e[2][1].i;
    c[6] = M.e[1][2].r - M.e[2][1].r;
    c[7] = (M.e[0][0].i + M.e[1][1].i - (R)2 * M.e[2][2].i) * is3;
}
// P = sum_a p_a T^a (Hermitian traceless)
__device__ __forceinline__ dmat herm_from_lie(const double p[8]) {
    const double is3 = 0.57735026918962576451;
    dmat P;
    P.e[0][0] = {0.5 * (p[2] + p[7] * is3), 0};
    P.e[1][1] = {0.5 * (-p[2] + p[7] * is3), 0};
    P.e[2][2] = {-p[7] * is3, 0};
    P.e[0][1] = {0.5 * p[0], -0.5 * p[1]};
    P.e[1][0] = {0.5 * p[0], 0.5 * p[1]};
    P.e[0][2] = {0.5 * p[3], -0.5 * p[4]};
    P.e[2][0] = {0.5 * p[3], 0.5 * p[4]};
    P.e[1][2] = {0.5 * p[5], -0.5 * p[6]};
    P.e[2][1] = {0.5 * p[5], 0.5 * p[6]};
    return P;
}

// ---------------------------------------------------------------- geometry
struct Geom {
    int L[4];
    int Vh;
    int V;
    int stride[4];   // lexicographic strides 1, L0, L0 L1, L0 L1 L2
};

// coordinates of even-odd site (parity p, index i); returns lexicographic index
__device__ __forceinline__ int eo_coords(const Geom& g, int p, int i, int x[4]) {
    int lex2 = 2 * i;
    int x0h = lex2 % g.L[0];
    int rest = lex2 / g.L[0];
    x[1] = rest % g.L[1]; rest /= g.L[1];
    x[2] = rest % g.L[2];
    x[3] = rest / g.L[2];
    x[0] = x0h + ((p + x[1] + x[2] + x[3]) & 1);
    return lex2 - x0h + x[0];
}
// lexicographic index of the neighbour one step along mu (dir +1 / -1)
__device__ __forceinline__ int nb_lex(const Geom& g, int lex, const int x[4], int mu, int dir) {
    if (dir > 0) return (x[mu] == g.L[mu] - 1) ? lex - (g.L[mu] - 1) * g.stride[mu] : lex + g.stride[mu];
    return (x[mu] == 0) ? lex + (g.L[mu] - 1) * g.stride[mu] : lex - g.stride[mu];
}

// ---------------------------------------------------------------- field access
// FP64 spinor half field: double2 [12][Vh]
struct SpinorD { dcx c[4][3]; };
struct SpinorF { fcx c[4][3]; };

__device__ __forceinline__ SpinorD load_spinor(const double2* __restrict__ f, int Vh, int i) {
    SpinorD s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 v = __ldg(f + (size_t)k * Vh + i);
        s.c[k / 3][k % 3] = {v.x, v.y};
    }
    return s;
}
__device__ __forceinline__ void store_spinor(double2* __restrict__ f, int Vh, int i, const SpinorD& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) f[(size_t)k * Vh + i] = make_double2(s.c[k / 3][k % 3].r, s.c[k / 3][k % 3].i);
}
__device__ __forceinline__ SpinorF load_spinor(const float4* __restrict__ f, int Vh, int i) {
    SpinorF s;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 v = __ldg(f + (size_t)k * Vh + i);
        int c0 = 2 * k, c1 = 2 * k + 1;
        s.c[c0 / 3][c0 % 3] = {v.x, v.y};
        s.c[c1 / 3][c1 % 3] = {v.z, v.w};
    }
    return s;
}
__device__ __forceinline__ void store_spinor(float4* __restrict__ f, int Vh, int i, const SpinorF& s) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        int c0 = 2 * k, c1 = 2 * k + 1;
        f[(size_t)k * Vh + i] = make_float4(s.c[c0 / 3][c0 % 3].r, s.c[c0 / 3][c0 % 3].i,
                                            s.c[c1 / 3][c1 % 3].r, s.c[c1 / 3][c1 % 3].i);
    }
}

// FP64 links: double2 [parity][4][9][Vh]
__device__ __forceinline__ dmat load_link(const double2* __restrict__ U, int Vh, int p, int mu, int i) {
    const double2* b = U + (size_t)((p * 4 + mu) * 9) * Vh + i;
    dmat m;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 v = __ldg(b + (size_t)k * Vh);
        m.e[k / 3][k % 3] = {v.x, v.y};
    }
    return m;
}
__device__ __forceinline__ void store_link(double2* __restrict__ U, int Vh, int p, int mu, int i, const dmat& m) {
    double2* b = U + (size_t)((p * 4 + mu) * 9) * Vh + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) b[(size_t)k * Vh] = make_double2(m.e[k / 3][k % 3].r, m.e[k / 3][k % 3].i);
}
// FP32 two-row links: float4 [parity][4][3][Vh]; row 3 = conj(row1 x row2)
// the SU(3) matrix from its first two rows, stored as the three float4 a, c, d
__device__ __forceinline__ mat3<float> link12_from(float4 a, float4 c, float4 d) {
    mat3<float> m;
    m.e[0][0] = {a.x, a.y}; m.e[0][1] = {a.z, a.w}; m.e[0][2] = {c.x, c.y};
    m.e[1][0] = {c.z, c.w}; m.e[1][1] = {d.x, d.y}; m.e[1][2] = {d.z, d.w};
    m.e[2][0] = conj(m.e[0][1] * m.e[1][2] - m.e[0][2] * m.e[1][1]);
    m.e[2][1] = conj(m.e[0][2] * m.e[1][0] - m.e[0][0] * m.e[1][2]);
    m.e[2][2] = conj(m.e[0][0] * m.e[1][1] - m.e[0][1] * m.e[1][0]);
    return m;
}
__device__ __forceinline__ mat3<float> load_link12(const float4* __restrict__ U, int Vh, int p, int mu, int i) {
    const float4* b = U + (size_t)((p * 4 + mu) * 3) * Vh + i;
    return link12_from(__ldg(b), __ldg(b + Vh), __ldg(b + 2 * (size_t)Vh));
}
__device__ __forceinline__ void store_link12(float4* __restrict__ U, int Vh, int p, int mu, int i, const dmat& m) {
    float4* b = U + (size_t)((p * 4 + mu) * 3) * Vh + i;
    b[0] = make_float4((float)m.e[0][0].r, (float)m.e[0][0].i, (float)m.e[0][1].r, (float)m.e[0][1].i);
    b[Vh] = make_float4((float)m.e[0][2].r, (float)m.e[0][2].i, (float)m.e[1][0].r, (float)m.e[1][0].i);
    b[2 * (size_t)Vh] = make_float4((float)m.e[1][1].r, (float)m.e[1][1].i, (float)m.e[1][2].r, (float)m.e[1][2].i);
}

// momenta: double2 [parity][4][4][Vh]
__device__ __forceinline__ void load_mom(const double2* __restrict__ m, int Vh, int p, int mu, int i, double v[8]) {
    const double2* b = m + (size_t)((p * 4 + mu) * 4) * Vh + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) { double2 t = b[(size_t)k * Vh]; v[2 * k] = t.x; v[2 * k + 1] = t.y; }
}
__device__ __forceinline__ void store_mom(double2* __restrict__ m, int Vh, int p, int mu, int i, const double v[8]) {
    double2* b = m + (size_t)((p * 4 + mu) * 4) * Vh + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) b[(size_t)k * Vh] = make_double2(v[2 * k], v[2 * k + 1]);
}

// ---------------------------------------------------------------- Philox-4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds, multipliers on words 0 and 2,
// Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}
// Box-Muller pair from one Philox block; counter (c0, c1, c2, c3), key = seed
__device__ __forceinline__ void gauss_pair(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           double& g0, double& g1) {
    uint4 o = philox(make_uint4(c0, c1, c2, c3), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    double v1 = u53(o.x, o.y), v2 = u53(o.z, o.w);
    double r = sqrt(-2.0 * log(v1));
    double s, c;
    sincospi(2.0 * v2, &s, &c);
    g0 = r * c;
    g1 = r * s;
}
enum { FIELD_MOMENTA = 1, FIELD_XI = 2, FIELD_LINKS = 3, FIELD_METROPOLIS = 4, FIELD_SOURCE = 5 };

// ---------------------------------------------------------------- solver scalars
struct Scalars {
    double rr;        // current |r|^2
    double rr_old;
    double pAp;
    double alpha, beta;
    double rr_max;    // max |r|^2 since the last reliable update
    double target;    // stop when rr <= target
    double delta2;    // reliable-update trigger: rr < delta2 * rr_max (0 disables)
    int done;         // 0 running; 1 stop condition fired; 2 final p-update done
    int iters;
    int nan;
    int pad;
    double slot[8];   // generic reduction results
};

enum ReduceOp { RED_STORE = 0, RED_PAP = 1, RED_RR = 2 };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
// fixed-order block sum of NT threads (result in thread 0)
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[NT / 32];
    __syncthreads();
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < NT / 32) ? sh[l] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

__device__ __forceinline__ void apply_reduce_op(Scalars* s, int op, int slot, double v) {
    if (op == RED_STORE) {
        s->slot[slot] = v;
    } else if (op == RED_PAP) {
        s->pAp = v;
        if (!(v > 0.0) || !isfinite(v)) { s->nan = 1; s->done = 2; s->alpha = 0.0; }
        else s->alpha = s->rr / v;
    } else {  // RED_RR
        double rr_new = v;
        s->beta = rr_new / s->rr;
        s->rr_old = s->rr;
        s->rr = rr_new;
        s->iters += 1;
        if (rr_new > s->rr_max) s->rr_max = rr_new;
        if (!isfinite(rr_new)) { s->nan = 1; s->done = 2; }
        else if (rr_new <= s->target || rr_new < s->delta2 * s->rr_max) s->done = 1;
    }
}

// Sum of partials[0 .. n) by the whole block in a fixed order (result in thread 0):
// eight independent loads in flight per thread, the same result on every run.
__device__ __forceinline__ double ordered_sum(const double* partials, int n) {
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < n; k += 8 * NT) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (k + j * NT < n) a[j] += __ldcg(partials + k + j * NT);
    }
    const double acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    return block_sum(acc);
}

// Deterministic grid reduction over the nblk blocks of one problem (blk = this
// block's index among them): each block stores its partial, the last block to
// finish sums all partials in index order and applies `op` to the scalars.
__device__ __forceinline__ void grid_reduce(double block_partial, double* partials, unsigned* counter,
                                            Scalars* s, int op, int slot, int blk, int nblk) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blk] = block_partial;
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double acc = ordered_sum(partials, nblk);
    if (threadIdx.x == 0) {
        *counter = 0u;
        apply_reduce_op(s, op, slot, acc);
    }
}
__device__ __forceinline__ void grid_reduce(double block_partial, double* partials, unsigned* counter,
                                            Scalars* s, int op, int slot) {
    grid_reduce(block_partial, partials, counter, s, op, slot, blockIdx.x, gridDim.x);
}

}  // namespace lgt
