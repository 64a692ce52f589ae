// lgt_df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  On this part an
// FP64 FMA issues at 1/64 of the FP32 rate, so FP64-accurate products of link
// matrices are cheaper as FP32 pairs.  Built from the error-free transformations
// TwoSum (Knuth) and TwoProduct with a fused multiply-add (Dekker's product without
// splitting); a dot product keeps one running FP32 sum with its rounding errors
// collected in a second FP32 word, as in the compensated dot product Dot2 of Ogita,
// Rump and Oishi (SIAM J. Sci. Comput. 26 (2005) 1955), with the low words of the
// operands entering through the error word.
//
// Every addition and product whose rounding error is captured uses the _rn
// intrinsics, which the compiler never contracts into an FMA.
#pragma once
#include "lgt_common.cuh"
#include "lgt_su3.cuh"

namespace lgt {

struct df { float h, l; };
struct dfc { df r, i; };
struct dfmat { dfc e[3][3]; };

__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }

__device__ __forceinline__ df df_from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// h + l = s + c with |l| <= ulp(h)/2 (needs |s| >= |c| or s = 0)
__device__ __forceinline__ df fast_renorm(float s, float c) {
    const float h = __fadd_rn(s, c);
    return {h, __fsub_rn(c, __fsub_rn(h, s))};
}

__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return fast_renorm(s, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfc operator+(const dfc& a, const dfc& b) { return {df_add(a.r, b.r), df_add(a.i, b.i)}; }
__device__ __forceinline__ dfc operator-(const dfc& a, const dfc& b) { return {df_sub(a.r, b.r), df_sub(a.i, b.i)}; }
__device__ __forceinline__ dfc operator-(const dfc& a) { return {df_neg(a.r), df_neg(a.i)}; }
__device__ __forceinline__ dfc times_i(const dfc& a) { return {df_neg(a.i), a.r}; }
__device__ __forceinline__ dfc times_mi(const dfc& a) { return {a.i, df_neg(a.r)}; }

// compensated accumulator: value s + c
struct dacc {
    float s, c;
};
__device__ __forceinline__ dacc dacc0() { return {0.f, 0.f}; }
// A += a * b  (a, b double-floats; the lo*lo term is below the format's precision)
__device__ __forceinline__ void dacc_mul(dacc& A, df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);   // exact rounding error of the product
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float s, t;
    two_sum(A.s, p, s, t);
    A.s = s;
    A.c = __fadd_rn(A.c, __fadd_rn(t, e));
}
// A += a (a double-float)
__device__ __forceinline__ void dacc_add(dacc& A, df a) {
    float s, t;
    two_sum(A.s, a.h, s, t);
    A.s = s;
    A.c = __fadd_rn(A.c, __fadd_rn(t, a.l));
}
__device__ __forceinline__ df dacc_get(const dacc& A) {
    // s carries the leading part; renormalise with TwoSum (no magnitude assumption)
    float h, l;
    two_sum(A.s, A.c, h, l);
    return {h, l};
}

// complex multiply-accumulate into a pair of accumulators (re, im):
//   conj flags select a, b or their conjugates
template <bool CA, bool CB>
__device__ __forceinline__ void cacc_mul(dacc& re, dacc& im, const dfc& a, const dfc& b) {
    const df ai = CA ? df_neg(a.i) : a.i;
    const df bi = CB ? df_neg(b.i) : b.i;
    dacc_mul(re, a.r, b.r);
    dacc_mul(re, df_neg(ai), bi);
    dacc_mul(im, a.r, bi);
    dacc_mul(im, ai, b.r);
}

// C = op(A) op(B) with op = identity or Hermitian conjugate
template <bool DA, bool DB>
__device__ __forceinline__ dfmat df_mul(const dfmat& A, const dfmat& B) {
    dfmat C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dacc re = dacc0(), im = dacc0();
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const dfc& a = DA ? A.e[k][i] : A.e[i][k];
                const dfc& b = DB ? B.e[j][k] : B.e[k][j];
                cacc_mul<DA, DB>(re, im, a, b);
            }
            C.e[i][j] = {dacc_get(re), dacc_get(im)};
        }
    return C;
}
// C = A B and C += A B with the row loop kept as a loop: a third of the code of the
// unrolled products, for kernels that chain many products per thread and would
// otherwise outgrow the instruction cache.  The row of A and the row of C are picked
// with selects, not by indexing with the loop counter: an indexed register array
// would live in local memory, and in the clover force that traffic went to DRAM.
__device__ __forceinline__ dfc dfc_sel3(int i, const dfc& a0, const dfc& a1, const dfc& a2) {
    return i == 0 ? a0 : (i == 1 ? a1 : a2);
}
__device__ __forceinline__ void df_mul_rows(dfmat& C, const dfmat& A, const dfmat& B, bool acc) {
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
        dfc a[3], c[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = dfc_sel3(i, A.e[0][k], A.e[1][k], A.e[2][k]);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const dfc c0 = dfc_sel3(i, C.e[0][j], C.e[1][j], C.e[2][j]);
            dacc re = acc ? dacc{c0.r.h, c0.r.l} : dacc0();
            dacc im = acc ? dacc{c0.i.h, c0.i.l} : dacc0();
#pragma unroll
            for (int k = 0; k < 3; ++k) cacc_mul<false, false>(re, im, a[k], B.e[k][j]);
            c[j] = {dacc_get(re), dacc_get(im)};
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (r == i) C.e[r][j] = c[j];
    }
}

// C += op(A) op(B): the accumulators start from the entries of C (hi, lo)
template <bool DA, bool DB>
__device__ __forceinline__ void df_mul_acc(dfmat& C, const dfmat& A, const dfmat& B) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dacc re = {C.e[i][j].r.h, C.e[i][j].r.l}, im = {C.e[i][j].i.h, C.e[i][j].i.l};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const dfc& a = DA ? A.e[k][i] : A.e[i][k];
                const dfc& b = DB ? B.e[j][k] : B.e[k][j];
                cacc_mul<DA, DB>(re, im, a, b);
            }
            C.e[i][j] = {dacc_get(re), dacc_get(im)};
        }
}
__device__ __forceinline__ void df_add_to(dfmat& A, const dfmat& B) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A.e[i][j].r = df_add(A.e[i][j].r, B.e[i][j].r);
            A.e[i][j].i = df_add(A.e[i][j].i, B.e[i][j].i);
        }
}
__device__ __forceinline__ dfmat df_zero3() {
    dfmat C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C.e[i][j] = {{0.f, 0.f}, {0.f, 0.f}};
    return C;
}

// double-float links: float4 [parity][4][9][Vh], entry k = (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ dfmat load_link_df(const float4* __restrict__ U, int Vh, int p, int mu, int i) {
    const float4* b = U + (size_t)((p * 4 + mu) * 9) * Vh + i;
    dfmat m;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float4 v = __ldg(b + (size_t)k * Vh);
        m.e[k / 3][k % 3] = {{v.x, v.y}, {v.z, v.w}};
    }
    return m;
}
__device__ __forceinline__ void store_link_df(float4* __restrict__ U, int Vh, int p, int mu, int i, const dmat& m) {
    float4* b = U + (size_t)((p * 4 + mu) * 9) * Vh + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const df r = df_from(m.e[k / 3][k % 3].r), im = df_from(m.e[k / 3][k % 3].i);
        b[(size_t)k * Vh] = make_float4(r.h, r.l, im.h, im.l);
    }
}

// double-float spinor half field: float4 [12][Vh], entry k = 3 spin + colour =
// (re.hi, re.lo, im.hi, im.lo)
struct SpinorDF { dfc c[4][3]; };
__device__ __forceinline__ SpinorDF load_spinor_df(const float4* __restrict__ f, int Vh, int i) {
    SpinorDF s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float4 v = __ldg(f + (size_t)k * Vh + i);
        s.c[k / 3][k % 3] = {{v.x, v.y}, {v.z, v.w}};
    }
    return s;
}
__device__ __forceinline__ void store_spinor_df(float4* __restrict__ f, int Vh, int i, const SpinorDF& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const dfc& v = s.c[k / 3][k % 3];
        f[(size_t)k * Vh + i] = make_float4(v.r.h, v.r.l, v.i.h, v.i.l);
    }
}

// the double-float link U_mu at coordinates x
__device__ __forceinline__ dfmat link_df_at(const float4* U, const Geom& g, const int x[4], int mu) {
    const int lex = lex_of(g, x);
    return load_link_df(U, g.Vh, (x[0] + x[1] + x[2] + x[3]) & 1, mu, lex >> 1);
}

// the double-float link U_mu at coordinates x, or its Hermitian conjugate
__device__ __forceinline__ dfmat link_df_op(const float4* U, const Geom& g, const int x[4], int mu, bool dag) {
    const int lex = lex_of(g, x);
    const float4* b = U + (size_t)((((x[0] + x[1] + x[2] + x[3]) & 1) * 4 + mu) * 9) * g.Vh + (lex >> 1);
    dfmat m;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 v = __ldg(b + (size_t)(dag ? 3 * c + a : 3 * a + c) * g.Vh);
            m.e[a][c] = {{v.x, v.y}, dag ? df{-v.z, -v.w} : df{v.z, v.w}};
        }
    return m;
}

// Lie components c_a = Im tr(lambda^a M) of a double-float matrix, in FP64
__device__ __forceinline__ void lie_im_tr_df(const dfmat& M, double c[8]) {
    c[0] = df_to(df_add(M.e[0][1].i, M.e[1][0].i));
    c[1] = df_to(df_sub(M.e[0][1].r, M.e[1][0].r));
    c[2] = df_to(df_sub(M.e[0][0].i, M.e[1][1].i));
    c[3] = df_to(df_add(M.e[0][2].i, M.e[2][0].i));
    c[4] = df_to(df_sub(M.e[0][2].r, M.e[2][0].r));
    c[5] = df_to(df_add(M.e[1][2].i, M.e[2][1].i));
    c[6] = df_to(df_sub(M.e[1][2].r, M.e[2][1].r));
    const df d = df_sub(df_add(M.e[0][0].i, M.e[1][1].i), df_add(M.e[2][2].i, M.e[2][2].i));
    c[7] = df_to(d) * 0.57735026918962576451;
}

}  // namespace lgt
