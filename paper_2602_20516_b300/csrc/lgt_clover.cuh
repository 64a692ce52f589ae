// lgt_clover.cuh -- the FP32 copy of a clover block field (1 + A or its inverse on
// the sites of a parity), stored Hermitian-packed: each of the two 6 x 6 chiral
// blocks is Hermitian, so its 6 real diagonal entries and the 15 entries above the
// diagonal determine it.
//
// Layout: float4 [parity][18][Vh]; chiral block c occupies float4 9c .. 9c+8 as 36
// floats: the diagonal d_0 .. d_5, then the entries (r, q), r < q, row by row, as
// (re, im).  288 B per site instead of 576 B for the full blocks; every CG operator
// application of the even-odd clover action reads such a field twice.
#pragma once
#include "lgt_common.cuh"

namespace lgt {

// float offset of entry (r, q), r < q, inside a packed block
__host__ __device__ constexpr int clover_upper_index(int r, int q) {
    // entries before row r: 5 + 4 + ... (r terms) = r (11 - r) / 2
    return 6 + 2 * (r * (11 - r) / 2 + (q - r - 1));
}

// w = B v for the two chiral blocks of site i (v, w: the 12 spin-colour components,
// chiral block c acting on components 6c .. 6c+5); Cp = the parity's [18][Vh] block
__device__ __forceinline__ void clover_mul_f32(const float4* __restrict__ Cp, int Vh, int i, const fcx (&v)[12],
                                               fcx (&w)[12]) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float f[36];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 z = __ldg(Cp + (size_t)(9 * c + k) * Vh + i);
            f[4 * k] = z.x; f[4 * k + 1] = z.y; f[4 * k + 2] = z.z; f[4 * k + 3] = z.w;
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const fcx vr = v[6 * c + r];
            fcx s = {f[r] * vr.r, f[r] * vr.i};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                if (q == r) continue;
                const int o = r < q ? clover_upper_index(r, q) : clover_upper_index(q, r);
                const fcx z = {f[o], r < q ? f[o + 1] : -f[o + 1]};   // B_rq = conj(B_qr) below the diagonal
                s = cmad(s, z, v[6 * c + q]);
            }
            w[6 * c + r] = s;
        }
    }
}

// write chiral block c (a full 6 x 6 Hermitian matrix in FP64) to the packed FP32 field
// (o32 = the parity's [18][Vh] block + site index)
__device__ __forceinline__ void clover_store_f32(float4* o32, int Vh, int c, const dcx (&B)[6][6]) {
    float f[36];
#pragma unroll
    for (int r = 0; r < 6; ++r) f[r] = (float)B[r][r].r;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int q = r + 1; q < 6; ++q) {
            f[clover_upper_index(r, q)] = (float)B[r][q].r;
            f[clover_upper_index(r, q) + 1] = (float)B[r][q].i;
        }
#pragma unroll
    for (int k = 0; k < 9; ++k)
        o32[(size_t)(9 * c + k) * Vh] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

}  // namespace lgt
