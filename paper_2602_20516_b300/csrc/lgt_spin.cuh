// lgt_spin.cuh -- spin projection of the Wilson hopping term in the chiral
// basis g_k = [[0,-i s_k],[i s_k,0]] (mu = k-1 < 3), g_4 = [[0,1],[1,0]] (mu = 3):
// (1 + S g_mu) psi has two independent spin rows h0, h1; rows 2, 3 are
// multiples (+-1, +-i) of them.
#pragma once
#include "lgt_common.cuh"

namespace lgt {

// (1 + S g_MU) psi = (h0, h1, recon): h_j are two colour vectors.  C is a complex
// type with +, - and times_i (cx<float>, cx<double> or the double-float dfc).
template <int MU, int S, typename C>
__device__ __forceinline__ void project(const C (&psi)[4][3], C (&h)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) {
            h[0][c] = (S < 0) ? psi[0][c] + times_i(psi[3][c]) : psi[0][c] - times_i(psi[3][c]);
            h[1][c] = (S < 0) ? psi[1][c] + times_i(psi[2][c]) : psi[1][c] - times_i(psi[2][c]);
        } else if (MU == 1) {
            h[0][c] = (S < 0) ? psi[0][c] + psi[3][c] : psi[0][c] - psi[3][c];
            h[1][c] = (S < 0) ? psi[1][c] - psi[2][c] : psi[1][c] + psi[2][c];
        } else if (MU == 2) {
            h[0][c] = (S < 0) ? psi[0][c] + times_i(psi[2][c]) : psi[0][c] - times_i(psi[2][c]);
            h[1][c] = (S < 0) ? psi[1][c] - times_i(psi[3][c]) : psi[1][c] + times_i(psi[3][c]);
        } else {
            h[0][c] = (S < 0) ? psi[0][c] - psi[2][c] : psi[0][c] + psi[2][c];
            h[1][c] = (S < 0) ? psi[1][c] - psi[3][c] : psi[1][c] + psi[3][c];
        }
    }
}

// out += (1 + S g_MU) reconstructed from the multiplied half spinor uh (C as in project,
// with times_mi as well)
template <int MU, int S, typename C>
__device__ __forceinline__ void accumulate(C (&out)[4][3], const C (&uh)[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        out[0][c] = out[0][c] + uh[0][c];
        out[1][c] = out[1][c] + uh[1][c];
        if (MU == 0) {
            out[2][c] = (S < 0) ? out[2][c] + times_mi(uh[1][c]) : out[2][c] + times_i(uh[1][c]);
            out[3][c] = (S < 0) ? out[3][c] + times_mi(uh[0][c]) : out[3][c] + times_i(uh[0][c]);
        } else if (MU == 1) {
            out[2][c] = (S < 0) ? out[2][c] - uh[1][c] : out[2][c] + uh[1][c];
            out[3][c] = (S < 0) ? out[3][c] + uh[0][c] : out[3][c] - uh[0][c];
        } else if (MU == 2) {
            out[2][c] = (S < 0) ? out[2][c] + times_mi(uh[0][c]) : out[2][c] + times_i(uh[0][c]);
            out[3][c] = (S < 0) ? out[3][c] + times_i(uh[1][c]) : out[3][c] + times_mi(uh[1][c]);
        } else {
            out[2][c] = (S < 0) ? out[2][c] - uh[0][c] : out[2][c] + uh[0][c];
            out[3][c] = (S < 0) ? out[3][c] - uh[1][c] : out[3][c] + uh[1][c];
        }
    }
}

}  // namespace lgt
