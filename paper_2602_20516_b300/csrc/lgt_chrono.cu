// lgt_chrono.cu -- initial guess for a solve from the solutions of earlier solves of
// the same system (the chronological inverter of Brower, Ivanenko, Levi and Orginos,
// Nucl. Phys. B484 (1997) 353): with V = (v_1 .. v_N) the last N solutions, the
// guess x0 = V c minimises the A-norm of the error over span(V), i.e.
//   (V^+ A V) c = V^+ b.
// Kernels: many complex inner products in one launch (deterministic two-level
// reduction per product), the N x N Hermitian solve (one thread, Cholesky), and the
// combination x0 = sum_i c_i v_i.
#include "lgt_internal.h"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

template <typename TB> struct CdotLoad;
template <> struct CdotLoad<double2> {
    // complex entries k = 0..11 of a site: double2 [12][Vh]
    static __device__ __forceinline__ void site(const double2* f, int Vh, int i, double (&re)[12], double (&im)[12]) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 v = __ldg(f + (size_t)k * Vh + i);
            re[k] = v.x; im[k] = v.y;
        }
    }
};
template <> struct CdotLoad<float4> {
    // float4 [6][Vh]: entry j holds components 2j, 2j+1
    static __device__ __forceinline__ void site(const float4* f, int Vh, int i, double (&re)[12], double (&im)[12]) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float4 v = __ldg(f + (size_t)j * Vh + i);
            re[2 * j] = v.x; im[2 * j] = v.y; re[2 * j + 1] = v.z; im[2 * j + 1] = v.w;
        }
    }
};

// out[m] = <a_m, b_m> = sum conj(a_m) b_m over the half field, m = blockIdx.y
template <typename TB>
__global__ void __launch_bounds__(NT) cdot_many_kernel(CdotArgs D) {
    const int m = blockIdx.y;
    const int i = blockIdx.x * NT + threadIdx.x;
    double sr = 0.0, si = 0.0;
    if (i < D.Vh) {
        double ar[12], ai[12], br[12], bi[12];
        CdotLoad<double2>::site((const double2*)D.a[m], D.Vh, i, ar, ai);
        CdotLoad<TB>::site((const TB*)D.b[m], D.Vh, i, br, bi);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            sr = fma(ar[k], br[k], fma(ai[k], bi[k], sr));
            si = fma(ar[k], bi[k], fma(-ai[k], br[k], si));
        }
    }
    sr = block_sum(sr);
    si = block_sum(si);
    __shared__ bool last;
    double2* part = D.partials + (size_t)m * gridDim.x;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = make_double2(sr, si);
        __threadfence();
        const unsigned prev = atomicAdd(D.counter + m, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double ar = 0.0, ai = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += NT) {
        const double2 v = __ldcg(part + k);
        ar += v.x;
        ai += v.y;
    }
    ar = block_sum(ar);
    ai = block_sum(ai);
    if (threadIdx.x == 0) {
        D.counter[m] = 0u;
        D.out[m] = make_double2(ar, ai);
    }
}

cudaError_t cdot_many(const CdotArgs& D, int M, bool b_fp32, cudaStream_t st) {
    if (M < 1 || M > CDOT_MAX) return cudaErrorInvalidValue;
    const dim3 grid(grid_for(D.Vh), M);
    if ((long)grid.x * M > D.capacity) return cudaErrorInvalidValue;
    if (b_fp32) cdot_many_kernel<float4><<<grid, NT, 0, st>>>(D);
    else cdot_many_kernel<double2><<<grid, NT, 0, st>>>(D);
    count_launch();
    return cudaGetLastError();
}

// G (N x N, row-major, G[i*N+j] = <v_i, A v_j>) and g (N) -> c with G c = g.  G is
// Hermitian positive definite for independent v; the Hermitian part is used.  The
// products A v are FP32 (relative error ~1e-7), and successive MD solutions are close
// to parallel: a vector whose Cholesky pivot (the squared A-norm of its part not
// spanned by the vectors before it) is below 1e-6 of the largest diagonal entry is
// at the FP32 noise level of G, gets c = 0 and is left out.  Result in c[0..N),
// count kept in *used.
__global__ void chrono_solve_kernel(const double2* G, const double2* g, double2* c, int N, int* used) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double Lr[CHRONO_MAX][CHRONO_MAX], Li[CHRONO_MAX][CHRONO_MAX];
    bool keep[CHRONO_MAX];
    double dmax = 0.0;
    for (int i = 0; i < N; ++i) dmax = fmax(dmax, G[i * N + i].x);
    int n_used = 0;
    // Cholesky G = L L^+ on the kept vectors (column by column)
    for (int j = 0; j < N; ++j) {
        double d = G[j * N + j].x;
        for (int k = 0; k < j; ++k)
            if (keep[k]) d -= Lr[j][k] * Lr[j][k] + Li[j][k] * Li[j][k];
        keep[j] = d > 1e-6 * dmax;
        for (int i = 0; i < N; ++i) { Lr[i][j] = 0.0; Li[i][j] = 0.0; }
        if (!keep[j]) continue;
        ++n_used;
        const double dj = sqrt(d);
        Lr[j][j] = dj;
        for (int i = j + 1; i < N; ++i) {
            // Hermitian part: (G_ij + conj(G_ji)) / 2
            double sr = 0.5 * (G[i * N + j].x + G[j * N + i].x);
            double si = 0.5 * (G[i * N + j].y - G[j * N + i].y);
            for (int k = 0; k < j; ++k) {
                if (!keep[k]) continue;
                // s -= L_ik conj(L_jk)
                sr -= Lr[i][k] * Lr[j][k] + Li[i][k] * Li[j][k];
                si -= Li[i][k] * Lr[j][k] - Lr[i][k] * Li[j][k];
            }
            Lr[i][j] = sr / dj;
            Li[i][j] = si / dj;
        }
    }
    // forward substitution L y = g, back substitution L^+ c = y (kept rows only)
    double yr[CHRONO_MAX], yi[CHRONO_MAX];
    for (int i = 0; i < N; ++i) {
        yr[i] = yi[i] = 0.0;
        if (!keep[i]) continue;
        double sr = g[i].x, si = g[i].y;
        for (int k = 0; k < i; ++k) {
            if (!keep[k]) continue;
            sr -= Lr[i][k] * yr[k] - Li[i][k] * yi[k];
            si -= Lr[i][k] * yi[k] + Li[i][k] * yr[k];
        }
        yr[i] = sr / Lr[i][i];
        yi[i] = si / Lr[i][i];
    }
    for (int i = N - 1; i >= 0; --i) {
        if (!keep[i]) { c[i] = make_double2(0.0, 0.0); continue; }
        double sr = yr[i], si = yi[i];
        for (int k = i + 1; k < N; ++k) {
            if (!keep[k]) continue;
            // s -= conj(L_ki) c_k
            const double2 ck = c[k];
            sr -= Lr[k][i] * ck.x + Li[k][i] * ck.y;
            si -= Lr[k][i] * ck.y - Li[k][i] * ck.x;
        }
        c[i] = make_double2(sr / Lr[i][i], si / Lr[i][i]);
    }
    *used = n_used;
}

cudaError_t chrono_solve(const double2* G, const double2* g, double2* c, int N, int* used, cudaStream_t st) {
    if (N < 1 || N > CHRONO_MAX) return cudaErrorInvalidValue;
    chrono_solve_kernel<<<1, 32, 0, st>>>(G, g, c, N, used);
    count_launch();
    return cudaGetLastError();
}

// x = sum_i c_i v_i over FP64 half fields (double2 [12][Vh])
struct CombineArgs {
    const double2* v[CHRONO_MAX];
    const double2* c;
    double2* x;
    int N;
    long ne;
};
__global__ void __launch_bounds__(NT) chrono_combine_kernel(CombineArgs C) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= C.ne) return;
    double xr = 0.0, xi = 0.0;
#pragma unroll
    for (int i = 0; i < CHRONO_MAX; ++i) {
        if (i >= C.N) break;
        const double2 ci = C.c[i], v = __ldg(C.v[i] + e);
        xr = fma(ci.x, v.x, fma(-ci.y, v.y, xr));
        xi = fma(ci.x, v.y, fma(ci.y, v.x, xi));
    }
    C.x[e] = make_double2(xr, xi);
}

cudaError_t chrono_combine(double2* x, const double2* const* v, const double2* c, int N, int Vh, cudaStream_t st) {
    if (N < 1 || N > CHRONO_MAX) return cudaErrorInvalidValue;
    CombineArgs C;
    for (int i = 0; i < CHRONO_MAX; ++i) C.v[i] = i < N ? v[i] : nullptr;
    C.c = c;
    C.x = x;
    C.N = N;
    C.ne = 12L * Vh;
    chrono_combine_kernel<<<grid_for(C.ne), NT, 0, st>>>(C);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lgt
