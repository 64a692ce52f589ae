// lgt_blas.cu -- CG vector kernels: norms and inner products with FP64
// accumulation and a deterministic two-level (block, then last-block) reduction,
// the search-direction update, precision conversions and axpby.
// A "field" of n sites is [n/Vh parities][components][Vh]; site t -> (t / Vh, t % Vh).
#include "lgt_internal.h"

namespace lgt {

static inline int grid_for(long n) { return (int)((n + NT - 1) / NT); }

cudaError_t blas_zero(void* f, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(f, 0, bytes, st); }

template <bool FP64>
__global__ void __launch_bounds__(NT) norm2_kernel(const void* a, int n, int Vh, RedArgs R, int slot) {
    const int t = blockIdx.x * NT + threadIdx.x;
    double acc = 0.0;
    if (t < n) {
        const int p = t / Vh, i = t - p * Vh;
        if (FP64) {
            const double2* b = (const double2*)a + (size_t)p * 12 * Vh + i;
#pragma unroll
            for (int k = 0; k < 12; ++k) { double2 v = __ldg(b + (size_t)k * Vh); acc += v.x * v.x + v.y * v.y; }
        } else {
            const float4* b = (const float4*)a + (size_t)p * 6 * Vh + i;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                float4 v = __ldg(b + (size_t)k * Vh);
                acc += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
            }
        }
    }
    double bs = block_sum(acc);
    grid_reduce(bs, R.partials, R.counter, R.s, RED_STORE, slot);
}

cudaError_t blas_norm2(const void* a, int n, int Vh, bool fp64, const RedArgs& R, int slot, cudaStream_t st) {
    if (grid_for(n) > R.capacity) return cudaErrorInvalidValue;   // partials too small
    if (fp64) norm2_kernel<true><<<grid_for(n), NT, 0, st>>>(a, n, Vh, R, slot);
    else norm2_kernel<false><<<grid_for(n), NT, 0, st>>>(a, n, Vh, R, slot);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) redot_kernel(const double2* a, const double2* b, int n, int Vh, RedArgs R,
                                                   int slot) {
    const int t = blockIdx.x * NT + threadIdx.x;
    double acc = 0.0;
    if (t < n) {
        const int p = t / Vh, i = t - p * Vh;
        const size_t o = (size_t)p * 12 * Vh + i;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 u = __ldg(a + o + (size_t)k * Vh), v = __ldg(b + o + (size_t)k * Vh);
            acc += u.x * v.x + u.y * v.y;
        }
    }
    double bs = block_sum(acc);
    grid_reduce(bs, R.partials, R.counter, R.s, RED_STORE, slot);
}

cudaError_t blas_redot(const double2* a, const double2* b, int n, int Vh, const RedArgs& R, int slot,
                       cudaStream_t st) {
    if (grid_for(n) > R.capacity) return cudaErrorInvalidValue;
    redot_kernel<<<grid_for(n), NT, 0, st>>>(a, b, n, Vh, R, slot);
    count_launch();
    return cudaGetLastError();
}

// x += alpha p, then p = r + beta p over the flat element array; the last block
// moves done 1 -> 2
__device__ __forceinline__ void axpy(double2& x, double2 p, double a) {
    x.x = fma(a, p.x, x.x);
    x.y = fma(a, p.y, x.y);
}
__device__ __forceinline__ void axpy(float4& x, float4 p, double ad) {
    const float a = (float)ad;
    x.x = fmaf(a, p.x, x.x);
    x.y = fmaf(a, p.y, x.y);
    x.z = fmaf(a, p.z, x.z);
    x.w = fmaf(a, p.w, x.w);
}
__device__ __forceinline__ void xpby(double2& p, double2 r, double b) {
    p.x = fma(b, p.x, r.x);
    p.y = fma(b, p.y, r.y);
}
__device__ __forceinline__ void xpby(float4& p, float4 r, double bd) {
    const float b = (float)bd;
    p.x = fmaf(b, p.x, r.x);
    p.y = fmaf(b, p.y, r.y);
    p.z = fmaf(b, p.z, r.z);
    p.w = fmaf(b, p.w, r.w);
}

template <typename T>
__device__ __forceinline__ void p_update_body(T* p, const T* r, T* x, long ne, const RedArgs& R, int blk,
                                              int nblk) {
    if (R.s->done >= 2) return;
    const long e = (long)blk * NT + threadIdx.x;
    if (e < ne) {
        T pv = p[e], xv = x[e];
        axpy(xv, pv, R.s->alpha);
        x[e] = xv;
        xpby(pv, __ldg(r + e), R.s->beta);
        p[e] = pv;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(R.counter, 1u);
        last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        *R.counter = 0u;
        if (R.s->done == 1) R.s->done = 2;
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) p_update_kernel(T* p, const T* r, T* x, long ne, RedArgs R) {
    p_update_body<T>(p, r, x, ne, R, blockIdx.x, gridDim.x);
}

// The same on one half field ([NC][Vh]) with a thread per site over its NC components,
// so that a block touches whole sites: block b works on site block nblk - 1 - b when
// reverse is set (the order of the sites only; the values are the same).
template <typename T, int NC>
__device__ __forceinline__ void p_update_sites_body(T* p, const T* r, T* x, int Vh, const RedArgs& R, int blk) {
    if (R.s->done >= 2) return;
    const int i = blk * NT + threadIdx.x;
    if (i < Vh) {
        const double a = R.s->alpha, b = R.s->beta;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const size_t e = (size_t)k * Vh + i;
            T pv = p[e], xv = x[e];
            axpy(xv, pv, a);
            x[e] = xv;
            xpby(pv, __ldg(r + e), b);
            p[e] = pv;
        }
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(R.counter, 1u);
        last = (prev == (unsigned)gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        *R.counter = 0u;
        if (R.s->done == 1) R.s->done = 2;
    }
}
template <typename T, int NC>
__global__ void __launch_bounds__(NT) p_update_sites_kernel(T* p, const T* r, T* x, int Vh, RedArgs R, int reverse) {
    p_update_sites_body<T, NC>(p, r, x, Vh, R, reverse ? gridDim.x - 1 - blockIdx.x : blockIdx.x);
}
// several systems (blockIdx.y), FP32 half fields
__global__ void __launch_bounds__(NT) p_update_sites_multi_kernel(PUpdateM P, int Vh) {
    const int k = blockIdx.y;
    if (k >= P.nrhs) return;
    p_update_sites_body<float4, 6>((float4*)P.p[k], (const float4*)P.r[k], (float4*)P.x[k], Vh, P.red[k], blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(NT) p_update_batch_kernel(const BatchAxpy* __restrict__ d, int n) {
    int lo = 0, hi = n - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d[mid].first <= b) lo = mid;
        else hi = mid - 1;
    }
    const BatchAxpy& e = d[lo];
    p_update_body<T>((T*)e.p, (const T*)e.r, (T*)e.x, e.ne, e.red, b - e.first, e.nblk);
}

cudaError_t launch_p_update_batch(const BatchAxpy* d, int n, int total_blocks, bool fp64, cudaStream_t st) {
    if (n <= 0 || total_blocks <= 0) return cudaSuccess;
    if (fp64) p_update_batch_kernel<double2><<<total_blocks, NT, 0, st>>>(d, n);
    else p_update_batch_kernel<float4><<<total_blocks, NT, 0, st>>>(d, n);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(NT) p_update_multi_kernel(PUpdateM P, long ne) {
    const int k = blockIdx.y;
    if (k >= P.nrhs) return;
    p_update_body<T>((T*)P.p[k], (const T*)P.r[k], (T*)P.x[k], ne, P.red[k], blockIdx.x, gridDim.x);
}
cudaError_t blas_cg_p_update_multi(const PUpdateM& P, int n, bool fp64, cudaStream_t st) {
    if (P.nrhs < 1 || P.nrhs > KMAX_RHS) return cudaErrorInvalidValue;
    if (!fp64) {   // one FP32 half field per system: site blocks
        p_update_sites_multi_kernel<<<dim3(grid_for(n), P.nrhs), NT, 0, st>>>(P, n);
        count_launch();
        return cudaGetLastError();
    }
    const long ne = (long)n * 12;
    const dim3 grid(grid_for(ne), P.nrhs);
    p_update_multi_kernel<double2><<<grid, NT, 0, st>>>(P, ne);
    count_launch();
    return cudaGetLastError();
}

cudaError_t blas_cg_p_update(void* p, const void* r, void* x, int n, int Vh, bool fp64, const RedArgs& R,
                             cudaStream_t st, bool reverse) {
    const int rev = reverse ? 1 : 0;
    if (n == Vh) {   // one half field: site blocks
        if (fp64)
            p_update_sites_kernel<double2, 12><<<grid_for(n), NT, 0, st>>>((double2*)p, (const double2*)r,
                                                                          (double2*)x, Vh, R, rev);
        else
            p_update_sites_kernel<float4, 6><<<grid_for(n), NT, 0, st>>>((float4*)p, (const float4*)r, (float4*)x,
                                                                        Vh, R, rev);
    } else if (fp64) {
        long ne = (long)n * 12;
        p_update_kernel<double2><<<grid_for(ne), NT, 0, st>>>((double2*)p, (const double2*)r, (double2*)x, ne, R);
    } else {
        long ne = (long)n * 6;
        p_update_kernel<float4><<<grid_for(ne), NT, 0, st>>>((float4*)p, (const float4*)r, (float4*)x, ne, R);
    }
    count_launch();
    return cudaGetLastError();
}

// FP64 [P][12][Vh] <-> FP32 [P][6][Vh]: float4 k of a site = double2 components 2k, 2k+1
__global__ void __launch_bounds__(NT) d2f_kernel(float4* y, const double2* x, int n, int Vh) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= (long)n * 6) return;
    const int site = (int)(e % n), k = (int)(e / n);
    const int p = site / Vh, i = site - p * Vh;
    const double2* b = x + (size_t)p * 12 * Vh + i;
    double2 u = b[(size_t)(2 * k) * Vh], v = b[(size_t)(2 * k + 1) * Vh];
    y[(size_t)p * 6 * Vh + (size_t)k * Vh + i] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
}

template <int MODE>  // 0: y = x, 1: y += x
__global__ void __launch_bounds__(NT) f2d_kernel(double2* y, const float4* x, int n, int Vh) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= (long)n * 6) return;
    const int site = (int)(e % n), k = (int)(e / n);
    const int p = site / Vh, i = site - p * Vh;
    float4 f = x[(size_t)p * 6 * Vh + (size_t)k * Vh + i];
    double2* b = y + (size_t)p * 12 * Vh + i;
    double2 u = make_double2(f.x, f.y), v = make_double2(f.z, f.w);
    if (MODE == 1) {
        double2 a = b[(size_t)(2 * k) * Vh], c = b[(size_t)(2 * k + 1) * Vh];
        u.x += a.x; u.y += a.y; v.x += c.x; v.y += c.y;
    }
    b[(size_t)(2 * k) * Vh] = u;
    b[(size_t)(2 * k + 1) * Vh] = v;
}

cudaError_t blas_d2f(float4* y, const double2* x, int n, int Vh, cudaStream_t st) {
    d2f_kernel<<<grid_for((long)n * 6), NT, 0, st>>>(y, x, n, Vh);
    count_launch();
    return cudaGetLastError();
}
cudaError_t blas_add_f2d(double2* y, const float4* x, int n, int Vh, cudaStream_t st) {
    f2d_kernel<1><<<grid_for((long)n * 6), NT, 0, st>>>(y, x, n, Vh);
    count_launch();
    return cudaGetLastError();
}
cudaError_t blas_f2d(double2* y, const float4* x, int n, int Vh, cudaStream_t st) {
    f2d_kernel<0><<<grid_for((long)n * 6), NT, 0, st>>>(y, x, n, Vh);
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) axpby_kernel(double2* y, const double2* x, double a, double b, long ne) {
    const long e = (long)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    double2 u = __ldg(x + e), v = y[e];
    v.x = fma(a, u.x, b * v.x);
    v.y = fma(a, u.y, b * v.y);
    y[e] = v;
}

cudaError_t blas_axpby(double2* y, const double2* x, double a, double b, int n, int Vh, cudaStream_t st) {
    (void)Vh;
    long ne = (long)n * 12;
    axpby_kernel<<<grid_for(ne), NT, 0, st>>>(y, x, a, b, ne);
    count_launch();
    return cudaGetLastError();
}

cudaError_t blas_action_parts(const double2* phi, const double2* chi, const double2* eta, int n, int Vh,
                              const RedArgs& R, cudaStream_t st) {
    cudaError_t e = blas_redot(phi, chi, n, Vh, R, 0, st);
    if (e != cudaSuccess) return e;
    return blas_norm2(eta, n, Vh, true, R, 1, st);
}

}  // namespace lgt
