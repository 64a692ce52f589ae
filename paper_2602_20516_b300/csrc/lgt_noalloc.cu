// lgt_noalloc.cu -- mean plaquette of a canonical-layout gauge field without any
// device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// result: code running inside another framework's memory pool or under a strict
// memory budget, allocator-free embedded runtimes, and hooks that run between the
// launches of someone else's pipeline, where a cudaMalloc would synchronise the
// device or fail.  lgt_plaquette_noalloc serves them: it reads the caller's links,
// writes the caller's output, and keeps its per-block partial sums in a fixed,
// file-scope device array instead of a lattice handle's workspace.
//
// Limits and sharing: the array holds one partial sum per block of 128 sites for
// at most 65536 blocks, so volumes above 8,388,608 sites are rejected (LGT_EINVAL).
// Every GPU that loads this library holds the array (about 0.5 MiB) until the
// process exits.  All calls share it and it keeps the last call's contents; the
// completion counter is cleared at the start of every call.  Two calls whose
// kernels overlap on the GPU (different streams, or different host threads on the
// same device) race on the array and give wrong results: serialise them.
#include <mutex>

#include "../../include/lgt.h"
#include "lgt_internal.h"

namespace {

using namespace lgt;

constexpr int kMaxBlocks = 65536;
constexpr long kMaxSites = (long)kMaxBlocks * NT;
constexpr int kMaxDevices = 64;

// partial sums [0, kMaxBlocks), then the completion counter (as 64-bit word)
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 32];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Re tr U_munu(x) / 3 summed over mu < nu at site s of a canonical [V][4][3][3] field
__device__ double site_plaquettes(const double2* __restrict__ U, const int L[4], long s) {
    int x[4];
    long r = s;
    x[0] = (int)(r % L[0]); r /= L[0];
    x[1] = (int)(r % L[1]); r /= L[1];
    x[2] = (int)(r % L[2]);
    x[3] = (int)(r / L[2]);
    const long stride[4] = {1, (long)L[0], (long)L[0] * L[1], (long)L[0] * L[1] * L[2]};
    auto link = [&](long site, int mu) {
        dmat m;
        const double2* b = U + (site * 4 + mu) * 9;
        for (int k = 0; k < 9; ++k) {
            double2 v = __ldg(b + k);
            m.e[k / 3][k % 3] = {v.x, v.y};
        }
        return m;
    };
    auto step = [&](int mu) { return (x[mu] == L[mu] - 1) ? s - (long)(L[mu] - 1) * stride[mu] : s + stride[mu]; };
    double acc = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        dmat Umu = link(s, mu);
        long sm = step(mu);
        for (int nu = mu + 1; nu < 4; ++nu) {
            long sn = step(nu);
            dmat a = mul(Umu, link(sm, nu));
            dmat b = mul_nd(a, link(sn, mu));
            dmat c = mul_nd(b, link(s, nu));
            acc += retrace(c);
        }
    }
    return acc / 3.0;
}

__global__ void __launch_bounds__(NT) plaquette_noalloc_kernel(const double2* __restrict__ U, int L0, int L1, int L2,
                                                               int L3, double* scratch, double* out) {
    const int L[4] = {L0, L1, L2, L3};
    const long V = (long)L0 * L1 * L2 * L3;
    const long s = (long)blockIdx.x * NT + threadIdx.x;
    double v = (s < V) ? site_plaquettes(U, L, s) : 0.0;
    v = block_sum(v);
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch + kMaxBlocks);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = v;
        __threadfence();
        last = (atomicAdd(counter, 1ull) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += NT) acc += __ldcg(scratch + k);
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        out[0] = acc / (6.0 * (double)V);
        *counter = 0ull;
    }
}

}  // namespace

extern "C" int lgt_plaquette_noalloc(const double* links_canonical, const int dims[4], double* plaq_dev,
                                     void* stream) {
    if (!links_canonical || !dims || !plaq_dev) return lgt::set_error(LGT_EINVAL, "null argument");
    // the limit is checked after every factor, so the product never exceeds
    // kMaxSites * INT_MAX and cannot overflow
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2) return lgt::set_error(LGT_EINVAL, "every extent must be even and >= 2");
        V *= dims[m];
        if (V > kMaxSites)
            return lgt::set_error(LGT_EINVAL, "volume exceeds the 8388608-site limit of the static scratch array");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return lgt::set_error(LGT_ECUDA, "no usable current CUDA device");
    double* scratch;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return lgt::set_error(LGT_ECUDA, "cudaGetSymbolAddress of the static scratch array failed");
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the completion counter must start at zero
    if (cudaMemsetAsync(scratch + kMaxBlocks, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return lgt::set_error(LGT_ECUDA, "clearing the scratch counter failed");
    const int grid = (int)((V + NT - 1) / NT);
    plaquette_noalloc_kernel<<<grid, NT, 0, st>>>(reinterpret_cast<const double2*>(links_canonical), dims[0],
                                                  dims[1], dims[2], dims[3], scratch, plaq_dev);
    lgt::count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lgt::set_error(LGT_ECUDA, cudaGetErrorString(e));
    return LGT_OK;
}
