// lgt_api.cu -- the C ABI of liblgt (include/lgt.h): lattice handles, the CG
// drivers (FP64, and mixed FP32-inner / FP64-reliable-update), actions, forces,
// molecular-dynamics updates and HMC trajectories.  All device work is in the
// kernels of the other translation units; this file only sequences launches on
// the handle's stream and reads back the few scalars the control flow needs.
#include <chrono>
#include <complex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unistd.h>
#include <vector>

#include "../../include/lgt.h"
#include "lgt_internal.h"

using namespace lgt;

// ---------------------------------------------------------------- errors
static thread_local std::string g_err = "";
static thread_local int64_t g_launches = 0;

// hop-kernel timing: event pairs recorded around each hop launch while enabled
struct KernelTiming {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    size_t used = 0;
    uint64_t seen = 0;   // hop launches since start
    int every = 1;       // record every `every`-th of them
};
static KernelTiming g_kt;

namespace lgt {
void count_launch() { ++g_launches; }
int set_error(int code, const char* msg) {
    g_err = msg;
    return code;
}
bool kernel_timing_slot(int kind, cudaEvent_t* a, cudaEvent_t* b) {
    if (!g_kt.on || g_kt.used + 2 > g_kt.ev.size() || g_kt.used / 2 >= g_kt.kind.size()) return false;
    if (g_kt.seen++ % g_kt.every != 0) return false;   // sampled: every `every`-th hop launch
    *a = g_kt.ev[g_kt.used];
    *b = g_kt.ev[g_kt.used + 1];
    g_kt.kind[g_kt.used / 2] = kind;
    g_kt.used += 2;
    return true;
}
}

// hop launch with optional CUDA-event timing; kind = 5 * fp64 + epilogue
static cudaError_t timed_hop(const HopArgs& A, bool fp64, bool dagger, int epi, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = kernel_timing_slot((fp64 ? 5 : 0) + epi, &e0, &e1);
    if (timed) cudaEventRecord(e0, st);
    cudaError_t e = launch_hop(A, fp64, dagger, epi, st);
    if (timed) cudaEventRecord(e1, st);
    return e;
}
// the double-float hop, timed as kind 10 + epilogue
static cudaError_t timed_hop_df(const HopArgs& A, bool dagger, int epi, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = kernel_timing_slot(10 + epi, &e0, &e1);
    if (timed) cudaEventRecord(e0, st);
    cudaError_t e = launch_hop_df(A, dagger, epi, st);
    if (timed) cudaEventRecord(e1, st);
    return e;
}

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(LGT_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                   \
    } while (0)
#define TRY(call)                        \
    do {                                 \
        int r_ = (call);                 \
        if (r_ != LGT_OK) return r_;     \
    } while (0)

// ---------------------------------------------------------------- host Philox (Metropolis draw)
static void philox_host(const uint32_t ctr[4], uint64_t seed, uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t a = (uint64_t)0xD2511F53u * c0, b = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0, n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        c0 = n0; c1 = (uint32_t)b; c2 = n2; c3 = (uint32_t)a;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ---------------------------------------------------------------- handle
constexpr int MAX_STOUT = LGT_MAX_STOUT;   // stout levels in front of D

struct Links {
    double2* U;
    float4* U12;
    // clover term 1 + A of these links (null: Wilson operator)
    const double2* C64 = nullptr;
    const float4* C32 = nullptr;
    // even-odd form: (1 + A)^{-1} on odd sites (layout of C64 / C32) and the sum over the
    // odd sites of ln det (1 + A)
    const double2* I64 = nullptr;
    const float4* I32 = nullptr;
    double logdet_odd = 0.0;
    // Hermitian-packed double-float copies of 1 + A (even sites) and of its inverse (odd
    // sites) for the mixed solver's double-float true residuals (null: FP64 residuals)
    const float4* Cdf = nullptr;
    const float4* Idf = nullptr;
};

struct lgt_lattice {
    int dims[4];
    Geom g;
    lgt_allocator alloc;
    bool custom_alloc;
    cudaStream_t st;
    std::vector<void*> blocks;
    size_t bytes;
    // gauge field
    Links thin;
    // solver workspace (full fields; even-odd solves use the even half)
    double2 *r, *p, *u, *t, *X, *Y, *b;
    // force vectors taken from the solver's final true residual: when cap_X / cap_Y
    // are set, the FP64 residual of a converged solve leaves X = (x_e, kappa H_oe x_e)
    // and Y = (Dhat x_e, kappa (H^+)_oe Dhat x_e) (full lattice: Y = D x) in them, and
    // cap_valid says so
    double2 *cap_X, *cap_Y;
    bool cap_valid;
    // the mixed even-odd Wilson solver forms its true residuals in double-float: the
    // same vectors are then left as double-float copies, x_e and X_o in Xdf, eta_e
    // and Y_o in Ydf, and cap_df_valid says so (cap_valid stays false until they are
    // converted to FP64 for a consumer that needs them there)
    bool cap_df_valid = false;
    // the FP64 links the double-float copy Udf was last built from, within one solve
    // or force evaluation (nullptr: rebuild)
    const double2* udf_src = nullptr;
    float4 *r32, *p32, *x32, *u32, *t32, *X32, *Y32;
    bool have_solver;
    // double-float copies for LGT_ARITH_DF64 forces: links, X, Y
    float4 *Udf, *Xdf, *Ydf;
    // clover term: fields of the thin links (lgt_set_clover) and of the links of a
    // force/action call (fermion_links), full spinor temporaries for (1 + A) y, and
    // the insertion field of the clover force
    double2 *thin_c64, *call_c64, *cins;
    float4* cins_df;   // double-float copy of the insertion field (double-float force arithmetic)
    float4 *call_cdf, *call_idf;   // packed double-float clover blocks (float4 [parity][36][Vh])
    float4 *thin_c32, *call_c32;
    // (1 + A)^{-1} on odd sites for the even-odd form, of the thin and of the call links
    double2 *thin_i64, *call_i64;
    float4 *thin_i32, *call_i32;
    double2* ct64;
    float4* ct32;
    // several right-hand sides (lgt_cg_solve_multi): per system FP32 even/odd half
    // fields, an FP64 residual, scalars, reduction partials and counter
    struct {
        float4 *x32[KMAX_RHS], *r32[KMAX_RHS], *p32[KMAX_RHS], *u32[KMAX_RHS], *t32[KMAX_RHS];
        double2* r64[KMAX_RHS];
        double* partials[KMAX_RHS];
        unsigned* counter;   // KMAX_RHS counters, 64 B apart
        Scalars* s;          // device [KMAX_RHS]
        Scalars* hs;         // pinned mirror
        bool ready;
    } mw;
    // chronological initial guesses: the last solutions (FP64 even halves) of the
    // operator with kappa ch.kappa, newest at hist[(head - 1) mod CHRONO_MAX]
    struct {
        double2* hist[CHRONO_MAX];
        int n, head;
        int last_iters;       // iterations of the last recorded solve
        double kappa;
        double2 *G, *g, *c;   // device: Gram matrix, projections, coefficients
        int* used;
        double2* partials;
        unsigned* counter;
        long cap;
    } ch;
    // alternate sweep order of the CG kernels (lgt_set_sweep_order) and the direction
    // of the last launch
    int alternate = 1;
    int sweep = 0;
    // staging of the FP32 hops' operands in shared memory (lgt_set_hop_staging)
    int stage = 0;
    // HMC / force workspace
    double2 *mom, *Ubak, *phi, *xi, *F, *G;
    // canonical links staged for lgt_save_checkpoint / lgt_load_checkpoint
    double2* ckpt = nullptr;
    bool have_md;
    // stout stack: a pool of FP64 link fields holding the smeared levels the adjoint
    // needs (placement by StoutPlan), the FP32 copy of the top level, gradient
    // ping-pong and the per-link G_C scratch of the adjoint
    double2* sbuf[MAX_STOUT];
    int n_sbuf;
    float4* stout_top12;
    double2* sgrad[3];
    // reductions
    double* partials;
    int n_partials;
    unsigned* counter;
    Scalars* s;
    Scalars* hs;   // pinned host mirror
};

static int lat_alloc(lgt_lattice* L, size_t bytes, void** out) {
    void* p = nullptr;
    if (L->custom_alloc) {
        p = L->alloc.alloc(L->alloc.ctx, bytes, (void*)L->st);
        if (!p) return fail(LGT_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return fail(LGT_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    L->blocks.push_back(p);
    L->bytes += bytes;
    *out = p;
    return LGT_OK;
}

template <typename T> static int A(lgt_lattice* L, size_t bytes, T** out) {
    void* p;
    int r = lat_alloc(L, bytes, &p);
    *out = (T*)p;
    return r;
}

static size_t spinor64_full(const lgt_lattice* L) { return (size_t)2 * 12 * L->g.Vh * sizeof(double2); }
static size_t spinor32_full(const lgt_lattice* L) { return (size_t)2 * 6 * L->g.Vh * sizeof(float4); }
static size_t links64(const lgt_lattice* L) { return (size_t)8 * 9 * L->g.Vh * sizeof(double2); }
static size_t links12(const lgt_lattice* L) { return (size_t)8 * 3 * L->g.Vh * sizeof(float4); }
static size_t mom_bytes(const lgt_lattice* L) { return (size_t)8 * 4 * L->g.Vh * sizeof(double2); }

static int ensure_solver(lgt_lattice* L) {
    if (L->have_solver) return LGT_OK;
    size_t s64 = spinor64_full(L), s32 = spinor32_full(L);
    TRY(A(L, s64, &L->r)); TRY(A(L, s64, &L->p)); TRY(A(L, s64, &L->u)); TRY(A(L, s64, &L->t));
    TRY(A(L, s64, &L->X)); TRY(A(L, s64, &L->Y)); TRY(A(L, s64, &L->b));
    TRY(A(L, s32, &L->r32)); TRY(A(L, s32, &L->p32)); TRY(A(L, s32, &L->x32)); TRY(A(L, s32, &L->u32));
    TRY(A(L, s32, &L->t32));
    TRY(A(L, s32, &L->X32)); TRY(A(L, s32, &L->Y32));
    L->have_solver = true;
    return LGT_OK;
}

static int ensure_df(lgt_lattice* L) {
    if (L->Udf) return LGT_OK;
    TRY(A(L, links64(L), &L->Udf));
    TRY(A(L, spinor64_full(L), &L->Xdf));
    TRY(A(L, spinor64_full(L), &L->Ydf));
    return LGT_OK;
}

static int ensure_multi(lgt_lattice* L) {
    if (L->mw.ready) return LGT_OK;
    const size_t h32 = (size_t)6 * L->g.Vh * sizeof(float4), h64 = (size_t)12 * L->g.Vh * sizeof(double2);
    for (int k = 0; k < KMAX_RHS; ++k) {
        TRY(A(L, h32, &L->mw.x32[k])); TRY(A(L, h32, &L->mw.r32[k])); TRY(A(L, h32, &L->mw.p32[k]));
        TRY(A(L, h32, &L->mw.u32[k])); TRY(A(L, h32, &L->mw.t32[k])); TRY(A(L, h64, &L->mw.r64[k]));
        TRY(A(L, sizeof(double) * (size_t)L->n_partials, &L->mw.partials[k]));
    }
    TRY(A(L, 64 * KMAX_RHS, &L->mw.counter));
    TRY(A(L, sizeof(Scalars) * KMAX_RHS, &L->mw.s));
    if (!L->mw.hs && cudaMallocHost((void**)&L->mw.hs, sizeof(Scalars) * KMAX_RHS) != cudaSuccess)
        return fail(LGT_ENOMEM, "cudaMallocHost failed");
    CK(cudaMemsetAsync(L->mw.counter, 0, 64 * KMAX_RHS, L->st));
    L->mw.ready = true;
    return LGT_OK;
}

static int ensure_clover(lgt_lattice* L, bool thin) {
    const size_t c64 = (size_t)2 * 72 * L->g.Vh * sizeof(double2), c32 = (size_t)2 * 18 * L->g.Vh * sizeof(float4);
    if (thin && !L->thin_c64) {
        TRY(A(L, c64, &L->thin_c64)); TRY(A(L, c32, &L->thin_c32));
        TRY(A(L, c64, &L->thin_i64)); TRY(A(L, c32, &L->thin_i32));
    }
    if (!thin && !L->call_c64) {
        TRY(A(L, c64, &L->call_c64));
        TRY(A(L, c32, &L->call_c32));
        TRY(A(L, c64, &L->call_i64)); TRY(A(L, c32, &L->call_i32));
        TRY(A(L, (size_t)2 * 54 * L->g.Vh * sizeof(double2), &L->cins));
        TRY(A(L, (size_t)2 * 54 * L->g.Vh * sizeof(float4), &L->cins_df));
    }
    if (!L->ct64) { TRY(A(L, spinor64_full(L), &L->ct64)); TRY(A(L, spinor32_full(L), &L->ct32)); }
    return LGT_OK;
}

// sigma_munu = (i/2)[g_mu, g_nu] in the chiral basis of the hop kernels
// (g_k = [[0, -i s_k], [i s_k, 0]] for mu = k - 1, g_4 = [[0, 1], [1, 0]]), as its two
// 2 x 2 chiral blocks; the off-diagonal blocks vanish because sigma commutes with g5
static CloverSigma clover_sigma() {
    typedef std::complex<double> C;
    const C I(0, 1);
    C pauli[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    C gam[4][4][4] = {};
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                gam[k][a][2 + b] = -I * pauli[k][a][b];
                gam[k][2 + a][b] = I * pauli[k][a][b];
            }
    for (int a = 0; a < 2; ++a) { gam[3][a][2 + a] = 1; gam[3][2 + a][a] = 1; }
    CloverSigma S;
    memset(&S, 0, sizeof S);
    const int pm[6] = {0, 0, 0, 1, 1, 2}, pn[6] = {1, 2, 3, 2, 3, 3};
    for (int pl = 0; pl < 6; ++pl)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                C acc = 0;
                for (int c = 0; c < 4; ++c)
                    acc += gam[pm[pl]][a][c] * gam[pn[pl]][c][b] - gam[pn[pl]][a][c] * gam[pm[pl]][c][b];
                acc *= 0.5 * I;
                if (a / 2 == b / 2) S.s[pl][a / 2][a % 2][b % 2] = make_double2(acc.real(), acc.imag());
            }
    return S;
}

static int ensure_chrono(lgt_lattice* L) {
    if (L->ch.G) return LGT_OK;
    const size_t h64 = (size_t)12 * L->g.Vh * sizeof(double2);
    for (int k = 0; k < CHRONO_MAX; ++k) TRY(A(L, h64, &L->ch.hist[k]));
    TRY(A(L, sizeof(double2) * CDOT_MAX, &L->ch.G));
    TRY(A(L, sizeof(double2) * CHRONO_MAX, &L->ch.g));
    TRY(A(L, sizeof(double2) * CHRONO_MAX, &L->ch.c));
    TRY(A(L, 64, &L->ch.used));
    L->ch.cap = (long)CDOT_MAX * ((L->g.Vh + NT - 1) / NT);
    TRY(A(L, sizeof(double2) * (size_t)L->ch.cap, &L->ch.partials));
    TRY(A(L, sizeof(unsigned) * CDOT_MAX, &L->ch.counter));
    CK(cudaMemsetAsync(L->ch.counter, 0, sizeof(unsigned) * CDOT_MAX, L->st));
    L->ch.n = L->ch.head = 0;
    return LGT_OK;
}

static int ensure_md(lgt_lattice* L) {
    if (L->have_md) return LGT_OK;
    TRY(A(L, mom_bytes(L), &L->mom));
    TRY(A(L, links64(L), &L->Ubak));
    TRY(A(L, spinor64_full(L), &L->phi));
    TRY(A(L, spinor64_full(L), &L->xi));
    TRY(A(L, mom_bytes(L), &L->F));
    TRY(A(L, links64(L), &L->G));
    L->have_md = true;
    return LGT_OK;
}

// Where the smeared levels live for n levels and mode m = stout_recompute:
//   m = 0  every level k in sbuf[k-1];
//   m = 1  only the top level (sbuf[0]) and one scratch field (sbuf[1]); the input
//          of each level is recomputed from the thin links in the adjoint (work
//          O(n^2) smearing steps, memory O(1));
//   m = c >= 2  checkpoints: levels c, 2c, ... below n in sbuf[0 .. nck), the top in
//          sbuf[nck], and c - 1 segment fields after it; the adjoint recomputes
//          each segment once from its checkpoint (about n extra smearing steps,
//          memory n/c + c levels).
// Every mode runs the same forward kernels on the same inputs, so the levels, and
// with them the gradients, are identical bit for bit.
struct StoutPlan {
    int n, m, c, nck;
    int buffers() const {
        if (m == 0) return n;
        if (m == 1) return n > 1 ? 2 : 1;
        return nck + 1 + std::min(c - 1, n - 1);
    }
    // field of level k (1..n) as written by the forward pass
    int slot(int k) const {
        if (m == 0) return k - 1;
        if (m == 1) return ((n - k) % 2 == 0) ? 0 : 1;
        if (k == n) return nck;
        if (k % c == 0) return k / c - 1;
        return nck + (k % c);
    }
};
static StoutPlan stout_plan(int n, int m) {
    StoutPlan P{n, m, m >= 2 ? m : 0, 0};
    if (m >= 2) P.nck = (n - 1) / m;
    return P;
}

static int ensure_stout(lgt_lattice* L, int n, int m) {
    if (n < 0 || n > MAX_STOUT) return fail(LGT_EINVAL, "n_stout = %d outside 0..%d", n, MAX_STOUT);
    if (m < 0) return fail(LGT_EINVAL, "stout_recompute = %d", m);
    if (n == 0) return LGT_OK;
    if (!L->stout_top12) TRY(A(L, links12(L), &L->stout_top12));
    if (!L->sgrad[0])
        for (int k = 0; k < 3; ++k) TRY(A(L, links64(L), &L->sgrad[k]));
    const int need = stout_plan(n, m).buffers();
    while (L->n_sbuf < need) TRY(A(L, links64(L), &L->sbuf[L->n_sbuf++]));
    return LGT_OK;
}

static RedArgs red(lgt_lattice* L) { return RedArgs{L->s, L->partials, L->counter, L->n_partials}; }



static int sync_scalars(lgt_lattice* L) {
    CK(cudaMemcpyAsync(L->hs, L->s, sizeof(Scalars), cudaMemcpyDeviceToHost, L->st));
    CK(cudaStreamSynchronize(L->st));
    return LGT_OK;
}
static int push_scalars(lgt_lattice* L) {
    CK(cudaMemcpyAsync(L->s, L->hs, sizeof(Scalars), cudaMemcpyHostToDevice, L->st));
    return LGT_OK;
}

// (1 + A)^{-1} on the odd sites of lk's clover term into I64 / I32, and the sum of
// ln det (1 + A) over them (synchronous: the sum is read back)
static int clover_inverse_odd(lgt_lattice* L, Links* lk, double2* I64, float4* I32) {
    CK(clover_invert(lk->C64, L->g, 1, I64, I32, red(L), 5, L->st));
    TRY(sync_scalars(L));
    if (!std::isfinite(L->hs->slot[5]))
        return fail(LGT_ENAN, "the clover term 1 + A is not positive definite on some odd site");
    lk->I64 = I64;
    lk->I32 = I32;
    lk->logdet_odd = L->hs->slot[5];
    return LGT_OK;
}

extern "C" const char* lgt_last_error(void) { return g_err.c_str(); }
extern "C" int lgt_version(void) { return 100; }
extern "C" int64_t lgt_launch_count(int reset) {
    int64_t v = g_launches;
    if (reset) g_launches = 0;
    return v;
}

extern "C" int lgt_create_lattice(const int dims[4], const lgt_allocator* alloc, void* stream, lgt_lattice_t* out) {
    if (!dims || !out) return fail(LGT_EINVAL, "null argument");
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2) return fail(LGT_EINVAL, "extent %d of direction %d must be even and >= 2", dims[m], m);
        V *= dims[m];
    }
    if (V > (1L << 30)) return fail(LGT_EINVAL, "volume %ld too large", V);
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(LGT_EINVAL, "allocator without alloc/free");
    lgt_lattice* L = new lgt_lattice();
    memcpy(L->dims, dims, sizeof L->dims);
    for (int m = 0; m < 4; ++m) L->g.L[m] = dims[m];
    L->g.V = (int)V;
    L->g.Vh = (int)(V / 2);
    L->g.stride[0] = 1;
    L->g.stride[1] = dims[0];
    L->g.stride[2] = dims[0] * dims[1];
    L->g.stride[3] = dims[0] * dims[1] * dims[2];
    L->custom_alloc = alloc != nullptr;
    if (alloc) L->alloc = *alloc;
    // one partial sum per block of the largest reducing grid: one thread per link (4V)
    L->n_partials = (int)((8L * L->g.Vh + NT - 1) / NT) + 64;
    L->st = (cudaStream_t)stream;
    int rc;
    if ((rc = A(L, links64(L), &L->thin.U)) || (rc = A(L, links12(L), &L->thin.U12)) ||
        (rc = A(L, sizeof(double) * (size_t)L->n_partials, &L->partials)) ||
        (rc = A(L, 64, &L->counter)) || (rc = A(L, sizeof(Scalars), &L->s))) {
        lgt_destroy_lattice(L);
        return rc;
    }
    if (cudaMallocHost((void**)&L->hs, sizeof(Scalars)) != cudaSuccess) {
        lgt_destroy_lattice(L);
        return fail(LGT_ENOMEM, "cudaMallocHost failed");
    }
    memset(L->hs, 0, sizeof(Scalars));
    cudaError_t e = cudaMemsetAsync(L->counter, 0, 64, L->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->s, 0, sizeof(Scalars), L->st);
    if (e == cudaSuccess) e = gauge_unit(L->thin.U, L->thin.U12, L->g, L->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->st);
    if (e != cudaSuccess) {
        lgt_destroy_lattice(L);
        return fail(LGT_ECUDA, "lattice initialisation: %s", cudaGetErrorString(e));
    }
    *out = L;
    return LGT_OK;
}

extern "C" int lgt_destroy_lattice(lgt_lattice_t L) {
    if (!L) return LGT_OK;
    cudaStreamSynchronize(L->st);
    for (void* p : L->blocks) {
        if (L->custom_alloc) L->alloc.free(L->alloc.ctx, p, (void*)L->st);
        else cudaFree(p);
    }
    if (L->hs) cudaFreeHost(L->hs);
    if (L->mw.hs) cudaFreeHost(L->mw.hs);
    delete L;
    return LGT_OK;
}

extern "C" int lgt_set_stream(lgt_lattice_t L, void* stream) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    L->st = (cudaStream_t)stream;
    return LGT_OK;
}

extern "C" int lgt_lattice_info(lgt_lattice_t L, int64_t* volume, size_t* bytes) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    if (volume) *volume = L->g.V;
    if (bytes) *bytes = L->bytes;
    return LGT_OK;
}

extern "C" int lgt_field_bytes(lgt_lattice_t L, int kind, int parity, int precision, size_t* bytes) {
    if (!L || !bytes) return fail(LGT_EINVAL, "null argument");
    if (kind == 0) {
        size_t half = (precision == LGT_FP32) ? (size_t)6 * L->g.Vh * 16 : (size_t)12 * L->g.Vh * 16;
        if (parity == LGT_FULL) half *= 2;
        *bytes = half;
    } else if (kind == 1) {
        *bytes = mom_bytes(L);
    } else if (kind == 2) {
        *bytes = links64(L);
    } else {
        return fail(LGT_EINVAL, "unknown field kind %d", kind);
    }
    return LGT_OK;
}

// ---------------------------------------------------------------- gauge field
extern "C" int lgt_set_links(lgt_lattice_t L, const double* canon) {
    if (!L || !canon) return fail(LGT_EINVAL, "null argument");
    CK(gauge_pack_links(L->thin.U, L->thin.U12, (const double2*)canon, L->g, L->st));
    L->udf_src = nullptr;
    return LGT_OK;
}
extern "C" int lgt_get_links(lgt_lattice_t L, double* canon) {
    if (!L || !canon) return fail(LGT_EINVAL, "null argument");
    CK(gauge_unpack_links(canon, L->thin.U, L->g, L->st));
    return LGT_OK;
}
// ---------------------------------------------------------------- checkpoint
// File: header of 7 little-endian 64-bit words (magic "LGTCKPT1"; version | flags << 32;
// dims[0] | dims[1] << 32; dims[2] | dims[3] << 32; seed; next trajectory; payload
// bytes), the canonical links (complex128 [V][4][3][3]), then the FNV-1a hash of the
// header and payload taken over 64-bit words (offset basis 0xcbf29ce484222325,
// prime 0x100000001b3).
namespace {
constexpr uint64_t kCkptMagic = 0x3154504b4354474cull;   // "LGTCKPT1" read little-endian
constexpr uint64_t kCkptVersion = 1;
uint64_t fnv1a_words(uint64_t h, const uint64_t* w, size_t n) {
    for (size_t k = 0; k < n; ++k) {
        h ^= w[k];
        h *= 0x100000001b3ull;
    }
    return h;
}
}  // namespace

static int ensure_ckpt(lgt_lattice* L) {
    if (!L->ckpt) TRY(A(L, links64(L), &L->ckpt));
    return LGT_OK;
}

extern "C" int lgt_save_checkpoint(lgt_lattice_t L, const char* path, uint64_t seed, uint64_t next_traj) {
    if (!L || !path) return fail(LGT_EINVAL, "null argument");
    TRY(ensure_ckpt(L));
    const size_t bytes = links64(L);
    std::vector<uint64_t> buf(7 + bytes / 8);
    uint64_t* h = buf.data();
    h[0] = kCkptMagic;
    h[1] = kCkptVersion;
    h[2] = (uint64_t)(uint32_t)L->dims[0] | ((uint64_t)(uint32_t)L->dims[1] << 32);
    h[3] = (uint64_t)(uint32_t)L->dims[2] | ((uint64_t)(uint32_t)L->dims[3] << 32);
    h[4] = seed;
    h[5] = next_traj;
    h[6] = bytes;
    CK(gauge_unpack_links((double*)L->ckpt, L->thin.U, L->g, L->st));
    CK(cudaMemcpyAsync(h + 7, L->ckpt, bytes, cudaMemcpyDeviceToHost, L->st));
    CK(cudaStreamSynchronize(L->st));
    const uint64_t sum = fnv1a_words(0xcbf29ce484222325ull, buf.data(), buf.size());
    // written beside the target and renamed over it once complete and flushed to disk,
    // so a crash or a full disk mid-write leaves the previous checkpoint intact
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(LGT_EINVAL, "cannot open %s for writing", tmp.c_str());
    bool ok = fwrite(buf.data(), 8, buf.size(), f) == buf.size() && fwrite(&sum, 8, 1, f) == 1;
    ok = fflush(f) == 0 && ok;
    ok = fsync(fileno(f)) == 0 && ok;
    if (fclose(f) != 0 || !ok) {
        remove(tmp.c_str());
        return fail(LGT_EINVAL, "writing %s failed", tmp.c_str());
    }
    if (rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(LGT_EINVAL, "renaming %s to %s failed", tmp.c_str(), path);
    }
    return LGT_OK;
}

extern "C" int lgt_load_checkpoint(lgt_lattice_t L, const char* path, uint64_t* seed, uint64_t* next_traj) {
    if (!L || !path) return fail(LGT_EINVAL, "null argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(LGT_EINVAL, "cannot open %s", path);
    const size_t bytes = links64(L);
    std::vector<uint64_t> buf(7 + bytes / 8);
    uint64_t sum = 0, extra = 0;
    const size_t got = fread(buf.data(), 8, buf.size(), f);
    const bool have_sum = fread(&sum, 8, 1, f) == 1;
    const bool at_end = fread(&extra, 1, 1, f) == 0;
    fclose(f);
    const uint64_t* h = buf.data();
    if (got < 7 || h[0] != kCkptMagic) return fail(LGT_EINVAL, "%s is not a checkpoint", path);
    if ((h[1] & 0xffffffffull) != kCkptVersion) return fail(LGT_EINVAL, "checkpoint version %llu", (unsigned long long)h[1]);
    const int d[4] = {(int)(uint32_t)h[2], (int)(uint32_t)(h[2] >> 32), (int)(uint32_t)h[3], (int)(uint32_t)(h[3] >> 32)};
    for (int m = 0; m < 4; ++m)
        if (d[m] != L->dims[m])
            return fail(LGT_EINVAL, "checkpoint lattice %dx%dx%dx%d differs from the handle's", d[0], d[1], d[2], d[3]);
    if (h[6] != bytes || got != buf.size() || !have_sum || !at_end)
        return fail(LGT_EINVAL, "checkpoint %s is truncated or too long", path);
    if (fnv1a_words(0xcbf29ce484222325ull, buf.data(), buf.size()) != sum)
        return fail(LGT_EINVAL, "checkpoint %s: checksum mismatch", path);
    TRY(ensure_ckpt(L));
    CK(cudaMemcpyAsync(L->ckpt, h + 7, bytes, cudaMemcpyHostToDevice, L->st));
    CK(gauge_pack_links(L->thin.U, L->thin.U12, L->ckpt, L->g, L->st));
    L->udf_src = nullptr;
    CK(cudaStreamSynchronize(L->st));
    if (seed) *seed = h[4];
    if (next_traj) *next_traj = h[5];
    return LGT_OK;
}

extern "C" int lgt_random_links(lgt_lattice_t L, uint64_t seed, double alpha) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    CK(gauge_random(L->thin.U, L->thin.U12, L->g, seed, alpha, L->st));
    L->udf_src = nullptr;
    return LGT_OK;
}
extern "C" int lgt_reunitarise(lgt_lattice_t L) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    L->udf_src = nullptr;
    CK(gauge_reunitarise(L->thin.U, L->thin.U12, L->g, L->st));
    return LGT_OK;
}
static int plaquette_sum(lgt_lattice* L, const double2* U, double* out) {
    CK(gauge_plaquette(U, L->g, red(L), 0, L->st));
    TRY(sync_scalars(L));
    *out = L->hs->slot[0];
    return LGT_OK;
}
static int rectangle_sum(lgt_lattice* L, const double2* U, double* out) {
    CK(gauge_rectangles(U, L->g, red(L), 0, L->st));
    TRY(sync_scalars(L));
    *out = L->hs->slot[0];
    return LGT_OK;
}
// S_G = beta [c0 (6V - sum Re tr P / 3) + c1 (12V - sum Re tr R / 3)], c0 = 1 - 8 c1
static int gauge_action_value(lgt_lattice* L, const lgt_action_params* ap, double* S) {
    double ps;
    TRY(plaquette_sum(L, L->thin.U, &ps));
    if (ap->c1 == 0.0) {
        *S = ap->beta * (6.0 * L->g.V - ps);
        return LGT_OK;
    }
    double rs;
    TRY(rectangle_sum(L, L->thin.U, &rs));
    *S = ap->beta * ((1.0 - 8.0 * ap->c1) * (6.0 * L->g.V - ps) + ap->c1 * (12.0 * L->g.V - rs));
    return LGT_OK;
}
extern "C" int lgt_rectangle(lgt_lattice_t L, double* rect) {
    if (!L || !rect) return fail(LGT_EINVAL, "null argument");
    double s;
    TRY(rectangle_sum(L, L->thin.U, &s));
    *rect = s / (12.0 * L->g.V);
    return LGT_OK;
}

extern "C" int lgt_plaquette(lgt_lattice_t L, double* plaq) {
    if (!L || !plaq) return fail(LGT_EINVAL, "null argument");
    double s;
    TRY(plaquette_sum(L, L->thin.U, &s));
    *plaq = s / (6.0 * L->g.V);
    return LGT_OK;
}

// ---------------------------------------------------------------- layouts
static int check_parity(int parity) {
    if (parity < 0 || parity > 2) return fail(LGT_EINVAL, "parity %d", parity);
    return LGT_OK;
}
static int check_precision(int precision) {
    if (precision != LGT_FP64 && precision != LGT_FP32 && precision != LGT_DF64)
        return fail(LGT_EINVAL, "precision %d", precision);
    return LGT_OK;
}
// complex entries of a spinor field of parity selector `parity`
static long spinor_entries(const lgt_lattice* L, int parity) { return (parity == LGT_FULL ? 24L : 12L) * L->g.Vh; }
extern "C" int lgt_pack_spinor(lgt_lattice_t L, const double* canon, void* field, int parity, int precision) {
    if (!L || !canon || !field) return fail(LGT_EINVAL, "null argument");
    TRY(check_parity(parity));
    TRY(check_precision(precision));
    CK(spinor_pack(field, (const double2*)canon, L->g, parity, precision != LGT_FP32, L->st));
    // double-float: the FP64 layout converted in place (each entry is read, then
    // rewritten as its pair, by the same thread)
    if (precision == LGT_DF64)
        CK(complex_to_df((float4*)field, (const double2*)field, spinor_entries(L, parity), L->st));
    return LGT_OK;
}
extern "C" int lgt_unpack_spinor(lgt_lattice_t L, const void* field, double* canon, int parity, int precision) {
    if (!L || !canon || !field) return fail(LGT_EINVAL, "null argument");
    TRY(check_parity(parity));
    TRY(check_precision(precision));
    if (precision == LGT_DF64) {   // through the FP64 layout in a workspace field
        TRY(ensure_solver(L));
        CK(complex_from_df(L->u, (const float4*)field, spinor_entries(L, parity), L->st));
        field = L->u;
    }
    CK(spinor_unpack((double2*)canon, field, L->g, parity, precision != LGT_FP32, L->st));
    return LGT_OK;
}
extern "C" int lgt_pack_momenta(lgt_lattice_t L, const double* canon, double* mom) {
    if (!L || !canon || !mom) return fail(LGT_EINVAL, "null argument");
    CK(mom_pack((double2*)mom, canon, L->g, L->st));
    return LGT_OK;
}
extern "C" int lgt_unpack_momenta(lgt_lattice_t L, const double* mom, double* canon) {
    if (!L || !canon || !mom) return fail(LGT_EINVAL, "null argument");
    CK(mom_unpack(canon, (const double2*)mom, L->g, L->st));
    return LGT_OK;
}
extern "C" int lgt_pack_links_field(lgt_lattice_t L, const double* canon, double* field) {
    if (!L || !canon || !field) return fail(LGT_EINVAL, "null argument");
    CK(gauge_pack_field((double2*)field, (const double2*)canon, L->g, L->st));
    return LGT_OK;
}
extern "C" int lgt_unpack_links_field(lgt_lattice_t L, const double* field, double* canon) {
    if (!L || !canon || !field) return fail(LGT_EINVAL, "null argument");
    CK(gauge_unpack_field(canon, (const double2*)field, L->g, L->st));
    return LGT_OK;
}

// ---------------------------------------------------------------- operators
static HopArgs hop_base(lgt_lattice* L, const Links& lk, bool fp64) {
    HopArgs a;
    memset(&a, 0, sizeof a);
    a.U = fp64 ? (const void*)lk.U : (const void*)lk.U12;
    a.g = L->g;
    a.s = L->s;
    a.partials = L->partials;
    a.red_capacity = L->n_partials;
    a.counter = L->counter;
    a.a = 1.0;
    a.stage = fp64 ? 0 : L->stage;
    return a;
}
static size_t half_elems(const lgt_lattice* L, bool fp64) { return (size_t)(fp64 ? 12 : 6) * L->g.Vh; }
// pointer to the half field of parity q inside a full field
static const void* half(const void* f, const lgt_lattice* L, bool fp64, int q) {
    return (const char*)f + (size_t)q * half_elems(L, fp64) * 16;
}
static void* half(void* f, const lgt_lattice* L, bool fp64, int q) {
    return (char*)f + (size_t)q * half_elems(L, fp64) * 16;
}

// single-parity hop: out_q = a H_{q,1-q} in (+ y)
static int hop1(lgt_lattice* L, const Links& lk, bool fp64, bool dag, int q, const void* in_half, void* out_half,
                double a, int epi = EPI_HOP, const void* y_half = nullptr) {
    HopArgs A = hop_base(L, lk, fp64);
    A.parity = q;
    A.in[1 - q] = in_half;
    A.out[q] = out_half;
    A.y[q] = y_half;
    A.a = a;
    CK(timed_hop(A, fp64, dag, epi, L->st));
    return LGT_OK;
}
// (1 + A) in into the clover temporary of the precision (full fields), or in itself
static const void* clover_y(lgt_lattice* L, const Links& lk, bool fp64, const void* in) {
    if (!lk.C64) return in;
    void* t = fp64 ? (void*)L->ct64 : (void*)L->ct32;
    if (clover_apply(fp64 ? (const void*)lk.C64 : (const void*)lk.C32, in, t, L->g, 2, fp64, L->st) != cudaSuccess)
        return nullptr;
    return t;
}

// full-lattice D or D^+: out = (1 + A) in - kappa H in (A = 0 without clover term)
static int dfull(lgt_lattice* L, const Links& lk, bool fp64, bool dag, const void* in, void* out, double kappa) {
    const void* yin = clover_y(L, lk, fp64, in);
    if (!yin) return fail(LGT_ECUDA, "clover apply failed");
    HopArgs A = hop_base(L, lk, fp64);
    A.parity = 2;
    for (int q = 0; q < 2; ++q) {
        A.in[q] = half(in, L, fp64, q);
        A.out[q] = half(out, L, fp64, q);
        A.y[q] = half(yin, L, fp64, q);
    }
    A.a = -kappa;
    CK(timed_hop(A, fp64, dag, EPI_XPAY, L->st));
    return LGT_OK;
}
// Dhat^(+) on even half fields: out = in - kappa^2 H_eo H_oe in, tmp an odd half field
static int dhat(lgt_lattice* L, const Links& lk, bool fp64, bool dag, const void* in, void* out, void* tmp,
                double kappa) {
    if (lk.C64) {
        // with the clover term: Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe, M = 1 + A Hermitian
        // (tmp: odd intermediate; the clover temporaries hold M_oo^{-1} tmp and M_ee in)
        if (!lk.I64) return fail(LGT_EINVAL, "the even-odd clover operator needs (1 + A)^{-1} on odd sites");
        void* ct = fp64 ? (void*)L->ct64 : (void*)L->ct32;
        void* t2 = half(ct, L, fp64, 1);
        void* y = half(ct, L, fp64, 0);
        TRY(hop1(L, lk, fp64, dag, 1, in, tmp, 1.0));
        CK(clover_apply(fp64 ? (const void*)lk.I64 : (const void*)lk.I32, tmp, t2, L->g, 1, fp64, L->st));
        CK(clover_apply(fp64 ? (const void*)lk.C64 : (const void*)lk.C32, in, y, L->g, 0, fp64, L->st));
        TRY(hop1(L, lk, fp64, dag, 0, t2, out, -kappa * kappa, EPI_XPAY, y));
        return LGT_OK;
    }
    TRY(hop1(L, lk, fp64, dag, 1, in, tmp, 1.0));
    TRY(hop1(L, lk, fp64, dag, 0, tmp, out, -kappa * kappa, EPI_XPAY, in));
    return LGT_OK;
}

extern "C" int lgt_set_clover(lgt_lattice_t L, double csw, double kappa) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    if (csw == 0.0) {
        L->thin.C64 = nullptr;
        L->thin.C32 = nullptr;
        L->thin.I64 = nullptr;
        L->thin.I32 = nullptr;
        L->thin.logdet_odd = 0.0;
        return LGT_OK;
    }
    TRY(ensure_clover(L, true));
    CK(clover_field(L->thin.U, L->g, clover_sigma(), kappa, csw, L->thin_c64, L->thin_c32, L->st));
    L->thin.C64 = L->thin_c64;
    L->thin.C32 = L->thin_c32;
    // the even-odd operators need (1 + A)^{-1} on the odd sites
    const int rc = clover_inverse_odd(L, &L->thin, L->thin_i64, L->thin_i32);
    if (rc != LGT_OK) {
        L->thin.C64 = nullptr;
        L->thin.C32 = nullptr;
        L->thin.I64 = nullptr;
        L->thin.I32 = nullptr;
        return rc;
    }
    return LGT_OK;
}

extern "C" int lgt_set_sweep_order(lgt_lattice_t L, int alternate) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    L->alternate = alternate != 0;
    return LGT_OK;
}

extern "C" int lgt_set_hop_staging(lgt_lattice_t L, int mode) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    if (mode < 0 || mode > 3) return fail(LGT_EINVAL, "staging mode %d (0..3)", mode);
    L->stage = mode;
    return LGT_OK;
}

extern "C" int lgt_hop_staging_status(lgt_lattice_t L, int* applies, unsigned* timeouts) {
    if (!L || !applies || !timeouts) return fail(LGT_EINVAL, "null argument");
    *applies = hop_stage_hr(L->g) > 0;
    *timeouts = hop_stage_timeouts();
    return *timeouts == ~0u ? fail(LGT_ECUDA, "reading the staging counter failed") : LGT_OK;
}

extern "C" int lgt_dslash(lgt_lattice_t L, const void* in, void* out, int op, int out_parity, int dagger,
                          double kappa, int precision) {
    if (!L || !in || !out) return fail(LGT_EINVAL, "null argument");
    if (in == out) return fail(LGT_EINVAL, "in and out must be distinct buffers");
    const bool dag = dagger != 0;
    if (precision == LGT_DF64) {
        if (op != LGT_OP_HOP) return fail(LGT_EINVAL, "LGT_DF64 applies LGT_OP_HOP only");
        if (out_parity != LGT_EVEN && out_parity != LGT_ODD) return fail(LGT_EINVAL, "hop needs EVEN or ODD");
        TRY(ensure_df(L));
        CK(links_to_df(L->Udf, L->thin.U, L->g, L->st));
        L->udf_src = L->thin.U;
        HopArgs A;
        memset(&A, 0, sizeof A);
        A.U = L->Udf;
        A.g = L->g;
        A.parity = out_parity;
        A.in[1 - out_parity] = in;
        A.out[out_parity] = out;
        A.a = 1.0;
        CK(timed_hop_df(A, dag, EPI_HOP, L->st));
        return LGT_OK;
    }
    if (precision != LGT_FP64 && precision != LGT_FP32) return fail(LGT_EINVAL, "precision %d", precision);
    const bool fp64 = precision == LGT_FP64;
    switch (op) {
    case LGT_OP_HOP:
        if (out_parity != LGT_EVEN && out_parity != LGT_ODD) return fail(LGT_EINVAL, "hop needs EVEN or ODD");
        return hop1(L, L->thin, fp64, dag, out_parity, in, out, 1.0);
    case LGT_OP_D:
        return dfull(L, L->thin, fp64, dag, in, out, kappa);
    case LGT_OP_DHAT:
    case LGT_OP_DHAT_NORMAL: {
        TRY(ensure_solver(L));
        void* tmp = fp64 ? (void*)L->t : (void*)L->t32;
        if (op == LGT_OP_DHAT) return dhat(L, L->thin, fp64, dag, in, out, tmp, kappa);
        void* mid = fp64 ? (void*)L->u : (void*)L->u32;
        TRY(dhat(L, L->thin, fp64, false, in, mid, tmp, kappa));
        return dhat(L, L->thin, fp64, true, mid, out, tmp, kappa);
    }
    default:
        return fail(LGT_EINVAL, "unknown operator %d", op);
    }
}

// ---------------------------------------------------------------- CG
// One CG iteration on A = M^+M, enqueued without host synchronisation.  Kernels
// return at once after the stop flag is raised on the device.
static int cg_iteration(lgt_lattice* L, const Links& lk, bool fp64, bool eo, double kappa, void* x, void* r, void* p,
                        void* u, void* t) {
    if (eo && lk.C64 && !fp64) {
        // FP32 even-odd clover (Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe) with the
        // site-local blocks fused into the hops: the odd hops store M_oo^{-1} H_oe in,
        // the even hops form M_ee y in their epilogue; the kernel sequence, deferred
        // <p, A p> reduction and sweep order of the Wilson iteration below
        auto dir = [&]() { return L->alternate ? (L->sweep ^= 1) : 0; };
        HopArgs A = hop_base(L, lk, false);
        A.skip = 1;
        A.parity = 1; A.in[0] = p; A.out[1] = t; A.clov = lk.I32; A.reverse = dir();
        CK(timed_hop(A, false, false, EPI_HOP, L->st));
        A = hop_base(L, lk, false);
        A.skip = 1;
        A.parity = 0; A.in[1] = t; A.out[0] = u; A.y[0] = p; A.clov = lk.C32; A.a = -kappa * kappa;
        A.red_op = RED_PAP; A.reverse = dir(); A.defer = 1;
        CK(timed_hop(A, false, false, EPI_XPAY_NORM, L->st));
        A = hop_base(L, lk, false);
        A.skip = 1;
        A.parity = 1; A.in[0] = u; A.out[1] = t; A.clov = lk.I32; A.reverse = dir();
        A.fin_n = hop_grid(L->g, 0); A.fin_op = RED_PAP;
        CK(timed_hop(A, false, true, EPI_HOP, L->st));
        A = hop_base(L, lk, false);
        A.skip = 1;
        A.parity = 0; A.in[1] = t; A.y[0] = u; A.clov = lk.C32; A.a = -kappa * kappa; A.red_op = RED_RR;
        A.r[0] = r; A.reverse = dir();
        CK(timed_hop(A, false, true, EPI_CG, L->st));
        CK(blas_cg_p_update(p, r, x, L->g.Vh, L->g.Vh, false, red(L), L->st, dir() != 0));
        return LGT_OK;
    }
    if (eo && lk.C64) {
        // with the clover term (Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe): the odd
        // intermediate goes through M_oo^{-1}, and M_ee p / M_ee u enter the xpay hops
        void* ct = fp64 ? (void*)L->ct64 : (void*)L->ct32;
        void* t2 = half(ct, L, fp64, 1);
        void* y = half(ct, L, fp64, 0);
        const void* Iv = fp64 ? (const void*)lk.I64 : (const void*)lk.I32;
        const void* Cv = fp64 ? (const void*)lk.C64 : (const void*)lk.C32;
        HopArgs A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 1; A.in[0] = p; A.out[1] = t;
        CK(timed_hop(A, fp64, false, EPI_HOP, L->st));
        CK(clover_apply(Iv, t, t2, L->g, 1, fp64, L->st));
        CK(clover_apply(Cv, p, y, L->g, 0, fp64, L->st));
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 0; A.in[1] = t2; A.out[0] = u; A.y[0] = y; A.a = -kappa * kappa; A.red_op = RED_PAP;
        CK(timed_hop(A, fp64, false, EPI_XPAY_NORM, L->st));
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 1; A.in[0] = u; A.out[1] = t;
        CK(timed_hop(A, fp64, true, EPI_HOP, L->st));
        CK(clover_apply(Iv, t, t2, L->g, 1, fp64, L->st));
        CK(clover_apply(Cv, u, y, L->g, 0, fp64, L->st));
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 0; A.in[1] = t2; A.y[0] = y; A.a = -kappa * kappa; A.red_op = RED_RR;
        A.r[0] = r;
        CK(timed_hop(A, fp64, true, EPI_CG, L->st));
        CK(blas_cg_p_update(p, r, x, L->g.Vh, L->g.Vh, fp64, red(L), L->st));
        return LGT_OK;
    }
    if (eo) {
        // with alternate order on, every launch walks the sites in the direction opposite
        // to the one before, so it starts on the sites whose data the previous launch
        // left in L2
        auto dir = [&]() { return L->alternate ? (L->sweep ^= 1) : 0; };
        HopArgs A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 1; A.in[0] = p; A.out[1] = t; A.reverse = dir();
        CK(timed_hop(A, fp64, false, EPI_HOP, L->st));
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 0; A.in[1] = t; A.out[0] = u; A.y[0] = p; A.a = -kappa * kappa; A.red_op = RED_PAP;
        A.reverse = dir(); A.defer = 1;
        CK(timed_hop(A, fp64, false, EPI_XPAY_NORM, L->st));
        // the hop of Dhat^+ does not need alpha: its block 0 finishes <p, A p> -> alpha
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 1; A.in[0] = u; A.out[1] = t; A.reverse = dir();
        A.fin_n = hop_grid(L->g, 0); A.fin_op = RED_PAP;
        CK(timed_hop(A, fp64, true, EPI_HOP, L->st));
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 0; A.in[1] = t; A.y[0] = u; A.a = -kappa * kappa; A.red_op = RED_RR;
        A.r[0] = r; A.reverse = dir();
        CK(timed_hop(A, fp64, true, EPI_CG, L->st));
        CK(blas_cg_p_update(p, r, x, L->g.Vh, L->g.Vh, fp64, red(L), L->st, dir() != 0));
    } else {
        const void* yp = clover_y(L, lk, fp64, p);
        if (!yp) return fail(LGT_ECUDA, "clover apply failed");
        HopArgs A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 2;
        for (int q = 0; q < 2; ++q) {
            A.in[q] = half(p, L, fp64, q); A.out[q] = half(u, L, fp64, q); A.y[q] = half(yp, L, fp64, q);
        }
        A.a = -kappa; A.red_op = RED_PAP;
        CK(timed_hop(A, fp64, false, EPI_XPAY_NORM, L->st));
        const void* yu = clover_y(L, lk, fp64, u);
        if (!yu) return fail(LGT_ECUDA, "clover apply failed");
        A = hop_base(L, lk, fp64);
        A.skip = 1;
        A.parity = 2;
        for (int q = 0; q < 2; ++q) {
            A.in[q] = half(u, L, fp64, q); A.y[q] = half(yu, L, fp64, q);
            A.r[q] = half(r, L, fp64, q);
        }
        A.a = -kappa; A.red_op = RED_RR;
        CK(timed_hop(A, fp64, true, EPI_CG, L->st));
        CK(blas_cg_p_update(p, r, x, 2 * L->g.Vh, L->g.Vh, fp64, red(L), L->st));
    }
    return LGT_OK;
}

// FP64 true residual res = b - A x, |res|^2 -> slot 0.  With L->cap_X / cap_Y set
// (x is then the even half of cap_X), the intermediate vectors of A x are written
// where the fermion force reads them:
//   even-odd: X_o = kappa H_oe x, eta = x - kappa H_eo X_o (= Dhat x), Y_o = kappa (H^+)_oe eta,
//             A x = eta - kappa (H^+)_eo Y_o;
//   full:     Y = D x, A x = D^+ Y.
// The force vectors of the even-odd clover operator from x_e (FP64):
//   X_o = kappa M_oo^{-1} H_oe x_e,  Y_e = M_ee x_e - kappa H_eo X_o (= Dhat x_e),
//   Y_o = kappa M_oo^{-1} (H^+)_oe Y_e;
// the odd half of the FP64 clover temporary is the scratch field (Xo and Yo may alias).
static int eo_clover_xy(lgt_lattice* L, const Links& lk, double kappa, const double2* x, double2* Xo, double2* Ye,
                        double2* Yo) {
    double2* cto = (double2*)half(L->ct64, L, true, 1);
    double2* cte = L->ct64;
    TRY(hop1(L, lk, true, false, 1, x, cto, kappa));
    CK(clover_apply(lk.I64, cto, Xo, L->g, 1, true, L->st));
    CK(clover_apply(lk.C64, x, cte, L->g, 0, true, L->st));
    TRY(hop1(L, lk, true, false, 0, Xo, Ye, -kappa, EPI_XPAY, cte));
    TRY(hop1(L, lk, true, true, 1, Ye, cto, kappa));
    CK(clover_apply(lk.I64, cto, Yo, L->g, 1, true, L->st));
    return LGT_OK;
}

static int true_residual(lgt_lattice* L, const Links& lk, bool eo, double kappa, const double2* b, const double2* x,
                         double2* res) {
    const bool cap = L->cap_X && L->cap_Y;
    if (eo && lk.C64) {
        // A x = Dhat^+ Y_e = M_ee Y_e - kappa (H^+)_eo Y_o
        double2* Xo = cap ? (double2*)half(L->cap_X, L, true, 1) : L->t;
        double2* Ye = cap ? L->cap_Y : L->u;
        double2* Yo = cap ? (double2*)half(L->cap_Y, L, true, 1) : L->t;
        TRY(eo_clover_xy(L, lk, kappa, x, Xo, Ye, Yo));
        CK(clover_apply(lk.C64, Ye, L->ct64, L->g, 0, true, L->st));
        HopArgs A = hop_base(L, lk, true);
        A.parity = 0; A.in[1] = Yo; A.y[0] = L->ct64; A.a = -kappa; A.out[0] = res; A.pv[0] = b;
        A.red_op = RED_STORE; A.red_slot = 0;
        CK(timed_hop(A, true, true, EPI_RESID, L->st));
    } else if (eo) {
        double2* Xo = cap ? (double2*)half(L->cap_X, L, true, 1) : L->t;
        double2* Ye = cap ? L->cap_Y : L->u;
        double2* Yo = cap ? (double2*)half(L->cap_Y, L, true, 1) : L->t;
        TRY(hop1(L, lk, true, false, 1, x, Xo, kappa));
        TRY(hop1(L, lk, true, false, 0, Xo, Ye, -kappa, EPI_XPAY, x));
        TRY(hop1(L, lk, true, true, 1, Ye, Yo, kappa));
        HopArgs A = hop_base(L, lk, true);
        A.parity = 0; A.in[1] = Yo; A.y[0] = Ye; A.a = -kappa; A.out[0] = res; A.pv[0] = b;
        A.red_op = RED_STORE; A.red_slot = 0;
        CK(timed_hop(A, true, true, EPI_RESID, L->st));
    } else {
        double2* Yf = cap ? L->cap_Y : L->u;
        TRY(dfull(L, lk, true, false, x, Yf, kappa));
        const void* yY = clover_y(L, lk, true, Yf);
        if (!yY) return fail(LGT_ECUDA, "clover apply failed");
        HopArgs A = hop_base(L, lk, true);
        A.parity = 2;
        for (int q = 0; q < 2; ++q) {
            A.in[q] = half(Yf, L, true, q); A.y[q] = half(yY, L, true, q);
            A.out[q] = half(res, L, true, q); A.pv[q] = half(b, L, true, q);
        }
        A.a = -kappa; A.red_op = RED_STORE; A.red_slot = 0;
        CK(timed_hop(A, true, true, EPI_RESID, L->st));
    }
    return LGT_OK;
}

// The even-odd Wilson true residual res = b - A x (A = Dhat^+ Dhat) with the four hops
// in double-float arithmetic on the double-float links Udf (built from lk.U); x, b and
// res are FP64, |res|^2 -> slot 0.  The intermediate vectors stay in double-float:
// x_e and X_o = kappa H_oe x_e in Xdf, eta_e = x_e - kappa H_eo X_o (= Dhat x_e) and
// Y_o = kappa (H^+)_oe eta_e in Ydf -- the force vectors X, Y of the solution.
static int true_residual_df(lgt_lattice* L, const Links& lk, double kappa, const double2* b, const double2* x,
                            double2* res) {
    if (L->udf_src != lk.U) {
        CK(links_to_df(L->Udf, lk.U, L->g, L->st));
        L->udf_src = lk.U;
    }
    const long hf = 12L * L->g.Vh;
    float4* xe = L->Xdf;
    float4* Xo = L->Xdf + hf;
    float4* Ye = L->Ydf;
    float4* Yo = L->Ydf + hf;
    CK(complex_to_df(xe, x, hf, L->st));
    // with the clover term: X_o = kappa M_oo^{-1} H_oe x_e, eta_e = M_ee x_e - kappa H_eo X_o,
    // Y_o = kappa M_oo^{-1} (H^+)_oe eta_e, A x = M_ee eta_e - kappa (H^+)_eo Y_o (the
    // blocks applied inside the hops)
    HopArgs A;
    memset(&A, 0, sizeof A);
    A.U = L->Udf;
    A.g = L->g;
    A.parity = 1; A.in[0] = xe; A.out[1] = Xo; A.a = kappa; A.clov = lk.Idf;
    CK(timed_hop_df(A, false, EPI_HOP, L->st));
    A.parity = 0; A.in[1] = Xo; A.out[0] = Ye; A.y[0] = xe; A.a = -kappa; A.clov = lk.Cdf;
    CK(timed_hop_df(A, false, EPI_XPAY, L->st));
    A.parity = 1; A.in[0] = Ye; A.out[1] = Yo; A.y[1] = nullptr; A.a = kappa; A.clov = lk.Idf;
    CK(timed_hop_df(A, true, EPI_HOP, L->st));
    HopArgs R = hop_base(L, lk, true);
    R.U = L->Udf;
    R.parity = 0; R.in[1] = Yo; R.y[0] = Ye; R.a = -kappa; R.out[0] = res; R.pv[0] = b; R.clov = lk.Cdf;
    R.red_op = RED_STORE; R.red_slot = 0;
    CK(timed_hop_df(R, true, EPI_RESID, L->st));
    return LGT_OK;
}

// The captured force vectors in FP64 (X_o, eta_e, Y_o converted from their
// double-float copies; X_e is the FP64 solution itself) for consumers of FP64 X, Y.
static int cap_to_fp64(lgt_lattice* L) {
    if (L->cap_valid || !L->cap_df_valid) return LGT_OK;
    const long hf = 12L * L->g.Vh;
    CK(complex_from_df((double2*)half(L->X, L, true, 1), L->Xdf + hf, hf, L->st));
    CK(complex_from_df(L->Y, L->Ydf, 2 * hf, L->st));
    L->cap_valid = true;
    return LGT_OK;
}

// Chronological initial guess for Dhat^+Dhat x = b on even sites (kappa): with the
// last N kept solutions v_i, x = sum c_i v_i with (V^+ A V) c = V^+ b.  The products
// A v_i use the FP32 operator on all of them at once (a guess needs no more).  The
// guess's residual is formed in FP64 by the solver: from the FP32 products it would be
// wrong by ~eps32 cond(A) |b|, as large as the residual of a good guess.
// *used = false (x untouched) when nothing of this operator is kept.
static int chrono_guess(lgt_lattice* L, const Links& lk, const double2* b, double2* x, double kappa, int want,
                        bool* used) {
    *used = false;
    auto& C = L->ch;
    if (C.n == 0 || C.kappa != kappa) return LGT_OK;
    TRY(ensure_multi(L));
    auto& W = L->mw;
    const int N = std::min(want, C.n);
    const double2* v[CHRONO_MAX];
    for (int i = 0; i < N; ++i) v[i] = C.hist[(C.head - 1 - i + 2 * CHRONO_MAX) % CHRONO_MAX];   // newest first
    // w_i = A v_i in FP32: t = H_oe v, u = v - kappa^2 H_eo t, t = H^+_oe u, w = u - kappa^2 H^+_eo t
    for (int i = 0; i < N; ++i) CK(blas_d2f(W.p32[i], v[i], L->g.Vh, L->g.Vh, L->st));
    HopArgsM H;
    memset(&H, 0, sizeof H);
    H.U = lk.U12;
    H.g = L->g;
    H.nrhs = N;
    for (int pass = 0; pass < 2; ++pass) {
        const bool dag = pass == 1;
        H.parity = 1;
        for (int i = 0; i < N; ++i) { H.in[i] = dag ? W.u32[i] : W.p32[i]; H.out[i] = W.t32[i]; H.a[i] = 1.0; }
        CK(launch_hop_multi(H, false, dag, EPI_HOP, L->st));
        H.parity = 0;
        for (int i = 0; i < N; ++i) {
            H.in[i] = W.t32[i];
            H.y[i] = dag ? W.u32[i] : W.p32[i];
            H.out[i] = dag ? W.r32[i] : W.u32[i];
            H.a[i] = -kappa * kappa;
        }
        CK(launch_hop_multi(H, false, dag, EPI_XPAY, L->st));
    }
    CdotArgs D;
    memset(&D, 0, sizeof D);
    D.Vh = L->g.Vh;
    D.partials = C.partials;
    D.counter = C.counter;
    D.capacity = C.cap;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) { D.a[i * N + j] = v[i]; D.b[i * N + j] = W.r32[j]; }
    D.out = C.G;
    CK(cdot_many(D, N * N, true, L->st));
    for (int i = 0; i < N; ++i) { D.a[i] = v[i]; D.b[i] = b; }
    D.out = C.g;
    CK(cdot_many(D, N, false, L->st));
    CK(chrono_solve(C.G, C.g, C.c, N, C.used, L->st));
    CK(chrono_combine(x, v, C.c, N, L->g.Vh, L->st));
    *used = true;
    return LGT_OK;
}
static int chrono_record(lgt_lattice* L, const double2* x, double kappa, int iters) {
    auto& C = L->ch;
    if (C.n > 0 && C.kappa != kappa) C.n = C.head = 0;
    C.kappa = kappa;
    if (iters > 0) C.last_iters = iters;
    CK(cudaMemcpyAsync(C.hist[C.head], x, (size_t)12 * L->g.Vh * sizeof(double2), cudaMemcpyDeviceToDevice, L->st));
    C.head = (C.head + 1) % CHRONO_MAX;
    C.n = std::min(C.n + 1, CHRONO_MAX);
    return LGT_OK;
}

static int cg_core(lgt_lattice* L, const Links& lk, const double2* b, double2* x, double kappa, bool eo,
                   const lgt_solver_params* sp, lgt_solve_stats* stats) {
    NvtxRange nvtx("lgt cg");
    auto t0 = std::chrono::steady_clock::now();
    if (!sp) return fail(LGT_EINVAL, "null solver parameters");
    if (sp->precision != LGT_FP64 && sp->precision != LGT_MIXED) return fail(LGT_EINVAL, "solver precision %d", sp->precision);
    if (!(sp->tol > 0) || sp->max_iter <= 0) return fail(LGT_EINVAL, "tol and max_iter must be positive");
    TRY(ensure_solver(L));
    L->cap_valid = false;
    L->cap_df_valid = false;
    L->udf_src = nullptr;   // the links may have changed since the last solve
    const int n = eo ? L->g.Vh : 2 * L->g.Vh;
    const int K = sp->check_every > 0 ? sp->check_every : 16;
    const bool mixed = sp->precision == LGT_MIXED;
    // the mixed even-odd Wilson solver forms its true residuals in double-float
    const bool dfres = mixed && eo && (!lk.C64 || (lk.Cdf && lk.Idf));
    if (dfres) TRY(ensure_df(L));
    auto residual = [&](double2* res) -> int {
        return dfres ? true_residual_df(L, lk, kappa, b, x, res) : true_residual(L, lk, eo, kappa, b, x, res);
    };
    // the vectors of the last residual are the force vectors of x (when x is cap_X)
    auto captured = [&]() {
        const bool cap = L->cap_X && L->cap_Y && (const double2*)x == L->cap_X;
        L->cap_valid = cap && !dfres;
        L->cap_df_valid = cap && dfres;
    };
    const size_t b64 = (size_t)n * 12 * sizeof(double2), b32 = (size_t)n * 6 * sizeof(float4);
    lgt_solve_stats st = {};

    CK(blas_norm2(b, n, L->g.Vh, true, red(L), 0, L->st));
    TRY(sync_scalars(L));
    const double bb = L->hs->slot[0];
    CK(cudaMemsetAsync(x, 0, b64, L->st));
    if (!std::isfinite(bb)) return fail(LGT_ENAN, "right-hand side is not finite");
    if (bb == 0.0) {
        CK(cudaStreamSynchronize(L->st));
        if (stats) *stats = st;
        return LGT_OK;
    }
    const double target = sp->tol * sp->tol * bb;
    Scalars* hs = L->hs;
    // start: x = 0, r = b; or the chronological guess x0 with its FP64 residual
    bool guess = false;
    // (the guess's FP32 products have no clover term: not used with one)
    if (eo && sp->chrono > 0 && !lk.C64) {
        TRY(ensure_chrono(L));
        TRY(chrono_guess(L, lk, b, x, kappa, std::min(sp->chrono, CHRONO_MAX), &guess));
    }
    double rr0 = bb;
    if (guess) {
        TRY(residual(L->r));
        TRY(sync_scalars(L));
        rr0 = hs->slot[0];
        st.reliable_updates += 1;
        // a guess no better than zero (e.g. from a history of another source) is dropped
        if (!(rr0 < bb)) {
            guess = false;
            rr0 = bb;
            CK(cudaMemsetAsync(x, 0, b64, L->st));
        }
    }
    if (!guess) CK(cudaMemcpyAsync(L->r, b, b64, cudaMemcpyDeviceToDevice, L->st));
    memset(hs, 0, sizeof(Scalars));
    hs->rr = rr0;
    hs->rr_max = rr0;
    hs->target = target;
    hs->delta2 = mixed ? sp->delta * sp->delta : 0.0;
    if (mixed) {
        CK(blas_d2f(L->r32, L->r, n, L->g.Vh, L->st));
        CK(cudaMemcpyAsync(L->p32, L->r32, b32, cudaMemcpyDeviceToDevice, L->st));
        CK(cudaMemsetAsync(L->x32, 0, b32, L->st));
    } else {
        CK(cudaMemcpyAsync(L->p, L->r, b64, cudaMemcpyDeviceToDevice, L->st));
    }
    TRY(push_scalars(L));
    double rr_true = rr0;
    int rc = LGT_OK;
    const bool record = eo && sp->chrono > 0 && !lk.C64;
    // Near a nearly singular operator the FP32 recursion can break down (<p, Ap> <= 0 from
    // FP32 rounding) or stop reducing the true residual; a chronological guess can then
    // also carry an error in the lowest modes that the FP32 recursion cannot remove, so
    // a guessed solve that breaks down, stalls or reduces its residual by less than 2x
    // across a reliable update is redone once from x = 0.  A breakdown is handled as a
    // reliable update that also restarts the search direction (at most 16 times); two
    // reliable updates in a row that each fail to halve the true residual (including
    // cycles ended after kMaxCycle iterations) end the FP32 iterations and the solve
    // continues in FP64 CG from the current x and residual.
    bool use32 = mixed;
    bool guessed = guess;   // still iterating from a chronological guess
    int breakdowns = 0, poor = 0, iters_at_update = 0, iters_handover = 0;
    double rr_prev = rr0;
    // an FP32 cycle that runs this long without its stop test firing is ended by a
    // reliable update as well (its progress is then judged like any other); a solve from
    // a guess gets 1.5 times the iterations of the last recorded solve before it is
    // redone from x = 0
    constexpr int kMaxCycle = 1000;
    const int guess_cap = std::max(64, (3 * L->ch.last_iters) / 2 + 32);
    // back to x = 0, r = b (the zero-guess solve), keeping the iteration count
    auto restart_from_zero = [&]() -> int {
        CK(cudaMemsetAsync(x, 0, b64, L->st));
        CK(cudaMemcpyAsync(L->r, b, b64, cudaMemcpyDeviceToDevice, L->st));
        use32 = mixed;
        if (mixed) {
            CK(blas_d2f(L->r32, b, n, L->g.Vh, L->st));
            CK(cudaMemcpyAsync(L->p32, L->r32, b32, cudaMemcpyDeviceToDevice, L->st));
            CK(cudaMemsetAsync(L->x32, 0, b32, L->st));
        } else {
            CK(cudaMemcpyAsync(L->p, b, b64, cudaMemcpyDeviceToDevice, L->st));
        }
        rr_true = rr_prev = bb;
        poor = breakdowns = 0;
        guessed = false;
        st.restarts += 1;
        hs->rr = hs->rr_max = bb;
        hs->done = 0;
        hs->nan = 0;
        hs->delta2 = mixed ? sp->delta * sp->delta : 0.0;
        TRY(push_scalars(L));
        return LGT_OK;
    };
    if (guess && rr0 <= target) {   // the guess already solves the system
        captured();
        if (record) TRY(chrono_record(L, x, kappa, hs->iters));
    }
    for (; !(guess && rr0 <= target);) {
        for (int k = 0; k < K; ++k) {
            if (use32) TRY(cg_iteration(L, lk, false, eo, kappa, L->x32, L->r32, L->p32, L->u32, L->t32));
            else TRY(cg_iteration(L, lk, true, eo, kappa, x, L->r, L->p, L->u, L->t));
        }
        TRY(sync_scalars(L));
        // An FP32 cycle whose recursion residual grew 1e3-fold (in |r|^2) above the true
        // residual it started from has diverged (seen when the search direction kept
        // across a reliable update no longer suits a residual that differed from the
        // recursion's by 2x): its correction is dropped, and the cycle restarts from that
        // residual with p = r (counted as a breakdown)
        if (use32 && !hs->nan && hs->rr_max > 1e3 * rr_prev) {
            if (guessed) {
                iters_at_update = hs->iters;
                TRY(restart_from_zero());
                continue;
            }
            if (++breakdowns > 16) {
                rc = fail(LGT_ENAN, "FP32 CG diverged repeatedly after %d iterations", hs->iters);
                break;
            }
            iters_at_update = hs->iters;
            st.diverged += 1;
            CK(cudaMemsetAsync(L->x32, 0, b32, L->st));
            CK(blas_d2f(L->r32, L->r, n, L->g.Vh, L->st));
            CK(cudaMemcpyAsync(L->p32, L->r32, b32, cudaMemcpyDeviceToDevice, L->st));
            hs->rr = rr_prev;
            hs->rr_max = rr_prev;
            hs->done = 0;
            TRY(push_scalars(L));
            continue;
        }
        const bool breakdown = hs->nan != 0;
        const bool hit_cap = hs->iters >= sp->max_iter;
        const bool long_cycle = guessed ? hs->iters - iters_at_update >= guess_cap
                                        : use32 && hs->iters - iters_at_update >= kMaxCycle;
        // a guessed solve that runs into trouble is redone from x = 0 (once)
        if (guessed && !hit_cap && (breakdown || long_cycle)) {
            iters_at_update = hs->iters;
            TRY(restart_from_zero());
            continue;
        }
        if (breakdown && (!use32 || ++breakdowns > 16)) {
            rc = fail(LGT_ENAN, "non-finite value in CG after %d iterations", hs->iters);
            break;
        }
        if (hs->done || hit_cap || breakdown || long_cycle) {
            iters_at_update = hs->iters;
            if (breakdown) st.breakdowns += 1;
            if (use32) {
                CK(blas_add_f2d(x, L->x32, n, L->g.Vh, L->st));
                CK(cudaMemsetAsync(L->x32, 0, b32, L->st));
            }
            TRY(residual(L->r));
            TRY(sync_scalars(L));
            rr_true = hs->slot[0];
            st.reliable_updates += 1;
            if (!std::isfinite(rr_true)) {
                if (guessed && !hit_cap) { TRY(restart_from_zero()); continue; }
                rc = fail(LGT_ENAN, "non-finite true residual");
                break;
            }
            if (rr_true <= target) {
                captured();
                if (record) TRY(chrono_record(L, x, kappa, hs->iters));
                break;
            }
            if (hit_cap) {
                rc = fail(LGT_ENOCONV, "CG reached max_iter=%d, true relative residual %.3e", sp->max_iter,
                          std::sqrt(rr_true / bb));
                break;
            }
            const bool slow = rr_true > 0.25 * rr_prev;   // |r| shrank by less than 2x since the last update
            if (guessed && slow) { TRY(restart_from_zero()); continue; }
            if (use32) {
                poor = slow ? poor + 1 : 0;
                if (poor >= 2) {   // the FP32 iterations stopped making progress: FP64 from here
                    use32 = false;
                    st.handovers = 1;
                    iters_handover = hs->iters;
                    CK(cudaMemcpyAsync(L->p, L->r, b64, cudaMemcpyDeviceToDevice, L->st));
                }
            }
            rr_prev = rr_true;
            if (use32) {
                CK(blas_d2f(L->r32, L->r, n, L->g.Vh, L->st));
                if (breakdown) CK(cudaMemcpyAsync(L->p32, L->r32, b32, cudaMemcpyDeviceToDevice, L->st));
            }
            hs->rr = rr_true;
            hs->rr_max = rr_true;
            hs->done = 0;
            hs->nan = 0;
            hs->delta2 = use32 ? sp->delta * sp->delta : 0.0;
            TRY(push_scalars(L));
        }
    }
    CK(cudaStreamSynchronize(L->st));
    st.iters = hs->iters;
    st.fp64_iters = mixed ? (st.handovers ? hs->iters - iters_handover : 0) : hs->iters;
    st.true_rel_residual = std::sqrt(rr_true / bb);
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = st;
    return rc;
}

static void add_stats(lgt_solve_stats* acc, const lgt_solve_stats& s) {
    acc->iters += s.iters;
    acc->reliable_updates += s.reliable_updates;
    acc->breakdowns += s.breakdowns;
    acc->diverged += s.diverged;
    acc->handovers += s.handovers;
    acc->fp64_iters += s.fp64_iters;
    acc->restarts += s.restarts;
    acc->true_rel_residual = s.true_rel_residual > acc->true_rel_residual ? s.true_rel_residual : acc->true_rel_residual;
    acc->seconds += s.seconds;
}

extern "C" int lgt_cg_solve(lgt_lattice_t L, const double* b, double* x, double kappa, int even_odd,
                            const lgt_solver_params* sp, lgt_solve_stats* stats) {
    if (!L || !b || !x) return fail(LGT_EINVAL, "null argument");
    if (b == x) return fail(LGT_EINVAL, "b and x must be distinct");
    return cg_core(L, L->thin, (const double2*)b, (double2*)x, kappa, even_odd != 0, sp, stats);
}

extern "C" int lgt_chrono_reset(lgt_lattice_t L) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    L->ch.n = L->ch.head = 0;
    return LGT_OK;
}

// ---------------------------------------------------------------- several right-hand sides
// launch arguments for the running systems sys[0..n): slot j holds system sys[j]
static HopArgsM hop_multi_base(lgt_lattice* L, int n, const int* sys) {
    HopArgsM a;
    memset(&a, 0, sizeof a);
    a.U = L->thin.U12;
    a.g = L->g;
    a.nrhs = n;
    a.skip = 1;
    a.red_capacity = L->n_partials;
    for (int j = 0; j < n; ++j) {
        const int k = sys[j];
        a.s[j] = L->mw.s + k;
        a.partials[j] = L->mw.partials[k];
        a.counter[j] = (unsigned*)((char*)L->mw.counter + 64 * k);
        a.a[j] = 1.0;
    }
    return a;
}

// One FP32 CG iteration of the running systems sys[0..n) (A_k = Dhat_k^+ Dhat_k, even
// sites): the kernel sequence of cg_iteration, each launch covering all of them.
static int cg_iteration_multi(lgt_lattice* L, int n, const int* sys, const double* kappa) {
    auto& W = L->mw;
    HopArgsM A = hop_multi_base(L, n, sys);
    A.parity = 1;
    for (int j = 0; j < n; ++j) { A.in[j] = W.p32[sys[j]]; A.out[j] = W.t32[sys[j]]; }
    CK(launch_hop_multi(A, false, false, EPI_HOP, L->st));
    A = hop_multi_base(L, n, sys);
    A.parity = 0; A.red_op = RED_PAP; A.defer = 1;
    for (int j = 0; j < n; ++j) {
        const int k = sys[j];
        A.in[j] = W.t32[k]; A.out[j] = W.u32[k]; A.y[j] = W.p32[k]; A.a[j] = -kappa[k] * kappa[k];
    }
    CK(launch_hop_multi(A, false, false, EPI_XPAY_NORM, L->st));
    // the hop of Dhat^+ does not need alpha: its block 0 finishes <p, A p> -> alpha
    A = hop_multi_base(L, n, sys);
    A.parity = 1; A.fin_n = hop_grid(L->g, 0); A.fin_op = RED_PAP;
    for (int j = 0; j < n; ++j) { A.in[j] = W.u32[sys[j]]; A.out[j] = W.t32[sys[j]]; }
    CK(launch_hop_multi(A, false, true, EPI_HOP, L->st));
    A = hop_multi_base(L, n, sys);
    A.parity = 0; A.red_op = RED_RR;
    for (int j = 0; j < n; ++j) {
        const int k = sys[j];
        A.in[j] = W.t32[k]; A.y[j] = W.u32[k]; A.a[j] = -kappa[k] * kappa[k];
        A.r[j] = W.r32[k];
    }
    CK(launch_hop_multi(A, false, true, EPI_CG, L->st));
    PUpdateM P;
    memset(&P, 0, sizeof P);
    P.nrhs = n;
    for (int j = 0; j < n; ++j) {
        const int k = sys[j];
        P.p[j] = W.p32[k]; P.r[j] = W.r32[k]; P.x[j] = W.x32[k];
        P.red[j] = RedArgs{W.s + k, W.partials[k], (unsigned*)((char*)W.counter + 64 * k), L->n_partials};
    }
    CK(blas_cg_p_update_multi(P, L->g.Vh, false, L->st));
    return LGT_OK;
}

// Mixed-precision CG on nrhs systems sharing the handle's links: each system has
// its own kappa, scalars, stop test and FP64 reliable updates (as cg_core), and
// the FP32 operator applications of all running systems share every link load.
// A system's iterates are the ones cg_core produces for it alone.
static int cg_multi(lgt_lattice* L, int nrhs, const double2* const* b, double2* const* x, const double* kappa,
                    const lgt_solver_params* sp, lgt_solve_stats* stats) {
    auto t0 = std::chrono::steady_clock::now();
    TRY(ensure_solver(L));
    TRY(ensure_multi(L));
    auto& W = L->mw;
    const int n = L->g.Vh;
    const int K = sp->check_every > 0 ? sp->check_every : 16;
    const size_t b64 = (size_t)n * 12 * sizeof(double2), b32 = (size_t)n * 6 * sizeof(float4);
    L->cap_valid = false;
    L->cap_df_valid = false;
    // true residuals in double-float, as the single-system mixed solver forms them
    TRY(ensure_df(L));
    L->udf_src = nullptr;
    for (int k = 0; k < nrhs; ++k) CK(blas_norm2(b[k], n, L->g.Vh, true, red(L), k, L->st));
    TRY(sync_scalars(L));
    double bb[KMAX_RHS], rr_true[KMAX_RHS];
    int rel[KMAX_RHS], div[KMAX_RHS] = {};
    bool fin[KMAX_RHS];
    int rc = LGT_OK;
    memset(W.hs, 0, sizeof(Scalars) * KMAX_RHS);
    for (int k = 0; k < nrhs; ++k) {
        bb[k] = L->hs->slot[k];
        rr_true[k] = bb[k];
        rel[k] = 0;
        CK(cudaMemsetAsync(x[k], 0, b64, L->st));
        if (!std::isfinite(bb[k])) return fail(LGT_ENAN, "right-hand side %d is not finite", k);
        fin[k] = bb[k] == 0.0;
        Scalars& h = W.hs[k];
        h.rr = h.rr_max = bb[k];
        h.target = sp->tol * sp->tol * bb[k];
        h.delta2 = sp->delta * sp->delta;
        h.done = fin[k] ? 2 : 0;
        CK(cudaMemcpyAsync(W.r64[k], b[k], b64, cudaMemcpyDeviceToDevice, L->st));
        CK(blas_d2f(W.r32[k], b[k], n, L->g.Vh, L->st));
        CK(cudaMemcpyAsync(W.p32[k], W.r32[k], b32, cudaMemcpyDeviceToDevice, L->st));
        CK(cudaMemsetAsync(W.x32[k], 0, b32, L->st));
    }
    CK(cudaMemcpyAsync(W.s, W.hs, sizeof(Scalars) * KMAX_RHS, cudaMemcpyHostToDevice, L->st));
    for (;;) {
        // the launches of this batch cover the systems still running at its start
        int sys[KMAX_RHS], nrun = 0;
        for (int k = 0; k < nrhs; ++k)
            if (!fin[k]) sys[nrun++] = k;
        if (nrun == 0) break;
        for (int it = 0; it < K; ++it) TRY(cg_iteration_multi(L, nrun, sys, kappa));
        CK(cudaMemcpyAsync(W.hs, W.s, sizeof(Scalars) * KMAX_RHS, cudaMemcpyDeviceToHost, L->st));
        CK(cudaStreamSynchronize(L->st));
        for (int k = 0; k < nrhs; ++k) {
            if (fin[k]) continue;
            Scalars& h = W.hs[k];
            // a diverged FP32 cycle restarts from its last true residual (as cg_core)
            if (!h.nan && h.rr_max > 1e3 * rr_true[k]) {
                div[k] += 1;
                CK(cudaMemsetAsync(W.x32[k], 0, b32, L->st));
                CK(blas_d2f(W.r32[k], W.r64[k], n, L->g.Vh, L->st));
                CK(cudaMemcpyAsync(W.p32[k], W.r32[k], b32, cudaMemcpyDeviceToDevice, L->st));
                h.rr = h.rr_max = rr_true[k];
                h.done = 0;
                continue;
            }
            if (h.nan) {
                if (rc == LGT_OK) rc = fail(LGT_ENAN, "non-finite value in CG of system %d", k);
                fin[k] = true; h.done = 2;
                continue;
            }
            const bool hit_cap = h.iters >= sp->max_iter;
            if (!(h.done || hit_cap)) continue;
            CK(blas_add_f2d(x[k], W.x32[k], n, L->g.Vh, L->st));
            CK(cudaMemsetAsync(W.x32[k], 0, b32, L->st));
            TRY(true_residual_df(L, L->thin, kappa[k], b[k], x[k], W.r64[k]));
            TRY(sync_scalars(L));
            rr_true[k] = L->hs->slot[0];
            rel[k] += 1;
            if (!std::isfinite(rr_true[k])) {
                if (rc == LGT_OK) rc = fail(LGT_ENAN, "non-finite true residual of system %d", k);
                fin[k] = true; h.done = 2;
            } else if (rr_true[k] <= h.target) {
                fin[k] = true; h.done = 2;
            } else if (hit_cap) {
                if (rc == LGT_OK)
                    rc = fail(LGT_ENOCONV, "CG of system %d reached max_iter=%d, true relative residual %.3e", k,
                              sp->max_iter, std::sqrt(rr_true[k] / bb[k]));
                fin[k] = true; h.done = 2;
            } else {
                CK(blas_d2f(W.r32[k], W.r64[k], n, L->g.Vh, L->st));
                h.rr = h.rr_max = rr_true[k];
                h.done = 0;
            }
        }
        CK(cudaMemcpyAsync(W.s, W.hs, sizeof(Scalars) * KMAX_RHS, cudaMemcpyHostToDevice, L->st));
    }
    CK(cudaStreamSynchronize(L->st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats)
        for (int k = 0; k < nrhs; ++k)
            stats[k] = lgt_solve_stats{W.hs[k].iters, rel[k], bb[k] > 0 ? std::sqrt(rr_true[k] / bb[k]) : 0.0, secs,
                                       0, div[k], 0, 0, 0};
    return rc;
}

extern "C" int lgt_cg_solve_multi(lgt_lattice_t L, int nrhs, const double* const* b, double* const* x,
                                  const double* kappa, const lgt_solver_params* sp, lgt_solve_stats* stats) {
    if (!L || !b || !x || !kappa || !sp) return fail(LGT_EINVAL, "null argument");
    if (nrhs < 1 || nrhs > KMAX_RHS) return fail(LGT_EINVAL, "nrhs = %d outside 1..%d", nrhs, KMAX_RHS);
    if (L->thin.C64) return fail(LGT_EINVAL, "the clover term is attached: even-odd solves are not available");
    if (sp->precision != LGT_FP64 && sp->precision != LGT_MIXED) return fail(LGT_EINVAL, "solver precision %d", sp->precision);
    if (!(sp->tol > 0) || sp->max_iter <= 0) return fail(LGT_EINVAL, "tol and max_iter must be positive");
    for (int k = 0; k < nrhs; ++k) {
        if (!b[k] || !x[k]) return fail(LGT_EINVAL, "null field of system %d", k);
        for (int j = 0; j < nrhs; ++j)
            if ((const double*)x[k] == b[j] || (j != k && x[k] == x[j]))
                return fail(LGT_EINVAL, "solution %d aliases another field", k);
    }
    if (sp->precision == LGT_FP64) {   // FP64 arithmetic bounds the FP64 hop: solve one after another
        for (int k = 0; k < nrhs; ++k)
            TRY(cg_core(L, L->thin, (const double2*)b[k], (double2*)x[k], kappa[k], true, sp, stats ? stats + k : nullptr));
        return LGT_OK;
    }
    return cg_multi(L, nrhs, (const double2* const*)b, (double2* const*)x, kappa, sp, stats);
}

extern "C" int lgt_hop_multi(lgt_lattice_t L, int nrhs, const void* const* in, void* const* out, int out_parity,
                             int dagger) {
    if (!L || !in || !out) return fail(LGT_EINVAL, "null argument");
    if (nrhs < 1 || nrhs > KMAX_RHS) return fail(LGT_EINVAL, "nrhs = %d outside 1..%d", nrhs, KMAX_RHS);
    if (out_parity != LGT_EVEN && out_parity != LGT_ODD) return fail(LGT_EINVAL, "hop needs EVEN or ODD");
    HopArgsM A;
    memset(&A, 0, sizeof A);
    A.U = L->thin.U12;
    A.g = L->g;
    A.parity = out_parity;
    A.nrhs = nrhs;
    for (int k = 0; k < nrhs; ++k) {
        if (!in[k] || !out[k]) return fail(LGT_EINVAL, "null field of system %d", k);
        A.in[k] = in[k]; A.out[k] = out[k]; A.a[k] = 1.0;
    }
    CK(launch_hop_multi(A, false, dagger != 0, EPI_HOP, L->st));
    return LGT_OK;
}

// ---------------------------------------------------------------- smearing
static int check_action(const lgt_action_params* ap) {
    if (!ap) return fail(LGT_EINVAL, "null action parameters");
    if (ap->n_stout < 0 || ap->n_stout > MAX_STOUT)
        return fail(LGT_EINVAL, "n_stout = %d outside 0..%d", ap->n_stout, MAX_STOUT);
    if (ap->stout_recompute < 0) return fail(LGT_EINVAL, "stout_recompute = %d", ap->stout_recompute);
    if (ap->force_arith < LGT_ARITH_FP64 || ap->force_arith > LGT_ARITH_DF64)
        return fail(LGT_EINVAL, "force_arith = %d", ap->force_arith);
    return LGT_OK;
}
// Smear the thin links through levels 1..n into the fields of the plan.
static int smear_to(lgt_lattice* L, const StoutPlan& P, double rho, double2** level_n) {
    const double2* src = L->thin.U;
    for (int k = 1; k <= P.n; ++k) {
        double2* dst = L->sbuf[P.slot(k)];
        CK(stout_forward(src, dst, L->g, rho, L->st));
        src = dst;
    }
    *level_n = (double2*)src;
    return LGT_OK;
}
// links seen by the Dirac operator: thin, or the top stout level (+ its FP32 copy)
// (+ the clover term of ap->csw built from them; lgt_set_clover's field is not used here)
// With a mixed solver and double-float force arithmetic (sp given) the clover field is
// built in double-float arithmetic as well (the FP64 field-strength products are FP64
// bound); the FP64 path and the actions build it in FP64.  With a mixed solver and the
// even-odd form, double-float copies of the blocks serve the solver's true residuals.
static int fermion_links(lgt_lattice* L, const lgt_action_params* ap, Links* out,
                         const lgt_solver_params* sp = nullptr) {
    Links lk{L->thin.U, L->thin.U12};
    if (ap->n_stout > 0) {
        TRY(ensure_stout(L, ap->n_stout, ap->stout_recompute));
        double2* top;
        TRY(smear_to(L, stout_plan(ap->n_stout, ap->stout_recompute), ap->rho, &top));
        CK(gauge_make12(L->stout_top12, top, L->g, L->st));
        lk = Links{top, L->stout_top12};
    }
    if (ap->fermions && ap->csw != 0.0) {
        TRY(ensure_clover(L, false));
        if (sp && sp->precision == LGT_MIXED && ap->force_arith == LGT_ARITH_DF64) {
            TRY(ensure_df(L));
            CK(links_to_df(L->Udf, lk.U, L->g, L->st));
            L->udf_src = nullptr;   // the solve rebuilds (or keeps) its own copy
            // the force insertion buffer is free until the force: scratch for the field strengths
            CK(clover_field_df(L->Udf, L->g, clover_sigma(), ap->kappa, ap->csw, L->cins, L->call_c64, L->call_c32,
                               L->st));
        } else {
            CK(clover_field(lk.U, L->g, clover_sigma(), ap->kappa, ap->csw, L->call_c64, L->call_c32, L->st));
        }
        lk.C64 = L->call_c64;
        lk.C32 = L->call_c32;
        if (ap->even_odd) TRY(clover_inverse_odd(L, &lk, L->call_i64, L->call_i32));
        if (ap->even_odd && sp && sp->precision == LGT_MIXED) {
            if (!L->call_cdf) {
                TRY(A(L, (size_t)2 * 36 * L->g.Vh * sizeof(float4), &L->call_cdf));
                TRY(A(L, (size_t)2 * 36 * L->g.Vh * sizeof(float4), &L->call_idf));
            }
            CK(clover_pack_df(lk.C64, L->g, 0, L->call_cdf, L->st));
            CK(clover_pack_df(lk.I64, L->g, 1, L->call_idf, L->st));
            lk.Cdf = L->call_cdf;
            lk.Idf = L->call_idf;
        }
    }
    *out = lk;
    return LGT_OK;
}
// the thin links without any clover term (what the gauge action and force see)
static Links gauge_links(lgt_lattice* L) { return Links{L->thin.U, L->thin.U12}; }

// ---------------------------------------------------------------- actions
// S_f pieces after a solve chi = X (even half or full): eta = M chi into Y
static int pf_action_on(lgt_lattice* L, const Links& lk, const lgt_action_params* ap, const double2* phi,
                        const lgt_solver_params* sp, double* S_f, lgt_solve_stats* stats) {
    TRY(ensure_solver(L));
    const bool eo = ap->even_odd != 0;
    const int n = eo ? L->g.Vh : 2 * L->g.Vh;
    L->cap_X = L->X;
    L->cap_Y = L->Y;
    const int rc = cg_core(L, lk, phi, L->X, ap->kappa, eo, sp, stats);
    L->cap_X = L->cap_Y = nullptr;
    TRY(rc);
    TRY(cap_to_fp64(L));
    // eta = M chi: left in Y by the solver's final residual, else computed here
    if (!L->cap_valid) {
        if (eo) TRY(dhat(L, lk, true, false, L->X, L->Y, L->t, ap->kappa));
        else TRY(dfull(L, lk, true, false, L->X, L->Y, ap->kappa));
    }
    CK(blas_action_parts(phi, L->X, L->Y, n, L->g.Vh, red(L), L->st));
    TRY(sync_scalars(L));
    *S_f = 2.0 * L->hs->slot[0] - L->hs->slot[1];
    // even-odd clover: det(D^+ D) = det(M_oo)^2 det(Dhat^+ Dhat), so S_f holds -2 ln det M_oo
    if (eo && lk.C64) *S_f -= 2.0 * lk.logdet_odd;
    return LGT_OK;
}

extern "C" int lgt_action(lgt_lattice_t L, const lgt_action_params* ap, const double* phi,
                          const lgt_solver_params* sp, double* S_g, double* S_f, lgt_solve_stats* stats) {
    if (!L) return fail(LGT_EINVAL, "null lattice");
    TRY(check_action(ap));
    if (stats) *stats = lgt_solve_stats{};
    if (S_g) {
        double s;
        TRY(gauge_action_value(L, ap, &s));
        *S_g = s;
    }
    if (S_f) {
        *S_f = 0.0;
        if (ap->fermions) {
            if (!phi) return fail(LGT_EINVAL, "null phi");
            Links lk;
            TRY(fermion_links(L, ap, &lk));
            TRY(pf_action_on(L, lk, ap, (const double2*)phi, sp, S_f, stats));
            if (!std::isfinite(*S_f)) return fail(LGT_ENAN, "non-finite S_f");
        }
    }
    return LGT_OK;
}

extern "C" int lgt_kinetic_energy(lgt_lattice_t L, const double* mom, double* K) {
    if (!L || !mom || !K) return fail(LGT_EINVAL, "null argument");
    CK(gauge_kinetic((const double2*)mom, L->g, red(L), 0, L->st));
    TRY(sync_scalars(L));
    *K = L->hs->slot[0];
    return LGT_OK;
}

// ---------------------------------------------------------------- forces
// Solve and build X, Y of the fermion force on links lk (FP64 X, Y; with fp32 the
// vectors are built in FP32 from the FP64 solution: X32, Y32).
static int force_vectors(lgt_lattice* L, const Links& lk, const lgt_action_params* ap, const double2* phi,
                         const lgt_solver_params* sp, lgt_solve_stats* stats, bool fp32, bool dfa) {
    const bool eo = ap->even_odd != 0;
    L->cap_X = L->X;
    L->cap_Y = L->Y;
    const int rc = cg_core(L, lk, phi, L->X, ap->kappa, eo, sp, stats);
    L->cap_X = L->cap_Y = nullptr;
    TRY(rc);
    if (eo && lk.C64) {
        // the FP64 vectors (from the solver's final residual, else computed here); the
        // FP32 force arithmetic takes their FP32 copies
        TRY(cap_to_fp64(L));
        if (!L->cap_valid)
            TRY(eo_clover_xy(L, lk, ap->kappa, L->X, (double2*)half(L->X, L, true, 1), L->Y,
                             (double2*)half(L->Y, L, true, 1)));
        if (fp32) {
            CK(blas_d2f(L->X32, L->X, 2 * L->g.Vh, L->g.Vh, L->st));
            CK(blas_d2f(L->Y32, L->Y, 2 * L->g.Vh, L->g.Vh, L->st));
        }
        return LGT_OK;
    }
    if (fp32) {
        if (eo) {
            float4* Xo = (float4*)half(L->X32, L, false, 1);
            float4* Yo = (float4*)half(L->Y32, L, false, 1);
            CK(blas_d2f(L->X32, L->X, L->g.Vh, L->g.Vh, L->st));
            TRY(hop1(L, lk, false, false, 1, L->X32, Xo, ap->kappa));
            TRY(hop1(L, lk, false, false, 0, Xo, L->Y32, -ap->kappa, EPI_XPAY, L->X32));
            TRY(hop1(L, lk, false, true, 1, L->Y32, Yo, ap->kappa));
        } else {
            CK(blas_d2f(L->X32, L->X, 2 * L->g.Vh, L->g.Vh, L->st));
            TRY(dfull(L, lk, false, false, L->X32, L->Y32, ap->kappa));
        }
        return LGT_OK;
    }
    // built by the solver's final residual: in double-float (read as such by the
    // double-float force) or in FP64
    if (L->cap_df_valid && dfa) return LGT_OK;
    TRY(cap_to_fp64(L));
    if (L->cap_valid) return LGT_OK;
    if (eo) {
        double2* Xo = (double2*)half(L->X, L, true, 1);
        double2* Yo = (double2*)half(L->Y, L, true, 1);
        // X_o = kappa H_oe chi_e;  eta_e = chi_e - kappa H_eo X_o;  Y_o = kappa (H^+)_oe eta_e
        TRY(hop1(L, lk, true, false, 1, L->X, Xo, ap->kappa));
        TRY(hop1(L, lk, true, false, 0, Xo, L->Y, -ap->kappa, EPI_XPAY, L->X));
        TRY(hop1(L, lk, true, true, 1, L->Y, Yo, ap->kappa));
    } else {
        TRY(dfull(L, lk, true, false, L->X, L->Y, ap->kappa));
    }
    return LGT_OK;
}

// out = keep*out + coef * (dS_G + dS_f) in Lie (form 0) or G (form 1) layout, on the
// links the actions see (no smearing here).  With the mixed solver, Lie-form forces
// use the arithmetic ap->force_arith: FP64 kernels, FP32 arithmetic on the FP32 links
// and FP32 X, Y, or double-float arithmetic on double-float copies of the FP64 links
// and FP64 X, Y; every variant accumulates into FP64.  FP64 solves, and the G form,
// always use the FP64 kernels.
static int force_on(lgt_lattice* L, const Links& gauge_lk, const Links& ferm_lk, const lgt_action_params* ap,
                    const double2* phi, const lgt_solver_params* sp, double coef, int keep, int form, double2* out,
                    lgt_solve_stats* stats) {
    NvtxRange nvtx("lgt force");
    const int arith = (form == 0 && sp && sp->precision == LGT_MIXED) ? ap->force_arith : LGT_ARITH_FP64;
    const bool fp32 = arith == LGT_ARITH_FP32, dfa = arith == LGT_ARITH_DF64;
    if (dfa) TRY(ensure_df(L));
    L->udf_src = nullptr;
    // the double-float copy of links U in Udf (the solve may have made it already)
    auto udf_of = [&](const double2* U) -> int {
        if (L->udf_src != U) {
            CK(links_to_df(L->Udf, U, L->g, L->st));
            L->udf_src = U;
        }
        return LGT_OK;
    };
    if (ap->fermions) {
        if (!phi) return fail(LGT_EINVAL, "null phi");
        TRY(ensure_solver(L));
        TRY(force_vectors(L, ferm_lk, ap, phi, sp, stats, fp32, dfa));
    }
    if (ap->beta != 0.0) {
        if (fp32) CK(gauge_force_fp32(gauge_lk.U12, L->g, ap->beta, ap->c1, coef, keep, out, L->st));
        else if (dfa && ap->c1 == 0.0) {
            TRY(udf_of(gauge_lk.U));
            CK(gauge_force_df(L->Udf, L->g, ap->beta, coef, keep, out, L->st));
        } else CK(gauge_force(gauge_lk.U, L->g, ap->beta, ap->c1, coef, keep, form, out, L->st));
        keep = 1;
    }
    if (ap->fermions) {
        if (fp32) CK(fermion_force_fp32(ferm_lk.U12, L->X32, L->Y32, L->g, ap->kappa, coef, keep, out, L->st));
        else if (dfa) {
            TRY(udf_of(ferm_lk.U));
            if (!L->cap_df_valid) {   // the vectors are in FP64: their double-float copies
                CK(spinor_to_df(L->Xdf, L->X, L->g, L->st));
                CK(spinor_to_df(L->Ydf, L->Y, L->g, L->st));
            }
            CK(fermion_force_df(L->Udf, L->Xdf, L->Ydf, L->g, ap->kappa, coef, keep, out, L->st));
        } else CK(fermion_force(ferm_lk.U, L->X, L->Y, L->g, ap->kappa, coef, keep, form, out, L->st));
        keep = 1;
        if (ferm_lk.C64) {   // clover part, FP64 from X, Y (full lattice: X = chi, Y = D chi)
            if (fp32 && !L->cap_valid && !ap->even_odd) TRY(dfull(L, ferm_lk, true, false, L->X, L->Y, ap->kappa));
            CK(clover_insertion(L->X, L->Y, L->g, clover_sigma(), ap->kappa, ap->csw, L->cins, L->st));
            // even-odd: the odd-site determinant -2 ln det M_oo
            if (ap->even_odd)
                CK(clover_det_insertion(ferm_lk.I64, L->g, 1, clover_sigma(), ap->kappa, ap->csw, L->cins, L->st));
            // double-float force arithmetic: the gather from the double-float links the
            // fermion force just used (Udf holds ferm_lk.U)
            if (dfa) {
                CK(complex_to_df(L->cins_df, L->cins, 2L * 54 * L->g.Vh, L->st));
                CK(clover_force_df(L->Udf, L->cins_df, L->g, coef, 1, out, L->st));
            }
            else CK(clover_force(ferm_lk.U, L->cins, L->g, coef, 1, form, out, L->st));
        }
    }
    if (!keep) CK(cudaMemsetAsync(out, 0, form == 0 ? mom_bytes(L) : links64(L), L->st));
    return LGT_OK;
}

// Adjoint of the smearing levels n..1 (after smear_to with the same plan): sgrad[0]
// holds the gradient w.r.t. the top level on entry; the gradient w.r.t. the thin
// links is written to G.  The input U_{k-1} of level k is read from where the plan
// keeps it, or recomputed (mode 1: from the thin links; checkpoint mode: each
// segment below the top one from its checkpoint, once).
static int stout_chain(lgt_lattice* L, const lgt_action_params* ap, double2* G) {
    const StoutPlan P = stout_plan(ap->n_stout, ap->stout_recompute);
    double2* ga = L->sgrad[0];
    double2* gb = L->sgrad[1];
    const double rho = ap->rho;
    auto step = [&](int k, const double2* Uin) -> int {
        double2* dst = (k == 1) ? G : gb;
        CK(stout_backward(Uin, ga, dst, L->sgrad[2], L->g, rho, L->st));
        std::swap(ga, gb);
        return LGT_OK;
    };
    if (P.m == 0) {
        for (int k = P.n; k >= 1; --k) TRY(step(k, k == 1 ? L->thin.U : L->sbuf[P.slot(k - 1)]));
    } else if (P.m == 1) {
        // U_{k-1} recomputed from the thin links into the field the top level does not use
        // (the top level itself is no longer needed once its gradient exists)
        for (int k = P.n; k >= 1; --k) {
            const double2* src = L->thin.U;
            for (int j = 1; j <= k - 1; ++j) {
                double2* dst = L->sbuf[((k - 1 - j) % 2 == 0) ? 1 : 0];
                CK(stout_forward(src, dst, L->g, rho, L->st));
                src = dst;
            }
            TRY(step(k, src));
        }
    } else {
        const int c = P.c;
        for (int s0 = ((P.n - 1) / c) * c; s0 >= 0; s0 -= c) {
            const int e = std::min(s0 + c, P.n);
            const double2* base = (s0 == 0) ? L->thin.U : L->sbuf[P.slot(s0)];
            // levels s0+1 .. e-1 into the segment fields (the top segment's are still
            // there from the forward pass)
            if (e != P.n || s0 + c < P.n) {
                const double2* src = base;
                for (int k = s0 + 1; k <= e - 1; ++k) {
                    double2* dst = L->sbuf[P.nck + (k - s0)];
                    CK(stout_forward(src, dst, L->g, rho, L->st));
                    src = dst;
                }
            }
            for (int k = e; k >= s0 + 1; --k)
                TRY(step(k, (k - 1 == s0) ? base : L->sbuf[P.nck + (k - 1 - s0)]));
        }
    }
    return LGT_OK;
}

// Smeared fermion action: G_fermion w.r.t. the top level, taken back level by
// level; the gauge action sees the thin links.  Result G in G layout (thin links).
static int force_grad_stout(lgt_lattice* L, const lgt_action_params* ap, const double2* phi,
                            const lgt_solver_params* sp, double2* G, lgt_solve_stats* stats) {
    Links top;
    TRY(fermion_links(L, ap, &top));
    double2* ga = L->sgrad[0];
    lgt_action_params fa = *ap;
    fa.beta = 0.0;
    if (ap->fermions) {
        TRY(force_on(L, L->thin, top, &fa, phi, sp, 1.0, 0, 1, ga, stats));
    } else {
        CK(cudaMemsetAsync(ga, 0, links64(L), L->st));
    }
    TRY(stout_chain(L, ap, G));
    if (ap->beta != 0.0) CK(gauge_force(L->thin.U, L->g, ap->beta, ap->c1, 1.0, 1, 1, G, L->st));
    return LGT_OK;
}

// Lie components F_a = Re tr(G^+ i T^a U) of a G-form gradient on the handle's links
extern "C" int lgt_grad_to_lie(lgt_lattice_t L, const double* G_field, double* F_mom) {
    if (!L || !G_field || !F_mom) return fail(LGT_EINVAL, "null argument");
    CK(grad_to_lie((double2*)F_mom, (const double2*)G_field, L->thin.U, L->g, L->st));
    return LGT_OK;
}

// smeared links of the handle's gauge field, in canonical layout
extern "C" int lgt_stout_smear(lgt_lattice_t L, double rho, int n_levels, int recompute, double* out_canonical) {
    if (!L || !out_canonical) return fail(LGT_EINVAL, "null argument");
    lgt_action_params ap = {0.0, 0.0, 0, 0, n_levels, rho, recompute};
    TRY(check_action(&ap));
    Links top;
    TRY(fermion_links(L, &ap, &top));
    CK(gauge_unpack_links(out_canonical, top.U, L->g, L->st));
    CK(cudaStreamSynchronize(L->st));
    return LGT_OK;
}

// adjoint of the n-level smearing: gradient w.r.t. the top level -> thin links
extern "C" int lgt_stout_backward(lgt_lattice_t L, double rho, int n_levels, int recompute,
                                  const double* G_top_canonical, double* G_thin_canonical) {
    if (!L || !G_top_canonical || !G_thin_canonical) return fail(LGT_EINVAL, "null argument");
    lgt_action_params ap = {0.0, 0.0, 0, 0, n_levels, rho, recompute};
    TRY(check_action(&ap));
    TRY(ensure_md(L));
    if (n_levels == 0) {
        CK(cudaMemcpyAsync(G_thin_canonical, G_top_canonical, links64(L), cudaMemcpyDeviceToDevice, L->st));
        CK(cudaStreamSynchronize(L->st));
        return LGT_OK;
    }
    Links top;
    TRY(fermion_links(L, &ap, &top));   // forward levels (stored mode needs them all)
    CK(gauge_pack_field(L->sgrad[0], (const double2*)G_top_canonical, L->g, L->st));
    TRY(stout_chain(L, &ap, L->G));
    CK(gauge_unpack_field(G_thin_canonical, L->G, L->g, L->st));
    CK(cudaStreamSynchronize(L->st));
    return LGT_OK;
}

extern "C" int lgt_force(lgt_lattice_t L, const lgt_action_params* ap, const double* phi,
                         const lgt_solver_params* sp, double* F_out, int form, lgt_solve_stats* stats) {
    if (!L || !F_out) return fail(LGT_EINVAL, "null argument");
    TRY(check_action(ap));
    if (form != LGT_FORCE_LIE && form != LGT_GRAD_G) return fail(LGT_EINVAL, "form %d", form);
    if (stats) *stats = lgt_solve_stats{};
    if (ap->n_stout == 0) {
        Links fl;
        TRY(fermion_links(L, ap, &fl, form == LGT_FORCE_LIE ? sp : nullptr));
        TRY(force_on(L, gauge_links(L), fl, ap, (const double2*)phi, sp, 1.0, 0, form, (double2*)F_out, stats));
    } else {
        TRY(ensure_solver(L));
        TRY(ensure_md(L));
        double2* G = form == LGT_GRAD_G ? (double2*)F_out : L->G;
        TRY(force_grad_stout(L, ap, (const double2*)phi, sp, G, stats));
        if (form == LGT_FORCE_LIE) CK(grad_to_lie((double2*)F_out, G, L->thin.U, L->g, L->st));
    }
    CK(cudaStreamSynchronize(L->st));
    return LGT_OK;
}

// mom -= eps F
static int kick(lgt_lattice* L, double2* mom, double eps, const lgt_action_params* ap, const double2* phi,
                const lgt_solver_params* sp, lgt_solve_stats* stats) {
    // the gauge action always sees thin links: only a fermion part goes through smearing
    if (ap->n_stout == 0 || !ap->fermions) {
        Links fl;
        TRY(fermion_links(L, ap, &fl, sp));
        return force_on(L, gauge_links(L), fl, ap, phi, sp, -eps, 1, 0, mom, stats);
    }
    TRY(ensure_md(L));
    TRY(force_grad_stout(L, ap, phi, sp, L->G, stats));
    CK(grad_to_lie(L->F, L->G, L->thin.U, L->g, L->st));
    CK(gauge_kick(mom, L->F, eps, L->g, L->st));
    return LGT_OK;
}

// U <- exp(i eps P) U.  With double-float arithmetic on the mixed path (df) and a
// double-float copy of exactly these links at hand (made by the force evaluation before
// the update), the update runs in double-float from that copy and keeps it current;
// otherwise in FP64, and the copy is dropped.
static int update_links(lgt_lattice* L, const double2* mom, double eps, bool df) {
    if (df && L->Udf && L->udf_src == L->thin.U) {
        CK(update_links_df(L->Udf, L->thin.U, L->thin.U12, mom, eps, L->g, L->st));
        return LGT_OK;
    }
    CK(gauge_update_links(L->thin.U, L->thin.U12, mom, eps, L->g, L->st));
    L->udf_src = nullptr;
    return LGT_OK;
}
static bool df_updates(const lgt_action_params* ap, const lgt_solver_params* sp) {
    return ap && sp && sp->precision == LGT_MIXED && ap->force_arith == LGT_ARITH_DF64;
}

extern "C" int lgt_md_update(lgt_lattice_t L, double* mom, double eps, int which, const lgt_action_params* ap,
                             const double* phi, const lgt_solver_params* sp, lgt_solve_stats* stats) {
    if (!L || !mom) return fail(LGT_EINVAL, "null argument");
    NvtxRange nvtx(which == LGT_UPDATE_U ? "lgt update U" : "lgt update P");
    if (stats) *stats = lgt_solve_stats{};
    if (which == LGT_UPDATE_U) return update_links(L, (const double2*)mom, eps, df_updates(ap, sp));
    if (which != LGT_UPDATE_P) return fail(LGT_EINVAL, "which = %d", which);
    TRY(check_action(ap));
    lgt_solve_stats s = {};
    TRY(kick(L, (double2*)mom, eps, ap, (const double2*)phi, sp, &s));
    CK(cudaStreamSynchronize(L->st));
    if (stats) *stats = s;
    return LGT_OK;
}

extern "C" int lgt_gaussian_momenta(lgt_lattice_t L, double* mom, uint64_t seed, uint32_t traj) {
    if (!L || !mom) return fail(LGT_EINVAL, "null argument");
    CK(gauge_momenta_heatbath((double2*)mom, L->g, seed, traj, L->st));
    return LGT_OK;
}

extern "C" int lgt_gaussian_spinor(lgt_lattice_t L, double* field, uint64_t seed, uint32_t traj, uint32_t field_id,
                                   int parity) {
    if (!L || !field) return fail(LGT_EINVAL, "null argument");
    TRY(check_parity(parity));
    CK(spinor_gaussian((double2*)field, L->g, parity, seed, traj, field_id, L->st));
    return LGT_OK;
}

// ---------------------------------------------------------------- HMC
static int integrate(lgt_lattice* L, const lgt_action_params* ap, const lgt_hmc_params* hp, const double2* phi,
                     lgt_solve_stats* tot, int* evals) {
    const double eps = hp->tau / hp->n_steps;
    lgt_solve_stats s;
    auto K = [&](double e) -> int {
        s = lgt_solve_stats{};
        int r = kick(L, L->mom, e, ap, phi, &hp->md_solver, &s);
        add_stats(tot, s);
        ++*evals;
        return r;
    };
    const bool dfu = df_updates(ap, &hp->md_solver);
    auto Uup = [&](double e) -> int { return update_links(L, L->mom, e, dfu); };
    if (hp->integrator == LGT_LEAPFROG) {
        TRY(K(0.5 * eps));
        for (int i = 0; i < hp->n_steps; ++i) {
            TRY(Uup(eps));
            TRY(K(i + 1 < hp->n_steps ? eps : 0.5 * eps));
        }
    } else if (hp->integrator == LGT_OMELYAN2MN) {
        // the second-order minimum-norm (2MN) position-velocity-position integrator of
        // Omelyan, Mryglod and Folk, Comput. Phys. Commun. 151 (2003) 272, Eq. (31):
        // lambda = 0.1931833275037836 minimises the norm of its leading error term
        const double lam = 0.1931833275037836;
        TRY(K(lam * eps));
        for (int i = 0; i < hp->n_steps; ++i) {
            TRY(Uup(0.5 * eps));
            TRY(K((1.0 - 2.0 * lam) * eps));
            TRY(Uup(0.5 * eps));
            TRY(K(i + 1 < hp->n_steps ? 2.0 * lam * eps : lam * eps));
        }
    } else if (hp->integrator == LGT_SEXTON_WEINGARTEN) {
        // outer leapfrog with the fermion force; each outer step runs n_inner leapfrog
        // steps of the gauge force (the cheap, stiff part) at eps / n_inner
        lgt_action_params apF = *ap, apG = *ap;
        apF.beta = 0.0;
        apG.fermions = 0;
        const int m = hp->n_inner > 0 ? hp->n_inner : 1;
        const double ein = eps / m;
        auto KP = [&](const lgt_action_params* a, double e) -> int {
            s = lgt_solve_stats{};
            int r = kick(L, L->mom, e, a, phi, &hp->md_solver, &s);
            add_stats(tot, s);
            ++*evals;
            return r;
        };
        TRY(KP(&apF, 0.5 * eps));
        for (int i = 0; i < hp->n_steps; ++i) {
            TRY(KP(&apG, 0.5 * ein));
            for (int j = 0; j < m; ++j) {
                TRY(Uup(ein));
                TRY(KP(&apG, j + 1 < m ? ein : 0.5 * ein));
            }
            TRY(KP(&apF, i + 1 < hp->n_steps ? eps : 0.5 * eps));
        }
    } else {
        return fail(LGT_EINVAL, "integrator %d", hp->integrator);
    }
    return LGT_OK;
}

extern "C" int lgt_hmc_trajectory(lgt_lattice_t L, const lgt_action_params* ap, const lgt_hmc_params* hp,
                                  uint64_t seed, uint32_t traj, lgt_hmc_result* res) {
    if (!L || !hp || !res) return fail(LGT_EINVAL, "null argument");
    NvtxRange nvtx("lgt trajectory");
    TRY(check_action(ap));
    if (hp->n_steps <= 0) return fail(LGT_EINVAL, "n_steps must be positive");
    TRY(ensure_md(L));
    TRY(ensure_solver(L));
    memset(res, 0, sizeof *res);
    const bool eo = ap->even_odd != 0;
    L->ch.n = L->ch.head = 0;   // a new pseudofermion source: earlier solutions do not apply
    CK(cudaMemcpyAsync(L->Ubak, L->thin.U, links64(L), cudaMemcpyDeviceToDevice, L->st));
    CK(gauge_momenta_heatbath(L->mom, L->g, seed, traj, L->st));
    TRY(lgt_kinetic_energy(L, (const double*)L->mom, &res->K_old));
    double ps;
    TRY(gauge_action_value(L, ap, &res->Sg_old));
    if (ap->fermions) {
        // phi = M^+ xi on the (smeared) links, S_f(old) = xi^+ xi
        CK(cudaMemsetAsync(L->xi, 0, spinor64_full(L), L->st));
        CK(spinor_gaussian(L->xi, L->g, eo ? 0 : 2, seed, traj, FIELD_XI, L->st));
        Links lk;
        TRY(fermion_links(L, ap, &lk));
        if (eo) TRY(dhat(L, lk, true, true, L->xi, L->phi, L->t, ap->kappa));
        else TRY(dfull(L, lk, true, true, L->xi, L->phi, ap->kappa));
        CK(blas_norm2(L->xi, eo ? L->g.Vh : 2 * L->g.Vh, L->g.Vh, true, red(L), 0, L->st));
        TRY(sync_scalars(L));
        res->Sf_old = L->hs->slot[0];
        if (eo && lk.C64) res->Sf_old -= 2.0 * lk.logdet_odd;
    }
    int evals = 0;
    TRY(integrate(L, ap, hp, L->phi, &res->total, &evals));
    res->force_evals = evals;
    TRY(lgt_kinetic_energy(L, (const double*)L->mom, &res->K_new));
    TRY(gauge_action_value(L, ap, &res->Sg_new));
    if (ap->fermions) {
        Links lk;
        TRY(fermion_links(L, ap, &lk));
        lgt_solve_stats s = {};
        TRY(pf_action_on(L, lk, ap, L->phi, &hp->action_solver, &res->Sf_new, &s));
        add_stats(&res->total, s);
    }
    res->dH = (res->K_new + res->Sg_new + res->Sf_new) - (res->K_old + res->Sg_old + res->Sf_old);
    if (!std::isfinite(res->dH)) return fail(LGT_ENAN, "non-finite Delta H");
    uint32_t ctr[4] = {0, 0, traj, FIELD_METROPOLIS}, o[4];
    philox_host(ctr, seed, o);
    double u = ((double)(o[0] >> 5) * 67108864.0 + (double)(o[1] >> 6) + 0.5) * (1.0 / 9007199254740992.0);
    res->accepted = u < std::exp(-res->dH);
    if (!res->accepted) {
        CK(cudaMemcpyAsync(L->thin.U, L->Ubak, links64(L), cudaMemcpyDeviceToDevice, L->st));
        L->udf_src = nullptr;
    }
    L->udf_src = nullptr;
    CK(gauge_reunitarise(L->thin.U, L->thin.U12, L->g, L->st));
    TRY(plaquette_sum(L, L->thin.U, &ps));
    res->plaquette = ps / (6.0 * L->g.V);
    return LGT_OK;
}

// ---------------------------------------------------------------- diagnostics
extern "C" int lgt_kernel_timing_start(int max_launches) {
    if (max_launches <= 0 || max_launches > (1 << 20)) return fail(LGT_EINVAL, "max_launches %d", max_launches);
    size_t need = 2 * (size_t)max_launches;
    while (g_kt.ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        g_kt.ev.push_back(e);
    }
    g_kt.kind.assign(max_launches, 0);
    g_kt.used = 0;
    g_kt.seen = 0;
    g_kt.on = true;
    return LGT_OK;
}

extern "C" int lgt_kernel_timing_sample(int every) {
    if (every < 1) return fail(LGT_EINVAL, "every = %d", every);
    g_kt.every = every;
    return LGT_OK;
}

extern "C" int lgt_kernel_timing_stop(double min_ms, double* ms, int64_t* n, int64_t* n_short) {
    g_kt.on = false;
    double acc[LGT_TIMING_KINDS] = {0};
    int64_t cnt[LGT_TIMING_KINDS] = {0}, nshort = 0;
    for (size_t k = 0; k + 1 < g_kt.used; k += 2) {
        CK(cudaEventSynchronize(g_kt.ev[k + 1]));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, g_kt.ev[k], g_kt.ev[k + 1]));
        if (t < min_ms) {   // returned at entry: its solver had already stopped
            ++nshort;
            continue;
        }
        int kind = g_kt.kind[k / 2];
        acc[kind] += t;
        cnt[kind] += 1;
    }
    g_kt.used = 0;
    for (int k = 0; k < LGT_TIMING_KINDS; ++k) {
        if (ms) ms[k] = acc[k];
        if (n) n[k] = cnt[k];
    }
    if (n_short) *n_short = nshort;
    return LGT_OK;
}

extern "C" int lgt_measure_fp64_peak(double* flops, double* seconds) {
    if (!flops) return fail(LGT_EINVAL, "null argument");
    double secs = 0;
    CK(fp64_peak_kernel_run(flops, &secs));
    if (seconds) *seconds = secs;
    return LGT_OK;
}
