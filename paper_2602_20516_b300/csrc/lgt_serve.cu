// lgt_serve.cu -- a request server for Dirac solves and force evaluations on a
// pool of resident gauge fields of different volumes, with continuous batching.
//
// Each scheduling tick (lgt_server_step):
//   1. admits queued requests in arrival order while slots and the HBM budget
//      allow, builds their right-hand sides on the device;
//   2. advances every running CG by `batch_iters` iterations with batched
//      launches: one launch per CG kernel step covers all running requests of a
//      precision (each request keeps its own geometry, fields, scalars and
//      deterministic reduction), so requests of any volume overlap on the GPU;
//   3. reads every running request's solver scalars with one copy, and for the
//      requests whose stop condition fired forms the true residual (mixed
//      requests first fold the FP32 iterate in: a reliable update), with the FP64
//      hop, or with the double-float hop for a mixed request on a gauge field
//      that has a double-float copy;
//   4. finishes converged requests (solution reconstruction or force kernels;
//      double-float forces for mixed requests with a double-float residual) and
//      releases their memory; completions carry host timestamps.
// A request's arithmetic does not depend on what else is running: results are
// the same alone and in any mix.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "../../include/lgt.h"
#include "lgt_internal.h"

using namespace lgt;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

#define SCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return set_error(LGT_ECUDA, cudaGetErrorString(e_));            \
    } while (0)
#define STRY(call)                   \
    do {                             \
        int r_ = (call);             \
        if (r_ != LGT_OK) return r_; \
    } while (0)

struct Gauge {
    Geom g;
    double2* U;
    float4* U12;
    float4* Udf = nullptr;   // double-float copy (when the budget allowed it at creation)
    size_t bytes;
};

struct Req {
    uint64_t id;
    lgt_request q;
    int slot = -1;
    bool fp64 = true;
    size_t bytes = 0;
    void* mem = nullptr;
    // FP64 half fields unless noted
    double2 *src = nullptr;   // full: b (solve) or phi on even sites (force)
    double2 *c = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *u = nullptr, *t = nullptr;
    float4 *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *u32 = nullptr, *t32 = nullptr;
    double2 *X = nullptr, *Y = nullptr;  // full, force requests
    double2* out = nullptr;              // solve: full solution; force: momenta layout
    double* partials = nullptr;
    unsigned* counter = nullptr;
    double bb = 0.0;
    int reliable = 0;
    int status = LGT_OK;
    double res = 0.0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int iters = 0;
    bool running = false;
    bool reported = false;
    // mixed requests near a nearly singular operator (as lgt_cg_solve): FP32 breakdowns
    // restart from the FP64 residual, two slow cycles in a row hand over to FP64 CG
    int breakdowns = 0, poor = 0, iters_at_update = 0;
    double rr_prev = 0.0;
    bool restart_p = false;
};

size_t half64(const Geom& g) { return (size_t)12 * g.Vh * sizeof(double2); }
size_t half32(const Geom& g) { return (size_t)6 * g.Vh * sizeof(float4); }
size_t mom_bytes(const Geom& g) { return (size_t)8 * 4 * g.Vh * sizeof(double2); }
int nblk(const Geom& g) { return (g.Vh + NT - 1) / NT; }

size_t request_bytes(const Geom& g, const lgt_request& q) {
    size_t b = 2 * half64(g) + 6 * half64(g);                     // src (full) + c x r p u t
    if (q.precision == LGT_MIXED) b += 5 * half32(g);
    b += (q.kind == LGT_REQ_FORCE) ? 4 * half64(g) + mom_bytes(g) : 2 * half64(g);
    b += sizeof(double) * (nblk(g) + 64) + 256;
    return b + 16 * 256;   // alignment slack
}

}  // namespace

struct lgt_server {
    lgt_allocator alloc;
    bool custom;
    cudaStream_t st;
    size_t budget, used = 0;
    int max_active, batch_iters;
    double delta;
    std::vector<Gauge> gauges;
    std::deque<Req*> queue;
    std::vector<Req*> active;
    std::vector<Req*> done;
    std::vector<int> free_slots;
    uint64_t next_id = 1;
    Scalars* s = nullptr;    // device, one slot per active request
    Scalars* hs = nullptr;   // pinned mirror
    BatchHop* d_hop = nullptr;   // device descriptors: [2 precisions][4 steps][max_active]
    BatchAxpy* d_axpy = nullptr; // [2][max_active]
    BatchHop* h_hop = nullptr;   // pinned staging
    BatchAxpy* h_axpy = nullptr;
    std::vector<void*> fixed;
};

namespace {

int srv_alloc(lgt_server* S, size_t bytes, void** p) {
    *p = nullptr;
    if (S->custom) *p = S->alloc.alloc(S->alloc.ctx, bytes, (void*)S->st);
    else if (cudaMalloc(p, bytes) != cudaSuccess) *p = nullptr;
    if (!*p) return set_error(LGT_ENOMEM, "server allocation failed");
    return LGT_OK;
}
void srv_free(lgt_server* S, void* p) {
    if (!p) return;
    if (S->custom) S->alloc.free(S->alloc.ctx, p, (void*)S->st);
    else cudaFree(p);
}

HopArgs req_hop(lgt_server* S, Req* R, const Gauge& G, bool fp64) {
    HopArgs a;
    memset(&a, 0, sizeof a);
    a.U = fp64 ? (const void*)G.U : (const void*)G.U12;
    a.g = G.g;
    a.s = S->s + R->slot;
    a.partials = R->partials;
    a.red_capacity = nblk(G.g) + 64;
    a.counter = R->counter;
    a.a = 1.0;
    return a;
}

// single-problem hop on a request: out_q = a H in (+ y)
int rhop(lgt_server* S, Req* R, bool fp64, bool dag, int q, const void* in, void* out, double a,
         int epi = EPI_HOP, const void* y = nullptr, const void* b = nullptr, int red_op = 0) {
    const Gauge& G = S->gauges[R->q.gauge_id];
    HopArgs A = req_hop(S, R, G, fp64);
    A.parity = q;
    A.in[1 - q] = in;
    A.out[q] = out;
    A.y[q] = y;
    A.pv[q] = b;
    A.a = a;
    A.red_op = red_op;
    SCK(launch_hop(A, fp64, dag, epi, S->st));
    return LGT_OK;
}

// res = c - Dhat^+ Dhat x with the double-float hop (a mixed request on a gauge field
// with a double-float copy), |res|^2 into the request's scalar slot 0.  A force request
// keeps the intermediate vectors X = (x_e, kappa H_oe x_e), Y = (Dhat x_e,
// kappa (H^+)_oe Dhat x_e) in double-float in its X, Y buffers (the converged
// residual's vectors feed the force); a solve request borrows its FP64 u, t, p (unused
// by the FP32 iterations) and its FP32 x, r pair, and x32 is cleared again afterwards.
int true_residual_df(lgt_server* S, Req* R) {
    const Gauge& G = S->gauges[R->q.gauge_id];
    const Geom& g = G.g;
    const long hf = 12L * g.Vh;
    const double kappa = R->q.kappa;
    float4 *xe, *Xo, *Ye, *Yo;
    if (R->q.kind == LGT_REQ_FORCE) {
        xe = (float4*)R->X; Xo = xe + hf;
        Ye = (float4*)R->Y; Yo = Ye + hf;
    } else {
        xe = (float4*)R->u; Xo = (float4*)R->t;
        Ye = (float4*)R->p; Yo = R->x32;
    }
    SCK(complex_to_df(xe, R->x, hf, S->st));
    HopArgs A;
    memset(&A, 0, sizeof A);
    A.U = G.Udf;
    A.g = g;
    A.parity = 1; A.in[0] = xe; A.out[1] = Xo; A.a = kappa;
    SCK(launch_hop_df(A, false, EPI_HOP, S->st));
    A.parity = 0; A.in[1] = Xo; A.out[0] = Ye; A.y[0] = xe; A.a = -kappa;
    SCK(launch_hop_df(A, false, EPI_XPAY, S->st));
    A.parity = 1; A.in[0] = Ye; A.out[1] = Yo; A.y[0] = nullptr; A.a = kappa;
    SCK(launch_hop_df(A, true, EPI_HOP, S->st));
    HopArgs B = req_hop(S, R, G, true);
    B.U = G.Udf;
    B.parity = 0; B.in[1] = Yo; B.y[0] = Ye; B.a = -kappa; B.out[0] = R->r; B.pv[0] = R->c;
    B.red_op = RED_STORE; B.red_slot = 0;
    SCK(launch_hop_df(B, true, EPI_RESID, S->st));
    if (R->q.kind == LGT_REQ_SOLVE) SCK(cudaMemsetAsync(R->x32, 0, half32(g), S->st));
    return LGT_OK;
}
bool df_residual(const lgt_server* S, const Req* R) { return !R->fp64 && S->gauges[R->q.gauge_id].Udf; }

// res = c - Dhat^+ Dhat x (FP64, or double-float for a mixed request on a gauge field
// with a double-float copy), |res|^2 into the request's scalar slot 0
int true_residual(lgt_server* S, Req* R) {
    if (df_residual(S, R)) return true_residual_df(S, R);
    const double k2 = R->q.kappa * R->q.kappa;
    STRY(rhop(S, R, true, false, 1, R->x, R->t, 1.0));
    STRY(rhop(S, R, true, false, 0, R->t, R->u, -k2, EPI_XPAY, R->x));
    STRY(rhop(S, R, true, true, 1, R->u, R->t, 1.0));
    STRY(rhop(S, R, true, true, 0, R->t, R->r, -k2, EPI_RESID, R->u, R->c, RED_STORE));
    return LGT_OK;
}

int admit(lgt_server* S, Req* R) {
    const Gauge& G = S->gauges[R->q.gauge_id];
    const Geom& g = G.g;
    void* mem;
    STRY(srv_alloc(S, R->bytes, &mem));
    R->mem = mem;
    S->used += R->bytes;
    char* p = (char*)mem;
    auto take = [&](size_t n) {
        void* q = p;
        p += (n + 255) & ~(size_t)255;
        return q;
    };
    R->src = (double2*)take(2 * half64(g));
    R->c = (double2*)take(half64(g));
    R->x = (double2*)take(half64(g));
    R->r = (double2*)take(half64(g));
    R->p = (double2*)take(half64(g));
    R->u = (double2*)take(half64(g));
    R->t = (double2*)take(half64(g));
    if (!R->fp64) {
        // x32 and r32 adjacent: together one double-float half field for the residual
        R->x32 = (float4*)take(2 * half32(g));
        R->r32 = R->x32 + (size_t)6 * g.Vh;
        R->p32 = (float4*)take(half32(g));
        R->u32 = (float4*)take(half32(g));
        R->t32 = (float4*)take(half32(g));
    }
    if (R->q.kind == LGT_REQ_FORCE) {
        R->X = (double2*)take(2 * half64(g));
        R->Y = (double2*)take(2 * half64(g));
        R->out = (double2*)take(mom_bytes(g));
    } else {
        R->out = (double2*)take(2 * half64(g));
    }
    R->partials = (double*)take(sizeof(double) * (nblk(g) + 64));
    R->counter = (unsigned*)take(256);
    R->slot = S->free_slots.back();
    S->free_slots.pop_back();
    SCK(cudaMemsetAsync(R->counter, 0, 256, S->st));
    const double kappa = R->q.kappa;
    const double2* b_e = R->src;
    const double2* b_o = R->src + (size_t)12 * g.Vh;
    if (R->q.kind == LGT_REQ_SOLVE) {
        // D x = b by even-odd CGNE: bhat_e = b_e + kappa H_eo b_o, c = Dhat^+ bhat_e
        SCK(spinor_gaussian(R->src, g, 2, R->q.source_seed, 0, FIELD_SOURCE, S->st));
        STRY(rhop(S, R, true, false, 0, b_o, R->u, kappa, EPI_XPAY, b_e));
        STRY(rhop(S, R, true, true, 1, R->u, R->t, 1.0));
        STRY(rhop(S, R, true, true, 0, R->t, R->c, -kappa * kappa, EPI_XPAY, R->u));
    } else {
        SCK(spinor_gaussian(R->src, g, 0, R->q.source_seed, 0, FIELD_SOURCE, S->st));
        SCK(cudaMemcpyAsync(R->c, R->src, half64(g), cudaMemcpyDeviceToDevice, S->st));
    }
    RedArgs red{S->s + R->slot, R->partials, R->counter, nblk(g) + 64};
    SCK(blas_norm2(R->c, g.Vh, g.Vh, true, red, 0, S->st));
    SCK(cudaMemsetAsync(R->x, 0, half64(g), S->st));
    SCK(cudaMemcpyAsync(R->r, R->c, half64(g), cudaMemcpyDeviceToDevice, S->st));
    if (R->fp64) {
        SCK(cudaMemcpyAsync(R->p, R->c, half64(g), cudaMemcpyDeviceToDevice, S->st));
    } else {
        SCK(blas_d2f(R->r32, R->c, g.Vh, g.Vh, S->st));
        SCK(cudaMemcpyAsync(R->p32, R->r32, half32(g), cudaMemcpyDeviceToDevice, S->st));
        SCK(cudaMemsetAsync(R->x32, 0, half32(g), S->st));
    }
    R->t_admit = now_s();
    return LGT_OK;
}

void release(lgt_server* S, Req* R) {
    if (R->mem) {
        srv_free(S, R->mem);
        S->used -= R->bytes;
        R->mem = nullptr;
    }
    if (R->slot >= 0) {
        S->free_slots.push_back(R->slot);
        R->slot = -1;
    }
}

// epilogue of a converged request
int finish(lgt_server* S, Req* R) {
    const Gauge& G = S->gauges[R->q.gauge_id];
    const Geom& g = G.g;
    const double kappa = R->q.kappa;
    if (R->q.kind == LGT_REQ_SOLVE) {
        // x_o = b_o + kappa H_oe x_e
        SCK(cudaMemcpyAsync(R->out, R->x, half64(g), cudaMemcpyDeviceToDevice, S->st));
        STRY(rhop(S, R, true, false, 1, R->x, R->out + (size_t)12 * g.Vh, kappa, EPI_XPAY,
                  R->src + (size_t)12 * g.Vh));
    } else if (df_residual(S, R)) {
        // the converged double-float residual left X, Y in double-float: the mixed
        // path's double-float forces (Lie form, FP64 accumulation)
        int keep = 0;
        if (R->q.beta != 0.0) {
            SCK(gauge_force_df(G.Udf, g, R->q.beta, 1.0, 0, R->out, S->st));
            keep = 1;
        }
        SCK(fermion_force_df(G.Udf, (const float4*)R->X, (const float4*)R->Y, g, kappa, 1.0, keep, R->out, S->st));
    } else {
        double2* Xo = R->X + (size_t)12 * g.Vh;
        double2* Yo = R->Y + (size_t)12 * g.Vh;
        SCK(cudaMemcpyAsync(R->X, R->x, half64(g), cudaMemcpyDeviceToDevice, S->st));
        STRY(rhop(S, R, true, false, 1, R->X, Xo, kappa));
        STRY(rhop(S, R, true, false, 0, Xo, R->Y, -kappa, EPI_XPAY, R->X));
        STRY(rhop(S, R, true, true, 1, R->Y, Yo, kappa));
        int keep = 0;
        if (R->q.beta != 0.0) {
            SCK(gauge_force(G.U, g, R->q.beta, 0.0, 1.0, 0, 0, R->out, S->st));
            keep = 1;
        }
        SCK(fermion_force(G.U, R->X, R->Y, g, kappa, 1.0, keep, 0, R->out, S->st));
    }
    return LGT_OK;
}

int sync_all_scalars(lgt_server* S) {
    SCK(cudaMemcpyAsync(S->hs, S->s, sizeof(Scalars) * S->max_active, cudaMemcpyDeviceToHost, S->st));
    SCK(cudaStreamSynchronize(S->st));
    return LGT_OK;
}

// K batched CG iterations over the running requests of one precision
int batch_iterations(lgt_server* S, bool fp64, int K) {
    const int grp = fp64 ? 1 : 0;
    BatchHop* h = S->h_hop + (size_t)grp * 4 * S->max_active;
    BatchAxpy* ha = S->h_axpy + (size_t)grp * S->max_active;
    int n = 0, total = 0, total_p = 0;
    for (Req* R : S->active) {
        if (!R->running || R->fp64 != fp64) continue;
        const Gauge& G = S->gauges[R->q.gauge_id];
        const int nb = nblk(G.g);
        const double k2 = R->q.kappa * R->q.kappa;
        void *x = fp64 ? (void*)R->x : (void*)R->x32, *r = fp64 ? (void*)R->r : (void*)R->r32;
        void *p = fp64 ? (void*)R->p : (void*)R->p32, *u = fp64 ? (void*)R->u : (void*)R->u32;
        void* t = fp64 ? (void*)R->t : (void*)R->t32;
        HopArgs a = req_hop(S, R, G, fp64);
        a.skip = 1;
        HopArgs s1 = a;
        s1.parity = 1; s1.in[0] = p; s1.out[1] = t;
        HopArgs s2 = a;
        s2.parity = 0; s2.in[1] = t; s2.out[0] = u; s2.y[0] = p; s2.a = -k2; s2.red_op = RED_PAP;
        HopArgs s3 = a;
        s3.parity = 1; s3.in[0] = u; s3.out[1] = t;
        HopArgs s4 = a;
        s4.parity = 0; s4.in[1] = t; s4.y[0] = u; s4.a = -k2; s4.red_op = RED_RR;
        s4.r[0] = r;
        h[0 * S->max_active + n] = BatchHop{s1, total, nb};
        h[1 * S->max_active + n] = BatchHop{s2, total, nb};
        h[2 * S->max_active + n] = BatchHop{s3, total, nb};
        h[3 * S->max_active + n] = BatchHop{s4, total, nb};
        const long ne = (long)G.g.Vh * (fp64 ? 12 : 6);
        const int nbp = (int)((ne + NT - 1) / NT);
        ha[n] = BatchAxpy{p, r, x, ne, RedArgs{S->s + R->slot, R->partials, R->counter, nblk(G.g) + 64}, total_p, nbp};
        total += nb;
        total_p += nbp;
        ++n;
    }
    if (n == 0) return LGT_OK;
    BatchHop* d = S->d_hop + (size_t)grp * 4 * S->max_active;
    BatchAxpy* da = S->d_axpy + (size_t)grp * S->max_active;
    SCK(cudaMemcpyAsync(d, h, sizeof(BatchHop) * 4 * S->max_active, cudaMemcpyHostToDevice, S->st));
    SCK(cudaMemcpyAsync(da, ha, sizeof(BatchAxpy) * S->max_active, cudaMemcpyHostToDevice, S->st));
    for (int k = 0; k < K; ++k) {
        SCK(launch_hop_batch(d + 0 * S->max_active, n, total, fp64, false, EPI_HOP, S->st));
        SCK(launch_hop_batch(d + 1 * S->max_active, n, total, fp64, false, EPI_XPAY_NORM, S->st));
        SCK(launch_hop_batch(d + 2 * S->max_active, n, total, fp64, true, EPI_HOP, S->st));
        SCK(launch_hop_batch(d + 3 * S->max_active, n, total, fp64, true, EPI_CG, S->st));
        SCK(launch_p_update_batch(da, n, total_p, fp64, S->st));
    }
    return LGT_OK;
}

}  // namespace

extern "C" int lgt_server_create(const lgt_allocator* alloc, size_t hbm_budget_bytes, int max_active,
                                 int batch_iters, double delta, void* stream, lgt_server_t* out) {
    if (!out || max_active <= 0 || max_active > 1024 || batch_iters <= 0)
        return set_error(LGT_EINVAL, "bad server arguments");
    if (alloc && (!alloc->alloc || !alloc->free)) return set_error(LGT_EINVAL, "allocator without alloc/free");
    *out = nullptr;
    lgt_server* S = new lgt_server();
    S->custom = alloc != nullptr;
    if (alloc) S->alloc = *alloc;
    S->st = (cudaStream_t)stream;
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    S->batch_iters = batch_iters;
    S->delta = delta > 0 ? delta : 1e-3;
    for (int k = max_active - 1; k >= 0; --k) S->free_slots.push_back(k);
    void* p;
    int rc;
    if ((rc = srv_alloc(S, sizeof(Scalars) * max_active, &p))) { lgt_server_destroy(S); return rc; }
    S->s = (Scalars*)p;
    S->fixed.push_back(p);
    if ((rc = srv_alloc(S, sizeof(BatchHop) * 8 * max_active, &p))) { lgt_server_destroy(S); return rc; }
    S->d_hop = (BatchHop*)p;
    S->fixed.push_back(p);
    if ((rc = srv_alloc(S, sizeof(BatchAxpy) * 2 * max_active, &p))) { lgt_server_destroy(S); return rc; }
    S->d_axpy = (BatchAxpy*)p;
    S->fixed.push_back(p);
    if (cudaMallocHost((void**)&S->hs, sizeof(Scalars) * max_active) != cudaSuccess ||
        cudaMallocHost((void**)&S->h_hop, sizeof(BatchHop) * 8 * max_active) != cudaSuccess ||
        cudaMallocHost((void**)&S->h_axpy, sizeof(BatchAxpy) * 2 * max_active) != cudaSuccess) {
        lgt_server_destroy(S);
        return set_error(LGT_ENOMEM, "pinned host allocation failed");
    }
    memset(S->hs, 0, sizeof(Scalars) * max_active);
    memset(S->h_hop, 0, sizeof(BatchHop) * 8 * max_active);
    memset(S->h_axpy, 0, sizeof(BatchAxpy) * 2 * max_active);
    if (cudaMemsetAsync(S->s, 0, sizeof(Scalars) * max_active, S->st) != cudaSuccess) {
        lgt_server_destroy(S);
        return set_error(LGT_ECUDA, "server initialisation failed");
    }
    *out = S;
    return LGT_OK;
}

extern "C" int lgt_server_destroy(lgt_server_t S) {
    if (!S) return LGT_OK;
    cudaStreamSynchronize(S->st);
    for (Req* R : S->queue) { release(S, R); delete R; }
    for (Req* R : S->active) { release(S, R); delete R; }
    for (Req* R : S->done) { release(S, R); delete R; }
    for (Gauge& G : S->gauges) {
        srv_free(S, G.U);
        srv_free(S, G.U12);
        srv_free(S, G.Udf);
    }
    for (void* p : S->fixed) srv_free(S, p);
    if (S->hs) cudaFreeHost(S->hs);
    if (S->h_hop) cudaFreeHost(S->h_hop);
    if (S->h_axpy) cudaFreeHost(S->h_axpy);
    delete S;
    return LGT_OK;
}

extern "C" int lgt_server_add_gauge(lgt_server_t S, const int dims[4], uint64_t seed, double alpha, int* gauge_id) {
    if (!S || !dims || !gauge_id) return set_error(LGT_EINVAL, "null argument");
    Gauge G;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2) return set_error(LGT_EINVAL, "every extent must be even and >= 2");
        G.g.L[m] = dims[m];
        V *= dims[m];
    }
    G.g.V = (int)V;
    G.g.Vh = (int)(V / 2);
    G.g.stride[0] = 1;
    G.g.stride[1] = dims[0];
    G.g.stride[2] = dims[0] * dims[1];
    G.g.stride[3] = dims[0] * dims[1] * dims[2];
    size_t b64 = (size_t)8 * 9 * G.g.Vh * sizeof(double2), b12 = (size_t)8 * 3 * G.g.Vh * sizeof(float4);
    if (S->used + b64 + b12 > S->budget) return set_error(LGT_ENOMEM, "gauge field exceeds the HBM budget");
    void *a, *b;
    STRY(srv_alloc(S, b64, &a));
    if (srv_alloc(S, b12, &b) != LGT_OK) {
        srv_free(S, a);
        return LGT_ENOMEM;
    }
    G.U = (double2*)a;
    G.U12 = (float4*)b;
    G.bytes = b64 + b12;
    // the double-float copy for the mixed requests' residuals and forces, when the
    // gauge fields with their copies stay within half the budget (the other half is
    // left to requests); decided once per field, so a request's arithmetic never
    // depends on the other requests
    void* c = nullptr;
    if (S->used + G.bytes + b64 <= S->budget / 2 && srv_alloc(S, b64, &c) == LGT_OK) {
        G.Udf = (float4*)c;
        G.bytes += b64;
    }
    S->used += G.bytes;
    SCK(gauge_random(G.U, G.U12, G.g, seed, alpha, S->st));
    if (G.Udf) SCK(links_to_df(G.Udf, G.U, G.g, S->st));
    SCK(cudaStreamSynchronize(S->st));
    S->gauges.push_back(G);
    *gauge_id = (int)S->gauges.size() - 1;
    return LGT_OK;
}

extern "C" int lgt_server_get_links(lgt_server_t S, int gauge_id, double* links_canonical) {
    if (!S || !links_canonical || gauge_id < 0 || gauge_id >= (int)S->gauges.size())
        return set_error(LGT_EINVAL, "bad argument");
    SCK(gauge_unpack_links(links_canonical, S->gauges[gauge_id].U, S->gauges[gauge_id].g, S->st));
    SCK(cudaStreamSynchronize(S->st));
    return LGT_OK;
}

extern "C" int lgt_server_submit(lgt_server_t S, const lgt_request* q, uint64_t* id) {
    if (!S || !q || !id) return set_error(LGT_EINVAL, "null argument");
    if (q->gauge_id < 0 || q->gauge_id >= (int)S->gauges.size()) return set_error(LGT_EINVAL, "unknown gauge_id");
    if (q->kind != LGT_REQ_SOLVE && q->kind != LGT_REQ_FORCE) return set_error(LGT_EINVAL, "unknown request kind");
    if (q->precision != LGT_FP64 && q->precision != LGT_MIXED) return set_error(LGT_EINVAL, "precision");
    if (!(q->tol > 0) || q->max_iter <= 0) return set_error(LGT_EINVAL, "tol and max_iter must be positive");
    Req* R = new Req();
    R->id = S->next_id++;
    R->q = *q;
    R->fp64 = q->precision == LGT_FP64;
    R->bytes = request_bytes(S->gauges[q->gauge_id].g, *q);
    R->t_submit = now_s();
    S->queue.push_back(R);
    *id = R->id;
    return LGT_OK;
}

extern "C" int lgt_server_step(lgt_server_t S, int* n_active, int* n_queued) {
    if (!S) return set_error(LGT_EINVAL, "null server");
    NvtxRange nvtx("lgt server step");
    // 1. admission (arrival order; a request that cannot fit even alone is refused)
    std::vector<Req*> admitted;
    while (!S->queue.empty() && (int)S->active.size() < S->max_active) {
        Req* R = S->queue.front();
        size_t gauge_bytes = 0;
        for (const Gauge& G : S->gauges) gauge_bytes += G.bytes;
        if (R->bytes + gauge_bytes > S->budget) {
            S->queue.pop_front();
            R->status = LGT_ENOMEM;
            R->t_admit = R->t_done = now_s();
            S->done.push_back(R);
            continue;
        }
        if (S->used + R->bytes > S->budget) break;
        S->queue.pop_front();
        int rc = admit(S, R);
        if (rc != LGT_OK) {
            release(S, R);
            R->status = rc;
            R->t_done = now_s();
            S->done.push_back(R);
            continue;
        }
        S->active.push_back(R);
        admitted.push_back(R);
    }
    if (!admitted.empty()) {
        STRY(sync_all_scalars(S));
        for (Req* R : admitted) {
            Scalars& h = S->hs[R->slot];
            R->bb = h.slot[0];
            R->rr_prev = R->bb;
            memset(&h, 0, sizeof(Scalars));
            h.rr = R->bb;
            h.rr_max = R->bb;
            h.target = R->q.tol * R->q.tol * R->bb;
            h.delta2 = R->fp64 ? 0.0 : S->delta * S->delta;
            h.done = (R->bb == 0.0) ? 2 : 0;
            SCK(cudaMemcpyAsync(S->s + R->slot, &h, sizeof(Scalars), cudaMemcpyHostToDevice, S->st));
            R->running = true;
        }
    }
    // 2. batched CG iterations
    STRY(batch_iterations(S, false, S->batch_iters));
    STRY(batch_iterations(S, true, S->batch_iters));
    // 3. stop conditions -> true residuals (reliable updates for mixed requests)
    STRY(sync_all_scalars(S));
    std::vector<Req*> check;
    // an FP32 cycle this long without its stop test firing is ended by a reliable
    // update as well
    constexpr int kMaxCycle = 1000;
    for (Req* R : S->active) {
        if (!R->running) continue;
        Scalars& h = S->hs[R->slot];
        // a diverged FP32 cycle (|r|^2 of the recursion 1e3 above the true residual it
        // started from): its correction is dropped and it restarts from that residual
        if (!R->fp64 && !h.nan && h.rr_max > 1e3 * R->rr_prev) {
            if (++R->breakdowns > 16) {
                R->status = LGT_ENAN;
                R->running = false;
                continue;
            }
            const Geom& g = S->gauges[R->q.gauge_id].g;
            R->iters_at_update = h.iters;
            SCK(cudaMemsetAsync(R->x32, 0, half32(g), S->st));
            SCK(blas_d2f(R->r32, R->r, g.Vh, g.Vh, S->st));
            SCK(cudaMemcpyAsync(R->p32, R->r32, half32(g), cudaMemcpyDeviceToDevice, S->st));
            h.rr = R->rr_prev;
            h.rr_max = R->rr_prev;
            h.done = 0;
            SCK(cudaMemcpyAsync(S->s + R->slot, &h, sizeof(Scalars), cudaMemcpyHostToDevice, S->st));
            continue;
        }
        const bool breakdown = h.nan != 0;
        if (breakdown && (R->fp64 || ++R->breakdowns > 16)) {
            R->status = LGT_ENAN;
            R->running = false;
            continue;
        }
        const bool long_cycle = !R->fp64 && h.iters - R->iters_at_update >= kMaxCycle;
        if (h.done >= 1 || h.iters >= R->q.max_iter || breakdown || long_cycle) {
            const Geom& g = S->gauges[R->q.gauge_id].g;
            if (!R->fp64) {
                SCK(blas_add_f2d(R->x, R->x32, g.Vh, g.Vh, S->st));
                SCK(cudaMemsetAsync(R->x32, 0, half32(g), S->st));
            }
            STRY(true_residual(S, R));
            R->restart_p = breakdown;
            check.push_back(R);
        }
    }
    std::vector<Req*> finished;
    if (!check.empty()) {
        STRY(sync_all_scalars(S));
        for (Req* R : check) {
            Scalars& h = S->hs[R->slot];
            const double rr = h.slot[0];
            R->reliable += 1;
            R->iters = h.iters;
            R->res = std::sqrt(rr / R->bb);
            if (!std::isfinite(rr)) {
                R->status = LGT_ENAN;
                R->running = false;
            } else if (rr <= h.target) {
                R->running = false;
                finished.push_back(R);
            } else if (h.iters >= R->q.max_iter) {
                R->status = LGT_ENOCONV;
                R->running = false;
            } else {
                const Geom& g = S->gauges[R->q.gauge_id].g;
                if (!R->fp64) {
                    // |r| shrank by less than 2x since the last update, twice in a row:
                    // the FP32 iterations stopped making progress, FP64 CG from here
                    const bool slow = rr > 0.25 * R->rr_prev;
                    R->poor = slow ? R->poor + 1 : 0;
                    if (R->poor >= 2) {
                        R->fp64 = true;
                        SCK(cudaMemcpyAsync(R->p, R->r, half64(g), cudaMemcpyDeviceToDevice, S->st));
                    }
                }
                R->rr_prev = rr;
                R->iters_at_update = h.iters;
                if (!R->fp64) {
                    SCK(blas_d2f(R->r32, R->r, g.Vh, g.Vh, S->st));
                    if (R->restart_p) SCK(cudaMemcpyAsync(R->p32, R->r32, half32(g), cudaMemcpyDeviceToDevice, S->st));
                }
                h.rr = rr;
                h.rr_max = rr;
                h.done = 0;
                h.nan = 0;
                h.delta2 = R->fp64 ? 0.0 : S->delta * S->delta;
                SCK(cudaMemcpyAsync(S->s + R->slot, &h, sizeof(Scalars), cudaMemcpyHostToDevice, S->st));
            }
        }
    }
    // 4. epilogues and retirement
    for (Req* R : finished) STRY(finish(S, R));
    bool any_retired = false;
    for (Req* R : S->active)
        if (!R->running) any_retired = true;
    if (any_retired) {
        SCK(cudaStreamSynchronize(S->st));
        const double t = now_s();
        std::vector<Req*> still;
        for (Req* R : S->active) {
            if (R->running) {
                still.push_back(R);
                continue;
            }
            R->t_done = t;
            if (R->slot >= 0) {
                S->free_slots.push_back(R->slot);
                R->slot = -1;
            }
            // a successful request's result is kept until fetched when asked for
            if (R->status != LGT_OK || !R->q.keep_result) release(S, R);
            S->done.push_back(R);
        }
        S->active.swap(still);
    }
    if (n_active) *n_active = (int)S->active.size();
    if (n_queued) *n_queued = (int)S->queue.size();
    return LGT_OK;
}

extern "C" int lgt_server_poll(lgt_server_t S, lgt_completion* out, int max, int* n) {
    if (!S || !n || (max > 0 && !out)) return set_error(LGT_EINVAL, "null argument");
    int k = 0;
    std::vector<Req*> keep;
    for (Req* R : S->done) {
        if (R->reported || k >= max) {   // reported earlier (result pending) or no room
            keep.push_back(R);
            continue;
        }
        lgt_completion& c = out[k++];
        c.id = R->id;
        c.status = R->status;
        c.iters = R->iters;
        c.reliable_updates = R->reliable;
        c.true_rel_residual = R->res;
        c.t_submit = R->t_submit;
        c.t_admit = R->t_admit;
        c.t_done = R->t_done;
        if (R->mem) {   // result kept for lgt_server_result
            R->reported = true;
            keep.push_back(R);
        } else {
            delete R;
        }
    }
    S->done.swap(keep);
    *n = k;
    return LGT_OK;
}

extern "C" int lgt_server_result(lgt_server_t S, uint64_t id, double* out_dev, size_t bytes) {
    if (!S) return set_error(LGT_EINVAL, "null server");
    for (size_t k = 0; k < S->done.size(); ++k) {
        Req* R = S->done[k];
        if (R->id != id) continue;
        if (!R->mem) return set_error(LGT_EINVAL, "request has no kept result");
        const Geom& g = S->gauges[R->q.gauge_id].g;
        size_t need = (R->q.kind == LGT_REQ_FORCE) ? mom_bytes(g) : 2 * half64(g);
        if (out_dev) {
            if (bytes < need) return set_error(LGT_EINVAL, "output buffer too small");
            SCK(cudaMemcpyAsync(out_dev, R->out, need, cudaMemcpyDeviceToDevice, S->st));
            SCK(cudaStreamSynchronize(S->st));
        }
        release(S, R);
        if (R->reported) {   // poll has already returned its completion
            delete R;
            S->done.erase(S->done.begin() + k);
        }
        return LGT_OK;
    }
    return set_error(LGT_EINVAL, "unknown or already released request id");
}

extern "C" int lgt_server_info(lgt_server_t S, size_t* used_bytes, size_t* budget_bytes, int* n_active,
                               int* n_queued) {
    if (!S) return set_error(LGT_EINVAL, "null server");
    if (used_bytes) *used_bytes = S->used;
    if (budget_bytes) *budget_bytes = S->budget;
    if (n_active) *n_active = (int)S->active.size();
    if (n_queued) *n_queued = (int)S->queue.size();
    return LGT_OK;
}

extern "C" double lgt_clock(void) { return now_s(); }
