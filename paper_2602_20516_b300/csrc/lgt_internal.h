// lgt_internal.h -- declarations shared by the liblgt translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lgt_common.cuh"
#include <nvtx3/nvToolsExt.h>

namespace lgt {

// NVTX range for the duration of a scope (a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

enum Epilogue { EPI_HOP = 0, EPI_XPAY = 1, EPI_XPAY_NORM = 2, EPI_CG = 3, EPI_RESID = 4 };

// Arguments of one hopping-term launch.  Field pointers are half fields indexed
// by parity (double2 [12][Vh] for FP64, float4 [6][Vh] for FP32); the input of
// output parity p is in[1-p].  parity = 0, 1 or 2 (both parities in one launch).
struct HopArgs {
    const void* U;        // FP64 links (double2) or FP32 two-row links (float4)
    const void* in[2];
    void* out[2];
    const void* y[2];     // xpay addend (same parity as the output)
    void* r[2];           // EPI_CG: residual
    const void* pv[2];    // EPI_RESID: right-hand side
    double a;             // coefficient of H in
    Geom g;
    int parity;
    Scalars* s;           // solver scalars (nullptr: no skip test, no reduction)
    double* partials;
    unsigned* counter;
    int red_op, red_slot;
    int skip;             // 1: return at once when the solver scalars say done
    int red_capacity;     // entries of partials (reducing epilogues need one per block)
    int reverse;          // 1: block b works on site block nblk - 1 - b (same results)
    // Deferred reduction: with defer set, a reducing epilogue only stores its block
    // partials (no per-block fence and atomic); a later hop launch with fin_n > 0 has
    // its block 0 sum those fin_n partials (the same fixed order as the last block of a
    // reducing launch) and apply fin_op to the scalars before its own work.  For an
    // epilogue whose result the next launch does not read (<p, A p> before the hop of
    // Dhat^+).
    int defer;
    int fin_n, fin_op;
    // Even-odd clover operator fused into the hop (Hermitian-packed block field of the
    // output parity: FP32 [parity][18][Vh] for the FP32 hop, lgt_clover.cuh; double-float
    // [parity][36][Vh] for the double-float hop): EPI_HOP stores clov(p) a H in (the
    // inverse block of the output site, M_oo^{-1}); EPI_XPAY_NORM, EPI_CG and (double-
    // float) EPI_XPAY, EPI_RESID take y -> clov(p) y (M_ee y) before adding a H in.
    // nullptr: no clover term.
    const void* clov;
    // FP32 one-parity hops on a lattice whose half-rows tile the block (hop_stage_hr):
    // bit 0 stages the block's links, bit 1 its input spinors and their neighbour halos
    // in shared memory by bulk copies before the arithmetic (same results); 0 reads
    // every operand through L1/L2.
    int stage;
};

cudaError_t launch_hop(const HopArgs& A, bool fp64, bool dagger, int epi, cudaStream_t st);
int hop_grid(const Geom& g, int parity);
// half-row length L0 / 2 when the staged FP32 hop applies to this geometry (whole
// half-rows tile a block and the rows of a block tile an x-y plane), else 0
int hop_stage_hr(const Geom& g);
// blocks of the staged hop whose wait for their bulk copies gave up (they stored NaN)
unsigned hop_stage_timeouts();

// Several right-hand sides (1..KMAX_RHS, every slot a valid system) on the same FP32
// links and output parity in one launch: each link is loaded once per site and
// direction for all of them.  System k is masked (skip = 1) once its scalars say
// done; its epilogue and its reduction (own scalars, partials and counter) are
// those of the single-system hop.
constexpr int KMAX_RHS = 4;
struct HopArgsM {
    const void* U;
    Geom g;
    int parity;           // output parity, 0 or 1
    int nrhs;
    int skip;
    int red_op;
    int red_capacity;
    const void* in[KMAX_RHS];   // half fields of parity 1 - parity
    void* out[KMAX_RHS];
    const void* y[KMAX_RHS];
    void* r[KMAX_RHS];
    double a[KMAX_RHS];
    Scalars* s[KMAX_RHS];
    double* partials[KMAX_RHS];
    unsigned* counter[KMAX_RHS];
    int defer;            // as HopArgs: the reducing epilogue only stores block partials,
    int fin_n, fin_op;    // block 0 of a later launch sums fin_n of them per system
};
cudaError_t launch_hop_multi(const HopArgsM& A, bool fp64, bool dagger, int epi, cudaStream_t st);

// One entry of a batched launch: the hop arguments of one problem and its block
// range [first, first + nblk) in the combined grid (entries sorted by first).
struct BatchHop {
    HopArgs a;
    int first, nblk;
};
cudaError_t launch_hop_batch(const BatchHop* d_desc, int n, int total_blocks, bool fp64, bool dagger, int epi,
                             cudaStream_t st);

// launch counting (per host thread)
void count_launch();
// record the thread-local message returned by lgt_last_error(); returns code
int set_error(int code, const char* msg);
// CUDA-event timing of hop launches (kind 0 FP32, 1 FP64): returns true and an
// event pair to record around the launch while timing is on and slots remain
bool kernel_timing_slot(int kind, cudaEvent_t* start, cudaEvent_t* stop);

// ---------------------------------------------------------------- BLAS (lgt_blas.cu)
struct RedArgs {
    Scalars* s;
    double* partials;
    unsigned* counter;
    int capacity;   // entries of partials: a reducing launch with more blocks is refused
};
// all operate on n "rows" = sites; FP64 rows are 12 double2, FP32 rows 6 float4
cudaError_t blas_zero(void* f, size_t bytes, cudaStream_t st);
// |a|^2 (FP64 accumulate) -> slot
cudaError_t blas_norm2(const void* a, int n, int Vh, bool fp64, const RedArgs& R, int slot, cudaStream_t st);
// Re <a, b> -> slot   (FP64 fields)
cudaError_t blas_redot(const double2* a, const double2* b, int n, int Vh, const RedArgs& R, int slot, cudaStream_t st);
// x += alpha p, then p = r + beta p  (alpha, beta from scalars), skipped once
// done >= 2; marks done 1 -> 2.  n == Vh (one half field): a thread per site, and
// reverse walks the site blocks from the end
cudaError_t blas_cg_p_update(void* p, const void* r, void* x, int n, int Vh, bool fp64, const RedArgs& R,
                             cudaStream_t st, bool reverse = false);
// the same for many problems in one launch (each with its own scalars and counter)
struct BatchAxpy {
    void* p;
    const void* r;
    void* x;
    long ne;         // elements (double2 for FP64, float4 for FP32)
    RedArgs red;
    int first, nblk;
};
cudaError_t launch_p_update_batch(const BatchAxpy* d_desc, int n, int total_blocks, bool fp64, cudaStream_t st);
// x_k += alpha_k p_k, p_k = r_k + beta_k p_k for nrhs systems of n sites each (one
// launch, blockIdx.y = k), each with its own scalars and counter, as blas_cg_p_update
struct PUpdateM {
    void* p[KMAX_RHS];
    const void* r[KMAX_RHS];
    void* x[KMAX_RHS];
    RedArgs red[KMAX_RHS];
    int nrhs;
};
cudaError_t blas_cg_p_update_multi(const PUpdateM& P, int n, bool fp64, cudaStream_t st);
// y = x (FP64 -> FP32 rounding) / y64 += x32 / y = x
cudaError_t blas_d2f(float4* y, const double2* x, int n, int Vh, cudaStream_t st);
cudaError_t blas_add_f2d(double2* y, const float4* x, int n, int Vh, cudaStream_t st);
cudaError_t blas_f2d(double2* y, const float4* x, int n, int Vh, cudaStream_t st);
// y = a x + b y  (FP64)
cudaError_t blas_axpby(double2* y, const double2* x, double a, double b, int n, int Vh, cudaStream_t st);
// S_f = 2 Re<phi, chi> - |eta|^2 pieces: slot0 = Re<phi,chi>, slot1 = |eta|^2 (single kernel)
cudaError_t blas_action_parts(const double2* phi, const double2* chi, const double2* eta, int n, int Vh,
                              const RedArgs& R, cudaStream_t st);

// ---------------------------------------------------------------- gauge (lgt_gauge.cu)
cudaError_t gauge_pack_links(double2* U, float4* U12, const double2* canon, const Geom& g, cudaStream_t st);
cudaError_t gauge_unpack_links(double* canon, const double2* U, const Geom& g, cudaStream_t st);
cudaError_t gauge_pack_field(double2* F, const double2* canon, const Geom& g, cudaStream_t st);
cudaError_t gauge_unpack_field(double* canon, const double2* F, const Geom& g, cudaStream_t st);
cudaError_t gauge_unit(double2* U, float4* U12, const Geom& g, cudaStream_t st);
cudaError_t gauge_random(double2* U, float4* U12, const Geom& g, uint64_t seed, double alpha, cudaStream_t st);
cudaError_t gauge_make12(float4* U12, const double2* U, const Geom& g, cudaStream_t st);
cudaError_t gauge_reunitarise(double2* U, float4* U12, const Geom& g, cudaStream_t st);
cudaError_t gauge_plaquette(const double2* U, const Geom& g, const RedArgs& R, int slot, cudaStream_t st);
// mom (or F) update from the gauge force: F_G -> out = keep*out + coef*F (Lie or G form);
// c1 = rectangle weight of the improved action (0: Wilson plaquette action)
cudaError_t gauge_force(const double2* U, const Geom& g, double beta, double c1, double coef, int keep, int form,
                        double2* out, cudaStream_t st);
// Lie-form gauge force with FP32 staple arithmetic on the two-row links,
// accumulated into FP64 (the mixed-precision MD path)
cudaError_t gauge_force_fp32(const float4* U12, const Geom& g, double beta, double c1, double coef, int keep,
                             double2* out, cudaStream_t st);
// sum_{x, mu != nu} Re tr R_munu(x) / 3 (2 x 1 rectangles) -> slot
cudaError_t gauge_rectangles(const double2* U, const Geom& g, const RedArgs& R, int slot, cudaStream_t st);
// U <- exp(i eps P) U, refresh FP32 copy
cudaError_t gauge_update_links(double2* U, float4* U12, const double2* mom, double eps, const Geom& g,
                               cudaStream_t st);
cudaError_t gauge_momenta_heatbath(double2* mom, const Geom& g, uint64_t seed, uint32_t traj, cudaStream_t st);
cudaError_t gauge_kinetic(const double2* mom, const Geom& g, const RedArgs& R, int slot, cudaStream_t st);
cudaError_t gauge_kick(double2* mom, const double2* F, double eps, const Geom& g, cudaStream_t st);
cudaError_t spinor_gaussian(double2* f, const Geom& g, int parity, uint64_t seed, uint32_t traj, uint32_t field,
                            cudaStream_t st);
cudaError_t spinor_pack(void* field, const double2* canon, const Geom& g, int parity, bool fp64, cudaStream_t st);
cudaError_t spinor_unpack(double2* canon, const void* field, const Geom& g, int parity, bool fp64, cudaStream_t st);
cudaError_t mom_pack(double2* mom, const double* canon, const Geom& g, cudaStream_t st);
cudaError_t mom_unpack(double* canon, const double2* mom, const Geom& g, cudaStream_t st);
// Lie components of a G-form field: F_a = Re tr(G^+ i T^a U)
cudaError_t grad_to_lie(double2* F, const double2* G, const double2* U, const Geom& g, cudaStream_t st);

// ---------------------------------------------------------------- fermion force (lgt_force.cu)
// X, Y: full FP64 fields [2][12][Vh].  form 0: out = keep*out + coef*F (Lie, momentum
// layout);  form 1: out = keep*out + coef*G (G-form layout).
cudaError_t fermion_force(const double2* U, const double2* X, const double2* Y, const Geom& g, double kappa,
                          double coef, int keep, int form, double2* out, cudaStream_t st);
// Lie form with FP32 arithmetic: X, Y float4 [2][6][Vh], two-row FP32 links; FP64 output
cudaError_t fermion_force_fp32(const float4* U12, const float4* X, const float4* Y, const Geom& g, double kappa,
                               double coef, int keep, double2* out, cudaStream_t st);

// ---------------------------------------------------------------- chronological guess (lgt_chrono.cu)
constexpr int CHRONO_MAX = KMAX_RHS;               // solutions kept
constexpr int CDOT_MAX = CHRONO_MAX * CHRONO_MAX;  // inner products per launch
// out[m] = <a_m, b_m> (complex, conj(a) b) over even-odd half fields of Vh sites:
// a_m FP64 (double2 [12][Vh]), b_m FP64 or FP32 (float4 [6][Vh]); m < M <= CDOT_MAX.
struct CdotArgs {
    const void* a[CDOT_MAX];
    const void* b[CDOT_MAX];
    double2* out;        // [M]
    double2* partials;   // [M][blocks]
    unsigned* counter;   // [M], zero between launches
    int Vh;
    long capacity;       // double2 entries of partials
};
cudaError_t cdot_many(const CdotArgs& D, int M, bool b_fp32, cudaStream_t st);
// G c = g for the N x N Hermitian G (row-major), dependent vectors dropped (c = 0)
cudaError_t chrono_solve(const double2* G, const double2* g, double2* c, int N, int* used, cudaStream_t st);
// x = sum_i c_i v_i (FP64 half fields)
cudaError_t chrono_combine(double2* x, const double2* const* v, const double2* c, int N, int Vh, cudaStream_t st);


// ---------------------------------------------------------------- double-float forces (lgt_force_df.cu)
// FP64 links / full spinor field -> double-float copies (float4 per complex entry)
cudaError_t links_to_df(float4* Udf, const double2* U, const Geom& g, cudaStream_t st);
// U <- exp(i eps P) U in double-float arithmetic from the double-float copy Udf of U;
// writes U (FP64), U12 and Udf
cudaError_t update_links_df(float4* Udf, double2* U, float4* U12, const double2* mom, double eps, const Geom& g,
                            cudaStream_t st);
// Wilson hop in double-float arithmetic (lgt_dirac_df.cu): U double-float links, in / y
// double-float half fields; epilogues EPI_HOP, EPI_XPAY (double-float out) and
// EPI_RESID (pv and out FP64, |out|^2 reduced like the FP64 hop's)
cudaError_t launch_hop_df(const HopArgs& A, bool dagger, int epi, cudaStream_t st);
// HopArgs.clov for launch_hop_df: the Hermitian-packed double-float copy float4
// [parity][36][Vh] of a clover block field's parity (from its FP64 field)
cudaError_t clover_pack_df(const double2* C64, const Geom& g, int parity, float4* Cdf, cudaStream_t st);
// ne complex entries FP64 <-> double-float
cudaError_t complex_to_df(float4* y, const double2* x, long ne, cudaStream_t st);
cudaError_t complex_from_df(double2* y, const float4* x, long ne, cudaStream_t st);
cudaError_t spinor_to_df(float4* y, const double2* x, const Geom& g, cudaStream_t st);
// Lie form, out = keep*out + coef*F, double-float arithmetic, FP64 accumulation
cudaError_t gauge_force_df(const float4* Udf, const Geom& g, double beta, double coef, int keep, double2* out,
                           cudaStream_t st);
cudaError_t fermion_force_df(const float4* Udf, const float4* Xdf, const float4* Ydf, const Geom& g, double kappa,
                             double coef, int keep, double2* out, cudaStream_t st);

// ---------------------------------------------------------------- clover term (lgt_clover.cu)
// sigma_munu = (i/2)[g_mu, g_nu] restricted to the chiral blocks: s[plane][block][row][col]
// (planes (0,1) (0,2) (0,3) (1,2) (1,3) (2,3); block 0 = spins 0,1, block 1 = spins 2,3)
struct CloverSigma {
    double2 s[6][2][2][2];
};
// 1 + A, A = -kappa c_sw sum sigma F, from the FP64 links: C64 double2 [parity][72][Vh],
// C32 float4 [parity][36][Vh]
cudaError_t clover_field(const double2* U, const Geom& g, const CloverSigma& S, double kappa, double csw,
                         double2* C64, float4* C32, cudaStream_t st);
// the same field with the leaves in double-float arithmetic on the double-float links;
// Fscratch: double2 [2][54][Vh] for the field strengths of the six planes
cudaError_t clover_field_df(const float4* Udf, const Geom& g, const CloverSigma& S, double kappa, double csw,
                            double2* Fscratch, double2* C64, float4* C32, cudaStream_t st);
// out = (1 + A) in on parity 0 / 1 (half fields) or 2 (full fields)
cudaError_t clover_apply(const void* C, const void* in, void* out, const Geom& g, int parity, bool fp64,
                         cudaStream_t st);
// insertion M = -i kappa c_sw (Lambda + Lambda^+)/4 per site and plane from full X, Y
cudaError_t clover_insertion(const double2* X, const double2* Y, const Geom& g, const CloverSigma& S, double kappa,
                             double csw, double2* M, cudaStream_t st);
// clover part of the force: form 0 Lie (out = keep*out + coef*F), form 1 G form
// (1 + A)^{-1} on the sites of `parity` (0 / 1) in the layout of the clover field (I64
// double2 [parity][72][Vh], I32 float4 [parity][36][Vh]; the other parity untouched), and
// the sum over those sites of ln det (1 + A) into R.s->slot[slot]
cudaError_t clover_invert(const double2* C64, const Geom& g, int parity, double2* I64, float4* I32, const RedArgs& R,
                          int slot, cudaStream_t st);
// adds the insertion of -2 ln det (1 + A) over the sites of `parity` to M (from I64)
cudaError_t clover_det_insertion(const double2* I64, const Geom& g, int parity, const CloverSigma& S, double kappa,
                                 double csw, double2* M, cudaStream_t st);
// the clover force gather (Lie form) in double-float arithmetic from the links' double-float
// copy and the insertions' (float4 [parity][54][Vh], converted from the FP64 field)
cudaError_t clover_force_df(const float4* Udf, const float4* Mdf, const Geom& g, double coef, int keep, double2* out,
                            cudaStream_t st);
cudaError_t clover_force(const double2* U, const double2* M, const Geom& g, double coef, int keep, int form,
                         double2* out, cudaStream_t st);

// ---------------------------------------------------------------- stout (lgt_stout.cu)
cudaError_t stout_forward(const double2* Uin, double2* Uout, const Geom& g, double rho, cudaStream_t st);
// Gin = adjoint of one level applied to Gout, for the level whose input is Uin
cudaError_t stout_backward(const double2* Uin, const double2* Gout, double2* Gin, double2* scratch, const Geom& g,
                           double rho, cudaStream_t st);

// ---------------------------------------------------------------- diagnostics
cudaError_t fp64_peak_kernel_run(double* flops, double* seconds);

}  // namespace lgt
