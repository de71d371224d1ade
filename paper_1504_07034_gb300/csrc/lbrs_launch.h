// Host-side launchers of the LBRS kernels (internal to the library).
//
// The FP64 step and every FP64-arithmetic helper kernel live in
// lbrs_kernels_f64.cu (compiled without FMA contraction); the FP32 step lives
// in lbrs_kernels_f32.cu.  The runtime (lbrs_runtime.cu) calls only these.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

namespace lbrs {
// A named range on the profiler's host timeline for the enclosing scope (header-only
// NVTX: without an attached tool the calls do nothing).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace lbrs

namespace lbrs {

template <typename T>
struct StepArgs;
template <typename T>
struct AdjArgs;
template <typename T>
struct BatchArgs;
struct BatchTile;

// The LBRS_DEBUG build's first out-of-bounds record of each kernel unit
// ((site << 40) | index, 0 if none; clear != 0 zeroes it); 0 in release builds.
unsigned long long debug_word_f32(int clear);
unsigned long long debug_word_f64(int clear);
unsigned long long debug_word_f16(int clear);

// Failure-detection self-test: a bounded wait on an mbarrier that nothing completes
// gives up and raises *wait_flag (one block, 4096 polls).
cudaError_t launch_wait_timeout_selftest(unsigned* wait_flag, cudaStream_t s);
cudaError_t launch_rcp_selftest(const float* x, float* r, int64_t n, cudaStream_t s);

// One time step src -> dst.  lattice: LAT_D1Q2 / LAT_D2Q4.
cudaError_t launch_step_f64(int lattice, const StepArgs<double>& a, cudaStream_t s);
cudaError_t launch_step_f32(int lattice, const StepArgs<float>& a, cudaStream_t s);
// D2Q4 FP32: two time steps in one launch, src -> dst (temporal blocking by two).
// With a valid tile map of src the kernel fetches its window by tensor copies and
// reports a bounded wait that gave up in *wait_flag; otherwise it loads directly.
// A non-null a.Uout records the moments of both steps: [2][4][N] from a.Uout.
struct alignas(64) TileMap {
    unsigned char bytes[128];   // an encoded CUtensorMap (36 x 18 x 4-field boxes of the state)
    int valid;
};
bool step2_f32_enabled();
bool encode_f32_tile_map(TileMap* map, const float* f, int64_t nx, int64_t ny);
cudaError_t launch_step2_f32(const StepArgs<float>& a, const TileMap* map, unsigned* wait_flag, cudaStream_t s);
// D2Q4 FP32: three time steps in one launch, src -> dst (temporal blocking by three; tensor
// copies of 40 x 20 boxes, so nx % 4 == 0), bit-identical to single steps.  Not for internal
// walls, halfway walls or recording steps.  Off when the environment sets LBRS_F32_FUSE3=0.
bool step3_f32_enabled();
bool encode_f32_tile_map3(TileMap* map, const float* f, int64_t nx, int64_t ny);
cudaError_t launch_step3_f32(const StepArgs<float>& a, const TileMap* map3, unsigned* wait_flag, cudaStream_t s);
// Two scalar D2Q4 (2-D Burgers) steps per launch, FP32: a.src -> a.dst.
cudaError_t launch_step2s_f32(const StepArgs<float>& a, cudaStream_t s);

// Dirichlet ghost tables: ghost[side][q*K + k] = f^eq(U(prim[side])) for every
// side whose kind is DIRICHLET, computed in FP64 and rounded to the storage type.
struct GhostSpec {
    double prim[4][4];
    int kind[4];
    double dx;       // the scalar lattice's boundary profiles are functions of the coordinate
};
cudaError_t launch_ghost(int lattice, int storage_f64, const GhostSpec& g, double gamma, double c, void* ghost,
                         cudaStream_t s);
// Adaptive lambda (D2Q4): st is an AdaptState in the workspace.
cudaError_t launch_adapt_reset(void* st, double lambda, cudaStream_t s);
cudaError_t launch_adapt_prep(int storage_f64, void* st, void* ghost, const GhostSpec& g, double gamma, double dx,
                              double safety, double t_final, cudaStream_t s);
cudaError_t launch_adapt_step_f64(const StepArgs<double>& a, void* st, double gamma, cudaStream_t s);
cudaError_t launch_adapt_step_f32(const StepArgs<float>& a, void* st, double gamma, cudaStream_t s);
cudaError_t launch_adapt_init_bound_f64(const void* fs, int64_t N, double gamma, void* st, cudaStream_t s);
cudaError_t launch_adapt_init_bound_f32(const void* fs, int64_t N, double gamma, void* st, cudaStream_t s);


// f = f^eq(U(W)) for every cell; W is [K][N] of w_dtype (0 f64, 1 f32), conserved or primitive;
// fs has planes of `plane` >= N elements (cell c of plane n at fs[n * plane + c]).
cudaError_t launch_set_state(int lattice, int storage_f64, const void* W, int w_dtype, int kind, void* fs,
                             int64_t N, int64_t plane, double gamma, double c, cudaStream_t s);

// U[k][c] = sum_q fs[q][k][c] in FP64, written as out_dtype (0 f64, 1 f32), for the N cells
// c of planes `plane` elements apart (U is [K][N]).
cudaError_t launch_moments(int lattice, int storage_f64, const void* fs, void* U, int out_dtype, int64_t N,
                           int64_t plane, cudaStream_t s);

// Fixed-order FP64 diagnostics: nblocks partial records of DIAG_W doubles, then
// one finalising pass into out[DIAG_W] = totals[4], min_rho, min_p,
// max_lambda_local, n_nonphysical, n_subchar, (unused).
int diag_blocks();
cudaError_t launch_diag(int lattice, int storage_f64, const void* fs, int64_t N, int64_t plane, double gamma,
                        double lambda, double cell_volume, double* partials, double* out, cudaStream_t s);

// Periodic device checks: reset the status record, fold one diagnostics result into it.
cudaError_t launch_status_reset(double* status, cudaStream_t s);
cudaError_t launch_status_update(const double* diag_out, double* status, int64_t step, cudaStream_t s);

// Recording step (D2Q4): the step above that also writes its moments to a.Uout.
cudaError_t launch_step_record_f64(const StepArgs<double>& a, cudaStream_t s);
// D2Q4 boundary balance of the next step: out[0..3] inflow, out[4..7] outflow (FP64, times vol).
cudaError_t launch_boundary_flux_f64(const StepArgs<double>& a, double vol, double* out, cudaStream_t s);
cudaError_t launch_boundary_flux_f32(const StepArgs<float>& a, double vol, double* out, cudaStream_t s);
cudaError_t launch_step_record_f32(const StepArgs<float>& a, cudaStream_t s);

// Adjoint of one periodic D2Q4 step, and the equilibrium VJP dL/dU0 (see lbrs_kernels.cuh).
cudaError_t launch_adjoint_f64(const AdjArgs<double>& a, cudaStream_t s);
cudaError_t launch_adjoint_f32(const AdjArgs<float>& a, cudaStream_t s);
// FP32 adjoint sweep on k = (1 - w) g + w J_E^T g (periodic D2Q4): pointwise k from
// g (a.U, a.gin -> a.gout); one pull step (with a.U: k, without: g); two fused steps
// k^s -> k^{s-2} with a.U = U_{s-1} and U2 = U_{s-2}.
cudaError_t launch_adj_local_f32(const AdjArgs<float>& a, cudaStream_t s);
cudaError_t launch_adj_pull_f32(const AdjArgs<float>& a, cudaStream_t s);
// With a valid tile map of a.gin (the k buffer, encode_f32_tile_map) the tensor-copy form on 32 x 16
// tiles, reporting a bounded wait that gave up in *wait_flag; otherwise direct loads.
cudaError_t launch_adj_fused2_f32(const AdjArgs<float>& a, const float* U2, const TileMap* map, unsigned* wait_flag,
                                  cudaStream_t s);
// FP32 sweep at omega = 1 in its moments form: the state kU = J_E(U)^T g (4 planes, the
// same for every population).  local: kU from a full g; pull: kU -> kU' (a.U set) or
// -> the full g (a.U NULL); fused2: kU^s -> kU^{s-2} (a.U = U_{s-1}, U2 = U_{s-2}).
bool adj_uform_enabled();
cudaError_t launch_adj_local_u_f32(const AdjArgs<float>& a, cudaStream_t s);
cudaError_t launch_adj_pull_u_f32(const AdjArgs<float>& a, cudaStream_t s);
cudaError_t launch_adj_fused2_u_f32(const AdjArgs<float>& a, const float* U2, cudaStream_t s);
cudaError_t launch_vjp_equilibrium_f64(const AdjArgs<double>& a, cudaStream_t s);
cudaError_t launch_vjp_equilibrium_f32(const AdjArgs<float>& a, cudaStream_t s);

// gbar[q][k][c] = dLdU[k][c] for every q (dLdU of in_dtype 0 f64 / 1 f32; gbar in storage type).
cudaError_t launch_adjoint_seed(int Q, int K, int storage_f64, const void* dLdU, int in_dtype, void* gbar, int64_t N,
                                cudaStream_t s);

// Density mismatch loss 0.5 sum (rho - target)^2 * cell_volume of fs (rho = sum_q fs[q][0]),
// reduced in FP64 in a fixed order into out[0], and its gradient seed
// gbar[q][0] = (rho - target) * cell_volume, gbar[q][k>0] = 0.
cudaError_t launch_density_loss(int Q, int K, int storage_f64, const void* fs, const void* target, int t_dtype,
                                void* gbar, int64_t N, int64_t plane, double cell_volume, double* partials, double* out,
                                cudaStream_t s);

// Batched D1Q2 / D1Q3 tubes with temporal blocking (lbrs_batch.cuh): one CTA of
// `block` threads per active tile; dynamic shared memory 2*3Q*(TILE+2H) elements.
cudaError_t launch_batch_f64(const BatchArgs<double>& a, int ntiles, int block, cudaStream_t s);
cudaError_t launch_batch_f32(const BatchArgs<float>& a, int ntiles, int block, cudaStream_t s);
// Raise the kernel's dynamic shared-memory limit to smem bytes (call before launching or capturing).
cudaError_t prepare_batch_f64(int block, size_t smem, int q);
cudaError_t prepare_batch_f32(int block, size_t smem, int q);
cudaError_t launch_batch_copy_f64(const double* src, double* dst, int64_t N, const BatchTile* tiles, int ntiles,
                                  const int64_t* tube_off, int planes, cudaStream_t s);
cudaError_t launch_batch_copy_f32(const float* src, float* dst, int64_t N, const BatchTile* tiles, int ntiles,
                                  const int64_t* tube_off, int planes, cudaStream_t s);

// Batched tubes: f = f^eq(U(W)) with each cell's tube lambda (bisection in tube_off).
cudaError_t launch_batch_set_state(int storage_f64, const void* W, int w_dtype, int kind, void* fs, int64_t N,
                                   const int64_t* tube_off, int64_t nb, const double* tube_lam, double gamma, int q,
                                   cudaStream_t s);

// FP16 non-equilibrium form (lbrs_kernels_f16.cu).  A state buffer holds U as
// [4][N] FP32, g as [3][4][N] FP16 and the four per-field scales (FP32):
// 40 N + 16 bytes.
struct F16StepArgs {
    const void* src;
    void* dst;
    const float* ghost;    // [4][GHOST_STRIDE] f of the Dirichlet states (FP32)
    int64_t N;
    int nx, ny;
    int bc[4];
    float om, om1, c, gm1;
};
cudaError_t launch_step_f16neq(const F16StepArgs& a, cudaStream_t s);
// Moments-only form (omega = 1): a state buffer is U [4][N] FP32.
cudaError_t launch_step_f32u(const F16StepArgs& a, cudaStream_t s);
// The same, two steps per launch (bit-identical to two single steps); off when the
// environment sets LBRS_F32U_FUSE=0.
cudaError_t launch_step2_f32u(const F16StepArgs& a, cudaStream_t s);
bool step2_f32u_enabled();
cudaError_t launch_set_state_f32u(const void* W, int w_dtype, int kind, void* fs, int64_t N, int64_t plane,
                                  double gamma, cudaStream_t s);
// U = U(W) in FP32, g = 0, then the per-field scales from max |U_k| (absmax_bits: 4 words of scratch).
cudaError_t launch_set_state_f16neq(const void* W, int w_dtype, int kind, void* fs, int64_t N, double gamma,
                                    unsigned int* absmax_bits, cudaStream_t s);

}  // namespace lbrs
