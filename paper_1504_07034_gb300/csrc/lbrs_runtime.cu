// Host runtime of the LBRS solver: the C ABI declared in include/lbrs.h.
//
// Owns nothing on the device: the caller's workspace is carved into two
// ping-pong distribution buffers, the Dirichlet ghost tables and the
// diagnostics scratch.  Steps are enqueued on the caller's stream; runs of
// many steps replay a CUDA graph of graph_steps() steps (captured once per
// context and buffer parity on a private stream).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <cuda_runtime.h>

#include "lbrs.h"
#include "lbrs_kernels.cuh"
#include "lbrs_batch.cuh"
#include "lbrs_launch.h"

using namespace lbrs;

namespace {

constexpr size_t kAlign = 256;
constexpr int kGraphSteps = 32;   // 16 two-step or 32 one-step launches: an even number

thread_local char g_err[512] = "";

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// f_bytes: the raw state of the context's own cells (what lbrs_get_distributions moves);
// store_bytes: one stored buffer, which also holds the ghost rows of cut sides;
// each of the two buffers takes a slot that can also stage K FP64 fields of host input.
struct Layout {
    size_t f_bytes, store_bytes, slot, f0, f1, ghost, partials, diag_out, scale, status, wait_flag, adapt, total;
};

bool two_d(int lat) { return lat == LBRS_D2Q4 || lat == LBRS_D2Q4S; }
int lattice_q(int lat) { return two_d(lat) ? 4 : (lat == LBRS_D1Q3 ? 3 : 2); }
int lattice_k(int lat) { return lat == LBRS_D2Q4 ? 4 : (lat == LBRS_D2Q4S ? 1 : 3); }

constexpr int kDefaultHaloRows = 2;   // the two-step kernel's depth
constexpr int kMaxHaloRows = 64;

// Ghost rows stored beyond y side s (2 = y-lo, 3 = y-hi): the side's halo depth if it is a cut.
int64_t ghost_rows(const lbrs_config* c, int s)
{
    if (c->lattice != LBRS_D2Q4 || s < 2 || c->bc[s].kind != LBRS_BC_CUT) return 0;
    return c->bc[s].halo_rows ? c->bc[s].halo_rows : kDefaultHaloRows;
}
int64_t stored_rows(const lbrs_config* c) { return c->ny + ghost_rows(c, 2) + ghost_rows(c, 3); }
// Planes of one stored buffer in the distribution forms and the moments-only form.
int state_planes(const lbrs_config* c)
{
    return c->precision == LBRS_F32U ? 4 : lattice_q(c->lattice) * lattice_k(c->lattice);
}
// kernel lattice code of a public lattice
int lat_code(int lat)
{
    return lat == LBRS_D2Q4 ? LAT_D2Q4 : (lat == LBRS_D2Q4S ? LAT_D2Q4S : (lat == LBRS_D1Q3 ? LAT_D1Q3 : LAT_D1Q2));
}

Layout layout_of(const lbrs_config* c)
{
    Layout L;
    const size_t elem = c->precision == LBRS_F64 ? 8 : 4;
    const size_t N = (size_t)c->nx * (size_t)c->ny;
    const size_t Ns = (size_t)c->nx * (size_t)stored_rows(c);
    if (c->precision == LBRS_F16NEQ) {
        L.f_bytes = L.store_bytes = N * (4 * 4 + 12 * 2) + 4 * sizeof(float);
    } else {
        L.f_bytes = N * (size_t)state_planes(c) * elem;
        L.store_bytes = Ns * (size_t)state_planes(c) * elem;
    }
    // host input and output are staged through the idle buffer: K FP64 fields of the own cells
    const size_t stage = N * (size_t)lattice_k(c->lattice) * sizeof(double);
    L.slot = align_up(L.store_bytes > stage ? L.store_bytes : stage);
    size_t off = 0;
    L.f0 = off;
    off += L.slot;
    L.f1 = off;
    off += L.slot;
    L.ghost = off;
    off += align_up(4 * GHOST_STRIDE * elem);
    L.partials = off;
    off += align_up((size_t)diag_blocks() * DIAG_W * sizeof(double));
    L.diag_out = off;
    off += align_up(DIAG_W * sizeof(double));
    L.scale = off;                                   // FP16 form: 4 words of scratch for the scales
    off += align_up(4 * sizeof(float));
    L.status = off;                                  // record of the periodic device checks
    off += align_up(4 * sizeof(double));
    L.wait_flag = off;                               // set by a bounded device wait that gave up
    off += align_up(sizeof(unsigned));
    L.adapt = off;                                   // the adaptive-lambda run's record
    off += align_up(sizeof(AdaptState));
    L.total = off;
    return L;
}

}  // namespace

struct lbrs_ctx {
    lbrs_config cfg;
    Layout L;
    int lattice, f64, f16, f32u, Q, K;
    int P;                   // planes of a stored buffer: Q * K, or 4 in the moments-only form
    int64_t N;               // stored cells nx * ny_store: the plane stride of the state buffers
    int64_t N_own;           // the context's own cells nx * ny
    int64_t ny_store;        // stored rows: ny plus the ghost rows of cut y sides
    int64_t row0;            // stored row of own row 0 (the ghost rows below it)
    int64_t halo[2];         // ghost rows below (y-lo) and above (y-hi); 0 where the side is not a cut
    int64_t halo_left[2];    // steps the last import of each cut side still covers
    char* ws;
    char* f[2];
    int cur;                 // index of the buffer holding the current state
    cudaStream_t stream;
    bool has_state;
    int64_t step;
    int64_t launches;
    double c;                // 1/(4 lambda) in 2-D, 1/(2 lambda) in 1-D
    cudaStream_t cap_stream;
    cudaGraphExec_t graph[2];
    TileMap tmap[2];         // tensor maps of the two state buffers (FP32 D2Q4 two-step kernel)
    TileMap tmap3[2];        // the same for the three-step kernel (larger boxes)
    int graph_launches[2];   // kernels in graph[b]
    const uint8_t* solid;    // caller-owned obstacle mask [ny][nx] (lbrs_set_obstacles), or NULL
    GhostSpec gspec;         // the sides' kinds and states (the adaptive run rebuilds the ghosts)
    bool adapt_ready;        // the adaptive record holds the current state's run
    bool adapt_used;         // the distributions carry an adaptive lambda
    cudaGraphExec_t agraph[2];   // kAdaptGraphSteps adaptive steps from buffer b
    double agraph_key[2];        // (safety, t_final) the adaptive graphs were captured with
    // checkpointed adjoint: the run recorded by lbrs_forward_checkpointed
    char* adj_ws;
    size_t adj_bytes;
    int64_t adj_n, adj_seg, adj_step0;
    char err[512];
};

namespace {

lbrs_status fail(lbrs_ctx* ctx, lbrs_status s, const char* fmt, ...)
{
    char* buf = ctx ? ctx->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (ctx) snprintf(g_err, sizeof g_err, "%s", ctx->err);
    return s;
}

lbrs_status cuda_fail(lbrs_ctx* ctx, cudaError_t e, const char* what)
{
    return fail(ctx, LBRS_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define LBRS_CUDA(ctx, call)                                        \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);  \
    } while (0)

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

lbrs_status validate(const lbrs_config* c)
{
    if (!c) return fail(nullptr, LBRS_EINVAL, "config is NULL");
    if (c->struct_size != sizeof(lbrs_config))
        return fail(nullptr, LBRS_EINVAL, "config.struct_size %u != sizeof(lbrs_config) %zu", c->struct_size,
                    sizeof(lbrs_config));
    if (c->lattice != LBRS_D1Q2 && c->lattice != LBRS_D2Q4 && c->lattice != LBRS_D1Q3 && c->lattice != LBRS_D2Q4S)
        return fail(nullptr, LBRS_EINVAL, "unknown lattice %d", c->lattice);
    if (c->precision < LBRS_F64 || c->precision > LBRS_F32U)
        return fail(nullptr, LBRS_EINVAL, "unknown precision %d", c->precision);
    if ((c->precision == LBRS_F16NEQ || c->precision == LBRS_F32U) && c->lattice != LBRS_D2Q4)
        return fail(nullptr, LBRS_EINVAL, "LBRS_F16NEQ and LBRS_F32U are D2Q4 storage forms");
    if (c->precision == LBRS_F32U && c->omega != 1.0)
        return fail(nullptr, LBRS_EINVAL, "LBRS_F32U stores only the moments and needs omega == 1");
    if (c->nx < 1 || c->ny < 1) return fail(nullptr, LBRS_EINVAL, "grid must have nx, ny >= 1");
    if (c->nx > (1LL << 30)) return fail(nullptr, LBRS_EINVAL, "nx too large (max 2^30)");
    if (!two_d(c->lattice) && c->ny != 1) return fail(nullptr, LBRS_EINVAL, "1-D lattices (D1Q2, D1Q3) need ny == 1");
    if (two_d(c->lattice) && stored_rows(c) > 2LL * 65535)
        return fail(nullptr, LBRS_EINVAL, "ny too large (max 131070 rows including the ghost rows of cuts)");
    if (!(c->gamma > 1.0) || !isfinite(c->gamma)) return fail(nullptr, LBRS_EINVAL, "gamma must be > 1");
    if (!finite_pos(c->lambda)) return fail(nullptr, LBRS_EINVAL, "lambda must be positive");
    if (!(c->omega > 0.0 && c->omega < 2.0)) return fail(nullptr, LBRS_EINVAL, "omega must lie in (0, 2)");
    if (!finite_pos(c->dx)) return fail(nullptr, LBRS_EINVAL, "dx must be positive");
    if (c->diag_every < 0) return fail(nullptr, LBRS_EINVAL, "diag_every must be >= 0");
    const int sides = two_d(c->lattice) ? 4 : 2;
    for (int s = 0; s < sides; ++s) {
        const int kind = c->bc[s].kind;
        if (kind < LBRS_BC_PERIODIC || kind > LBRS_BC_WALL_HALFWAY)
            return fail(nullptr, LBRS_EINVAL, "side %d: unknown boundary kind %d", s, kind);
        if (kind == LBRS_BC_WALL_HALFWAY &&
            (c->lattice != LBRS_D2Q4 || s < 2 || (c->precision != LBRS_F64 && c->precision != LBRS_F32)))
            return fail(nullptr, LBRS_EINVAL,
                        "side %d: halfway walls are defined on the y sides of D2Q4 in LBRS_F64 or LBRS_F32", s);
        if (kind == LBRS_BC_CUT) {
            if (c->lattice != LBRS_D2Q4 || s < 2)
                return fail(nullptr, LBRS_EINVAL, "side %d: cuts are defined on the y sides of D2Q4 only", s);
            if (c->precision == LBRS_F16NEQ)
                return fail(nullptr, LBRS_EINVAL, "side %d: cuts cover the F64, F32 and F32U forms", s);
            const int h = c->bc[s].halo_rows;
            if (h < 0 || h > kMaxHaloRows)
                return fail(nullptr, LBRS_EINVAL, "side %d: halo_rows must lie in [0, %d]", s, kMaxHaloRows);
            if (c->ny < ghost_rows(c, s))
                return fail(nullptr, LBRS_EINVAL, "side %d: a cut needs ny >= its halo rows", s);
            continue;
        }
        if (kind == LBRS_BC_WALL && (c->lattice != LBRS_D2Q4 || s < 2))
            return fail(nullptr, LBRS_EINVAL, "side %d: walls are defined on the y sides of D2Q4 only", s);
        if (kind == LBRS_BC_PERIODIC && c->bc[s ^ 1].kind != LBRS_BC_PERIODIC)
            return fail(nullptr, LBRS_EINVAL, "side %d: periodic must pair with periodic", s);
        if (kind == LBRS_BC_DIRICHLET) {
            const double* w = c->bc[s].prim;
            const int K = lattice_k(c->lattice);
            if (c->lattice == LBRS_D2Q4S) {       // the scalar's linear profile (value, slope)
                if (!isfinite(w[0]) || !isfinite(w[1]))
                    return fail(nullptr, LBRS_EINVAL, "side %d: non-finite Dirichlet profile", s);
                continue;
            }
            for (int k = 0; k < K; ++k)
                if (!isfinite(w[k])) return fail(nullptr, LBRS_EINVAL, "side %d: non-finite Dirichlet state", s);
            if (!(w[0] > 0.0) || !(w[K - 1] > 0.0))
                return fail(nullptr, LBRS_EINVAL, "side %d: Dirichlet state needs rho > 0 and p > 0", s);
        }
    }
    if (c->lattice == LBRS_D2Q4 && (c->bc[2].kind == LBRS_BC_WALL || c->bc[3].kind == LBRS_BC_WALL) && c->ny < 2)
        return fail(nullptr, LBRS_EINVAL, "walls need ny >= 2");
    return LBRS_OK;
}

// Boundary kind of side s as the kernels see it.  A cut side's stored grid ends in
// its ghost rows, which the kernels close like a transmissive side: the rows next to
// that edge go wrong one row per step, and within the halo depth they stay ghost rows
// (the own rows never read them), until the next import replaces them.
int kernel_bc(const lbrs_ctx* ctx, int s)
{
    const int kind = ctx->cfg.bc[s].kind;
    return kind == LBRS_BC_CUT ? (int)LBRS_BC_TRANSMISSIVE : kind;
}

template <typename T>
StepArgs<T> step_args(const lbrs_ctx* ctx, int from)
{
    StepArgs<T> a;
    a.src = (const T*)ctx->f[from];
    a.dst = (T*)ctx->f[from ^ 1];
    a.ghost = (const T*)(ctx->ws + ctx->L.ghost);
    a.N = ctx->N;
    a.nx = (int)ctx->cfg.nx;
    a.ny = (int)ctx->ny_store;
    for (int s = 0; s < 4; ++s) a.bc[s] = kernel_bc(ctx, s);
    a.om = (T)ctx->cfg.omega;
    a.om1 = (T)(1.0 - ctx->cfg.omega);
    a.c = (T)ctx->c;
    a.gm1 = (T)(ctx->cfg.gamma - 1.0);
    a.Uout = nullptr;
    a.solid = ctx->solid;
    return a;
}

// Arguments of the reduced-state kernels (FP16 non-equilibrium and moments-only forms).
F16StepArgs f16_args(const lbrs_ctx* ctx, int from)
{
    F16StepArgs a;
    a.src = ctx->f[from];
    a.dst = ctx->f[from ^ 1];
    a.ghost = (const float*)(ctx->ws + ctx->L.ghost);
    a.N = ctx->N;
    a.nx = (int)ctx->cfg.nx;
    a.ny = (int)ctx->ny_store;
    for (int k = 0; k < 4; ++k) a.bc[k] = kernel_bc(ctx, k);
    a.om = (float)ctx->cfg.omega;
    a.om1 = (float)(1.0 - ctx->cfg.omega);
    a.c = (float)ctx->c;
    a.gm1 = (float)(ctx->cfg.gamma - 1.0);
    return a;
}

cudaError_t launch_one_step(lbrs_ctx* ctx, int from, cudaStream_t s)
{
    const int lat = lat_code(ctx->lattice);
    if (ctx->f64) return launch_step_f64(lat, step_args<double>(ctx, from), s);
    if (ctx->f16) return launch_step_f16neq(f16_args(ctx, from), s);
    if (ctx->f32u) return launch_step_f32u(f16_args(ctx, from), s);
    return launch_step_f32(lat, step_args<float>(ctx, from), s);
}

// FP32 1-D (D1Q2, D1Q3) with both ends transmissive or both periodic: steps taken by the batched
// tubes' temporal-blocking kernel as a tube of one, up to kOneHalo steps per launch in shared memory
// (tiles of 4 kOneBlock - 2 kOneHalo cells; the single-tube arithmetic, bit-identical to one step a
// launch).  LBRS_1D_BLOCKED=0 keeps one step a launch.
constexpr int kOneBlock = 256, kOneCellsPerThread = 4, kOneHalo = 32;
constexpr int kOneTile = kOneBlock * kOneCellsPerThread - 2 * kOneHalo;

bool blocked_1d(const lbrs_ctx* ctx)
{
    static const int enabled = [] {
        const char* e = getenv("LBRS_1D_BLOCKED");
        return (e && !strcmp(e, "0")) ? 0 : 1;
    }();
    if (!enabled || ctx->f64 || (ctx->lattice != LBRS_D1Q2 && ctx->lattice != LBRS_D1Q3)) return false;
    const int k0 = ctx->cfg.bc[0].kind, k1 = ctx->cfg.bc[1].kind;
    return k0 == k1 && (k0 == LBRS_BC_TRANSMISSIVE || k0 == LBRS_BC_PERIODIC);
}

size_t blocked_1d_smem(const lbrs_ctx* ctx) { return 2 * 3 * (size_t)ctx->Q * (kOneTile + 2 * kOneHalo) * sizeof(float); }

// m <= kOneHalo steps of a blocked 1-D context from buffer `from` in one launch.
cudaError_t launch_blocked_1d(const lbrs_ctx* ctx, int from, int m, cudaStream_t s)
{
    BatchArgs<float> a{};
    a.src = (const float*)ctx->f[from];
    a.dst = (float*)ctx->f[from ^ 1];
    a.N = ctx->N;
    a.tiles = nullptr;
    a.tile_cells = kOneTile;
    a.halo = kOneHalo;
    a.periodic = ctx->cfg.bc[0].kind == LBRS_BC_PERIODIC;
    a.launch = 0;
    a.q = ctx->Q;
    a.om = (float)ctx->cfg.omega;
    a.om1 = (float)(1.0 - ctx->cfg.omega);
    a.gm1 = (float)(ctx->cfg.gamma - 1.0);
    a.one_len = (int)ctx->cfg.nx;
    a.one_steps = m;
    a.one_c = (float)ctx->c;
    const int ntiles = (int)((ctx->cfg.nx + kOneTile - 1) / kOneTile);
    // the kernel's shared-memory limit is shared with the batched tubes, which set it per tuning
    const cudaError_t e = prepare_batch_f32(kOneBlock, blocked_1d_smem(ctx), ctx->Q);
    if (e != cudaSuccess) return e;
    return launch_batch_f32(a, ntiles, kOneBlock, s);
}

// The FP32 distribution form's two-steps-per-launch kernel available for this context?
// With internal walls only in its tensor-copy form.
bool fused2_f32(const lbrs_ctx* ctx)
{
    if (ctx->f64 || ctx->f16 || ctx->f32u || ctx->lattice != LBRS_D2Q4 || !step2_f32_enabled()) return false;
    return !ctx->solid || (ctx->tmap[0].valid && ctx->tmap[1].valid);
}

// Does lbrs_step advance this context two steps per launch (FP32 distributions, or the
// moments-only form)?
// Scalar D2Q4 (2-D Burgers) in FP32: two steps per launch; LBRS_F32S_FUSE=0 keeps one.
bool fused2_scalar(const lbrs_ctx* ctx)
{
    static const int enabled = [] {
        const char* e = getenv("LBRS_F32S_FUSE");
        return (e && !strcmp(e, "0")) ? 0 : 1;
    }();
    return enabled && !ctx->f64 && ctx->lattice == LBRS_D2Q4S;
}

bool fused2(const lbrs_ctx* ctx)
{
    return fused2_f32(ctx) || (ctx->f32u && step2_f32u_enabled()) || fused2_scalar(ctx);
}

unsigned* wait_flag(const lbrs_ctx* ctx) { return (unsigned*)(ctx->ws + ctx->L.wait_flag); }

// The FP32 three-steps-per-launch kernel available for this context?  Not with internal
// walls or halfway walls (their populations break the one-reader rule of its in-place phases).
bool fused3(const lbrs_ctx* ctx)
{
    if (!fused2_f32(ctx) || ctx->solid || !step3_f32_enabled()) return false;
    if (ctx->cfg.bc[2].kind == LBRS_BC_WALL_HALFWAY || ctx->cfg.bc[3].kind == LBRS_BC_WALL_HALFWAY) return false;
    return ctx->tmap3[0].valid && ctx->tmap3[1].valid;
}

// Steps the next launch takes out of `left`: three where the three-step kernel applies (but
// 2 + 2 rather than 3 + 1), else two where the two-step kernel does, else one.
int next_launch_steps(const lbrs_ctx* ctx, int64_t left)
{
    if (left >= 3 && left != 4 && fused3(ctx)) return 3;
    if (left >= 2 && fused2(ctx)) return 2;
    return 1;
}

// Steps per captured graph: 12 three-step launches, else kGraphSteps (an even number of
// launches either way, so that a graph returns the buffers to their parity).
int graph_steps(const lbrs_ctx* ctx) { return fused3(ctx) ? 36 : kGraphSteps; }

// Three steps from buffer b into buffer b ^ 1.
cudaError_t launch_step3(const lbrs_ctx* ctx, int b, cudaStream_t s)
{
    return launch_step3_f32(step_args<float>(ctx, b), &ctx->tmap3[b], wait_flag(ctx), s);
}

// Two steps from buffer b into buffer b ^ 1.
cudaError_t launch_step2(const lbrs_ctx* ctx, int b, cudaStream_t s)
{
    if (ctx->f32u) return launch_step2_f32u(f16_args(ctx, b), s);
    if (fused2_scalar(ctx)) return launch_step2s_f32(step_args<float>(ctx, b), s);
    return launch_step2_f32(step_args<float>(ctx, b), &ctx->tmap[b], wait_flag(ctx), s);
}

// Lattice code of the read-out kernels (moments, diagnostics) for this storage.
int readout_lattice(const lbrs_ctx* ctx)
{
    if (ctx->f16 || ctx->f32u) return LAT_U2D;
    return lat_code(ctx->lattice);
}

// Capture graph_steps() steps starting from buffer `from` into graph[from].
lbrs_status ensure_graph(lbrs_ctx* ctx, int from)
{
    if (ctx->graph[from]) return LBRS_OK;
    if (!ctx->cap_stream) LBRS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    LBRS_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    int b = from, launches = 0;
    const int G = graph_steps(ctx);
    for (int n = 0; n < G && le == cudaSuccess; ++launches) {
        const int m = next_launch_steps(ctx, G - n);
        le = m == 3 ? launch_step3(ctx, b, ctx->cap_stream)
                    : (m == 2 ? launch_step2(ctx, b, ctx->cap_stream) : launch_one_step(ctx, b, ctx->cap_stream));
        n += m;
        b ^= 1;
    }
    ctx->graph_launches[from] = launches;
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, le, "step launch during graph capture");
    }
    if (ee != cudaSuccess) return cuda_fail(ctx, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&ctx->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        ctx->graph[from] = nullptr;
        return cuda_fail(ctx, ie, "cudaGraphInstantiate");
    }
    return LBRS_OK;
}

size_t field_bytes(const lbrs_ctx* ctx, int dtype)
{
    return (size_t)ctx->K * (size_t)ctx->N_own * (dtype == LBRS_F64 ? 8 : 4);
}

size_t elem_bytes(const lbrs_ctx* ctx) { return ctx->f64 ? 8 : 4; }

// Cell 0 of the own rows in plane 0 of a stored buffer (the planes are ctx->N cells apart).
char* own_ptr(const lbrs_ctx* ctx, char* buf) { return buf + (size_t)ctx->row0 * ctx->cfg.nx * elem_bytes(ctx); }

// The raw state of the own cells between a stored buffer and contiguous planes elsewhere.
cudaError_t copy_own_out(const lbrs_ctx* ctx, char* buf, void* dst, cudaMemcpyKind kind)
{
    if (ctx->N == ctx->N_own) return cudaMemcpyAsync(dst, buf, ctx->L.f_bytes, kind, ctx->stream);
    const size_t e = elem_bytes(ctx), row = (size_t)ctx->N_own * e;
    return cudaMemcpy2DAsync(dst, row, own_ptr(ctx, buf), (size_t)ctx->N * e, row, (size_t)ctx->P, kind, ctx->stream);
}

cudaError_t copy_own_in(const lbrs_ctx* ctx, char* buf, const void* src, cudaMemcpyKind kind)
{
    if (ctx->N == ctx->N_own) return cudaMemcpyAsync(buf, src, ctx->L.f_bytes, kind, ctx->stream);
    const size_t e = elem_bytes(ctx), row = (size_t)ctx->N_own * e;
    return cudaMemcpy2DAsync(own_ptr(ctx, buf), (size_t)ctx->N * e, src, row, row, (size_t)ctx->P, kind, ctx->stream);
}

int readout_lattice(const lbrs_ctx* ctx);

// One periodic check of the current state: the FP64 diagnostics reduction,
// folded into the device status record under the current step number.
cudaError_t periodic_check(lbrs_ctx* ctx)
{
    const double vol = two_d(ctx->lattice) ? ctx->cfg.dx * ctx->cfg.dx : ctx->cfg.dx;
    double* partials = (double*)(ctx->ws + ctx->L.partials);
    double* dout = (double*)(ctx->ws + ctx->L.diag_out);
    cudaError_t e = launch_diag(readout_lattice(ctx), ctx->f64, own_ptr(ctx, ctx->f[ctx->cur]), ctx->N_own, ctx->N,
                                ctx->cfg.gamma, ctx->cfg.lambda, vol, partials, dout, ctx->stream);
    if (e != cudaSuccess) return e;
    ctx->launches += 3;
    return launch_status_update(dout, (double*)(ctx->ws + ctx->L.status), ctx->step, ctx->stream);
}

// A new state clears the record of the periodic checks and the wait flag, ends an
// adaptive-lambda run (the ghosts return to the configured lambda) and leaves the
// ghost rows of cut sides stale until their next import.
lbrs_status reset_status(lbrs_ctx* ctx)
{
    ctx->halo_left[0] = ctx->halo_left[1] = 0;
    if (ctx->adapt_used) {
        LBRS_CUDA(ctx, launch_ghost(lat_code(ctx->lattice), ctx->f64, ctx->gspec, ctx->cfg.gamma, ctx->c,
                                    ctx->ws + ctx->L.ghost, ctx->stream));
        ctx->launches += 1;
    }
    ctx->adapt_ready = ctx->adapt_used = false;
    LBRS_CUDA(ctx, launch_status_reset((double*)(ctx->ws + ctx->L.status), ctx->stream));
    LBRS_CUDA(ctx, cudaMemsetAsync(wait_flag(ctx), 0, sizeof(unsigned), ctx->stream));
    ctx->launches += 1;
    return LBRS_OK;
}

// The adjoint covers the periodic D2Q4 step, and y-slabs of a periodic grid (x periodic,
// y sides cut): its kernels wrap the stored rows in y, which spoils only ghost rows.
lbrs_status adjoint_supported(lbrs_ctx* ctx)
{
    if (ctx->lattice != LBRS_D2Q4) return fail(ctx, LBRS_EINVAL, "the adjoint covers D2Q4 only");
    if (ctx->f16 || ctx->f32u) return fail(ctx, LBRS_EINVAL, "the adjoint covers the F64 and F32 forms only");
    for (int s = 0; s < 4; ++s) {
        const int kind = ctx->cfg.bc[s].kind;
        if (kind != LBRS_BC_PERIODIC && !(s >= 2 && kind == LBRS_BC_CUT))
            return fail(ctx, LBRS_EINVAL, "the adjoint covers periodic domains and their y-slabs only");
    }
    if (ctx->solid) return fail(ctx, LBRS_EINVAL, "the adjoint does not cover internal walls");
    return LBRS_OK;
}

// Host check of an obstacle mask: every population of a fluid cell whose pull comes
// from a solid cell must be replaced by one that is pulled from a fluid cell or a
// Dirichlet ghost (not itself unknown, not behind a domain wall).  Returns the
// number of (cell, population) pairs that break this.
int64_t obstacle_violations(const lbrs_config* c, const uint8_t* m)
{
    const int64_t nx = c->nx, ny = c->ny;
    static const int SX[4] = {-1, 1, 1, -1}, SY[4] = {-1, -1, 1, 1};
    // solidity of a cell index after the domain mapping; Dirichlet and wall sides are fluid
    auto solid = [&](int64_t i, int64_t j) -> bool {
        if (i < 0 || i >= nx) {
            const int kind = c->bc[i < 0 ? 0 : 1].kind;
            if (kind == LBRS_BC_PERIODIC) i = i < 0 ? i + nx : i - nx;
            else if (kind == LBRS_BC_TRANSMISSIVE) i = i < 0 ? 0 : nx - 1;
            else return false;
        }
        if (j < 0 || j >= ny) {
            const int kind = c->bc[j < 0 ? 2 : 3].kind;
            if (kind == LBRS_BC_PERIODIC) j = j < 0 ? j + ny : j - ny;
            else if (kind == LBRS_BC_TRANSMISSIVE) j = j < 0 ? 0 : ny - 1;
            else return false;
        }
        return m[j * nx + i] != 0;
    };
    // is population q of cell (i, j) unknown after streaming (wall side or solid source)?
    auto unknown = [&](int64_t i, int64_t j, int q) -> bool {
        const int64_t si = i - SX[q], sj = j - SY[q];
        const bool out_y = sj < 0 || sj >= ny, out_x = si < 0 || si >= nx;
        if (out_y && c->bc[sj < 0 ? 2 : 3].kind == LBRS_BC_WALL) return true;
        if (out_x && c->bc[si < 0 ? 0 : 1].kind == LBRS_BC_DIRICHLET) return false;
        if (out_y && c->bc[sj < 0 ? 2 : 3].kind == LBRS_BC_DIRICHLET) return false;
        return solid(si, sj);
    };
    int64_t bad = 0;
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            if (m[j * nx + i]) continue;
            for (int q = 0; q < 4; ++q) {
                const int64_t sj = j - SY[q];
                const bool out_y = sj < 0 || sj >= ny;
                if (out_y && c->bc[sj < 0 ? 2 : 3].kind == LBRS_BC_WALL) continue;   // a domain wall's population
                if (!unknown(i, j, q)) continue;
                const bool xn = solid(i - SX[q], j), yn = solid(i, j - SY[q]);
                const int mx = (xn && !yn) || xn == yn ? -SX[q] : SX[q];
                const int my = (!xn && yn) || xn == yn ? -SY[q] : SY[q];
                int mq = 0;
                while (SX[mq] != mx || SY[mq] != my) ++mq;
                if (unknown(i, j, mq)) ++bad;
            }
        }
    return bad;
}

template <typename T>
AdjArgs<T> adj_args(const lbrs_ctx* ctx, const void* U, const void* gin, void* gout)
{
    AdjArgs<T> a;
    a.U = (const T*)U;
    a.gin = (const T*)gin;
    a.gout = (T*)gout;
    a.N = ctx->N;
    a.nx = (int)ctx->cfg.nx;
    a.ny = (int)ctx->ny_store;
    a.om = (T)ctx->cfg.omega;
    a.om1 = (T)(1.0 - ctx->cfg.omega);
    a.c = (T)ctx->c;
    a.gm1 = (T)(ctx->cfg.gamma - 1.0);
    a.gamma = (T)ctx->cfg.gamma;
    return a;
}

// One recording step from the current buffer: writes the step's moments to Uout.
cudaError_t launch_record_step(lbrs_ctx* ctx, void* Uout)
{
    if (ctx->f64) {
        StepArgs<double> a = step_args<double>(ctx, ctx->cur);
        a.Uout = (double*)Uout;
        return launch_step_record_f64(a, ctx->stream);
    }
    StepArgs<float> a = step_args<float>(ctx, ctx->cur);
    a.Uout = (float*)Uout;
    return launch_step_record_f32(a, ctx->stream);
}

// Two recording steps in one launch (FP32 D2Q4): the moments of both steps go to
// Uout and Uout + K N.
cudaError_t launch_record_step2(lbrs_ctx* ctx, void* Uout)
{
    StepArgs<float> a = step_args<float>(ctx, ctx->cur);
    a.Uout = (float*)Uout;
    return launch_step2_f32(a, &ctx->tmap[ctx->cur], wait_flag(ctx), ctx->stream);
}

// Three recording steps in one launch (FP32 D2Q4, where the three-step kernel applies).
cudaError_t launch_record_step3(lbrs_ctx* ctx, void* Uout)
{
    StepArgs<float> a = step_args<float>(ctx, ctx->cur);
    a.Uout = (float*)Uout;
    return launch_step3_f32(a, &ctx->tmap3[ctx->cur], wait_flag(ctx), ctx->stream);
}

// n recording steps from the current buffer into U_hist (stride: one step's moments),
// in threes where the three-step kernel applies (but 2 + 2 rather than 3 + 1), then in pairs
// where the two-step kernel does.
lbrs_status record_steps(lbrs_ctx* ctx, int64_t n, char* U_hist)
{
    const size_t stride = (size_t)ctx->K * ctx->N * elem_bytes(ctx);
    int64_t m = 0;
    for (; m + 3 <= n && n - m != 4 && fused3(ctx); m += 3) {
        LBRS_CUDA(ctx, launch_record_step3(ctx, U_hist + m * stride));
        ctx->cur ^= 1;
        ctx->launches += 1;
    }
    for (; m + 2 <= n && fused2_f32(ctx) && !ctx->solid; m += 2) {
        LBRS_CUDA(ctx, launch_record_step2(ctx, U_hist + m * stride));
        ctx->cur ^= 1;
        ctx->launches += 1;
    }
    for (; m < n; ++m) {
        LBRS_CUDA(ctx, launch_record_step(ctx, U_hist + m * stride));
        ctx->cur ^= 1;
        ctx->launches += 1;
    }
    return LBRS_OK;
}

cudaError_t launch_adjoint_step_raw(lbrs_ctx* ctx, const void* U_next, const void* gin, void* gout)
{
    if (ctx->f64) return launch_adjoint_f64(adj_args<double>(ctx, U_next, gin, gout), ctx->stream);
    return launch_adjoint_f32(adj_args<float>(ctx, U_next, gin, gout), ctx->stream);
}

cudaError_t launch_vjp_eq_raw(lbrs_ctx* ctx, const void* U0, const void* g0, void* grad)
{
    if (ctx->f64) return launch_vjp_equilibrium_f64(adj_args<double>(ctx, U0, g0, grad), ctx->stream);
    return launch_vjp_equilibrium_f32(adj_args<float>(ctx, U0, g0, grad), ctx->stream);
}

struct AdjLayout {
    int64_t nseg;
    size_t ckpt0, ckpt_stride, uhist, gbar0, gbar1, total;
};

AdjLayout adj_layout(const lbrs_ctx* ctx, int64_t n, int64_t seg)
{
    AdjLayout A;
    A.nseg = (n + seg - 1) / seg;
    A.ckpt_stride = align_up(ctx->L.f_bytes);
    size_t off = 0;
    A.ckpt0 = off;
    off += (size_t)(A.nseg + 1) * A.ckpt_stride;          // segment starts plus the final state
    A.uhist = off;
    off += align_up((size_t)seg * ctx->K * ctx->N * elem_bytes(ctx));
    A.gbar0 = off;
    off += A.ckpt_stride;
    A.gbar1 = off;
    off += A.ckpt_stride;
    A.total = off;
    return A;
}

}  // namespace

// Shared with other translation units of the library: configuration checks
// and the thread's last-error text for calls that have no context.
namespace lbrs {
lbrs_status validate_config(const lbrs_config* c) { return validate(c); }
lbrs_status set_error(lbrs_status s, const char* msg) { return fail(nullptr, s, "%s", msg); }
}  // namespace lbrs

// ====================================================================== C ABI

extern "C" {

int lbrs_abi_version(void) { return LBRS_ABI_VERSION; }

lbrs_status lbrs_selftest_wait_timeout(lbrs_ctx* ctx)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    LBRS_CUDA(ctx, launch_wait_timeout_selftest(wait_flag(ctx), ctx->stream));
    ctx->launches += 1;
    return LBRS_OK;
}

lbrs_status lbrs_selftest_rcp_f32(const float* x, float* r, int64_t n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !r))) return fail(nullptr, LBRS_EINVAL, "x and r must be device buffers of n >= 0 floats");
    const cudaError_t e = launch_rcp_selftest(x, r, n, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(nullptr, LBRS_ECUDA, cudaGetErrorString(e));
    return LBRS_OK;
}

int lbrs_debug_build(void)
{
#ifdef LBRS_DEBUG
    return 1;
#else
    return 0;
#endif
}

lbrs_status lbrs_debug_check(uint64_t* first)
{
    if (!first) return fail(nullptr, LBRS_EINVAL, "first is NULL");
    unsigned long long w = 0ull;
    for (unsigned long long v : {debug_word_f32(1), debug_word_f64(1), debug_word_f16(1)})
        if (!w) w = v;
    *first = (uint64_t)w;
    if (w)
        return fail(nullptr, LBRS_ECUDA, "index out of bounds (bounds-checked build): site %llu, index %llu",
                    w >> 40, w & ((1ull << 40) - 1));
    return LBRS_OK;
}

const char* lbrs_status_string(lbrs_status s)
{
    switch (s) {
        case LBRS_OK: return "LBRS_OK";
        case LBRS_EINVAL: return "LBRS_EINVAL";
        case LBRS_ENOMEM: return "LBRS_ENOMEM";
        case LBRS_ECUDA: return "LBRS_ECUDA";
        case LBRS_ENONPHYS: return "LBRS_ENONPHYS";
        case LBRS_ESUBCHAR: return "LBRS_ESUBCHAR";
        case LBRS_ETIMEOUT: return "LBRS_ETIMEOUT";
        case LBRS_ESTATE: return "LBRS_ESTATE";
    }
    return "LBRS_UNKNOWN";
}

lbrs_status lbrs_workspace_size(const lbrs_config* cfg, size_t* bytes)
{
    if (!bytes) return fail(nullptr, LBRS_EINVAL, "bytes is NULL");
    lbrs_status st = validate(cfg);
    if (st != LBRS_OK) return st;
    *bytes = layout_of(cfg).total;
    return LBRS_OK;
}

lbrs_status lbrs_create(const lbrs_config* cfg, void* d_workspace, size_t bytes, lbrs_ctx** out)
{
    if (!out) return fail(nullptr, LBRS_EINVAL, "out is NULL");
    *out = nullptr;
    lbrs_status st = validate(cfg);
    if (st != LBRS_OK) return st;
    const Layout L = layout_of(cfg);
    if (!d_workspace) return fail(nullptr, LBRS_EINVAL, "workspace is NULL");
    if ((uintptr_t)d_workspace % kAlign) return fail(nullptr, LBRS_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < L.total)
        return fail(nullptr, LBRS_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, L.total);

    lbrs_ctx* ctx = (lbrs_ctx*)calloc(1, sizeof(lbrs_ctx));
    if (!ctx) return fail(nullptr, LBRS_ENOMEM, "host allocation of the context failed");
    ctx->cfg = *cfg;
    ctx->L = L;
    ctx->lattice = cfg->lattice;
    ctx->f64 = cfg->precision == LBRS_F64;
    ctx->f16 = cfg->precision == LBRS_F16NEQ;
    ctx->f32u = cfg->precision == LBRS_F32U;
    ctx->Q = lattice_q(cfg->lattice);
    ctx->K = lattice_k(cfg->lattice);
    ctx->P = state_planes(cfg);
    ctx->halo[0] = ghost_rows(cfg, 2);
    ctx->halo[1] = ghost_rows(cfg, 3);
    ctx->row0 = ctx->halo[0];
    ctx->ny_store = stored_rows(cfg);
    ctx->N_own = cfg->nx * cfg->ny;
    ctx->N = cfg->nx * ctx->ny_store;
    ctx->ws = (char*)d_workspace;
    ctx->f[0] = ctx->ws + L.f0;
    ctx->f[1] = ctx->ws + L.f1;
    ctx->stream = (cudaStream_t)cfg->cuda_stream;
    ctx->c = two_d(cfg->lattice) ? 1.0 / (4.0 * cfg->lambda) : 1.0 / (2.0 * cfg->lambda);   // both 1-D lattices: 1/(2 lambda)

    GhostSpec g;
    memset(&g, 0, sizeof g);
    g.dx = cfg->dx;
    for (int s = 0; s < 4; ++s) {
        g.kind[s] = cfg->bc[s].kind;
        for (int k = 0; k < 4; ++k) g.prim[s][k] = cfg->bc[s].prim[k];
    }
    ctx->gspec = g;
    const int lat = lat_code(cfg->lattice);
    cudaError_t e = launch_ghost(lat, ctx->f64, g, cfg->gamma, ctx->c, ctx->ws + L.ghost, ctx->stream);
    if (e != cudaSuccess) {
        lbrs_status s = cuda_fail(nullptr, e, "ghost-table kernel");
        free(ctx);
        return s;
    }
    ctx->launches = 1;
    e = cudaMemsetAsync(wait_flag(ctx), 0, sizeof(unsigned), ctx->stream);
    if (e != cudaSuccess) {
        lbrs_status s = cuda_fail(nullptr, e, "clearing the wait flag");
        free(ctx);
        return s;
    }
    if (fused2_f32(ctx))
        for (int b = 0; b < 2; ++b) {
            encode_f32_tile_map(&ctx->tmap[b], (const float*)ctx->f[b], cfg->nx, ctx->ny_store);
            encode_f32_tile_map3(&ctx->tmap3[b], (const float*)ctx->f[b], cfg->nx, ctx->ny_store);
        }
    *out = ctx;
    return LBRS_OK;
}

void lbrs_destroy(lbrs_ctx* ctx)
{
    if (!ctx) return;
    for (int b = 0; b < 2; ++b) {
        if (ctx->graph[b]) cudaGraphExecDestroy(ctx->graph[b]);
        if (ctx->agraph[b]) cudaGraphExecDestroy(ctx->agraph[b]);
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    free(ctx);
}

lbrs_status lbrs_set_state(lbrs_ctx* ctx, const void* W, int on_device, int dtype, int kind)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!W) return fail(ctx, LBRS_EINVAL, "W is NULL");
    if (dtype != LBRS_F64 && dtype != LBRS_F32) return fail(ctx, LBRS_EINVAL, "dtype must be LBRS_F64 or LBRS_F32");
    if (kind != LBRS_CONSERVED && kind != LBRS_PRIMITIVE) return fail(ctx, LBRS_EINVAL, "unknown state kind %d", kind);
    const void* src = W;
    if (!on_device) {
        // stage through the idle buffer: K*N*8 bytes always fit in Q*K*N*elem
        char* stage = ctx->f[ctx->cur ^ 1];
        LBRS_CUDA(ctx, cudaMemcpyAsync(stage, W, field_bytes(ctx, dtype), cudaMemcpyHostToDevice, ctx->stream));
        src = stage;
    }
    const int lat = lat_code(ctx->lattice);
    if (ctx->f32u) {
        LBRS_CUDA(ctx, launch_set_state_f32u(src, dtype == LBRS_F32, kind, own_ptr(ctx, ctx->f[ctx->cur]), ctx->N_own,
                                             ctx->N, ctx->cfg.gamma, ctx->stream));
    } else if (ctx->f16) {
        LBRS_CUDA(ctx, launch_set_state_f16neq(src, dtype == LBRS_F32, kind, ctx->f[ctx->cur], ctx->N, ctx->cfg.gamma,
                                               (unsigned int*)(ctx->ws + ctx->L.scale), ctx->stream));
        ctx->launches += 3;
    } else {
        LBRS_CUDA(ctx, launch_set_state(lat, ctx->f64, src, dtype == LBRS_F32, kind, own_ptr(ctx, ctx->f[ctx->cur]),
                                        ctx->N_own, ctx->N, ctx->cfg.gamma, ctx->c, ctx->stream));
    }
    ctx->launches += 1;
    lbrs_status rs = reset_status(ctx);
    if (rs != LBRS_OK) return rs;
    if (!on_device) LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // host W is consumed on return
    ctx->has_state = true;
    ctx->step = 0;
    return LBRS_OK;
}

static lbrs_status step_plain(lbrs_ctx* ctx, int64_t n);

lbrs_status lbrs_step(lbrs_ctx* ctx, int64_t n)
{
    NvtxRange range("lbrs_step");
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (n < 0) return fail(ctx, LBRS_EINVAL, "negative step count");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    if (ctx->adapt_used)
        return fail(ctx, LBRS_ESTATE, "the distributions carry an adaptive lambda: continue with "
                                      "lbrs_step_adaptive or set a state");
    for (int h = 0; h < 2; ++h)
        if (ctx->halo[h] && n > ctx->halo_left[h])
            return fail(ctx, LBRS_ESTATE, "%lld steps requested, but the ghost rows of the %s cut cover %lld more "
                        "steps: import the neighbour's rows (lbrs_halo_import) first", (long long)n,
                        h ? "y-hi" : "y-lo", (long long)ctx->halo_left[h]);
    for (int h = 0; h < 2; ++h)
        if (ctx->halo[h]) ctx->halo_left[h] -= n;
    const int64_t every = ctx->cfg.diag_every;
    if (every <= 0) return step_plain(ctx, n);
    // run to each multiple of diag_every, check there
    while (n > 0) {
        const int64_t to_check = every - ctx->step % every;
        const int64_t m = to_check < n ? to_check : n;
        lbrs_status st = step_plain(ctx, m);
        if (st != LBRS_OK) return st;
        n -= m;
        if (ctx->step % every == 0) LBRS_CUDA(ctx, periodic_check(ctx));
    }
    return LBRS_OK;
}

static lbrs_status step_plain(lbrs_ctx* ctx, int64_t n)
{
    if (blocked_1d(ctx)) {
        for (int64_t left = n; left > 0;) {
            const int m = (int)(left < kOneHalo ? left : kOneHalo);
            LBRS_CUDA(ctx, launch_blocked_1d(ctx, ctx->cur, m, ctx->stream));
            ctx->cur ^= 1;
            ctx->step += m;
            ctx->launches += 1;
            left -= m;
        }
        return LBRS_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LBRS_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
    int64_t left = n;
    const int G = graph_steps(ctx);
    if (cap == cudaStreamCaptureStatusNone && n >= 2 * G) {
        lbrs_status st = ensure_graph(ctx, ctx->cur);
        if (st != LBRS_OK) return st;
        while (left >= G) {
            LBRS_CUDA(ctx, cudaGraphLaunch(ctx->graph[ctx->cur], ctx->stream));
            left -= G;
            ctx->step += G;
            ctx->launches += ctx->graph_launches[ctx->cur];
        }
    }
    while (left > 0) {
        const int m = next_launch_steps(ctx, left);
        LBRS_CUDA(ctx, m == 3 ? launch_step3(ctx, ctx->cur, ctx->stream)
                              : (m == 2 ? launch_step2(ctx, ctx->cur, ctx->stream)
                                        : launch_one_step(ctx, ctx->cur, ctx->stream)));
        ctx->cur ^= 1;
        ctx->step += m;
        ctx->launches += 1;
        left -= m;
    }
    return LBRS_OK;
}

lbrs_status lbrs_sync(lbrs_ctx* ctx)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    {
        unsigned flag = 0;
        LBRS_CUDA(ctx, cudaMemcpyAsync(&flag, wait_flag(ctx), sizeof flag, cudaMemcpyDeviceToHost, ctx->stream));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (flag == 1) return fail(ctx, LBRS_ETIMEOUT, "a bounded wait for a tile copy gave up; the state is not valid");
        if (flag)
            return fail(ctx, LBRS_ETIMEOUT, "a bounded wait for a tile copy gave up and the copy had not landed when "
                        "its block left: the state is not valid, and the copy may have completed into shared "
                        "memory of a later block of the same launch or of a later kernel");
    }
#ifdef LBRS_DEBUG
    {
        uint64_t w = 0;
        if (lbrs_debug_check(&w) != LBRS_OK)
            return fail(ctx, LBRS_ECUDA, "index out of bounds (bounds-checked build): site %llu, index %llu",
                        (unsigned long long)(w >> 40), (unsigned long long)(w & ((1ull << 40) - 1)));
    }
#endif
    if (ctx->cfg.diag_every > 0 && ctx->has_state) {
        double st[4];
        LBRS_CUDA(ctx, cudaMemcpyAsync(st, ctx->ws + ctx->L.status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (st[0] >= 0.0) {
            if (st[1] > 0.0)
                return fail(ctx, LBRS_ENONPHYS, "%lld non-physical cells at step %lld", (long long)st[1], (long long)st[0]);
            return fail(ctx, LBRS_ESUBCHAR, "%lld cells exceed lambda at step %lld (max local bound %.6g)",
                        (long long)st[2], (long long)st[0], st[3]);
        }
    }
    return LBRS_OK;
}

lbrs_status lbrs_first_bad_step(lbrs_ctx* ctx, int64_t* step)
{
    if (!ctx || !step) return fail(ctx, LBRS_EINVAL, "NULL argument");
    *step = -1;
    if (!ctx->has_state) return LBRS_OK;
    double st[4];
    LBRS_CUDA(ctx, cudaMemcpyAsync(st, ctx->ws + ctx->L.status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *step = (int64_t)st[0];
    return LBRS_OK;
}

lbrs_status lbrs_moments(lbrs_ctx* ctx, void* U_out, int on_device, int dtype)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!U_out) return fail(ctx, LBRS_EINVAL, "U_out is NULL");
    if (dtype != LBRS_F64 && dtype != LBRS_F32) return fail(ctx, LBRS_EINVAL, "dtype must be LBRS_F64 or LBRS_F32");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    void* dst = on_device ? U_out : (void*)ctx->f[ctx->cur ^ 1];
    LBRS_CUDA(ctx, launch_moments(readout_lattice(ctx), ctx->f64, own_ptr(ctx, ctx->f[ctx->cur]), dst,
                                  dtype == LBRS_F32, ctx->N_own, ctx->N, ctx->stream));
    ctx->launches += 1;
    if (!on_device) {
        LBRS_CUDA(ctx, cudaMemcpyAsync(U_out, dst, field_bytes(ctx, dtype), cudaMemcpyDeviceToHost, ctx->stream));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBRS_OK;
}

lbrs_status lbrs_diagnostics(lbrs_ctx* ctx, lbrs_diag* out)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!out) return fail(ctx, LBRS_EINVAL, "out is NULL");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    const int lat = readout_lattice(ctx);
    const double vol = two_d(ctx->lattice) ? ctx->cfg.dx * ctx->cfg.dx : ctx->cfg.dx;
    double* partials = (double*)(ctx->ws + ctx->L.partials);
    double* dout = (double*)(ctx->ws + ctx->L.diag_out);
    LBRS_CUDA(ctx, launch_diag(lat, ctx->f64, own_ptr(ctx, ctx->f[ctx->cur]), ctx->N_own, ctx->N, ctx->cfg.gamma,
                               ctx->cfg.lambda, vol, partials, dout, ctx->stream));
    ctx->launches += 2;
    double h[DIAG_W];
    LBRS_CUDA(ctx, cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    memset(out, 0, sizeof *out);
    for (int k = 0; k < ctx->K; ++k) out->totals[k] = h[k];
    out->min_rho = h[4];
    out->min_p = h[5];
    out->max_lambda_local = h[6];
    out->n_nonphysical = (int64_t)h[7];
    out->n_subchar = (int64_t)h[8];
    if (out->n_nonphysical > 0) return fail(ctx, LBRS_ENONPHYS, "%lld non-physical cells at step %lld",
                                            (long long)out->n_nonphysical, (long long)ctx->step);
    if (out->n_subchar > 0) return fail(ctx, LBRS_ESUBCHAR, "%lld cells exceed lambda at step %lld",
                                        (long long)out->n_subchar, (long long)ctx->step);
    return LBRS_OK;
}

lbrs_status lbrs_boundary_flux(lbrs_ctx* ctx, double inflow[4], double outflow[4])
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!inflow || !outflow) return fail(ctx, LBRS_EINVAL, "inflow or outflow is NULL");
    if (ctx->lattice != LBRS_D2Q4 || ctx->f16 || ctx->f32u)
        return fail(ctx, LBRS_EINVAL, "the boundary balance covers D2Q4 with stored distributions (F64, F32)");
    if (ctx->solid) return fail(ctx, LBRS_EINVAL, "the boundary balance covers the domain's sides, not internal walls");
    if (ctx->halo[0] || ctx->halo[1]) return fail(ctx, LBRS_EINVAL, "the boundary balance is not defined on a cut grid");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    if (ctx->adapt_used)
        return fail(ctx, LBRS_ESTATE, "the distributions carry an adaptive lambda: the ghosts of the next step are not built");
    const double vol = ctx->cfg.dx * ctx->cfg.dx;
    double* dout = (double*)(ctx->ws + ctx->L.diag_out);
    LBRS_CUDA(ctx, ctx->f64 ? launch_boundary_flux_f64(step_args<double>(ctx, ctx->cur), vol, dout, ctx->stream)
                            : launch_boundary_flux_f32(step_args<float>(ctx, ctx->cur), vol, dout, ctx->stream));
    ctx->launches += 1;
    double h[8];
    LBRS_CUDA(ctx, cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 4; ++k) {
        inflow[k] = h[k];
        outflow[k] = h[4 + k];
    }
    return LBRS_OK;
}

lbrs_status lbrs_get_distributions(lbrs_ctx* ctx, void* dst, int on_device)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!dst) return fail(ctx, LBRS_EINVAL, "dst is NULL");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    LBRS_CUDA(ctx, copy_own_out(ctx, ctx->f[ctx->cur], dst, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    if (!on_device) LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LBRS_OK;
}

lbrs_status lbrs_set_obstacles(lbrs_ctx* ctx, const uint8_t* d_solid)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (d_solid) {
        if (ctx->lattice != LBRS_D2Q4 || ctx->f16 || ctx->f32u)
            return fail(ctx, LBRS_EINVAL, "internal walls cover the F64 and F32 D2Q4 forms");
        if (ctx->halo[0] || ctx->halo[1]) return fail(ctx, LBRS_EINVAL, "internal walls are not covered on cut grids");
        if (ctx->cfg.bc[2].kind == LBRS_BC_WALL_HALFWAY || ctx->cfg.bc[3].kind == LBRS_BC_WALL_HALFWAY)
            return fail(ctx, LBRS_EINVAL, "internal walls are not combined with halfway walls");
        std::vector<uint8_t> m((size_t)ctx->N);
        LBRS_CUDA(ctx, cudaMemcpyAsync(m.data(), d_solid, m.size(), cudaMemcpyDeviceToHost, ctx->stream));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const int64_t bad = obstacle_violations(&ctx->cfg, m.data());
        if (bad)
            return fail(ctx, LBRS_EINVAL,
                        "obstacle geometry: %lld populations of fluid cells have no known mirror "
                        "(fluid channels must be at least two cells wide)", (long long)bad);
    }
    // the captured step graphs hold the previous mask
    for (int b = 0; b < 2; ++b)
        if (ctx->graph[b]) {
            cudaGraphExecDestroy(ctx->graph[b]);
            ctx->graph[b] = nullptr;
        }
    ctx->solid = d_solid;
    return LBRS_OK;
}

// One adaptive step from the current buffer on stream s (a prep launch and a step launch).
static cudaError_t launch_adapt_pair(lbrs_ctx* ctx, int from, double safety, double t_final, cudaStream_t s)
{
    void* st = ctx->ws + ctx->L.adapt;
    cudaError_t e = launch_adapt_prep(ctx->f64, st, ctx->ws + ctx->L.ghost, ctx->gspec, ctx->cfg.gamma, ctx->cfg.dx,
                                      safety, t_final, s);
    if (e != cudaSuccess) return e;
    if (ctx->f64) return launch_adapt_step_f64(step_args<double>(ctx, from), st, ctx->cfg.gamma, s);
    return launch_adapt_step_f32(step_args<float>(ctx, from), st, ctx->cfg.gamma, s);
}

constexpr int kAdaptGraphSteps = 32;   // even: a graph returns the buffers to their parity

// The graph of kAdaptGraphSteps adaptive steps from buffer `from` for (safety, t_final).
static lbrs_status ensure_adapt_graph(lbrs_ctx* ctx, int from, double safety, double t_final)
{
    if (ctx->agraph[from] && ctx->agraph_key[0] == safety && ctx->agraph_key[1] == t_final) return LBRS_OK;
    if (ctx->agraph_key[0] != safety || ctx->agraph_key[1] != t_final) {
        for (int b = 0; b < 2; ++b)
            if (ctx->agraph[b]) {
                cudaGraphExecDestroy(ctx->agraph[b]);
                ctx->agraph[b] = nullptr;
            }
        ctx->agraph_key[0] = safety;
        ctx->agraph_key[1] = t_final;
    }
    if (!ctx->cap_stream) LBRS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    LBRS_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    int b = from;
    for (int m = 0; m < kAdaptGraphSteps && le == cudaSuccess; ++m) {
        le = launch_adapt_pair(ctx, b, safety, t_final, ctx->cap_stream);
        b ^= 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, le, "adaptive step launch during graph capture");
    }
    if (ee != cudaSuccess) return cuda_fail(ctx, ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&ctx->agraph[from], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        ctx->agraph[from] = nullptr;
        return cuda_fail(ctx, ie, "cudaGraphInstantiate");
    }
    return LBRS_OK;
}

lbrs_status lbrs_step_adaptive(lbrs_ctx* ctx, int64_t n, double safety, double t_final)
{
    NvtxRange range("lbrs_step_adaptive");
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (n < 0) return fail(ctx, LBRS_EINVAL, "negative step count");
    if (ctx->lattice != LBRS_D2Q4 || ctx->f16 || ctx->f32u || ctx->solid)
        return fail(ctx, LBRS_EINVAL, "the adaptive lambda covers the F64 and F32 D2Q4 forms without internal walls");
    if (ctx->halo[0] || ctx->halo[1])
        return fail(ctx, LBRS_EINVAL, "the adaptive lambda is a global maximum: not covered on cut grids");
    if (!(safety >= 1.0) || !isfinite(safety)) return fail(ctx, LBRS_EINVAL, "safety must be >= 1");
    if (!(t_final >= 0.0) || !isfinite(t_final)) return fail(ctx, LBRS_EINVAL, "t_final must be >= 0");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    void* st = ctx->ws + ctx->L.adapt;
    if (!ctx->adapt_ready) {
        if (t_final > 0.0 && ctx->cfg.dx / ctx->cfg.lambda > t_final)
            return fail(ctx, LBRS_EINVAL, "the first step alone (dx / lambda) passes t_final");
        LBRS_CUDA(ctx, launch_adapt_reset(st, ctx->cfg.lambda, ctx->stream));
        if (ctx->f64)
            LBRS_CUDA(ctx, launch_adapt_init_bound_f64(ctx->f[ctx->cur], ctx->N, ctx->cfg.gamma, st, ctx->stream));
        else
            LBRS_CUDA(ctx, launch_adapt_init_bound_f32(ctx->f[ctx->cur], ctx->N, ctx->cfg.gamma, st, ctx->stream));
        ctx->launches += 2;
        ctx->adapt_ready = true;
    }
    ctx->adapt_used = true;
    int64_t left = n;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LBRS_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
    if (cap == cudaStreamCaptureStatusNone && n >= kAdaptGraphSteps) {
        lbrs_status gs = ensure_adapt_graph(ctx, ctx->cur, safety, t_final);
        if (gs != LBRS_OK) return gs;
        for (; left >= kAdaptGraphSteps; left -= kAdaptGraphSteps) {
            LBRS_CUDA(ctx, cudaGraphLaunch(ctx->agraph[ctx->cur], ctx->stream));
            ctx->step += kAdaptGraphSteps;
            ctx->launches += 2 * kAdaptGraphSteps;
        }
    }
    for (; left > 0; --left) {
        LBRS_CUDA(ctx, launch_adapt_pair(ctx, ctx->cur, safety, t_final, ctx->stream));
        ctx->cur ^= 1;
        ctx->step += 1;
        ctx->launches += 2;
    }
    return LBRS_OK;
}

lbrs_status lbrs_adaptive_state(lbrs_ctx* ctx, double* t, double* lambda, int64_t* steps, int* done)
{
    if (!ctx || !t || !lambda || !steps || !done) return fail(ctx, LBRS_EINVAL, "NULL argument");
    if (!ctx->adapt_ready) {
        *t = 0.0;
        *lambda = ctx->cfg.lambda;
        *steps = 0;
        *done = 0;
        return LBRS_OK;
    }
    AdaptState h;
    LBRS_CUDA(ctx, cudaMemcpyAsync(&h, ctx->ws + ctx->L.adapt, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *t = h.t;
    *lambda = h.lam_cur;
    *steps = h.steps;
    *done = h.done;
    return LBRS_OK;
}

// ---------------------------------------------------------------- checkpoints

namespace {
// Header of a checkpoint blob; the raw distributions follow at kCkptHeader bytes.
struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t lattice, precision;
    int32_t bc_kind[4];
    int32_t reserved;
    int64_t nx, ny, step;
    double lambda, omega, gamma, dx;
    double bc_prim[4][4];
    uint64_t f_bytes;
};
constexpr size_t kCkptHeader = 256;
static_assert(sizeof(CkptHeader) <= kCkptHeader, "checkpoint header size");
constexpr char kCkptMagic[8] = {'L', 'B', 'R', 'S', 'C', 'K', 'P', '1'};

CkptHeader header_of(const lbrs_ctx* ctx)
{
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.version = 1;
    h.lattice = ctx->cfg.lattice;
    h.precision = ctx->cfg.precision;
    for (int s = 0; s < 4; ++s) {
        h.bc_kind[s] = ctx->cfg.bc[s].kind;
        for (int k = 0; k < 4; ++k) h.bc_prim[s][k] = ctx->cfg.bc[s].prim[k];
    }
    h.nx = ctx->cfg.nx;
    h.ny = ctx->cfg.ny;
    h.step = ctx->step;
    h.lambda = ctx->cfg.lambda;
    h.omega = ctx->cfg.omega;
    h.gamma = ctx->cfg.gamma;
    h.dx = ctx->cfg.dx;
    h.f_bytes = ctx->L.f_bytes;
    return h;
}
}  // namespace

lbrs_status lbrs_checkpoint_size(const lbrs_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return fail(nullptr, LBRS_EINVAL, "NULL argument");
    *bytes = kCkptHeader + ctx->L.f_bytes;
    return LBRS_OK;
}

lbrs_status lbrs_checkpoint_save(lbrs_ctx* ctx, void* dst, int on_device)
{
    if (!ctx || !dst) return fail(ctx, LBRS_EINVAL, "NULL argument");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    if (ctx->adapt_used) return fail(ctx, LBRS_EINVAL, "an adaptive run's state is not covered by checkpoints");
    unsigned char head[kCkptHeader];
    memset(head, 0, sizeof head);
    const CkptHeader h = header_of(ctx);
    memcpy(head, &h, sizeof h);
    char* d = (char*)dst;
    if (on_device) {
        LBRS_CUDA(ctx, cudaMemcpyAsync(d, head, kCkptHeader, cudaMemcpyHostToDevice, ctx->stream));
        LBRS_CUDA(ctx, copy_own_out(ctx, ctx->f[ctx->cur], d + kCkptHeader, cudaMemcpyDeviceToDevice));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // the header's host copy goes out of scope
    } else {
        memcpy(d, head, kCkptHeader);
        LBRS_CUDA(ctx, copy_own_out(ctx, ctx->f[ctx->cur], d + kCkptHeader, cudaMemcpyDeviceToHost));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBRS_OK;
}

lbrs_status lbrs_checkpoint_load(lbrs_ctx* ctx, const void* src, int on_device)
{
    if (!ctx || !src) return fail(ctx, LBRS_EINVAL, "NULL argument");
    CkptHeader h;
    const char* s = (const char*)src;
    if (on_device) {
        LBRS_CUDA(ctx, cudaMemcpyAsync(&h, s, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    } else {
        memcpy(&h, s, sizeof h);
    }
    if (memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0 || h.version != 1)
        return fail(ctx, LBRS_EINVAL, "not a checkpoint of this library (magic or version)");
    const CkptHeader want = header_of(ctx);
    bool same = h.lattice == want.lattice && h.precision == want.precision && h.nx == want.nx && h.ny == want.ny &&
                h.lambda == want.lambda && h.omega == want.omega && h.gamma == want.gamma && h.dx == want.dx &&
                h.f_bytes == want.f_bytes;
    for (int q = 0; q < 4 && same; ++q) {
        same = h.bc_kind[q] == want.bc_kind[q];
        for (int k = 0; k < 4 && same; ++k) same = h.bc_prim[q][k] == want.bc_prim[q][k];
    }
    if (!same) return fail(ctx, LBRS_EINVAL, "checkpoint of another configuration (grid, lattice, precision, "
                                             "lambda, omega, gamma, dx or boundaries differ)");
    LBRS_CUDA(ctx, copy_own_in(ctx, ctx->f[ctx->cur], s + kCkptHeader,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    if (!on_device) LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->has_state = true;
    ctx->step = h.step;
    lbrs_status rs = reset_status(ctx);
    if (rs != LBRS_OK) return rs;
    return LBRS_OK;
}

lbrs_status lbrs_set_distributions(lbrs_ctx* ctx, const void* src, int on_device, int64_t step)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!src) return fail(ctx, LBRS_EINVAL, "src is NULL");
    if (step < 0) return fail(ctx, LBRS_EINVAL, "negative step");
    LBRS_CUDA(ctx, copy_own_in(ctx, ctx->f[ctx->cur], src, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    lbrs_status rs = reset_status(ctx);
    if (rs != LBRS_OK) return rs;
    if (!on_device) LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->has_state = true;
    ctx->step = step;
    return LBRS_OK;
}

// ---------------------------------------------------------------- cuts (y-slab decomposition)

namespace {
// First stored row of the H rows an export reads (the own rows next to the side) or an
// import writes (the ghost rows beyond it); side 2 is y-lo, 3 is y-hi.
int64_t halo_first_row(const lbrs_ctx* ctx, int side, bool import)
{
    if (side == 2) return import ? 0 : ctx->row0;
    return import ? ctx->row0 + ctx->cfg.ny : ctx->row0 + ctx->cfg.ny - ctx->halo[1];
}

// Arguments of the row exchanges; the state's own exchanges also need a state.
lbrs_status halo_args(lbrs_ctx* ctx, int side, const void* buf, bool need_state = true)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!buf) return fail(ctx, LBRS_EINVAL, "halo buffer is NULL");
    if (side != 2 && side != 3) return fail(ctx, LBRS_EINVAL, "side must be 2 (y-lo) or 3 (y-hi), got %d", side);
    if (!ctx->halo[side - 2]) return fail(ctx, LBRS_EINVAL, "side %d is not a cut", side);
    if (need_state && !ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    return LBRS_OK;
}
}  // namespace

lbrs_status lbrs_halo_size(const lbrs_ctx* ctx, int side, int64_t* rows, size_t* bytes)
{
    if (!ctx || !rows || !bytes) return fail(nullptr, LBRS_EINVAL, "NULL argument");
    if (side != 2 && side != 3) return fail(nullptr, LBRS_EINVAL, "side must be 2 (y-lo) or 3 (y-hi)");
    *rows = ctx->halo[side - 2];
    *bytes = (size_t)ctx->P * (size_t)*rows * (size_t)ctx->cfg.nx * elem_bytes(ctx);
    return LBRS_OK;
}

namespace {
// The H rows next to cut `side` of a buffer in the stored layout ([planes][ny_store][nx], storage
// precision) to or from a block [planes][H][nx] elsewhere: the own rows out (export), the ghost
// rows in (import).
lbrs_status copy_rows(lbrs_ctx* ctx, int side, char* buf, int planes, void* block, bool import, int on_device)
{
    const size_t e = elem_bytes(ctx), w = (size_t)ctx->halo[side - 2] * ctx->cfg.nx * e;
    char* rows = buf + (size_t)halo_first_row(ctx, side, import) * ctx->cfg.nx * e;
    if (import)
        LBRS_CUDA(ctx, cudaMemcpy2DAsync(rows, (size_t)ctx->N * e, block, w, w, (size_t)planes,
                                         on_device ? cudaMemcpyDefault : cudaMemcpyHostToDevice, ctx->stream));
    else
        LBRS_CUDA(ctx, cudaMemcpy2DAsync(block, w, rows, (size_t)ctx->N * e, w, (size_t)planes,
                                         on_device ? cudaMemcpyDefault : cudaMemcpyDeviceToHost, ctx->stream));
    if (!on_device) LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LBRS_OK;
}
}  // namespace

lbrs_status lbrs_halo_export(lbrs_ctx* ctx, int side, void* dst, int on_device)
{
    lbrs_status st = halo_args(ctx, side, dst);
    if (st != LBRS_OK) return st;
    return copy_rows(ctx, side, ctx->f[ctx->cur], ctx->P, dst, false, on_device);
}

lbrs_status lbrs_halo_import(lbrs_ctx* ctx, int side, const void* src, int on_device)
{
    lbrs_status st = halo_args(ctx, side, src);
    if (st != LBRS_OK) return st;
    st = copy_rows(ctx, side, ctx->f[ctx->cur], ctx->P, (void*)src, true, on_device);
    if (st != LBRS_OK) return st;
    ctx->halo_left[side - 2] = ctx->halo[side - 2];
    return LBRS_OK;
}

lbrs_status lbrs_store_rows(const lbrs_ctx* ctx, int64_t* ny_store, int64_t* row0)
{
    if (!ctx || !ny_store || !row0) return fail(nullptr, LBRS_EINVAL, "NULL argument");
    *ny_store = ctx->ny_store;
    *row0 = ctx->row0;
    return LBRS_OK;
}

lbrs_status lbrs_rows_export(lbrs_ctx* ctx, int side, const void* d_buf, int planes, void* dst, int on_device)
{
    lbrs_status st = halo_args(ctx, side, dst, false);
    if (st != LBRS_OK) return st;
    if (!d_buf || planes < 1) return fail(ctx, LBRS_EINVAL, "buffer NULL or planes < 1");
    return copy_rows(ctx, side, (char*)d_buf, planes, dst, false, on_device);
}

lbrs_status lbrs_rows_import(lbrs_ctx* ctx, int side, void* d_buf, int planes, const void* src, int on_device)
{
    lbrs_status st = halo_args(ctx, side, src, false);
    if (st != LBRS_OK) return st;
    if (!d_buf || planes < 1) return fail(ctx, LBRS_EINVAL, "buffer NULL or planes < 1");
    return copy_rows(ctx, side, (char*)d_buf, planes, (void*)src, true, on_device);
}

lbrs_status lbrs_step_count(const lbrs_ctx* ctx, int64_t* steps)
{
    if (!ctx || !steps) return fail(nullptr, LBRS_EINVAL, "NULL argument");
    *steps = ctx->step;
    return LBRS_OK;
}

lbrs_status lbrs_launch_count(const lbrs_ctx* ctx, int64_t* launches)
{
    if (!ctx || !launches) return fail(nullptr, LBRS_EINVAL, "NULL argument");
    *launches = ctx->launches;
    return LBRS_OK;
}

lbrs_status lbrs_step_record(lbrs_ctx* ctx, int64_t n, void* d_U_hist)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (n < 0) return fail(ctx, LBRS_EINVAL, "negative step count");
    if (n > 0 && !d_U_hist) return fail(ctx, LBRS_EINVAL, "d_U_hist is NULL");
    if (ctx->lattice != LBRS_D2Q4 || ctx->f16 || ctx->f32u)
        return fail(ctx, LBRS_EINVAL, "recording steps cover the F64 and F32 D2Q4 forms only");
    if (ctx->halo[0] || ctx->halo[1]) {
        lbrs_status hs = adjoint_supported(ctx);
        if (hs != LBRS_OK) return hs;
        for (int h = 0; h < 2; ++h)
            if (ctx->halo[h] && n > ctx->halo_left[h])
                return fail(ctx, LBRS_ESTATE, "%lld recording steps requested, but the ghost rows of the %s cut "
                            "cover %lld more steps: import the neighbour's rows first", (long long)n,
                            h ? "y-hi" : "y-lo", (long long)ctx->halo_left[h]);
        for (int h = 0; h < 2; ++h)
            if (ctx->halo[h]) ctx->halo_left[h] -= n;
    }
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    lbrs_status st = record_steps(ctx, n, (char*)d_U_hist);
    if (st != LBRS_OK) return st;
    ctx->step += n;
    return LBRS_OK;
}

lbrs_status lbrs_adjoint_seed(lbrs_ctx* ctx, const void* d_dLdU, int dtype, void* d_gbar)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!d_dLdU || !d_gbar) return fail(ctx, LBRS_EINVAL, "NULL buffer");
    if (dtype != LBRS_F64 && dtype != LBRS_F32) return fail(ctx, LBRS_EINVAL, "dtype must be LBRS_F64 or LBRS_F32");
    LBRS_CUDA(ctx, launch_adjoint_seed(ctx->Q, ctx->K, ctx->f64, d_dLdU, dtype == LBRS_F32, d_gbar, ctx->N, ctx->stream));
    ctx->launches += 1;
    return LBRS_OK;
}

lbrs_status lbrs_vjp_loss(lbrs_ctx* ctx, const void* d_rho_target, int dtype, void* d_gbar, double* loss)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!d_rho_target || !d_gbar) return fail(ctx, LBRS_EINVAL, "NULL buffer");
    if (dtype != LBRS_F64 && dtype != LBRS_F32) return fail(ctx, LBRS_EINVAL, "dtype must be LBRS_F64 or LBRS_F32");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    if (ctx->f16 || ctx->f32u) return fail(ctx, LBRS_EINVAL, "the adjoint covers the F64 and F32 forms only");
    const double vol = two_d(ctx->lattice) ? ctx->cfg.dx * ctx->cfg.dx : ctx->cfg.dx;
    double* partials = (double*)(ctx->ws + ctx->L.partials);
    double* dout = (double*)(ctx->ws + ctx->L.diag_out);
    // own rows only (a cut context's buffers hold ghost rows, which the loss does not cover)
    const size_t own = (size_t)ctx->row0 * ctx->cfg.nx;
    LBRS_CUDA(ctx, launch_density_loss(ctx->Q, ctx->K, ctx->f64, own_ptr(ctx, ctx->f[ctx->cur]),
                                       (const char*)d_rho_target + own * (dtype == LBRS_F64 ? 8 : 4),
                                       dtype == LBRS_F32, (char*)d_gbar + own * elem_bytes(ctx), ctx->N_own, ctx->N,
                                       vol, partials, dout, ctx->stream));
    ctx->launches += 2;
    if (loss) {
        LBRS_CUDA(ctx, cudaMemcpyAsync(loss, dout, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        LBRS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return LBRS_OK;
}

lbrs_status lbrs_adjoint_step(lbrs_ctx* ctx, const void* d_U_next, const void* d_gbar_in, void* d_gbar_out)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    lbrs_status st = adjoint_supported(ctx);
    if (st != LBRS_OK) return st;
    if (!d_U_next || !d_gbar_in || !d_gbar_out) return fail(ctx, LBRS_EINVAL, "NULL buffer");
    if (d_gbar_in == d_gbar_out) return fail(ctx, LBRS_EINVAL, "d_gbar_in and d_gbar_out must differ");
    LBRS_CUDA(ctx, launch_adjoint_step_raw(ctx, d_U_next, d_gbar_in, d_gbar_out));
    ctx->launches += 1;
    return LBRS_OK;
}

lbrs_status lbrs_vjp_equilibrium(lbrs_ctx* ctx, const void* d_U0, const void* d_gbar0, void* d_gradU0)
{
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    lbrs_status st = adjoint_supported(ctx);
    if (st != LBRS_OK) return st;
    if (!d_U0 || !d_gbar0 || !d_gradU0) return fail(ctx, LBRS_EINVAL, "NULL buffer");
    LBRS_CUDA(ctx, launch_vjp_eq_raw(ctx, d_U0, d_gbar0, d_gradU0));
    ctx->launches += 1;
    return LBRS_OK;
}

lbrs_status lbrs_adjoint_workspace_size(const lbrs_ctx* ctx, int64_t n_steps, int64_t segment, size_t* bytes)
{
    if (!ctx || !bytes) return fail(nullptr, LBRS_EINVAL, "NULL argument");
    if (n_steps < 1 || segment < 1) return fail(nullptr, LBRS_EINVAL, "n_steps and segment must be >= 1");
    *bytes = adj_layout(ctx, n_steps, segment).total;
    return LBRS_OK;
}

lbrs_status lbrs_forward_checkpointed(lbrs_ctx* ctx, int64_t n_steps, int64_t segment, void* d_adj_ws, size_t bytes)
{
    NvtxRange range("lbrs_forward_checkpointed");
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    lbrs_status st = adjoint_supported(ctx);
    if (st != LBRS_OK) return st;
    if (ctx->halo[0] || ctx->halo[1])
        return fail(ctx, LBRS_EINVAL, "the checkpointed driver steps without the neighbours' rows: on a cut grid, "
                                      "drive recording and adjoint steps between row exchanges");
    if (n_steps < 1 || segment < 1) return fail(ctx, LBRS_EINVAL, "n_steps and segment must be >= 1");
    if (!ctx->has_state) return fail(ctx, LBRS_ESTATE, "no state set");
    if (!d_adj_ws || (uintptr_t)d_adj_ws % kAlign) return fail(ctx, LBRS_EINVAL, "adjoint workspace NULL or not 256-byte aligned");
    const AdjLayout A = adj_layout(ctx, n_steps, segment);
    if (bytes < A.total) return fail(ctx, LBRS_ENOMEM, "adjoint workspace has %zu bytes, needs %zu", bytes, A.total);
    char* ws = (char*)d_adj_ws;
    ctx->adj_ws = nullptr;
    ctx->adj_step0 = ctx->step;
    for (int64_t s = 0; s < A.nseg; ++s) {
        LBRS_CUDA(ctx, cudaMemcpyAsync(ws + A.ckpt0 + s * A.ckpt_stride, ctx->f[ctx->cur], ctx->L.f_bytes,
                                       cudaMemcpyDeviceToDevice, ctx->stream));
        const int64_t len = (s + 1) * segment <= n_steps ? segment : n_steps - s * segment;
        st = lbrs_step(ctx, len);
        if (st != LBRS_OK) return st;
    }
    LBRS_CUDA(ctx, cudaMemcpyAsync(ws + A.ckpt0 + A.nseg * A.ckpt_stride, ctx->f[ctx->cur], ctx->L.f_bytes,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->adj_ws = ws;
    ctx->adj_bytes = bytes;
    ctx->adj_n = n_steps;
    ctx->adj_seg = segment;
    return LBRS_OK;
}

lbrs_status lbrs_backward_checkpointed(lbrs_ctx* ctx, void* d_adj_ws, const void* d_gbar_T, void* d_gradU0)
{
    NvtxRange range("lbrs_backward_checkpointed");
    if (!ctx) return fail(nullptr, LBRS_EINVAL, "ctx is NULL");
    if (!ctx->adj_ws || d_adj_ws != ctx->adj_ws)
        return fail(ctx, LBRS_ESTATE, "no checkpointed forward run recorded on this adjoint workspace");
    if (!d_gbar_T || !d_gradU0) return fail(ctx, LBRS_EINVAL, "NULL buffer");
    const AdjLayout A = adj_layout(ctx, ctx->adj_n, ctx->adj_seg);
    char* ws = ctx->adj_ws;
    char* g[2] = {ws + A.gbar0, ws + A.gbar1};
    TileMap gmap[2];                 // tensor maps of the two k buffers (FP32 fused sweep)
    for (int b = 0; b < 2; ++b)
        if (ctx->f64 || !encode_f32_tile_map(&gmap[b], (const float*)g[b], ctx->cfg.nx, ctx->cfg.ny)) gmap[b].valid = 0;
    char* uhist = ws + A.uhist;
    const size_t ustride = (size_t)ctx->K * ctx->N * elem_bytes(ctx);
    LBRS_CUDA(ctx, cudaMemcpyAsync(g[0], d_gbar_T, ctx->L.f_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    int gc = 0;
    for (int64_t s = A.nseg - 1; s >= 0; --s) {
        NvtxRange seg_range("adjoint segment");
        const int64_t start = s * ctx->adj_seg;
        const int64_t len = start + ctx->adj_seg <= ctx->adj_n ? ctx->adj_seg : ctx->adj_n - start;
        // recompute the segment from its checkpoint, recording U^{start+1 .. start+len}
        LBRS_CUDA(ctx, cudaMemcpyAsync(ctx->f[ctx->cur], ws + A.ckpt0 + s * A.ckpt_stride, ctx->L.f_bytes,
                                       cudaMemcpyDeviceToDevice, ctx->stream));
        lbrs_status rs = record_steps(ctx, len, uhist);
        if (rs != LBRS_OK) return rs;
        if (fused2_f32(ctx)) {
            // sweep on k = fbar: k^{end} from g^{end}, two steps per launch while U_{s-1} and
            // U_{s-2} lie in this segment, one more step if needed, then the pull that hands
            // g^{start} to the earlier segment.  uhist[m] holds U_{start+m+1}.
            // at omega = 1 the sweep's state is the same for every population: kept as 4 fields
            const bool uform = ctx->cfg.omega == 1.0 && adj_uform_enabled();
            AdjArgs<float> aa = adj_args<float>(ctx, uhist + (len - 1) * ustride, g[gc], g[gc ^ 1]);
            LBRS_CUDA(ctx, uform ? launch_adj_local_u_f32(aa, ctx->stream) : launch_adj_local_f32(aa, ctx->stream));
            gc ^= 1;
            int64_t t = len;                                   // g[gc] holds k^{start+t}
            for (; t >= 3; t -= 2) {
                aa = adj_args<float>(ctx, uhist + (t - 2) * ustride, g[gc], g[gc ^ 1]);
                const float* U2 = (const float*)(uhist + (t - 3) * ustride);
                LBRS_CUDA(ctx, uform ? launch_adj_fused2_u_f32(aa, U2, ctx->stream)
                                     : launch_adj_fused2_f32(aa, U2, &gmap[gc], wait_flag(ctx), ctx->stream));
                gc ^= 1;
            }
            if (t == 2) {
                aa = adj_args<float>(ctx, uhist, g[gc], g[gc ^ 1]);
                LBRS_CUDA(ctx, uform ? launch_adj_pull_u_f32(aa, ctx->stream) : launch_adj_pull_f32(aa, ctx->stream));
                gc ^= 1;
            }
            aa = adj_args<float>(ctx, nullptr, g[gc], g[gc ^ 1]);
            LBRS_CUDA(ctx, uform ? launch_adj_pull_u_f32(aa, ctx->stream) : launch_adj_pull_f32(aa, ctx->stream));
            gc ^= 1;
            ctx->launches += 2 + (len - 1) / 2 + ((len - 1) % 2);
        } else {
            for (int64_t m = len - 1; m >= 0; --m) {
                LBRS_CUDA(ctx, launch_adjoint_step_raw(ctx, uhist + m * ustride, g[gc], g[gc ^ 1]));
                gc ^= 1;
                ctx->launches += 1;
            }
        }
    }
    // dL/dU0 = J_E(U0)^T gbar^0 with U0 the moments of the first checkpoint
    const int lat = LAT_D2Q4;
    LBRS_CUDA(ctx, launch_moments(lat, ctx->f64, ws + A.ckpt0, uhist, ctx->f64 ? 0 : 1, ctx->N, ctx->N, ctx->stream));
    LBRS_CUDA(ctx, launch_vjp_eq_raw(ctx, uhist, g[gc], d_gradU0));
    ctx->launches += 2;
    // restore the final forward state
    LBRS_CUDA(ctx, cudaMemcpyAsync(ctx->f[ctx->cur], ws + A.ckpt0 + A.nseg * A.ckpt_stride, ctx->L.f_bytes,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->step = ctx->adj_step0 + ctx->adj_n;
    return LBRS_OK;
}

const char* lbrs_last_error(const lbrs_ctx* ctx) { return ctx ? ctx->err : g_err; }

}  // extern "C"
