// FP64 kernels of the LBRS solver: the FP64 time step and every helper whose
// arithmetic is FP64 whatever the storage precision (initial equilibria,
// Dirichlet ghost tables, moments read-out, diagnostics).
//
// Compiled with -fmad=false: no FMA contraction, IEEE division and square
// root, so each expression rounds as written.
#include <math.h>

#include "lbrs_kernels.cuh"
#include "lbrs_batch.cuh"
#include "lbrs_launch.h"

namespace lbrs {

namespace {

constexpr int kThreads = 256;
constexpr int kDiagBlocks = 608;   // 4 x 152 SMs; fixed so the reduction order never changes

int grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = 152 * 16;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

template <int LAT>
struct Dims;
template <>
struct Dims<LAT_D2Q4> {
    static constexpr int Q = 4, K = 4;
};
template <>
struct Dims<LAT_D1Q2> {
    static constexpr int Q = 2, K = 3;
};
template <>
struct Dims<LAT_U2D> {
    static constexpr int Q = 1, K = 4;
};
template <>
struct Dims<LAT_D1Q3> {
    static constexpr int Q = 3, K = 3;
};
template <>
struct Dims<LAT_D2Q4S> {
    static constexpr int Q = 4, K = 1;
};

// f^eq in FP64 for either lattice, e[q*K + k]
template <int LAT>
__device__ __forceinline__ void equilibria_flat(const double* U, double gm1, double c, double* e)
{
    if constexpr (LAT == LAT_D2Q4S) {
        equilibria2ds<double>(U[0], c, e);
    } else if constexpr (LAT == LAT_D2Q4) {
        double t[4][4];
        equilibria2d<double>(U, gm1, c, t);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) e[q * 4 + k] = t[q][k];
    } else if constexpr (LAT == LAT_D1Q3) {
        double t[3][3];
        equilibria1d3<double>(U, gm1, c, t);
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) e[q * 3 + k] = t[q][k];
    } else {
        double t[2][3];
        equilibria1d<double>(U, gm1, c, t);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) e[q * 3 + k] = t[q][k];
    }
}

template <int LAT>
__device__ __forceinline__ void prim_to_cons(const double* w, double gamma, double* U)
{
    if constexpr (LAT == LAT_D2Q4S) U[0] = w[0];
    else if constexpr (LAT == LAT_D2Q4) prim_to_cons2d(w, gamma, U);
    else prim_to_cons1d(w, gamma, U);
}

template <typename Ts, int LAT>
__global__ void ghost_kernel(GhostSpec g, double gamma, double c, Ts* ghost)
{
    constexpr int Q = Dims<LAT>::Q, K = Dims<LAT>::K;
    const int side = threadIdx.x;
    if (side >= 4) return;
    double e[16];
    static_assert(Q * K <= GHOST_STRIDE, "ghost table stride");
    for (int n = 0; n < GHOST_STRIDE; ++n) e[n] = 0.0;
    if (g.kind[side] == BC_DIRICHLET) {
        if constexpr (LAT == LAT_D2Q4S) {
            e[0] = g.prim[side][0];            // the profile: u0, slope, dx
            e[1] = g.prim[side][1];
            e[2] = g.dx;
        } else {
            double U[4];
            prim_to_cons<LAT>(g.prim[side], gamma, U);
            equilibria_flat<LAT>(U, gamma - 1.0, c, e);
        }
    }
    for (int n = 0; n < GHOST_STRIDE; ++n) ghost[side * GHOST_STRIDE + n] = (Ts)e[n];
}

template <typename Tin, typename Ts, int LAT>
__global__ void __launch_bounds__(kThreads) set_state_kernel(const Tin* __restrict__ W, Ts* __restrict__ fs,
                                                             int64_t N, int64_t P, int kind, double gamma,
                                                             double c)
{
    constexpr int Q = Dims<LAT>::Q, K = Dims<LAT>::K;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double w[4], U[4], e[16];
#pragma unroll
        for (int k = 0; k < K; ++k) w[k] = (double)W[k * N + i];
        if (kind == KIND_PRIMITIVE) {
            prim_to_cons<LAT>(w, gamma, U);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) U[k] = w[k];
        }
        equilibria_flat<LAT>(U, gamma - 1.0, c, e);
#pragma unroll
        for (int n = 0; n < Q * K; ++n) fs[n * P + i] = (Ts)e[n];
    }
}

template <typename Ts, typename To, int LAT>
__global__ void __launch_bounds__(kThreads) moments_kernel(const Ts* __restrict__ fs, To* __restrict__ U, int64_t N,
                                                          int64_t P)
{
    constexpr int Q = Dims<LAT>::Q, K = Dims<LAT>::K;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = (double)fs[(0 * K + k) * P + i];
#pragma unroll
            for (int q = 1; q < Q; ++q) s += (double)fs[(q * K + k) * P + i];
            U[k * N + i] = (To)s;
        }
    }
}

// ---------------------------------------------------------------- diagnostics

struct DiagAcc {
    double tot[4];
    double min_rho, min_p, max_lam, nbad, nsub;
};

__device__ __forceinline__ void diag_combine(DiagAcc& a, const DiagAcc& b)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) a.tot[k] += b.tot[k];
    a.min_rho = fmin(a.min_rho, b.min_rho);
    a.min_p = fmin(a.min_p, b.min_p);
    a.max_lam = fmax(a.max_lam, b.max_lam);
    a.nbad += b.nbad;
    a.nsub += b.nsub;
}

__device__ __forceinline__ DiagAcc diag_shfl_down(const DiagAcc& a, int off)
{
    DiagAcc b;
#pragma unroll
    for (int k = 0; k < 4; ++k) b.tot[k] = __shfl_down_sync(0xffffffffu, a.tot[k], off);
    b.min_rho = __shfl_down_sync(0xffffffffu, a.min_rho, off);
    b.min_p = __shfl_down_sync(0xffffffffu, a.min_p, off);
    b.max_lam = __shfl_down_sync(0xffffffffu, a.max_lam, off);
    b.nbad = __shfl_down_sync(0xffffffffu, a.nbad, off);
    b.nsub = __shfl_down_sync(0xffffffffu, a.nsub, off);
    return b;
}

// Per-cell checks of Sections II.A/II.D: rho > 0, p > 0, finite moments, and
// the local bound |u| + a (1-D) or max(|u+v|, |u-v|) + sqrt(2) a (2-D) <= lambda.
// The checks run in the storage precision R (FP64 arithmetic is slow on this
// GPU and FP32 states gain nothing from it); the totals accumulate in FP64.
template <typename Ts, int LAT>
__global__ void __launch_bounds__(kThreads) diag_partial_kernel(const Ts* __restrict__ fs, int64_t N, int64_t P,
                                                                double gamma, double lambda,
                                                                double* __restrict__ partials)
{
    constexpr int Q = Dims<LAT>::Q, K = Dims<LAT>::K;
    using R = Ts;
    const R g = (R)gamma, gm1 = (R)(gamma - 1.0), lam_max = (R)lambda;
    DiagAcc acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.tot[k] = 0.0;
    acc.min_rho = acc.min_p = INFINITY;
    acc.max_lam = 0.0;
    acc.nbad = acc.nsub = 0.0;
    R mn_rho = (R)INFINITY, mn_p = (R)INFINITY, mx_lam = (R)0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        R U[4] = {0, 0, 0, 0};
        bool finite = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            R s = fs[(0 * K + k) * P + i];
#pragma unroll
            for (int q = 1; q < Q; ++q) s += fs[(q * K + k) * P + i];
            U[k] = s;
            acc.tot[k] += (double)s;
            finite = finite && isfinite(s);
        }
        R p, lam;
        if constexpr (K == 1) {
            // the scalar law: no density or pressure; f^eq is monotone in u iff lambda >= |u| + 1
            p = (R)1;
            lam = fabs(U[0]) + (R)1;
        } else if constexpr (K == 4) {
            const R inv = (R)1 / U[0];
            const R u = U[1] * inv, v = U[2] * inv;
            p = gm1 * (U[3] - (R)0.5 * (U[1] * u + U[2] * v));
            const R s1 = fabs(u + v), s2 = fabs(u - v);
            lam = (s1 > s2 ? s1 : s2) + sqrt((R)2 * g * p * inv);
        } else {
            const R inv = (R)1 / U[0];
            const R u = U[1] * inv;
            p = gm1 * (U[2] - (R)0.5 * (U[1] * u));
            lam = fabs(u) + sqrt(g * p * inv);
            if constexpr (LAT == LAT_D1Q3) lam *= (R)1.224744871391589;   // sqrt(3/2)
        }
        if (finite) {
            mn_rho = fmin(mn_rho, U[0]);
            mn_p = fmin(mn_p, p);
        }
        if (!finite || (K > 1 && (!(U[0] > (R)0) || !(p > (R)0)))) {
            acc.nbad += 1.0;
        } else {
            mx_lam = fmax(mx_lam, lam);
            if (lam > lam_max) acc.nsub += 1.0;
        }
    }
    acc.min_rho = (double)mn_rho;
    acc.min_p = (double)mn_p;
    acc.max_lam = (double)mx_lam;
    // warp, then block, in a fixed order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) diag_combine(acc, diag_shfl_down(acc, off));
    __shared__ DiagAcc warp_acc[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        DiagAcc b = warp_acc[0];
        for (int w = 1; w < kThreads / 32; ++w) diag_combine(b, warp_acc[w]);
        double* out = partials + (int64_t)blockIdx.x * DIAG_W;
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = b.tot[k];
        out[4] = b.min_rho;
        out[5] = b.min_p;
        out[6] = b.max_lam;
        out[7] = b.nbad;
        out[8] = b.nsub;
        out[9] = 0.0;
    }
}

__global__ void diag_final_kernel(const double* __restrict__ partials, int nblocks, double cell_volume,
                                  double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    double mn_r = INFINITY, mn_p = INFINITY, mx_l = 0.0, nb = 0.0, ns = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double* p = partials + (int64_t)b * DIAG_W;
        for (int k = 0; k < 4; ++k) tot[k] += p[k];
        mn_r = fmin(mn_r, p[4]);
        mn_p = fmin(mn_p, p[5]);
        mx_l = fmax(mx_l, p[6]);
        nb += p[7];
        ns += p[8];
    }
    for (int k = 0; k < 4; ++k) out[k] = tot[k] * cell_volume;
    out[4] = mn_r;
    out[5] = mn_p;
    out[6] = mx_l;
    out[7] = nb;
    out[8] = ns;
    out[9] = 0.0;
}

template <typename Ts, typename Tin>
__global__ void __launch_bounds__(kThreads) adjoint_seed_kernel(int Q, int K, const Tin* __restrict__ dLdU,
                                                                Ts* __restrict__ gbar, int64_t N)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < K; ++k) {
            const Ts g = (Ts)dLdU[k * N + i];
            for (int q = 0; q < Q; ++q) gbar[(q * K + k) * N + i] = g;
        }
}

template <typename Ts, typename Tt>
__global__ void __launch_bounds__(kThreads) density_loss_kernel(int Q, int K, const Ts* __restrict__ fs,
                                                                const Tt* __restrict__ target, Ts* __restrict__ gbar,
                                                                int64_t N, int64_t P, double cell,
                                                                double* __restrict__ partials)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double rho = (double)fs[i];
        for (int q = 1; q < Q; ++q) rho += (double)fs[(q * K) * P + i];
        const double r = rho - (double)target[i];
        acc += 0.5 * r * r;
        const Ts g = (Ts)(r * cell);
        for (int q = 0; q < Q; ++q) {
            gbar[(q * K) * P + i] = g;
            for (int k = 1; k < K; ++k) gbar[(q * K + k) * P + i] = (Ts)0;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    __shared__ double warp_acc[kThreads / 32];
    if ((threadIdx.x & 31) == 0) warp_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = warp_acc[0];
        for (int w = 1; w < kThreads / 32; ++w) b += warp_acc[w];
        partials[blockIdx.x] = b;
    }
}

__global__ void sum_final_kernel(const double* __restrict__ partials, int n, double scale, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += partials[b];
    out[0] = s * scale;
}

// Batched tubes: f = f^eq(U(W)) with the cell's own tube lambda, in FP64.
template <typename Tin, typename Ts>
__global__ void __launch_bounds__(kThreads) batch_set_state_kernel(const Tin* __restrict__ W, Ts* __restrict__ fs,
                                                                   int64_t N, int kind, double gamma,
                                                                   const int64_t* __restrict__ tube_off, int64_t nb,
                                                                   const double* __restrict__ tube_lam, int q)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nb - 1;             // last tube with off <= i
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (tube_off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const double c = 1.0 / (2.0 * tube_lam[lo]);
        double w[3], U[3], e[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) w[k] = (double)W[k * N + i];
        if (kind == KIND_PRIMITIVE) {
            prim_to_cons1d(w, gamma, U);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) U[k] = w[k];
        }
        if (q == 3) equilibria_flat<LAT_D1Q3>(U, gamma - 1.0, c, e);
        else equilibria_flat<LAT_D1Q2>(U, gamma - 1.0, c, e);
        for (int n = 0; n < 3 * q; ++n) fs[n * N + i] = (Ts)e[n];
    }
}

// Record of the periodic checks: [0] first bad step (-1 none), [1] non-physical
// cells then, [2] cells over lambda then, [3] max local bound over all checks.
__global__ void status_reset_kernel(double* status)
{
    if (threadIdx.x == 0) {
        status[0] = -1.0;
        status[1] = status[2] = status[3] = 0.0;
    }
}

__global__ void status_update_kernel(const double* __restrict__ diag, double* __restrict__ status, double step)
{
    if (threadIdx.x != 0) return;
    status[3] = fmax(status[3], diag[6]);
    if ((diag[7] > 0.0 || diag[8] > 0.0) && status[0] < 0.0) {
        status[0] = step;
        status[1] = diag[7];
        status[2] = diag[8];
    }
}

// Adaptive lambda: reset the run's record (time 0, the configured lambda).
__global__ void adapt_reset_kernel(AdaptState* st, double lambda)
{
    if (threadIdx.x != 0) return;
    for (int n = 0; n < 3; ++n) st->bound_bits[n] = 0ull;
    st->t = 0.0;
    st->lam_cur = lambda;
    st->c_new = 1.0 / (4.0 * lambda);
    st->steps = 0;
    st->last = st->done = st->slot_cur = st->skip = 0;
}

// Adaptive lambda, before each step (one thread; FP64 without contraction, the
// oracle's expressions): the next lambda from the bound of the current state and of
// the Dirichlet states, the stop at t_final, the clock, the ghosts of this step's
// stream (with the current lambda) and a cleared slot for the step's bound.
template <typename Ts>
__global__ void adapt_prep_kernel(AdaptState* st, Ts* ghost, GhostSpec g, double gamma, double dx, double safety,
                                  double t_final)
{
    if (threadIdx.x != 0) return;
    if (st->done) {
        st->skip = 1;
        return;
    }
    st->skip = 0;
    double bound = __longlong_as_double((long long)st->bound_bits[st->slot_cur]);
    double Ub[4][4];
    for (int s = 0; s < 4; ++s) {
        if (g.kind[s] != BC_DIRICHLET) continue;
        prim_to_cons2d(g.prim[s], gamma, Ub[s]);
        bound = fmax(bound, bound2d<double>(Ub[s], gamma));
    }
    const double t_next = st->last ? t_final : st->t + dx / st->lam_cur;
    double lam_new = safety * bound;
    int next_last = 0;
    if (!st->last && t_final > 0.0 && t_next + dx / lam_new >= t_final) {
        lam_new = dx / (t_final - t_next);
        next_last = 1;
    }
    const double c_cur = 1.0 / (4.0 * st->lam_cur);
    for (int s = 0; s < 4; ++s) {
        if (g.kind[s] != BC_DIRICHLET) continue;
        double e[4][4];
        equilibria2d<double>(Ub[s], gamma - 1.0, c_cur, e);
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < 4; ++k) ghost[s * GHOST_STRIDE + q * 4 + k] = (Ts)e[q][k];
    }
    st->c_new = 1.0 / (4.0 * lam_new);
    const int acc = (st->slot_cur + 1) % 3;
    st->bound_bits[acc] = 0ull;
    st->slot_cur = acc;
    st->t = t_next;
    st->lam_cur = lam_new;
    st->steps += 1;
    if (st->last) st->done = 1;
    st->last = next_last;
}

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_status_reset(double* status, cudaStream_t s)
{
    status_reset_kernel<<<1, 32, 0, s>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_status_update(const double* diag_out, double* status, int64_t step, cudaStream_t s)
{
    status_update_kernel<<<1, 32, 0, s>>>(diag_out, status, (double)step);
    return cudaGetLastError();
}

cudaError_t launch_batch_set_state(int storage_f64, const void* W, int w_dtype, int kind, void* fs, int64_t N,
                                   const int64_t* tube_off, int64_t nb, const double* tube_lam, double gamma, int q,
                                   cudaStream_t s)
{
    const int g = grid_for(N);
    if (storage_f64) {
        if (w_dtype == 0) batch_set_state_kernel<double, double><<<g, kThreads, 0, s>>>((const double*)W, (double*)fs, N, kind, gamma, tube_off, nb, tube_lam, q);
        else batch_set_state_kernel<float, double><<<g, kThreads, 0, s>>>((const float*)W, (double*)fs, N, kind, gamma, tube_off, nb, tube_lam, q);
    } else {
        if (w_dtype == 0) batch_set_state_kernel<double, float><<<g, kThreads, 0, s>>>((const double*)W, (float*)fs, N, kind, gamma, tube_off, nb, tube_lam, q);
        else batch_set_state_kernel<float, float><<<g, kThreads, 0, s>>>((const float*)W, (float*)fs, N, kind, gamma, tube_off, nb, tube_lam, q);
    }
    return cudaGetLastError();
}

static dim3 grid2d(int nx, int ny, dim3 block)
{
    return dim3((unsigned)((nx + block.x - 1) / block.x), (unsigned)((ny + block.y - 1) / block.y));
}

// ---------------------------------------------------------------- boundary balance (D2Q4)
//
// The populations that the next step moves across the domain's sides, summed in FP64 per field:
// inflow, the populations of side cells whose pull source lies beyond a non-periodic side, with
// the values the step gives them (pull_edge_2d: a Dirichlet ghost, the clamped cell's population,
// a wall relation); outflow, the current post-collision populations of side cells whose
// destination x + c_q lies beyond a non-periodic side.  Every other population stays inside, so
// the totals of the next state are the current ones plus inflow minus outflow (the collision
// keeps the moments).  One block visits each side cell once in a fixed order and reduces in a
// fixed tree: the sums are bitwise reproducible.  out[0..3] inflow, out[4..7] outflow, times vol.
constexpr int kFluxThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFluxThreads) boundary_flux2d_kernel(const StepArgs<T> a, double vol, double* out)
{
    __shared__ double red[8][kFluxThreads];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int nx = a.nx, ny = a.ny;
    const int64_t rows = ny > 1 ? 2 : 1;                       // the bottom row, and the top one
    const int64_t inner = ny > 2 ? ny - 2 : 0;                 // rows between them
    const int64_t cols = nx > 1 ? 2 : 1;                       // their first and last cells
    const int64_t P = rows * nx + cols * inner;
    const bool px = a.bc[0] == BC_PERIODIC, py = a.bc[2] == BC_PERIODIC;
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    for (int64_t p = threadIdx.x; p < P; p += kFluxThreads) {
        int i, j;
        if (p < nx) {
            i = (int)p;
            j = 0;
        } else if (p < rows * nx) {
            i = (int)(p - nx);
            j = ny - 1;
        } else {
            const int64_t r = p - rows * nx;
            j = 1 + (int)(r % inner);
            i = r / inner ? nx - 1 : 0;
        }
        T f[4][4];
        pull_edge_2d<T>(a, i, j, f);
        const int64_t c = (int64_t)j * nx + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int si = i - SX[q], sj = j - SY[q], di = i + SX[q], dj = j + SY[q];
            const bool in = (!px && (si < 0 || si >= nx)) || (!py && (sj < 0 || sj >= ny));
            const bool leaves = (!px && (di < 0 || di >= nx)) || (!py && (dj < 0 || dj >= ny));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (in) acc[k] += (double)f[q][k];
                if (leaves) acc[4 + k] += (double)a.src[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 50)];
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) red[m][threadIdx.x] = acc[m];
    __syncthreads();
    for (int h = kFluxThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int m = 0; m < 8; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 8) out[threadIdx.x] = red[threadIdx.x][0] * vol;
}

cudaError_t launch_boundary_flux_f64(const StepArgs<double>& a, double vol, double* out, cudaStream_t s)
{
    boundary_flux2d_kernel<double><<<1, kFluxThreads, 0, s>>>(a, vol, out);
    return cudaGetLastError();
}

cudaError_t launch_boundary_flux_f32(const StepArgs<float>& a, double vol, double* out, cudaStream_t s)
{
    boundary_flux2d_kernel<float><<<1, kFluxThreads, 0, s>>>(a, vol, out);
    return cudaGetLastError();
}

cudaError_t launch_step_record_f64(const StepArgs<double>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    if (a.solid) step2d_obstacle_kernel<double, true><<<grid2d(a.nx, a.ny, block), block, 0, s>>>(a);
    else step2d_kernel<double, true><<<grid2d(a.nx, a.ny, block), block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_f64(const AdjArgs<double>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    adjoint2d_kernel<double><<<grid2d(a.nx, a.ny, block), block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_vjp_equilibrium_f64(const AdjArgs<double>& a, cudaStream_t s)
{
    vjp_equilibrium2d_kernel<double><<<grid_for(a.N), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(int Q, int K, int storage_f64, const void* dLdU, int in_dtype, void* gbar, int64_t N,
                                cudaStream_t s)
{
    const int g = grid_for(N);
    if (storage_f64) {
        if (in_dtype == 0) adjoint_seed_kernel<double, double><<<g, kThreads, 0, s>>>(Q, K, (const double*)dLdU, (double*)gbar, N);
        else adjoint_seed_kernel<double, float><<<g, kThreads, 0, s>>>(Q, K, (const float*)dLdU, (double*)gbar, N);
    } else {
        if (in_dtype == 0) adjoint_seed_kernel<float, double><<<g, kThreads, 0, s>>>(Q, K, (const double*)dLdU, (float*)gbar, N);
        else adjoint_seed_kernel<float, float><<<g, kThreads, 0, s>>>(Q, K, (const float*)dLdU, (float*)gbar, N);
    }
    return cudaGetLastError();
}

cudaError_t launch_density_loss(int Q, int K, int storage_f64, const void* fs, const void* target, int t_dtype,
                                void* gbar, int64_t N, int64_t plane, double cell_volume, double* partials, double* out,
                                cudaStream_t s)
{
    const int g = kDiagBlocks;
    if (storage_f64) {
        if (t_dtype == 0) density_loss_kernel<double, double><<<g, kThreads, 0, s>>>(Q, K, (const double*)fs, (const double*)target, (double*)gbar, N, plane, cell_volume, partials);
        else density_loss_kernel<double, float><<<g, kThreads, 0, s>>>(Q, K, (const double*)fs, (const float*)target, (double*)gbar, N, plane, cell_volume, partials);
    } else {
        if (t_dtype == 0) density_loss_kernel<float, double><<<g, kThreads, 0, s>>>(Q, K, (const float*)fs, (const double*)target, (float*)gbar, N, plane, cell_volume, partials);
        else density_loss_kernel<float, float><<<g, kThreads, 0, s>>>(Q, K, (const float*)fs, (const float*)target, (float*)gbar, N, plane, cell_volume, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_final_kernel<<<1, 32, 0, s>>>(partials, g, cell_volume, out);
    return cudaGetLastError();
}

cudaError_t launch_step_f64(int lattice, const StepArgs<double>& a, cudaStream_t s)
{
    if (lattice == LAT_D2Q4) {
        const dim3 block(128, 2);
        unsigned gy = (unsigned)((a.ny + block.y - 1) / block.y);
        const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), gy);
        if (a.solid) step2d_obstacle_kernel<double><<<grid, block, 0, s>>>(a);
        else step2d_kernel<double><<<grid, block, 0, s>>>(a);
    } else if (lattice == LAT_D2Q4S) {
        const dim3 block(128, 2);
        step2ds_kernel<double><<<grid2d(a.nx, a.ny, block), block, 0, s>>>(a);
    } else if (lattice == LAT_D1Q3) {
        step1d_q3_kernel<double><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    } else {
        step1d_kernel<double><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_ghost(int lattice, int storage_f64, const GhostSpec& g, double gamma, double c, void* ghost,
                         cudaStream_t s)
{
    if (lattice == LAT_D2Q4S) {
        if (storage_f64) ghost_kernel<double, LAT_D2Q4S><<<1, 32, 0, s>>>(g, gamma, c, (double*)ghost);
        else ghost_kernel<float, LAT_D2Q4S><<<1, 32, 0, s>>>(g, gamma, c, (float*)ghost);
    } else if (lattice == LAT_D2Q4) {
        if (storage_f64) ghost_kernel<double, LAT_D2Q4><<<1, 32, 0, s>>>(g, gamma, c, (double*)ghost);
        else ghost_kernel<float, LAT_D2Q4><<<1, 32, 0, s>>>(g, gamma, c, (float*)ghost);
    } else if (lattice == LAT_D1Q3) {
        if (storage_f64) ghost_kernel<double, LAT_D1Q3><<<1, 32, 0, s>>>(g, gamma, c, (double*)ghost);
        else ghost_kernel<float, LAT_D1Q3><<<1, 32, 0, s>>>(g, gamma, c, (float*)ghost);
    } else {
        if (storage_f64) ghost_kernel<double, LAT_D1Q2><<<1, 32, 0, s>>>(g, gamma, c, (double*)ghost);
        else ghost_kernel<float, LAT_D1Q2><<<1, 32, 0, s>>>(g, gamma, c, (float*)ghost);
    }
    return cudaGetLastError();
}

template <int LAT>
static void set_state_dispatch(int storage_f64, const void* W, int w_dtype, int kind, void* fs, int64_t N,
                               int64_t P, double gamma, double c, cudaStream_t s)
{
    const int g = grid_for(N);
    if (storage_f64) {
        if (w_dtype == 0) set_state_kernel<double, double, LAT><<<g, kThreads, 0, s>>>((const double*)W, (double*)fs, N, P, kind, gamma, c);
        else set_state_kernel<float, double, LAT><<<g, kThreads, 0, s>>>((const float*)W, (double*)fs, N, P, kind, gamma, c);
    } else {
        if (w_dtype == 0) set_state_kernel<double, float, LAT><<<g, kThreads, 0, s>>>((const double*)W, (float*)fs, N, P, kind, gamma, c);
        else set_state_kernel<float, float, LAT><<<g, kThreads, 0, s>>>((const float*)W, (float*)fs, N, P, kind, gamma, c);
    }
}

cudaError_t launch_set_state(int lattice, int storage_f64, const void* W, int w_dtype, int kind, void* fs,
                             int64_t N, int64_t plane, double gamma, double c, cudaStream_t s)
{
    if (lattice == LAT_D2Q4S) set_state_dispatch<LAT_D2Q4S>(storage_f64, W, w_dtype, kind, fs, N, plane, gamma, c, s);
    else if (lattice == LAT_D2Q4) set_state_dispatch<LAT_D2Q4>(storage_f64, W, w_dtype, kind, fs, N, plane, gamma, c, s);
    else if (lattice == LAT_D1Q3) set_state_dispatch<LAT_D1Q3>(storage_f64, W, w_dtype, kind, fs, N, plane, gamma, c, s);
    else set_state_dispatch<LAT_D1Q2>(storage_f64, W, w_dtype, kind, fs, N, plane, gamma, c, s);
    return cudaGetLastError();
}

template <int LAT>
static void moments_dispatch(int storage_f64, const void* fs, void* U, int out_dtype, int64_t N, int64_t P,
                             cudaStream_t s)
{
    const int g = grid_for(N);
    if (storage_f64) {
        if (out_dtype == 0) moments_kernel<double, double, LAT><<<g, kThreads, 0, s>>>((const double*)fs, (double*)U, N, P);
        else moments_kernel<double, float, LAT><<<g, kThreads, 0, s>>>((const double*)fs, (float*)U, N, P);
    } else {
        if (out_dtype == 0) moments_kernel<float, double, LAT><<<g, kThreads, 0, s>>>((const float*)fs, (double*)U, N, P);
        else moments_kernel<float, float, LAT><<<g, kThreads, 0, s>>>((const float*)fs, (float*)U, N, P);
    }
}

cudaError_t launch_moments(int lattice, int storage_f64, const void* fs, void* U, int out_dtype, int64_t N,
                           int64_t plane, cudaStream_t s)
{
    if (lattice == LAT_U2D) moments_dispatch<LAT_U2D>(0, fs, U, out_dtype, N, plane, s);
    else if (lattice == LAT_D2Q4S) moments_dispatch<LAT_D2Q4S>(storage_f64, fs, U, out_dtype, N, plane, s);
    else if (lattice == LAT_D2Q4) moments_dispatch<LAT_D2Q4>(storage_f64, fs, U, out_dtype, N, plane, s);
    else if (lattice == LAT_D1Q3) moments_dispatch<LAT_D1Q3>(storage_f64, fs, U, out_dtype, N, plane, s);
    else moments_dispatch<LAT_D1Q2>(storage_f64, fs, U, out_dtype, N, plane, s);
    return cudaGetLastError();
}

int diag_blocks() { return kDiagBlocks; }

cudaError_t launch_diag(int lattice, int storage_f64, const void* fs, int64_t N, int64_t plane, double gamma,
                        double lambda, double cell_volume, double* partials, double* out, cudaStream_t s)
{
    if (lattice == LAT_U2D) {
        diag_partial_kernel<float, LAT_U2D><<<kDiagBlocks, kThreads, 0, s>>>((const float*)fs, N, plane, gamma, lambda, partials);
    } else if (lattice == LAT_D1Q3) {
        if (storage_f64) diag_partial_kernel<double, LAT_D1Q3><<<kDiagBlocks, kThreads, 0, s>>>((const double*)fs, N, plane, gamma, lambda, partials);
        else diag_partial_kernel<float, LAT_D1Q3><<<kDiagBlocks, kThreads, 0, s>>>((const float*)fs, N, plane, gamma, lambda, partials);
    } else if (lattice == LAT_D2Q4S) {
        if (storage_f64) diag_partial_kernel<double, LAT_D2Q4S><<<kDiagBlocks, kThreads, 0, s>>>((const double*)fs, N, plane, gamma, lambda, partials);
        else diag_partial_kernel<float, LAT_D2Q4S><<<kDiagBlocks, kThreads, 0, s>>>((const float*)fs, N, plane, gamma, lambda, partials);
    } else if (lattice == LAT_D2Q4) {
        if (storage_f64) diag_partial_kernel<double, LAT_D2Q4><<<kDiagBlocks, kThreads, 0, s>>>((const double*)fs, N, plane, gamma, lambda, partials);
        else diag_partial_kernel<float, LAT_D2Q4><<<kDiagBlocks, kThreads, 0, s>>>((const float*)fs, N, plane, gamma, lambda, partials);
    } else {
        if (storage_f64) diag_partial_kernel<double, LAT_D1Q2><<<kDiagBlocks, kThreads, 0, s>>>((const double*)fs, N, plane, gamma, lambda, partials);
        else diag_partial_kernel<float, LAT_D1Q2><<<kDiagBlocks, kThreads, 0, s>>>((const float*)fs, N, plane, gamma, lambda, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, 32, 0, s>>>(partials, kDiagBlocks, cell_volume, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched tubes

template <int Q>
static cudaError_t launch_batch_q_f64(const BatchArgs<double>& a, int ntiles, int block, cudaStream_t s)
{
    const size_t smem = 2 * 3 * Q * (size_t)(a.tile_cells + 2 * a.halo) * sizeof(double);
    switch (block) {
        case 128:
            batch1d_kernel<double, 128, Q><<<ntiles, 128, smem, s>>>(a);
            break;
        case 256:
            batch1d_kernel<double, 256, Q><<<ntiles, 256, smem, s>>>(a);
            break;
        case 512:
            batch1d_kernel<double, 512, Q><<<ntiles, 512, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_f64(const BatchArgs<double>& a, int ntiles, int block, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    return a.q == 3 ? launch_batch_q_f64<3>(a, ntiles, block, s) : launch_batch_q_f64<2>(a, ntiles, block, s);
}

template <int Q>
static cudaError_t prepare_batch_q_f64(int block, size_t smem)
{
    // opt in to more than the default 48 KiB of dynamic shared memory
    switch (block) {
        case 128:
            return cudaFuncSetAttribute(batch1d_kernel<double, 128, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 256:
            return cudaFuncSetAttribute(batch1d_kernel<double, 256, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 512:
            return cudaFuncSetAttribute(batch1d_kernel<double, 512, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_batch_f64(int block, size_t smem, int q)
{
    return q == 3 ? prepare_batch_q_f64<3>(block, smem) : prepare_batch_q_f64<2>(block, smem);
}

cudaError_t launch_batch_copy_f64(const double* src, double* dst, int64_t N, const BatchTile* tiles, int ntiles,
                                     const int64_t* tube_off, int planes, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    batch_copy_kernel<double><<<ntiles, 256, 0, s>>>(src, dst, N, tiles, tube_off, planes);
    return cudaGetLastError();
}

}  // namespace lbrs

namespace lbrs {

cudaError_t launch_adapt_reset(void* st, double lambda, cudaStream_t s)
{
    adapt_reset_kernel<<<1, 32, 0, s>>>((AdaptState*)st, lambda);
    return cudaGetLastError();
}

cudaError_t launch_adapt_prep(int storage_f64, void* st, void* ghost, const GhostSpec& g, double gamma, double dx,
                              double safety, double t_final, cudaStream_t s)
{
    if (storage_f64)
        adapt_prep_kernel<double><<<1, 32, 0, s>>>((AdaptState*)st, (double*)ghost, g, gamma, dx, safety, t_final);
    else
        adapt_prep_kernel<float><<<1, 32, 0, s>>>((AdaptState*)st, (float*)ghost, g, gamma, dx, safety, t_final);
    return cudaGetLastError();
}

cudaError_t launch_adapt_step_f64(const StepArgs<double>& a, void* st, double gamma, cudaStream_t s)
{
    const dim3 block(128, 2);
    step2d_adapt_kernel<double><<<grid2d(a.nx, a.ny, block), block, 0, s>>>(a, (AdaptState*)st, gamma);
    return cudaGetLastError();
}

cudaError_t launch_adapt_init_bound_f64(const void* fs, int64_t N, double gamma, void* st, cudaStream_t s)
{
    adapt_init_bound_kernel<double><<<grid_for(N), 256, 0, s>>>((const double*)fs, N, gamma, (AdaptState*)st);
    return cudaGetLastError();
}

// First out-of-bounds index recorded by this unit's kernels (LBRS_DEBUG builds; 0 otherwise).
LBRS_DEBUG_WORD(debug_word_f64)

}  // namespace lbrs
