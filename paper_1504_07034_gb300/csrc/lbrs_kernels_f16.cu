// Reduced-state D2Q4 steps: the FP16 non-equilibrium form (LBRS_F16NEQ) and
// the omega = 1 moments-only form (LBRS_F32U).
//
// LBRS_F16NEQ.  State per cell: the moments U (4 x FP32) and, per field k, the
// post-collision non-equilibrium parts g_q = f*_q - f^eq_q(U) of populations
// q = 0, 1, 2 in FP16, scaled by a per-field power of two s_k (stored value
// g / s_k).  A state buffer is U [4][N] FP32, g [3][4][N] FP16, then the four
// scales (FP32), so a copy of the buffer is a complete checkpoint; every step
// carries the scales over to its output buffer.  The fourth part follows from
// sum_q g_q = 0: the collision leaves the moments unchanged, sum_q f*_q = U =
// sum_q f^eq_q(U).  40 bytes per cell instead of 64: 80 B per lattice update.
//
// LBRS_F32U.  At omega = 1 the relaxation returns f* = f^eq(U) exactly (Section
// II.A with omega = 1), so the state is the moments U alone: 16 bytes per
// cell, 32 B per lattice update.
//
// Both stream by reconstruction: f*_q(x - c_q) = f^eq_q(U(x - c_q)) [+ s_k g_q].
// One CTA owns a 32 x 16 tile; it first rebuilds f* of the 34 x 18 window (tile
// plus one cell of halo, sources outside the domain resolved by the boundary
// kind exactly as the pull of the distribution-storing kernel does) in shared
// memory, each window cell once, then every tile cell gathers its four pulled
// populations, applies the wall relations, forms U and -- for the FP16 form --
// the new non-equilibrium parts g = (1 - omega)(f - f^eq(U)).  The window keeps
// the four fields of a population together (one 16-byte word per population and
// slot), so a slot is written and a cell's pull is read in four vector accesses;
// a tile whose window lies inside the domain skips the boundary resolution.
#include <stdlib.h>
#include <string.h>

#include <cuda_fp16.h>

#include "lbrs_kernels.cuh"
#include "lbrs_launch.h"

namespace lbrs {

namespace {

struct F16Args {
    const float* __restrict__ Uin;     // [4][N]
    const __half* __restrict__ gin;    // [3][4][N]
    float* __restrict__ Uout;
    __half* __restrict__ gout;
    const float* __restrict__ ghost;   // [4][GHOST_STRIDE] full f of the Dirichlet states
    const float* __restrict__ scale;   // [4] s_k, tail of the input buffer
    float* __restrict__ scale_out;     // tail of the output buffer
    int64_t N;
    int nx, ny;
    int bc[4];
    float om, om1, c, gm1;
};

constexpr int kTX = 32, kTY = 16, kWX = kTX + 2, kWY = kTY + 2, kWN = kWX * kWY;
constexpr int kThreads = kTX * kTY;

template <bool F16>
__global__ void __launch_bounds__(kThreads) step2d_tile_kernel(const F16Args a)
{
    __shared__ float4 s_f[4 * kWN];      // f*_{q,k} of every window slot: [q][slot].(k = x, y, z, w)
    const int i0 = blockIdx.x * kTX - 1, j0 = blockIdx.y * kTY - 1;
    float sc[4] = {1.f, 1.f, 1.f, 1.f}, inv[4] = {1.f, 1.f, 1.f, 1.f};
    if constexpr (F16) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sc[k] = a.scale[k];
            inv[k] = 1.f / sc[k];          // exact: the scales are powers of two
        }
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 4) a.scale_out[threadIdx.x] = a.scale[threadIdx.x];
    }

    // phase 1: f* of each window slot, its source resolved like the pull does
    const bool inside = i0 >= 0 && j0 >= 0 && i0 + kWX <= a.nx && j0 + kWY <= a.ny;
    for (int w = threadIdx.x; w < kWN; w += kThreads) {
        int i = i0 + w % kWX, j = j0 + w / kWX;
        if (!inside) {
            // a slot more than one cell outside the grid is no tile cell's source (and one
            // wrap would not bring it inside a periodic grid narrower than the tile)
            if (i < -1 || i > a.nx || j < -1 || j > a.ny) continue;
            const int side_x = i < 0 ? 0 : (i >= a.nx ? 1 : -1);
            const int side_y = j < 0 ? 2 : (j >= a.ny ? 3 : -1);
            const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
            const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
            const float* g = nullptr;
            if (side_x >= 0) {
                if (kind_x == BC_DIRICHLET) g = a.ghost + side_x * GHOST_STRIDE;
                else if (kind_x == BC_PERIODIC) i = i < 0 ? i + a.nx : i - a.nx;
                else i = i < 0 ? 0 : a.nx - 1;
            }
            if (!g && side_y >= 0) {
                // a wall side's slot is never used (the wall relation replaces those
                // populations); clamp it like a transmissive side
                if (kind_y == BC_DIRICHLET) g = a.ghost + side_y * GHOST_STRIDE;
                else if (kind_y == BC_PERIODIC) j = j < 0 ? j + a.ny : j - a.ny;
                else j = j < 0 ? 0 : a.ny - 1;
            }
            if (g) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    s_f[LBRS_IX(q * kWN + w, 4 * kWN, 40)] = make_float4(g[q * 4], g[q * 4 + 1], g[q * 4 + 2], g[q * 4 + 3]);
                continue;
            }
        }
        const int64_t c = (int64_t)j * a.nx + i;
        float U[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.Uin[LBRS_IX(k * a.N + c, 4 * a.N, 41)];
        float e[4][4];
        equilibria2d<float>(U, a.gm1, a.c, e);
        if constexpr (F16) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float g0 = __half2float(a.gin[LBRS_IX(k * a.N + c, 12 * a.N, 41)]);
                const float g1 = __half2float(a.gin[LBRS_IX((4 + k) * a.N + c, 12 * a.N, 41)]);
                const float g2 = __half2float(a.gin[LBRS_IX((8 + k) * a.N + c, 12 * a.N, 41)]);
                e[0][k] += sc[k] * g0;
                e[1][k] += sc[k] * g1;
                e[2][k] += sc[k] * g2;
                e[3][k] += sc[k] * -((g0 + g1) + g2);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) s_f[LBRS_IX(q * kWN + w, 4 * kWN, 40)] = make_float4(e[q][0], e[q][1], e[q][2], e[q][3]);
    }
    __syncthreads();

    // phase 2: pull, wall relations, moments [, non-equilibrium parts]
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const int i = blockIdx.x * kTX + tx, j = blockIdx.y * kTY + ty;
    if (i >= a.nx || j >= a.ny) return;
    const int slot = (ty + 1) * kWX + (tx + 1);
    // sources x - c_q: q0 (-,-) <- (+1,+1); q1 (+,-) <- (-1,+1); q2 (+,+) <- (-1,-1); q3 (-,+) <- (+1,-1)
    const int src[4] = {slot + kWX + 1, slot + kWX - 1, slot - kWX - 1, slot - kWX + 1};
    float f[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = s_f[LBRS_IX(q * kWN + src[q], 4 * kWN, 40)];
        f[q][0] = v.x;
        f[q][1] = v.y;
        f[q][2] = v.z;
        f[q][3] = v.w;
    }
    const bool wall_bottom = j == 0 && a.bc[2] == BC_WALL;
    const bool wall_top = j == a.ny - 1 && a.bc[3] == BC_WALL;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float sgn = k == 2 ? -1.f : 1.f;
        if (wall_top) {
            f[0][k] = sgn * f[3][k];
            f[1][k] = sgn * f[2][k];
        }
        if (wall_bottom) {
            f[3][k] = sgn * f[0][k];
            f[2][k] = sgn * f[1][k];
        }
    }
    const int64_t c = (int64_t)j * a.nx + i;
    float U[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        U[k] = ((f[0][k] + f[1][k]) + f[2][k]) + f[3][k];
        a.Uout[LBRS_IX(k * a.N + c, 4 * a.N, 41)] = U[k];
    }
    if constexpr (F16) {
        float e[4][4];
        equilibria2d<float>(U, a.gm1, a.c, e);
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                a.gout[LBRS_IX((q * 4 + k) * a.N + c, 12 * a.N, 41)] = __float2half_rn(a.om1 * (f[q][k] - e[q][k]) * inv[k]);
    }
}

// ---------------------------------------------------------------- moments-only form, two steps per launch
//
// At omega = 1 one step of the moments-only form is U'(x) = sum_q f^eq_q(U(x - c_q)) (with the
// boundary resolution and the wall relations of the pull).  One CTA advances a 32 x 16 tile by two
// steps and reads and writes the state once:
//   phase A  f*^n = f^eq(U^n) of the 36 x 20 window (two cells of halo) into shared memory;
//   phase B  U^{n+1} of the 34 x 18 inner window gathered from it; after a barrier the inner slots
//            are overwritten in place with f*^{n+1} = f^eq(U^{n+1});
//   phase C  U^{n+2} of the tile gathered from the inner window and stored.
// Window slots beyond a periodic side hold the wrapped cells (their own pulls stay inside the
// window).  A slot beyond another side stands for the source that the single-step pull would
// resolve there: a Dirichlet side's ghost f, else the clamped cell (transmissive; a wall side's
// slots are never read, the wall relations replace those populations), the x side taking
// precedence at corners.  In phase A the clamped cell is loaded; in phase B the thread of such a
// slot gathers U^{n+1} of the clamped slot itself, so every inner slot is written after one barrier.
// Every value is formed by the arithmetic of the single-step kernel (step2d_tile_kernel<false>), so
// the result is bit-identical to two single steps.  State traffic: 16 B read and 16 B written per
// cell and launch, 16 B per lattice update.

constexpr int kUX = 32, kUY = 16;                       // tile
constexpr int kAX = kUX + 4, kAY = kUY + 4, kAN = kAX * kAY;   // phase-A window (two cells of halo)
constexpr int kBX = kUX + 2, kBY = kUY + 2, kBN = kBX * kBY;   // phase-B inner window
constexpr int kUThreads = kUX * kUY;
constexpr int kBPer = (kBN + kUThreads - 1) / kUThreads;       // inner slots per thread

// Cells beyond side s of an axis of n cells that a coordinate lies (0 inside).
__device__ __forceinline__ int beyond(int i, int n) { return i < 0 ? -i : (i >= n ? i - n + 1 : 0); }

__device__ __forceinline__ int wrap_mod(int i, int n)
{
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// The two-step kernel.  a.Uin / a.Uout as in step2d_tile_kernel<false>.
__global__ void __launch_bounds__(kUThreads) step2d_u2_kernel(const F16Args a)
{
    __shared__ float4 s_f[4 * kAN];      // [q][slot], slot = wy * kAX + wx
    const int ti0 = blockIdx.x * kUX, tj0 = blockIdx.y * kUY;
    const int i0 = ti0 - 2, j0 = tj0 - 2;                  // global cell of window slot (0, 0)
    const bool inside = i0 >= 0 && j0 >= 0 && i0 + kAX <= a.nx && j0 + kAY <= a.ny;
    const bool per_x = a.bc[0] == BC_PERIODIC, per_y = a.bc[2] == BC_PERIODIC;

    // phase A: f*^n of every window slot that a later phase reads
    for (int w = threadIdx.x; w < kAN; w += kUThreads) {
        int i = i0 + w % kAX, j = j0 + w / kAX;
        if (!inside) {
            const int bx = beyond(i, a.nx), by = beyond(j, a.ny);
            // two cells beyond a non-periodic side: only inner slots beyond that side would pull
            // from here, and those are not gathered from their own position
            if ((bx > 1 && !per_x) || (by > 1 && !per_y) || bx > 2 || by > 2) continue;
            const float* g = nullptr;
            if (bx) {
                const int side = i < 0 ? 0 : 1;
                const int kind = side == 0 ? a.bc[0] : a.bc[1];
                if (kind == BC_DIRICHLET) g = a.ghost + side * GHOST_STRIDE;
                else if (kind == BC_PERIODIC) i = wrap_mod(i, a.nx);
                else i = i < 0 ? 0 : a.nx - 1;
            }
            if (!g && by) {
                const int side = j < 0 ? 2 : 3;
                const int kind = side == 2 ? a.bc[2] : a.bc[3];
                if (kind == BC_DIRICHLET) g = a.ghost + side * GHOST_STRIDE;
                else if (kind == BC_PERIODIC) j = wrap_mod(j, a.ny);
                else j = j < 0 ? 0 : a.ny - 1;
            }
            if (g) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    s_f[LBRS_IX(q * kAN + w, 4 * kAN, 42)] = make_float4(g[q * 4], g[q * 4 + 1], g[q * 4 + 2], g[q * 4 + 3]);
                continue;
            }
        }
        const int64_t c = (int64_t)j * a.nx + i;
        float U[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.Uin[LBRS_IX(k * a.N + c, 4 * a.N, 43)];
        float e[4][4];
        equilibria2d<float>(U, a.gm1, a.c, e);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            s_f[LBRS_IX(q * kAN + w, 4 * kAN, 42)] = make_float4(e[q][0], e[q][1], e[q][2], e[q][3]);
    }
    __syncthreads();

    // phase B: U^{n+1} of the inner slots (kind 0: skip, 1: gathered, 2: Dirichlet ghost of side gs)
    float U1[kBPer][4];
    int kind1[kBPer], gs1[kBPer];
#pragma unroll
    for (int r = 0; r < kBPer; ++r) {
        kind1[r] = 0;
        gs1[r] = 0;
        const int b = threadIdx.x + r * kUThreads;
        if (b >= kBN) continue;
        int wx = 1 + b % kBX, wy = 1 + b / kBX;             // window position of the slot
        if (!inside) {
            const int i = i0 + wx, j = j0 + wy;
            const int bx = beyond(i, a.nx), by = beyond(j, a.ny);
            if (bx > 1 || by > 1) continue;                  // beyond a ragged tile's edge: no cell pulls it
            bool ghost = false;
            if (bx && !per_x) {
                const int side = i < 0 ? 0 : 1;
                if ((side == 0 ? a.bc[0] : a.bc[1]) == BC_DIRICHLET) {
                    ghost = true;
                    gs1[r] = side;
                } else {
                    wx += i < 0 ? -i : a.nx - 1 - i;        // the clamped cell's slot
                }
            }
            if (!ghost && by && !per_y) {
                const int side = j < 0 ? 2 : 3;
                if ((side == 2 ? a.bc[2] : a.bc[3]) == BC_DIRICHLET) {
                    ghost = true;
                    gs1[r] = side;
                } else {
                    wy += j < 0 ? -j : a.ny - 1 - j;
                }
            }
            if (ghost) {
                kind1[r] = 2;
                continue;
            }
        }
        const int slot = wy * kAX + wx;
        const int src[4] = {slot + kAX + 1, slot + kAX - 1, slot - kAX - 1, slot - kAX + 1};
        float f[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = s_f[LBRS_IX(q * kAN + src[q], 4 * kAN, 44)];
            f[q][0] = v.x;
            f[q][1] = v.y;
            f[q][2] = v.z;
            f[q][3] = v.w;
        }
        const int j = j0 + wy;                               // the gathering cell's row (unwrapped)
        const bool wall_bottom = j == 0 && a.bc[2] == BC_WALL;
        const bool wall_top = j == a.ny - 1 && a.bc[3] == BC_WALL;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float sgn = k == 2 ? -1.f : 1.f;
            if (wall_top) {
                f[0][k] = sgn * f[3][k];
                f[1][k] = sgn * f[2][k];
            }
            if (wall_bottom) {
                f[3][k] = sgn * f[0][k];
                f[2][k] = sgn * f[1][k];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) U1[r][k] = ((f[0][k] + f[1][k]) + f[2][k]) + f[3][k];
        kind1[r] = 1;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kBPer; ++r) {
        const int b = threadIdx.x + r * kUThreads;
        if (b >= kBN || kind1[r] == 0) continue;
        const int w = (1 + b / kBX) * kAX + 1 + b % kBX;
        if (kind1[r] == 2) {
            const float* g = a.ghost + gs1[r] * GHOST_STRIDE;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                s_f[LBRS_IX(q * kAN + w, 4 * kAN, 45)] = make_float4(g[q * 4], g[q * 4 + 1], g[q * 4 + 2], g[q * 4 + 3]);
            continue;
        }
        float e[4][4];
        equilibria2d<float>(U1[r], a.gm1, a.c, e);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            s_f[LBRS_IX(q * kAN + w, 4 * kAN, 45)] = make_float4(e[q][0], e[q][1], e[q][2], e[q][3]);
    }
    __syncthreads();

    // phase C: U^{n+2} of the tile
    const int tx = threadIdx.x % kUX, ty = threadIdx.x / kUX;
    const int i = ti0 + tx, j = tj0 + ty;
    if (i >= a.nx || j >= a.ny) return;
    const int slot = (ty + 2) * kAX + (tx + 2);
    const int src[4] = {slot + kAX + 1, slot + kAX - 1, slot - kAX - 1, slot - kAX + 1};
    float f[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 v = s_f[LBRS_IX(q * kAN + src[q], 4 * kAN, 46)];
        f[q][0] = v.x;
        f[q][1] = v.y;
        f[q][2] = v.z;
        f[q][3] = v.w;
    }
    const bool wall_bottom = j == 0 && a.bc[2] == BC_WALL;
    const bool wall_top = j == a.ny - 1 && a.bc[3] == BC_WALL;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float sgn = k == 2 ? -1.f : 1.f;
        if (wall_top) {
            f[0][k] = sgn * f[3][k];
            f[1][k] = sgn * f[2][k];
        }
        if (wall_bottom) {
            f[3][k] = sgn * f[0][k];
            f[2][k] = sgn * f[1][k];
        }
    }
    const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) a.Uout[LBRS_IX(k * a.N + c, 4 * a.N, 47)] = ((f[0][k] + f[1][k]) + f[2][k]) + f[3][k];
}

// Initial state: U from W (conserved or primitive, FP64 arithmetic), g = 0.
template <typename Tin>
__global__ void __launch_bounds__(256) set_state_f16neq_kernel(const Tin* __restrict__ W, float* __restrict__ U,
                                                               __half* __restrict__ g, int64_t N, int64_t P,
                                                               int kind, double gamma)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double w[4], u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = (double)W[k * N + i];
        if (kind == KIND_PRIMITIVE) {
            prim_to_cons2d(w, gamma, u);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) u[k] = w[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k * P + i] = (float)u[k];
        if (g) {
#pragma unroll
            for (int n = 0; n < 12; ++n) g[n * N + i] = __float2half_rn(0.f);
        }
    }
}

// Per-field scale: the power of two at or above max_cells |U_k| (1 for an all-zero field).
__global__ void __launch_bounds__(256) field_absmax_kernel(const float* __restrict__ U, int64_t N,
                                                           unsigned int* __restrict__ absmax_bits)
{
    float m[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) m[k] = fmaxf(m[k], fabsf(U[k * N + i]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m[k] = fmaxf(m[k], __shfl_down_sync(0xffffffffu, m[k], off));
        // non-negative floats order like their bit patterns
        if ((threadIdx.x & 31) == 0) atomicMax(absmax_bits + k, __float_as_uint(m[k]));
    }
}

__global__ void field_scale_kernel(const unsigned int* __restrict__ absmax_bits, float* __restrict__ scale)
{
    const int k = threadIdx.x;
    if (k >= 4) return;
    const float m = __uint_as_float(absmax_bits[k]);
    scale[k] = (m > 0.f && isfinite(m)) ? exp2f(ceilf(log2f(m))) : 1.f;
}

}  // namespace

static F16Args tile_args(const F16StepArgs& s, bool f16)
{
    F16Args a;
    a.Uin = (const float*)s.src;
    a.gin = f16 ? (const __half*)((const char*)s.src + 16 * s.N) : nullptr;
    a.Uout = (float*)s.dst;
    a.gout = f16 ? (__half*)((char*)s.dst + 16 * s.N) : nullptr;
    a.ghost = s.ghost;
    a.scale = f16 ? (const float*)((const char*)s.src + 40 * s.N) : nullptr;
    a.scale_out = f16 ? (float*)((char*)s.dst + 40 * s.N) : nullptr;
    a.N = s.N;
    a.nx = s.nx;
    a.ny = s.ny;
    for (int k = 0; k < 4; ++k) a.bc[k] = s.bc[k];
    a.om = s.om;
    a.om1 = s.om1;
    a.c = s.c;
    a.gm1 = s.gm1;
    return a;
}

cudaError_t launch_step_f16neq(const F16StepArgs& s, cudaStream_t st)
{
    const dim3 grid((unsigned)((s.nx + kTX - 1) / kTX), (unsigned)((s.ny + kTY - 1) / kTY));
    step2d_tile_kernel<true><<<grid, kThreads, 0, st>>>(tile_args(s, true));
    return cudaGetLastError();
}

cudaError_t launch_step_f32u(const F16StepArgs& s, cudaStream_t st)
{
    const dim3 grid((unsigned)((s.nx + kTX - 1) / kTX), (unsigned)((s.ny + kTY - 1) / kTY));
    step2d_tile_kernel<false><<<grid, kThreads, 0, st>>>(tile_args(s, false));
    return cudaGetLastError();
}

cudaError_t launch_step2_f32u(const F16StepArgs& s, cudaStream_t st)
{
    const dim3 grid((unsigned)((s.nx + kUX - 1) / kUX), (unsigned)((s.ny + kUY - 1) / kUY));
    step2d_u2_kernel<<<grid, kUThreads, 0, st>>>(tile_args(s, false));
    return cudaGetLastError();
}

bool step2_f32u_enabled()
{
    static int v = [] {
        const char* e = getenv("LBRS_F32U_FUSE");
        return (e && !strcmp(e, "0")) ? 0 : 1;
    }();
    return v != 0;
}

cudaError_t launch_set_state_f32u(const void* W, int w_dtype, int kind, void* fs, int64_t N, int64_t plane,
                                  double gamma, cudaStream_t st)
{
    int64_t b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    const int g = (int)(b < 1 ? 1 : b);
    if (w_dtype == 0) set_state_f16neq_kernel<double><<<g, 256, 0, st>>>((const double*)W, (float*)fs, nullptr, N, plane, kind, gamma);
    else set_state_f16neq_kernel<float><<<g, 256, 0, st>>>((const float*)W, (float*)fs, nullptr, N, plane, kind, gamma);
    return cudaGetLastError();
}

cudaError_t launch_set_state_f16neq(const void* W, int w_dtype, int kind, void* fs, int64_t N, double gamma,
                                    unsigned int* absmax_bits, cudaStream_t st)
{
    float* scale = (float*)((char*)fs + 40 * N);
    int64_t b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    const int g = (int)(b < 1 ? 1 : b);
    float* U = (float*)fs;
    __half* gq = (__half*)((char*)fs + 16 * N);
    if (w_dtype == 0) set_state_f16neq_kernel<double><<<g, 256, 0, st>>>((const double*)W, U, gq, N, N, kind, gamma);
    else set_state_f16neq_kernel<float><<<g, 256, 0, st>>>((const float*)W, U, gq, N, N, kind, gamma);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(absmax_bits, 0, 4 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    field_absmax_kernel<<<g, 256, 0, st>>>(U, N, absmax_bits);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    field_scale_kernel<<<1, 32, 0, st>>>(absmax_bits, scale);
    return cudaGetLastError();
}

// First out-of-bounds index recorded by this unit's kernels (LBRS_DEBUG builds; 0 otherwise).
LBRS_DEBUG_WORD(debug_word_f16)

}  // namespace lbrs
