// FP32 time step of the LBRS solver (distributions stored and updated in FP32).
//
// Compiled with FMA contraction allowed; velocities use one reciprocal per cell
// (rcp_f32: the hardware approximation refined by one Newton-Raphson step).  The numerics differ from the FP64 path by rounding
// only; their distance to the FP64 oracle is measured, not assumed.
//
// D2Q4 uses a vectorised kernel when nx is a multiple of the vector width V:
// each thread owns V consecutive cells of one row and reads each of the 16
// (q, k) planes with one V-wide load.  The +-1 column shift of the pull is
// realigned with one warp shuffle per plane; the lane at the warp's edge
// fetches the missing neighbour itself (resolving the x boundary when the
// neighbour lies outside the domain).  The first and last rows, whose sources
// cross the y boundaries (walls, ghosts, wrap), take the scalar path.
#include <stdlib.h>
#include <string.h>
#include <mutex>

#include <cuda.h>

#include "lbrs_kernels.cuh"
#include "lbrs_batch.cuh"
#include "lbrs_launch.h"

namespace lbrs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int V>
struct Vec;
template <>
struct Vec<2> {
    using type = float2;
    static __device__ __forceinline__ float get(const float2& v, int c) { return c == 0 ? v.x : v.y; }
    static __device__ __forceinline__ float2 make(const float* f) { return make_float2(f[0], f[1]); }
    static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};
template <>
struct Vec<4> {
    using type = float4;
    static __device__ __forceinline__ float get(const float4& v, int c)
    {
        return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
    }
    static __device__ __forceinline__ float4 make(const float* f) { return make_float4(f[0], f[1], f[2], f[3]); }
    static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};

// Value of plane (q, k) at column -1 (side 0) or nx (side 1) of a row whose y
// source is inside the domain: Dirichlet ghost, periodic wrap or clamp.
__device__ __forceinline__ float x_outside(int kind, const float* __restrict__ ghost, const float* row, int nx,
                                           int side, int q, int k)
{
    if (kind == BC_DIRICHLET) return ghost[side * GHOST_STRIDE + q * 4 + k];
    if (kind == BC_PERIODIC) return side == 0 ? row[nx - 1] : row[0];
    return side == 0 ? row[0] : row[nx - 1];
}

template <int V>
__global__ void __launch_bounds__(128) step2d_f32_vec_kernel(const StepArgs<float> a)
{
    using VT = typename Vec<V>::type;
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.y;
    const int i0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const bool active = i0 < a.nx;

    if (j == 0 || j == a.ny - 1) {     // rows touching a y boundary: scalar path
        if (!active) return;
#pragma unroll 1
        for (int c = 0; c < V; ++c) {
            float f[4][4];
            pull_edge_2d<float>(a, i0 + c, j, f);
            collide_store_2d<float>(a, (int64_t)j * a.nx + i0 + c, f);
        }
        return;
    }

    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    // The lane at the left edge of a warp needs column i0-1 (planes pulling
    // from i-1); the lane at the right edge (or the last active one) needs
    // column i0+V.  Outside the domain the column is wrapped, clamped or
    // replaced by the Dirichlet ghost below.
    const bool left_lane = lane == 0;
    const bool right_lane = lane == 31 || i0 + V >= a.nx;
    const int bc0 = a.bc[0], bc1 = a.bc[1];
    const int idx_left = i0 > 0 ? i0 - 1 : (bc0 == BC_PERIODIC ? a.nx - 1 : 0);
    const int idx_right = i0 + V < a.nx ? i0 + V : (bc1 == BC_PERIODIC ? 0 : a.nx - 1);
    const bool ghost_left = i0 == 0 && bc0 == BC_DIRICHLET;
    const bool ghost_right = i0 + V >= a.nx && bc1 == BC_DIRICHLET;

    // phase 1: every load of the cell group is issued before any is used
    VT v[4][4];
    float ex[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t row_off = (int64_t)(j - SY[q]) * a.nx;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float* row = a.src + (q * 4 + k) * a.N + row_off;
            v[q][k] = active ? *reinterpret_cast<const VT*>(row + i0) : Vec<V>::zero();
            if (SX[q] > 0) ex[q][k] = (left_lane && active) ? row[idx_left] : 0.f;
            else ex[q][k] = (right_lane && active) ? row[idx_right] : 0.f;
        }
    }
    // phase 2: realign the +-1 column shift with warp shuffles
    float f[4][4][V];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (SX[q] > 0) {
                // pull from i - 1: cells i0..i0+V-1 take columns i0-1 .. i0+V-2
                float prev = __shfl_up_sync(kFull, Vec<V>::get(v[q][k], V - 1), 1);
                if (left_lane) prev = ghost_left ? a.ghost[q * 4 + k] : ex[q][k];
                f[q][k][0] = prev;
#pragma unroll
                for (int c = 1; c < V; ++c) f[q][k][c] = Vec<V>::get(v[q][k], c - 1);
            } else {
                // pull from i + 1: cells i0..i0+V-1 take columns i0+1 .. i0+V
                float next = __shfl_down_sync(kFull, Vec<V>::get(v[q][k], 0), 1);
                if (right_lane) next = ghost_right ? a.ghost[GHOST_STRIDE + q * 4 + k] : ex[q][k];
#pragma unroll
                for (int c = 0; c < V - 1; ++c) f[q][k][c] = Vec<V>::get(v[q][k], c + 1);
                f[q][k][V - 1] = next;
            }
        }
    }
    if (!active) return;

#pragma unroll
    for (int c = 0; c < V; ++c) {
        float U[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = ((f[0][k][c] + f[1][k][c]) + f[2][k][c]) + f[3][k][c];
        float e[4][4];
        equilibria2d<float>(U, a.gm1, a.c, e);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k][c] = a.om1 * f[q][k][c] + a.om * e[q][k];
    }
    const int64_t base = (int64_t)j * a.nx + i0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) *reinterpret_cast<VT*>(a.dst + (q * 4 + k) * a.N + base) = Vec<V>::make(f[q][k]);
}

// R cells per thread, strided by the warp width: a warp owns 32 R consecutive
// cells of one row and lane l takes cells l, l + 32, ...  Every load is a plain
// coalesced 4-byte load at the +-1 column offset, R independent cells give R
// times the bytes in flight of the one-cell kernel, and no shuffles are needed.
template <int R>
__global__ void __launch_bounds__(128) step2d_f32_ilp_kernel(const StepArgs<float> a)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int j = blockIdx.y;
    const int ibase = warp * 32 * R + lane;
    if (j == 0 || j == a.ny - 1) {
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            const int i = ibase + 32 * r;
            if (i >= a.nx) break;
            float f[4][4];
            pull_edge_2d<float>(a, i, j, f);
            collide_store_2d<float>(a, (int64_t)j * a.nx + i, f);
        }
        return;
    }
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    const int bc0 = a.bc[0], bc1 = a.bc[1];
    float f[R][4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t row_off = (int64_t)(j - SY[q]) * a.nx;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = ibase + 32 * r;
            int si = i - SX[q];
            bool ghost = false;
            int side = 0;
            if (si < 0) {
                ghost = bc0 == BC_DIRICHLET;
                si = bc0 == BC_PERIODIC ? a.nx - 1 : 0;
            } else if (si >= a.nx) {
                ghost = bc1 == BC_DIRICHLET;
                side = 1;
                si = bc1 == BC_PERIODIC ? 0 : a.nx - 1;
            }
            const bool ok = i < a.nx;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float* row = a.src + (q * 4 + k) * a.N + row_off;
                f[r][q][k] = ok ? row[si] : 0.f;
            }
            if (ghost && ok) {
#pragma unroll
                for (int k = 0; k < 4; ++k) f[r][q][k] = a.ghost[side * GHOST_STRIDE + q * 4 + k];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = ibase + 32 * r;
        if (i < a.nx) collide_store_2d<float>(a, (int64_t)j * a.nx + i, f[r]);
    }
}

// ---------------------------------------------------------------- two steps per launch
//
// Temporal blocking by two: one CTA owns a 32 x 8 tile.  Phase 1 performs step
// n -> n+1 (the same pull, boundary resolution and collision as step2d_kernel)
// for the 34 x 10 window of the tile plus one cell of halo and keeps the result
// in shared memory; window slots beyond a periodic side hold the wrapped cells,
// slots beyond any other side are not computed.  Phase 2 performs step
// n+1 -> n+2 for the tile, pulling from shared memory: a source outside the
// domain is resolved exactly as in pull_edge_2d (Dirichlet ghost, clamp into
// the domain, whose cell is then in the window, or the wall relations); a
// periodic source keeps its unwrapped coordinate, whose slot holds the wrapped
// cell.  The state is read and written once per two steps.
constexpr int kFTX = 32, kFTY = 8, kFWX = kFTX + 2, kFWY = kFTY + 2, kFWN = kFWX * kFWY;

// x modulo n in [0, n): without a division for x within one period of the range, the case of
// every neighbour and window offset on a grid at least as wide as the window.
__device__ __forceinline__ int wrap_index(int x, int n)
{
    if (x >= 0 && x < n) return x;
    if (x < 0 && x >= -n) return x + n;
    if (x >= n && x - n < n) return x - n;
    x %= n;
    return x < 0 ? x + n : x;
}

// Phase 2 of the two-step kernels: step n+1 -> n+2 for the tile (i0, j0), pulling
// from the window of post-collision populations in shared memory.
// STORE_U: a.Uout receives the moments of this (second) step.
template <bool STORE_U, bool HALF>
__device__ __forceinline__ void step2_phase2(const StepArgs<float>& a, const float* s_f, int i0, int j0)
{
    const int ti = threadIdx.x % kFTX, tj = threadIdx.x / kFTX;
    const int i = i0 + ti, j = j0 + tj;
    if (i >= a.nx || j >= a.ny) return;
    float f[4][4];
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        // the cell's own slot s0; sources (i + 1, j + 1), (i - 1, j + 1), (i - 1, j - 1), (i + 1, j - 1)
        const int s0 = (tj + 1) * kFWX + ti + 1;
        const int sl[4] = {s0 + kFWX + 1, s0 + kFWX - 1, s0 - kFWX - 1, s0 - kFWX + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = s_f[LBRS_IX((q * 4 + k) * kFWN + sl[q], 16 * kFWN, 12)];
        collide_store_2d<float, STORE_U>(a, (int64_t)j * a.nx + i, f);
        return;
    }
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    bool wall_top = false, wall_bottom = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int si = i - SX[q], sj = j - SY[q];
        const int side_y = sj < 0 ? 2 : (sj >= a.ny ? 3 : -1);
        const int side_x = si < 0 ? 0 : (si >= a.nx ? 1 : -1);
        const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
        const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
        if (side_y >= 0 && kind_y == BC_WALL) {
            if (side_y == 3) wall_top = true; else wall_bottom = true;
            continue;
        }
        if (HALF && side_y >= 0 && kind_y == BC_WALL_HALFWAY) {
            // the mirror image of this population leaving the horizontal neighbour on the wall
            // row (a periodic neighbour keeps its unwrapped slot, which holds the wrapped cell)
            const int m = 3 - q;
            const float* gm = nullptr;
            if (side_x >= 0) {
                if (kind_x == BC_DIRICHLET) gm = a.ghost + side_x * GHOST_STRIDE + m * 4;
                else if (kind_x != BC_PERIODIC) si = si < 0 ? 0 : a.nx - 1;
            }
            const int slot = (j - (j0 - 1)) * kFWX + (si - (i0 - 1));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float sgn = k == 2 ? -1.f : 1.f;
                f[q][k] = sgn * (gm ? gm[k] : s_f[LBRS_IX((m * 4 + k) * kFWN + slot, 16 * kFWN, 12)]);
            }
            continue;
        }
        const float* g = nullptr;
        if (side_x >= 0) {
            if (kind_x == BC_DIRICHLET) g = a.ghost + side_x * GHOST_STRIDE + q * 4;
            else if (kind_x != BC_PERIODIC) si = si < 0 ? 0 : a.nx - 1;
        }
        if (!g && side_y >= 0) {
            if (kind_y == BC_DIRICHLET) g = a.ghost + side_y * GHOST_STRIDE + q * 4;
            else if (kind_y != BC_PERIODIC) sj = sj < 0 ? 0 : a.ny - 1;
        }
        if (g) {
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = g[k];
        } else {
            const int slot = (sj - (j0 - 1)) * kFWX + (si - (i0 - 1));
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = s_f[LBRS_IX((q * 4 + k) * kFWN + slot, 16 * kFWN, 12)];
        }
    }
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
    collide_store_2d<float, STORE_U>(a, (int64_t)j * a.nx + i, f);
}

// Phase-1 output of window slot w = (wi, wj): the post-collision populations into
// shared memory and, with STORE_U, the moments of a tile cell (the first step's)
// into a.Uout.
template <bool STORE_U>
__device__ __forceinline__ void step2_store_slot(const StepArgs<float>& a, float* s_f, int w, int wi, int wj, int i0,
                                                 int j0, const float U[4], const float out[4][4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_f[LBRS_IX((q * 4 + k) * kFWN + w, 16 * kFWN, 11)] = out[q][k];
    if constexpr (STORE_U) {
        const int i = i0 - 1 + wi, j = j0 - 1 + wj;
        if (wi >= 1 && wi <= kFTX && wj >= 1 && wj <= kFTY && i < a.nx && j < a.ny) {
#pragma unroll
            for (int k = 0; k < 4; ++k) a.Uout[LBRS_IX(k * a.N + (int64_t)j * a.nx + i, 4 * a.N, 11)] = U[k];
        }
    }
}

// The arguments of the second step: with STORE_U its moments go to the next
// record of the history, K * N values after the first step's.
__device__ __forceinline__ StepArgs<float> second_step_args(const StepArgs<float>& a, bool store_u)
{
    StepArgs<float> b = a;
    if (store_u) b.Uout = a.Uout + 4 * a.N;
    return b;
}

template <bool STORE_U, bool HALF>
__global__ void __launch_bounds__(kFTX * kFTY, 4) step2d_f32_fused2_kernel(const StepArgs<float> a)
{
    __shared__ float s_f[16 * kFWN];
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * kFTY;
    const bool px = a.bc[0] == BC_PERIODIC, py = a.bc[2] == BC_PERIODIC;

    // phase 1: step n -> n+1 on the window
    for (int w = threadIdx.x; w < kFWN; w += kFTX * kFTY) {
        int i = i0 - 1 + w % kFWX, j = j0 - 1 + w / kFWX;
        if (i < 0 || i >= a.nx) {
            if (!px) continue;
            i = wrap_index(i, a.nx);
        }
        if (j < 0 || j >= a.ny) {
            if (!py) continue;
            j = wrap_index(j, a.ny);
        }
        const int64_t c = (int64_t)j * a.nx + i;
        float f[4][4];
        if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
            const int64_t src[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = a.src[LBRS_IX((q * 4 + k) * a.N + src[q], 16 * a.N, 10)];
        } else {
            pull_edge_2d<float, HALF>(a, i, j, f);
        }
        float U[4], out[4][4];
        collide_2d<float>(a, f, U, out);
        step2_store_slot<STORE_U>(a, s_f, w, w % kFWX, w / kFWX, i0, j0, U, out);
    }
    __syncthreads();

    step2_phase2<STORE_U, HALF>(second_step_args(a, STORE_U), s_f, i0, j0);
}

// ---------------------------------------------------------------- two steps per launch, TMA-fed
//
// The same two steps on tiles of 32 x 16 cells, with the state the tile needs
// fetched by tensor copies (cp.async.bulk.tensor) into shared memory.  Population q
// of a window slot (i, j) is pulled from (i - sx_q, j - sy_q), so each population
// needs the window shifted by its own velocity: one copy per population of its 4
// fields over a 36 x 18 box, x from i0 (q = 1, 4: sources right of the slot) or
// i0 - 4 (q = 2, 3), y from j0 (sources above) or j0 - 2 (below); x starts on a
// 16-byte boundary.  Phase 1 computes the 34 x 18 window and writes each slot's
// post-collision populations over the box positions it pulled them from:
// population q of a slot is pulled from exactly one position, which no other slot
// reads, so each thread overwrites the 16 values it has just read (no hazard
// between threads) and the boxes are the only buffer (40.5 KB, five blocks per SM).
// Phase 2 computes the tile's second step, two cells per thread, reading population
// q of a source slot where it was pulled from.  Cells outside the grid arrive as
// zeros and are never read: a window slot whose pull leaves the grid interior takes
// the general path (global loads through pull_edge_2d).  One elected thread arms an
// mbarrier with the byte count and issues the copies; every thread waits on the
// barrier's phase with a bounded number of polls.  A wait that gives up sets
// *wait_flag (see give_up_tile), and the block leaves without touching the destination.
constexpr int kPX = 36;                                   // box columns (the 34-slot window, 16-byte aligned)
constexpr int kTY = 16, kTWY = kTY + 2, kTWN = kFWX * kTWY, kTPY = kTY + 2, kTPN = kPX * kTPY;
constexpr size_t kTallSmemBytes = 128 + 16u * kTPN * sizeof(float) + 16;
constexpr int kWaitPolls = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int polls)
{
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// A block whose bounded wait for its tile copies gave up.  The thread that issued the
// copies waits once more, again bounded, before the block leaves: while it waits the
// block (and its shared memory) stays resident, so copies that land in that time land
// in this block's own buffer.  The flag records the outcome: 1 if the copies landed
// (nothing is in flight when the block leaves), 2 if they did not (a copy may still
// complete into shared memory that a later block owns).  The host reports either as
// LBRS_ETIMEOUT; the other threads leave at once (the block's shared memory is
// released only when all of them have left).
__device__ __forceinline__ void give_up_tile(uint32_t bar, unsigned* wait_flag)
{
    if (threadIdx.x == 0) {
        const bool landed = mbar_wait_bounded(bar, 0, kWaitPolls);
        atomicMax(wait_flag, landed ? 1u : 2u);
    }
}

// The four population boxes of tile (i0, j0), each PN floats per field (36 columns
// and PN / 36 rows), onto one mbarrier.
template <int PN>
__device__ __forceinline__ void issue_tile_copy(const CUtensorMap* tmap, float* s_raw, uint32_t bar, int i0, int j0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(16u * PN * 4u) : "memory");
    const int x0[4] = {i0, i0 - 4, i0 - 4, i0};
    const int y0[4] = {j0, j0, j0 - 2, j0 - 2};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(s_raw + q * 4 * PN)),
            "l"((uint64_t)tmap), "r"(x0[q]), "r"(y0[q]), "r"(q * 4), "r"(bar)
            : "memory");
}

// An L2 prefetch of the boxes issue_tile_copy copies for tile (i0, j0).
__device__ __forceinline__ void prefetch_tile_l2(const CUtensorMap* tmap, int i0, int j0)
{
    const int x0[4] = {i0, i0 - 4, i0 - 4, i0};
    const int y0[4] = {j0, j0, j0 - 2, j0 - 2};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"((uint64_t)tmap),
                     "r"(x0[q]), "r"(y0[q]), "r"(q * 4)
                     : "memory");
}

// Position of population q, field k of window slot (wi, wj) in the boxes.
__device__ __forceinline__ int tall_pos(int q, int k, int wi, int wj)
{
    return (q * 4 + k) * kTPN + wj * kPX + wi + ((q == 1 || q == 2) ? 2 : 0);
}

template <bool STORE_U>
__device__ __forceinline__ void tall_store_slot(const StepArgs<float>& a, float* s_raw, int wi, int wj, int i0, int j0,
                                                const float U[4], const float out[4][4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) s_raw[LBRS_IX(tall_pos(q, k, wi, wj), 16 * kTPN, 16)] = out[q][k];
    if constexpr (STORE_U) {
        const int i = i0 - 1 + wi, j = j0 - 1 + wj;
        if (wi >= 1 && wi <= kFTX && wj >= 1 && wj <= kTY && i < a.nx && j < a.ny) {
#pragma unroll
            for (int k = 0; k < 4; ++k) a.Uout[LBRS_IX(k * a.N + (int64_t)j * a.nx + i, 4 * a.N, 16)] = U[k];
        }
    }
}

// Phase 1 on the 34 x 18 window, in place.
template <bool STORE_U, bool HALF>
__device__ __forceinline__ void tall_phase1(const StepArgs<float>& a, float* s_raw, int i0, int j0)
{
    if (i0 >= 2 && j0 >= 2 && i0 + kFTX + 2 <= a.nx && j0 + kTY + 2 <= a.ny) {
        // every window slot is an interior cell (the whole block takes this branch):
        // all pulls come from the copied boxes
        for (int w = threadIdx.x; w < kTWN; w += kFTX * kFTY) {
            const int wi = w % kFWX, wj = w / kFWX;
            float f[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = s_raw[LBRS_IX(tall_pos(q, k, wi, wj), 16 * kTPN, 16)];
            float U[4], out[4][4];
            collide_2d<float>(a, f, U, out);
            tall_store_slot<STORE_U>(a, s_raw, wi, wj, i0, j0, U, out);
        }
        return;
    }
    const bool px = a.bc[0] == BC_PERIODIC, py = a.bc[2] == BC_PERIODIC;
    for (int w = threadIdx.x; w < kTWN; w += kFTX * kFTY) {
        const int wi = w % kFWX, wj = w / kFWX;
        int i = i0 - 1 + wi, j = j0 - 1 + wj;
        if (i < 0 || i >= a.nx) {
            if (!px) continue;
            i = wrap_index(i, a.nx);
        }
        if (j < 0 || j >= a.ny) {
            if (!py) continue;
            j = wrap_index(j, a.ny);
        }
        float f[4][4];
        if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = s_raw[LBRS_IX(tall_pos(q, k, wi, wj), 16 * kTPN, 16)];
        } else {
            pull_edge_2d<float, HALF>(a, i, j, f);
        }
        float U[4], out[4][4];
        collide_2d<float>(a, f, U, out);
        tall_store_slot<STORE_U>(a, s_raw, wi, wj, i0, j0, U, out);
    }
}

// Phase 2 for tile cell (ti, tj), pulling from the window in the boxes.
template <bool STORE_U, bool HALF>
__device__ __forceinline__ void tall_phase2(const StepArgs<float>& a, const float* s_f, int i0, int j0, int ti, int tj)
{
    const int i = i0 + ti, j = j0 + tj;
    if (i >= a.nx || j >= a.ny) return;
    float f[4][4];
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        // sources (i + 1, j + 1), (i - 1, j + 1), (i - 1, j - 1), (i + 1, j - 1): window slots
        const int swi[4] = {ti + 2, ti, ti, ti + 2};
        const int swj[4] = {tj + 2, tj + 2, tj, tj};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = s_f[LBRS_IX(tall_pos(q, k, swi[q], swj[q]), 16 * kTPN, 17)];
        collide_store_2d<float, STORE_U>(a, (int64_t)j * a.nx + i, f);
        return;
    }
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    bool wall_top = false, wall_bottom = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int si = i - SX[q], sj = j - SY[q];
        const int side_y = sj < 0 ? 2 : (sj >= a.ny ? 3 : -1);
        const int side_x = si < 0 ? 0 : (si >= a.nx ? 1 : -1);
        const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
        const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
        if (side_y >= 0 && kind_y == BC_WALL) {
            if (side_y == 3) wall_top = true; else wall_bottom = true;
            continue;
        }
        if (HALF && side_y >= 0 && kind_y == BC_WALL_HALFWAY) {
            // the mirror image of this population leaving the horizontal neighbour on the wall
            // row (a periodic neighbour keeps its unwrapped slot, which holds the wrapped cell)
            const int m = 3 - q;
            const float* gm = nullptr;
            if (side_x >= 0) {
                if (kind_x == BC_DIRICHLET) gm = a.ghost + side_x * GHOST_STRIDE + m * 4;
                else if (kind_x != BC_PERIODIC) si = si < 0 ? 0 : a.nx - 1;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float sgn = k == 2 ? -1.f : 1.f;
                f[q][k] = sgn * (gm ? gm[k] : s_f[LBRS_IX(tall_pos(m, k, si - (i0 - 1), j - (j0 - 1)), 16 * kTPN, 17)]);
            }
            continue;
        }
        const float* g = nullptr;
        if (side_x >= 0) {
            if (kind_x == BC_DIRICHLET) g = a.ghost + side_x * GHOST_STRIDE + q * 4;
            else if (kind_x != BC_PERIODIC) si = si < 0 ? 0 : a.nx - 1;
        }
        if (!g && side_y >= 0) {
            if (kind_y == BC_DIRICHLET) g = a.ghost + side_y * GHOST_STRIDE + q * 4;
            else if (kind_y != BC_PERIODIC) sj = sj < 0 ? 0 : a.ny - 1;
        }
        if (g) {
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = g[k];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                f[q][k] = s_f[LBRS_IX(tall_pos(q, k, si - (i0 - 1), sj - (j0 - 1)), 16 * kTPN, 17)];
        }
    }
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
    collide_store_2d<float, STORE_U>(a, (int64_t)j * a.nx + i, f);
}

// Internal walls in the two-step kernel.  The block keeps the solidity of the
// tile's pull range, the 36 x 20 cells from (i0 - 2, j0 - 2), in shared memory:
// every cell whose solidity the two steps consult lies there (window slots, their
// sources and the x and y neighbours of the mirror rule).  A coordinate outside
// the domain takes solid_at's value (wrapped, clamped, or fluid beyond a Dirichlet
// or wall side), wrapped as often as needed: the sources of a periodic window slot
// lie two cells out, and a solid one among them must send the tile down the
// obstacle path even though the slot's own pull reads the global mask.
constexpr int kMX = kFTX + 4, kMY = kTY + 4, kMN = kMX * kMY;
constexpr size_t kTallObstSmemBytes = kTallSmemBytes + kMN;

// Fill the mask window; true when any of its cells is solid (for the whole block).
__device__ __forceinline__ bool load_mask_window(const StepArgs<float>& a, uint8_t* s_m, int i0, int j0)
{
    int any = 0;
    for (int m = threadIdx.x; m < kMN; m += kFTX * kFTY) {
        int i = i0 - 2 + m % kMX, j = j0 - 2 + m / kMX;
        bool fluid = false;
        if (i < 0 || i >= a.nx) {
            const int kind = i < 0 ? a.bc[0] : a.bc[1];
            if (kind == BC_PERIODIC) i = wrap_index(i, a.nx);
            else if (kind == BC_TRANSMISSIVE) i = i < 0 ? 0 : a.nx - 1;
            else fluid = true;
        }
        if (j < 0 || j >= a.ny) {
            const int kind = j < 0 ? a.bc[2] : a.bc[3];
            if (kind == BC_PERIODIC) j = wrap_index(j, a.ny);
            else if (kind == BC_TRANSMISSIVE) j = j < 0 ? 0 : a.ny - 1;
            else fluid = true;
        }
        const uint8_t v = !fluid && a.solid[LBRS_IX((int64_t)j * a.nx + i, a.N, 14)] ? 1 : 0;
        s_m[m] = v;
        any |= v;
    }
    return __syncthreads_or(any) != 0;
}

__device__ __forceinline__ bool msolid(const uint8_t* s_m, int i, int j, int i0, int j0)
{
    return s_m[LBRS_IX((j - j0 + 2) * kMX + (i - i0 + 2), kMN, 14)] != 0;
}

// Phase 1 with internal walls: solid window slots are skipped (phase 2 never
// reads them: a population pulled from a solid cell is replaced by the mirror
// rule); a fluid slot with a solid source, or on a domain side, takes the
// single-step kernel's obstacle pull from global memory.
__device__ __forceinline__ void tall_phase1_obst(const StepArgs<float>& a, float* s_raw, const uint8_t* s_m, int i0,
                                                 int j0)
{
    const bool px = a.bc[0] == BC_PERIODIC, py = a.bc[2] == BC_PERIODIC;
    for (int w = threadIdx.x; w < kTWN; w += kFTX * kFTY) {
        const int wi = w % kFWX, wj = w / kFWX;
        const int ui = i0 - 1 + wi, uj = j0 - 1 + wj;
        int i = ui, j = uj;
        if (i < 0 || i >= a.nx) {
            if (!px) continue;
            i = wrap_index(i, a.nx);
        }
        if (j < 0 || j >= a.ny) {
            if (!py) continue;
            j = wrap_index(j, a.ny);
        }
        if (msolid(s_m, ui, uj, i0, j0)) continue;
        float f[4][4];
        if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1 && !msolid(s_m, ui + 1, uj + 1, i0, j0) &&
            !msolid(s_m, ui - 1, uj + 1, i0, j0) && !msolid(s_m, ui - 1, uj - 1, i0, j0) &&
            !msolid(s_m, ui + 1, uj - 1, i0, j0)) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = s_raw[LBRS_IX(tall_pos(q, k, wi, wj), 16 * kTPN, 13)];
        } else {
            pull_obstacle_2d<float>(a, i, j, f);
        }
        float U[4], out[4][4];
        collide_2d<float>(a, f, U, out);
        tall_store_slot<false>(a, s_raw, wi, wj, i0, j0, U, out);
    }
}

// Phase 2 with internal walls: a solid tile cell is carried unchanged (its two
// steps copy it); a fluid cell pulls from the window and resolves solid sources
// and domain sides in pull_obstacle_2d's order.
__device__ __forceinline__ void tall_phase2_obst(const StepArgs<float>& a, const float* s_f, const uint8_t* s_m, int i0,
                                                 int j0, int ti, int tj)
{
    const int i = i0 + ti, j = j0 + tj;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    if (msolid(s_m, i, j, i0, j0)) {
#pragma unroll
        for (int n = 0; n < 16; ++n) a.dst[LBRS_IX(n * a.N + c, 16 * a.N, 15)] = a.src[LBRS_IX(n * a.N + c, 16 * a.N, 15)];
        return;
    }
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    float f[4][4];
    bool wall_top = false, wall_bottom = false;
    bool unknown[4] = {false, false, false, false};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int si = i - SX[q], sj = j - SY[q];
        const int side_y = sj < 0 ? 2 : (sj >= a.ny ? 3 : -1);
        const int side_x = si < 0 ? 0 : (si >= a.nx ? 1 : -1);
        const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
        const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
        if (side_y >= 0 && kind_y == BC_WALL) {
            if (side_y == 3) wall_top = true; else wall_bottom = true;
            continue;
        }
        const float* g = nullptr;
        if (side_x >= 0) {
            if (kind_x == BC_DIRICHLET) g = a.ghost + side_x * GHOST_STRIDE + q * 4;
            else if (kind_x != BC_PERIODIC) si = si < 0 ? 0 : a.nx - 1;
        }
        if (!g && side_y >= 0) {
            if (kind_y == BC_DIRICHLET) g = a.ghost + side_y * GHOST_STRIDE + q * 4;
            else if (kind_y != BC_PERIODIC) sj = sj < 0 ? 0 : a.ny - 1;
        }
        if (!g && msolid(s_m, si, sj, i0, j0)) {
            unknown[q] = true;
            continue;
        }
        if (g) {
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = g[k];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                f[q][k] = s_f[LBRS_IX(tall_pos(q, k, si - (i0 - 1), sj - (j0 - 1)), 16 * kTPN, 12)];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!unknown[q]) continue;
        const bool xn = msolid(s_m, i - SX[q], j, i0, j0), yn = msolid(s_m, i, j - SY[q], i0, j0);
        const bool flip_x = !(yn && !xn), flip_y = !(xn && !yn);
        const int mx = flip_x ? -SX[q] : SX[q], my = flip_y ? -SY[q] : SY[q];
        const int m = my < 0 ? (mx < 0 ? 0 : 1) : (mx > 0 ? 2 : 3);
        const float su = flip_x ? -1.f : 1.f, sv = flip_y ? -1.f : 1.f;
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
            if (mm != m) continue;
            f[q][0] = f[mm][0];
            f[q][1] = su * f[mm][1];
            f[q][2] = sv * f[mm][2];
            f[q][3] = f[mm][3];
        }
    }
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
    collide_store_2d<float>(a, c, f);
}

// One block per 32 x 16 tile, five resident blocks per SM (48 registers, 40.5 KB of
// shared memory; 41.2 KB with the obstacle mask window of OBST).  Forms measured
// slower: 32 x 8 tiles with a separate window buffer (the same time on a flushed
// 1024^2 grid, 10 % less throughput on large grids); blocks reused for further
// tiles with the next copy issued early (fewer resident warps).  Once its boxes have
// landed, a block asks the L2 for the boxes of the block `ahead` places later in launch
// order (half a wave; an earlier form that prefetched the following tile's boxes early
// evicted halo rows still to be read).
template <bool STORE_U, bool OBST = false, bool HALF = false>
__global__ void __launch_bounds__(kFTX * kFTY, 5)
    step2d_f32_fused2_tall_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs<float> a,
                                  unsigned* wait_flag, int ahead)
{
    static_assert(!(STORE_U && OBST), "the recording form has no internal walls");
    extern __shared__ unsigned char smem_dyn[];
    float* s_raw = (float*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
    uint64_t* bar_p = (uint64_t*)(s_raw + 16 * kTPN);
    const uint32_t bar = smem_addr(bar_p);
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * kTY;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_tile_copy<kTPN>(&tmap, s_raw, bar, i0, j0);
    }
    __syncthreads();
    bool obst = false;
    uint8_t* s_m = (uint8_t*)(bar_p + 2);
    if constexpr (OBST) obst = load_mask_window(a, s_m, i0, j0);   // while the copies are in flight
    const bool arrived = mbar_wait_bounded(bar, 0, kWaitPolls);
    if (!__syncthreads_and(arrived)) {
        give_up_tile(bar, wait_flag);
        return;
    }
    if (threadIdx.x == 0 && ahead > 0) {
        const int64_t later = (int64_t)blockIdx.y * gridDim.x + blockIdx.x + ahead;
        if (later < (int64_t)gridDim.x * gridDim.y)
            prefetch_tile_l2(&tmap, (int)(later % gridDim.x) * kFTX, (int)(later / gridDim.x) * kTY);
    }
    const int ti = threadIdx.x % kFTX, tj = threadIdx.x / kFTX;
    if (OBST && obst) {
        tall_phase1_obst(a, s_raw, s_m, i0, j0);
        __syncthreads();
        tall_phase2_obst(a, s_raw, s_m, i0, j0, ti, tj);
        tall_phase2_obst(a, s_raw, s_m, i0, j0, ti, tj + kFTY);
        return;
    }
    tall_phase1<STORE_U, HALF>(a, s_raw, i0, j0);
    __syncthreads();
    const StepArgs<float> b = second_step_args(a, STORE_U);
    tall_phase2<STORE_U, HALF>(b, s_raw, i0, j0, ti, tj);
    tall_phase2<STORE_U, HALF>(b, s_raw, i0, j0, ti, tj + kFTY);
}

// ---------------------------------------------------------------- three steps per launch, TMA-fed
//
// The state is read and written once per three steps (128 B per cell and launch, 42.7 B per
// lattice update).  A block of 192 threads owns a 32 x 12 tile (five blocks per SM: 41 KB of boxes and
// 64 registers each); window slot (wi, wj), wi < 36, wj < 16, is the
// cell (i0 - 2 + wi, j0 - 2 + wj) (the tile and two cells of halo).  Four tensor copies bring,
// per population q, the 40 x 16 x 4-field box of the values that the window's slots pull
// (shifted by the velocity, x starting on a 16-byte boundary at i0 - 4): position f3_pos(q, k,
// wi, wj) holds what slot (wi, wj) pulls.
//   phase 1  step n -> n+1 on the window, each slot's results written over the positions it
//            pulled them from (one reader per position);
//   phase 2  step n+1 -> n+2 on the 34 x 14 inner slots: slot (u, v) pulls population q from
//            slot (u - sx, v - sy), at f3_pos(q, ., u - sx, v - sy), and writes its own
//            population q over that same position (again one reader per position);
//   phase 3  step n+2 -> n+3 for the tile: cell (x, y) finds population q of its source slot
//            (x - sx, y - sy) at f3_pos(q, ., x - 2 sx, y - 2 sy); the result goes to global memory.
// Slots beyond a non-periodic side are not computed; on tiles at the grid's edge a fix-up pass
// after phases 1 and 2 writes into them what the single-step pull resolves there (a Dirichlet
// ghost, or the clamped cell's values, x side first), so phases 2 and 3 gather uniformly.  Slots
// beyond a periodic side compute the wrapped cell (by the global pull of the single-step kernel:
// the boxes hold the copy's fill there).  Every value is formed with the single-step kernel's
// arithmetic, so three steps are bit-identical to single steps.  Not for internal walls or halfway
// walls (those take the two-step kernel).
constexpr int kT3Y = 12, kT3T = 192, kT3B = 5;             // tile rows, threads and blocks per SM
constexpr int kP3X = 40;                                    // box columns
constexpr int kW3X = 36, kW3Y = kT3Y + 4, kW3N = kW3X * kW3Y;  // phase-1 window (tile + 2 halo)
constexpr int kB3X = 34, kB3Y = kT3Y + 2, kB3N = kB3X * kB3Y;  // phase-2 slots (tile + 1 halo)
constexpr int kP3N = kP3X * kW3Y;                           // floats per field plane of a box
constexpr size_t kF3SmemBytes = 128 + 16u * kP3N * sizeof(float) + 16;

// Position of population q, field k, as pulled by window slot (wi, wj).
__device__ __forceinline__ int f3_pos(int q, int k, int wi, int wj)
{
    return (q * 4 + k) * kP3N + wj * kP3X + wi + ((q == 0 || q == 3) ? 3 : 1);
}

// The four population boxes of tile (i0, j0) onto one mbarrier.
__device__ __forceinline__ void issue_tile_copy3(const CUtensorMap* tmap, float* s_raw, uint32_t bar, int i0, int j0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(16u * kP3N * 4u) : "memory");
    const int y0[4] = {j0 - 1, j0 - 1, j0 - 3, j0 - 3};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(s_raw + q * 4 * kP3N)),
            "l"((uint64_t)tmap), "r"(i0 - 4), "r"(y0[q]), "r"(q * 4), "r"(bar)
            : "memory");
}

// An L2 prefetch of the four population boxes of tile (i0, j0), the boxes issue_tile_copy3 copies.
__device__ __forceinline__ void prefetch_tile_l2_3(const CUtensorMap* tmap, int i0, int j0)
{
    const int y0[4] = {j0 - 1, j0 - 1, j0 - 3, j0 - 3};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"((uint64_t)tmap),
                     "r"(i0 - 4), "r"(y0[q]), "r"(q * 4)
                     : "memory");
}

// How the window slot of unwrapped cell (ui, uj) gets its values: 0 computed there (inside the
// grid, or beyond a periodic side: the wrapped cell); 1 the ghost of Dirichlet side *gs; 2 the
// values of the slot of unwrapped cell (*ci, *cj) (a transmissive side's clamped cell); 3 none
// (beyond a wall side, whose populations the wall relations replace, or farther beyond a side
// than `reach` cells -- 2 for phase 1, 1 for phase 2 -- which no later phase pulls).
__device__ __forceinline__ int f3_resolve(const StepArgs<float>& a, int ui, int uj, int& ci, int& cj, int& gs,
                                          int reach)
{
    ci = ui;
    cj = uj;
    const int bx = ui < 0 ? -ui : (ui >= a.nx ? ui - a.nx + 1 : 0);
    const int by = uj < 0 ? -uj : (uj >= a.ny ? uj - a.ny + 1 : 0);
    const bool px = a.bc[0] == BC_PERIODIC, py = a.bc[2] == BC_PERIODIC;
    if (bx > reach || by > reach || (bx > 1 && !px) || (by > 1 && !py)) return 3;
    if (bx && !px) {
        const int side = ui < 0 ? 0 : 1;
        if ((side == 0 ? a.bc[0] : a.bc[1]) == BC_DIRICHLET) {
            gs = side;
            return 1;
        }
        ci = ui < 0 ? 0 : a.nx - 1;
    }
    if (by && !py) {
        const int side = uj < 0 ? 2 : 3;
        const int kind = side == 2 ? a.bc[2] : a.bc[3];
        if (kind == BC_DIRICHLET) {
            gs = side;
            return 1;
        }
        if (kind == BC_WALL) return 3;
        cj = uj < 0 ? 0 : a.ny - 1;
    }
    return (ci == ui && cj == uj) ? 0 : 2;
}

// The on-node wall relations (Section II.E) for a cell on row j.
__device__ __forceinline__ void f3_walls(const StepArgs<float>& a, int j, float f[4][4])
{
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
}

// Window slots by warp: pass p < WY is window row p, one slot a lane (32 contiguous positions of a
// box row, so no two lanes share a bank); the passes after it take the columns beyond 32.  Returns
// false for the lanes of the last pass that have no slot.
template <int WX, int WY>
__host__ __device__ constexpr int window_passes()
{
    return WY + ((WX - 32) * WY + 31) / 32;
}

template <int WX, int WY>
__device__ __forceinline__ bool window_slot(int p, int lane, int& wi, int& wj)
{
    if (p < WY) {
        wi = lane;
        wj = p;
        return true;
    }
    const int L = (p - WY) * 32 + lane;
    wi = 32 + L % (WX - 32);
    wj = L / (WX - 32);
    return L < (WX - 32) * WY;
}

// The three steps of tile (i0, j0) from its boxes at s (landed), by THR threads.  STORE_U: a
// recording launch, which also writes the moments of each step's collision for the tile's cells to
// a.Uout (step n+1), a.Uout + 4N (n+2) and a.Uout + 8N (n+3), as three recording steps would.
template <int THR, bool STORE_U>
__device__ __forceinline__ void f3_tile(const StepArgs<float>& a, float* s, int i0, int j0)
{
    constexpr int kThr = THR;
    // every slot and every source of phase 1 inside the grid: no resolution anywhere
    const bool inside = i0 >= 3 && j0 >= 3 && i0 + kFTX + 3 <= a.nx && j0 + kT3Y + 3 <= a.ny;

    // slots go to warps by window row (window_slot)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kNW = kThr / 32;

    // phase 1: step n -> n+1 on the window, in place
    for (int p = warp; p < window_passes<kW3X, kW3Y>(); p += kNW) {
        int wi, wj;
        if (!window_slot<kW3X, kW3Y>(p, lane, wi, wj)) continue;
        float f[4][4];
        bool boxed = inside;
        if (!inside) {
            const int ui = i0 - 2 + wi, uj = j0 - 2 + wj;
            int ci, cj, gs;
            if (f3_resolve(a, ui, uj, ci, cj, gs, 2) != 0) continue;
            boxed = ui >= 1 && ui <= a.nx - 2 && uj >= 1 && uj <= a.ny - 2;
            if (!boxed) {
                const int i = (ui < 0 || ui >= a.nx) ? wrap_index(ui, a.nx) : ui;
                const int j = (uj < 0 || uj >= a.ny) ? wrap_index(uj, a.ny) : uj;
                pull_edge_2d<float, false>(a, i, j, f);
            }
        }
        if (boxed) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = s[LBRS_IX(f3_pos(q, k, wi, wj), 16 * kP3N, 23)];
        }
        float U[4], out[4][4];
        collide_2d<float>(a, f, U, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) s[LBRS_IX(f3_pos(q, k, wi, wj), 16 * kP3N, 23)] = out[q][k];
        if constexpr (STORE_U) {
            const int i = i0 - 2 + wi, j = j0 - 2 + wj;
            if (wi >= 2 && wi < 2 + kFTX && wj >= 2 && wj < 2 + kT3Y && i < a.nx && j < a.ny) {
#pragma unroll
                for (int k = 0; k < 4; ++k) a.Uout[LBRS_IX(k * a.N + (int64_t)j * a.nx + i, 4 * a.N, 29)] = U[k];
            }
        }
    }
    __syncthreads();
    if (!inside) {
        // window slots beyond a non-periodic side: what the single-step pull resolves there
        for (int w = threadIdx.x; w < kW3N; w += kThr) {
            const int wi = w % kW3X, wj = w / kW3X;
            int ci, cj, gs;
            const int r = f3_resolve(a, i0 - 2 + wi, j0 - 2 + wj, ci, cj, gs, 2);
            if (r != 1 && r != 2) continue;
            const int cwi = ci - (i0 - 2), cwj = cj - (j0 - 2);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    s[LBRS_IX(f3_pos(q, k, wi, wj), 16 * kP3N, 23)] =
                        r == 1 ? a.ghost[gs * GHOST_STRIDE + q * 4 + k] : s[LBRS_IX(f3_pos(q, k, cwi, cwj), 16 * kP3N, 23)];
        }
        __syncthreads();
    }

    // phase 2: step n+1 -> n+2 on the inner slots, each written over the positions it pulled
    for (int p = warp; p < window_passes<kB3X, kB3Y>(); p += kNW) {
        int u, v;
        if (!window_slot<kB3X, kB3Y>(p, lane, u, v)) continue;
        ++u;                                          // slot (u, v) of the window, u, v >= 1
        ++v;
        const int uj = j0 - 2 + v;
        if (!inside) {
            int ci, cj, gs;
            if (f3_resolve(a, i0 - 2 + u, uj, ci, cj, gs, 1) != 0) continue;
        }
        // sources (u - sx, v - sy): q0 (u+1, v+1), q1 (u-1, v+1), q2 (u-1, v-1), q3 (u+1, v-1)
        const int su[4] = {u + 1, u - 1, u - 1, u + 1};
        const int sv[4] = {v + 1, v + 1, v - 1, v - 1};
        float f[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = s[LBRS_IX(f3_pos(q, k, su[q], sv[q]), 16 * kP3N, 24)];
        if (!inside) f3_walls(a, uj, f);
        float U[4], out[4][4];
        collide_2d<float>(a, f, U, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) s[LBRS_IX(f3_pos(q, k, su[q], sv[q]), 16 * kP3N, 24)] = out[q][k];
        if constexpr (STORE_U) {
            const int i = i0 - 2 + u;
            if (u >= 2 && u < 2 + kFTX && v >= 2 && v < 2 + kT3Y && i < a.nx && uj < a.ny) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    a.Uout[LBRS_IX((4 + k) * a.N + (int64_t)uj * a.nx + i, 8 * a.N, 29)] = U[k];
            }
        }
    }
    __syncthreads();
    if (!inside) {
        // inner slots beyond a non-periodic side, stored where phase 3 looks for them
        for (int b = threadIdx.x; b < kB3N; b += kThr) {
            const int u = 1 + b % kB3X, v = 1 + b / kB3X;
            int ci, cj, gs;
            const int r = f3_resolve(a, i0 - 2 + u, j0 - 2 + v, ci, cj, gs, 1);
            if (r != 1 && r != 2) continue;
            const int cu = ci - (i0 - 2), cv = cj - (j0 - 2);
            const int du[4] = {1, -1, -1, 1}, dv[4] = {1, 1, -1, -1};   // -sx, -sy
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    s[LBRS_IX(f3_pos(q, k, u + du[q], v + dv[q]), 16 * kP3N, 24)] =
                        r == 1 ? a.ghost[gs * GHOST_STRIDE + q * 4 + k]
                               : s[LBRS_IX(f3_pos(q, k, cu + du[q], cv + dv[q]), 16 * kP3N, 24)];
        }
        __syncthreads();
    }

    // phase 3: step n+2 -> n+3 for the tile, one tile row a warp (kFTX * kT3Y / THR rows a warp)
#pragma unroll
    for (int rep = 0; rep < kFTX * kT3Y / THR; ++rep) {
        const int ty = warp + rep * kNW;
        const int i = i0 + lane, j = j0 + ty;
        if (i >= a.nx || j >= a.ny) continue;
        const int x = lane + 2, y = ty + 2;
        // population q of source slot (x - sx, y - sy) lies at (x - 2 sx, y - 2 sy)
        const int px[4] = {x + 2, x - 2, x - 2, x + 2};
        const int py[4] = {y + 2, y + 2, y - 2, y - 2};
        float f[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = s[LBRS_IX(f3_pos(q, k, px[q], py[q]), 16 * kP3N, 25)];
        if (!inside) f3_walls(a, j, f);
        if constexpr (STORE_U) {
            StepArgs<float> c = a;
            c.Uout = a.Uout + 8 * a.N;
            collide_store_2d<float, true>(c, (int64_t)j * a.nx + i, f);
        } else {
            collide_store_2d<float>(a, (int64_t)j * a.nx + i, f);
        }
    }
}

// One block a tile.  Once its own boxes have landed, the block asks the L2 for the boxes of the
// block `ahead` places later in launch order (ahead = half the resident blocks of the device, 0
// for none): that block starts about half a wave later, and its copies then find their data in the
// L2 instead of queueing behind the wave's DRAM reads.  The prefetch moves no byte that the launch
// would not read anyway; it only reads it earlier.
template <bool STORE_U>
__global__ void __launch_bounds__(kT3T, kT3B)
    step2d_f32_fused3_kernel(const __grid_constant__ CUtensorMap tmap, const StepArgs<float> a, unsigned* wait_flag,
                             int ahead)
{
    extern __shared__ unsigned char smem_dyn[];
    float* s = (float*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
    uint64_t* bar_p = (uint64_t*)(s + 16 * kP3N);
    const uint32_t bar = smem_addr(bar_p);
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * kT3Y;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_tile_copy3(&tmap, s, bar, i0, j0);
    }
    __syncthreads();
    const bool arrived = mbar_wait_bounded(bar, 0, kWaitPolls);
    if (!__syncthreads_and(arrived)) {
        give_up_tile(bar, wait_flag);
        return;
    }
    if (threadIdx.x == 0 && ahead > 0) {
        const int64_t later = (int64_t)blockIdx.y * gridDim.x + blockIdx.x + ahead;
        if (later < (int64_t)gridDim.x * gridDim.y)
            prefetch_tile_l2_3(&tmap, (int)(later % gridDim.x) * kFTX, (int)(later / gridDim.x) * kT3Y);
    }
    f3_tile<kT3T, STORE_U>(a, s, i0, j0);
}

// ---------------------------------------------------------------- scalar D2Q4, two steps per launch
//
// One block of 256 threads per 32 x TY tile (TY = 16, 24 or 32 rows); the state (4 populations of one
// field) is read and written once per two steps, 32 B per cell and launch.  Phase 1 computes step n+1 on
// the 34 x (TY + 2) window (the tile and one cell of halo) into shared memory with the single-step kernel's pull and collision; slots beyond
// a periodic side compute the wrapped cell, slots beyond another side are not needed.  Phase 2 computes
// step n+2 for the tile, taking population q from where the single-step pull resolves its source: within
// the grid or beyond a periodic side the source's (unwrapped) slot, beyond a transmissive side the clamped
// cell's slot, beyond a Dirichlet side the ghost of the side's profile (x side first).  The ghosts do not
// change between the steps, so the result is bit-identical to two single steps.
template <int TY>
__global__ void __launch_bounds__(kFTX * kFTY) step2ds_fused2_kernel(const StepArgs<float> a)
{
    constexpr int kTWN = kFWX * (TY + 2);   // window slots: the tile and one cell of halo
    __shared__ float s_f[4 * kTWN];
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * TY;
    const bool px = a.bc[0] == BC_PERIODIC, py = a.bc[2] == BC_PERIODIC;
    // the window and every source of its slots inside the grid: direct offsets in both phases
    const bool inside = i0 >= 2 && j0 >= 2 && i0 + kFTX + 2 <= a.nx && j0 + TY + 2 <= a.ny;
    if (inside) {
        // every load of the thread's window slots (kPass of them: three at 16 rows, five at 32) is issued
        // before the first collision: the phase is bound by the latency of these loads, and kPass slots a
        // thread keep kPass times as many in flight as one slot at a time
        constexpr int kThr = kFTX * kFTY, kPass = (kTWN + kThr - 1) / kThr;
        static_assert((kPass - 1) * kThr <= kTWN, "every pass but the last is full");
        float f[kPass][4];
#pragma unroll
        for (int p = 0; p < kPass; ++p) {
            const int w = threadIdx.x + p * kThr;
            if (p < kPass - 1 || w < kTWN) {
                const int64_t c = (int64_t)(j0 - 1 + w / kFWX) * a.nx + (i0 - 1 + w % kFWX);
                const int64_t src[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
                for (int q = 0; q < 4; ++q) f[p][q] = a.src[LBRS_IX(q * a.N + src[q], 4 * a.N, 51)];
            }
        }
#pragma unroll
        for (int p = 0; p < kPass; ++p) {
            const int w = threadIdx.x + p * kThr;
            if (p < kPass - 1 || w < kTWN) {
                float out[4];
                collide_2ds<float>(a, f[p], out);
#pragma unroll
                for (int q = 0; q < 4; ++q) s_f[LBRS_IX(q * kTWN + w, 4 * kTWN, 52)] = out[q];
            }
        }
        __syncthreads();
        const int ti = threadIdx.x % kFTX;
        for (int tj = threadIdx.x / kFTX; tj < TY; tj += kFTY) {
            // the source x - c_q of cell (ti, tj) is window slot (ti + 1 - sx_q, tj + 1 - sy_q)
            const int s0 = (tj + 1) * kFWX + ti + 1;
            const int sl[4] = {s0 + kFWX + 1, s0 + kFWX - 1, s0 - kFWX - 1, s0 - kFWX + 1};
            float f[4], out[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) f[q] = s_f[LBRS_IX(q * kTWN + sl[q], 4 * kTWN, 53)];
            collide_2ds<float>(a, f, out);
            const int64_t c = (int64_t)(j0 + tj) * a.nx + i0 + ti;
#pragma unroll
            for (int q = 0; q < 4; ++q) a.dst[LBRS_IX(q * a.N + c, 4 * a.N, 53)] = out[q];
        }
        return;
    }
    for (int w = threadIdx.x; w < kTWN; w += kFTX * kFTY) {
        int i = i0 - 1 + w % kFWX, j = j0 - 1 + w / kFWX;
        if (i < 0 || i >= a.nx) {
            if (!px) continue;
            i = wrap_index(i, a.nx);
        }
        if (j < 0 || j >= a.ny) {
            if (!py) continue;
            j = wrap_index(j, a.ny);
        }
        float f[4];
        if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
            const int64_t c = (int64_t)j * a.nx + i;
            const int64_t src[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
            for (int q = 0; q < 4; ++q) f[q] = a.src[LBRS_IX(q * a.N + src[q], 4 * a.N, 51)];
        } else {
            pull_edge_2ds<float>(a, i, j, f);
        }
        float out[4];
        collide_2ds<float>(a, f, out);
#pragma unroll
        for (int q = 0; q < 4; ++q) s_f[LBRS_IX(q * kTWN + w, 4 * kTWN, 52)] = out[q];
    }
    __syncthreads();
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    const int ti = threadIdx.x % kFTX;
    for (int tj = threadIdx.x / kFTX; tj < TY; tj += kFTY) {
        const int i = i0 + ti, j = j0 + tj;
        if (i >= a.nx || j >= a.ny) continue;
        float f[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int si = i - SX[q], sj = j - SY[q];     // the source, wrapped or clamped as the single step does
            int ui = si, uj = sj;                   // its slot: unwrapped beyond a periodic side
            const int side_y = sj < 0 ? 2 : (sj >= a.ny ? 3 : -1);
            const int side_x = si < 0 ? 0 : (si >= a.nx ? 1 : -1);
            const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
            const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
            const float* g = nullptr;
            int m = 0;
            if (side_x >= 0) {
                if (kind_x == BC_DIRICHLET) {
                    g = a.ghost + side_x * GHOST_STRIDE;
                    m = sj;
                } else if (kind_x == BC_PERIODIC) {
                    si = si < 0 ? si + a.nx : si - a.nx;
                } else {
                    si = si < 0 ? 0 : a.nx - 1;
                    ui = si;
                }
            }
            if (!g && side_y >= 0) {
                if (kind_y == BC_DIRICHLET) {
                    g = a.ghost + side_y * GHOST_STRIDE;
                    m = si;
                } else if (kind_y != BC_PERIODIC) {
                    sj = sj < 0 ? 0 : a.ny - 1;
                    uj = sj;
                }
            }
            f[q] = g ? ghost_population_2ds<float>(a, g, m, q)
                     : s_f[LBRS_IX(q * kTWN + (uj - (j0 - 1)) * kFWX + (ui - (i0 - 1)), 4 * kTWN, 53)];
        }
        float out[4];
        collide_2ds<float>(a, f, out);
        const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) a.dst[LBRS_IX(q * a.N + c, 4 * a.N, 53)] = out[q];
    }
}

// Failure-detection self-test: one block waits, with the tile kernels' bounded wait,
// on an mbarrier that nothing completes (no copy, no arrival); the wait gives up after
// `polls` polls and the block raises *wait_flag as the tile kernels do.  Nothing is in
// flight when it returns.
__global__ void __launch_bounds__(32) wait_timeout_selftest_kernel(unsigned* wait_flag, int polls)
{
    __shared__ uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool arrived = mbar_wait_bounded(b, 0, polls);
    if (!__syncthreads_and(arrived) && threadIdx.x == 0) atomicExch(wait_flag, 1u);
}

// ---------------------------------------------------------------- adjoint, two steps per launch
//
// The adjoint step pushes fbar(x) = (1 - w) g(x) + w J_E(U(x))^T g(x) to x - c_q.
// Read as a pull, g^{s-1}(y)_q = k^s_q(y + c_q) with k^s = fbar computed at its own
// cell.  Storing k instead of g makes the adjoint sweep the same shape as the
// forward step -- gather, then a local operator -- so two steps fuse like the
// forward's: phase 1 forms k^{s-1} on the tile's 34 x 10 window (periodic wrap)
// into shared memory, phase 2 forms k^{s-2} on the tile.  Every value is the push
// kernel's expression at the same cell, so the sweep is bit-identical to it.

__device__ __forceinline__ void adj_local(const AdjArgs<float>& a, const float U[4], const float g[4][4],
                                          float out[4][4])
{
    float ubar[4];
    equilibrium_vjp2d<float>(U, g, a.gamma, a.gm1, a.c, ubar);
    const bool eq_only = a.om1 == 0.f;   // omega = 1: as in the push kernel
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[q][k] = eq_only ? ubar[k] : a.om1 * g[q][k] + a.om * ubar[k];
}

// g(x)_q = k_q(x + c_q) for a cell (i, j) of the periodic grid.
__device__ __forceinline__ void adj_gather(const AdjArgs<float>& a, int i, int j, float g[4][4])
{
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        const int64_t c = (int64_t)j * a.nx + i;
        const int64_t src[4] = {c - a.nx - 1, c - a.nx + 1, c + a.nx + 1, c + a.nx - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX((q * 4 + k) * a.N + src[q], 16 * a.N, 32)];
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t s = (int64_t)wrap_index(j + SY[q], a.ny) * a.nx + wrap_index(i + SX[q], a.nx);
#pragma unroll
        for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX((q * 4 + k) * a.N + s, 16 * a.N, 32)];
    }
}

// k(x) = (1 - w) g(x) + w J_E(U(x))^T g(x), pointwise (the start of a sweep).
__global__ void __launch_bounds__(256) adj_local_kernel(const AdjArgs<float> a)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += (int64_t)gridDim.x * blockDim.x) {
        float g[4][4], U[4], out[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 32)];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 32)];
        adj_local(a, U, g, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) a.gout[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 32)] = out[q][k];
    }
}

// One step: g = gathered k; with a.U, out = the local operator of g, else out = g
// (the last step of a segment, which hands g to the earlier segment).
__global__ void __launch_bounds__(256) adj_pull_kernel(const AdjArgs<float> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    float g[4][4], out[4][4];
    adj_gather(a, i, j, g);
    if (a.U) {
        float U[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 32)];
        adj_local(a, U, g, out);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) out[q][k] = g[q][k];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) a.gout[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 32)] = out[q][k];
}

// Two steps: k^s (a.gin) -> k^{s-2} (a.gout); a.U = U_{s-1}, U2 = U_{s-2}.
__global__ void __launch_bounds__(kFTX * kFTY, 4) adj_fused2_kernel(const AdjArgs<float> a, const float* __restrict__ U2)
{
    __shared__ float s_k[16 * kFWN];
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * kFTY;
    for (int w = threadIdx.x; w < kFWN; w += kFTX * kFTY) {
        const int i = wrap_index(i0 - 1 + w % kFWX, a.nx), j = wrap_index(j0 - 1 + w / kFWX, a.ny);
        float g[4][4], U[4], out[4][4];
        adj_gather(a, i, j, g);
        const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 33)];
        adj_local(a, U, g, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) s_k[LBRS_IX((q * 4 + k) * kFWN + w, 16 * kFWN, 33)] = out[q][k];
    }
    __syncthreads();
    const int ti = threadIdx.x % kFTX, tj = threadIdx.x / kFTX;
    const int i = i0 + ti, j = j0 + tj;
    if (i >= a.nx || j >= a.ny) return;
    // sources y + c_q: slots (ti + 1 + sx_q, tj + 1 + sy_q)
    const int s0 = (tj + 1) * kFWX + ti + 1;
    const int sl[4] = {s0 - kFWX - 1, s0 - kFWX + 1, s0 + kFWX + 1, s0 + kFWX - 1};
    float g[4][4], U[4], out[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[q][k] = s_k[LBRS_IX((q * 4 + k) * kFWN + sl[q], 16 * kFWN, 33)];
    const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = U2[LBRS_IX(k * a.N + c, 4 * a.N, 33)];
    adj_local(a, U, g, out);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) a.gout[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 33)] = out[q][k];
}

// The two adjoint steps on 32 x 16 tiles, fed like the forward's tall kernel: the
// gather g(x)_q = k_q(x + c_q) pulls population q from the cell one step along
// +c_q, so its box starts at x = i0 - 4 (sx_q = -1) or i0, y = j0 - 2 (sy_q = -1)
// or j0 (the mirror of the forward's boxes), 36 x 18 per field.  Phase 1 forms
// k^{s-1} on the 34 x 18 window in place over the boxes (each position is gathered
// by one slot only); slots whose sources wrap around the periodic grid gather from
// global memory.  Phase 2 forms k^{s-2} for the tile, two cells per thread.  The
// same expressions in the same order as the push kernel: bit-identical.
__device__ __forceinline__ int adj_pos(int q, int k, int wi, int wj)
{
    return (q * 4 + k) * kTPN + wj * kPX + wi + ((q == 0 || q == 3) ? 2 : 0);
}

__device__ __forceinline__ void issue_adj_copy(const CUtensorMap* tmap, float* s_raw, uint32_t bar, int i0, int j0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(16u * kTPN * 4u) : "memory");
    const int x0[4] = {i0 - 4, i0, i0, i0 - 4};
    const int y0[4] = {j0 - 2, j0 - 2, j0, j0};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(s_raw + q * 4 * kTPN)),
            "l"((uint64_t)tmap), "r"(x0[q]), "r"(y0[q]), "r"(q * 4), "r"(bar)
            : "memory");
}

// Two steps: k^s (a.gin, through tmap) -> k^{s-2} (a.gout); a.U = U_{s-1}, U2 = U_{s-2}.
__global__ void __launch_bounds__(kFTX * kFTY, 5)
    adj_fused2_tall_kernel(const __grid_constant__ CUtensorMap tmap, const AdjArgs<float> a,
                           const float* __restrict__ U2, unsigned* wait_flag)
{
    extern __shared__ unsigned char smem_dyn[];
    float* s_raw = (float*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
    uint64_t* bar_p = (uint64_t*)(s_raw + 16 * kTPN);
    const uint32_t bar = smem_addr(bar_p);
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * kTY;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue_adj_copy(&tmap, s_raw, bar, i0, j0);
    }
    __syncthreads();
    const bool arrived = mbar_wait_bounded(bar, 0, kWaitPolls);
    if (!__syncthreads_and(arrived)) {
        give_up_tile(bar, wait_flag);
        return;
    }
    // phase 1: k^{s-1} on the window (periodic: every slot is a cell of the grid)
    for (int w = threadIdx.x; w < kTWN; w += kFTX * kFTY) {
        const int wi = w % kFWX, wj = w / kFWX;
        const int ui = i0 - 1 + wi, uj = j0 - 1 + wj;
        const int i = wrap_index(ui, a.nx), j = wrap_index(uj, a.ny);
        float g[4][4], U[4], out[4][4];
        if (ui > 0 && ui < a.nx - 1 && uj > 0 && uj < a.ny - 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) g[q][k] = s_raw[LBRS_IX(adj_pos(q, k, wi, wj), 16 * kTPN, 34)];
        } else {
            adj_gather(a, i, j, g);
        }
        const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 34)];
        adj_local(a, U, g, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) s_raw[LBRS_IX(adj_pos(q, k, wi, wj), 16 * kTPN, 34)] = out[q][k];
    }
    __syncthreads();
    // phase 2: k^{s-2} on the tile; the source of population q is slot (ti + 1 + sx_q, tj + 1 + sy_q)
    const int ti = threadIdx.x % kFTX;
    for (int tj = threadIdx.x / kFTX; tj < kTY; tj += kFTY) {
        const int i = i0 + ti, j = j0 + tj;
        if (i >= a.nx || j >= a.ny) continue;
        const int swi[4] = {ti, ti + 2, ti + 2, ti};
        const int swj[4] = {tj, tj, tj + 2, tj + 2};
        float g[4][4], U[4], out[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[q][k] = s_raw[LBRS_IX(adj_pos(q, k, swi[q], swj[q]), 16 * kTPN, 35)];
        const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = U2[LBRS_IX(k * a.N + c, 4 * a.N, 35)];
        adj_local(a, U, g, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) a.gout[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 35)] = out[q][k];
    }
}

// ---------------------------------------------------------------- adjoint at omega = 1, moments form
//
// At omega = 1 the local operator returns k_q = J_E(U)^T g for every q: the sweep's
// state is q-independent, so it is kept as its 4 fields kU (the adjoint's analogue of
// the forward's moments-only form; exact, the same values as the 16-value sweep).
// The gather becomes g_q(x) = kU(x + c_q): 4 fields of each of the 4 neighbours.

// g_q(x) = kU(x + c_q) for cell (i, j) of the periodic grid (kU: 4 planes).
__device__ __forceinline__ void adj_gather_u(const float* __restrict__ kU, int64_t N, int nx, int ny, int i, int j,
                                             float g[4][4])
{
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t s = (int64_t)wrap_index(j + SY[q], ny) * nx + wrap_index(i + SX[q], nx);
#pragma unroll
        for (int k = 0; k < 4; ++k) g[q][k] = kU[LBRS_IX(k * N + s, 4 * N, 36)];
    }
}

// kU = J_E(U)^T g from the full g (a.gin, 16 planes): the start of a sweep.
__global__ void __launch_bounds__(256) adj_local_u_kernel(const AdjArgs<float> a)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += (int64_t)gridDim.x * blockDim.x) {
        float g[4][4], U[4], ubar[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 36)];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 36)];
        equilibrium_vjp2d<float>(U, g, a.gamma, a.gm1, a.c, ubar);
#pragma unroll
        for (int k = 0; k < 4; ++k) a.gout[LBRS_IX(k * a.N + c, 4 * a.N, 36)] = ubar[k];
    }
}

// One step from kU (a.gin, 4 planes): with a.U, kU' = J_E(U)^T g; without, the full
// g (16 planes) for the earlier segment.
__global__ void __launch_bounds__(256) adj_pull_u_kernel(const AdjArgs<float> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    float g[4][4];
    adj_gather_u(a.gin, a.N, a.nx, a.ny, i, j, g);
    if (a.U) {
        float U[4], ubar[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 36)];
        equilibrium_vjp2d<float>(U, g, a.gamma, a.gm1, a.c, ubar);
#pragma unroll
        for (int k = 0; k < 4; ++k) a.gout[LBRS_IX(k * a.N + c, 4 * a.N, 36)] = ubar[k];
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) a.gout[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 36)] = g[q][k];
    }
}

// Two steps kU^s -> kU^{s-2} on a 32 x TY tile (TY = 16, 24 or 32 rows): phase 1 forms kU^{s-1} on
// the 34 x (TY + 2) window (4 fields per slot in shared memory), phase 2 kU^{s-2} for the tile.  A tile whose
// window and the window's neighbours lie inside the grid gathers without wrapping (the same
// cells, so the same values).  Six blocks per SM (40 registers, no spills): the sweep waits on its
// gathers, and a sixth block hides more of that latency than the registers of a fifth buy.
template <int TY>
__global__ void __launch_bounds__(kFTX * kFTY, 6) adj_fused2_u_kernel(const AdjArgs<float> a, const float* __restrict__ U2)
{
    constexpr int kTWN = kFWX * (TY + 2);   // window slots: the tile and one cell of halo
    __shared__ float s_w[4 * kTWN];
    const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * TY;
    const bool inside = i0 >= 2 && j0 >= 2 && i0 + kFTX + 2 <= a.nx && j0 + TY + 2 <= a.ny;
    for (int w = threadIdx.x; w < kTWN; w += kFTX * kFTY) {
        float g[4][4], U[4], ubar[4];
        int64_t c;
        if (inside) {
            c = (int64_t)(j0 - 1 + w / kFWX) * a.nx + (i0 - 1 + w % kFWX);
            // x + c_q: q0 (i-1, j-1), q1 (i+1, j-1), q2 (i+1, j+1), q3 (i-1, j+1)
            const int64_t s[4] = {c - a.nx - 1, c - a.nx + 1, c + a.nx + 1, c + a.nx - 1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX(k * a.N + s[q], 4 * a.N, 37)];
        } else {
            const int i = wrap_index(i0 - 1 + w % kFWX, a.nx), j = wrap_index(j0 - 1 + w / kFWX, a.ny);
            adj_gather_u(a.gin, a.N, a.nx, a.ny, i, j, g);
            c = (int64_t)j * a.nx + i;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 37)];
        equilibrium_vjp2d<float>(U, g, a.gamma, a.gm1, a.c, ubar);
#pragma unroll
        for (int k = 0; k < 4; ++k) s_w[LBRS_IX(k * kTWN + w, 4 * kTWN, 37)] = ubar[k];
    }
    __syncthreads();
    const int ti = threadIdx.x % kFTX;
    for (int tj = threadIdx.x / kFTX; tj < TY; tj += kFTY) {
        const int i = i0 + ti, j = j0 + tj;
        if (i >= a.nx || j >= a.ny) continue;
        // the source of population q, x + c_q, is window slot (ti + 1 + sx_q, tj + 1 + sy_q)
        const int s0 = (tj + 1) * kFWX + ti + 1;
        const int sl[4] = {s0 - kFWX - 1, s0 - kFWX + 1, s0 + kFWX + 1, s0 + kFWX - 1};
        float g[4][4], U[4], ubar[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[q][k] = s_w[LBRS_IX(k * kTWN + sl[q], 4 * kTWN, 37)];
        const int64_t c = (int64_t)j * a.nx + i;
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = U2[LBRS_IX(k * a.N + c, 4 * a.N, 37)];
        equilibrium_vjp2d<float>(U, g, a.gamma, a.gm1, a.c, ubar);
#pragma unroll
        for (int k = 0; k < 4; ++k) a.gout[LBRS_IX(k * a.N + c, 4 * a.N, 37)] = ubar[k];
    }
}

// Kernel variant for D2Q4 FP32: 0 = scalar one cell per thread, 2 or 4 =
// vector width, 12 / 14 = 2 / 4 strided cells per thread.  The default can be
// overridden for tuning sweeps with the environment variable LBRS_F32_STEP_VARIANT.
int step2d_f32_variant()
{
    static int v = [] {
        const char* s = getenv("LBRS_F32_STEP_VARIANT");
        if (s) {
            const int x = atoi(s);
            if (x == 0 || x == 2 || x == 4 || x == 12 || x == 14) return x;
        }
        return 0;
    }();
    return v;
}

}  // namespace

cudaError_t launch_step_f32(int lattice, const StepArgs<float>& a, cudaStream_t s)
{
    if (lattice == LAT_D2Q4 && a.solid) {
        const dim3 block(128, 2);
        const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
        step2d_obstacle_kernel<float><<<grid, block, 0, s>>>(a);
    } else if (lattice == LAT_D2Q4) {
        const int var = step2d_f32_variant();
        if ((var == 2 || var == 4) && a.nx % var == 0 && a.ny <= 65535) {
            const unsigned per_block = 128u * var;
            const dim3 grid((unsigned)((a.nx + per_block - 1) / per_block), (unsigned)a.ny);
            if (var == 4) step2d_f32_vec_kernel<4><<<grid, 128, 0, s>>>(a);
            else step2d_f32_vec_kernel<2><<<grid, 128, 0, s>>>(a);
        } else if ((var == 12 || var == 14) && a.ny <= 65535) {
            const unsigned per_block = 128u * (var - 10);
            const dim3 grid((unsigned)((a.nx + per_block - 1) / per_block), (unsigned)a.ny);
            if (var == 14) step2d_f32_ilp_kernel<4><<<grid, 128, 0, s>>>(a);
            else step2d_f32_ilp_kernel<2><<<grid, 128, 0, s>>>(a);
        } else {
            const dim3 block(128, 2);
            const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
            step2d_kernel<float><<<grid, block, 0, s>>>(a);
        }
    } else if (lattice == LAT_D2Q4S) {
        const dim3 block(128, 2);
        const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
        step2ds_kernel<float><<<grid, block, 0, s>>>(a);
    } else if (lattice == LAT_D1Q3) {
        step1d_q3_kernel<float><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    } else {
        step1d_kernel<float><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// Two steps per launch (temporal blocking by two); on by default, LBRS_F32_FUSE=0 turns it off.
bool step2_f32_enabled()
{
    static int v = [] {
        const char* s = getenv("LBRS_F32_FUSE");
        return (s && !strcmp(s, "0")) ? 0 : 1;
    }();
    return v != 0;
}

// Tensor copies for the two-step kernel; on by default, LBRS_F32_TMA=0 turns them off.
static bool tma_enabled()
{
    static int v = [] {
        const char* s = getenv("LBRS_F32_TMA");
        return (s && !strcmp(s, "0")) ? 0 : 1;
    }();
    return v != 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// The distance of the two-step kernel's L2 prefetch (the boxes of the block that many places later
// in launch order, after a block's own boxes have landed): half its resident blocks on the current
// device, as for the three-step kernel (measured +1.5 % on the flushed 1024^2 grid, +3.9 % with
// internal walls on 6144 x 2048); LBRS_F32_PREFETCH2=n > 1 sets it, =0 turns it off; 0 if the
// query fails.
static int step2_prefetch_ahead()
{
    static int v = [] {
        const char* e = getenv("LBRS_F32_PREFETCH2");
        if (e && !strcmp(e, "0")) return 0;
        if (e && atoi(e) > 1) return atoi(e);
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step2d_f32_fused2_tall_kernel<false>, kFTX * kFTY,
                                                          kTallSmemBytes) != cudaSuccess)
            return 0;
        return sms * per / 2;
    }();
    return v;
}

bool encode_f32_tile_map(TileMap* map, const float* f, int64_t nx, int64_t ny)
{
    static_assert(sizeof(map->bytes) == sizeof(CUtensorMap), "TileMap holds one CUtensorMap");
    map->valid = 0;
    if (!tma_enabled() || nx % 4 != 0 || ((uintptr_t)f & 15)) return false;   // row and field strides: 16-byte multiples
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(step2d_f32_fused2_tall_kernel<false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(step2d_f32_fused2_tall_kernel<true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(step2d_f32_fused2_tall_kernel<false, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallObstSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(step2d_f32_fused2_tall_kernel<false, false, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallSmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(step2d_f32_fused2_tall_kernel<true, false, true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallSmemBytes);
    });
    if (attr_err != cudaSuccess) return false;
    step2_prefetch_ahead();   // its device queries now, not first inside a graph capture
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 16};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)(nx * ny) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kPX, (cuuint32_t)kTPY, 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    memcpy(map->bytes, &m, sizeof m);
    map->valid = 1;
    return true;
}

// The distance of the three-step kernel's L2 prefetch: half its resident blocks on the current
// device (SMs x blocks per SM / 2; measured on 1024^2 and 4096 x 1024 grids: a plateau from 0.5 to
// 0.8 of a wave, below it at one wave or more); LBRS_F32_PREFETCH=n > 1 sets it, =0 turns the
// prefetch off; 0 if the query fails.
static int step3_prefetch_ahead()
{
    static int v = [] {
        const char* e = getenv("LBRS_F32_PREFETCH");
        if (e && !strcmp(e, "0")) return 0;
        if (e && atoi(e) > 1) return atoi(e);
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step2d_f32_fused3_kernel<false>, kT3T,
                                                          kF3SmemBytes) != cudaSuccess)
            return 0;
        return sms * per / 2;
    }();
    return v;
}

// The tensor map of the three-step kernel: 40 x 16 x 4-field boxes of the state.
bool encode_f32_tile_map3(TileMap* map, const float* f, int64_t nx, int64_t ny)
{
    map->valid = 0;
    if (!tma_enabled() || nx % 4 != 0 || ((uintptr_t)f & 15)) return false;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(step2d_f32_fused3_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kF3SmemBytes);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(step2d_f32_fused3_kernel<true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kF3SmemBytes);
    });
    if (attr_err != cudaSuccess) return false;
    step3_prefetch_ahead();   // its device queries now, not first inside a graph capture
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 16};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)(nx * ny) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kP3X, (cuuint32_t)kW3Y, 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    memcpy(map->bytes, &m, sizeof m);
    map->valid = 1;
    return true;
}

bool step3_f32_enabled()
{
    static int v = [] {
        const char* e = getenv("LBRS_F32_FUSE3");
        return (e && !strcmp(e, "0")) ? 0 : 1;
    }();
    return v != 0;
}

// Three steps; with a.Uout set, three recording steps (the moments of each step to a.Uout, one
// step's 4 N values after another).
cudaError_t launch_step3_f32(const StepArgs<float>& a, const TileMap* map3, unsigned* wait_flag, cudaStream_t s)
{
    if (!map3 || !map3->valid || !wait_flag || a.solid) return cudaErrorInvalidValue;
    CUtensorMap m;
    memcpy(&m, map3->bytes, sizeof m);
    const dim3 grid((unsigned)((a.nx + kFTX - 1) / kFTX), (unsigned)((a.ny + kT3Y - 1) / kT3Y));
    const int ahead = step3_prefetch_ahead();
    if (a.Uout)
        step2d_f32_fused3_kernel<true><<<grid, kT3T, kF3SmemBytes, s>>>(m, a, wait_flag, ahead);
    else
        step2d_f32_fused3_kernel<false><<<grid, kT3T, kF3SmemBytes, s>>>(m, a, wait_flag, ahead);
    return cudaGetLastError();
}

cudaError_t launch_step2_f32(const StepArgs<float>& a, const TileMap* map, unsigned* wait_flag, cudaStream_t s)
{
    const int ahead = step2_prefetch_ahead();
    const bool rec = a.Uout != nullptr;
    const bool half = a.bc[2] == BC_WALL_HALFWAY || a.bc[3] == BC_WALL_HALFWAY;   // the variants that resolve it
    if (map && map->valid && wait_flag) {
        CUtensorMap m;
        memcpy(&m, map->bytes, sizeof m);
        const dim3 grid((unsigned)((a.nx + kFTX - 1) / kFTX), (unsigned)((a.ny + kTY - 1) / kTY));
        if (a.solid) {
            if (rec || half) return cudaErrorInvalidValue;   // no recording form or halfway walls with obstacles
            step2d_f32_fused2_tall_kernel<false, true><<<grid, kFTX * kFTY, kTallObstSmemBytes, s>>>(m, a, wait_flag, ahead);
        } else if (rec) {
            if (half) step2d_f32_fused2_tall_kernel<true, false, true><<<grid, kFTX * kFTY, kTallSmemBytes, s>>>(m, a, wait_flag, ahead);
            else step2d_f32_fused2_tall_kernel<true><<<grid, kFTX * kFTY, kTallSmemBytes, s>>>(m, a, wait_flag, ahead);
        } else {
            if (half) step2d_f32_fused2_tall_kernel<false, false, true><<<grid, kFTX * kFTY, kTallSmemBytes, s>>>(m, a, wait_flag, ahead);
            else step2d_f32_fused2_tall_kernel<false><<<grid, kFTX * kFTY, kTallSmemBytes, s>>>(m, a, wait_flag, ahead);
        }
    } else if (a.solid) {
        return cudaErrorInvalidValue;                // internal walls need the tensor-copy form
    } else {
        const dim3 grid((unsigned)((a.nx + kFTX - 1) / kFTX), (unsigned)((a.ny + kFTY - 1) / kFTY));
        if (rec) {
            if (half) step2d_f32_fused2_kernel<true, true><<<grid, kFTX * kFTY, 0, s>>>(a);
            else step2d_f32_fused2_kernel<true, false><<<grid, kFTX * kFTY, 0, s>>>(a);
        } else {
            if (half) step2d_f32_fused2_kernel<false, true><<<grid, kFTX * kFTY, 0, s>>>(a);
            else step2d_f32_fused2_kernel<false, false><<<grid, kFTX * kFTY, 0, s>>>(a);
        }
    }
    return cudaGetLastError();
}

// Two scalar D2Q4 steps from a.src into a.dst (step2ds_fused2_kernel).
// Rows of a tile for the kernels with a tile-height parameter: a value of `allowed` (zero-terminated)
// from the environment variable `name` (a tuning override), else `dflt`.
static int tile_rows(const char* name, int dflt, const int* allowed)
{
    const char* e = getenv(name);
    const int v = e ? atoi(e) : 0;
    for (; *allowed; ++allowed)
        if (v == *allowed) return v;
    return dflt;
}

template <int TY, typename Kernel, typename... Args>
static cudaError_t launch_tiled(Kernel k, int nx, int ny, cudaStream_t s, Args... args)
{
    const dim3 grid((unsigned)((nx + kFTX - 1) / kFTX), (unsigned)((ny + TY - 1) / TY));
    k<<<grid, kFTX * kFTY, 0, s>>>(args...);
    return cudaGetLastError();
}

cudaError_t launch_step2s_f32(const StepArgs<float>& a, cudaStream_t s)
{
    // 32 rows measured fastest (8192^2 steady: 16 rows 339 k, 24 rows 399 k, 32 rows 406-408 k, 48 rows
    // 361 k, 64 rows 351 k MLUPS)
    static const int allowed[] = {16, 24, 32, 0};
    static const int ty = tile_rows("LBRS_F32S_TILE_Y", 32, allowed);
    if (ty == 24) return launch_tiled<24>(step2ds_fused2_kernel<24>, a.nx, a.ny, s, a);
    if (ty == 16) return launch_tiled<16>(step2ds_fused2_kernel<16>, a.nx, a.ny, s, a);
    return launch_tiled<32>(step2ds_fused2_kernel<32>, a.nx, a.ny, s, a);
}

// rcp_f32 over n inputs, for its error-bound test.
__global__ void rcp_selftest_kernel(const float* __restrict__ x, float* __restrict__ r, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = rcp_f32(x[i]);
}

cudaError_t launch_rcp_selftest(const float* x, float* r, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    rcp_selftest_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(x, r, n);
    return cudaGetLastError();
}

cudaError_t launch_wait_timeout_selftest(unsigned* wait_flag, cudaStream_t s)
{
    wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(wait_flag, 1 << 12);
    return cudaGetLastError();
}

cudaError_t launch_adapt_step_f32(const StepArgs<float>& a, void* st, double gamma, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    step2d_adapt_kernel<float><<<grid, block, 0, s>>>(a, (AdaptState*)st, gamma);
    return cudaGetLastError();
}

cudaError_t launch_adapt_init_bound_f32(const void* fs, int64_t N, double gamma, void* st, cudaStream_t s)
{
    int64_t b = (N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    adapt_init_bound_kernel<float><<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>((const float*)fs, N, gamma, (AdaptState*)st);
    return cudaGetLastError();
}

cudaError_t launch_step_record_f32(const StepArgs<float>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    if (a.solid) step2d_obstacle_kernel<float, true><<<grid, block, 0, s>>>(a);
    else step2d_kernel<float, true><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    adjoint2d_kernel<float><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_local_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    int64_t b = (a.N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    adj_local_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_pull_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    adj_pull_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_fused2_f32(const AdjArgs<float>& a, const float* U2, const TileMap* map, unsigned* wait_flag,
                                  cudaStream_t s)
{
    if (map && map->valid && wait_flag) {
        static const cudaError_t attr = cudaFuncSetAttribute(
            adj_fused2_tall_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallSmemBytes);
        if (attr != cudaSuccess) return attr;
        CUtensorMap m;
        memcpy(&m, map->bytes, sizeof m);
        const dim3 grid((unsigned)((a.nx + kFTX - 1) / kFTX), (unsigned)((a.ny + kTY - 1) / kTY));
        adj_fused2_tall_kernel<<<grid, kFTX * kFTY, kTallSmemBytes, s>>>(m, a, U2, wait_flag);
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)((a.nx + kFTX - 1) / kFTX), (unsigned)((a.ny + kFTY - 1) / kFTY));
    adj_fused2_kernel<<<grid, kFTX * kFTY, 0, s>>>(a, U2);
    return cudaGetLastError();
}

// The omega = 1 sweep in its moments form; on by default, LBRS_ADJ_UFORM=0 turns it off.
bool adj_uform_enabled()
{
    static int v = [] {
        const char* e = getenv("LBRS_ADJ_UFORM");
        return (e && !strcmp(e, "0")) ? 0 : 1;
    }();
    return v != 0;
}

cudaError_t launch_adj_local_u_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    int64_t b = (a.N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    adj_local_u_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_pull_u_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    adj_pull_u_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_fused2_u_f32(const AdjArgs<float>& a, const float* U2, cudaStream_t s)
{
    // 24 rows measured fastest (2048^2 x 2000 steps: sweep 77.5 ms at 16 rows, 74.6 ms at 24, 76.0 ms at 32)
    static const int allowed[] = {16, 24, 32, 0};
    static const int ty = tile_rows("LBRS_ADJU_TILE_Y", 24, allowed);
    if (ty == 32) return launch_tiled<32>(adj_fused2_u_kernel<32>, a.nx, a.ny, s, a, U2);
    if (ty == 16) return launch_tiled<16>(adj_fused2_u_kernel<16>, a.nx, a.ny, s, a, U2);
    return launch_tiled<24>(adj_fused2_u_kernel<24>, a.nx, a.ny, s, a, U2);
}

cudaError_t launch_vjp_equilibrium_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    int64_t b = (a.N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    vjp_equilibrium2d_kernel<float><<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched tubes

template <int Q>
static cudaError_t launch_batch_q_f32(const BatchArgs<float>& a, int ntiles, int block, cudaStream_t s)
{
    const size_t smem = 2 * 3 * Q * (size_t)(a.tile_cells + 2 * a.halo) * sizeof(float);
    switch (block) {
        case 128:
            batch1d_kernel<float, 128, Q><<<ntiles, 128, smem, s>>>(a);
            break;
        case 256:
            batch1d_kernel<float, 256, Q><<<ntiles, 256, smem, s>>>(a);
            break;
        case 512:
            batch1d_kernel<float, 512, Q><<<ntiles, 512, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_f32(const BatchArgs<float>& a, int ntiles, int block, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    return a.q == 3 ? launch_batch_q_f32<3>(a, ntiles, block, s) : launch_batch_q_f32<2>(a, ntiles, block, s);
}

template <int Q>
static cudaError_t prepare_batch_q_f32(int block, size_t smem)
{
    // opt in to more than the default 48 KiB of dynamic shared memory
    switch (block) {
        case 128:
            return cudaFuncSetAttribute(batch1d_kernel<float, 128, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 256:
            return cudaFuncSetAttribute(batch1d_kernel<float, 256, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 512:
            return cudaFuncSetAttribute(batch1d_kernel<float, 512, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_batch_f32(int block, size_t smem, int q)
{
    return q == 3 ? prepare_batch_q_f32<3>(block, smem) : prepare_batch_q_f32<2>(block, smem);
}

cudaError_t launch_batch_copy_f32(const float* src, float* dst, int64_t N, const BatchTile* tiles, int ntiles,
                                     const int64_t* tube_off, int planes, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    batch_copy_kernel<float><<<ntiles, 256, 0, s>>>(src, dst, N, tiles, tube_off, planes);
    return cudaGetLastError();
}

// First out-of-bounds index recorded by this unit's kernels (LBRS_DEBUG builds; 0 otherwise).
LBRS_DEBUG_WORD(debug_word_f32)

}  // namespace lbrs
