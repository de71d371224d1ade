// FP32 time step of the LBRS solver (distributions stored and updated in FP32).
//
// Compiled with FMA contraction allowed; velocities use one correctly rounded
// reciprocal per cell.  The numerics differ from the FP64 path by rounding
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
    if (lattice == LAT_D2Q4) {
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
    } else if (lattice == LAT_D1Q3) {
        step1d_q3_kernel<float><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    } else {
        step1d_kernel<float><<<(unsigned)((a.nx + 255) / 256), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_record_f32(const StepArgs<float>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    step2d_kernel<float, true><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((a.nx + block.x - 1) / block.x), (unsigned)((a.ny + block.y - 1) / block.y));
    adjoint2d_kernel<float><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_vjp_equilibrium_f32(const AdjArgs<float>& a, cudaStream_t s)
{
    int64_t b = (a.N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    vjp_equilibrium2d_kernel<float><<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batched tubes

cudaError_t launch_batch_f32(const BatchArgs<float>& a, int ntiles, int block, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    const size_t smem = 2 * 6 * (size_t)(a.tile_cells + 2 * a.halo) * sizeof(float);
    switch (block) {
        case 128:
            batch1d_kernel<float, 128><<<ntiles, 128, smem, s>>>(a);
            break;
        case 256:
            batch1d_kernel<float, 256><<<ntiles, 256, smem, s>>>(a);
            break;
        case 512:
            batch1d_kernel<float, 512><<<ntiles, 512, smem, s>>>(a);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t prepare_batch_f32(int block, size_t smem)
{
    // opt in to more than the default 48 KiB of dynamic shared memory
    switch (block) {
        case 128:
            return cudaFuncSetAttribute(batch1d_kernel<float, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 256:
            return cudaFuncSetAttribute(batch1d_kernel<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 512:
            return cudaFuncSetAttribute(batch1d_kernel<float, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_copy_f32(const float* src, float* dst, int64_t N, const BatchTile* tiles, int ntiles,
                                     const int64_t* tube_off, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    batch_copy_kernel<float><<<ntiles, 256, 0, s>>>(src, dst, N, tiles, tube_off);
    return cudaGetLastError();
}

}  // namespace lbrs
