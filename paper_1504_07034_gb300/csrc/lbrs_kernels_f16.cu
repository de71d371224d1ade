// D2Q4 step with FP16 storage of the non-equilibrium part (precision LBRS_F16NEQ).
//
// State per cell: the moments U (4 x FP32) and, per field k, the post-collision
// non-equilibrium parts g_q = f*_q - f^eq_q(U) of populations q = 0, 1, 2 in
// FP16, scaled by a per-field power of two s_k (stored value g / s_k).  A state
// buffer is U [4][N] FP32, g [3][4][N] FP16, then the four scales (FP32), so a
// copy of the buffer is a complete checkpoint; every step carries the scales
// over to its output buffer.  The
// fourth follows from sum_q g_q = 0: the collision leaves the moments
// unchanged, sum_q f*_q = U = sum_q f^eq_q(U).  40 bytes per cell instead of
// 64, so a step moves 80 B instead of 128 B per lattice update.
//
// Streaming pulls f*_q(x - c_q) = f^eq_q(U(x - c_q)) + s_k g_q(x - c_q): the
// equilibrium of the source cell is re-evaluated from its stored moments
// (Sections II.C/II.D), then the step is the FP32 step: moments, fluxes,
// equilibria, relaxation; the new g = (1 - omega)(f - f^eq(U)) (the
// relaxation written on the non-equilibrium part) is rounded to FP16.
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

// f*_q of one source cell, all four fields.
__device__ __forceinline__ void load_pop(const F16Args& a, int q, int64_t s, const float sc[4], float f[4])
{
    float U[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = a.Uin[k * a.N + s];
    float g[4];
    if (q < 3) {
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] = __half2float(a.gin[(q * 4 + k) * a.N + s]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            g[k] = -((__half2float(a.gin[k * a.N + s]) + __half2float(a.gin[(4 + k) * a.N + s])) +
                     __half2float(a.gin[(8 + k) * a.N + s]));
    }
    float e[4][4];
    equilibria2d<float>(U, a.gm1, a.c, e);
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = e[q][k] + sc[k] * g[k];
}

__device__ __forceinline__ void pull_edge_f16(const F16Args& a, int i, int j, const float sc[4], float f[4][4])
{
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
        const float* g = nullptr;
        if (side_x >= 0) {
            if (kind_x == BC_DIRICHLET) g = a.ghost + side_x * GHOST_STRIDE + q * 4;
            else if (kind_x == BC_PERIODIC) si = si < 0 ? si + a.nx : si - a.nx;
            else si = si < 0 ? 0 : a.nx - 1;
        }
        if (!g && side_y >= 0) {
            if (kind_y == BC_DIRICHLET) g = a.ghost + side_y * GHOST_STRIDE + q * 4;
            else if (kind_y == BC_PERIODIC) sj = sj < 0 ? sj + a.ny : sj - a.ny;
            else sj = sj < 0 ? 0 : a.ny - 1;
        }
        if (g) {
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = g[k];
        } else {
            load_pop(a, q, (int64_t)sj * a.nx + si, sc, f[q]);
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
}

__global__ void __launch_bounds__(256) step2d_f16neq_kernel(const F16Args a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    if (c < 4) a.scale_out[c] = a.scale[c];
    float sc[4], inv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sc[k] = a.scale[k];
        inv[k] = 1.f / sc[k];          // exact: the scales are powers of two
    }
    float f[4][4];
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        const int64_t s[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) load_pop(a, q, s[q], sc, f[q]);
    } else {
        pull_edge_f16(a, i, j, sc, f);
    }
    float U[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = ((f[0][k] + f[1][k]) + f[2][k]) + f[3][k];
    float e[4][4];
    equilibria2d<float>(U, a.gm1, a.c, e);
#pragma unroll
    for (int k = 0; k < 4; ++k) a.Uout[k * a.N + c] = U[k];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            a.gout[(q * 4 + k) * a.N + c] = __float2half_rn(a.om1 * (f[q][k] - e[q][k]) * inv[k]);
}

// Initial state: U from W (conserved or primitive, FP64 arithmetic), g = 0.
template <typename Tin>
__global__ void __launch_bounds__(256) set_state_f16neq_kernel(const Tin* __restrict__ W, float* __restrict__ U,
                                                               __half* __restrict__ g, int64_t N, int kind,
                                                               double gamma)
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
        for (int k = 0; k < 4; ++k) U[k * N + i] = (float)u[k];
#pragma unroll
        for (int n = 0; n < 12; ++n) g[n * N + i] = __float2half_rn(0.f);
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

cudaError_t launch_step_f16neq(const F16StepArgs& s, cudaStream_t st)
{
    F16Args a;
    a.Uin = (const float*)s.src;
    a.gin = (const __half*)((const char*)s.src + 16 * s.N);
    a.Uout = (float*)s.dst;
    a.gout = (__half*)((char*)s.dst + 16 * s.N);
    a.ghost = s.ghost;
    a.scale = (const float*)((const char*)s.src + 40 * s.N);
    a.scale_out = (float*)((char*)s.dst + 40 * s.N);
    a.N = s.N;
    a.nx = s.nx;
    a.ny = s.ny;
    for (int k = 0; k < 4; ++k) a.bc[k] = s.bc[k];
    a.om = s.om;
    a.om1 = s.om1;
    a.c = s.c;
    a.gm1 = s.gm1;
    const dim3 block(128, 2);
    const dim3 grid((unsigned)((s.nx + block.x - 1) / block.x), (unsigned)((s.ny + block.y - 1) / block.y));
    step2d_f16neq_kernel<<<grid, block, 0, st>>>(a);
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
    if (w_dtype == 0) set_state_f16neq_kernel<double><<<g, 256, 0, st>>>((const double*)W, U, gq, N, kind, gamma);
    else set_state_f16neq_kernel<float><<<g, 256, 0, st>>>((const float*)W, U, gq, N, kind, gamma);
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

}  // namespace lbrs
