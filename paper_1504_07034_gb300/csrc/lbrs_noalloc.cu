// lbrs_diagnostics_noalloc: the FP64 diagnostics reduction without a
// workspace and without any device allocation.
//
// Some callers cannot hand this library a workspace for the reduction's
// per-block partial sums: loops that must not stall on the implicit device
// synchronisation of cudaMalloc/cudaFree, and processes whose device memory is
// fully held by another allocator (for instance a framework's caching pool).  For them this variant keeps its scratch in a
// file-scope static __device__ array of fixed size, which the CUDA runtime
// places in device memory when the library's module is loaded and which stays
// there, on every GPU that loads the library, until the process exits.
//
// The scratch holds kMaxBlocks partial records of DIAG_W doubles plus the
// DIAG_W-double result (kMaxBlocks * 80 + 80 bytes = 320.1 KiB).  One record
// covers kCellsPerBlock cells, so grids of up to kMaxBlocks * kCellsPerBlock
// = 33,554,432 cells are accepted; larger grids are rejected with
// LBRS_EINVAL.  Every record the final pass reads is written earlier in the
// same call, so nothing in the scratch has to start at zero.  All calls share
// the one array: calls that overlap on the GPU (on different streams without
// ordering between them) race on it.
//
// Host code must not pass the array's name to a kernel: on the host it is a
// stand-in symbol, not a device address.  The device address is looked up
// with cudaGetSymbolAddress once per device, with that device current, on the
// first call made while it is current (that first call should therefore come
// before any stream capture), and kept for the life of the process's context
// on that device: after a cudaDeviceReset the kept address is stale.  Device
// code here names the array directly.  Each call ends by copying the result
// to the caller's host struct and synchronising its stream.
//
// Compiled with -fmad=false, like the other FP64 kernels.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include <cuda_runtime.h>

#include "lbrs.h"
#include "lbrs_kernels.cuh"

namespace lbrs {
lbrs_status validate_config(const lbrs_config* c);
lbrs_status set_error(lbrs_status s, const char* msg);
}  // namespace lbrs

namespace {

using namespace lbrs;

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 32;
constexpr int64_t kCellsPerBlock = (int64_t)kThreads * kCellsPerThread;   // 8192
constexpr int kMaxBlocks = 4096;
constexpr int64_t kMaxCells = kMaxBlocks * kCellsPerBlock;                 // 33,554,432
constexpr int kMaxDevices = 64;

// partial records [kMaxBlocks][DIAG_W], then the result [DIAG_W]
static __device__ __align__(256) double g_diag_scratch[(kMaxBlocks + 1) * DIAG_W];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

struct Acc {
    double tot[4];
    double min_rho, min_p, max_lam, nbad, nsub;
};

__device__ __forceinline__ void combine(Acc& a, const Acc& b)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) a.tot[k] += b.tot[k];
    a.min_rho = fmin(a.min_rho, b.min_rho);
    a.min_p = fmin(a.min_p, b.min_p);
    a.max_lam = fmax(a.max_lam, b.max_lam);
    a.nbad += b.nbad;
    a.nsub += b.nsub;
}

__device__ __forceinline__ Acc shfl_down(const Acc& a, int off)
{
    Acc b;
#pragma unroll
    for (int k = 0; k < 4; ++k) b.tot[k] = __shfl_down_sync(0xffffffffu, a.tot[k], off);
    b.min_rho = __shfl_down_sync(0xffffffffu, a.min_rho, off);
    b.min_p = __shfl_down_sync(0xffffffffu, a.min_p, off);
    b.max_lam = __shfl_down_sync(0xffffffffu, a.max_lam, off);
    b.nbad = __shfl_down_sync(0xffffffffu, a.nbad, off);
    b.nsub = __shfl_down_sync(0xffffffffu, a.nsub, off);
    return b;
}

// Same per-cell checks (in the storage precision, totals in FP64) and fixed-order
// reduction as lbrs_diagnostics; the partial records go to the static scratch
// (its device address is `scratch`).
template <typename Ts, int Q, int K>
__global__ void __launch_bounds__(kThreads) noalloc_partial_kernel(const Ts* __restrict__ fs, int64_t N, double gamma,
                                                                   double lambda, double* __restrict__ scratch)
{
    using R = Ts;
    const R g = (R)gamma, gm1 = (R)(gamma - 1.0), lam_max = (R)lambda;
    Acc acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc.tot[k] = 0.0;
    acc.nbad = acc.nsub = 0.0;
    R mn_rho = (R)INFINITY, mn_p = (R)INFINITY, mx_lam = (R)0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        R U[4] = {0, 0, 0, 0};
        bool finite = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            R s = fs[(0 * K + k) * N + i];
#pragma unroll
            for (int q = 1; q < Q; ++q) s += fs[(q * K + k) * N + i];
            U[k] = s;
            acc.tot[k] += (double)s;
            finite = finite && isfinite(s);
        }
        const R inv = (R)1 / U[0];
        R p, lam;
        if (K == 4) {
            const R u = U[1] * inv, v = U[2] * inv;
            p = gm1 * (U[3] - (R)0.5 * (U[1] * u + U[2] * v));
            const R s1 = fabs(u + v), s2 = fabs(u - v);
            lam = (s1 > s2 ? s1 : s2) + sqrt((R)2 * g * p * inv);
        } else {
            const R u = U[1] * inv;
            p = gm1 * (U[2] - (R)0.5 * (U[1] * u));
            lam = fabs(u) + sqrt(g * p * inv);
            if (Q == 3) lam *= (R)1.224744871391589;   // D1Q3 bound: sqrt(3/2)(|u| + a)
        }
        if (finite) {
            mn_rho = fmin(mn_rho, U[0]);
            mn_p = fmin(mn_p, p);
        }
        if (!finite || !(U[0] > (R)0) || !(p > (R)0)) {
            acc.nbad += 1.0;
        } else {
            mx_lam = fmax(mx_lam, lam);
            if (lam > lam_max) acc.nsub += 1.0;
        }
    }
    acc.min_rho = (double)mn_rho;
    acc.min_p = (double)mn_p;
    acc.max_lam = (double)mx_lam;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) combine(acc, shfl_down(acc, off));
    __shared__ Acc warp_acc[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_acc[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc b = warp_acc[0];
        for (int w = 1; w < kThreads / 32; ++w) combine(b, warp_acc[w]);
        double* out = scratch + (int64_t)blockIdx.x * DIAG_W;
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

// Folds the nblocks records in block order into the result slot after the
// last possible record.
__global__ void noalloc_final_kernel(int nblocks, double cell_volume)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    double mn_r = INFINITY, mn_p = INFINITY, mx_l = 0.0, nb = 0.0, ns = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double* p = g_diag_scratch + (int64_t)b * DIAG_W;
        for (int k = 0; k < 4; ++k) tot[k] += p[k];
        mn_r = fmin(mn_r, p[4]);
        mn_p = fmin(mn_p, p[5]);
        mx_l = fmax(mx_l, p[6]);
        nb += p[7];
        ns += p[8];
    }
    double* out = g_diag_scratch + (int64_t)kMaxBlocks * DIAG_W;
    for (int k = 0; k < 4; ++k) out[k] = tot[k] * cell_volume;
    out[4] = mn_r;
    out[5] = mn_p;
    out[6] = mx_l;
    out[7] = nb;
    out[8] = ns;
    out[9] = 0.0;
}

// Device address of the scratch on the current device, looked up once per device.
lbrs_status scratch_address(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(LBRS_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(LBRS_EINVAL, "device ordinal out of range for the scratch table");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the diagnostics scratch failed: %s",
                     cudaGetErrorString(e));
            return set_error(LBRS_ECUDA, msg);
        }
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return LBRS_OK;
}

}  // namespace

extern "C" lbrs_status lbrs_diagnostics_noalloc(const lbrs_config* cfg, const void* d_fs, lbrs_diag* out)
{
    lbrs_status st = validate_config(cfg);
    if (st != LBRS_OK) return st;
    if (cfg->precision == LBRS_F16NEQ || cfg->precision == LBRS_F32U)
        return set_error(LBRS_EINVAL, "the no-allocation diagnostics read the F64 and F32 forms only");
    if (!d_fs) return set_error(LBRS_EINVAL, "d_fs is NULL");
    if (!out) return set_error(LBRS_EINVAL, "out is NULL");
    const int64_t N = cfg->nx * cfg->ny;
    if (N > kMaxCells) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "grid of %lld cells exceeds the no-allocation diagnostics limit of %lld cells "
                 "(static scratch of %d partial records); use lbrs_diagnostics with a workspace",
                 (long long)N, (long long)kMaxCells, kMaxBlocks);
        return set_error(LBRS_EINVAL, msg);
    }
    if (cfg->lattice == LBRS_D2Q4S) return set_error(LBRS_EINVAL, "the scalar lattice is not covered here; use lbrs_diagnostics");
    double* scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != LBRS_OK) return st;

    const cudaStream_t stream = (cudaStream_t)cfg->cuda_stream;
    const int nblocks = (int)((N + kCellsPerBlock - 1) / kCellsPerBlock);
    const double vol = cfg->lattice == LBRS_D2Q4 ? cfg->dx * cfg->dx : cfg->dx;
    if (cfg->lattice == LBRS_D2Q4) {
        if (cfg->precision == LBRS_F64)
            noalloc_partial_kernel<double, 4, 4><<<nblocks, kThreads, 0, stream>>>((const double*)d_fs, N, cfg->gamma, cfg->lambda, scratch);
        else
            noalloc_partial_kernel<float, 4, 4><<<nblocks, kThreads, 0, stream>>>((const float*)d_fs, N, cfg->gamma, cfg->lambda, scratch);
    } else if (cfg->lattice == LBRS_D1Q3) {
        if (cfg->precision == LBRS_F64)
            noalloc_partial_kernel<double, 3, 3><<<nblocks, kThreads, 0, stream>>>((const double*)d_fs, N, cfg->gamma, cfg->lambda, scratch);
        else
            noalloc_partial_kernel<float, 3, 3><<<nblocks, kThreads, 0, stream>>>((const float*)d_fs, N, cfg->gamma, cfg->lambda, scratch);
    } else {
        if (cfg->precision == LBRS_F64)
            noalloc_partial_kernel<double, 2, 3><<<nblocks, kThreads, 0, stream>>>((const double*)d_fs, N, cfg->gamma, cfg->lambda, scratch);
        else
            noalloc_partial_kernel<float, 2, 3><<<nblocks, kThreads, 0, stream>>>((const float*)d_fs, N, cfg->gamma, cfg->lambda, scratch);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        noalloc_final_kernel<<<1, 32, 0, stream>>>(nblocks, vol);
        e = cudaGetLastError();
    }
    double h[DIAG_W];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, scratch + (int64_t)kMaxBlocks * DIAG_W, sizeof h, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return set_error(LBRS_ECUDA, cudaGetErrorString(e));

    const int K = cfg->lattice == LBRS_D2Q4 ? 4 : 3;
    for (int k = 0; k < 4; ++k) out->totals[k] = k < K ? h[k] : 0.0;
    out->min_rho = h[4];
    out->min_p = h[5];
    out->max_lambda_local = h[6];
    out->reserved = 0.0;
    out->n_nonphysical = (int64_t)h[7];
    out->n_subchar = (int64_t)h[8];
    if (out->n_nonphysical > 0) return set_error(LBRS_ENONPHYS, "non-physical cells present");
    if (out->n_subchar > 0) return set_error(LBRS_ESUBCHAR, "cells exceed lambda");
    return LBRS_OK;
}
