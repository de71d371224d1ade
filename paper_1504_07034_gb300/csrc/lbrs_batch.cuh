// Batched D1Q2 or D1Q3 time steps for many independent shock tubes (device code).
//
// Each tube b has its own length N_b, lattice speed lambda_b (c_b = 1/(2 lambda_b))
// and number of steps; all share gamma, omega and the boundary kind
// (transmissive or periodic at both ends).  The tubes are concatenated:
// f[q][k][off_b + x], x in [0, N_b), plane stride N = sum N_b; Q = 2 (D1Q2) or 3
// (D1Q3, the rest particle of Section II.C).
//
// Temporal blocking.  A launch advances every active tube by up to H steps.
// One CTA owns a tile of TILE cells of one tube and stages the window
// [t0 - H, t0 + TILE + H) of it (clamped to the tube, or wrapped for periodic
// tubes) in shared memory; it then applies the D1Q2 step (pull-stream,
// moments, flux, equilibria, relaxation; Section II.C) H times in shared
// memory.  Velocities are +-1 cell per step, so after s steps the window's
// cells within s of a cut edge are stale while the tile's own TILE cells,
// H away from the cuts, stay exact; at a tube's own ends the transmissive
// clamp is applied exactly as in the single-tube kernel.  The tile is then
// written back to the other ping-pong buffer.  Per cell update the
// arithmetic is that of step1d_kernel, in the same order.
#pragma once

#include "lbrs_kernels.cuh"

namespace lbrs {

struct BatchTile {
    int tube;     // tube index
    int t0;       // first cell of the tile within the tube
    int len;      // cells in the tile (<= TILE)
    int pad;
};

template <typename T>
struct BatchArgs {
    const T* __restrict__ src;
    T* __restrict__ dst;
    int64_t N;                              // plane stride: total cells
    const BatchTile* __restrict__ tiles;    // active tiles first
    const int64_t* __restrict__ tube_off;   // first cell of each tube in the planes
    const int* __restrict__ tube_len;
    const int* __restrict__ tube_steps;     // steps of each tube in this run
    const T* __restrict__ tube_c;           // 1/(2 lambda_b)
    // one tube (tiles == nullptr): tile blockIdx.x covers cells [blockIdx.x * TILE, + TILE) of a
    // tube of one_len cells at offset 0, stepped one_steps - launch * H times (at most H), c = one_c
    int one_len, one_steps;
    T one_c;
    int tile_cells;                         // TILE
    int halo;                               // H
    int periodic;                           // 1: periodic tubes, 0: transmissive ends
    int launch;                             // index of this launch within the run
    int q;                                  // 2 (D1Q2) or 3 (D1Q3)
    T om, om1, gm1;
};

// Window of W = TILE + 2H cells: W slots per (q, k) plane in shared memory, two
// buffers of 3Q planes.  BLOCK threads, each owning slots i = tid, tid + BLOCK, ...
template <typename T, int BLOCK, int Q>
__global__ void __launch_bounds__(BLOCK) batch1d_kernel(const BatchArgs<T> a)
{
    constexpr int P = 3 * Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const bool one = a.tiles == nullptr;
    const int4 tile = one ? make_int4(0, (int)blockIdx.x * a.tile_cells, 0, 0)
                          : __ldg(reinterpret_cast<const int4*>(a.tiles) + blockIdx.x);   // {tube, t0, len, pad}
    const int b = tile.x;
    const int H = a.halo;
    const int W = a.tile_cells + 2 * H;
    const int len = one ? a.one_len : a.tube_len[b];
    const int ns = min(H, (one ? a.one_steps : a.tube_steps[b]) - a.launch * H);   // >= 1 for an active tile
    const int64_t off = one ? 0 : a.tube_off[b];
    const T c = one ? a.one_c : a.tube_c[b];
    const int t0 = tile.y, tlen = one ? min(a.tile_cells, len - t0) : tile.z;
    const int x0 = t0 - H;                  // tube coordinate of window slot 0
    // slots whose tube coordinate is outside [0, len) exist only for periodic tubes

    for (int i = threadIdx.x; i < W; i += BLOCK) {
        int x = x0 + i;
        if (a.periodic) {
            x %= len;
            x += (x >> 31) & len;
        }
        if (x >= 0 && x < len) {
#pragma unroll
            for (int n = 0; n < P; ++n) sm[LBRS_IX(n * W + i, P * W, 20)] = a.src[LBRS_IX(n * a.N + off + x, P * a.N, 21)];
        }
    }
    __syncthreads();

    // the window slots that exist: all of them for periodic tubes, the tube's
    // own cells otherwise
    const int lo = a.periodic ? 0 : max(0, -x0);
    const int hi = a.periodic ? W : min(W, len - x0);
    int cur = 0;
    for (int s = 0; s < ns; ++s) {
        const T* in = sm + cur * P * W;
        T* out = sm + (cur ^ 1) * P * W;
        for (int i = lo + threadIdx.x; i < hi; i += BLOCK) {
            // velocity -1 pulls from i + 1, +1 from i - 1; at a tube end the
            // transmissive clamp returns the cell itself; at a window cut the
            // slot is stale anyway (outside the valid cone), clamp to stay in bounds
            const int ip = i + 1 < hi ? i + 1 : hi - 1;
            const int im = i - 1 >= lo ? i - 1 : lo;
            // D1Q3: the rest population stays in its cell
            T f[Q][3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[0][k] = in[LBRS_IX(k * W + ip, P * W, 20)];
                if constexpr (Q == 3) {
                    f[1][k] = in[LBRS_IX((3 + k) * W + i, P * W, 20)];
                    f[2][k] = in[LBRS_IX((6 + k) * W + im, P * W, 20)];
                } else {
                    f[1][k] = in[LBRS_IX((3 + k) * W + im, P * W, 20)];
                }
            }
            T U[3];
            T e[Q][3];
            if constexpr (Q == 3) {
#pragma unroll
                for (int k = 0; k < 3; ++k) U[k] = (f[0][k] + f[1][k]) + f[2][k];
                equilibria1d3<T>(U, a.gm1, c, e);
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) U[k] = f[0][k] + f[1][k];
                equilibria1d<T>(U, a.gm1, c, e);
            }
            if (a.om1 == T(0)) {
                // omega = 1 (uniform over the launch): the relaxation returns f^eq, which is
                // what the general expression rounds to for any finite f
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int k = 0; k < 3; ++k) out[LBRS_IX((q * 3 + k) * W + i, P * W, 20)] = e[q][k];
            } else {
#pragma unroll
                for (int q = 0; q < Q; ++q)
#pragma unroll
                    for (int k = 0; k < 3; ++k) out[LBRS_IX((q * 3 + k) * W + i, P * W, 20)] = a.om1 * f[q][k] + a.om * e[q][k];
            }
        }
        __syncthreads();
        cur ^= 1;
    }

    const T* fin = sm + cur * P * W;
    for (int i = threadIdx.x; i < tlen; i += BLOCK) {
        const int slot = H + i;
        const int64_t g = off + t0 + i;
#pragma unroll
        for (int n = 0; n < P; ++n) a.dst[LBRS_IX(n * a.N + g, P * a.N, 21)] = fin[LBRS_IX(n * W + slot, P * W, 20)];
    }
}

// Copy the cells of the listed tiles from src to dst (tubes whose final state
// ended in the other ping-pong buffer).
template <typename T>
__global__ void batch_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t N,
                                  const BatchTile* __restrict__ tiles, const int64_t* __restrict__ tube_off, int planes)
{
    const int4 tile = __ldg(reinterpret_cast<const int4*>(tiles) + blockIdx.x);   // {tube, t0, len, pad}
    const int64_t base = tube_off[tile.x] + tile.y;
    for (int i = threadIdx.x; i < tile.z; i += blockDim.x)
        for (int n = 0; n < planes; ++n) dst[n * N + base + i] = src[n * N + base + i];
}

}  // namespace lbrs
