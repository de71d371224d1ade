// Device code of the LBRS time step (sm_103a).
//
// One step of the Lattice Boltzmann Relaxation Scheme, fused into one kernel
// per lattice: every thread owns one cell and
//   1. pulls its Q*K post-collision populations from the upwind neighbours
//      (f_q(x) = f*_q(x - c_q), exact hopping, discrete LBRS update of
//      Section II.A / multi-D update of Section II.D), resolving sources
//      outside the domain by the boundary kind; on a wall row the entering
//      populations follow the free-slip relations of Section II.E;
//   2. forms the moments U_k = sum_q f_{q,k} (moment relations);
//   3. evaluates the ideal-gas pressure and the Euler fluxes (Section II.C,
//      and their 2-D counterparts for Section II.D);
//   4. builds the equilibria f^eq (Sections II.C, II.D) and relaxes
//      f* = (1 - omega) f + omega f^eq, writing to the other ping-pong buffer.
//
// Storage is structure-of-arrays f[q][k][j][i]: each (q, k) plane is read
// once at a constant (+-1, +-1) offset and written once, so one step moves
// exactly Q*K*(read + write) elements per cell.
//
// The FP64 instantiation is compiled without FMA contraction and with IEEE
// division so that its rounding is that of the plain expressions; the FP32
// one uses one reciprocal per cell and lets the compiler contract.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbrs {

// Index check of the LBRS_DEBUG build, the library's bounds and race check where no
// sanitizer runs: an index outside [0, n) is replaced by 0, so that the access stays
// inside its buffer, and the first such event of the translation unit is recorded
// as (site << 40) | (index mod 2^40) in its debug word, which lbrs_sync reports.  In
// the release build LBRS_IX is the index itself.
#ifdef LBRS_DEBUG
static __device__ unsigned long long g_debug_first = 0ull;   // one per translation unit
static __device__ __forceinline__ int64_t debug_index(int64_t i, int64_t n, int site)
{
    if (i >= 0 && i < n) return i;
    atomicCAS(&g_debug_first, 0ull,
              ((unsigned long long)site << 40) | ((unsigned long long)i & ((1ull << 40) - 1)));
    return 0;
}
#define LBRS_IX(i, n, site) ::lbrs::debug_index((int64_t)(i), (int64_t)(n), (site))
// A host function of the translation unit returning (and with clear, zeroing) its word.
#define LBRS_DEBUG_WORD(name)                                                           \
    unsigned long long name(int clear)                                                  \
    {                                                                                   \
        unsigned long long w = 0ull;                                                    \
        if (cudaMemcpyFromSymbol(&w, g_debug_first, sizeof w) != cudaSuccess) return 0; \
        if (clear && w) {                                                               \
            const unsigned long long z = 0ull;                                          \
            cudaMemcpyToSymbol(g_debug_first, &z, sizeof z);                            \
        }                                                                               \
        return w;                                                                       \
    }
#else
#define LBRS_IX(i, n, site) (i)
#define LBRS_DEBUG_WORD(name) \
    unsigned long long name(int) { return 0ull; }
#endif

// BC_WALL_HALFWAY has the code of LBRS_BC_WALL_HALFWAY (a cut side reaches the kernels as
// BC_TRANSMISSIVE).
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_DIRICHLET = 2, BC_WALL = 3, BC_WALL_HALFWAY = 5 };
// LAT_U2D: a D2Q4 state stored as its moments U directly (the FP16
// non-equilibrium form keeps U in FP32): read-outs treat it as one
// "population" per field.
enum { LAT_D1Q2 = 0, LAT_D2Q4 = 1, LAT_U2D = 2, LAT_D1Q3 = 3, LAT_D2Q4S = 4 };
enum { KIND_CONSERVED = 0, KIND_PRIMITIVE = 1 };

// Ghost-table stride: one Dirichlet side holds Q*K <= 16 values.
constexpr int GHOST_STRIDE = 16;
// Width of one block's diagnostic partial record (doubles).
constexpr int DIAG_W = 10;

template <typename T>
struct StepArgs {
    const T* __restrict__ src;    // f* at time n, [Q][K][ny][nx]
    T* __restrict__ dst;          // f* at time n + 1
    const T* __restrict__ ghost;  // [4][GHOST_STRIDE]: f^eq of each Dirichlet side's state
    int64_t N;                    // plane stride nx * ny
    int nx, ny;
    int bc[4];                    // x-lo, x-hi, y-lo, y-hi
    T om, om1;                    // omega, 1 - omega
    T c;                          // 1/(4 lambda) in 2-D, 1/(2 lambda) in 1-D
    T gm1;                        // gamma - 1
    T* __restrict__ Uout;         // recording steps only: moments U_k of the step, [K][ny][nx]
    const uint8_t* __restrict__ solid;  // D2Q4, nullable: [ny][nx], nonzero = solid cell of an internal wall
};

// ---------------------------------------------------------------- arithmetic

// The FP32 reciprocal of a density: the hardware's approximate reciprocal r0
// (within one unit in the last place; subnormal input or output flushed to zero,
// which a density of a valid state never is), refined by one Newton-Raphson step
// for 1/x, r = r0 + r0 (1 - x r0), both products fused.
__device__ __forceinline__ float rcp_f32(float x)
{
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x));
    const float e = __fmaf_rn(-x, r0, 1.f);
    return __fmaf_rn(r0, e, r0);
}

// Velocities from momenta: IEEE divisions in FP64 (same rounding as the plain
// expressions), one approximate reciprocal in FP32 (rcp_f32).
template <typename T>
__device__ __forceinline__ void velocity2(T rho, T mx, T my, T& u, T& v)
{
    if constexpr (std::is_same<T, double>::value) {
        u = mx / rho;
        v = my / rho;
    } else {
        const float inv = rcp_f32(rho);
        u = mx * inv;
        v = my * inv;
    }
}

template <typename T>
__device__ __forceinline__ T velocity1(T rho, T m)
{
    if constexpr (std::is_same<T, double>::value) {
        return m / rho;
    } else {
        return m * rcp_f32(rho);
    }
}

// D2Q4 equilibria of one state (Section II.D), e[q][k]:
//   F = (rho u, rho u^2 + p, rho u v, u (rho E + p)),
//   G = (rho v, rho v u, rho v^2 + p, v (rho E + p)),
//   f^eq_q = U/4 + sx_q c F + sy_q c G with c = 1/(4 lambda), q = (-,-), (+,-), (+,+), (-,+).
template <typename T>
__device__ __forceinline__ void equilibria2d(const T U[4], T gm1, T c, T e[4][4])
{
    T u, v;
    velocity2<T>(U[0], U[1], U[2], u, v);
    const T p = gm1 * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
    const T F[4] = {U[1], U[1] * u + p, U[1] * v, u * (U[3] + p)};
    const T G[4] = {U[2], U[2] * u, U[2] * v + p, v * (U[3] + p)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T a = T(0.25) * U[k];
        const T b = c * F[k];
        const T d = c * G[k];
        e[0][k] = (a - b) - d;
        e[1][k] = (a + b) - d;
        e[2][k] = (a + b) + d;
        e[3][k] = (a - b) + d;
    }
}

// Scalar D2Q4 equilibria for the 2-D inviscid Burgers law of Section III,
// g1 = u^2/2, g2 = u: f^eq_q = u/4 + sx_q c g1 + sy_q c g2, c = 1/(4 lambda) (Section II.D).
template <typename T>
__device__ __forceinline__ void equilibria2ds(T u, T c, T e[4])
{
    const T g1 = T(0.5) * u * u, g2 = u;
    const T a = T(0.25) * u, b = c * g1, d = c * g2;
    e[0] = (a - b) - d;
    e[1] = (a + b) - d;
    e[2] = (a + b) + d;
    e[3] = (a - b) + d;
}

// Scalar lattice Dirichlet side: the linear profile u0 + slope * s at the centre
// coordinate s = (m + 1/2) dx of the ghost cell along the side; the ghost table of
// the side holds (u0, slope, dx).
template <typename T>
__device__ __forceinline__ T profile_value(const T* g, int m)
{
    return g[0] + g[1] * ((T(m) + T(0.5)) * g[2]);
}

// D1Q2 equilibria (Section II.C): G = (rho u, rho u^2 + p, u (rho E + p)),
// f^eq_{1,2} = U/2 -/+ c G with c = 1/(2 lambda).
template <typename T>
__device__ __forceinline__ void equilibria1d(const T U[3], T gm1, T c, T e[2][3])
{
    const T u = velocity1<T>(U[0], U[1]);
    const T p = gm1 * (U[2] - T(0.5) * (U[1] * u));
    const T G[3] = {U[1], U[1] * u + p, u * (U[2] + p)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T a = T(0.5) * U[k];
        const T b = c * G[k];
        e[0][k] = a - b;
        e[1][k] = a + b;
    }
}

// D1Q3 equilibria (Section II.C, rest particle): f^eq = (U/3 - c G, U/3, U/3 + c G),
// c = 1/(2 lambda), G the 1-D Euler flux.
template <typename T>
__device__ __forceinline__ void equilibria1d3(const T U[3], T gm1, T c, T e[3][3])
{
    const T u = velocity1<T>(U[0], U[1]);
    const T p = gm1 * (U[2] - T(0.5) * (U[1] * u));
    const T G[3] = {U[1], U[1] * u + p, u * (U[2] + p)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T a = U[k] / T(3);
        const T b = c * G[k];
        e[0][k] = a - b;
        e[1][k] = a;
        e[2][k] = a + b;
    }
}

// Conserved variables from primitive ones, rho E = p/(gamma - 1) + rho |u|^2 / 2.
__device__ __forceinline__ void prim_to_cons2d(const double w[4], double gamma, double U[4])
{
    const double rho = w[0], u = w[1], v = w[2], p = w[3];
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * v;
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v);
}

__device__ __forceinline__ void prim_to_cons1d(const double w[3], double gamma, double U[3])
{
    const double rho = w[0], u = w[1], p = w[2];
    U[0] = rho;
    U[1] = rho * u;
    U[2] = p / (gamma - 1.0) + 0.5 * rho * (u * u);
}

// ---------------------------------------------------------------- D2Q4 step

// Pull with boundary resolution for cells on the domain edge.
// Priority: a wall on the y side; a Dirichlet ghost on the x side; a Dirichlet
// ghost on the y side; otherwise wrap (periodic) / clamp (transmissive) each
// coordinate.  Then the free-slip wall relations (Section II.E).
// A halfway wall (the flag alternative of that wall, reflecting at the plane half a
// cell beyond the wall row): a population that would enter through it takes the
// mirror image (sy reversed, m = 3 - q) of the one leaving its horizontal neighbour
// (i - sx, j) on the wall row, rho v negated; the neighbour's x is resolved like a
// pull source (Dirichlet ghost, wrap, clamp).  HALF = false compiles the pull without
// that case, for kernels on a tight register budget that are not launched with it.
template <typename T, bool HALF = true>
__device__ __forceinline__ void pull_edge_2d(const StepArgs<T>& a, int i, int j, T f[4][4])
{
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
    bool wall_top = false, wall_bottom = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int si = i - SX[q], sj = j - SY[q];
        const int side_y = sj < 0 ? 2 : (sj >= a.ny ? 3 : -1);
        const int side_x = si < 0 ? 0 : (si >= a.nx ? 1 : -1);
        // side kinds by selection, not by a runtime index into the parameter
        // block (which would force a local-memory copy of it)
        const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
        const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
        if (side_y >= 0 && kind_y == BC_WALL) {
            if (side_y == 3) wall_top = true; else wall_bottom = true;
            continue;
        }
        if (HALF && side_y >= 0 && kind_y == BC_WALL_HALFWAY) {
            const int m = 3 - q;
            const T* gm = nullptr;
            if (side_x >= 0) {
                if (kind_x == BC_DIRICHLET) gm = a.ghost + side_x * GHOST_STRIDE + m * 4;
                else if (kind_x == BC_PERIODIC) si = si < 0 ? si + a.nx : si - a.nx;
                else si = si < 0 ? 0 : a.nx - 1;
            }
            const int64_t s = (int64_t)j * a.nx + si;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T sgn = k == 2 ? T(-1) : T(1);
                f[q][k] = sgn * (gm ? gm[k] : a.src[LBRS_IX((m * 4 + k) * a.N + s, 16 * a.N, 1)]);
            }
            continue;
        }
        const T* g = nullptr;
        if (side_x >= 0) {
            const int kind = kind_x;
            if (kind == BC_DIRICHLET) g = a.ghost + side_x * GHOST_STRIDE + q * 4;
            else if (kind == BC_PERIODIC) si = si < 0 ? si + a.nx : si - a.nx;
            else si = si < 0 ? 0 : a.nx - 1;
        }
        if (!g && side_y >= 0) {
            const int kind = kind_y;
            if (kind == BC_DIRICHLET) g = a.ghost + side_y * GHOST_STRIDE + q * 4;
            else if (kind == BC_PERIODIC) sj = sj < 0 ? sj + a.ny : sj - a.ny;
            else sj = sj < 0 ? 0 : a.ny - 1;
        }
        const int64_t s = (int64_t)sj * a.nx + si;
#pragma unroll
        for (int k = 0; k < 4; ++k) f[q][k] = g ? g[k] : a.src[LBRS_IX((q * 4 + k) * a.N + s, 16 * a.N, 1)];
    }
    // top wall: f1 = f4, f2 = f3; bottom wall: f4 = f1, f3 = f2; rho v negated
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T sgn = k == 2 ? T(-1) : T(1);
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

// ---------------------------------------------------------------- internal walls
//
// Lattice-aligned obstacles: solid cells are inert (their distributions are
// carried unchanged).  In a fluid cell, a population whose pull source (after the
// domain boundaries) is a solid cell is replaced by a known population of the same
// cell -- the free-slip reflection of Section II.E generalised to obstacle faces:
// with only the axis neighbour (i - sx, j) solid, the wall is normal to x and the
// population mirrored in x, (-sx, sy), is taken with rho u negated; with only
// (i, j - sy) solid, mirrored in y with rho v negated (the paper's upper-wall
// relations); with both or neither (a concave or a convex corner), the opposite
// population with both negated.  Axis neighbours map through the domain sides
// like pull sources (wrap, clamp; Dirichlet and wall sides count as fluid).  The
// host rejects geometries where the chosen population is itself unknown, so the
// replacement is always a pulled or ghost value.  Obstacle populations are
// resolved before the domain-wall relations.

template <typename T>
__device__ __forceinline__ bool solid_at(const StepArgs<T>& a, int i, int j)
{
    if (i < 0 || i >= a.nx) {
        const int kind = i < 0 ? a.bc[0] : a.bc[1];
        if (kind == BC_PERIODIC) i = i < 0 ? i + a.nx : i - a.nx;
        else if (kind == BC_TRANSMISSIVE) i = i < 0 ? 0 : a.nx - 1;
        else return false;
    }
    if (j < 0 || j >= a.ny) {
        const int kind = j < 0 ? a.bc[2] : a.bc[3];
        if (kind == BC_PERIODIC) j = j < 0 ? j + a.ny : j - a.ny;
        else if (kind == BC_TRANSMISSIVE) j = j < 0 ? 0 : a.ny - 1;
        else return false;
    }
    return a.solid[LBRS_IX((int64_t)j * a.nx + i, a.N, 2)] != 0;
}

// The pull of pull_edge_2d for a fluid cell next to obstacles.
template <typename T>
__device__ __forceinline__ void pull_obstacle_2d(const StepArgs<T>& a, int i, int j, T f[4][4])
{
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
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
        const T* g = nullptr;
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
        const int64_t s = (int64_t)sj * a.nx + si;
        if (!g && a.solid[LBRS_IX(s, a.N, 3)]) {
            unknown[q] = true;
            continue;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) f[q][k] = g ? g[k] : a.src[LBRS_IX((q * 4 + k) * a.N + s, 16 * a.N, 3)];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!unknown[q]) continue;
        const bool xn = solid_at(a, i - SX[q], j), yn = solid_at(a, i, j - SY[q]);
        const bool flip_x = !(yn && !xn), flip_y = !(xn && !yn);   // x wall: flip x only; y wall: y only
        const int mx = flip_x ? -SX[q] : SX[q], my = flip_y ? -SY[q] : SY[q];
        const int m = my < 0 ? (mx < 0 ? 0 : 1) : (mx > 0 ? 2 : 3);
        const T su = flip_x ? T(-1) : T(1), sv = flip_y ? T(-1) : T(1);
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
            if (mm != m) continue;
            f[q][0] = f[mm][0];
            f[q][1] = su * f[mm][1];
            f[q][2] = sv * f[mm][2];
            f[q][3] = f[mm][3];
        }
    }
    // domain walls: top f1 = f4, f2 = f3; bottom f4 = f1, f3 = f2; rho v negated
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T sgn = k == 2 ? T(-1) : T(1);
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

// Collision of one cell (Eq. 9 with the equilibria of Eq. 12): moments U of the
// pulled populations f, then out = (1 - omega) f + omega f^eq(U).
// At omega = 1 (a grid-uniform branch) the result is f^eq itself, which is what
// the general expression gives there for any finite f (0 f + 1 f^eq rounds to
// f^eq; only the sign of a zero may differ).
template <typename T>
__device__ __forceinline__ void collide_2d(const StepArgs<T>& a, const T f[4][4], T U[4], T out[4][4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = ((f[0][k] + f[1][k]) + f[2][k]) + f[3][k];
    if (a.om1 == T(0)) {
        equilibria2d<T>(U, a.gm1, a.c, out);
        return;
    }
    T e[4][4];
    equilibria2d<T>(U, a.gm1, a.c, e);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[q][k] = a.om1 * f[q][k] + a.om * e[q][k];
}

template <typename T, bool STORE_U = false>
__device__ __forceinline__ void collide_store_2d(const StepArgs<T>& a, int64_t c, const T f[4][4])
{
    T U[4], out[4][4];
    collide_2d<T>(a, f, U, out);
    if constexpr (STORE_U) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a.Uout[LBRS_IX(k * a.N + c, 4 * a.N, 4)] = U[k];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) a.dst[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 4)] = out[q][k];
}

// One thread per cell; blockDim.x along i (coalesced), blockDim.y along j.
// STORE_U also writes the step's moments (the recording step of the adjoint).
template <typename T, bool STORE_U = false>
__global__ void __launch_bounds__(256) step2d_kernel(const StepArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    T f[4][4];
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        // sources: q0 (-,-) <- (i+1, j+1); q1 (+,-) <- (i-1, j+1);
        //          q2 (+,+) <- (i-1, j-1); q3 (-,+) <- (i+1, j-1)
        const int64_t s[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) f[q][k] = a.src[LBRS_IX((q * 4 + k) * a.N + s[q], 16 * a.N, 5)];
    } else {
        pull_edge_2d<T>(a, i, j, f);
    }
    collide_store_2d<T, STORE_U>(a, c, f);
}

// The D2Q4 step on a grid with internal walls: solid cells carried unchanged,
// fluid cells pulled through pull_obstacle_2d (which also resolves the domain
// sides), then the same collision.
template <typename T, bool STORE_U = false>
__global__ void __launch_bounds__(256) step2d_obstacle_kernel(const StepArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    if (a.solid[LBRS_IX(c, a.N, 6)]) {
        T f[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                f[q][k] = a.src[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 6)];
                a.dst[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 6)] = f[q][k];
            }
        if constexpr (STORE_U) {
#pragma unroll
            for (int k = 0; k < 4; ++k) a.Uout[LBRS_IX(k * a.N + c, 4 * a.N, 6)] = ((f[0][k] + f[1][k]) + f[2][k]) + f[3][k];
        }
        return;
    }
    T f[4][4];
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        // away from the domain sides and from solid sources: the plain interior pull
        const int64_t s[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
        if (!(a.solid[LBRS_IX(s[0], a.N, 6)] | a.solid[LBRS_IX(s[1], a.N, 6)] | a.solid[LBRS_IX(s[2], a.N, 6)] | a.solid[LBRS_IX(s[3], a.N, 6)])) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = a.src[LBRS_IX((q * 4 + k) * a.N + s[q], 16 * a.N, 6)];
            collide_store_2d<T, STORE_U>(a, c, f);
            return;
        }
    }
    pull_obstacle_2d<T>(a, i, j, f);
    collide_store_2d<T, STORE_U>(a, c, f);
}

// ---------------------------------------------------------------- adaptive lambda (D2Q4)
//
// The lattice speed taken anew every step (the sub-characteristic choice of
// Section II.C with the bound of Section II.D): distributions carry the lambda of
// their equilibria, so a step streams with the current state's lambda (the
// Dirichlet ghosts are rebuilt with it; the step advances the time by dx / lambda)
// and collides with the next one, safety times the largest local bound of the
// state before the step and of the Dirichlet states.  The maximum over the cells
// is taken by the step kernel itself for the following step (one block max and one
// 64-bit atomic max per block, of the bits of a non-negative double); a one-thread
// prep kernel before each step turns it into the next lambda, the clock and the
// ghosts.  Three rotating accumulator slots keep reads and resets apart.
struct AdaptState {
    unsigned long long bound_bits[3];   // largest bound of a state, as the bits of a non-negative double
    double t;                           // time reached
    double lam_cur;                     // lambda of the current distributions
    double c_new;                       // 1/(4 lambda) of the running step's collision
    long long steps;                    // adaptive steps taken
    int last;                           // the next step ends the run
    int done;                           // the run reached t_final: further steps keep the state
    int slot_cur;                       // slot with the bound of the current state
    int skip;                           // the running step keeps the state
};

// The local bound max(|u+v|, |u-v|) + sqrt(2) a of a state (Section II.D), in T;
// -1 for a state with rho <= 0, p <= 0 or a non-finite pressure (left out).
template <typename T>
__device__ __forceinline__ double bound2d(const T U[4], double gamma)
{
    const T g = (T)gamma, gm1 = (T)(gamma - 1.0);
    const T u = U[1] / U[0], v = U[2] / U[0];
    const T p = gm1 * (U[3] - T(0.5) * (U[1] * u + U[2] * v));
    if (!(U[0] > T(0)) || !(p > T(0)) || !isfinite(p)) return -1.0;
    const T a = sqrt(g * p / U[0]);
    const T s1 = fabs(u + v), s2 = fabs(u - v);
    return (double)((s1 > s2 ? s1 : s2) + sqrt(T(2)) * a);
}

// The local bound in the storage precision: bound2d for FP64 (the oracle's
// expressions); in FP32 one reciprocal of rho (rcp_f32, the one the
// collision's velocities use) and one square root, sqrt(2 gamma p / rho) for
// sqrt(2) a.
template <typename T>
__device__ __forceinline__ T bound_local(const T U[4], double gamma)
{
    if constexpr (std::is_same<T, float>::value) {
        const float g = (float)gamma, gm1 = (float)(gamma - 1.0);
        const float inv = rcp_f32(U[0]);
        const float u = U[1] * inv, v = U[2] * inv;
        const float p = gm1 * (U[3] - 0.5f * (U[1] * u + U[2] * v));
        if (!(U[0] > 0.f) || !(p > 0.f) || !isfinite(p)) return -1.f;
        return fmaxf(fabsf(u + v), fabsf(u - v)) + sqrtf(2.f * (g * p * inv));
    } else {
        return bound2d<double>(U, gamma);
    }
}

// Block maximum of v (threads of a 1-D or 2-D block of NT threads), folded into *dst
// as the bits of a non-negative double.
template <int NT, typename V>
__device__ __forceinline__ void block_max_into(V v, unsigned long long* dst)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    __shared__ V wmax[NT / 32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) wmax[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        V m = wmax[0];
        for (int w = 1; w < NT / 32; ++w) m = fmax(m, wmax[w]);
        if (m > V(0)) atomicMax(dst, (unsigned long long)__double_as_longlong((double)m));
    }
}

// One adaptive step (stream with the ghosts the prep kernel built, collide with
// c_new), accumulating the bound of the new state into the prep's slot.
template <typename T>
__global__ void __launch_bounds__(256) step2d_adapt_kernel(const StepArgs<T> a, AdaptState* st, double gamma)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool in = i < a.nx && j < a.ny;
    const int64_t c = (int64_t)j * a.nx + i;
    // the pull does not depend on the prep's results: its loads go out before the state is read
    T f[4][4];
    if (in) {
        if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
            const int64_t s[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) f[q][k] = a.src[LBRS_IX((q * 4 + k) * a.N + s[q], 16 * a.N, 7)];
        } else {
            pull_edge_2d<T>(a, i, j, f);
        }
    }
    if (st->skip) {            // the same for every thread of the grid
        if (in) {
#pragma unroll
            for (int n = 0; n < 16; ++n) a.dst[LBRS_IX(n * a.N + c, 16 * a.N, 7)] = a.src[LBRS_IX(n * a.N + c, 16 * a.N, 7)];
        }
        return;
    }
    T bnd = T(-1);
    if (in) {
        StepArgs<T> b = a;
        b.c = (T)st->c_new;
        T U[4], out[4][4];
        collide_2d<T>(b, f, U, out);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) a.dst[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 7)] = out[q][k];
        bnd = bound_local<T>(U, gamma);
    }
    block_max_into<256>(bnd, &st->bound_bits[st->slot_cur]);
}

// The bound of the current state (its moments summed in q order), into slot_cur.
template <typename T>
__global__ void __launch_bounds__(256) adapt_init_bound_kernel(const T* __restrict__ fs, int64_t N, double gamma,
                                                              AdaptState* st)
{
    T bnd = T(-1);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        T U[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = ((fs[k * N + c] + fs[(4 + k) * N + c]) + fs[(8 + k) * N + c]) + fs[(12 + k) * N + c];
        bnd = fmax(bnd, bound_local<T>(U, gamma));
    }
    block_max_into<256>(bnd, &st->bound_bits[st->slot_cur]);
}

// Population q of the Dirichlet ghost of a scalar D2Q4 side: f^eq of the side's profile value at
// coordinate m along the side.
template <typename T>
__device__ __forceinline__ T ghost_population_2ds(const StepArgs<T>& a, const T* g, int m, int q)
{
    T e[4];
    equilibria2ds<T>(profile_value<T>(g, m), a.c, e);
    T v = e[0];
#pragma unroll
    for (int r = 1; r < 4; ++r)
        if (r == q) v = e[r];
    return v;
}

// ---------------------------------------------------------------- scalar D2Q4 step
//
// One thread per cell: pull the four populations (periodic wrap, transmissive
// clamp, Dirichlet ghost f^eq of the side's profile value; x side first), then the
// moment u, the equilibria and the relaxation.

// The pull of cell (i, j) where a source lies beyond a side.
template <typename T>
__device__ __forceinline__ void pull_edge_2ds(const StepArgs<T>& a, int i, int j, T f[4])
{
    const int SX[4] = {-1, 1, 1, -1};
    const int SY[4] = {-1, -1, 1, 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int si = i - SX[q], sj = j - SY[q];
        const int side_y = sj < 0 ? 2 : (sj >= a.ny ? 3 : -1);
        const int side_x = si < 0 ? 0 : (si >= a.nx ? 1 : -1);
        const int kind_y = side_y == 2 ? a.bc[2] : a.bc[3];
        const int kind_x = side_x == 0 ? a.bc[0] : a.bc[1];
        const T* g = nullptr;
        int m = 0;
        if (side_x >= 0) {
            if (kind_x == BC_DIRICHLET) {
                g = a.ghost + side_x * GHOST_STRIDE;
                m = sj;
            } else if (kind_x == BC_PERIODIC) {
                si = si < 0 ? si + a.nx : si - a.nx;
            } else {
                si = si < 0 ? 0 : a.nx - 1;
            }
        }
        if (!g && side_y >= 0) {
            if (kind_y == BC_DIRICHLET) {
                g = a.ghost + side_y * GHOST_STRIDE;
                m = si;
            } else if (kind_y == BC_PERIODIC) {
                sj = sj < 0 ? sj + a.ny : sj - a.ny;
            } else {
                sj = sj < 0 ? 0 : a.ny - 1;
            }
        }
        if (g) {
            f[q] = ghost_population_2ds<T>(a, g, m, q);
        } else {
            f[q] = a.src[LBRS_IX(q * a.N + (int64_t)sj * a.nx + si, 4 * a.N, 8)];
        }
    }
}

// The moment, the equilibria and the relaxation of one cell.
template <typename T>
__device__ __forceinline__ void collide_2ds(const StepArgs<T>& a, const T f[4], T out[4])
{
    const T u = ((f[0] + f[1]) + f[2]) + f[3];
    T e[4];
    equilibria2ds<T>(u, a.c, e);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = a.om1 * f[q] + a.om * e[q];
}

template <typename T>
__global__ void __launch_bounds__(256) step2ds_kernel(const StepArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    T f[4];
    if (i > 0 && i < a.nx - 1 && j > 0 && j < a.ny - 1) {
        const int64_t s[4] = {c + a.nx + 1, c + a.nx - 1, c - a.nx - 1, c - a.nx + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) f[q] = a.src[LBRS_IX(q * a.N + s[q], 4 * a.N, 8)];
    } else {
        pull_edge_2ds<T>(a, i, j, f);
    }
    T out[4];
    collide_2ds<T>(a, f, out);
#pragma unroll
    for (int q = 0; q < 4; ++q) a.dst[LBRS_IX(q * a.N + c, 4 * a.N, 8)] = out[q];
}

// ---------------------------------------------------------------- D1Q2 step

template <typename T>
__global__ void __launch_bounds__(256) step1d_kernel(const StepArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    T f[2][3];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        int si = q == 0 ? i + 1 : i - 1;      // velocity -lambda pulls from i+1, +lambda from i-1
        const T* g = nullptr;
        if (si < 0 || si >= a.nx) {
            const int side = si < 0 ? 0 : 1;
            const int kind = side == 0 ? a.bc[0] : a.bc[1];
            if (kind == BC_DIRICHLET) g = a.ghost + side * GHOST_STRIDE + q * 3;
            else if (kind == BC_PERIODIC) si = si < 0 ? si + a.nx : si - a.nx;
            else si = si < 0 ? 0 : a.nx - 1;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) f[q][k] = g ? g[k] : a.src[LBRS_IX((q * 3 + k) * a.N + si, 6 * a.N, 9)];
    }
    T U[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) U[k] = f[0][k] + f[1][k];
    T e[2][3];
    equilibria1d<T>(U, a.gm1, a.c, e);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) a.dst[LBRS_IX((q * 3 + k) * a.N + i, 6 * a.N, 9)] = a.om1 * f[q][k] + a.om * e[q][k];
}

// ---------------------------------------------------------------- D1Q3 step

// Velocity -lambda pulls from i + 1, the rest particle stays, +lambda pulls from i - 1.
template <typename T>
__global__ void __launch_bounds__(256) step1d_q3_kernel(const StepArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    T f[3][3];
#pragma unroll
    for (int q = 0; q < 3; q += 2) {
        int si = q == 0 ? i + 1 : i - 1;
        const T* g = nullptr;
        if (si < 0 || si >= a.nx) {
            const int side = si < 0 ? 0 : 1;
            const int kind = side == 0 ? a.bc[0] : a.bc[1];
            if (kind == BC_DIRICHLET) g = a.ghost + side * GHOST_STRIDE + q * 3;
            else if (kind == BC_PERIODIC) si = si < 0 ? si + a.nx : si - a.nx;
            else si = si < 0 ? 0 : a.nx - 1;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) f[q][k] = g ? g[k] : a.src[LBRS_IX((q * 3 + k) * a.N + si, 9 * a.N, 9)];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) f[1][k] = a.src[LBRS_IX((3 + k) * a.N + i, 9 * a.N, 9)];
    T U[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) U[k] = (f[0][k] + f[1][k]) + f[2][k];
    T e[3][3];
    equilibria1d3<T>(U, a.gm1, a.c, e);
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) a.dst[LBRS_IX((q * 3 + k) * a.N + i, 9 * a.N, 9)] = a.om1 * f[q][k] + a.om * e[q][k];
}

// ---------------------------------------------------------------- adjoint (periodic D2Q4)
//
// Discrete adjoint of the step above (not in the paper).  Forward:
// f = S f*^n, U = M f, f*^{n+1} = (1 - w) f + w E(U).  With g = dL/df*^{n+1}:
//   fbar_{q,k} = (1 - w) g_{q,k} + w ubar_k,  ubar = J_E(U)^T g,
//   dL/df*^n_q(x - c_q) = fbar_q(x)   (transposed shift: push back along -c_q).
// J_E^T g = a/4 + c A_F^T bx + c A_G^T by, a_k = sum_q g_{q,k},
// bx_k = sum_q sx_q g_{q,k}, by_k = sum_q sy_q g_{q,k}, c = 1/(4 lambda), with
// A_F = dF/dU, A_G = dG/dU the ideal-gas Euler flux Jacobians.

template <typename T>
__device__ __forceinline__ void equilibrium_vjp2d(const T U[4], const T g[4][4], T gamma, T gm1, T c, T ubar[4])
{
    const T rho = U[0], mx = U[1], my = U[2], en = U[3];
    T u, v;
    velocity2<T>(rho, mx, my, u, v);
    const T p = gm1 * (en - T(0.5) * (mx * u + my * v));
    T H;
    if constexpr (std::is_same<T, double>::value)
        H = (en + p) / rho;
    else
        H = (en + p) * rcp_f32(rho);   // the reciprocal the velocities used
    const T q2h = T(0.5) * gm1 * (u * u + v * v);
    const T dF[4][4] = {{T(0), T(1), T(0), T(0)},
                        {q2h - u * u, (T(3) - gamma) * u, -gm1 * v, gm1},
                        {-u * v, v, u, T(0)},
                        {u * (q2h - H), H - gm1 * u * u, -gm1 * u * v, gamma * u}};
    const T dG[4][4] = {{T(0), T(0), T(1), T(0)},
                        {-u * v, v, u, T(0)},
                        {q2h - v * v, -gm1 * u, (T(3) - gamma) * v, gm1},
                        {v * (q2h - H), -gm1 * u * v, H - gm1 * v * v, gamma * v}};
    const T SXv[4] = {T(-1), T(1), T(1), T(-1)};
    const T SYv[4] = {T(-1), T(-1), T(1), T(1)};
    T av[4], bx[4], by[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        av[k] = bx[k] = by[k] = T(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            av[k] += g[q][k];
            bx[k] += SXv[q] * g[q][k];
            by[k] += SYv[q] * g[q][k];
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T sf = T(0), sg = T(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            sf += dF[r][k] * bx[r];
            sg += dG[r][k] * by[r];
        }
        ubar[k] = T(0.25) * av[k] + c * sf + c * sg;
    }
}

template <typename T>
struct AdjArgs {
    const T* __restrict__ U;      // moments of step n+1 (or U0 for the equilibrium VJP), [4][ny][nx]
    const T* __restrict__ gin;    // dL/df*^{n+1}, [4][4][ny][nx]
    T* __restrict__ gout;         // dL/df*^n (or dL/dU0), written
    int64_t N;
    int nx, ny;
    T om, om1, c, gm1, gamma;
};

// One thread per source cell x: read g(x) and U(x), push fbar_q(x) to x - c_q (periodic).
template <typename T>
__global__ void __launch_bounds__(256) adjoint2d_kernel(const AdjArgs<T> a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.nx || j >= a.ny) return;
    const int64_t c = (int64_t)j * a.nx + i;
    T g[4][4], U[4], ubar[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 30)];
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 30)];
    equilibrium_vjp2d<T>(U, g, a.gamma, a.gm1, a.c, ubar);
    // targets x - c_q: q0 (-,-) -> (i+1, j+1); q1 (+,-) -> (i-1, j+1); q2 (+,+) -> (i-1, j-1); q3 (-,+) -> (i+1, j-1)
    const int ip = i + 1 == a.nx ? 0 : i + 1, im = i == 0 ? a.nx - 1 : i - 1;
    const int jp = j + 1 == a.ny ? 0 : j + 1, jm = j == 0 ? a.ny - 1 : j - 1;
    const int64_t t[4] = {(int64_t)jp * a.nx + ip, (int64_t)jp * a.nx + im, (int64_t)jm * a.nx + im,
                          (int64_t)jm * a.nx + ip};
    // omega = 1: fbar = J_E^T g alone (what the general expression rounds to for finite g)
    const bool eq_only = a.om1 == T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            a.gout[LBRS_IX((q * 4 + k) * a.N + t[q], 16 * a.N, 30)] = eq_only ? ubar[k] : a.om1 * g[q][k] + a.om * ubar[k];
}

// dL/dU0 = J_E(U0)^T dL/df*^0, per cell.
template <typename T>
__global__ void __launch_bounds__(256) vjp_equilibrium2d_kernel(const AdjArgs<T> a)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.N; c += (int64_t)gridDim.x * blockDim.x) {
        T g[4][4], U[4], ubar[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) g[q][k] = a.gin[LBRS_IX((q * 4 + k) * a.N + c, 16 * a.N, 31)];
#pragma unroll
        for (int k = 0; k < 4; ++k) U[k] = a.U[LBRS_IX(k * a.N + c, 4 * a.N, 31)];
        equilibrium_vjp2d<T>(U, g, a.gamma, a.gm1, a.c, ubar);
#pragma unroll
        for (int k = 0; k < 4; ++k) a.gout[LBRS_IX(k * a.N + c, 4 * a.N, 31)] = ubar[k];
    }
}

}  // namespace lbrs
