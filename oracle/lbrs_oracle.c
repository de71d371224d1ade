/*
 * Plain FP64 CPU oracle of the Lattice Boltzmann Relaxation Scheme (LBRS).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never
 * does, and it shares no code with the CUDA library.
 *
 * It follows the paper (Raghurama Rao, Deshmukh, Kotnala, "A Lattice
 * Boltzmann Relaxation Scheme for Inviscid Compressible Flows") step by step,
 * in the paper's order, on separate arrays:
 *
 *   state      fs[q][k][cell] : post-collision distributions at time n
 *   initialise fs = f^eq(U0)                                 (Section II.A)
 *   one step   1. stream:   f_q(x) = fs_q(x - c_q dt)       (discrete LBRS update)
 *              2. boundary: ghosts / wall relations          (Section II.E)
 *              3. moments:  U_k = sum_q f_{q,k}               (moment relations)
 *              4. fluxes:   Euler F(U), G(U), ideal gas       (Sections II.C, II.D)
 *              5. equilibria f^eq from U and the fluxes        (Sections II.C, II.D)
 *              6. relax:    fs = (1 - w) f + w f^eq           (discrete LBRS update)
 *
 * Lattices (q is 0-based; the paper numbers them from 1):
 *   D1Q2 : c = (-1, +1) lattice units, K = 3 fields (rho, rho u, rho E).
 *          f^eq_{1,2} = U/2 -/+ G/(2 lambda)                  (Section II.C)
 *   D1Q3 : c = (-1, 0, +1), K = 3 (rest particle added, Section II.C):
 *          f^eq = (U/3 - G/(2 lambda), U/3, U/3 + G/(2 lambda))
 *   D2Q4 : c = (-1,-1), (+1,-1), (+1,+1), (-1,+1), K = 4 fields
 *          (rho, rho u, rho v, rho E);
 *          f^eq_q = U/4 + sx_q F/(4 lambda) + sy_q G/(4 lambda) (Section II.D)
 *
 * Readings where the paper is silent (stated once here):
 *   - lambda is one global constant and dt = dx / lambda (exact hopping).
 *   - transmissive boundary: the pull source index is clamped into the domain;
 *     Dirichlet boundary: the ghost holds f^eq of the boundary state with the
 *     run's lambda; periodic: the source index wraps.
 *   - the free-slip wall (Section II.E) is applied on the wall row itself
 *     after streaming: at a top wall the unknown downward populations are
 *     f1 = f4, f2 = f3 (negated for the rho v field); a bottom wall mirrors
 *     it: f4 = f1, f3 = f2 (negated for rho v).  Walls exist on the y sides.
 *   - the halfway alternative of that wall (a flag, ORC_WALL_HALFWAY): the
 *     wall lies half a cell beyond the wall row, and a population that would
 *     enter through it takes, by specular reflection there, the post-collision
 *     value of its mirror image: at a bottom wall f3(i, 0) = f*2(i - 1, 0) and
 *     f4(i, 0) = f*1(i + 1, 0), at a top wall f1(i, ny-1) = f*4(i + 1, ny-1)
 *     and f2(i, ny-1) = f*3(i - 1, ny-1), negated for rho v; the horizontal
 *     neighbour is resolved by the x sides like any pull source.  A domain
 *     with such walls on both y sides is the lower half of a periodic domain
 *     of twice the height whose upper half is its mirror image.
 *   - priority at a corner: a wall on the y side first, then a Dirichlet
 *     ghost on the x side, then a Dirichlet ghost on the y side, otherwise the
 *     source index is wrapped/clamped coordinate by coordinate.
 *   - the pressure is p = (gamma - 1)(rho E - |rho u|^2 / (2 rho)), written as
 *     (gamma - 1)(rho E - (rho u * u + rho v * v) / 2) with u = rho u / rho.
 *
 * Build (the flags matter: no FMA contraction, so that rounding is that of
 * the plain expressions below):
 *   gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC lbrs_oracle.c -o liblbrs_oracle.so -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

enum { ORC_PERIODIC = 0, ORC_TRANSMISSIVE = 1, ORC_DIRICHLET = 2, ORC_WALL = 3, ORC_WALL_HALFWAY = 4 };
enum { ORC_D1Q2 = 2, ORC_D1Q3 = 3, ORC_D2Q4 = 4, ORC_D2Q4S = 5 };

typedef struct {
    int32_t lattice;      /* ORC_D1Q2, ORC_D1Q3, ORC_D2Q4 or ORC_D2Q4S (scalar Burgers) */
    int32_t nthreads;     /* OpenMP threads, 0 = library default */
    int64_t nx, ny;       /* ny = 1 for D1Q2 */
    double gamma, lambda, omega;
    int32_t bc_kind[4];   /* x-lo, x-hi, y-lo, y-hi */
    double bc_prim[4][4]; /* Dirichlet primitive state per side: (rho,u,p) in 1-D, (rho,u,v,p) in 2-D */
    const uint8_t* solid; /* D2Q4 only, nullable: [ny][nx], nonzero = solid (internal wall) cell */
    double dx;            /* lattice spacing (the scalar lattice's boundary profiles) */
} orc_params;

typedef struct {
    int64_t first_bad_step;   /* first step with rho <= 0, p <= 0, NaN or lambda_loc > lambda; -1 if none */
    int64_t n_nonphysical;    /* cells with rho <= 0, p <= 0 or a non-finite value (last bad step) */
    int64_t n_subchar;        /* cells with lambda_loc > lambda (last bad step) */
    double max_lambda_local;  /* max over all checked steps and cells */
} orc_check;

/* velocity signs, q = 0..3 <-> the paper's f1..f4 */
static const int SX2[4] = {-1, +1, +1, -1};
static const int SY2[4] = {-1, -1, +1, +1};
static const int SX1[2] = {-1, +1};
static const int SX13[3] = {-1, 0, +1};

static int threads_of(const orc_params* P) { return P->nthreads > 0 ? P->nthreads : omp_get_max_threads(); }
static int two_d(const orc_params* P) { return P->lattice == ORC_D2Q4 || P->lattice == ORC_D2Q4S; }
static int nq(const orc_params* P) { return two_d(P) ? 4 : (P->lattice == ORC_D1Q3 ? 3 : 2); }
static int nk(const orc_params* P) { return P->lattice == ORC_D2Q4 ? 4 : (P->lattice == ORC_D2Q4S ? 1 : 3); }

/* ---------------------------------------------------------------- state */

/* Conserved variables from primitive ones, E = p/(rho (gamma-1)) + |u|^2/2 (Section II.C). */
static void prim_to_cons_cell(const orc_params* P, const double* w, double* U)
{
    double g = P->gamma;
    if (P->lattice == ORC_D2Q4S) {
        U[0] = w[0];                 /* the scalar is its own conserved variable */
        return;
    }
    if (P->lattice == ORC_D2Q4) {
        double rho = w[0], u = w[1], v = w[2], p = w[3];
        U[0] = rho;
        U[1] = rho * u;
        U[2] = rho * v;
        U[3] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
    } else {
        double rho = w[0], u = w[1], p = w[2];
        U[0] = rho;
        U[1] = rho * u;
        U[2] = p / (g - 1.0) + 0.5 * rho * (u * u);
    }
}

/* Ideal-gas pressure from conserved variables (inverse of the E definition). */
static double pressure(const orc_params* P, const double* U)
{
    double g = P->gamma;
    if (P->lattice == ORC_D2Q4) {
        double u = U[1] / U[0], v = U[2] / U[0];
        return (g - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));
    }
    double u = U[1] / U[0];
    return (g - 1.0) * (U[2] - 0.5 * (U[1] * u));
}

/* Equilibria of one cell, feq[q*K + k] (Sections II.C and II.D). */
static void feq_cell(const orc_params* P, const double* U, double* feq)
{
    double g = P->gamma;
    if (P->lattice == ORC_D2Q4S) {
        /* scalar law u_t + g1(u)_x + g2(u)_y = 0 with the inviscid Burgers fluxes of
         * Section III, g1 = u^2/2, g2 = u; f^eq_q = u/4 + sx g1/(4 lambda) + sy g2/(4 lambda)
         * (Section II.D) */
        double u = U[0];
        double g1 = 0.5 * u * u, g2 = u;
        double c = 1.0 / (4.0 * P->lambda);
        for (int q = 0; q < 4; ++q) {
            double a = 0.25 * u;
            double b = c * g1;
            double d = c * g2;
            double t = SX2[q] < 0 ? a - b : a + b;
            feq[q] = SY2[q] < 0 ? t - d : t + d;
        }
        return;
    }
    if (P->lattice == ORC_D2Q4) {
        /* 2-D Euler fluxes: F = (rho u, rho u^2 + p, rho u v, u(rho E + p)),
         *                   G = (rho v, rho v u, rho v^2 + p, v(rho E + p)). */
        double rho = U[0], mx = U[1], my = U[2], en = U[3];
        double u = mx / rho, v = my / rho;
        double p = (g - 1.0) * (en - 0.5 * (mx * u + my * v));
        double F[4], G[4];
        F[0] = mx;         G[0] = my;
        F[1] = mx * u + p; G[1] = my * u;
        F[2] = mx * v;     G[2] = my * v + p;
        F[3] = u * (en + p); G[3] = v * (en + p);
        double c = 1.0 / (4.0 * P->lambda);
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < 4; ++k) {
                double a = 0.25 * U[k];
                double b = c * F[k];
                double d = c * G[k];
                /* U/4 + sx F/(4 lambda) + sy G/(4 lambda), summed left to right */
                double t = SX2[q] < 0 ? a - b : a + b;
                feq[q * 4 + k] = SY2[q] < 0 ? t - d : t + d;
            }
    } else {
        /* 1-D Euler flux G = (rho u, p + rho u^2, p u + rho u E) */
        double rho = U[0], m = U[1], en = U[2];
        double u = m / rho;
        double p = (g - 1.0) * (en - 0.5 * (m * u));
        double G[3] = {m, m * u + p, u * (en + p)};
        double c = 1.0 / (2.0 * P->lambda);
        if (P->lattice == ORC_D1Q3) {
            for (int k = 0; k < 3; ++k) {
                double a = U[k] / 3.0;
                double b = c * G[k];
                feq[0 * 3 + k] = a - b;   /* velocity -lambda */
                feq[1 * 3 + k] = a;       /* rest particle */
                feq[2 * 3 + k] = a + b;   /* velocity +lambda */
            }
        } else {
            for (int k = 0; k < 3; ++k) {
                double a = 0.5 * U[k];
                double b = c * G[k];
                feq[0 * 3 + k] = a - b;   /* velocity -lambda */
                feq[1 * 3 + k] = a + b;   /* velocity +lambda */
            }
        }
    }
}

/* Local wave-speed bound: |u| + a for D1Q2 (Section II.C), max(|u+v|,|u-v|) + sqrt(2) a
 * for D2Q4 (Section II.D).  For D1Q3 the Chapman-Enskog analysis of Section II.B
 * with sum_q lambda_q^2 f^eq_q = (2/3) lambda^2 U gives a positive diffusion for a
 * wave of speed c only if c^2 < (2/3) lambda^2, hence the bound sqrt(3/2)(|u| + a). */
static double lambda_local(const orc_params* P, const double* U, double p)
{
    /* scalar D2Q4: f^eq_q is non-decreasing in u for every q iff lambda >= |g1'| + |g2'| = |u| + 1 */
    if (P->lattice == ORC_D2Q4S) return fabs(U[0]) + 1.0;
    double a = sqrt(P->gamma * p / U[0]);
    if (P->lattice == ORC_D2Q4) {
        double u = U[1] / U[0], v = U[2] / U[0];
        double s1 = fabs(u + v), s2 = fabs(u - v);
        return (s1 > s2 ? s1 : s2) + sqrt(2.0) * a;
    }
    if (P->lattice == ORC_D1Q3) return sqrt(1.5) * (fabs(U[1] / U[0]) + a);
    return fabs(U[1] / U[0]) + a;
}

/* ---------------------------------------------------------------- exported */

void orc_prim_to_cons(const orc_params* P, const double* W, double* U)
{
    int64_t N = P->nx * P->ny;
    int K = nk(P);
    for (int64_t c = 0; c < N; ++c) {
        double w[4], u[4];
        for (int k = 0; k < K; ++k) w[k] = W[k * N + c];
        prim_to_cons_cell(P, w, u);
        for (int k = 0; k < K; ++k) U[k * N + c] = u[k];
    }
}

/* Primitive variables (rho, u, [v,] p) from conserved ones. */
void orc_cons_to_prim(const orc_params* P, const double* U, double* W)
{
    int64_t N = P->nx * P->ny;
    int K = nk(P);
    for (int64_t c = 0; c < N; ++c) {
        double u[4];
        for (int k = 0; k < K; ++k) u[k] = U[k * N + c];
        W[0 * N + c] = u[0];
        if (K == 1) continue;
        W[1 * N + c] = u[1] / u[0];
        if (K == 4) W[2 * N + c] = u[2] / u[0];
        W[(K - 1) * N + c] = pressure(P, u);
    }
}

/* f^eq of a batch of states: U[k*n + c] -> feq[(q*K + k)*n + c]. */
void orc_feq(const orc_params* P, int64_t n, const double* U, double* feq)
{
    int Q = nq(P), K = nk(P);
    for (int64_t c = 0; c < n; ++c) {
        double u[4], f[16];
        for (int k = 0; k < K; ++k) u[k] = U[k * n + c];
        feq_cell(P, u, f);
        for (int q = 0; q < Q; ++q)
            for (int k = 0; k < K; ++k) feq[(q * K + k) * n + c] = f[q * K + k];
    }
}

/* Initialisation f_i = f^eq_i(U0) (Section II.A). */
void orc_init(const orc_params* P, const double* U0, double* fs)
{
    orc_feq(P, P->nx * P->ny, U0, fs);
}

/* Moments U_k = sum_q fs_{q,k}, summed in q order (moment relations, Section II). */
void orc_moments(const orc_params* P, const double* fs, double* U)
{
    int64_t N = P->nx * P->ny;
    int Q = nq(P), K = nk(P);
    for (int k = 0; k < K; ++k)
        for (int64_t c = 0; c < N; ++c) {
            double s = fs[(0 * K + k) * N + c];
            for (int q = 1; q < Q; ++q) s += fs[(q * K + k) * N + c];
            U[k * N + c] = s;
        }
}

int orc_validate(const orc_params* P)
{
    if (P->lattice != ORC_D1Q2 && P->lattice != ORC_D1Q3 && P->lattice != ORC_D2Q4 && P->lattice != ORC_D2Q4S)
        return 1;
    if (P->nx < 1 || P->ny < 1) return 2;
    if (!two_d(P) && P->ny != 1) return 3;
    if (!(P->lambda > 0.0) || !(P->omega > 0.0 && P->omega < 2.0) || !(P->gamma > 1.0)) return 4;
    int sides = two_d(P) ? 4 : 2;
    for (int s = 0; s < sides; ++s) {
        int kind = P->bc_kind[s];
        if (kind < ORC_PERIODIC || kind > ORC_WALL_HALFWAY) return 5;
        if ((kind == ORC_WALL || kind == ORC_WALL_HALFWAY) && P->lattice == ORC_D2Q4S) return 11;   /* no wall rule for a scalar */
        if ((kind == ORC_WALL || kind == ORC_WALL_HALFWAY) && s < 2) return 6;   /* walls on the y sides only */
        if (kind == ORC_WALL_HALFWAY && P->solid) return 13;  /* not combined with internal walls */
        if (kind == ORC_PERIODIC && P->bc_kind[s ^ 1] != ORC_PERIODIC) return 7;
    }
    if (P->lattice == ORC_D2Q4 && (P->bc_kind[2] == ORC_WALL || P->bc_kind[3] == ORC_WALL) && P->ny < 2)
        return 8;
    if (P->solid && P->lattice != ORC_D2Q4) return 9;
    if (P->lattice == ORC_D2Q4S && !(P->dx > 0.0)) return 12;
    return 0;
}

/*
 * Internal walls (lattice-aligned obstacles), extending the free-slip wall of
 * Section II.E to solid cells.  Readings (the paper gives the rule for a
 * straight upper wall only):
 *   - solid cells are inert: their distributions are carried unchanged;
 *   - in a fluid cell, a population whose pull source (after the domain
 *     boundaries) is a solid cell is unknown after streaming.  It takes the
 *     value of a known population of the same cell, chosen by which of the two
 *     axis neighbours towards the source, (i - sx, j) and (i, j - sy), is solid:
 *       only the x neighbour: a wall normal to x -> the population mirrored in x,
 *                             (-sx, sy), with rho u negated;
 *       only the y neighbour: a wall normal to y -> mirrored in y, (sx, -sy),
 *                             with rho v negated (the paper's upper-wall rule);
 *       both or neither (a concave or a convex corner): the opposite population
 *                             (-sx, -sy), with rho u and rho v negated;
 *   - the axis neighbours are mapped through the domain boundaries like a
 *     pull source (wrap, clamp); a Dirichlet or wall side counts as fluid;
 *   - a geometry where the chosen population is itself unknown (a fluid
 *     channel one cell wide, say) is rejected;
 *   - obstacle populations are resolved before the domain-wall relations.
 */
static int is_solid(const orc_params* P, int64_t i, int64_t j)
{
    const int64_t nx = P->nx, ny = P->ny;
    if (i < 0 || i >= nx) {
        int kind = P->bc_kind[i < 0 ? 0 : 1];
        if (kind == ORC_PERIODIC) i = (i + nx) % nx;
        else if (kind == ORC_TRANSMISSIVE) i = i < 0 ? 0 : nx - 1;
        else return 0;
    }
    if (j < 0 || j >= ny) {
        int kind = P->bc_kind[j < 0 ? 2 : 3];
        if (kind == ORC_PERIODIC) j = (j + ny) % ny;
        else if (kind == ORC_TRANSMISSIVE) j = j < 0 ? 0 : ny - 1;
        else return 0;
    }
    return P->solid[j * nx + i] != 0;
}

/* The population that replaces q (unknown at cell (i, j)) and the signs of rho u, rho v. */
static int obstacle_mirror(const orc_params* P, int64_t i, int64_t j, int q, double* sgn_u, double* sgn_v)
{
    int sx = SX2[q], sy = SY2[q];
    int xn = is_solid(P, i - sx, j), yn = is_solid(P, i, j - sy);
    int mx = sx, my = sy;
    if (xn && !yn) {
        mx = -sx;
    } else if (!xn && yn) {
        my = -sy;
    } else {
        mx = -sx;
        my = -sy;
    }
    *sgn_u = mx != sx ? -1.0 : 1.0;
    *sgn_v = my != sy ? -1.0 : 1.0;
    for (int m = 0; m < 4; ++m)
        if (SX2[m] == mx && SY2[m] == my) return m;
    return -1;
}

/* How the pull of population q into (i, j) resolves: 0 a grid cell that is fluid,
 * 1 a Dirichlet ghost, 2 a wall side, 3 a solid cell. */
static int pull_kind(const orc_params* P, int64_t i, int64_t j, int q)
{
    const int64_t nx = P->nx, ny = P->ny;
    int64_t si = i - SX2[q], sj = j - SY2[q];
    int side_y = sj < 0 ? 2 : (sj >= ny ? 3 : -1);
    int side_x = si < 0 ? 0 : (si >= nx ? 1 : -1);
    if (side_y >= 0 && P->bc_kind[side_y] == ORC_WALL) return 2;
    if (side_x >= 0 && P->bc_kind[side_x] == ORC_DIRICHLET) return 1;
    if (side_y >= 0 && P->bc_kind[side_y] == ORC_DIRICHLET) return 1;
    return is_solid(P, si, sj) ? 3 : 0;
}

/* Number of (cell, population) pairs whose replacement is itself unknown (0 = valid geometry). */
int64_t orc_obstacle_check(const orc_params* P)
{
    if (!P->solid || P->lattice != ORC_D2Q4) return 0;
    int64_t bad = 0;
    for (int64_t j = 0; j < P->ny; ++j)
        for (int64_t i = 0; i < P->nx; ++i) {
            if (P->solid[j * P->nx + i]) continue;
            for (int q = 0; q < 4; ++q) {
                if (pull_kind(P, i, j, q) != 3) continue;
                double su, sv;
                int m = obstacle_mirror(P, i, j, q, &su, &sv);
                int km = pull_kind(P, i, j, m);
                if (km == 2 || km == 3) ++bad;
            }
        }
    return bad;
}

/* Ghost distributions of each Dirichlet side: f^eq of the boundary state. */
static void ghost_tables(const orc_params* P, double ghost[4][16])
{
    int sides = P->lattice == ORC_D2Q4 ? 4 : (P->lattice == ORC_D2Q4S ? 0 : 2);
    for (int s = 0; s < sides; ++s) {
        double U[4];
        prim_to_cons_cell(P, P->bc_prim[s], U);
        feq_cell(P, U, ghost[s]);
    }
}

/* Scalar lattice: a Dirichlet side holds the linear profile u_b = prim[0] + prim[1] s,
 * s the centre coordinate (m + 1/2) dx of the ghost cell along that side (m may lie
 * outside the side at a corner: the profile is extended); the ghost is f^eq(u_b). */
static const double* profile_ghost(const orc_params* P, int side, int64_t m, double* buf)
{
    double ub = P->bc_prim[side][0] + P->bc_prim[side][1] * (((double)m + 0.5) * P->dx);
    feq_cell(P, &ub, buf);
    return buf;
}

/*
 * Streaming plus boundary conditions: f_q(x) = fs_q(x - c_q), then the
 * free-slip wall relations on wall rows (Section II.E).  fs and f are
 * [Q][K][ny][nx].  Returns 0, or a nonzero code if the parameters are invalid.
 */
int orc_stream(const orc_params* P, const double* fs, double* f)
{
    int err = orc_validate(P);
    if (err) return err;
    if (orc_obstacle_check(P)) return 10;
    const int64_t nx = P->nx, ny = P->ny, N = nx * ny;
    const int Q = nq(P), K = nk(P);
    double ghost[4][16];
    ghost_tables(P, ghost);
    const int is2d = two_d(P), scalar = P->lattice == ORC_D2Q4S;

#pragma omp parallel for schedule(static) num_threads(threads_of(P))
    for (int64_t j = 0; j < ny; ++j) {
        for (int64_t i = 0; i < nx; ++i) {
            const int64_t c = j * nx + i;
            if (P->solid && P->solid[c]) {                    /* inert solid cell */
                for (int q = 0; q < Q; ++q)
                    for (int k = 0; k < K; ++k) f[(q * K + k) * N + c] = fs[(q * K + k) * N + c];
                continue;
            }
            int wall_pop[4] = {0, 0, 0, 0};
            int solid_pop[4] = {0, 0, 0, 0};
            for (int q = 0; q < Q; ++q) {
                int sx = is2d ? SX2[q] : (Q == 3 ? SX13[q] : SX1[q]);
                int sy = is2d ? SY2[q] : 0;
                double gbuf[4];
                int64_t si = i - sx, sj = j - sy;
                int side_y = sj < 0 ? 2 : (sj >= ny ? 3 : -1);
                int side_x = si < 0 ? 0 : (si >= nx ? 1 : -1);
                const double* g = NULL;
                if (side_y >= 0 && P->bc_kind[side_y] == ORC_WALL) {
                    wall_pop[q] = 1;          /* set below from the wall relation */
                    continue;
                }
                if (side_y >= 0 && P->bc_kind[side_y] == ORC_WALL_HALFWAY) {
                    /* the mirror image of this population (sy reversed) leaving the
                     * horizontal neighbour on the wall row (x resolved as a pull source) */
                    const int m = 3 - q;
                    const double* gm = NULL;
                    if (side_x >= 0) {
                        int kind = P->bc_kind[side_x];
                        if (kind == ORC_DIRICHLET) gm = ghost[side_x];
                        else if (kind == ORC_PERIODIC) si = (si + nx) % nx;
                        else si = si < 0 ? 0 : nx - 1;
                    }
                    for (int k = 0; k < K; ++k) {
                        double sgn = (k == 2) ? -1.0 : 1.0;
                        f[(q * K + k) * N + c] = sgn * (gm ? gm[m * K + k] : fs[(m * K + k) * N + j * nx + si]);
                    }
                    continue;
                }
                if (side_x >= 0) {
                    int kind = P->bc_kind[side_x];
                    if (kind == ORC_DIRICHLET) g = scalar ? profile_ghost(P, side_x, sj, gbuf) : ghost[side_x];
                    else if (kind == ORC_PERIODIC) si = (si + nx) % nx;
                    else si = si < 0 ? 0 : nx - 1;              /* transmissive */
                }
                if (!g && side_y >= 0) {
                    int kind = P->bc_kind[side_y];
                    if (kind == ORC_DIRICHLET) g = scalar ? profile_ghost(P, side_y, si, gbuf) : ghost[side_y];
                    else if (kind == ORC_PERIODIC) sj = (sj + ny) % ny;
                    else sj = sj < 0 ? 0 : ny - 1;              /* transmissive */
                }
                if (!g && P->solid && P->solid[sj * nx + si]) {
                    solid_pop[q] = 1;         /* set below from the internal-wall relation */
                    continue;
                }
                for (int k = 0; k < K; ++k)
                    f[(q * K + k) * N + c] = g ? g[q * K + k] : fs[(q * K + k) * N + sj * nx + si];
            }
            /* Internal walls: an unknown population takes a known one of this cell. */
            for (int q = 0; q < Q; ++q) {
                if (!solid_pop[q]) continue;
                double sgn_u, sgn_v;
                int m = obstacle_mirror(P, i, j, q, &sgn_u, &sgn_v);
                for (int k = 0; k < K; ++k) {
                    double sgn = k == 1 ? sgn_u : (k == 2 ? sgn_v : 1.0);
                    f[(q * K + k) * N + c] = sgn * f[(m * K + k) * N + c];
                }
            }
            /* Free-slip wall (Section II.E).  Top wall: the incoming downward
             * populations f1, f2 (q = 0, 1) take f1 = f4, f2 = f3, negated for
             * the rho v field.  Bottom wall: f4 = f1, f3 = f2, negated for rho v. */
            if (wall_pop[0] || wall_pop[1]) {
                for (int k = 0; k < K; ++k) {
                    double sgn = (k == 2) ? -1.0 : 1.0;
                    f[(0 * K + k) * N + c] = sgn * f[(3 * K + k) * N + c];
                    f[(1 * K + k) * N + c] = sgn * f[(2 * K + k) * N + c];
                }
            }
            if (wall_pop[2] || wall_pop[3]) {
                for (int k = 0; k < K; ++k) {
                    double sgn = (k == 2) ? -1.0 : 1.0;
                    f[(3 * K + k) * N + c] = sgn * f[(0 * K + k) * N + c];
                    f[(2 * K + k) * N + c] = sgn * f[(1 * K + k) * N + c];
                }
            }
        }
    }
    return 0;
}

/*
 * Collision: moments, fluxes, equilibria, relaxation fs = (1-w) f + w f^eq.
 * Writes the moments of the streamed f to U (nullable).  Updates chk with the
 * physical-admissibility and sub-characteristic checks (nullable), tagging a
 * violation with `step`.
 */
void orc_collide(const orc_params* P, const double* f, double* fs, double* U, orc_check* chk, int64_t step)
{
    const int64_t N = P->nx * P->ny;
    const int Q = nq(P), K = nk(P);
    const double om = P->omega, om1 = 1.0 - P->omega;
    int64_t bad = 0, sub = 0;
    double lmax = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : bad, sub) reduction(max : lmax) \
    num_threads(threads_of(P))
    for (int64_t c = 0; c < N; ++c) {
        double u[4], feq[16];
        for (int k = 0; k < K; ++k) {
            double s = f[(0 * K + k) * N + c];
            for (int q = 1; q < Q; ++q) s += f[(q * K + k) * N + c];
            u[k] = s;
            if (U) U[k * N + c] = s;
        }
        feq_cell(P, u, feq);
        const int inert = P->solid && P->solid[c];          /* solid cells are carried unchanged */
        for (int q = 0; q < Q; ++q)
            for (int k = 0; k < K; ++k) {
                int64_t idx = (q * K + k) * N + c;
                fs[idx] = inert ? f[idx] : om1 * f[idx] + om * feq[q * K + k];
            }
        const int scalar = P->lattice == ORC_D2Q4S;          /* a scalar has no density or pressure */
        double p = scalar ? 1.0 : pressure(P, u);
        int finite = 1;
        for (int k = 0; k < K; ++k) finite &= isfinite(u[k]);
        if (!finite || (!scalar && (!(u[0] > 0.0) || !(p > 0.0)))) {
            ++bad;
        } else {
            double l = lambda_local(P, u, p);
            if (l > lmax) lmax = l;
            if (l > P->lambda) ++sub;
        }
    }
    if (chk) {
        if (lmax > chk->max_lambda_local) chk->max_lambda_local = lmax;
        if (bad || sub) {
            if (chk->first_bad_step < 0) chk->first_bad_step = step;
            chk->n_nonphysical = bad;
            chk->n_subchar = sub;
        }
    }
}

/*
 * Advance fs (in place) by nsteps steps; work is scratch of the same size.
 * The step counter of the checks starts at step0 + 1.  Returns 0 or an error code.
 */
int orc_run(const orc_params* P, double* fs, double* work, int64_t nsteps, int64_t step0, orc_check* chk)
{
    int err = orc_validate(P);
    if (err) return err;
    for (int64_t n = 0; n < nsteps; ++n) {
        orc_stream(P, fs, work);
        orc_collide(P, work, fs, NULL, chk, step0 + n + 1);
    }
    return 0;
}

/* Largest local bound over the cells' moments U (physical cells only) and the
 * Dirichlet states of the sides. */
static double max_bound(const orc_params* P, const double* U)
{
    const int64_t N = P->nx * P->ny;
    const int K = nk(P);
    double m = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        double u[4];
        for (int k = 0; k < K; ++k) u[k] = U[k * N + c];
        double p = pressure(P, u);
        if (!(u[0] > 0.0) || !(p > 0.0) || !isfinite(p)) continue;
        double l = lambda_local(P, u, p);
        if (l > m) m = l;
    }
    int sides = two_d(P) ? 4 : 2;
    for (int s = 0; s < sides; ++s) {
        if (P->bc_kind[s] != ORC_DIRICHLET) continue;
        double u[4];
        prim_to_cons_cell(P, P->bc_prim[s], u);
        double l = lambda_local(P, u, pressure(P, u));
        if (l > m) m = l;
    }
    return m;
}

/*
 * Adaptive lattice speed: the sub-characteristic choice of Section II.C (the bound
 * of Section II.D in 2-D) taken anew every step.  The post-collision distributions
 * carry the lambda of their equilibria, and streaming them one cell advances the
 * solution by dt = dx / (that lambda) (at omega = 1 the update is Lax-Friedrichs
 * with that lambda).  So each step streams with the lambda of the current state
 * (P->lambda for the first; Dirichlet ghosts built with it too), advancing the time
 * by dx / lambda, and its collision builds the equilibria with the next lambda:
 * safety times the largest local bound over the moments of the state before the
 * step and the Dirichlet states (one step behind, so that the GPU can take the max
 * in the same pass).  With t_final > 0 the collision whose state would stream past
 * t_final takes lambda = dx / (t_final - t) instead (larger, hence admissible), and
 * the run stops after that stream, at t_final exactly.  lam_out (nullable, nsteps
 * entries) receives each step's stream lambda; *lam_next the lambda of the final
 * state.  Returns the number of steps taken (negative on invalid parameters, or if
 * the first stream alone passes t_final); *t is the time reached.  Euler lattices,
 * no obstacles.
 */
int64_t orc_run_adaptive(const orc_params* P, double* fs, double* work, int64_t nsteps, double dx, double safety,
                         double t_final, double* lam_out, double* t, double* lam_next)
{
    if (orc_validate(P) || P->lattice == ORC_D2Q4S || P->solid || !(dx > 0.0) || !(safety >= 1.0)) return -1;
    if (t_final > 0.0 && dx / P->lambda > t_final) return -3;
    const int64_t N = P->nx * P->ny;
    double* U = (double*)malloc((size_t)nk(P) * (size_t)N * sizeof(double));
    if (!U) return -2;
    orc_params Qs = *P, Qc = *P;
    orc_moments(P, fs, U);
    double bound = max_bound(P, U), tt = 0.0, lam_cur = P->lambda;
    int last = 0;
    int64_t n = 0;
    while (n < nsteps) {
        double t_next = last ? t_final : tt + dx / lam_cur;
        double lam_new = safety * bound;
        int next_last = 0;
        if (!last && t_final > 0.0 && t_next + dx / lam_new >= t_final) {
            lam_new = dx / (t_final - t_next);
            next_last = 1;
        }
        Qs.lambda = lam_cur;
        Qc.lambda = lam_new;
        orc_stream(&Qs, fs, work);
        orc_collide(&Qc, work, fs, U, NULL, n + 1);
        if (lam_out) lam_out[n] = lam_cur;
        tt = t_next;
        lam_cur = lam_new;
        bound = max_bound(P, U);
        ++n;
        if (last) break;
        last = next_last;
    }
    free(U);
    *t = tt;
    *lam_next = lam_cur;
    return n;
}

/* FP64 totals sum_cells U_k * cell volume (cell volume = dx for 1-D, dx^2 for 2-D). */
void orc_totals(const orc_params* P, const double* fs, double cell_volume, double* totals)
{
    const int64_t N = P->nx * P->ny;
    const int Q = nq(P), K = nk(P);
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int64_t c = 0; c < N; ++c) {
            double u = fs[(0 * K + k) * N + c];
            for (int q = 1; q < Q; ++q) u += fs[(q * K + k) * N + c];
            s += u;
        }
        totals[k] = s * cell_volume;
    }
}

/* Boundary balance of the next step (D2Q4 and the scalar D2Q4, no internal walls): streaming
 * (Section II.D) moves fs_q(y) to y + c_q.  A population whose destination lies beyond a non-periodic
 * side leaves the domain (outflow); a cell whose pull source x - c_q lies beyond one receives what the
 * side condition gives it, the streamed f_q(x) of orc_stream with the wall relations of Section II.E
 * (inflow).  Per conserved field, both sums times cell_volume; `work` holds the streamed f
 * ([Q][K][ny][nx], like fs).  Since the collision keeps the moments, the totals after one step are
 * the totals before plus inflow minus outflow.  Returns 0, or the code of orc_stream, or 11 for
 * another lattice or internal walls. */
int orc_boundary_flux(const orc_params* P, const double* fs, double* work, double cell_volume, double* inflow,
                      double* outflow)
{
    if (!two_d(P) || P->solid) return 11;
    int err = orc_stream(P, fs, work);
    if (err) return err;
    const int64_t nx = P->nx, ny = P->ny, N = nx * ny;
    const int Q = nq(P), K = nk(P);
    const int px = P->bc_kind[0] == ORC_PERIODIC, py = P->bc_kind[2] == ORC_PERIODIC;
    for (int k = 0; k < K; ++k) {
        double in = 0.0, out = 0.0;
        for (int q = 0; q < Q; ++q)
            for (int64_t j = 0; j < ny; ++j)
                for (int64_t i = 0; i < nx; ++i) {
                    const int64_t c = j * nx + i;
                    const int64_t si = i - SX2[q], sj = j - SY2[q], di = i + SX2[q], dj = j + SY2[q];
                    if ((!px && (si < 0 || si >= nx)) || (!py && (sj < 0 || sj >= ny)))
                        in += work[(q * K + k) * N + c];
                    if ((!px && (di < 0 || di >= nx)) || (!py && (dj < 0 || dj >= ny)))
                        out += fs[(q * K + k) * N + c];
                }
        inflow[k] = in * cell_volume;
        outflow[k] = out * cell_volume;
    }
    return 0;
}

int orc_max_threads(void) { return omp_get_max_threads(); }

/* ====================================================================== adjoint
 *
 * Discrete adjoint of the D2Q4 step on a fully periodic domain (not in the
 * paper; the transpose of the step defined above, used for gradients).
 *
 * Forward step n -> n+1:  f = S fs^n,  U = M f,  fs^{n+1} = (1-w) f + w E(U),
 * with S the periodic shift f_q(x) = fs_q(x - c_q), M the moment sum over q and
 * E the equilibria.  With gbar = dL/dfs^{n+1}:
 *   fbar_{q,k} = (1-w) gbar_{q,k} + w ubar_k,   ubar = J_E(U)^T gbar,
 *   dL/dfs^n_q(x) = fbar_q(x + c_q)   (S^T: the shift back along c_q).
 * J_E^T gbar = a/4 + c A_F^T bx + c A_G^T by with a_k = sum_q gbar_{q,k},
 * bx_k = sum_q sx_q gbar_{q,k}, by_k = sum_q sy_q gbar_{q,k}, c = 1/(4 lambda),
 * and A_F = dF/dU, A_G = dG/dU the Euler flux Jacobians of the ideal gas.
 */

/* ubar_k = sum_{q,k'} gq[q*4+k'] dE_{q,k'}/dU_k at state U. */
static void equilibrium_vjp_2d(const orc_params* P, const double* U, const double* gq, double* ubar)
{
    const double g = P->gamma, gm1 = P->gamma - 1.0;
    const double rho = U[0], mx = U[1], my = U[2], en = U[3];
    const double u = mx / rho, v = my / rho;
    const double p = gm1 * (en - 0.5 * (mx * u + my * v));
    const double H = (en + p) / rho;
    const double q2h = 0.5 * gm1 * (u * u + v * v);
    /* dF[r][k] = dF_r / dU_k, dG likewise */
    const double dF[4][4] = {{0.0, 1.0, 0.0, 0.0},
                             {q2h - u * u, (3.0 - g) * u, -gm1 * v, gm1},
                             {-u * v, v, u, 0.0},
                             {u * (q2h - H), H - gm1 * u * u, -gm1 * u * v, g * u}};
    const double dG[4][4] = {{0.0, 0.0, 1.0, 0.0},
                             {-u * v, v, u, 0.0},
                             {q2h - v * v, -gm1 * u, (3.0 - g) * v, gm1},
                             {v * (q2h - H), -gm1 * u * v, H - gm1 * v * v, g * v}};
    const double c = 1.0 / (4.0 * P->lambda);
    double a[4], bx[4], by[4];
    for (int k = 0; k < 4; ++k) {
        a[k] = bx[k] = by[k] = 0.0;
        for (int q = 0; q < 4; ++q) {
            a[k] += gq[q * 4 + k];
            bx[k] += SX2[q] * gq[q * 4 + k];
            by[k] += SY2[q] * gq[q * 4 + k];
        }
    }
    for (int k = 0; k < 4; ++k) {
        double sf = 0.0, sg = 0.0;
        for (int r = 0; r < 4; ++r) {
            sf += dF[r][k] * bx[r];
            sg += dG[r][k] * by[r];
        }
        ubar[k] = 0.25 * a[k] + c * sf + c * sg;
    }
}

static int adjoint_supported(const orc_params* P)
{
    if (orc_validate(P)) return 0;
    if (P->lattice != ORC_D2Q4) return 0;
    for (int s = 0; s < 4; ++s)
        if (P->bc_kind[s] != ORC_PERIODIC) return 0;
    return 1;
}

/* One backward step: gout = dL/dfs^n from gin = dL/dfs^{n+1} and U_next =
 * the moments of step n+1 (the U the forward collision used). Returns 0, or
 * nonzero if the problem is not a periodic D2Q4 one. */
int orc_adjoint_step(const orc_params* P, const double* U_next, const double* gin, double* gout)
{
    if (!adjoint_supported(P)) return 1;
    const int64_t nx = P->nx, ny = P->ny, N = nx * ny;
    const double om = P->omega, om1 = 1.0 - P->omega;
#pragma omp parallel for schedule(static) num_threads(threads_of(P))
    for (int64_t j = 0; j < ny; ++j) {
        for (int64_t i = 0; i < nx; ++i) {
            const int64_t c = j * nx + i;
            double gq[16], U[4], ubar[4];
            for (int n = 0; n < 16; ++n) gq[n] = gin[n * N + c];
            for (int k = 0; k < 4; ++k) U[k] = U_next[k * N + c];
            equilibrium_vjp_2d(P, U, gq, ubar);
            for (int q = 0; q < 4; ++q) {
                const int64_t ti = (i - SX2[q] + nx) % nx, tj = (j - SY2[q] + ny) % ny;
                for (int k = 0; k < 4; ++k)
                    gout[(q * 4 + k) * N + tj * nx + ti] = om1 * gq[q * 4 + k] + om * ubar[k];
            }
        }
    }
    return 0;
}

/* Gradient with respect to the initial conserved state: fs^0 = E(U0), so
 * dL/dU0 = J_E(U0)^T dL/dfs^0, per cell. Returns 0 or nonzero as above. */
int orc_vjp_equilibrium(const orc_params* P, const double* U0, const double* g0, double* grad)
{
    if (!adjoint_supported(P)) return 1;
    const int64_t N = P->nx * P->ny;
    for (int64_t c = 0; c < N; ++c) {
        double gq[16], U[4], ubar[4];
        for (int n = 0; n < 16; ++n) gq[n] = g0[n * N + c];
        for (int k = 0; k < 4; ++k) U[k] = U0[k * N + c];
        equilibrium_vjp_2d(P, U, gq, ubar);
        for (int k = 0; k < 4; ++k) grad[k * N + c] = ubar[k];
    }
    return 0;
}
