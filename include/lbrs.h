/*
 * lbrs.h -- C ABI of the GB300 Lattice Boltzmann Relaxation Scheme (LBRS) solver.
 *
 * The method (Raghurama Rao, Deshmukh, Kotnala, "A Lattice Boltzmann
 * Relaxation Scheme for Inviscid Compressible Flows"):
 *
 *   distributions f_q, one per lattice velocity c_q and conserved field k;
 *   one time step = stream every population one lattice spacing along its
 *   velocity (exact hopping, lambda dt = dx), apply the boundary conditions,
 *   take the moments U_k = sum_q f_{q,k}, evaluate the Euler fluxes with the
 *   ideal-gas pressure, build the algebraic equilibria and relax:
 *       f*_q = (1 - omega) f_q + omega f^eq_q(U)      (discrete LBRS update, Section II.A)
 *
 *   D1Q2 (Section II.C): velocities (-lambda, +lambda), fields (rho, rho u, rho E),
 *       f^eq_{1,2} = U/2 -/+ G(U)/(2 lambda).
 *   D2Q4 (Section II.D): diagonal velocities f1 (-,-), f2 (+,-), f3 (+,+), f4 (-,+)
 *       times lambda, fields (rho, rho u, rho v, rho E),
 *       f^eq_q = U/4 + sx_q F(U)/(4 lambda) + sy_q G(U)/(4 lambda).
 *   Free-slip wall (Section II.E): the populations entering through a wall
 *       are replaced by specular reflection of the outgoing ones, negated for
 *       the wall-normal momentum field.
 *
 * Conventions
 *   Layout.    Distributions are structure-of-arrays f[q][k][j][i] (i fastest),
 *              q in the paper's order, Q = 2, 3 or 4, K = 3 or 4, N = nx * ny.
 *              Field arrays are [k][j][i].  1-D problems have ny = 1.
 *              Cells are cell-centred; dx = dy (exact hopping on the diagonals).
 *   Memory.    The caller owns every buffer.  Device memory for the solver
 *              state is ONE caller-provided workspace (e.g. a torch tensor) of
 *              lbrs_workspace_size() bytes, 256-byte aligned, which must
 *              outlive the context.  The library itself never allocates device
 *              memory; it allocates its host-side context and, on first use
 *              of a multi-step call, one private capture stream and CUDA
 *              graphs, released by lbrs_destroy.
 *   Streams.   All device work is enqueued on cfg.cuda_stream (0 = legacy
 *              default stream).  Calls are asynchronous unless they return
 *              data to host memory.  One context per stream; a context is not
 *              thread-safe.
 *   Errors.    Every call returns an lbrs_status; nothing aborts, traps or
 *              throws across the ABI.  LBRS_EINVAL leaves the state unchanged.
 *              lbrs_last_error() gives a one-line description of the last
 *              failure on a context.
 */
#ifndef LBRS_H
#define LBRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBRS_ABI_VERSION 1

typedef struct lbrs_ctx lbrs_ctx;

typedef enum {
    LBRS_OK = 0,
    LBRS_EINVAL = 1,    /* invalid argument or configuration */
    LBRS_ENOMEM = 2,    /* workspace too small */
    LBRS_ECUDA = 3,     /* a CUDA runtime call failed (see lbrs_last_error) */
    LBRS_ENONPHYS = 4,  /* a cell has rho <= 0, p <= 0 or a non-finite value */
    LBRS_ESUBCHAR = 5,  /* a cell violates lambda >= local wave-speed bound (Sections II.A, II.D) */
    LBRS_ETIMEOUT = 6,  /* a bounded device wait gave up (lbrs_sync; the state is then not valid) */
    LBRS_ESTATE = 7     /* call out of order (e.g. stepping before a state was set) */
} lbrs_status;

/* LBRS_D1Q3 adds a rest particle (Section II.C): velocities (-lambda, 0, +lambda),
 * f^eq = (U/3 - G/(2 lambda), U/3, U/3 + G/(2 lambda)).  Its Chapman-Enskog
 * diffusion dt (1/omega - 1/2)(2 lambda^2/3 - c^2) stays positive only for
 * wave speeds c below sqrt(2/3) lambda: the diagnostics' local bound for D1Q3 is
 * sqrt(3/2)(|u| + a). */
/* LBRS_D2Q4S is the D2Q4 lattice for one scalar conserved variable u with the
 * fluxes of the 2-D inviscid Burgers law of Section III, g1 = u^2/2, g2 = u:
 * f^eq_q = u/4 + sx_q g1/(4 lambda) + sy_q g2/(4 lambda) (Section II.D).  Fields
 * are [1][ny][nx]; LBRS_F64 or LBRS_F32 only; no walls, obstacles or adjoint.  A
 * Dirichlet side holds the linear profile u_b = prim[0] + prim[1] s, s = (m + 1/2) dx
 * the centre coordinate of the ghost cell along that side (m its index, extended
 * past the side's ends at corners).  The diagnostics report min u as min_rho, 1 as
 * min_p, and the local bound |u| + 1 (f^eq_q non-decreasing in u for every q iff
 * lambda >= |g1'| + |g2'|); only non-finite values count as non-physical. */
typedef enum { LBRS_D1Q2 = 0, LBRS_D2Q4 = 1, LBRS_D1Q3 = 2, LBRS_D2Q4S = 3 } lbrs_lattice;

/* Storage and arithmetic precision of the distributions.
 *   LBRS_F64     FP64 storage and arithmetic (the parity path);
 *   LBRS_F32     FP32 storage and arithmetic;
 *   LBRS_F16NEQ  D2Q4 only: per cell the moments U in FP32 plus the
 *                post-collision non-equilibrium parts f*_q - f^eq_q(U) of
 *                populations 1-3 in FP16 (per-field power-of-two scale; the
 *                fourth follows from their zero sum), FP32 arithmetic.
 *                40 instead of 64 bytes per cell.  Not differentiable (the
 *                adjoint calls reject it); lbrs_get/set_distributions move the
 *                raw buffer: U [4][N] FP32, g [3][4][N] FP16, 4 FP32 scales
 *                (40 N + 16 bytes);
 *   LBRS_F32U    D2Q4 with omega = 1 exactly: the post-collision state is then
 *                f^eq(U) (Section II.A with omega = 1), so only the moments U
 *                are stored (FP32, 16 bytes per cell) and each step rebuilds
 *                the pulled populations from the neighbours' moments.  Same
 *                restrictions as LBRS_F16NEQ; raw buffer U [4][N] FP32. */
typedef enum { LBRS_F64 = 0, LBRS_F32 = 1, LBRS_F16NEQ = 2, LBRS_F32U = 3 } lbrs_precision;

/* Boundary kinds.  The paper defines only the free-slip wall (Section II.E);
 * the others are this library's readings:
 *   PERIODIC     the pull source wraps around (both sides of an axis must be periodic);
 *   TRANSMISSIVE the pull source index is clamped into the domain (zero-order extrapolation);
 *   DIRICHLET    populations entering from outside are f^eq of the given state;
 *   WALL         free-slip wall on a y side (D2Q4 only), applied on the wall row;
 *   CUT          a y side (D2Q4; LBRS_F64, LBRS_F32 or LBRS_F32U) where this context's rows
 *                meet a neighbouring context's rows: the context is one y-slab of a larger
 *                grid (see lbrs_halo_export below);
 *   WALL_HALFWAY the halfway alternative of the free-slip wall (a y side of D2Q4 in LBRS_F64
 *                or LBRS_F32; not with internal walls): the wall lies half a cell beyond the
 *                wall row, and a population that would enter through it takes, by specular
 *                reflection there, the post-collision value of its mirror image leaving the
 *                horizontal neighbour on the wall row, rho v negated -- bottom:
 *                f3(i, 0) = f*2(i - 1, 0), f4(i, 0) = f*1(i + 1, 0); top:
 *                f1(i, ny-1) = f*4(i + 1, ny-1), f2(i, ny-1) = f*3(i - 1, ny-1); the neighbour's
 *                x is resolved like a pull source.  A grid with it on both y sides is the lower
 *                half of a periodic grid of twice the height holding its mirror image. */
typedef enum {
    LBRS_BC_PERIODIC = 0,
    LBRS_BC_TRANSMISSIVE = 1,
    LBRS_BC_DIRICHLET = 2,
    LBRS_BC_WALL = 3,
    LBRS_BC_CUT = 4,
    LBRS_BC_WALL_HALFWAY = 5
} lbrs_bc_kind;

/* Kind of the fields passed to lbrs_set_state. */
typedef enum { LBRS_CONSERVED = 0, LBRS_PRIMITIVE = 1 } lbrs_state_kind;

typedef struct {
    int32_t kind;       /* lbrs_bc_kind */
    int32_t halo_rows;  /* CUT only: ghost rows H stored beyond the side, 1..64 (0: 2); ignored otherwise */
    double prim[4];     /* DIRICHLET state: (rho, u, v, p) in 2-D, (rho, u, p) in 1-D */
} lbrs_bc;

typedef struct {
    uint32_t struct_size;   /* = sizeof(lbrs_config), for ABI growth */
    int32_t lattice;        /* lbrs_lattice */
    int32_t precision;      /* lbrs_precision */
    int32_t diag_every;     /* > 0: check the state every diag_every steps on the device (see lbrs_sync); 0: off */
    int64_t nx, ny;         /* cells; ny = 1 for D1Q2 */
    double gamma;           /* ratio of specific heats, > 1 */
    double lambda;          /* lattice speed, > 0; dt = dx / lambda */
    double omega;           /* relaxation parameter dt/epsilon, in (0, 2) (Section II.B) */
    double dx;              /* lattice spacing, > 0 (cell volume of the totals) */
    lbrs_bc bc[4];          /* x-lo, x-hi, y-lo, y-hi; 1-D uses the first two */
    void* cuda_stream;      /* cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream */
} lbrs_config;

/* Global diagnostics of the current state, reduced in FP64 in a fixed order
 * (bitwise reproducible run to run). */
typedef struct {
    double totals[4];          /* sum over cells of U_k * dx^d (d = 1 or 2); K entries used */
    double min_rho;            /* minimum density */
    double min_p;              /* minimum pressure */
    double max_lambda_local;   /* max |u| + a (1-D) or max(|u+v|,|u-v|) + sqrt(2) a (2-D), Sections II.C, II.D */
    double reserved;
    int64_t n_nonphysical;     /* cells with rho <= 0, p <= 0 or a non-finite moment */
    int64_t n_subchar;         /* cells whose local bound exceeds lambda */
} lbrs_diag;

/* Library ABI version (LBRS_ABI_VERSION of the build). */
int lbrs_abi_version(void);

/* Bounds-checked build (not a method of the paper: the library's own check of its
 * index arithmetic, where no memory sanitizer can run).  The library built with
 * -DLBRS_DEBUG (liblbrs_debug.so, `python -m paper_1504_07034_gb300.build --debug`)
 * checks the indices of its kernels' global and shared-memory accesses; an index
 * outside its buffer is replaced by 0 (the access stays inside the buffer, its value
 * is wrong) and the first such event of each kernel unit is recorded.
 * lbrs_debug_build: 1 for that build, 0 for the release build (which records
 * nothing).  lbrs_debug_check: after the caller has synchronised the device, writes
 * the first record, (site << 40) | index, to *first (0 if none), clears the records
 * and returns LBRS_ECUDA if there was one (LBRS_EINVAL for a NULL pointer); in
 * that build lbrs_sync also reports a record as LBRS_ECUDA.  Device-wide, not per
 * context: records of concurrent contexts are not told apart. */
int lbrs_debug_build(void);
lbrs_status lbrs_debug_check(uint64_t* first);

/* Failure-detection self-test (not a method of the paper).  Every device wait of the
 * library is bounded: the tile kernels' waits for their tensor copies give up after a
 * fixed number of polls, raise a flag in the workspace and leave their tile unwritten,
 * and lbrs_sync reports the flag as LBRS_ETIMEOUT; setting a state clears it.  This call
 * enqueues on the context's stream one block whose bounded wait, on an mbarrier that
 * nothing completes, runs out and raises the same flag, so that the reporting path can
 * be exercised without a fault.  The distributions are not touched. */
lbrs_status lbrs_selftest_wait_timeout(lbrs_ctx* ctx);

/* Arithmetic self-test (not a method of the paper).  The FP32 kernels form the
 * velocities u = (rho u) / rho with one reciprocal of rho: the hardware's approximate
 * reciprocal refined by one Newton-Raphson step for 1/x, r = r0 + r0 (1 - x r0).  This
 * call writes that reciprocal of x[i] to r[i], i < n, so that its error can be checked
 * against the exact quotient.  x and r: device buffers of n floats (caller-owned, not
 * aliased); the work is enqueued on cuda_stream (a cudaStream_t, NULL for the legacy
 * default stream) and not waited for.  LBRS_EINVAL for n < 0 or a NULL buffer with
 * n > 0; LBRS_ECUDA if the launch fails. */
lbrs_status lbrs_selftest_rcp_f32(const float* x, float* r, int64_t n, void* cuda_stream);

/* Human-readable name of a status code. Never NULL. */
const char* lbrs_status_string(lbrs_status s);

/* Bytes of device workspace a configuration needs: two distribution buffers
 * (ping-pong), boundary tables and reduction scratch.  EINVAL on a bad config. */
lbrs_status lbrs_workspace_size(const lbrs_config* cfg, size_t* bytes);

/* Create a solver context on the caller's workspace.  Validates cfg (EINVAL),
 * checks bytes >= lbrs_workspace_size (ENOMEM), computes the Dirichlet ghost
 * tables on the device.  *out receives the context; no state is set yet. */
lbrs_status lbrs_create(const lbrs_config* cfg, void* d_workspace, size_t bytes, lbrs_ctx** out);

/* Release a context (host memory, graphs, private stream).  NULL is a no-op.
 * Does not free the workspace. */
void lbrs_destroy(lbrs_ctx* ctx);

/* Set the state at step 0: f = f^eq(U0) (initialisation, Section II.A).
 *   W        K fields [k][ny][nx]; conserved (rho, rho u, [rho v,] rho E) or primitive
 *            (rho, u, [v,] p) according to `kind`;
 *   on_device nonzero if W is device memory, zero for host memory (copied on the stream
 *            through the idle half of the workspace);
 *   dtype    LBRS_F64 or LBRS_F32: element type of W.
 * The conversion and f^eq are computed in FP64 and rounded to the storage precision. */
lbrs_status lbrs_set_state(lbrs_ctx* ctx, const void* W, int on_device, int dtype, int kind);

/* Enqueue n >= 0 time steps (stream, boundary conditions, moments, fluxes,
 * equilibria, relaxation; discrete LBRS update, Sections II.A and II.D).
 * Asynchronous.  ESTATE if no state was set.  D2Q4 in LBRS_F32 advances several
 * steps per read and write of the state, bit-identical to single steps: where
 * nx % 4 == 0 and the grid has no internal or halfway walls, three steps per launch
 * (a group of four as 2 + 2), else two, an odd remainder one single step; the
 * multi-step kernels fetch their tiles by tensor copies with bounded waits (see
 * LBRS_ETIMEOUT).  LBRS_F32U and the scalar D2Q4S in LBRS_F32 advance pairs of steps in
 * one launch.  D1Q2 and D1Q3 in
 * LBRS_F32 with both ends transmissive or both periodic advance up to 32 steps per
 * launch in shared memory (the batched tubes' kernel as a tube of one), bit-identical to
 * single steps. */
lbrs_status lbrs_step(lbrs_ctx* ctx, int64_t n);

/* Adaptive lattice speed (D2Q4, LBRS_F64 or LBRS_F32, no internal walls): the
 * sub-characteristic choice of Section II.C with the bound of Section II.D, taken
 * anew every step.  Distributions carry the lambda of their equilibria and streaming
 * them one cell advances the solution by dt = dx / that lambda; so each step streams
 * with the current state's lambda (Dirichlet ghosts rebuilt with it) and collides
 * with the next one, safety times the largest local bound max(|u+v|, |u-v|) +
 * sqrt(2) a over the moments of the state before the step and the Dirichlet states.
 * The maximum over the cells is taken inside the step kernel (for the step after);
 * one small kernel per step turns it into lambda and the clock.  The first call after
 * a state was set starts a run at t = 0 with the configured lambda (whose first step
 * must not pass t_final: EINVAL).  With t_final > 0, the collision whose state would
 * stream past t_final takes lambda = dx / (t_final - t), so the run ends exactly at
 * t_final; steps enqueued after that keep the state unchanged (keep t_final fixed
 * over one run).  n steps are enqueued asynchronously (2 launches each).  After an
 * adaptive step, lbrs_step returns ESTATE until a state is set again (the ghosts
 * return to the configured lambda); lbrs_diagnostics compares the bounds with the
 * configured lambda.  safety >= 1, t_final >= 0 (0: no end). */
lbrs_status lbrs_step_adaptive(lbrs_ctx* ctx, int64_t n, double safety, double t_final);

/* The adaptive run's time reached, the lambda of the current distributions, the
 * adaptive steps taken and whether t_final was reached; synchronises. */
lbrs_status lbrs_adaptive_state(lbrs_ctx* ctx, double* t, double* lambda, int64_t* steps, int* done);

/* Wait for the context's stream; reports a CUDA error raised by earlier work,
 * and LBRS_ETIMEOUT if a tile copy of a multi-step kernel did not arrive within
 * its bounded wait (the blocks concerned left their tiles unwritten; setting a
 * state clears the flag).
 * With cfg.diag_every > 0, lbrs_step runs the FP64 diagnostics reduction of
 * lbrs_diagnostics on the device after every diag_every-th step and records
 * the first step at which a cell was non-physical or exceeded the lattice
 * speed bound (Sections II.A, II.D); lbrs_sync then returns LBRS_ENONPHYS or
 * LBRS_ESUBCHAR from that step on (the state is left as computed, for
 * inspection) and lbrs_first_bad_step gives the step.  Setting a state clears
 * the record. */
lbrs_status lbrs_sync(lbrs_ctx* ctx);

/* First step flagged by the periodic device checks (-1 if none); synchronises. */
lbrs_status lbrs_first_bad_step(lbrs_ctx* ctx, int64_t* step);

/* Conserved moments U_k = sum_q f_{q,k} of the current state (moment relations,
 * Section II), summed in FP64 in q order and written as `dtype` to U_out [K][ny][nx].
 * Host output (on_device == 0) synchronises the stream before returning. */
lbrs_status lbrs_moments(lbrs_ctx* ctx, void* U_out, int on_device, int dtype);

/* FP64 diagnostics of the current state (see lbrs_diag); synchronises.
 * Returns ENONPHYS if any cell is non-physical, else ESUBCHAR if any cell
 * violates the sub-characteristic bound, else OK; *out is filled in every case. */
lbrs_status lbrs_diagnostics(lbrs_ctx* ctx, lbrs_diag* out);

/* Boundary balance of the next step (D2Q4, F64 or F32 distributions; Section II.D's
 * streaming with the side conditions of Section II.E and the readings for the other
 * sides): FP64 sums, per conserved field and times the cell volume dx^2, of the
 * populations the next step brings into the domain -- those of side cells whose pull
 * source x - c_q lies beyond a non-periodic side, with the values the step gives them
 * (a Dirichlet ghost, the clamped cell's population, a wall relation) -- (inflow) and
 * of the current post-collision populations it takes out -- those of side cells whose
 * destination x + c_q lies beyond a non-periodic side -- (outflow).  Every other
 * population stays inside and the collision keeps the moments, so after one lbrs_step
 * the totals of lbrs_diagnostics equal the current totals plus inflow minus outflow,
 * up to rounding.  Bitwise reproducible (one block, fixed order).  Synchronises the
 * stream.  inflow, outflow: host arrays of 4 doubles.  LBRS_EINVAL for NULL arrays,
 * another lattice or form (F16NEQ, F32U), internal walls or cut sides; LBRS_ESTATE
 * without a state or after adaptive steps. */
lbrs_status lbrs_boundary_flux(lbrs_ctx* ctx, double inflow[4], double outflow[4]);

/* The same diagnostics for callers that cannot allocate device memory: no
 * context, no workspace, and no cudaMalloc/cudaFree or allocating library call.
 * The paper has no counterpart; it exists because some callers cannot provide
 * scratch memory -- loops that must not stall on the implicit device
 * synchronisation of cudaMalloc/cudaFree, and processes whose device memory is
 * fully held by another allocator (for instance a framework's caching pool).
 *   cfg   the configuration the distributions belong to (lattice, precision,
 *         nx, ny, gamma, lambda, dx are used; cuda_stream is the stream).
 *         Accepted: LBRS_D1Q2, LBRS_D1Q3 and LBRS_D2Q4 in LBRS_F64 or LBRS_F32;
 *         LBRS_D2Q4S, LBRS_F16NEQ and LBRS_F32U get LBRS_EINVAL;
 *   d_fs  device distributions f[q][k][j][i] in cfg->precision, e.g. from
 *         lbrs_get_distributions;
 *   out   host struct, filled as by lbrs_diagnostics (same status rules).
 * Scratch: a static device array of 320.1 KiB inside the library, held on every
 * GPU that loads the library until the process exits.  Grids of more than
 * 33,554,432 cells are rejected with LBRS_EINVAL.  The first call on each
 * device (made while that device is current) looks up the array's device
 * address with cudaGetSymbolAddress and keeps it for the life of the process's
 * context on that device (a cudaDeviceReset invalidates it); make that first
 * call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU race.  The call reads the result back to host memory and
 * synchronises cfg->cuda_stream before returning. */
lbrs_status lbrs_diagnostics_noalloc(const lbrs_config* cfg, const void* d_fs, lbrs_diag* out);

/* Copy the raw distributions f[q][k][j][i] (storage precision) out of / into
 * the context, e.g. for checkpoints.  Host transfers synchronise.  set also
 * sets the step counter. */
lbrs_status lbrs_get_distributions(lbrs_ctx* ctx, void* dst, int on_device);
lbrs_status lbrs_set_distributions(lbrs_ctx* ctx, const void* src, int on_device, int64_t step);

/* Checkpoints: a self-describing copy of the state, a 256-byte header (magic
 * "LBRSCKP1", version 1; lattice, precision, grid, step, lambda, omega, gamma, dx,
 * boundary kinds and states; the size of the distributions) followed by the raw
 * distributions (the FP16 form's scales included).  lbrs_checkpoint_size gives the
 * blob's bytes; save writes it to host or device memory and synchronises; load
 * checks the header against the context's configuration (EINVAL on any difference
 * or a foreign blob), restores the distributions and the step counter, and clears
 * the record of the periodic checks (as setting a state does).  Resuming from a
 * checkpoint is bit-identical to an uninterrupted run.  The state of an adaptive-
 * lambda run is not covered (EINVAL). */
lbrs_status lbrs_checkpoint_size(const lbrs_ctx* ctx, size_t* bytes);
lbrs_status lbrs_checkpoint_save(lbrs_ctx* ctx, void* dst, int on_device);
lbrs_status lbrs_checkpoint_load(lbrs_ctx* ctx, const void* src, int on_device);

/* Lattice-aligned internal walls (obstacles such as the forward-facing step and the
 * backward-facing step of the shock-diffraction problem, Section III), D2Q4 in
 * LBRS_F64 or LBRS_F32.  d_solid: device mask [ny][nx] of uint8, nonzero = solid
 * cell; owned by the caller, read at every step until replaced, so it must outlive
 * the context or a later call with NULL (which removes the walls).  Solid cells are
 * inert (their distributions are carried unchanged).  In a fluid cell, a population
 * pulled from a solid cell takes the free-slip reflection of Section II.E, applied
 * to the obstacle face: the population mirrored in x (rho u negated) when only the
 * axis neighbour (i - sx, j) is solid, mirrored in y (rho v negated) when only
 * (i, j - sy) is, the opposite one (both negated) at corners.  The mask is checked
 * on the host (one synchronous copy): EINVAL if a replacement would itself be
 * unknown (fluid channels one cell wide), for other lattices or storage forms.
 * With walls set, FP32 steps keep running two per launch where nx % 4 == 0 (the
 * tensor-copy form), one per launch otherwise; the adjoint calls return EINVAL. */
lbrs_status lbrs_set_obstacles(lbrs_ctx* ctx, const uint8_t* d_solid);

/* ---------------------------------------------------------------- y-slabs
 *
 * One grid split into y-slabs, one context per slab (on one GPU or one per GPU).
 * The pull of the multi-D update (Section II.D) reads, for the row j, the rows
 * j - 1 and j + 1 only, so a step of a slab needs, at each cut, the neighbouring
 * slab's row next to the cut.  A context whose y side is LBRS_BC_CUT stores H
 * ghost rows beyond that side (lbrs_bc.halo_rows) and closes its stored grid
 * there like a transmissive side.  After a rows' import, up to H steps leave the
 * context's own rows exactly as in the unsplit grid: each step spoils one more
 * ghost row from the outer edge inwards and never an own row.  Hence:
 *   - nx, ny, the fields of lbrs_set_state and lbrs_moments, the distributions of
 *     lbrs_get/set_distributions and checkpoints, and the diagnostics cover the
 *     context's own rows only (ny of them);
 *   - after lbrs_set_state, lbrs_set_distributions or lbrs_checkpoint_load, and
 *     after every H steps, lbrs_step returns LBRS_ESTATE until each cut side has
 *     been imported again; a step count larger than what the last imports cover
 *     is refused the same way (no step is taken);
 *   - a slab's own rows evolve bit for bit as the same rows of the unsplit grid
 *     do (same kernels, same per-cell arithmetic), provided that every import
 *     carries the neighbour's rows of the same step number.
 * Not covered on cut grids (LBRS_EINVAL): internal walls, the adaptive lambda and
 * the checkpointed adjoint driver; the adjoint steps themselves are (see
 * lbrs_rows_export).  The diagnostics totals of the slabs add up to the unsplit grid's
 * up to the order of the FP64 additions.
 *
 * lbrs_halo_size: the rows H of a cut side (2 = y-lo, 3 = y-hi; 0 rows if the side is
 *   not a cut) and the bytes of one exchanged block: P planes x H rows x nx cells in
 *   the storage precision, P = Q K = 16 in the distribution forms, 4 in LBRS_F32U.
 * lbrs_halo_export: copies the H own rows next to `side` (rows 0..H-1 for y-lo,
 *   ny-H..ny-1 for y-hi), every plane, to dst as [P][H][nx] (rows in increasing y).
 *   dst is caller-owned, host (on_device = 0; the call then synchronises) or device
 *   memory of any GPU (a peer copy).  Enqueued on the context's stream.
 * lbrs_halo_import: writes such a block, exported by the neighbour across `side` (its
 *   y-hi block for our y-lo side, its y-lo block for our y-hi side), into the ghost
 *   rows beyond `side`, and lets H more steps run.  src as dst above; the caller keeps
 *   it unchanged until the stream has passed the call.
 * Both return LBRS_EINVAL for a side that is not a cut and LBRS_ESTATE without a state. */
lbrs_status lbrs_halo_size(const lbrs_ctx* ctx, int side, int64_t* rows, size_t* bytes);
lbrs_status lbrs_halo_export(lbrs_ctx* ctx, int side, void* dst, int on_device);
lbrs_status lbrs_halo_import(lbrs_ctx* ctx, int side, const void* src, int on_device);

/* The adjoint on y-slabs of a periodic grid (x periodic, y sides cut): the reverse halo.
 * On such a context the adjoint calls below (lbrs_step_record, lbrs_adjoint_seed,
 * lbrs_vjp_loss, lbrs_adjoint_step, lbrs_vjp_equilibrium) take their buffers in the stored
 * layout: [planes][ny_s][nx] with ny_s = ny plus the ghost rows of both cuts and own row 0 at
 * stored row row0 (lbrs_store_rows).  The adjoint step pulls, for row j, from rows j - 1 and
 * j + 1 (the transpose of the streaming moves the same rows the other way), and its kernels
 * wrap the stored rows in y, which spoils ghost rows only; so H adjoint steps give exact own
 * rows when the ghost rows of the adjoint state and of the H recorded moment fields they use
 * hold the neighbours' rows.  lbrs_rows_export copies the H own rows next to cut `side` of a
 * stored-layout buffer (planes planes in the storage precision, e.g. 16 for dL/df*, 4 T for T
 * recorded steps of moments) to a block [planes][H][nx]; lbrs_rows_import writes such a block,
 * exported by the neighbour across `side`, into the buffer's ghost rows.  Memory and stream
 * rules as for lbrs_halo_export / lbrs_halo_import; no state needs to be set.  Recording steps follow the same import rule
 * as lbrs_step (LBRS_ESTATE beyond what the imports cover); lbrs_vjp_loss sums the own rows
 * only (the grid's loss is the sum over the slabs); the checkpointed driver below is not
 * covered on cut grids (it would step without the neighbours' rows: LBRS_EINVAL). */
lbrs_status lbrs_store_rows(const lbrs_ctx* ctx, int64_t* ny_store, int64_t* row0);
lbrs_status lbrs_rows_export(lbrs_ctx* ctx, int side, const void* d_buf, int planes, void* dst, int on_device);
lbrs_status lbrs_rows_import(lbrs_ctx* ctx, int side, void* d_buf, int planes, const void* src, int on_device);

/* ---------------------------------------------------------------- adjoint
 *
 * Discrete adjoint of the D2Q4 step on a fully periodic domain.  The paper
 * has no adjoint; these calls transpose the step defined above so that
 * gradients of a loss of the final state with respect to the initial
 * conserved fields can be computed:
 *   forward   f = S f*^n, U = M f, f*^{n+1} = (1 - omega) f + omega E(U)
 *   backward  fbar = (1 - omega) gbar + omega J_E(U)^T gbar,
 *             dL/df*^n_q(x - c_q) = fbar_q(x)       (gbar = dL/df*^{n+1})
 * with J_E the Jacobian of the equilibria (through the ideal-gas Euler flux
 * Jacobians).  Buffers are device memory in the storage precision unless a
 * dtype is given; distributions are [4][4][ny][nx], fields [4][ny][nx] (on a
 * y-slab context, the stored layout: see lbrs_rows_export above).
 * Contexts that are neither periodic nor a y-slab of a periodic grid, and D1Q2
 * contexts, get LBRS_EINVAL. */

/* Enqueue n steps like lbrs_step, also writing each step's moments U^{s+m+1}
 * (the U its collision used) to d_U_hist + m*K*N elements, m = 0..n-1. */
lbrs_status lbrs_step_record(lbrs_ctx* ctx, int64_t n, void* d_U_hist);

/* gbar[q][k] = dL/dU_k for every q (U_k = sum_q f*_{q,k}); d_dLdU is [K][ny][nx] of dtype. */
lbrs_status lbrs_adjoint_seed(lbrs_ctx* ctx, const void* d_dLdU, int dtype, void* d_gbar);

/* Density mismatch loss of the current state, L = 1/2 sum_cells (rho - rho_target)^2 dx^d,
 * reduced in FP64 in a fixed order (loss: host pointer, nullable; synchronises
 * when given), and its seed d_gbar = dL/df*.  d_rho_target is [ny][nx] of dtype. */
lbrs_status lbrs_vjp_loss(lbrs_ctx* ctx, const void* d_rho_target, int dtype, void* d_gbar, double* loss);

/* One backward step: d_gbar_out = dL/df*^n from d_gbar_in = dL/df*^{n+1} and
 * d_U_next = the moments of step n+1.  In and out buffers must differ. */
lbrs_status lbrs_adjoint_step(lbrs_ctx* ctx, const void* d_U_next, const void* d_gbar_in, void* d_gbar_out);

/* dL/dU0 = J_E(U0)^T dL/df*^0 per cell (the initial state is f*^0 = E(U0)). */
lbrs_status lbrs_vjp_equilibrium(lbrs_ctx* ctx, const void* d_U0, const void* d_gbar0, void* d_gradU0);

/* sqrt(T) checkpointing.  Bytes of the caller-owned adjoint workspace for a run
 * of n_steps in segments of `segment` steps: ceil(n/segment)+1 distribution
 * checkpoints, `segment` recorded moment fields and two gradient buffers. */
lbrs_status lbrs_adjoint_workspace_size(const lbrs_ctx* ctx, int64_t n_steps, int64_t segment, size_t* bytes);

/* Run n_steps from the current state, storing the state at each segment start
 * and at the end in d_adj_ws (256-byte aligned, >= lbrs_adjoint_workspace_size). */
lbrs_status lbrs_forward_checkpointed(lbrs_ctx* ctx, int64_t n_steps, int64_t segment, void* d_adj_ws, size_t bytes);

/* Backward sweep of the run recorded by lbrs_forward_checkpointed on d_adj_ws:
 * each segment, last first, is recomputed from its checkpoint while recording
 * its moments, then swept with lbrs_adjoint_step; finally d_gradU0 = dL/dU0.
 * d_gbar_T = dL/df* of the final state (e.g. from lbrs_vjp_loss).  The
 * context's state is the final forward state again on return. */
lbrs_status lbrs_backward_checkpointed(lbrs_ctx* ctx, void* d_adj_ws, const void* d_gbar_T, void* d_gradU0);

/* ---------------------------------------------------------------- batched D1Q2 / D1Q3 tubes
 *
 * Many independent 1-D problems (shock tubes) of uneven length advanced
 * together, each with its own lattice speed lambda_b and number of steps.
 * All tubes share gamma, omega and the end condition (transmissive or
 * periodic at both ends).  Distributions are stored concatenated:
 * f[q][k][off_b + x], off_b = sum of the lengths of the tubes before b;
 * field arrays are [3][sum N_b].  The step per cell is the D1Q2 (or D1Q3,
 * cfg.lattice) step of Section II.C, identical in arithmetic to the single-tube path; the
 * kernels advance a tile of a tube by up to `halo` steps in shared memory per
 * launch (temporal blocking, see lbrs_batch_tuning). */
typedef struct lbrs_batch lbrs_batch;

typedef struct {
    uint32_t struct_size;    /* = sizeof(lbrs_batch_config) */
    int32_t precision;       /* LBRS_F64 or LBRS_F32 */
    int32_t boundary;        /* LBRS_BC_TRANSMISSIVE or LBRS_BC_PERIODIC, both ends of every tube */
    int32_t lattice;         /* LBRS_D1Q2 (0) or LBRS_D1Q3 (the rest particle; lambda per tube accordingly) */
    int64_t batch;           /* number of tubes, >= 1 */
    const int64_t* lengths;  /* host [batch]: cells per tube (>= 1); copied at create */
    const double* lambda;    /* host [batch]: lattice speed per tube (> 0); copied at create */
    double gamma, omega;
    void* cuda_stream;
} lbrs_batch_config;

/* Launch shape of the batched kernel: `block` threads (128, 256 or 512), each
 * owning `cells_per_thread` window cells; a window is block*cells_per_thread
 * cells, of which `halo` on each side are recomputed context and the rest
 * (the tile, >= 32 cells) is advanced by up to `halo` steps per launch. */
typedef struct {
    int32_t block, cells_per_thread, halo, reserved;
} lbrs_batch_tuning;

lbrs_status lbrs_batch_workspace_size(const lbrs_batch_config* cfg, size_t* bytes);
lbrs_status lbrs_batch_create(const lbrs_batch_config* cfg, void* d_workspace, size_t bytes, lbrs_batch** out);
void        lbrs_batch_destroy(lbrs_batch* batch);

/* f = f^eq(U(W)) per cell with the cell's tube lambda; W [3][sum N] as in lbrs_set_state. */
lbrs_status lbrs_batch_set_state(lbrs_batch* batch, const void* W, int on_device, int dtype, int kind);

/* Advance tube b by steps[b] >= 0 steps (host array [batch]).  Asynchronous.
 * The launch sequence is captured in a CUDA graph and replayed while steps and
 * tuning stay the same. */
lbrs_status lbrs_batch_run(lbrs_batch* batch, const int64_t* steps);

/* Conserved fields [3][sum N] of the current state (FP64 sums, written as dtype). */
lbrs_status lbrs_batch_moments(lbrs_batch* batch, void* U_out, int on_device, int dtype);
lbrs_status lbrs_batch_get_distributions(lbrs_batch* batch, void* dst, int on_device);

lbrs_status lbrs_batch_get_tuning(const lbrs_batch* batch, lbrs_batch_tuning* tuning);
lbrs_status lbrs_batch_set_tuning(lbrs_batch* batch, const lbrs_batch_tuning* tuning);

/* Time one launch of every candidate tuning (block in {128, 256, 512},
 * cells per thread in {1, 2, 4, 8}, halo in {8, 16, 32, 64}) from the current
 * state for the given steps, keep the fastest per lattice update and return
 * it (chosen, ns_per_update nullable).  The state is not changed. */
lbrs_status lbrs_batch_autotune(lbrs_batch* batch, const int64_t* steps, lbrs_batch_tuning* chosen,
                                double* ns_per_update);

lbrs_status lbrs_batch_launch_count(const lbrs_batch* batch, int64_t* launches);
const char* lbrs_batch_last_error(const lbrs_batch* batch);

/* Number of time steps taken since the state was set. */
lbrs_status lbrs_step_count(const lbrs_ctx* ctx, int64_t* steps);

/* Number of kernels this context has launched (graph launches count each kernel). */
lbrs_status lbrs_launch_count(const lbrs_ctx* ctx, int64_t* launches);

/* Description of the last error on ctx ("" if none). Never NULL. */
const char* lbrs_last_error(const lbrs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBRS_H */
