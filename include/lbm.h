/*
 * lbm.h -- C interface of the GB300 library for the lattice Boltzmann method
 * with fully resolved moving rigid particles (Bartuschat, Fischermeier,
 * Gustavsson, Ruede, "Two computational models for simulating the tumbling
 * motion of elongated particles in fluids", Sec. 4).
 *
 * The problem the interface states (Sec. 4.2-4.3): a box of fluid on a
 * Cartesian lattice, with periodic or moving-wall boundaries, holding rigid
 * bodies mapped onto the lattice as obstacle cells; fluid and bodies advance
 * together, two-way coupled, and the hydrodynamic force and torque on every
 * body and the fluid fields can be read back.
 *
 * Conventions
 *  - Lattice units throughout: dx = dt = 1.  Cell (i,j,k) has centre (i,j,k)
 *    and linear index idx = i + nx*(j + ny*k) (x fastest).
 *  - D3Q19 velocities (Sec. 4.1, weights 1/3, 1/18, 1/36), numbered
 *      0: (0,0,0)
 *      1..6: +x, -x, +y, -y, +z, -z
 *      7..18: (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),
 *             (1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1)
 *    so that the opposite of q > 0 is the other member of its pair.
 *  - Canonical populations ("pdfs") are the post-stream values f_q(x) at the
 *    start of the next collision, stored as double f[q*n + idx], n = nx*ny*nz.
 *    Non-fluid cells report 0 for populations, density and velocity.
 *  - Every call returns an lbm_status; 0 is success.  No exception crosses the
 *    interface.  lbm_last_error() gives a message for the last failure.
 *  - The caller owns every host buffer passed in; the library never keeps or
 *    frees caller memory.  Device memory is taken from the caller's allocator
 *    callbacks when given, otherwise from cudaMalloc, and is released by
 *    lbm_destroy.
 *  - Work is ordered on the stream given at creation.  lbm_step is
 *    asynchronous; calls that return host data synchronise that stream.
 *  - A context is used by one host thread at a time.
 *  - A context belongs to the CUDA device that was current when it was
 *    created; every call makes that device current for its duration and
 *    restores the caller's device before returning.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 19

typedef struct lbm_ctx lbm_ctx;

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,         /* invalid argument (sizes, tau <= 1/2, NULL ...) */
    LBM_ERR_STATE = 2,       /* call not valid in the context's state */
    LBM_ERR_OOM = 3,         /* device allocation failed */
    LBM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    LBM_ERR_NUMERIC = 5,     /* non-finite force or particle state detected */
    LBM_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out */
    LBM_ERR_UNSUPPORTED = 7  /* request outside what this build supports */
} lbm_status;

/* How populations are stored in device memory.  Every form stores the offset
 * g_q = f_q - w_q*rho0 from the rest state.  F64 computes in double; the others
 * compute in float.  The force/torque accumulators and the rigid-body update
 * are always double; on the float forms the per-cell and per-warp partial
 * sums before them are compensated float pairs (about 48 bits). */
typedef enum lbm_precision {
    LBM_F64 = 0,
    LBM_F32 = 1,
    LBM_F16_OFFSET = 2,   /* IEEE binary16 offsets, round to nearest even */
    LBM_BF16_OFFSET = 3   /* bfloat16 offsets; the sweep's stores round stochastically
                           * (up with probability equal to the discarded fraction,
                           * bits from a counter-based generator seeded by the cell
                           * index and the step count: deterministic for a given
                           * state and step), other stores to nearest even */
} lbm_precision;

/* Particle-id map codes of cells that are not particle cells. */
#define LBM_PID_FLUID    0xFFFFFFFFu
#define LBM_PID_WALL_YLO 0xFFFFFFFEu  /* wall layer y = 0, moves at wall_u_lo */
#define LBM_PID_WALL_YHI 0xFFFFFFFDu  /* wall layer y = ny-1, moves at wall_u_hi */
#define LBM_PID_WALL     0xFFFFFFFCu  /* resting wall layer of a non-periodic x or z face */

/* Canonical cell flags returned by lbm_get_fields. */
#define LBM_FLAG_FLUID    0
#define LBM_FLAG_WALL     1
#define LBM_FLAG_PARTICLE 2

/* One lattice (Sec. 4.1).  A non-periodic axis is closed by one layer of wall
 * cells on each side: the y layers move with wall_u_lo / wall_u_hi (velocity
 * bounce-back, Eq. LBMMovWall), x and z layers rest (Eq. BBBC).  With the TRT
 * "magic" product Lambda = (tau - 1/2)(tau_odd - 1/2) = 3/16 the walls sit half-way
 * between cells (Sec. 4.1).  body_force is a constant force density on the
 * fluid, entered as the odd source 3 w_q rho0 c_q.g after collision. */
typedef struct lbm_grid_desc {
    int nx, ny, nz;            /* >= 3 each */
    double tau;                /* > 1/2; viscosity (tau - 1/2)/3 (Eq. kinVisc) */
    double magic;              /* TRT Lambda > 0; 3/16 in all of Sec. 5-6 */
    double rho0;               /* mean density, > 0 (usually 1) */
    int periodic[3];           /* 1 = periodic along x, y, z */
    double wall_u_lo[3];       /* velocity of the y = 0 wall layer, |u| < 0.1 */
    double wall_u_hi[3];       /* velocity of the y = ny-1 wall layer, |u| < 0.1 */
    double body_force[3];      /* fluid body-force density */
    lbm_precision prec;        /* storage form (same for every cell of a batch) */
    void *cuda_stream;         /* cudaStream_t for all work; NULL = legacy default stream */
    void *(*dev_alloc)(size_t bytes, void *user); /* optional device allocator */
    void (*dev_free)(void *ptr, void *user);       /* its matching free */
    void *user;                /* passed to dev_alloc / dev_free */
    int free_slip[3];          /* 1 = the wall layers of non-periodic axis x, y, z are
                                * free-slip walls (Eq. FreeSlipBC: a population leaving a
                                * fluid cell into the wall is reflected, its normal
                                * component reversed; at edges every crossed layer
                                * reflects).  Needs periodic[a] = 0; with free_slip[1]
                                * the y wall speeds must be 0.  Bodies must keep off the
                                * fluid layer next to a free-slip wall (lbm_set_particles
                                * returns LBM_ERR_ARG, a step that moves a body there
                                * LBM_ERR_UNSUPPORTED).  No momentum is booked to
                                * free-slip walls (lbm_get_wall_forces covers the
                                * no-slip y walls). */
} lbm_grid_desc;

/* One rigid body (Sec. 4.2-4.3).  shape LBM_SHAPE_ELLIPSOID: semi-axes
 * (a, b, c) along the body x, y, z axes, mass = density * 4/3 pi a b c.
 * shape LBM_SHAPE_SPHEROCYLINDER (the particles of Sec. 5.1, Fig. Capsule): a
 * cylinder of radius r with hemispherical end caps, total length L along body
 * x, given as semi_axes = (L/2, r, r) with L/2 >= r; mass = density *
 * (pi r^2 (L - 2r) + 4/3 pi r^3).  Inertia of the homogeneous solid.  quat =
 * (w, x, y, z) rotates body to world coordinates and is normalised by the
 * library; density is relative to rho0 = 1 units.  ext_force and ext_torque
 * are added to the hydrodynamic force and torque every step.  A fixed body
 * keeps its pose and velocities.  cell selects the lattice of a batch (0 for
 * a single lattice).  Along a periodic axis of extent n a body must stay
 * shorter than n/2 - 1 from its centre in every orientation (longest semi-axis
 * a with 2a + 2 < n): the obstacle mapping and the surface velocity of a
 * boundary link take the minimum image of the displacement from the centre,
 * and for a longer body the two can pick different images. */
#define LBM_SHAPE_ELLIPSOID 0
#define LBM_SHAPE_SPHEROCYLINDER 1
typedef struct lbm_particle {
    double pos[3];
    double quat[4];
    double vel[3];
    double omega[3];
    double semi_axes[3];
    double density;
    double ext_force[3];
    double ext_torque[3];
    int cell;
    int fixed;
    int shape;                 /* LBM_SHAPE_* */
} lbm_particle;

/* Create one lattice, fluid at rest with density rho0 (f_q = w_q rho0).
 * Errors: LBM_ERR_ARG for a NULL pointer, a size < 3, tau <= 1/2, magic <= 0,
 * rho0 <= 0, a wall speed component >= 0.1 in magnitude, an unknown precision,
 * or a lattice above 2^31 cells; LBM_ERR_OOM; LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_grid_desc *desc, lbm_ctx **out);

/* Create a batch of independent lattices advanced together (one sweep launch
 * per step over all of them).  prec, cuda_stream and the allocator are taken
 * from cells[0] and must be the same in every entry.  Errors as lbm_create. */
lbm_status lbm_create_batch(const lbm_grid_desc *cells, int ncells, lbm_ctx **out);

/* Replace the particle set and re-map the obstacle cells from the given poses
 * (Sec. 4.2: a non-wall cell is an obstacle cell of a body iff its centre lies
 * inside it; a cell inside several bodies belongs to the lowest index).
 * Particle cells that become fluid are refilled with f^eq(rho0, 0); cells that
 * become obstacles drop their populations.  n = 0 removes all particles.
 * Errors: LBM_ERR_ARG for n < 0, p == NULL with n > 0, a cell index out of
 * range, semi-axes <= 0, density <= 0, an unknown shape, a spherocylinder
 * whose semi_axes are not (L/2, r, r) with L/2 >= r, a body not inside the
 * fluid region of a non-periodic axis, or a body on the fluid layer next to a
 * free-slip wall. */
lbm_status lbm_set_particles(lbm_ctx *ctx, const lbm_particle *p, int n);

/* Advance nsteps time steps, asynchronously on the context's stream.  One step
 * (Sec. 4.1-4.3): the fused stream-collide sweep over every fluid cell with
 * velocity bounce-back at walls and obstacle cells and the momentum-exchange
 * force/torque sums (Eqs. LBMCollide, LBMStream, LBMMovWall,
 * LBMhydrodynForce); the rigid-body update; the re-mapping of obstacle cells
 * with equilibrium refill of uncovered cells (Sec. 4.2).
 * Device-side conditions (a non-finite force or body state, a body reaching
 * the fluid layer next to a free-slip wall, a bounded wait that ran out) are
 * reported by the next synchronising call (lbm_sync, lbm_get_forces).
 * Errors: LBM_ERR_ARG for nsteps < 0; LBM_ERR_STATE after such a condition
 * was reported; LBM_ERR_CUDA. */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps);

/* Wait for all queued work; reports LBM_ERR_NUMERIC (non-finite force, body
 * state or wall momentum), LBM_ERR_UNSUPPORTED (a body reached the fluid layer next to a
 * free-slip wall) or LBM_ERR_TIMEOUT (a bounded device wait ran out) if met
 * since the last check; the context then refuses further steps. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Hydrodynamic force and torque (Eq. LBMhydrodynForce; torque about the
 * centre of mass with lever arm x_s - x_C) of the last completed step, for the
 * first n particles, as force3n[3*i + a], torque3n[3*i + a].  External loads
 * are not included.  Synchronises and reports the device-side conditions as
 * lbm_sync does.  Either pointer may be NULL. */
lbm_status lbm_get_forces(lbm_ctx *ctx, double *force3n, double *torque3n, int n);

/* Momentum handed per step to the y = 0 and y = ny-1 wall layers of lattice
 * `cell` in the last step: f6[0..2] low wall, f6[3..5] high wall (no-slip
 * walls; free-slip walls book no momentum). */
lbm_status lbm_get_wall_forces(lbm_ctx *ctx, int cell, double *f6);

/* Current particle states (pose, velocities) of the first n particles. */
lbm_status lbm_get_particles(lbm_ctx *ctx, lbm_particle *p, int n);

/* Set external force/torque of the first n particles (host arrays of 3n
 * doubles; either may be NULL to leave that part unchanged).  Asynchronous
 * host-to-device copy on the context's stream: pageable arrays may be reused
 * as soon as the call returns, page-locked ones must stay unchanged until the
 * next synchronising call. */
lbm_status lbm_set_external(lbm_ctx *ctx, const double *force3n, const double *torque3n, int n);

/* Fields of lattice `cell` in canonical form (see Conventions): density
 * rho[n], velocity u3[3*n] (component-major, u = sum(c f)/rho0 + g/2),
 * flags[n] (LBM_FLAG_*), particle ids pid[n] (LBM_PID_* or the particle
 * index), populations pdfs[19*n].  Any pointer may be NULL.  Synchronises. */
lbm_status lbm_get_fields(lbm_ctx *ctx, int cell, double *rho, double *u3, uint8_t *flags,
                          uint32_t *pid, double *pdfs);

/* Overwrite the populations of the fluid cells of lattice `cell` from a
 * canonical host array pdfs[19*n] (checkpoint restore, test set-up). */
lbm_status lbm_set_pdfs(lbm_ctx *ctx, int cell, const double *pdfs);

/* Boundary links {(x_F, q): x_F fluid, x_F + c_q a wall or obstacle cell} of
 * lattice `cell`, ordered by cell index then q (the direction sets D_s of
 * Eq. LBMhydrodynForce, walls included), with the id of the cell hit.  Writes
 * at most cap entries; *count receives the total.  Any output array may be
 * NULL when cap = 0. */
lbm_status lbm_get_links(lbm_ctx *ctx, int cell, int32_t *idx, int8_t *q, uint32_t *pid, int cap,
                         int *count);

/* Allocation-free form of the link compaction (the paper has no counterpart).
 * Some callers cannot allocate device memory at the moment they need the link
 * list: a solver embedded in a host application whose memory manager owns all
 * device memory, or a latency-critical loop in which an allocation (which can
 * synchronise the device) is not acceptable.  This call allocates nothing:
 * the caller passes device buffers for the results and the per-block counts
 * live in one fixed array in device memory that every GPU loading this library
 * holds until the process exits (256 KiB).
 *   d_idx, d_q, d_pid: device arrays of at least cap entries (may be NULL when
 *     cap = 0); same content and order as lbm_get_links.
 *   d_count: device int receiving the total number of links (may exceed cap).
 * Asynchronous on the context's stream; nothing is copied to the host.
 * Lattices above 16,777,216 cells (65,536 tiles of 256) are rejected with
 * LBM_ERR_ARG.  The first call on a device looks up the device address of the
 * fixed array for that device; make that first call before any stream capture.
 * All calls share the array: calls whose work overlaps on the GPU (another
 * stream, another context, another host thread) race on it and must be
 * ordered by the caller. */
lbm_status lbm_get_links_noalloc(lbm_ctx *ctx, int cell, int32_t *d_idx, int8_t *d_q, uint32_t *d_pid,
                                 int cap, int *d_count);

typedef struct lbm_info {
    long long ncells_total;     /* cells over all lattices */
    long long nfluid_hint;      /* not computed: -1 */
    int nlattices;
    int nparticles;
    long long steps_done;
    size_t device_bytes;        /* device memory held by the context */
    int sweep_grid, sweep_block;/* launch shape of the sweep kernel */
    int bytes_per_population;   /* 8, 4 or 2 */
    int sweep_split;            /* 1: the direct sweep runs split (lbm_set_sweep_split) */
    int remap_fused;            /* 1: the re-mapping step runs as one cooperative launch */
    int remap_grid;             /* blocks of that launch (0 when not fused) */
    int cells_per_thread;       /* direct sweep: consecutive cells per thread (1, 2, 4) */
    int device;                 /* CUDA device of the context */
    int sweep_prefetch;         /* tiles ahead that the direct sweep prefetches into L2 (0: none) */
    int sweep_prefetch_mode;    /* LBM_PREFETCH_* in effect (LBM_PREFETCH_OFF outside the direct sweep) */
} lbm_info;

lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *info);

/* Sweep launch shape.  block = 0 selects the ring sweep (256 threads, each
 * keeping its next cells' populations in flight through asynchronous copies
 * into shared memory); block = -1 selects the staged sweep (tiles of 256
 * cells brought into shared memory by asynchronous bulk copies, several tiles
 * in flight per block); block = 32..256 (multiple of 32) selects the direct
 * sweep with that many threads, one cell each.  grid = number of blocks
 * (<= 0: one block per tile for the direct sweep, one resident wave on every
 * SM otherwise; capped at the tile count).  Used by the autotuner; takes
 * effect at the next lbm_step.  Any other block value returns LBM_ERR_ARG.
 * The default is the direct sweep with 128 threads. */
lbm_status lbm_set_launch(lbm_ctx *ctx, int block, int grid);

/* Consecutive cells per thread of the direct sweep: 1, 2 or 4 (FP64 storage:
 * 1 or 2).  With 2 or 4 a thread loads all its cells' populations before
 * colliding any of them (more bytes in flight per thread) and moves the
 * values of one population plane for its cells with one vector access
 * wherever they are contiguous and aligned (every plane on even steps; on odd
 * steps the planes of directions without an x component, when nx is a
 * multiple of the group size), and the FP32 / FP16 / BF16 sweeps collide two
 * cells at once on paired FP32 instructions; a direct-sweep tile then covers
 * block * cpt cells.  Results agree to rounding for every setting (the same
 * arithmetic, contracted into fused multiply-adds differently).  Default 1;
 * the autotuner chooses.  Takes effect at the next lbm_step.  Errors:
 * LBM_ERR_ARG for any other value. */
lbm_status lbm_set_cells_per_thread(lbm_ctx *ctx, int cpt);

/* Split direct sweep (enable != 0): near-obstacle cells (those next to a
 * body or a resting wall) leave the sweep kernel; a list kernel compacts them
 * from the marked tiles and a third kernel updates them, one cell per
 * thread, so that warps in the near-obstacle path are full.  The two kernels
 * touch disjoint population slots.  Worth it when bodies are many (dense
 * suspensions); the autotuner decides.  Applies to the direct sweep only;
 * takes effect at the next lbm_step. */
lbm_status lbm_set_sweep_split(lbm_ctx *ctx, int enable);

/* L2 prefetch in the direct sweep: a block that starts a tile first asks the
 * L2 for the population ranges of a later tile (the tile one resident wave
 * ahead, or the block's own next tile on a persistent grid) with one
 * asynchronous bulk prefetch per population plane, so that tile's loads find
 * their data in the L2.  mode: LBM_PREFETCH_OFF (0, the default),
 * LBM_PREFETCH_ALL (1: every sweep), LBM_PREFETCH_EVEN (2: only the sweeps of
 * even time steps, which read and write each cell's own slots) or
 * LBM_PREFETCH_ODD (3: only the sweeps of odd time steps, which read and
 * write the neighbours' slots); the two kinds of sweep gain or lose from it
 * differently.  Any other mode: LBM_ERR_ARG.  A hint only: results do not
 * change.  Chosen per context by lbm_autotune (for each parity on its own);
 * takes effect at the next lbm_step.  No counterpart in the paper (a launch
 * parameter like the block size). */
#define LBM_PREFETCH_OFF 0
#define LBM_PREFETCH_ALL 1
#define LBM_PREFETCH_EVEN 2
#define LBM_PREFETCH_ODD 3
lbm_status lbm_set_sweep_prefetch(lbm_ctx *ctx, int mode);

/* Fused re-mapping step (enable != 0; default 0): the rigid-body update
 * (Sec. 4.3) and the four passes of the obstacle re-mapping (Sec. 4.2:
 * uncover, claim, refill/fix-up, flags) run as one cooperative launch of at
 * most one resident wave, with grid-wide barriers between the passes, instead
 * of five launches.  Used only where the device and driver accept cooperative
 * launches (probed once per context, eagerly and inside a captured graph);
 * otherwise the separate kernels run.  The arithmetic is the same either way
 * (results differ only by the order of the sweep's FP64 force atomics).  On
 * GB300 the five launches with programmatic dependent launch are faster, so
 * the default is the separate form.  A barrier wait that runs out (it cannot
 * while the launch is resident) makes lbm_step return LBM_ERR_TIMEOUT.  Takes
 * effect at the next lbm_step. */
lbm_status lbm_set_remap_fused(lbm_ctx *ctx, int enable);

/* Poll limit of the bounded device-side waits of the fused re-mapping step
 * (its grid barriers): a waiting block gives up after `polls` polls, sets the
 * timeout condition and returns; 0 restores the default (2^20 polls, far
 * above any wait of a resident launch).  A small limit makes such waits run
 * out: the next synchronising call reports LBM_ERR_TIMEOUT and the context
 * refuses further steps.  For tests of that path; synchronises the stream. */
lbm_status lbm_set_wait_limit(lbm_ctx *ctx, unsigned polls);

/* Momentum stabilisation (Sec. 4.1; enable != 0; default 0): before every
 * sweep the mean velocity ubar = sum(j) / (rho0 N_fluid) over all fluid cells
 * of the current state is computed (two extra launches per step, one read of
 * the populations), and every cell's equilibrium is taken at u - ubar, so
 * that a fully periodic domain with constant forces on its particles does not
 * accelerate without bound (the total fluid momentum relaxes by
 * 1 - omega_odd per step).  Single-lattice contexts only: a batch returns
 * LBM_ERR_UNSUPPORTED.  Takes effect at the next lbm_step. */
lbm_status lbm_set_momentum_stabilisation(lbm_ctx *ctx, int enable);

/* Choose the sweep launch shape by timing candidates on this context (runs
 * sweeps on scratch copies: the state is restored afterwards): the ring and
 * staged sweeps and the direct sweep with 128 or 256 threads, 1, 2 or 4 cells
 * per thread, fused or split, on persistent and one-tile-per-block grids,
 * each direct-sweep shape with and without the L2 prefetch, timed for the
 * even- and odd-step sweeps separately (the prefetch is then chosen for each
 * parity on its own).  The chosen shape is kept and returned through
 * block/grid (either may be NULL); lbm_get_info reports the cells per
 * thread, the split and the prefetch mode. */
lbm_status lbm_autotune(lbm_ctx *ctx, int *block, int *grid);

/* CUDA graphs: when enabled, lbm_step replays a captured two-step graph for
 * pairs of steps that start on an even step, and a captured one-step graph
 * (one per parity) for a leading odd step or a trailing single step (default
 * on; needs a non-NULL stream).  Replay and eager launches give the same
 * flags and particle ids, and fields equal up to the order of the FP64
 * force sums. */
lbm_status lbm_set_graphs(lbm_ctx *ctx, int enable);

/* Sweep-kernel timing: when enabled, every sweep launch is bracketed by CUDA
 * events on the context's stream; lbm_get_sweep_timing returns the summed
 * device time in milliseconds and the number of launches since enabling
 * (synchronises) and resets the tally.  Enabling turns graph replay off. */
lbm_status lbm_set_sweep_timing(lbm_ctx *ctx, int enable);
lbm_status lbm_get_sweep_timing(lbm_ctx *ctx, double *ms, long long *launches);

/* Number of kernel launches issued by the library since creation. */
lbm_status lbm_get_launch_count(lbm_ctx *ctx, long long *launches);

/* ---------------------------------------------------------------------------
 * Learned force/torque closure.  The paper has none: its force and torque
 * are the momentum exchange of Eqs. TransferredMomentum / LBMhydrodynForce
 * (Sec. 4.2), applied in the rigid-body update (Sec. 4.3).  A closure adds a
 * correction predicted by a 86-64-64-64-6 ReLU network from the flow around
 * each body, before that update.
 *
 * Features (LBM_CLOSURE_IN per body): 27 sample points in the body frame at
 * offsets (1.5a i, 1.5b j, 1.5c k), i,j,k in {-1,0,1}, point s = 9(i+1) +
 * 3(j+1) + (k+1), (a,b,c) the semi-axes; at the world point x_C + R o_s the
 * velocity field (as lbm_get_fields reports it: zero on wall and particle
 * cells) is interpolated trilinearly between cell centres (periodic axes
 * wrap, the others clamp to the lattice); feature 3s+d is component d of
 * R^T (u - U - Omega x R o_s) / V (the flow relative to the body's rigid
 * motion continued to the sample point; U, Omega the body's velocity and
 * angular velocity), V = gamma * a.  Features 81..83: the
 * body x axis in world coordinates (first column of R); 84: a/b; 85: b.
 * gamma is the shear rate of the channel between the moving y walls,
 * |u_hi,x - u_lo,x| / (ny - 2); a lattice without moving y walls has gamma
 * = 0 (V = 1) and its bodies get no correction.
 *
 * Network parameters: one flat vector of LBM_CLOSURE_PARAMS values, W1 (64 x
 * 86, row-major [out][in]), b1 (64), W2 (64 x 64), b2, W3 (64 x 64), b3, W4
 * (6 x 64), b4 (6); ReLU after the three hidden layers.  Outputs o: the
 * body-frame correction dF = o[0..2] * mu gamma a b, dM = o[3..5] *
 * mu gamma a^2 b, mu = rho0 (tau - 1/2) / 3, rotated to the world frame.
 * Inference runs on the FP16 tensor cores with FP32 accumulation.
 * ------------------------------------------------------------------------- */
#define LBM_CLOSURE_IN 86
#define LBM_CLOSURE_OUT 6
#define LBM_CLOSURE_PARAMS 14278

/* Enable the closure with FP16 parameters (host array of LBM_CLOSURE_PARAMS
 * IEEE half values, bytes = 2 * LBM_CLOSURE_PARAMS), or disable it (params =
 * NULL).  While enabled every time step evaluates the network after the
 * sweep and adds the correction to the force and torque of every body; the
 * forces lbm_get_forces reports then include the correction.  Synchronises
 * the stream.  Errors: LBM_ERR_ARG for a wrong size. */
lbm_status lbm_set_closure(lbm_ctx *ctx, const void *params, size_t bytes);

/* Features of every body in the current state (the velocity field the next
 * sweep starts from, the bodies' current pose and velocity): n x
 * LBM_CLOSURE_IN floats into the host array features; n must equal the
 * number of bodies.  Synchronises the stream. */
lbm_status lbm_closure_features(lbm_ctx *ctx, float *features, int n);

/* Training of the closure network on the GPU.  An lbm_mlp holds FP32 master
 * parameters, the Adam moments and an FP16 working copy in device memory
 * (cudaMalloc, released by lbm_mlp_destroy); its work is ordered on the given
 * CUDA stream (NULL: the legacy default stream).  Samples are device arrays:
 * x (n x LBM_CLOSURE_IN floats), y (n x LBM_CLOSURE_OUT floats).  Loss: the
 * mean over samples and outputs of (o - y)^2.  The forward and backward
 * passes run on the FP16 tensor cores with FP32 accumulation; the output
 * delta is kept unscaled (o - y) in FP16 and the factor 2/(6n) is applied to
 * the FP32 gradient. */
typedef struct lbm_mlp lbm_mlp;

/* Create a trainer from initial FP32 parameters (host, LBM_CLOSURE_PARAMS). */
lbm_status lbm_mlp_create(const float *params, void *cuda_stream, lbm_mlp **out);
/* Network outputs for n samples: y (device, n x LBM_CLOSURE_OUT floats). */
lbm_status lbm_mlp_forward(lbm_mlp *m, const float *x, float *y, int n);
/* Loss and gradient over n samples without changing the parameters: grad
 * (device, LBM_CLOSURE_PARAMS floats, may be NULL) and loss (host, may be
 * NULL; synchronises). */
lbm_status lbm_mlp_grad(lbm_mlp *m, const float *x, const float *y, int n, float *grad, float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * gradient over the n samples; loss (host, may be NULL; synchronises)
 * receives the loss before the step. */
lbm_status lbm_mlp_train_step(lbm_mlp *m, const float *x, const float *y, int n, float lr, float *loss);
/* Current parameters: FP32 master values (host, may be NULL) and the FP16
 * copy lbm_set_closure takes (host, 2 * LBM_CLOSURE_PARAMS bytes, may be
 * NULL).  Synchronises. */
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *params, void *params_fp16);
lbm_status lbm_mlp_destroy(lbm_mlp *m);

lbm_status lbm_destroy(lbm_ctx *ctx);
const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif
#endif
