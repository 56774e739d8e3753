/*
 * sbot.h -- C ABI of the GB300 (sm_103a) library for the lattice-Boltzmann /
 * immersed-boundary / block-refinement time step of Nguyen & Duong,
 * "SBoTFlow" (arXiv 2402.04606).
 *
 * The calls follow the paper's statement of the problem (Sec. 2.5): the
 * domain and its refinement are created, the body geometry and kinematics
 * are set, the time loop advances the flow, and forces and fields are read.
 *
 * Conventions (all calls):
 *  - Every call returns an sbot_status; SBOT_OK is 0.  Nothing aborts or
 *    exits.  sbot_last_error() gives a message for the last failing call on a
 *    context (the pointer stays valid until the next call on that context).
 *  - Pointers to host memory are owned by the caller and only read or
 *    written during the call; the library keeps none of them.  The library
 *    owns all device memory of a context and frees it in sbot_destroy.
 *  - Lengths are in lattice units of the finest level ("finest cells")
 *    unless a comment says otherwise; level l has cells of 2^(m-1-l) finest
 *    cells, level 0 is the coarsest, m the number of levels.
 *  - Dense per-level arrays are row-major [ny_l][nx_l] with nx_l = nx0 * 2^l;
 *    population arrays are [9][ny_l][nx_l] in the direction order of Eq. 1
 *    (c_x = 0,1,0,-1,0,1,-1,-1,1; c_y = 0,0,1,0,-1,1,1,-1,-1).
 *  - Work is enqueued on the CUDA stream given at creation; calls that
 *    return host data synchronise that stream first.
 */
#ifndef SBOT_H
#define SBOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbot_ctx* sbot_ctx_t;

typedef enum {
    SBOT_OK = 0,
    SBOT_ERR_ARG = 1,       /* invalid argument or description */
    SBOT_ERR_OOM = 2,       /* device allocation failed or over the memory budget */
    SBOT_ERR_CUDA = 3,      /* a CUDA call failed */
    SBOT_ERR_TIMEOUT = 4,   /* a bounded device wait gave up */
    SBOT_ERR_NONFINITE = 5, /* NaN or Inf found in the state */
    SBOT_ERR_STATE = 6      /* call not valid in the current state (e.g. a marker left the finest region) */
} sbot_status;

/* storage of the populations.  SBOT_F64 stores f_i and computes in FP64.
 * The other kinds compute in FP32 on the deviation f_i - w_i (rho = 1 +
 * sum, f^eq - w_i = w_i (rho - 1 + rho X)), so rounding is relative to O(u)
 * quantities rather than to the weights.  SBOT_F32 stores that deviation;
 * the 16-bit kinds store the deviation from the instance's free-stream
 * equilibrium, f_i - f^eq_i(rho0, u_in), so that a flow close to its free
 * stream stores small values (with u_in = 0 the two are the same). */
typedef enum {
    SBOT_F64 = 0,
    SBOT_F32 = 1,    /* FP32 deviation f_i - w_i */
    SBOT_F16DEV = 2, /* FP16 deviation f_i - f^eq_i(rho0, u_in) */
    SBOT_BF16DEV = 3 /* BF16 deviation f_i - f^eq_i(rho0, u_in) */
} sbot_storage;

/* domain sides: index 0 W (x = 0), 1 E, 2 S (y = 0), 3 N.  W/E (and S/N) are
 * both periodic or both not.  The paper names the kinds (Sec. 2.1 after
 * Eq. 10, Sec. 3.3) without formulas; this library uses: equilibrium inlet =
 * the boundary column is reset to f^eq(rho0, u_in) after streaming; open
 * outlet = the unknown populations are copied from the neighbouring interior
 * cell (zero gradient); symmetry = half-way specular mirror (the virtual cell
 * beyond the side is the boundary cell with the normal velocity reflected).
 * At a corner the S/N rule is applied before the W/E rule. */
typedef enum {
    SBOT_BC_PERIODIC = 0,
    SBOT_BC_EQ_INLET = 1,
    SBOT_BC_OPEN_OUTLET = 2,
    SBOT_BC_SYMMETRY = 3,
    SBOT_BC_WALL = 4 /* no-slip wall half a cell beyond the side (bounce-back), moving at wall_velocity */
} sbot_bc;

/* a region, in finest units, that must be refined to at least `level` */
typedef struct {
    int level;
    double x0, y0, x1, y1;
} sbot_box;

/* Domain (Sec. 2.3-2.4): nx0 * ny0 coarsest cells, multiples of `block`;
 * `levels` = m (1..8); square blocks of block * block cells of their own
 * level (8, 16 or 32); tau of the finest level, tau_l = 1/2 + (tau - 1/2) / 2^(m-1-l)
 * (acoustic scaling, Eq. 9); rho0 and u_in give the inlet state.
 * Refinement: the static boxes, plus (when a body is set) the body's marker
 * bounding box over one coarse step widened by refine_margin[l] on all sides
 * and refine_wake[l] on the +x side, for each level l = 1..m-1, then 2:1
 * balanced over faces and corners.  retag = 1 re-evaluates the body boxes
 * every coarse step and moves the refined region with the body.
 * Refinement must stay clear of non-periodic sides (SBOT_ERR_ARG). */
typedef struct {
    int nx0, ny0;
    int levels;
    int block;
    int bc[4];
    double tau_finest;
    double rho0;
    double u_in[2];
    int storage; /* sbot_storage */
    int ibm_iters; /* K of the multi-direct forcing (Sec. 2.2); 0 means 5 */
    int retag;
    double refine_margin[8];
    double refine_wake[8];
    int n_boxes;
    const sbot_box* boxes; /* read during sbot_create_domain only */
    /* collision: 0 BGK (Eq. 6); 1 multiple relaxation times (the MRT option
     * of Sec. 2.1): the D2Q9 moment basis (rho, e, eps, j_x, q_x, j_y, q_y,
     * p_xx, p_xy), the equilibrium moments of Eq. 7, Guo forcing in moment
     * space, the stress moments relaxed at 1 / tau_l (the viscosity of Eq. 9)
     * and e, eps, q at mrt_rates[0..2] (0 selects 1.64, 1.54, 1.9); 2 large-
     * eddy (the LES option of Sec. 2.1): BGK at tau_l + 3 nu_t with the
     * Smagorinsky viscosity nu_t = les_cs^2 |S| in each level's units, |S|
     * from the cell's non-equilibrium stress (0 selects les_cs = 0.17).  All
     * instances of a batch share the collision kind of the first one. */
    int collision;
    double mrt_rates[3];
    double les_cs;
    /* Walls and solids (the bounce-back family of Sec. 2.1 after Eq. 10,
     * whose formulas the paper leaves to its reference; half-way and
     * linearly interpolated bounce-back of Bouzidi et al.):
     * wall_velocity[2 s], [2 s + 1] is the velocity of side s (W, E, S, N)
     * when it is an SBOT_BC_WALL: the population that left a boundary cell
     * toward it returns reversed plus 2 w_i rho0 (c_i . u_w) / c_s^2.
     * solid_kind 1: a circle (solid[0], solid[1]) of radius solid[2], kind 2:
     * the half-plane y < solid[0] (finest units), on the finest level: cells
     * whose centre lies inside are solid (cell type 4, never updated, left
     * out of the checksum); a population whose streaming source is solid is
     * the interpolated bounce-back at the exact fraction t of the link
     * outside the solid: 2t f*_o(x) + (1 - 2t) f*_o(x + c_i) for t < 1/2
     * (when x + c_i is fluid), else f*_o(x) / 2t + (1 - 1/2t) f*_i(x).
     * A solid needs a static refinement (retag 0), no IBM body in the same
     * instance, and two finest interior cells of clearance around it. */
    double wall_velocity[8];
    int solid_kind;
    double solid[3];
} sbot_domain_desc;

/* Body (Sec. 2.2, Sec. 3.3-3.6).  Shapes, in the body frame (x along the
 * chord), with n_markers Lagrangian markers at equal arc length
 * (Delta s_b = perimeter / n):
 *   kind 0  circle of radius a
 *   kind 1  ellipse with semi-axes a (x) and b (y)
 *   kind 2  rectangle with half-sides a and b: a flat plate with square
 *           edges (Sec. 3.4)
 *   kind 3  symmetric NACA four-digit airfoil (Sec. 3.5) of chord 2a,
 *           leading edge at x = -a, thickness ratio b / a (b is about the
 *           maximum half-thickness), closed trailing edge
 * Kinematics, time t in finest steps; the body is rotated by alpha(t) about
 * `pivot` (body frame, relative to the centre):
 *   motion 0  static, alpha = alpha_mean
 *   motion 1  alpha = alpha_mean - alpha_amp sin(2 pi t / period + phase)
 *   motion 2  motion 1 plus the heave of Sec. 3.6 (Eqs. 25-27):
 *             centre = x0 + (heave_amp / 2) cos(2 pi t / period) (cos beta, sin beta)
 *   motion 3  pitch-up ramp (Sec. 3.4, Eqs. 20-21): alpha = alpha_mean - A G / max G
 *             with A = alpha_amp, a_s = ramp_as, K = ramp_rate,
 *             t1* = ramp_t1, t* = t / t_ref (t_ref: finest steps per c / U)
 *   motion 4  smoothed asymmetric triangular pitch (Sec. 3.5, Eqs. 22-24):
 *             amplitude alpha_amp, period `period`, asymmetry asym_xi in
 *             (0, 1), corner time accel_frac * period (at most
 *             min(xi, 1 - xi) / 2 of it), time shifted by phase period / (2 pi)
 * Motions 3 and 4 keep the centre at x0.  u_ref and l_ref scale the force
 * coefficients returned with the forces.  Fields a motion does not use are
 * ignored. */
typedef struct {
    int kind;
    double a, b;
    int n_markers;
    double pivot[2];
    int motion;
    double x0[2];
    double alpha_mean, alpha_amp, period, phase, heave_amp, stroke_beta;
    double u_ref, l_ref;
    double ramp_as, ramp_rate, ramp_t1, t_ref; /* motion 3 */
    double asym_xi, accel_frac;                /* motion 4 */
} sbot_body_desc;

/* Per-instance calls.  A context made by sbot_create_domain holds one
 * instance; a batch (below) holds many, and the calls that read or set one
 * instance's state (sbot_set_body_kinematics, sbot_set_fields,
 * sbot_set_populations, sbot_get_forces, sbot_get_fields,
 * sbot_get_populations, sbot_get_celltypes, sbot_get_topology,
 * sbot_get_checksum(_noalloc), sbot_get_level_info, sbot_get_work) address
 * the instance chosen by sbot_batch_select (initially slot 0).  They fail
 * with SBOT_ERR_STATE when that slot holds no live instance. */

/* Create a domain (one instance).  `cuda_stream` is a cudaStream_t; with
 * NULL the context creates and owns a non-blocking stream.  The initial state is the equilibrium at (rho0, u_in)
 * until sbot_set_fields / sbot_set_populations change it.
 * Errors: SBOT_ERR_ARG (bad description), SBOT_ERR_OOM, SBOT_ERR_CUDA. */
sbot_status sbot_create_domain(const sbot_domain_desc* desc, void* cuda_stream, sbot_ctx_t* out);

/* Set the immersed body (Sec. 2.2) before the first step; copies `desc`.
 * The refinement is rebuilt around the body.  Errors: SBOT_ERR_ARG (the
 * marker patch is too large for one thread block), SBOT_ERR_STATE (after
 * stepping). */
sbot_status sbot_set_body_kinematics(sbot_ctx_t ctx, const sbot_body_desc* desc);

/* Initial state of level `level`: f = f^eq(rho, u) (Eq. 7) on its interior
 * cells, from dense host arrays [ny_l][nx_l]; only before the first step. */
sbot_status sbot_set_fields(sbot_ctx_t ctx, int level, const double* rho, const double* ux, const double* uy);

/* Initial pre-collision populations of level `level`, dense host [9][ny_l][nx_l]. */
sbot_status sbot_set_populations(sbot_ctx_t ctx, int level, const double* f);

/* Advance n coarse steps (each = 2^(m-1) finest steps of an instance with m
 * levels) by the recursive sub-cycled time step of Algorithm 1, for every live
 * instance of the context at once.  Asynchronous on the context stream.
 * Every coarse step replays one of two CUDA graphs (one per buffer parity of
 * level 0), captured on first use and again only when the slot pool or a work
 * list outgrows its capacity; the graphs read the list lengths on the device,
 * so a re-tag or an admission usually replays without recapture.  The first
 * call of a context should therefore not itself be inside a stream capture.
 * Errors: SBOT_ERR_STATE when a body leaves the finest region or the
 * refinement reaches a non-periodic side, SBOT_ERR_CUDA. */
sbot_status sbot_step(sbot_ctx_t ctx, int n_coarse_steps);

/* Body force history (Eq. 16 and its moment about the pivot): one entry per
 * finest step not yet returned, oldest first: fx, fy, mz (FP64).  On input
 * *n_inout is the capacity of the arrays, on output the count written.
 * Synchronises.  Entries beyond the device history capacity (65536 per
 * call) are lost and reported as SBOT_ERR_STATE. */
sbot_status sbot_get_forces(sbot_ctx_t ctx, double* fx, double* fy, double* mz, int* n_inout);

/* rho and the velocity sum_i c_i f_i / rho of the canonical (pre-collision)
 * state of level `level`, dense host arrays [ny_l][nx_l]; cells that are not
 * interior to that level are 0.  *n_cells_inout: capacity in, nx_l * ny_l out. */
sbot_status sbot_get_fields(sbot_ctx_t ctx, int level, double* rho, double* ux, double* uy, int64_t* n_cells_inout);

/* Canonical pre-collision populations of level `level`, dense host
 * [9][ny_l][nx_l] in FP64 (non-interior cells 0). *n_inout: capacity in
 * elements, 9 * nx_l * ny_l out. */
sbot_status sbot_get_populations(sbot_ctx_t ctx, int level, double* f, int64_t* n_inout);

/* Cell kinds of level `level`, dense [ny_l][nx_l]: 0 none, 1 interior,
 * 2 fine-side halo, 3 coarse-side mailbox (Sec. 2.4). */
sbot_status sbot_get_celltypes(sbot_ctx_t ctx, int level, uint8_t* types, int64_t* n_inout);

/* Block states of level `level` on its block lattice [ny_l/B][nx_l/B]:
 * 0 absent, 1 leaf, 2 refined (Sec. 2.3, Fig. 2).  The origin of block
 * (bx, by) is (bx B, by B) cells of level `level`, so the lattice of states
 * gives every leaf's origin and level; no separate origin list is returned. */
sbot_status sbot_get_topology(sbot_ctx_t ctx, int level, uint8_t* states, int* n_blocks_inout);

/* Mass and momentum of the canonical state, sum over interior cells of all
 * levels weighted by the cell area in finest cells (FP64 on the device). */
sbot_status sbot_get_checksum(sbot_ctx_t ctx, double out3[3]);

/* Same result as sbot_get_checksum, for callers that cannot allocate device
 * memory: code whose device memory is fully reserved by another allocator
 * (for example a framework's caching pool), or latency-critical loops that
 * must not pay for cudaMalloc, which can synchronise the whole device.
 * sbot_get_checksum allocates its partial-sum buffer on first use; this call
 * allocates nothing: its partial sums go to one file-scope static device
 * array of the library, sized for 4096 thread-block partial sums (96 KB, held
 * by every GPU that loads the library until the process exits).  A domain
 * needs one partial sum per 256 interior cells of a level, at most 1024 per
 * level; one that needs more than 4096 in total is rejected with
 * SBOT_ERR_ARG (use sbot_get_checksum for it).  Every call looks up the
 * array's device address in the current device's context (the context's
 * device must be current: SBOT_ERR_STATE otherwise); the first call on a
 * device may load the library's device code there, so make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (several
 * contexts on different streams at once) race and must be serialised by the
 * caller.  The paper has no counterpart; this is a library service. */
sbot_status sbot_get_checksum_noalloc(sbot_ctx_t ctx, double out3[3]);

/* Level sizes: nx_l, ny_l, and the number of interior cells of the level. */
sbot_status sbot_get_level_info(sbot_ctx_t ctx, int level, int* nx, int* ny, int64_t* n_interior);

/* Cell updates per coarse step summed over levels (interior cells * 2^l),
 * and the fine-equivalent count (domain area in finest cells * 2^(m-1)). */
sbot_status sbot_get_work(sbot_ctx_t ctx, int64_t* cell_updates, int64_t* fine_equivalent);

/* Kernel timing of the hot path with CUDA events on the context stream.
 * sbot_set_profiling(ctx, mask): bit k enables kind k -- 0 fused
 * stream-collide, 1 coarse-to-fine halo copy, 2 fine-to-coarse merge (done
 * inside the coarse fused sweep, so it reports no launches of its own), 3 IBM;
 * 0 disables.  The events are recorded inside the step's CUDA graph (a new
 * mask recaptures it), which a profiled step captures on the context stream
 * alone: the kernels run one after another, so their times never overlap
 * (and add up to at most the profiled step); while enabled, sbot_step waits
 * for each coarse step to finish.  sbot_get_profile(ctx, kind, ...) returns launches, summed
 * device milliseconds and algorithmic bytes of that kind since profiling was
 * last enabled (the bytes each launch must move: 9 populations read and
 * written per interior or halo cell).  Kind 4 counts every kernel that
 * sbot_step launched (persistent step kernels, table-update and re-tag
 * kernels, the first collision, and the kernel nodes of each replayed step
 * graph) since the last sbot_set_profiling call, profiling on or off; its
 * milliseconds and bytes are 0.  While profiling is on, steps run as the
 * per-phase graphs (the persistent kernel has no per-kernel events). */
sbot_status sbot_set_profiling(sbot_ctx_t ctx, int mask);
sbot_status sbot_get_profile(sbot_ctx_t ctx, int kind, int64_t* launches, double* ms, double* bytes);

/* Phase trace of the persistent step kernel (SBOT_TUNE_PERSISTENT): with bit
 * 4 (16) of the profiling mask set, and no other bit, steps keep running as
 * the persistent kernel and each records, per phase of its list, when its
 * tasks started and ended (device time) and how many ran.
 * sbot_get_step_trace returns the last traced step: per phase its kind
 * (0 poses, 1 IBM geometry, 2 coarse-to-fine copy, 3 stream-collide sweep,
 * 4 IBM, 5 force sums), level, queue (1 bulk, 0 critical), tasks, and in
 * us4[4 p .. 4 p + 3] the first task's start, the last task's start, the
 * first task's end and the last task's end, in microseconds after the
 * launch's first thread block started (-1 for a phase that ran no task),
 * in list order.  *n_inout: capacity in phases in, phases out (SBOT_ERR_ARG
 * with the count when too small).  Synchronises.  Errors: SBOT_ERR_STATE (no
 * traced persistent step yet). */
sbot_status sbot_get_step_trace(sbot_ctx_t ctx, int* n_inout, int* kind, int* level, int* bulk, int* tasks,
                                double* us4);

/* Tuning knobs of a context (a library service; the paper has none).
 * SBOT_TUNE_VECTOR_MIN_CELLS: a fused stream-collide launch over at least this
 * many cells uses the vector kernel (4 cells per thread, 8 in 16-bit storage,
 * 16-byte-class loads; blocks of 16 or 32 only), a smaller one the one-cell-per-thread kernel;
 * negative = never the vector kernel.  Default 2^19.  Results agree to
 * rounding either way (so in a batch, whose launches list the cells of all
 * its instances, an instance equals itself run alone bit for bit when the
 * threshold is 0 or negative, and to rounding otherwise).  A change takes effect at the next sbot_step (which
 * recaptures its graphs).  Errors: SBOT_ERR_ARG (unknown parameter). */
#define SBOT_TUNE_VECTOR_MIN_CELLS 0
/* SBOT_TUNE_STAGED (0 or 1, default 0): the launches that take the vector
 * kernel use its variant that stages each block's populations and neighbour
 * rows in shared memory with bulk asynchronous copies (an mbarrier with a
 * bounded wait: a copy that never lands is reported as SBOT_ERR_TIMEOUT by
 * the next call that reads the device error word). */
#define SBOT_TUNE_STAGED 1
/* SBOT_TUNE_PDL (0 or 1; default 1 for a context of sbot_create_domain, 0
 * for a batch): consecutive kernels of a step on one stream use programmatic
 * dependent launch: a kernel may be scheduled while its predecessor still
 * runs and waits on the device until the predecessor has finished and its
 * writes are visible, which hides part of the launch gap between dependent
 * kernels.  In a busy batch the early blocks hold SMs that other instances'
 * kernels need, hence the different defaults. */
#define SBOT_TUNE_PDL 2
/* SBOT_TUNE_PERSISTENT (0 or 1; default 1 for a context of
 * sbot_create_domain, 0 for a batch): each coarse step runs as one
 * persistent, cooperatively launched kernel that walks the step's phases of
 * Algorithm 1 over every live instance (coarse-to-fine copies, the IBM, the
 * per-level sweeps, the force sums), each phase waiting on the device for
 * the phases it depends on; level-0 blocks that depend on nothing inside the
 * step fill the thread blocks that would otherwise wait.  0 (or a context
 * that profiles kernels, stages blocks with SBOT_TUNE_STAGED or holds a
 * solid obstacle) replays the per-phase CUDA graphs instead.  Each cell's
 * arithmetic is the same either way; results are equal bit for bit when
 * both take the same cell mapping (SBOT_TUNE_VECTOR_MIN_CELLS 0 or -1, or
 * blocks of 8), else to rounding. */
#define SBOT_TUNE_PERSISTENT 3
/* SBOT_TUNE_STEP_THREADS (0, 256 or 768; default 0): thread-block size of
 * the persistent kernel, which is also the number of threads that run one
 * body's IBM; 0 takes 256 when three blocks fit on an SM with the IBM's
 * shared memory, else 768 (FP64 storage always uses 256). */
#define SBOT_TUNE_STEP_THREADS 4
/* SBOT_TUNE_SPIN_NS (>= 0, default 10^9): the longest time, in nanoseconds
 * of device time, a thread block of the persistent kernel waits for a phase
 * it depends on.  Past it the launch stops (every thread block leaves at its
 * next decision) and the next call that reads the device error word returns
 * SBOT_ERR_TIMEOUT; the instances' state is then undefined. */
#define SBOT_TUNE_SPIN_NS 5
/* SBOT_TUNE_BULK_ROUNDS (1..64, default 8): thread-block fillings of blocks
 * per task of the persistent kernel's bulk queue, and of a critical sweep
 * that would otherwise hand out more than 8 tasks per thread block (fewer
 * tasks to hand out, coarser filling). */
#define SBOT_TUNE_BULK_ROUNDS 6
/* SBOT_TUNE_IBM_THREADS (256, 512, 768 or 1024; default 1024): threads of the
 * thread block that runs one body's multi-direct forcing in the per-phase
 * graphs (the persistent kernel runs it with its own block size,
 * SBOT_TUNE_STEP_THREADS).  Results are equal bit for bit either way. */
#define SBOT_TUNE_IBM_THREADS 7
/* SBOT_TUNE_CRIT_BLOCKS (0..64, default 0): blocks per task of the
 * persistent kernel's sweeps that other phases wait for (the level-0 blocks
 * that wait for nothing are the bulk queue, SBOT_TUNE_BULK_ROUNDS); 0 gives
 * each task as many blocks as fill its thread block.  Fewer blocks per task
 * spread a short sweep over more SMs.  Results are equal bit for bit either
 * way. */
#define SBOT_TUNE_CRIT_BLOCKS 8
/* SBOT_TUNE_STEPS_PER_LAUNCH (1..16, default 8): coarse steps one launch of
 * the persistent kernel runs when at least that many are asked for (fewer
 * launches, whose start and end cost some microseconds each, and the end of
 * one step overlaps the start of the next).  A launch still runs one step
 * when the host has work between steps: a traced step, or an instance whose
 * moving body changes its refinement footprint within them; and when the
 * phase list of several steps does not fit the kernel.  Results are equal
 * bit for bit either way. */
#define SBOT_TUNE_STEPS_PER_LAUNCH 9
/* SBOT_TUNE_VEC_WAVES (-1..64, default 8): thread blocks of a vector-kernel
 * launch, in waves of resident blocks (3 per SM): at most this many waves,
 * each block walking the launch's cell list with a grid stride; 0 or
 * negative = one block per 4 (8 in 16-bit storage) cells of each thread,
 * every block short-lived.  Fewer, longer-lived blocks sweep a large list
 * faster (less block launch and tail); short ones leave their SMs sooner to
 * launches running beside them.  Results are the same bit for bit.  Takes
 * effect at the next sbot_step.  Errors: SBOT_ERR_ARG (out of range). */
#define SBOT_TUNE_VEC_WAVES 10
sbot_status sbot_set_tuning(sbot_ctx_t ctx, int what, int64_t value);
sbot_status sbot_get_tuning(sbot_ctx_t ctx, int what, int64_t* value);

/* Host-only planning (no GPU needed): the block states of level `level`
 * ([ny_l/B][nx_l/B], 0 absent, 1 leaf, 2 refined) that sbot_create_domain
 * plus sbot_set_body_kinematics (body may be NULL) would build for the
 * coarse step [coarse_step, coarse_step + 1].  *n_inout: capacity in, count
 * out.  Errors: SBOT_ERR_ARG (bad description or capacity), SBOT_ERR_STATE
 * (refinement reaches a non-periodic side). */
sbot_status sbot_plan_blocks(const sbot_domain_desc* desc, const sbot_body_desc* body, int64_t coarse_step,
                             int level, uint8_t* states, int* n_inout);

/* ------------------------------------------------------------------------
 * Batches.  Many independent instances (each its own domain, refinement and
 * body, any sizes and level counts, one block size and storage kind) share
 * one slot pool and are advanced together by sbot_step: one launch per phase
 * of Algorithm 1 covers the blocks of every instance on that level, so small
 * instances fill the GPU together.  The paper runs one case per job; batching
 * is this library's extension of the same time step.
 * ------------------------------------------------------------------------ */

#define SBOT_MAX_INSTANCES 4096

/* An empty batch of up to `max_instances` (1..SBOT_MAX_INSTANCES) instances
 * with blocks of `block` cells (8, 16, 32) and storage `storage`.
 * `hbm_budget_bytes` (0 = no limit) bounds the device memory the instances
 * may hold: admissions that would exceed it are refused.  `cuda_stream` as
 * in sbot_create_domain.  Errors: SBOT_ERR_ARG, SBOT_ERR_OOM, SBOT_ERR_CUDA. */
sbot_status sbot_batch_create(int max_instances, int block, int storage, int64_t hbm_budget_bytes, void* cuda_stream,
                              sbot_ctx_t* out);

/* Admit an instance: `desc` as in sbot_create_domain (its block and storage
 * must be the batch's), `body` as in sbot_set_body_kinematics or NULL.  Its
 * state is the equilibrium at (rho0, u_in) and its own time starts at 0; it
 * joins the next sbot_step.  *slot receives its index (the lowest free one).
 * The budget check counts two population buffers for every block the
 * instance needs at time 0 (1.5 times as many when a moving body re-tags),
 * its body buffers and lattice maps, against what the live instances hold.
 * Errors: SBOT_ERR_ARG, SBOT_ERR_OOM (no free slot, over the budget, or a
 * failed allocation; the batch is unchanged), SBOT_ERR_STATE (refinement
 * reaches a non-periodic side). */
sbot_status sbot_batch_admit(sbot_ctx_t ctx, const sbot_domain_desc* desc, const sbot_body_desc* body, int* slot);

/* Advance every live instance of the batch by n coarse steps: the same call
 * as sbot_step on the batch context (each instance by its own 2^(m-1)
 * finest steps of Algorithm 1), under the name the batch calls use. */
sbot_status sbot_batch_step(sbot_ctx_t ctx, int n_coarse_steps);

/* Retire the instance in `slot`: its blocks and buffers return to the batch
 * at once (read its results first).  Errors: SBOT_ERR_ARG (no live instance). */
sbot_status sbot_batch_retire(sbot_ctx_t ctx, int slot);

/* Choose the instance the per-instance calls address.  Errors: SBOT_ERR_ARG. */
sbot_status sbot_batch_select(sbot_ctx_t ctx, int slot);

/* Live instances, device bytes they hold (population slots in use plus body
 * buffers and lattice maps), cell updates of one coarse step summed over them,
 * and the coarse steps the selected instance has taken (-1 if none is
 * selected).  Any pointer may be NULL.  Host only, no synchronisation. */
sbot_status sbot_batch_info(sbot_ctx_t ctx, int* live, int64_t* bytes_in_use, int64_t* cell_updates_per_step,
                            int64_t* coarse_steps_of_selected);

sbot_status sbot_destroy(sbot_ctx_t ctx);
const char* sbot_last_error(sbot_ctx_t ctx);

#ifdef __cplusplus
}
#endif
#endif /* SBOT_H */
