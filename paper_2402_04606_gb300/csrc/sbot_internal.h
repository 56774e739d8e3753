// Internal structures of the GB300 library (host and device).  Not part of the ABI.
//
// Data layout in HBM: every refinement level of every instance is a sparse
// set of B x B blocks living in ONE slot pool.  A slot holds the 9
// populations of its block as structure-of-arrays: f[slot][q][y][x]
// (q in the order of Eq. 1), in two ping-pong buffers.  A slot is one of
//   ST_INT  leaf block (Sec. 2.3): interior cells, collided and streamed;
//   ST_GF   fine-side halo block (Sec. 2.4): a block of this level inside a
//           coarser leaf, whose cells within 2 cells of the interior form the
//           two halo layers; filled by the coarse-to-fine copy, streamed, never
//           collided;
//   ST_GC   coarse-side mailbox block: a block of this level inside the finer
//           region; the cells next to the interior receive the merged fine
//           halo values that the coarse interior pulls (volumetric scheme).
// A 3x3 neighbour table per slot (self in the middle, periodic wrap applied,
// -1 outside the domain or where no block of that level exists) makes every
// pull a table lookup; per-(instance, level) lattice maps give the slot of
// any block position.
#pragma once
#include <cstdint>
#include <cstddef>

#define SBOT_MAXLEV 8
#define SBOT_HIST_CAP 65536

enum { ST_FREE = 0, ST_INT = 1, ST_GF = 2, ST_GC = 3 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { BCK_PERIODIC = 0, BCK_INLET = 1, BCK_OUTLET = 2, BCK_SYMMETRY = 3, BCK_WALL = 4 };
enum {
    SLOTF_EDGE = 1,    // block touches a non-periodic domain side
    SLOTF_MAILBOX = 2, // interior block with a neighbour inside the finer region
    SLOTF_SOLID = 4    // finest interior block within two cells of a solid obstacle
};

// device error word bits
enum {
    ERRB_STENCIL = 1,     // a marker stencil cell is not a finest interior cell
    ERRB_PATCH = 2,       // marker patch larger than its capacity
    ERRB_NOSOURCE = 4,    // an interior cell found no streaming source
    ERRB_HALO = 8,        // coalescence found no fine halo cell
    ERRB_NONFINITE = 16,  // NaN/Inf in a checksum
    ERRB_TIMEOUT = 32,    // a bounded device wait gave up (a bulk copy, or a dependency of the step kernel)
    ERRB_SCHED = 64,      // the step kernel's phase bookkeeping overflowed (an internal error)
};

// Per-instance constants (device copy in InstParams[]).
struct InstParams {
    int m;
    int nx0, ny0;
    int bc[4];
    int periodic_x, periodic_y;
    double tau[SBOT_MAXLEV];
    double rho0, uin_x, uin_y;
    float dref[9];  // 16-bit storage: f^eq_q(rho0, u_in) - w_q, the storage form's shift from the compute form
    int dref_on;    // some dref[q] is not zero
    const int* latmap;                  // this instance's lattice maps (all levels)
    long long latmap_off[SBOT_MAXLEV];  // offset of each level's map in `latmap`
    int nbx[SBOT_MAXLEV], nby[SBOT_MAXLEV];
    // body (Sec. 2.2); positions in finest units
    int has_body;
    int n_markers;
    const double* qx;  // body-frame marker coordinates (relative to the centre)
    const double* qy;
    int K;
    double ds;
    double pivot[2];
    int motion;
    double x0[2], alpha_mean, alpha_amp, period, phase, heave_amp, beta;
    double cos_mean, sin_mean;  // cos, sin of alpha_mean (static bodies skip the trigonometry)
    double cos_beta, sin_beta;  // of the stroke-plane angle
    double mrt_s[3];                            // MRT rates of e, eps, q (collision kind of the context)
    double les_cs;                              // Smagorinsky constant of the LES collision
    double uwall[4][2];                         // velocity of each wall side
    int solid;                                  // 0 none, 1 circle, 2 half-plane y < y0 (finest level)
    double sol[3];
    double ramp_as, ramp_rate, ramp_t1, t_ref;  // motion 3 (pitch-up ramp)
    double asym_xi, accel_frac;                 // motion 4 (triangular pitch)
    void* patch;     // force patch, compute type, [2][patch_cap]
    int patch_cap;   // cells of the force patch
    double* hist;    // force history ring, [SBOT_HIST_CAP][3]
    double* pose_tab;  // moving bodies: [pose_n][4] centre x, y, cos, sin of the pose at pose_k0 + i
    int pose_n;        // 2^(m-1) + 1 poses: every finest time of one coarse step and the next one
    void* ibm_cache;   // stored IBM geometry: one entry (static body) or pose_n - 1 entries (moving body)
    long long ibm_cache_stride;  // bytes per entry, ibm_cache_bytes()
    void* fterm;       // per-marker force terms of the coarse step's finest steps, compute type, [fterm_n][3][N]
    int fterm_n;       // 2^(m-1)
};

// Per-instance state written by kernels.
struct InstState {
    long long fine_step;  // IBM evaluations done (= finest collisions done)
    int patch_x0, patch_y0, patch_w, patch_h;
    long long pose_k0;    // finest time of pose_tab[0], -1 before the first table
    int ibm_cached;       // the IBM cache holds this body's geometry
    int pad;
};

// Everything a kernel needs, passed by value.
struct DevPool {
    int B;
    int mask_words;  // 32-bit words of a per-slot cell mask
    const int* nbr;  // [S][9]
    const int* slot_inst;
    const int* slot_level;
    const int* slot_type;
    const int* slot_ox;  // cell origin of the block at its level
    const int* slot_oy;
    const int* slot_flags;
    const int* slot_parent;  // ST_GF: parent slot (ST_INT, level - 1), else -1
    const int* slot_child;   // [S][4]: ST_INT: the slots of its 4 quarter blocks on level + 1 ((qy * 2 + qx)), else -1
    const unsigned* slot_mask;  // [S][mask_words]: halo / mailbox cells
    const InstParams* inst;
    InstState* ist;
    int* err;
    int pdl;   // host side: launch the step kernels with programmatic dependent launch
    int vec_waves;  // host side: waves of resident blocks in a vector-kernel launch (<= 0: one per chunk)
    // host side, picks the kernel variants at launch: the collision kind of
    // every instance (0 BGK, 1 MRT, 2 LES) in the low 4 bits, plus COLL_SOLID
    // when some instance holds a solid obstacle.  (One word: growing this
    // by-value kernel parameter measured 2 % slower on the vector kernel.)
    int coll;
};

// ---------------------------------------------------------------------------
// launch wrappers (kernels.cu)
// ---------------------------------------------------------------------------
typedef struct CUstream_st* sbot_stream_t;
constexpr int COLL_SOLID = 16;
// ... and COLL_SHIFT when some instance of the context has stored a 16-bit
// state shifted from the compute form (a free stream: InstParams::dref); the
// 8-cell kernel then takes its variant with the shift
constexpr int COLL_SHIFT = 32;

// storage kinds as in sbot.h
// Hot-path launches read their list length from device memory (*pn) and run
// over a fixed capacity `cap`, so a CUDA graph survives changes of the lists.
// A launch of n_hint blocks of at least vec_min_cells cells takes the vector
// kernel (4 cells per thread, 8 in 16-bit storage; B = 16 or 32), a smaller one the scalar kernel
// (one cell per thread); vec_min_cells < 0 never takes the vector kernel.
// allow_force = 0: the launch reads no IBM force (blocks known to lie outside
// every patch).
// ffine: the next finer level's buffer after its two sub-steps (read by the
// merge of populations streaming in from the finer region; unused on levels
// without a finer one).
// staged = 1: launches that take the vector path use the variant whose
// blocks' populations are staged in shared memory by bulk copies.
// fhalo (non-null, the buffer ffine points to): the launch's cells next to
// the finer region also write the post-collision values into the finer
// level's halo cells they contain (the coarse-to-fine copy of the next
// sub-step); such a launch takes the one-cell-per-thread kernel.
void launch_fused(int storage, const DevPool& P, const int* list, const int* pn, int cap, int n_hint,
                  long long vec_min_cells, int staged, const void* fin, void* fout, const void* ffine, int level,
                  sbot_stream_t s, int allow_force = 1, void* fhalo = nullptr);
void launch_collide_init(int storage, const DevPool& P, const int* list, int n, const void* fpre, void* fpost,
                         int level, sbot_stream_t s);
void launch_c2f(int storage, const DevPool& P, const int* list, const int* pn, int cap, const void* fcoarse,
                void* ffine, sbot_stream_t s);
// the poses of one coarse step of every moving body in an instance list (Sec. 3.6)
void launch_pose(const DevPool& P, const int* inst_list, const int* pn, int cap, sbot_stream_t s);
// deferred = 1: the force and moment (Eq. 16) are left as per-marker terms
// for launch_force_sum, which sums the `steps` finest steps of the coarse
// step just run
// threads: the thread block that runs one body (at most 1024)
void launch_ibm(int storage, const DevPool& P, const int* inst_list, const int* pn, int cap, const void* f,
                int level, int direct, size_t smem, sbot_stream_t s, int deferred = 0, int threads = 1024);
void launch_force_sum(int storage, const DevPool& P, const int* inst_list, const int* pn, int cap, int steps,
                      sbot_stream_t s);
void launch_ibm_geom(int storage, const DevPool& P, const int* inst_list, const int* pn, int cap, int steps,
                     size_t smem, sbot_stream_t s);
size_t ibm_smem_bytes(int storage, int patch_cap, int n_markers);
size_t ibm_smem_limit(int storage);  // largest dynamic shared memory k_ibm can launch with
size_t ibm_cache_bytes(int storage, int patch_cap, int n_markers);
void launch_export(int storage, const DevPool& P, const int* list, int n, const void* f, const void* ffine, int level,
                   int direct, int nx, double* dense, long long plane, int mode, sbot_stream_t s);
void launch_set_pre(int storage, const DevPool& P, const int* list, int n, void* f, int nx, const double* dense,
                    long long plane, int from_fields, sbot_stream_t s);
int checksum_blocks(int n_slots, int B);
void launch_checksum_partials(int storage, const DevPool& P, const int* list, int n, const void* f, const void* ffine,
                              int level, int direct, double weight, double* partials, int nblocks, sbot_stream_t s);
void launch_reduce_partials(const double* partials, int n, double* out3, int* err, sbot_stream_t s);
// re-tag transfer jobs, RETAG_JOB_INTS ints each: destination slot, kind (0
// copy of the covering coarser cell, 1 mean of the 4 children), 4 source
// slots (kind 0: source, levels up, unused, unused), source buffer,
// destination buffer, destination block origin x, y (own level), 2 unused
#define RETAG_JOB_INTS 12
void launch_retag(int storage, const DevPool& P, const int* jobs, int n, void* f0, void* f1, sbot_stream_t s);

// one int of a device table and the value to store there
struct ScatterRec {
    int* dst;
    int value;
    int pad;
};
void launch_scatter(const ScatterRec* recs, int n, sbot_stream_t s);
int storage_bytes(int storage);

// ---------------------------------------------------------------------------
// persistent step kernel (step_impl.cuh): one launch runs a whole coarse step
// of every live instance as a list of phases (Algorithm 1 unrolled).  Each
// phase is a work list cut into tasks of one thread block; a phase waits for
// the phases it depends on (counters of finished tasks).  Critical phases are
// taken in list order (a topological order); bulk phases (level-0 blocks that
// depend on nothing inside the step) fill thread blocks that would wait.
// ---------------------------------------------------------------------------
#define STEP_MAX_PHASES 512
#define STEP_MAX_DEPS 8
enum { PH_POSE = 0, PH_GEOM, PH_C2F, PH_FUSED, PH_IBM, PH_FSUM };
struct StepPhase {
    int kind;         // PH_*
    int bulk;         // 1: bulk queue (no dependencies); 0: critical queue
    int level;
    int allow_force;  // PH_FUSED: 0 when no block of the list meets a force patch
    int fin, fout, ffine;  // population buffers by index (0, 1), -1 none
    int list_off;     // the work list: offset in the device list array
    int count_idx;    // its length: index in the device count array
    int fold;         // PH_FUSED: its cells next to the finer region also write the finer level's halo (in ffine)
    int arg;          // PH_GEOM: finest step of the coarse step; PH_FSUM: finest steps per coarse step;
                      // PH_FUSED: 1 to keep one cell per thread (blocks whose pulls merge fine values)
    int ndep;
    int dep[STEP_MAX_DEPS];   // the phases this one waits for (all earlier; a bulk phase waits for none)
};
// The launch's control block, zero before a launch and set back to zero by
// the last thread block to leave.  Per phase: tasks taken and tasks finished
// (a phase may start once every phase it depends on has finished all its
// tasks).
struct StepCtl {
    int head;       // critical phases before this position (in the critical order) have no task left to take
    int bulk_next;  // bulk task cursor
    int abort, exited;
    int taken[STEP_MAX_PHASES];
    int done[STEP_MAX_PHASES];
};
struct StepArgs {
    const StepPhase* ph;
    int nph;
    StepCtl* ctl;
    const int* lists;
    const int* counts;
    void* f0;
    void* f1;
    long long vec_min_cells;  // fused phases of at least this many cells take the vector mapping
    long long spin_ns;        // longest wait for a dependency before the launch gives up (ERRB_TIMEOUT)
    int bulk_rounds;          // vector rounds per bulk task
    int crit_items;           // > 0: at most this many list items per task of a critical fused phase
    // phase trace (nullptr: off): device ns of each phase's first task start
    // and last task end, its task count, and the launch's first start
    // (start[STEP_MAX_PHASES])
    unsigned long long* tr_start;  // [STEP_MAX_PHASES + 1] first task start, set to all ones before the launch
    unsigned long long* tr_end;    // [STEP_MAX_PHASES] last task end, zero before the launch
    unsigned long long* tr_start2; // [STEP_MAX_PHASES] last task start, zero before the launch
    unsigned long long* tr_end1;   // [STEP_MAX_PHASES] first task end, all ones before the launch
    int* tr_tasks;                 // [STEP_MAX_PHASES], zero before the launch
};
// launch the step kernel for this storage kind (grid, threads and dynamic
// shared memory from step_config); returns the CUDA error code
int launch_step(int storage, const DevPool& P, const StepArgs& A, int grid, int threads, size_t smem,
                sbot_stream_t s);
// thread blocks per SM that fit with `threads` threads and `smem` bytes of
// dynamic shared memory (0 when the kernel cannot launch so), and the
// kernel's static shared memory
int step_occupancy(int storage, int B, int coll, int threads, size_t smem, size_t* static_smem);

// allocation-free checksum: capacity of the static scratch (partial sums)
#define SBOT_NOALLOC_MAX_PARTIALS 4096
double* noalloc_scratch();
