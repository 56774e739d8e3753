// C ABI of the GB300 library (declared in include/sbot.h): contexts holding
// one or many simulation instances in one shared slot pool, the recursive
// sub-cycled schedule of Algorithm 1, re-tagging, admission and state
// input/output.  Host code plans and launches; every step of the method runs
// in the kernels of kernels.cu.
//
// Host/device bookkeeping.  The host keeps mirrors of every device table
// (slot tables, lattice maps, work lists).  A change edits the mirror and
// marks the address dirty; once per frame (a coarse step, an admission, a
// retirement) the dirty addresses are resolved against the mirrors, staged
// in pinned memory and written by one scatter kernel, in stream order before
// the next launch that reads them.  Re-tagging a few moving bodies therefore
// costs a few kilobytes of transfers and never waits for the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sbot.h"
#include "kinematics.h"
#include "sbot_internal.h"
#include "topology.h"

namespace {

struct HostBody {
    int kind = 0;
    double a = 0, b = 0;
    int n = 0;
    std::vector<double> qx, qy;
    double ds = 0;
    double pivot[2] = {0, 0};
    int motion = 0;
    double x0[2] = {0, 0}, alpha_mean = 0, alpha_amp = 0, period = 1, phase = 0, heave_amp = 0, beta = 0;
    double u_ref = 1, l_ref = 1;
    double ramp_as = 0, ramp_rate = 0, ramp_t1 = 0, t_ref = 1, asym_xi = 0.5, accel_frac = 0;
};

// work lists kept per group and level over every live instance (a group is
// the instances with the same number of levels m; each group runs its own
// branch of the step's graph, so instances of different depths overlap):
//   FUSED  interior + fine-side halo blocks (one fused launch when not split)
//   GF     fine-side halo blocks (coarse-to-fine copy)
//   GC     coarse-side mailbox blocks (no launch of their own: the coarse
//          pull merges the fine values; the list keeps their membership)
//   INDEP  fused blocks that need neither a mailbox nor a force patch
//   DEP    the other interior blocks
//   IBM    instances whose finest level this is
// Lists are unordered: every block of a launch is independent of the others.
enum { LK_FUSED = 0, LK_GF, LK_GC, LK_INDEP, LK_DEP, LK_IBM, LK_COUNT };
constexpr int SLOT_KINDS = 5;  // kinds that hold slots; LK_IBM holds instances
constexpr int NGL = SBOT_MAXLEV * SBOT_MAXLEV;   // (group, level) pairs: gl = (m - 1) * SBOT_MAXLEV + level
constexpr int NLISTS = NGL * LK_COUNT;
inline int gl_of(int m, int level) { return (m - 1) * SBOT_MAXLEV + level; }

struct WorkList {
    std::vector<int> items;
    int cap = 0, off = 0;  // region [off, off + cap) of the device list array
    double units = 0;      // cells covered (IBM: patch cells), for the algorithmic bytes
    bool dirty = false;    // length changed since the last flush
};

// namespaces of marked addresses
enum { A_NBR = 0, A_INST, A_LEVEL, A_TYPE, A_OX, A_OY, A_FLAGS, A_PARENT, A_MASK, A_CHILD };
constexpr int A_LIST = 16;              // + gl * LK_COUNT + kind
constexpr int A_LAT = A_LIST + NLISTS;  // + instance
struct Dirty {
    int arr;
    long long idx;
    bool operator<(const Dirty& o) const { return arr != o.arr ? arr < o.arr : idx < o.idx; }
    bool operator==(const Dirty& o) const { return arr == o.arr && idx == o.idx; }
};

// pinned staging memory for one frame's host-to-device copies
struct Arena {
    char* host = nullptr;
    size_t cap = 0, used = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

struct Inst {
    bool live = false;
    sbot_domain_desc d{};
    std::vector<RefBox> static_boxes;
    int m = 1;
    bool has_body = false;
    HostBody body;
    TopoSpec ts;
    BlockStates bs;
    std::vector<PlannedBlock> planned;
    std::vector<int> slot_of;           // slot of every planned block
    std::vector<std::vector<int>> lat;  // per level, slot of each block position or -1
    std::vector<long long> box_sig;     // blocks met by the refinement boxes of the last plan
    InstParams ip{};
    size_t ibm_smem = 0;
    int* d_latmap = nullptr;
    long long latmap_n = 0;
    int* d_int = nullptr;  // this instance's interior slots, level after level
    long long int_cap = 0;
    int int_off[SBOT_MAXLEV] = {}, int_n[SBOT_MAXLEV] = {};
    double *d_qx = nullptr, *d_qy = nullptr;
    void* d_patch = nullptr;
    double* d_hist = nullptr;
    double* d_pose = nullptr;
    void* d_ibmcache = nullptr;
    void* d_fterm = nullptr;
    long long coarse_step = 0;  // this instance's own time
    long long forces_read = 0;
    bool finalized = false;
    long long extra_bytes = 0;  // device bytes besides its slots
};

}  // namespace

struct sbot_ctx {
    cudaStream_t s = nullptr;
    bool own_stream = false;
    int device = 0;
    std::string err;
    int storage = 1, B = 16, words = 8;
    long long budget = 0;  // device bytes the instances may hold, 0 = no limit
    std::vector<Inst> inst;
    int sel = 0;  // instance addressed by the per-instance calls
    unsigned groups = 0;  // bit m-1 set: some live instance has m levels
    unsigned moving = 0;  // bit m-1 set: such an instance has a moving body (its group needs pose tables)
    // slot pool and its host mirrors
    int cap = 0;
    std::vector<int> h_type, h_level, h_ox, h_oy, h_flags, h_parent, h_nbr, h_inst, h_child;
    std::vector<uint32_t> h_mask;
    std::vector<int> free_slots;
    void* f[2] = {nullptr, nullptr};
    int *d_nbr = nullptr, *d_inst = nullptr, *d_level = nullptr, *d_type = nullptr, *d_ox = nullptr, *d_oy = nullptr,
        *d_flags = nullptr, *d_parent = nullptr, *d_child = nullptr;
    unsigned* d_mask = nullptr;
    InstParams* d_ip = nullptr;
    InstState* d_ist = nullptr;
    int* d_err = nullptr;
    // work lists [gl * LK_COUNT + kind] and each slot's (for LK_IBM: instance's) membership
    WorkList wl[NLISTS];
    std::vector<int> lpos[LK_COUNT];  // position in its list, or -1
    std::vector<uint8_t> lmask;       // list kinds a slot belongs to
    std::vector<int8_t> llev;         // (group, level) of those lists
    std::vector<int> lunits;          // cells the slot covers
    bool lists_grow = false;
    int* d_lists = nullptr;
    int* d_counts = nullptr;            // list lengths, [NLISTS]
    size_t ibm_smem[SBOT_MAXLEV] = {};  // dynamic shared memory of each group's IBM launch (never shrinks)
    long long cap_version = 0;          // bumps whenever a captured graph would be stale
    long long vec_min_cells = 1LL << 19;  // tuning: smallest fused launch (cells) for the vector kernel
    int staged = 0;                       // tuning: vector launches stage the blocks in shared memory
    int pdl = 1;                          // tuning: programmatic dependent launch inside the step
    int coll = 0;                         // collision kind of the live instances (0 BGK, 1 MRT)
    // staged updates
    std::vector<Dirty> dirty;
    bool dirty_bad = false;  // a marked address fell outside its table (an internal error)
    Arena arena[2];
    int cur_arena = 0;
    ScatterRec* d_recs = nullptr;
    size_t recs_cap = 0;
    int* d_jobs = nullptr;
    size_t jobs_cap = 0;   // ints
    int* d_one = nullptr;  // a one-entry instance list and its length
    double* d_partials = nullptr;
    int partials_cap = 0;
    double* d_out3 = nullptr;
    // concurrency: a stream per group, and per (group, level) a side stream
    // for the blocks that need not wait (created when the group first appears)
    cudaStream_t gstream[SBOT_MAXLEV] = {};
    cudaEvent_t ev_gfork = nullptr, ev_gjoin[SBOT_MAXLEV] = {};
    cudaStream_t pstream[SBOT_MAXLEV] = {};  // per group: the poses of the coarse step, ahead of its IBM launches
    cudaEvent_t ev_pose[SBOT_MAXLEV] = {};
    cudaEvent_t ev_ibm_last[SBOT_MAXLEV] = {}, ev_fsum[SBOT_MAXLEV] = {};  // the step's force sums, off the chain
    int ibm_left[SBOT_MAXLEV] = {};  // IBM launches still to record in the coarse step being captured
    int gsub[SBOT_MAXLEV] = {};      // sub-steps of each level recorded so far in the group being captured
    cudaStream_t side[NGL] = {};
    cudaEvent_t ev_fork[NGL] = {}, ev_join[NGL] = {};
    // profiling: kinds 0 fused, 1 c2f, 2 f2c, 3 ibm
    int prof_mask = 0;
    bool capturing = false;
    struct Rec {
        int kind, gl, list;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    long long prof_n[4] = {};
    long long launch_n = 0;          // kernels launched by sbot_step since the last sbot_set_profiling
    int graph_kernels[2] = {0, 0};   // kernel nodes of each step graph
    double prof_ms[4] = {}, prof_bytes[4] = {};
    // CUDA graphs of one coarse step, one per parity of level 0
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long graph_version[2] = {-1, -1};
    int graph_mask[2] = {-1, -1};
    std::vector<Rec> graph_recs[2];
    // buffer parity per level, shared by all instances: at the start of every
    // coarse step, level l holds its post-collision state in f[par[l]]
    int par[SBOT_MAXLEV] = {};
    // the persistent step kernel: its phase lists (one per parity of level
    // 0), control block and launch shape
    int persist = 1;                  // tuning: run steps with the persistent kernel when the context allows
    int ibm_threads = 1024;           // tuning: thread block of one body's IBM in the per-phase graphs
    int step_threads = 0;             // tuning: its thread-block size (0: chosen from its shared memory)
    long long spin_ns = 1000000000;   // tuning: longest wait for a dependency inside a step (ns)
    int bulk_rounds = 8;              // tuning: vector rounds per bulk task
    int crit_items = 0;               // tuning: blocks per task of a critical sweep (0: fill the thread block)
    // phase lists of the persistent kernel: [parity of level 0 + 2 * (several steps)]
    StepPhase* d_ph[4] = {nullptr, nullptr, nullptr, nullptr};
    int nph[4] = {0, 0, 0, 0};
    int ph_steps[4] = {0, 0, 0, 0};   // coarse steps the list covers
    long long ph_version[4] = {-1, -1, -1, -1};
    bool ph_ok[4] = {false, false, false, false};  // the list fits the kernel (else the graph path runs)
    int steps_per_launch = 8;         // tuning: coarse steps per persistent launch
    int vec_waves = 8;                // tuning: waves of blocks in a vector-kernel launch
    bool shift_seen = false;          // an instance with a shifted 16-bit storage form has been admitted
    StepCtl* d_ctl = nullptr;
    unsigned long long* d_trace = nullptr;  // phase trace: starts [STEP_MAX_PHASES + 1], ends, task counts
    int trace_g = -1;                       // level-0 parity of the traced step, -1 none
    int step_T = 0, step_grid = 0;    // launch shape of the last phase list built
    size_t step_smem = 0;
};

namespace {

sbot_status fail(sbot_ctx* c, sbot_status st, const std::string& m) {
    if (c) c->err = m;
    return st;
}

#define CK(call)                                                                                               \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess) return fail(c, SBOT_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                       \
    do {                                \
        sbot_status st_ = (expr);       \
        if (st_ != SBOT_OK) return st_; \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

DevPool pool_view(sbot_ctx* c) {
    DevPool P;
    P.B = c->B;
    P.mask_words = c->words;
    P.nbr = c->d_nbr;
    P.slot_inst = c->d_inst;
    P.slot_level = c->d_level;
    P.slot_type = c->d_type;
    P.slot_ox = c->d_ox;
    P.slot_oy = c->d_oy;
    P.slot_flags = c->d_flags;
    P.slot_parent = c->d_parent;
    P.slot_child = c->d_child;
    P.slot_mask = c->d_mask;
    P.inst = c->d_ip;
    P.ist = c->d_ist;
    P.err = c->d_err;
    P.pdl = c->pdl;
    P.vec_waves = c->vec_waves;
    P.coll = c->coll;
    for (const Inst& I : c->inst)
        if (I.live && I.ip.solid != 0) P.coll |= COLL_SOLID;
    if (c->shift_seen) P.coll |= COLL_SHIFT;
    return P;
}

WorkList& W_of(sbot_ctx* c, int gl, int k) { return c->wl[gl * LK_COUNT + k]; }
const int* lptr(sbot_ctx* c, int gl, int k) { return c->d_lists + W_of(c, gl, k).off; }
const int* cptr(sbot_ctx* c, int gl, int k) { return c->d_counts + gl * LK_COUNT + k; }
const int* int_part(const Inst& I, int l) { return I.d_int + I.int_off[l]; }
size_t slot_bytes(const sbot_ctx* c) { return (size_t)9 * c->B * c->B * storage_bytes(c->storage); }

// ---------------------------------------------------------------------------
// staging
// ---------------------------------------------------------------------------

// pinned staging copy of `bytes` of `src` (16-byte aligned) in this frame's arena
sbot_status arena_put(sbot_ctx* c, const void* src, size_t bytes, const char** out) {
    Arena& a = c->arena[c->cur_arena];
    size_t at = (a.used + 15) & ~size_t(15);
    if (at + bytes > a.cap) {
        // copies from this arena may still be queued: let them run first
        CK(cudaStreamSynchronize(c->s));
        size_t ncap = std::max<size_t>(2 * (at + bytes), size_t(1) << 20);
        char* h = nullptr;
        CK(cudaHostAlloc((void**)&h, ncap, cudaHostAllocDefault));
        if (a.host) cudaFreeHost(a.host);
        a.host = h;
        a.cap = ncap;
        at = 0;
    }
    std::memcpy(a.host + at, src, bytes);
    a.used = at + bytes;
    *out = a.host + at;
    return SBOT_OK;
}

// asynchronous host-to-device copy through the staging memory
sbot_status upload(sbot_ctx* c, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return SBOT_OK;
    const char* p = nullptr;
    TRY(arena_put(c, src, bytes, &p));
    CK(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, c->s));
    return SBOT_OK;
}

// end of a frame: the next frame stages into the other arena once the copies
// queued from that arena (two frames ago) have run
sbot_status end_frame(sbot_ctx* c) {
    Arena& a = c->arena[c->cur_arena];
    if (a.used == 0) return SBOT_OK;  // nothing staged: keep filling this arena
    CK(cudaEventRecord(a.done, c->s));
    a.pending = true;
    c->cur_arena ^= 1;
    Arena& b = c->arena[c->cur_arena];
    if (b.pending) CK(cudaEventSynchronize(b.done));
    b.pending = false;
    b.used = 0;
    return SBOT_OK;
}

void mark(sbot_ctx* c, int arr, long long idx) { c->dirty.push_back({arr, idx}); }

// set one entry of a slot-table mirror; mark it when it changes
template <class T>
void set_tab(sbot_ctx* c, std::vector<T>& mirror, int arr, long long idx, T v) {
    if (mirror[idx] != v) {
        mirror[idx] = v;
        mark(c, arr, idx);
    }
}

// (re)allocate the device work lists with room to grow and upload them whole
sbot_status realloc_lists(sbot_ctx* c) {
    int off = 0;
    for (WorkList& W : c->wl) {
        int n = (int)W.items.size();
        if (n > W.cap) W.cap = n + n / 4 + 16;
        W.off = off;
        off += W.cap;
    }
    CK(cudaStreamSynchronize(c->s));
    dfree(c->d_lists);
    c->d_lists = nullptr;
    c->cap_version++;
    CK(dalloc(&c->d_lists, (size_t)off));
    std::vector<int> flat((size_t)off, -1), counts((size_t)NLISTS, 0);
    for (int i = 0; i < NLISTS; i++) {
        WorkList& W = c->wl[i];
        std::copy(W.items.begin(), W.items.end(), flat.begin() + W.off);
        counts[i] = (int)W.items.size();
        W.dirty = false;
    }
    TRY(upload(c, c->d_lists, flat.data(), flat.size() * sizeof(int)));
    TRY(upload(c, c->d_counts, counts.data(), counts.size() * sizeof(int)));
    c->lists_grow = false;
    return SBOT_OK;
}

// Write every marked address (its value taken from the mirror now, so an
// address marked twice gets its last value) and every changed list length,
// with one scatter launch.
sbot_status flush(sbot_ctx* c) {
    if (c->dirty_bad) {
        c->dirty_bad = false;
        c->dirty.clear();
        return fail(c, SBOT_ERR_STATE, "internal error: a table update fell outside its table");
    }
    if (c->lists_grow) TRY(realloc_lists(c));
    std::vector<Dirty>& D = c->dirty;
    std::sort(D.begin(), D.end());
    D.erase(std::unique(D.begin(), D.end()), D.end());
    std::vector<ScatterRec> recs;
    recs.reserve(D.size() + 16);
    bool bad = false;
    auto put = [&](int* base, long long len, long long idx, int v) {
        if (!base || idx < 0 || idx >= len) {
            bad = true;
            return;
        }
        recs.push_back({base + idx, v, 0});
    };
    const long long cap = c->cap;
    for (const Dirty& d : D) {
        const long long i = d.idx;
        switch (d.arr) {
            case A_NBR: put(c->d_nbr, cap * 9, i, c->h_nbr[i]); break;
            case A_INST: put(c->d_inst, cap, i, c->h_inst[i]); break;
            case A_LEVEL: put(c->d_level, cap, i, c->h_level[i]); break;
            case A_TYPE: put(c->d_type, cap, i, c->h_type[i]); break;
            case A_OX: put(c->d_ox, cap, i, c->h_ox[i]); break;
            case A_OY: put(c->d_oy, cap, i, c->h_oy[i]); break;
            case A_FLAGS: put(c->d_flags, cap, i, c->h_flags[i]); break;
            case A_PARENT: put(c->d_parent, cap, i, c->h_parent[i]); break;
            case A_MASK: put((int*)c->d_mask, cap * c->words, i, (int)c->h_mask[i]); break;
            case A_CHILD: put(c->d_child, cap * 4, i, c->h_child[i]); break;
            default:
                if (d.arr >= A_LIST && d.arr < A_LAT) {
                    const WorkList& W = c->wl[d.arr - A_LIST];
                    if (i < (long long)W.items.size()) put(c->d_lists + W.off, W.cap, i, W.items[i]);
                } else {
                    int ii = d.arr - A_LAT;
                    if (ii < 0 || ii >= (int)c->inst.size() || !c->inst[ii].live) break;  // retired since
                    const Inst& I = c->inst[ii];
                    int l = 0;
                    while (l + 1 < I.m && i >= I.ip.latmap_off[l + 1]) l++;
                    long long p = i - I.ip.latmap_off[l];
                    if (p < 0 || p >= (long long)I.lat[l].size()) {
                        bad = true;
                        break;
                    }
                    put(I.d_latmap, I.latmap_n, i, I.lat[l][p]);
                }
        }
    }
    for (int i = 0; i < NLISTS; i++) {
        WorkList& W = c->wl[i];
        if (!W.dirty) continue;
        put(c->d_counts, NLISTS, i, (int)W.items.size());
        W.dirty = false;
    }
    D.clear();
    if (bad) return fail(c, SBOT_ERR_STATE, "internal error: a table update fell outside its table");
    if (recs.empty()) return SBOT_OK;
    if (recs.size() > c->recs_cap) {
        CK(cudaStreamSynchronize(c->s));
        dfree(c->d_recs);
        c->d_recs = nullptr;
        c->recs_cap = 0;
        size_t ncap = std::max<size_t>(2 * recs.size(), 4096);
        CK(dalloc(&c->d_recs, ncap));
        c->recs_cap = ncap;
    }
    TRY(upload(c, c->d_recs, recs.data(), recs.size() * sizeof(ScatterRec)));
    launch_scatter(c->d_recs, (int)recs.size(), c->s);
    c->launch_n++;
    CK(cudaGetLastError());
    return SBOT_OK;
}

// ---------------------------------------------------------------------------
// work-list membership
// ---------------------------------------------------------------------------

void list_add(sbot_ctx* c, int gl, int k, int id, int units) {
    WorkList& W = W_of(c, gl, k);
    W.items.push_back(id);
    int p = (int)W.items.size() - 1;
    c->lpos[k][id] = p;
    W.units += units;
    W.dirty = true;
    if (p >= W.cap) c->lists_grow = true;
    else mark(c, A_LIST + gl * LK_COUNT + k, p);
}

void list_remove(sbot_ctx* c, int gl, int k, int id, int units) {
    WorkList& W = W_of(c, gl, k);
    int p = c->lpos[k][id];
    if (p < 0) return;
    int last = W.items.back();
    W.items[p] = last;
    c->lpos[k][last] = p;
    W.items.pop_back();
    c->lpos[k][id] = -1;
    W.units -= units;
    W.dirty = true;
    if (p < (int)W.items.size()) mark(c, A_LIST + gl * LK_COUNT + k, p);
}

// the lists a slot of `type` belongs to
uint8_t kinds_of(int type, bool dep) {
    if (type == ST_INT) return (uint8_t)((1 << LK_FUSED) | (1 << (dep ? LK_DEP : LK_INDEP)));
    if (type == ST_GF) return (uint8_t)((1 << LK_FUSED) | (1 << LK_GF) | (1 << LK_INDEP));
    if (type == ST_GC) return (uint8_t)(1 << LK_GC);
    return 0;
}

void set_membership(sbot_ctx* c, int sl, int gl, uint8_t want, int units) {
    const uint8_t have = c->lmask[sl];
    const int lev0 = c->llev[sl], u0 = c->lunits[sl];
    for (int k = 0; k < SLOT_KINDS; k++) {
        bool a = (have >> k) & 1, b = (want >> k) & 1;
        bool same_place = a && b && lev0 == gl;
        if (a && !same_place) list_remove(c, lev0, k, sl, u0);
        if (b && !same_place) list_add(c, gl, k, sl, units);
        if (same_place && units != u0) W_of(c, gl, k).units += units - u0;
    }
    c->lmask[sl] = want;
    c->llev[sl] = (int8_t)gl;
    c->lunits[sl] = units;
}

void free_slot(sbot_ctx* c, int sl) {
    set_membership(c, sl, 0, 0, 0);
    set_tab(c, c->h_type, A_TYPE, sl, (int)ST_FREE);
    c->free_slots.push_back(sl);
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------

// Sec. 3.4-3.6 kinematics, for planning on the host (the kernels evaluate it again)
void host_pose(const HostBody& b, double t, double& cx, double& cy, double& al) {
    al = b.alpha_mean;
    double hx = 0, hy = 0;
    if (b.motion == 1 || b.motion == 2)
        al = b.alpha_mean - b.alpha_amp * std::sin(2.0 * M_PI * t / b.period + b.phase);
    if (b.motion == 3)
        al = b.alpha_mean - sbot_kin::ramp_alpha(b.alpha_amp, b.ramp_as, b.ramp_rate, b.ramp_t1, t / b.t_ref);
    if (b.motion == 4)
        al = b.alpha_mean - sbot_kin::triangle_alpha(b.alpha_amp, b.asym_xi, b.accel_frac, b.period,
                                                     t + b.phase * b.period / (2.0 * M_PI));
    if (b.motion == 2) {
        double h = 0.5 * b.heave_amp * std::cos(2.0 * M_PI * t / b.period);
        hx = h * std::cos(b.beta);
        hy = h * std::sin(b.beta);
    }
    cx = b.x0[0] + hx;
    cy = b.x0[1] + hy;
}

// markers at equal arc length: the perimeter is the length of the polygon of
// 64 n vertices at equal parameter steps t_k = 2 pi k / (64 n) on
// (a cos t, b sin t); marker j sits at arc length j P / n, its parameter
// interpolated linearly inside the polygon edge that holds it.  A circle is
// placed at equal angles directly.
double place_markers(double a, double b, int n, std::vector<double>& qx, std::vector<double>& qy) {
    qx.resize(n);
    qy.resize(n);
    if (a == b) {
        for (int j = 0; j < n; j++) {
            double t = 2.0 * M_PI * j / n;
            qx[j] = a * std::cos(t);
            qy[j] = a * std::sin(t);
        }
        return 2.0 * M_PI * a;
    }
    const int M = 64 * n;
    std::vector<double> arc(M + 1, 0.0);
    for (int k = 0; k < M; k++) {
        double t0 = 2.0 * M_PI * k / M, t1 = 2.0 * M_PI * (k + 1) / M;
        double ex = a * std::cos(t1) - a * std::cos(t0), ey = b * std::sin(t1) - b * std::sin(t0);
        arc[k + 1] = arc[k] + std::sqrt(ex * ex + ey * ey);
    }
    double P = arc[M];
    int k = 0;
    for (int j = 0; j < n; j++) {
        double want = P * j / n;
        while (k < M - 1 && arc[k + 1] <= want) k++;
        double fr = (want - arc[k]) / (arc[k + 1] - arc[k]);
        double t = 2.0 * M_PI * (k + fr) / M;
        qx[j] = a * std::cos(t);
        qy[j] = b * std::sin(t);
    }
    return P;
}

// markers at equal arc length on a rectangle of half-sides a, b (a flat
// plate, Sec. 3.4), walking its perimeter 4a + 4b counter-clockwise from (a, 0)
double place_rectangle(double a, double b, int n, std::vector<double>& qx, std::vector<double>& qy) {
    qx.resize(n);
    qy.resize(n);
    const double P = 4.0 * a + 4.0 * b;
    const double edge[5] = {b, 2.0 * a, 2.0 * b, 2.0 * a, b};
    const double sx[5] = {a, a, -a, -a, a}, sy[5] = {0.0, b, b, -b, -b};  // edge starts
    const double dx[5] = {0, -1, 0, 1, 0}, dy[5] = {1, 0, -1, 0, 1};       // edge directions
    for (int j = 0; j < n; j++) {
        double s = P * j / n;
        int e = 0;
        while (e < 4 && s >= edge[e]) s -= edge[e++];
        qx[j] = sx[e] + dx[e] * s;
        qy[j] = sy[e] + dy[e] * s;
    }
    return P;
}

// symmetric NACA four-digit section (Sec. 3.5), chord 2a from the leading edge
// at -a, thickness ratio b / a, closed trailing edge: markers at equal arc
// length on the polygon of 64 n vertices through x = a cos t,
// y = +-c y_t((1 + cos t) / 2), upper surface for 0 < t < pi
double place_naca(double a, double b, int n, std::vector<double>& qx, std::vector<double>& qy) {
    qx.resize(n);
    qy.resize(n);
    const double th = b / a, c = 2.0 * a;
    auto point = [&](double t, double& x, double& y) {
        const double u = 0.5 * (1.0 + std::cos(t));
        const double yt = c * 5.0 * th *
                          (0.2969 * std::sqrt(u) - 0.1260 * u - 0.3516 * u * u + 0.2843 * u * u * u -
                           0.1036 * u * u * u * u);
        x = a * std::cos(t);
        y = std::sin(t) >= 0.0 ? yt : -yt;
    };
    const int M = 64 * n;
    std::vector<double> arc(M + 1, 0.0);
    double px = a, py = 0.0;
    for (int k = 0; k < M; k++) {
        double x, y;
        if (k + 1 == M) {
            x = a, y = 0.0;
        } else {
            point(2.0 * M_PI * (k + 1) / M, x, y);
        }
        arc[k + 1] = arc[k] + std::sqrt((x - px) * (x - px) + (y - py) * (y - py));
        px = x, py = y;
    }
    const double P = arc[M];
    int k = 0;
    for (int j = 0; j < n; j++) {
        const double want = P * j / n;
        while (k < M - 1 && arc[k + 1] <= want) k++;
        const double fr = (want - arc[k]) / (arc[k + 1] - arc[k]);
        point(2.0 * M_PI * (k + fr) / M, qx[j], qy[j]);
    }
    return P;
}

bool host_body_from_desc(const sbot_body_desc* b, HostBody& hb) {
    if (b->n_markers < 3 || b->n_markers > 8192 || b->a <= 0 || b->kind < 0 || b->kind > 3 ||
        (b->kind != 0 && !(b->b > 0)) || !(b->period > 0) || b->motion < 0 || b->motion > 4)
        return false;
    if (b->kind == 3 && !(b->b < b->a)) return false;
    if (b->motion == 3 && !(b->ramp_as > 0 && b->ramp_rate > 0 && b->t_ref > 0 && b->alpha_amp != 0)) return false;
    if (b->motion == 4) {
        const double xi = b->asym_xi, acc = b->accel_frac;
        if (!(xi > 0 && xi < 1 && acc > 0 && acc <= 0.5 * std::min(xi, 1.0 - xi))) return false;
    }
    hb.kind = b->kind;
    hb.a = b->a;
    hb.b = b->kind == 0 ? b->a : b->b;
    hb.n = b->n_markers;
    double P = hb.kind == 2   ? place_rectangle(hb.a, hb.b, hb.n, hb.qx, hb.qy)
               : hb.kind == 3 ? place_naca(hb.a, hb.b, hb.n, hb.qx, hb.qy)
                              : place_markers(hb.a, hb.b, hb.n, hb.qx, hb.qy);
    hb.ds = P / hb.n;  // Delta s_b = perimeter / n
    hb.pivot[0] = b->pivot[0];
    hb.pivot[1] = b->pivot[1];
    hb.motion = b->motion;
    hb.x0[0] = b->x0[0];
    hb.x0[1] = b->x0[1];
    hb.alpha_mean = b->alpha_mean;
    hb.alpha_amp = b->alpha_amp;
    hb.period = b->period;
    hb.phase = b->phase;
    hb.heave_amp = b->heave_amp;
    hb.beta = b->stroke_beta;
    hb.u_ref = b->u_ref;
    hb.l_ref = b->l_ref;
    hb.ramp_as = b->ramp_as;
    hb.ramp_rate = b->ramp_rate;
    hb.ramp_t1 = b->ramp_t1;
    hb.t_ref = b->t_ref;
    hb.asym_xi = b->asym_xi;
    hb.accel_frac = b->accel_frac;
    return true;
}

// refinement boxes of the coarse step [n, n+1]: static ones plus the body's
// marker bounding box over its finest steps, widened per level
void window_boxes(const Inst& I, long long n, std::vector<RefBox>& out) {
    out = I.static_boxes;
    if (!I.has_body) return;
    const HostBody& b = I.body;
    long long nf = 1LL << (I.m - 1);
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
    for (long long k = n * nf; k <= (n + 1) * nf; k++) {
        double cx, cy, al;
        host_pose(b, (double)k, cx, cy, al);
        double ca = std::cos(al), sa = std::sin(al);
        for (int j = 0; j < b.n; j++) {
            double px = b.qx[j] - b.pivot[0], py = b.qy[j] - b.pivot[1];
            double rx = cx + b.pivot[0] + ca * px - sa * py;
            double ry = cy + b.pivot[1] + sa * px + ca * py;
            mnx = std::min(mnx, rx);
            mxx = std::max(mxx, rx);
            mny = std::min(mny, ry);
            mxy = std::max(mxy, ry);
        }
        if (b.motion == 0) break;  // one pose
    }
    for (int l = 1; l < I.m; l++) {
        double g = I.d.refine_margin[l];
        if (g <= 0) continue;
        out.push_back({l, mnx - g, mny - g, mxx + g + I.d.refine_wake[l], mxy + g});
    }
}

// The planner splits a level-l block [bx s, (bx+1) s) when a box of a finer
// level overlaps it, so the blocks a box meets on level l run from
// floor(x0 / s) to ceil(x1 / s) - 1 (s a power of two: the divisions are
// exact).  Equal signatures give equal topologies, and the plan is skipped.
std::vector<long long> box_signature(const Inst& I, const std::vector<RefBox>& boxes) {
    std::vector<long long> sig;
    for (const RefBox& r : boxes)
        for (int l = 0; l + 1 < I.m; l++) {
            if (r.level <= l) continue;
            double side = (double)I.d.block * (double)(1 << (I.m - 1 - l));
            sig.push_back((long long)std::floor(r.x0 / side));
            sig.push_back((long long)std::ceil(r.x1 / side));
            sig.push_back((long long)std::floor(r.y0 / side));
            sig.push_back((long long)std::ceil(r.y1 / side));
        }
    return sig;
}

TopoSpec topo_spec(const Inst& I, int B) {
    TopoSpec ts;
    ts.m = I.m;
    ts.B = B;
    ts.nx0 = I.d.nx0;
    ts.ny0 = I.d.ny0;
    ts.periodic_x = I.d.bc[SIDE_W] == BCK_PERIODIC;
    ts.periodic_y = I.d.bc[SIDE_S] == BCK_PERIODIC;
    return ts;
}

int popcount_mask(const std::vector<uint32_t>& m) {
    int n = 0;
    for (uint32_t w : m) n += __builtin_popcount(w);
    return n;
}

// more slots: bigger population buffers (contents kept) and tables (uploaded whole)
sbot_status grow_pool(sbot_ctx* c, int need) {
    if (need <= c->cap) return SBOT_OK;
    const int ncap = std::max(need, c->cap + c->cap / 2);
    const size_t per = slot_bytes(c);
    void* nf[2] = {nullptr, nullptr};
    CK(cudaStreamSynchronize(c->s));
    for (int i = 0; i < 2; i++) {
        if (cudaMalloc(&nf[i], (size_t)ncap * per) != cudaSuccess) {
            cudaGetLastError();
            dfree(nf[0]);
            return fail(c, SBOT_ERR_OOM, "population pool allocation failed");
        }
        if (c->f[i]) CK(cudaMemcpyAsync(nf[i], c->f[i], (size_t)c->cap * per, cudaMemcpyDeviceToDevice, c->s));
    }
    CK(cudaStreamSynchronize(c->s));
    for (int i = 0; i < 2; i++) {
        dfree(c->f[i]);
        c->f[i] = nf[i];
    }
    for (int sl = ncap - 1; sl >= c->cap; sl--) c->free_slots.push_back(sl);
    c->h_type.resize(ncap, ST_FREE);
    c->h_level.resize(ncap, 0);
    c->h_ox.resize(ncap, 0);
    c->h_oy.resize(ncap, 0);
    c->h_flags.resize(ncap, 0);
    c->h_parent.resize(ncap, -1);
    c->h_inst.resize(ncap, 0);
    c->h_nbr.resize((size_t)ncap * 9, -1);
    c->h_child.resize((size_t)ncap * 4, -1);
    c->h_mask.resize((size_t)ncap * c->words, 0u);
    for (int k = 0; k < SLOT_KINDS; k++) c->lpos[k].resize(ncap, -1);
    c->lmask.resize(ncap, 0);
    c->llev.resize(ncap, 0);
    c->lunits.resize(ncap, 0);
    int** arrs[] = {&c->d_nbr,  &c->d_inst,  &c->d_level,  &c->d_type, &c->d_ox,
                    &c->d_oy,   &c->d_flags, &c->d_parent, &c->d_child};
    for (int** a : arrs) {
        dfree(*a);
        *a = nullptr;
    }
    dfree(c->d_mask);
    c->d_mask = nullptr;
    c->cap_version++;
    CK(dalloc(&c->d_nbr, (size_t)ncap * 9));
    CK(dalloc(&c->d_inst, ncap));
    CK(dalloc(&c->d_level, ncap));
    CK(dalloc(&c->d_type, ncap));
    CK(dalloc(&c->d_ox, ncap));
    CK(dalloc(&c->d_oy, ncap));
    CK(dalloc(&c->d_flags, ncap));
    CK(dalloc(&c->d_parent, ncap));
    CK(dalloc(&c->d_child, (size_t)ncap * 4));
    CK(dalloc(&c->d_mask, (size_t)ncap * c->words));
    c->cap = ncap;
    const size_t n = (size_t)ncap * sizeof(int);
    TRY(upload(c, c->d_nbr, c->h_nbr.data(), 9 * n));
    TRY(upload(c, c->d_inst, c->h_inst.data(), n));
    TRY(upload(c, c->d_level, c->h_level.data(), n));
    TRY(upload(c, c->d_type, c->h_type.data(), n));
    TRY(upload(c, c->d_ox, c->h_ox.data(), n));
    TRY(upload(c, c->d_oy, c->h_oy.data(), n));
    TRY(upload(c, c->d_flags, c->h_flags.data(), n));
    TRY(upload(c, c->d_parent, c->h_parent.data(), n));
    TRY(upload(c, c->d_child, c->h_child.data(), 4 * n));
    TRY(upload(c, c->d_mask, c->h_mask.data(), c->h_mask.size() * sizeof(uint32_t)));
    return SBOT_OK;
}

// Build (or rebuild) instance ii's blocks for its coarse step [n, n+1].  With
// `transfer`, interior blocks that stay keep their slot and state, and new
// interior blocks get the post-collision state of the old grid (reading R5):
// a copy of the covering coarser cell, or the mean of the 4 children.  The
// table changes are marked; the caller flushes them before the next step.
// Reading R15 on the host: the solid's extent, for the block flags and the
// clearance check (the kernels test the cells themselves)
bool host_in_solid(const InstParams& ip, double px, double py) {
    if (ip.solid == 1) {
        const double dx = px - ip.sol[0], dy = py - ip.sol[1];
        return dx * dx + dy * dy < ip.sol[2] * ip.sol[2];
    }
    if (ip.solid == 2) return py < ip.sol[0];
    return false;
}

// the solid's bounding box widened by `pad` finest cells (x0, y0, x1, y1)
void solid_box(const InstParams& ip, double pad, double* b) {
    if (ip.solid == 1) {
        b[0] = ip.sol[0] - ip.sol[2] - pad, b[1] = ip.sol[1] - ip.sol[2] - pad;
        b[2] = ip.sol[0] + ip.sol[2] + pad, b[3] = ip.sol[1] + ip.sol[2] + pad;
    } else {
        b[0] = -1e300, b[1] = -1e300, b[2] = 1e300, b[3] = ip.sol[0] + pad;
    }
}

bool solid_near_block(const InstParams& ip, int x0, int y0, int B) {
    if (ip.solid == 0) return false;
    double b[4];
    solid_box(ip, 2.0, b);
    return x0 < b[2] && b[0] < x0 + B && y0 < b[3] && b[1] < y0 + B;
}

// every cell within two cells of a solid cell is a finest interior cell (or
// solid) and inside the domain (a circle), under a static refinement
bool solid_clear(const InstParams& ip, int m, const BlockStates& bs, int B, bool px, bool py) {
    if (ip.solid == 0) return true;
    const int l = m - 1, nxl = ip.nx0 << l, nyl = ip.ny0 << l;
    double b[4];
    solid_box(ip, 0.0, b);
    const int x0 = std::max(0, (int)std::floor(b[0]) - 1), x1 = std::min(nxl - 1, (int)std::ceil(b[2]) + 1);
    const int y0 = std::max(0, (int)std::floor(b[1]) - 1), y1 = std::min(nyl - 1, (int)std::ceil(b[3]) + 1);
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) {
            if (!host_in_solid(ip, x + 0.5, y + 0.5)) continue;
            for (int dy = -2; dy <= 2; dy++)
                for (int dx = -2; dx <= 2; dx++) {
                    int wx = x + dx, wy = y + dy;
                    if (wx < 0 || wx >= nxl) {
                        if (!px) {
                            if (ip.solid == 1) return false;
                            continue;
                        }
                        wx = (wx + nxl) % nxl;
                    }
                    if (wy < 0 || wy >= nyl) {
                        if (!py) {
                            if (ip.solid == 1) return false;
                            continue;
                        }
                        wy = (wy + nyl) % nyl;
                    }
                    if (bs.at(l, wx / B, wy / B) != 1) return false;  // not a leaf block of the finest level
                }
        }
    return true;
}

sbot_status build_topology(sbot_ctx* c, int ii, long long n, bool transfer) {
    Inst& I = c->inst[ii];
    TopoSpec ts = topo_spec(I, c->B);
    window_boxes(I, n, ts.boxes);
    std::vector<long long> sig = box_signature(I, ts.boxes);
    if (transfer && !I.bs.s.empty() && sig == I.box_sig) return SBOT_OK;
    BlockStates bs;
    const char* why = nullptr;
    if (!plan_blocks(ts, bs, &why)) return fail(c, SBOT_ERR_STATE, why);
    if (!solid_clear(I.ip, I.m, bs, c->B, ts.periodic_x, ts.periodic_y))
        return fail(c, SBOT_ERR_ARG, "the solid must lie in the finest level with two interior cells of clearance");
    I.box_sig = sig;
    if (transfer && !I.bs.s.empty() && bs.s == I.bs.s) return SBOT_OK;
    std::vector<PlannedBlock> planned;
    plan_slots(ts, bs, planned);

    const bool have_old = transfer && !I.bs.s.empty();
    const BlockStates& old = I.bs;
    const std::vector<std::vector<int>>& old_lat = I.lat;

    // interior blocks that remain interior keep their slot
    std::vector<int> keep_slot(planned.size(), -1);
    std::vector<char> still_used(c->cap, 0);
    if (have_old) {
        for (size_t i = 0; i < planned.size(); i++) {
            const PlannedBlock& pb = planned[i];
            if (pb.type != ST_INT || old.at(pb.level, pb.bx, pb.by) != 1) continue;
            int sl = old_lat[pb.level][(size_t)pb.by * old.nbx[pb.level] + pb.bx];
            keep_slot[i] = sl;
            still_used[sl] = 1;
        }
    }
    // this instance's other old slots: halo and mailbox slots are free now;
    // interior slots after the transfer has been queued
    std::vector<int> release_after;
    for (int sl : I.slot_of) {
        if (still_used[sl]) continue;
        if (c->h_type[sl] == ST_INT && have_old) release_after.push_back(sl);
        else free_slot(c, sl);
    }
    int need_new = 0;
    for (size_t i = 0; i < planned.size(); i++)
        if (keep_slot[i] < 0) need_new++;
    if ((int)c->free_slots.size() < need_new) {
        int in_use = c->cap - (int)c->free_slots.size();
        TRY(grow_pool(c, in_use + need_new + 16));
    }
    std::sort(c->free_slots.begin(), c->free_slots.end(), std::greater<int>());
    std::vector<int> slot_of(planned.size());
    for (size_t i = 0; i < planned.size(); i++) {
        if (keep_slot[i] >= 0) {
            slot_of[i] = keep_slot[i];
        } else {
            slot_of[i] = c->free_slots.back();
            c->free_slots.pop_back();
        }
    }
    std::vector<std::vector<int>> lat(I.m);
    for (int l = 0; l < I.m; l++) lat[l].assign((size_t)bs.nbx[l] * bs.nby[l], -1);
    for (size_t i = 0; i < planned.size(); i++)
        lat[planned[i].level][(size_t)planned[i].by * bs.nbx[planned[i].level] + planned[i].bx] = slot_of[i];
    // transfer jobs for the new interior blocks
    std::vector<int> jobs;
    if (have_old) {
        for (size_t i = 0; i < planned.size(); i++) {
            const PlannedBlock& pb = planned[i];
            if (pb.type != ST_INT || keep_slot[i] >= 0) continue;
            int l = pb.level, ost = old.at(l, pb.bx, pb.by);
            int j[RETAG_JOB_INTS] = {};
            j[0] = slot_of[i];
            if (ost == 0) {  // was inside a coarser leaf
                int ll = l, bx = pb.bx, by = pb.by;
                while (ll > 0) {
                    ll--;
                    bx >>= 1;
                    by >>= 1;
                    if (old.at(ll, bx, by) == 1) break;
                }
                if (old.at(ll, bx, by) != 1) return fail(c, SBOT_ERR_STATE, "re-tag: no covering coarser block");
                j[1] = 0;
                j[2] = old_lat[ll][(size_t)by * old.nbx[ll] + bx];
                j[3] = l - ll;
                j[6] = c->par[ll];
            } else {  // was refined: mean of the children (one level down)
                j[1] = 1;
                for (int qd = 0; qd < 4; qd++) {
                    int cbx = 2 * pb.bx + (qd & 1), cby = 2 * pb.by + (qd >> 1);
                    if (l + 1 >= I.m || old.at(l + 1, cbx, cby) != 1)
                        return fail(c, SBOT_ERR_STATE, "re-tag changed a region by more than one level in one step");
                    j[2 + qd] = old_lat[l + 1][(size_t)cby * old.nbx[l + 1] + cbx];
                }
                j[6] = c->par[l + 1];
            }
            j[7] = c->par[l];
            j[8] = pb.bx * c->B;
            j[9] = pb.by * c->B;
            jobs.insert(jobs.end(), j, j + RETAG_JOB_INTS);
        }
    }
    // queue the transfer now: it reads old interior slots, whose table entries
    // are still the device's, and writes the new slots at the origins it carries
    if (!jobs.empty()) {
        if (jobs.size() > c->jobs_cap) {
            CK(cudaStreamSynchronize(c->s));
            dfree(c->d_jobs);
            c->d_jobs = nullptr;
            c->jobs_cap = 0;
            CK(dalloc(&c->d_jobs, 2 * jobs.size()));
            c->jobs_cap = 2 * jobs.size();
        }
        TRY(upload(c, c->d_jobs, jobs.data(), jobs.size() * sizeof(int)));
        DevPool P = pool_view(c);
        // at the start of a coarse step every level holds its post-collision state in f[par[l]]
        launch_retag(c->storage, P, c->d_jobs, (int)(jobs.size() / RETAG_JOB_INTS), c->f[0], c->f[1], c->s);
        c->launch_n++;
        CK(cudaGetLastError());
    }
    for (int sl : release_after) free_slot(c, sl);
    // slot tables
    const bool px = ts.periodic_x, py = ts.periodic_y;
    for (size_t i = 0; i < planned.size(); i++) {
        const PlannedBlock& pb = planned[i];
        const int sl = slot_of[i], l = pb.level;
        set_tab(c, c->h_type, A_TYPE, sl, pb.type);
        set_tab(c, c->h_level, A_LEVEL, sl, l);
        set_tab(c, c->h_inst, A_INST, sl, ii);
        set_tab(c, c->h_ox, A_OX, sl, pb.bx * c->B);
        set_tab(c, c->h_oy, A_OY, sl, pb.by * c->B);
        bool edge = (!px && (pb.bx == 0 || pb.bx == bs.nbx[l] - 1)) || (!py && (pb.by == 0 || pb.by == bs.nby[l] - 1));
        set_tab(c, c->h_flags, A_FLAGS, sl, edge ? (int)SLOTF_EDGE : 0);
        int parent = (pb.type == ST_GF) ? lat[l - 1][(size_t)(pb.by >> 1) * bs.nbx[l - 1] + (pb.bx >> 1)] : -1;
        set_tab(c, c->h_parent, A_PARENT, sl, parent);
        for (int qd = 0; qd < 4; qd++) {
            int ch = -1;
            if (pb.type == ST_INT && l + 1 < I.m)
                ch = lat[l + 1][(size_t)(2 * pb.by + (qd >> 1)) * bs.nbx[l + 1] + 2 * pb.bx + (qd & 1)];
            set_tab(c, c->h_child, A_CHILD, (long long)sl * 4 + qd, ch);
        }
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int x = pb.bx + dx, y = pb.by + dy, v = -1;
                bool inx = x >= 0 && x < bs.nbx[l], iny = y >= 0 && y < bs.nby[l];
                if (!inx && px) {
                    x = (x + bs.nbx[l]) % bs.nbx[l];
                    inx = true;
                }
                if (!iny && py) {
                    y = (y + bs.nby[l]) % bs.nby[l];
                    iny = true;
                }
                if (inx && iny) v = lat[l][(size_t)y * bs.nbx[l] + x];
                set_tab(c, c->h_nbr, A_NBR, (long long)sl * 9 + (dy + 1) * 3 + (dx + 1), v);
            }
        for (int w = 0; w < c->words; w++)
            set_tab(c, c->h_mask, A_MASK, (long long)sl * c->words + w, pb.mask[w]);
    }
    // lattice map: uploaded whole the first time, then by changed entries
    long long tot = 0;
    for (int l = 0; l < I.m; l++) {
        I.ip.latmap_off[l] = tot;
        I.ip.nbx[l] = bs.nbx[l];
        I.ip.nby[l] = bs.nby[l];
        tot += (long long)lat[l].size();
    }
    const bool first = I.d_latmap == nullptr;
    if (first) {
        CK(dalloc(&I.d_latmap, (size_t)tot));
        I.latmap_n = tot;
        std::vector<int> flat;
        flat.reserve(tot);
        for (int l = 0; l < I.m; l++) flat.insert(flat.end(), lat[l].begin(), lat[l].end());
        TRY(upload(c, I.d_latmap, flat.data(), tot * sizeof(int)));
    } else {
        for (int l = 0; l < I.m; l++)
            for (size_t p = 0; p < lat[l].size(); p++)
                if (lat[l][p] != old_lat[l][p]) mark(c, A_LAT + ii, I.ip.latmap_off[l] + (long long)p);
    }
    I.ip.latmap = I.d_latmap;
    if (first) TRY(upload(c, c->d_ip + ii, &I.ip, sizeof(InstParams)));
    // interior blocks that must wait: a mailbox neighbour (coarse side of an
    // interface), or, on the finest level, the force patch of the body (every
    // finest block for a moving body; the stencil box for a static one)
    int bx0 = 1 << 30, by0 = 1 << 30, bx1 = -(1 << 30), by1 = -(1 << 30);
    const bool static_body = I.has_body && I.body.motion == 0;
    if (static_body) {
        double cs = std::cos(I.body.alpha_mean), sn = std::sin(I.body.alpha_mean);
        for (int j = 0; j < I.body.n; j++) {
            double qx = I.body.qx[j] - I.body.pivot[0], qy = I.body.qy[j] - I.body.pivot[1];
            double rx = I.body.x0[0] + I.body.pivot[0] + cs * qx - sn * qy;
            double ry = I.body.x0[1] + I.body.pivot[1] + sn * qx + cs * qy;
            int i0 = (int)std::floor(rx - 0.5) - 1, j0 = (int)std::floor(ry - 0.5) - 1;
            bx0 = std::min(bx0, i0 - 1);
            by0 = std::min(by0, j0 - 1);
            bx1 = std::max(bx1, i0 + 4);
            by1 = std::max(by1, j0 + 4);
        }
    }
    std::vector<int> ints;
    for (int l = 0; l < I.m; l++) {
        I.int_off[l] = (int)ints.size();
        for (size_t i = 0; i < planned.size(); i++) {
            const PlannedBlock& pb = planned[i];
            if (pb.level != l) continue;
            const int sl = slot_of[i];
            bool dep = false;
            int units = c->B * c->B;
            if (pb.type == ST_INT) {
                ints.push_back(sl);
                for (int k = 0; k < 9; k++) {
                    int nb = c->h_nbr[(size_t)sl * 9 + k];
                    if (nb >= 0 && c->h_type[nb] == ST_GC) dep = true;
                }
                if (dep) set_tab(c, c->h_flags, A_FLAGS, sl, c->h_flags[sl] | (int)SLOTF_MAILBOX);
                if (l == I.m - 1 && solid_near_block(I.ip, pb.bx * c->B, pb.by * c->B, c->B))
                    set_tab(c, c->h_flags, A_FLAGS, sl, c->h_flags[sl] | (int)SLOTF_SOLID);
                if (l == I.m - 1 && I.has_body) {
                    int x0 = pb.bx * c->B, y0 = pb.by * c->B;
                    dep = dep || !static_body || (x0 <= bx1 && bx0 < x0 + c->B && y0 <= by1 && by0 < y0 + c->B);
                }
            } else {
                units = popcount_mask(pb.mask);
            }
            set_membership(c, sl, gl_of(I.m, l), kinds_of(pb.type, dep), units);
        }
        I.int_n[l] = (int)ints.size() - I.int_off[l];
    }
    // this instance's interior list (state input/output, first collision, checksum)
    if ((long long)ints.size() > I.int_cap) {
        CK(cudaStreamSynchronize(c->s));
        dfree(I.d_int);
        I.d_int = nullptr;
        I.int_cap = 0;
        long long ncap = (long long)ints.size() + (long long)ints.size() / 2 + 16;
        CK(dalloc(&I.d_int, (size_t)ncap));
        I.int_cap = ncap;
    }
    TRY(upload(c, I.d_int, ints.data(), ints.size() * sizeof(int)));
    I.ts = ts;
    I.bs = std::move(bs);
    I.planned = std::move(planned);
    I.slot_of = std::move(slot_of);
    I.lat = std::move(lat);
    return SBOT_OK;
}

// the deepest level, the IBM launch sizes: after an admission or a retirement
// the groups present, their streams and IBM launch sizes: after an admission
// or a retirement
sbot_status refresh_groups(sbot_ctx* c) {
    unsigned groups = 0, moving = 0;
    for (auto& I : c->inst)
        if (I.live) {
            const int g = I.m - 1;
            groups |= 1u << g;
            if (I.has_body && I.body.motion != 0) moving |= 1u << g;
            if (I.has_body && I.ibm_smem > c->ibm_smem[g]) {
                c->ibm_smem[g] = I.ibm_smem;
                c->cap_version++;
            }
        }
    // the chain of dependent launches (transfers, IBM, the blocks that wait)
    // runs at the highest stream priority, the independent blocks at the
    // lowest, so that the CTA scheduler serves the critical path first
    int prio_low = 0, prio_high = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
    for (int g = 0; g < SBOT_MAXLEV; g++) {
        if (!((groups >> g) & 1) || c->gstream[g]) continue;
        CK(cudaStreamCreateWithPriority(&c->gstream[g], cudaStreamNonBlocking, prio_high));
        CK(cudaEventCreateWithFlags(&c->ev_gjoin[g], cudaEventDisableTiming));
        CK(cudaStreamCreateWithPriority(&c->pstream[g], cudaStreamNonBlocking, prio_high));
        CK(cudaEventCreateWithFlags(&c->ev_pose[g], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_ibm_last[g], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_fsum[g], cudaEventDisableTiming));
        for (int l = 0; l <= g; l++) {
            const int gl = gl_of(g + 1, l);
            CK(cudaStreamCreateWithPriority(&c->side[gl], cudaStreamNonBlocking, prio_low));
            CK(cudaEventCreateWithFlags(&c->ev_fork[gl], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->ev_join[gl], cudaEventDisableTiming));
        }
    }
    if (groups != c->groups || moving != c->moving) {
        c->groups = groups;
        c->moving = moving;
        c->cap_version++;
    }
    return SBOT_OK;
}

// ---------------------------------------------------------------------------
// the time step
// ---------------------------------------------------------------------------

cudaEvent_t new_event() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// events around a launch recorded into the graph being captured (external
// record nodes); they live as long as the graph
struct ProfScope {
    sbot_ctx* c;
    int kind, gl, list;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(sbot_ctx* c_, int k, int gl_, int lk, cudaStream_t s_) : c(c_), kind(k), gl(gl_), list(lk), st(s_) {
        if (c->capturing && (c->prof_mask & (1 << kind))) {
            a = new_event();
            cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = new_event();
        cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
        c->pending.push_back({kind, gl, list, a, b});
    }
};

// algorithmic bytes of one launch over a list: an interior or halo cell reads
// and writes its 9 populations once; the IBM pulls its patch once (the GC
// entry counts the merge's 4 fine reads and one write for about 3 populations
// of each mailbox cell, for a launch that the merge inside the pull no longer
// makes)
double list_bytes(const sbot_ctx* c, int gl, int k) {
    const double sb = storage_bytes(c->storage), u = c->wl[gl * LK_COUNT + k].units;
    if (k == LK_GC) return u * 3.0 * 5.0 * sb;
    if (k == LK_IBM) return u * 9.0 * sb;
    return u * 18.0 * sb;
}

// events of one graph replay: read them once it has finished
void account(sbot_ctx* c, const std::vector<sbot_ctx::Rec>& recs) {
    for (auto& r : recs) cudaEventSynchronize(r.b);
    for (auto& r : recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        c->prof_n[r.kind]++;
        c->prof_ms[r.kind] += ms;
        c->prof_bytes[r.kind] += list_bytes(c, r.gl, r.list);
    }
}

void drop_graph(sbot_ctx* c, int g) {
    if (c->gexec[g]) cudaGraphExecDestroy(c->gexec[g]);
    c->gexec[g] = nullptr;
    for (auto& r : c->graph_recs[g]) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    c->graph_recs[g].clear();
}

// One substep of level l of every instance of group g (m = g + 1 levels) and,
// recursively, two of every finer level: Algorithm 1 with each stream+collide
// pair fused into one pull kernel, on the group's stream.  Blocks that need
// neither a finer level nor the IBM run on a side stream from the start of
// the substep.  Launch sizes are the list capacities; the kernels read the
// current lengths on the device.
void advance(sbot_ctx* c, const DevPool& P, int g, int l) {
    const int storage = c->storage, gl = gl_of(g + 1, l);
    // a profiled step is captured on the context stream alone, so that the
    // kernels' events never overlap (the per-kind times then add up)
    const bool serial = c->prof_mask != 0;
    cudaStream_t st = serial ? c->s : c->gstream[g], sd = serial ? c->s : c->side[gl];
    const WorkList& Wi = W_of(c, gl, LK_INDEP);
    const WorkList& Wd = W_of(c, gl, LK_DEP);
    const bool fork = Wi.cap > 0 && Wd.cap > 0 && sd;
    void* cur = c->f[c->par[l]];
    void* nxt = c->f[1 - c->par[l]];
    // the finer level's buffer after its two sub-steps: the coarse pull merges
    // the populations streaming in from the finer region from its halo cells
    void* fine = l < g ? c->f[c->par[l + 1]] : nullptr;
    // the coarse-to-fine copy of the first sub-step is its own launch; at the
    // later ones the previous sweep of this level, whose cells next to the
    // finer region own the copied values, writes the halo (fold)
    const int sub = c->gsub[l]++;
    void* fold = (l < g && sub + 1 < (1 << l)) ? fine : nullptr;
    if (fork) {
        if (!serial) {
            cudaEventRecord(c->ev_fork[gl], st);
            cudaStreamWaitEvent(sd, c->ev_fork[gl], 0);
        }
        {
            ProfScope ps(c, 0, gl, LK_INDEP, sd);
            launch_fused(storage, P, lptr(c, gl, LK_INDEP), cptr(c, gl, LK_INDEP), Wi.cap, Wi.cap, c->vec_min_cells, c->staged, cur,
                         nxt, fine, l, sd, 0);
        }
        if (!serial) cudaEventRecord(c->ev_join[gl], sd);
    }
    if (l < g) {
        const int glf = gl + 1;  // the next finer level of the same group
        if (sub == 0) {
            ProfScope ps(c, 1, glf, LK_GF, st);
            launch_c2f(storage, P, lptr(c, glf, LK_GF), cptr(c, glf, LK_GF), W_of(c, glf, LK_GF).cap, cur,
                       c->f[c->par[l + 1]], st);
        }
        advance(c, P, g, l + 1);
        advance(c, P, g, l + 1);
    }
    const WorkList& Wb = W_of(c, gl, LK_IBM);
    if (Wb.cap > 0) {
        if ((c->moving >> g) & 1) cudaStreamWaitEvent(st, c->ev_pose[g], 0);
        {
            ProfScope ps(c, 3, gl, LK_IBM, st);
            launch_ibm(storage, P, lptr(c, gl, LK_IBM), cptr(c, gl, LK_IBM), Wb.cap, cur, l, 0, c->ibm_smem[g], st, 1,
                       c->ibm_threads);
        }
        if (--c->ibm_left[g] == 0) {  // the coarse step's last IBM: its force sums run beside the rest
            cudaStream_t sp = serial ? st : c->pstream[g];
            cudaEventRecord(c->ev_ibm_last[g], st);
            cudaStreamWaitEvent(sp, c->ev_ibm_last[g], 0);
            launch_force_sum(storage, P, lptr(c, gl, LK_IBM), cptr(c, gl, LK_IBM), Wb.cap, 1 << g, sp);
            cudaEventRecord(c->ev_fsum[g], sp);
        }
    }
    if (fork) {
        {
            // below the finest level these are the blocks next to the finer
            // region: their pulls merge fine values cell by cell, so they take
            // the one-cell-per-thread kernel whatever their number
            ProfScope ps(c, 0, gl, LK_DEP, st);
            launch_fused(storage, P, lptr(c, gl, LK_DEP), cptr(c, gl, LK_DEP), Wd.cap, Wd.cap,
                         l < g ? -1 : c->vec_min_cells, c->staged, cur, nxt, fine, l, st, 1, fold);
        }
        if (!serial) cudaStreamWaitEvent(st, c->ev_join[gl], 0);
    } else {
        const WorkList& Wf = W_of(c, gl, LK_FUSED);
        ProfScope ps(c, 0, gl, LK_FUSED, st);
        launch_fused(storage, P, lptr(c, gl, LK_FUSED), cptr(c, gl, LK_FUSED), Wf.cap, Wf.cap,
                     l < g ? -1 : c->vec_min_cells, c->staged, cur, nxt, fine, l, st, 1, fold);
    }
    c->par[l] ^= 1;
}

// one coarse step of every group, each on its own stream, forked from and
// joined back into the context stream
void advance_all(sbot_ctx* c) {
    const DevPool P = pool_view(c);
    int saved[SBOT_MAXLEV];
    std::memcpy(saved, c->par, sizeof saved);
    cudaEventRecord(c->ev_gfork, c->s);
    const bool serial = c->prof_mask != 0;  // a profiled step: everything on the context stream
    for (int g = 0; g < SBOT_MAXLEV; g++) {
        if (!((c->groups >> g) & 1)) continue;
        std::memcpy(c->par, saved, sizeof saved);
        cudaStream_t gs = serial ? c->s : c->gstream[g], ps = serial ? c->s : c->pstream[g];
        if (!serial) cudaStreamWaitEvent(gs, c->ev_gfork, 0);
        const int glb = gl_of(g + 1, g);  // the group's finest level holds its bodies
        if (W_of(c, glb, LK_IBM).cap > 0 && ((c->moving >> g) & 1)) {
            if (!serial) cudaStreamWaitEvent(ps, c->ev_gfork, 0);
            launch_pose(P, lptr(c, glb, LK_IBM), cptr(c, glb, LK_IBM), W_of(c, glb, LK_IBM).cap, ps);
            // the IBM geometry of every finest step of this coarse step, ahead of the IBM launches
            launch_ibm_geom(c->storage, P, lptr(c, glb, LK_IBM), cptr(c, glb, LK_IBM), W_of(c, glb, LK_IBM).cap,
                            1 << g, c->ibm_smem[g], ps);
            cudaEventRecord(c->ev_pose[g], ps);
        }
        const bool bodies = W_of(c, glb, LK_IBM).cap > 0;
        c->ibm_left[g] = bodies ? 1 << g : -1;
        std::memset(c->gsub, 0, sizeof c->gsub);
        advance(c, P, g, 0);
        if (!serial) {
            if (bodies) cudaStreamWaitEvent(gs, c->ev_fsum[g], 0);
            cudaEventRecord(c->ev_gjoin[g], gs);
            cudaStreamWaitEvent(c->s, c->ev_gjoin[g], 0);
        }
    }
    std::memcpy(c->par, saved, sizeof saved);
}

// ---------------------------------------------------------------------------
// the persistent step: Algorithm 1 as a phase list for the step kernel
// ---------------------------------------------------------------------------

// The phases of one coarse step of group g (its instances have m = g + 1
// levels), in the order of Algorithm 1 as advance() launches them, each with
// the phases it must wait for:
//   coarse-to-fine copy into level l+1: the last sweep of level l (the coarse
//     post-collision state it copies, and the merge that read the halo it
//     overwrites);
//   IBM of a finest sub-step: the level's previous sweep (the pre-collision
//     state it pulls) and, for a moving body, the geometry of that step;
//   sweep of level l, blocks needing no finer level and no force (A): the
//     level's previous sweep (neighbours; the buffer it overwrites) and the
//     copy into level l (halo cells);
//   the other blocks (B): the same, plus the IBM of the sub-step and the two
//     sweeps of level l+1 (whose halo values the coarse pull merges).
struct PhaseEmit {
    sbot_ctx* c;
    int g;
    std::vector<StepPhase> ph;
    int lastA[SBOT_MAXLEV], lastB[SBOT_MAXLEV], c2f_into[SBOT_MAXLEV], par[SBOT_MAXLEV], sub[SBOT_MAXLEV];
    int last_ibm = -1, n_ibm = 0;
    int prev_fsum = -1;  // the previous coarse step's force sums (their term slots are the next IBMs')
    bool bodies = false, moving = false;
    std::vector<int> geom;

    int add(int kind, int level, int gl, int lk, std::initializer_list<int> deps, int fin = -1, int fout = -1,
            int ffine = -1, int allow_force = 0, int arg = 0) {
        const WorkList& W = W_of(c, gl, lk);
        if (W.cap <= 0) return -1;
        StepPhase p{};
        p.kind = kind;
        p.bulk = 0;
        p.level = level;
        p.allow_force = allow_force;
        p.fin = fin;
        p.fout = fout;
        p.ffine = ffine;
        p.list_off = W.off;
        p.count_idx = gl * LK_COUNT + lk;
        p.arg = arg;
        p.fold = 0;
        p.ndep = 0;
        for (int d : deps)
            if (d >= 0) {
                bool dup = false;
                for (int k = 0; k < p.ndep; k++) dup |= p.dep[k] == d;
                if (!dup && p.ndep < STEP_MAX_DEPS) p.dep[p.ndep++] = d;
            }
        ph.push_back(p);
        return (int)ph.size() - 1;
    }

    void adv(int l) {
        const int gl = gl_of(g + 1, l);
        const int cur = par[l], nxt = 1 - par[l], fine = l < g ? par[l + 1] : -1;
        const bool fork = W_of(c, gl, LK_INDEP).cap > 0 && W_of(c, gl, LK_DEP).cap > 0;
        const int s = sub[l]++;                    // this level's sub-step within the coarse step
        const bool fold = l < g && s + 1 < (1 << l);  // a later sub-step of this level follows
        if (l < g) {
            // the halo of level l+1: copied at the first sub-step, written by
            // this level's previous sweep (fold) at the others
            if (s == 0) c2f_into[l + 1] = add(PH_C2F, l + 1, gl + 1, LK_GF, {lastA[l], lastB[l]}, cur, par[l + 1]);
            adv(l + 1);
            adv(l + 1);
        }
        int ibm = -1;
        if (l == g && bodies) {
            ibm = add(PH_IBM, l, gl, LK_IBM,
                      {lastA[l], lastB[l], moving ? geom[n_ibm] : -1, n_ibm == 0 ? prev_fsum : -1}, cur);
            n_ibm++;
            last_ibm = ibm;
        }
        const int c2 = l > 0 ? c2f_into[l] : -1;
        const int fa = l < g ? lastA[l + 1] : -1, fb = l < g ? lastB[l + 1] : -1;
        int A = -1, Bp;
        if (fork) {
            A = add(PH_FUSED, l, gl, LK_INDEP, {lastA[l], lastB[l], c2}, cur, nxt, fine, 0);
            Bp = add(PH_FUSED, l, gl, LK_DEP, {lastA[l], lastB[l], c2, ibm, fa, fb}, cur, nxt, fine, 1,
                     l < g ? 1 : 0);  // next to the finer region: one cell per thread
        } else {
            Bp = add(PH_FUSED, l, gl, LK_FUSED, {lastA[l], lastB[l], c2, ibm, fa, fb}, cur, nxt, fine, 1,
                     l < g ? 1 : 0);
        }
        if (fold && Bp >= 0) {
            ph[Bp].fold = 1;
            c2f_into[l + 1] = Bp;  // the next fine sub-steps read the halo it writes
        }
        lastA[l] = A;
        lastB[l] = Bp;
        par[l] ^= 1;
    }

    // `steps` coarse steps in a row: a step's phases wait for the previous
    // step's by the same rules as a level's sub-steps; besides, a moving
    // body's poses of the next step wait for this step's last IBM (which
    // comes after every reader of the poses and geometries), and the next
    // step's first IBM waits for this step's force sums (which read the
    // per-step terms it overwrites and the step counter it advances)
    void run(int steps) {
        for (int l = 0; l < SBOT_MAXLEV; l++) lastA[l] = lastB[l] = c2f_into[l] = -1;
        const int glb = gl_of(g + 1, g);
        bodies = W_of(c, glb, LK_IBM).cap > 0;
        moving = bodies && ((c->moving >> g) & 1);
        for (int k = 0; k < steps; k++) {
            for (int l = 0; l < SBOT_MAXLEV; l++) sub[l] = 0;
            n_ibm = 0;
            geom.clear();
            if (moving) {
                const int pose = add(PH_POSE, g, glb, LK_IBM, {last_ibm});
                for (int i = 0; i < (1 << g); i++)
                    geom.push_back(add(PH_GEOM, g, glb, LK_IBM, {pose}, -1, -1, -1, 0, i));
            }
            adv(0);
            if (bodies) prev_fsum = add(PH_FSUM, g, glb, LK_IBM, {last_ibm}, -1, -1, -1, 0, 1 << g);
        }
    }
};

// Every group's phases of `steps` coarse steps merged into one list: a
// group's phases keep their order, and groups interleave by their position
// along their own steps (deeper groups first at equal position), so that
// every group's chain of dependent phases advances from the start.  Level-0
// sweeps that wait for nothing go to the bulk queue.  Returns false when the
// list does not fit the kernel's limits.
bool build_step_phases(sbot_ctx* c, std::vector<StepPhase>& out, int steps) {
    struct Ref {
        double key;
        int g, i;
    };
    std::vector<PhaseEmit> em;
    std::vector<Ref> order;
    for (int g = SBOT_MAXLEV - 1; g >= 0; g--) {
        if (!((c->groups >> g) & 1)) continue;
        PhaseEmit e;
        e.c = c;
        e.g = g;
        std::memcpy(e.par, c->par, sizeof e.par);
        e.run(steps);
        em.push_back(std::move(e));
    }
    for (int k = 0; k < (int)em.size(); k++) {
        const int n = (int)em[k].ph.size();
        for (int i = 0; i < n; i++) order.push_back({(i + 0.5) / n, k, i});
    }
    std::stable_sort(order.begin(), order.end(), [](const Ref& a, const Ref& b) { return a.key < b.key; });
    if (order.empty() || order.size() > STEP_MAX_PHASES) return false;
    std::vector<std::vector<int>> where(em.size());
    for (size_t k = 0; k < em.size(); k++) where[k].assign(em[k].ph.size(), -1);
    out.clear();
    for (const Ref& r : order) {
        where[r.g][r.i] = (int)out.size();
        StepPhase p = em[r.g].ph[r.i];
        for (int k = 0; k < p.ndep; k++) p.dep[k] = where[r.g][p.dep[k]];
        p.bulk = (p.kind == PH_FUSED && p.level == 0 && p.ndep == 0) ? 1 : 0;
        out.push_back(p);
    }
    // every dependency is an earlier phase and only critical phases have any
    // (what the kernel's progress guarantee rests on: bulk tasks never wait)
    for (size_t i = 0; i < out.size(); i++)
        for (int k = 0; k < out[i].ndep; k++) {
            const int d = out[i].dep[k];
            if (d < 0 || d >= (int)i || out[i].bulk) return false;
        }
    return true;
}

// The launch shape of the step kernel: 256 threads per block when three
// blocks fit on an SM with the IBM's shared memory, else 768 (one block);
// FP64 always 256.  Returns false when it cannot launch.
bool step_launch_shape(sbot_ctx* c, int& T, int& grid, size_t& smem) {
    size_t need = 0;
    for (int g = 0; g < SBOT_MAXLEV; g++)
        if ((c->groups >> g) & 1) need = std::max(need, c->ibm_smem[g]);
    smem = (need + 15) & ~(size_t)15;
    const int coll = pool_view(c).coll;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return false;
    }
    size_t st = 0;
    auto occ = [&](int t) { return step_occupancy(c->storage, c->B, coll, t, smem, &st); };
    if (c->storage == 0) {
        T = 256;
    } else if (c->step_threads == 256 || c->step_threads == 768) {
        T = c->step_threads;
    } else {
        T = occ(256) >= 3 ? 256 : 768;
    }
    const int per_sm = occ(T);
    if (per_sm <= 0) return false;
    grid = per_sm * sms;
    return true;
}

// the phase list of `steps` coarse steps from level-0 parity g, in list slot
// g + 2 * (steps > 1), uploaded (rebuilt when a list moved or grew, the groups
// changed or the step count changed)
sbot_status ensure_step_phases(sbot_ctx* c, int g, int steps) {
    const int k = g + (steps > 1 ? 2 : 0);
    if (c->ph_version[k] == c->cap_version && c->ph_steps[k] == steps) return SBOT_OK;
    c->ph_version[k] = c->cap_version;
    c->ph_steps[k] = steps;
    c->ph_ok[k] = false;
    std::vector<StepPhase> ph;
    if (!build_step_phases(c, ph, steps)) return SBOT_OK;
    int T = 0, grid = 0;
    size_t smem = 0;
    if (!step_launch_shape(c, T, grid, smem)) return SBOT_OK;
    if (!c->d_ph[k]) CK(dalloc(&c->d_ph[k], (size_t)STEP_MAX_PHASES));
    if (!c->d_ctl) {
        CK(dalloc(&c->d_ctl, 1));
        CK(cudaMemsetAsync(c->d_ctl, 0, sizeof(StepCtl), c->s));
    }
    TRY(upload(c, c->d_ph[k], ph.data(), ph.size() * sizeof(StepPhase)));
    c->nph[k] = (int)ph.size();
    c->step_T = T;
    c->step_grid = grid;
    c->step_smem = smem;
    c->ph_ok[k] = true;
    return SBOT_OK;
}

// whether the refinement of instance I (re-tagged for coarse step n) stays
// as it is for steps n + 1 .. n + m - 1: their re-tag checks would do
// nothing, so those steps may run in the same launch as step n
bool footprint_kept(const Inst& I, long long n, int m) {
    std::vector<RefBox> boxes;
    for (int j = 1; j < m; j++) {
        window_boxes(I, n + j, boxes);
        if (box_signature(I, boxes) != I.box_sig) return false;
    }
    return true;
}

// Up to `most` coarse steps of every live instance with one launch of the
// persistent kernel: *ran = the steps it ran, 0 when this context takes the
// graph path instead.  A launch runs SBOT_TUNE_STEPS_PER_LAUNCH steps when
// that many are left and nothing has to happen on the host between them (no
// traced step; no re-tagging body whose footprint changes within them) and
// their phase list fits the kernel; else one.
sbot_status step_persistent(sbot_ctx* c, int most, int* ran) {
    *ran = 0;
    const DevPool P = pool_view(c);
    if (!c->persist || c->staged || (P.coll & COLL_SOLID) || (c->prof_mask & 15)) return SBOT_OK;
    const int g = c->par[0];
    int steps = most >= c->steps_per_launch ? c->steps_per_launch : 1;  // one list of each length
    if (c->prof_mask & 16) steps = 1;
    for (const Inst& I : c->inst)
        if (steps > 1 && I.live && I.d.retag && I.has_body && I.body.motion != 0 &&
            !footprint_kept(I, I.coarse_step, steps))
            steps = 1;
    int k = g + (steps > 1 ? 2 : 0);
    if (steps > 1) {
        TRY(ensure_step_phases(c, g, steps));
        if (!c->ph_ok[k]) steps = 1, k = g;
    }
    if (steps == 1) {
        TRY(ensure_step_phases(c, g, 1));
        if (!c->ph_ok[k]) return SBOT_OK;
    }
    StepArgs A{};
    A.ph = c->d_ph[k];
    A.nph = c->nph[k];
    A.ctl = c->d_ctl;
    A.lists = c->d_lists;
    A.counts = c->d_counts;
    A.f0 = c->f[0];
    A.f1 = c->f[1];
    A.vec_min_cells = c->vec_min_cells;
    A.spin_ns = c->spin_ns;
    A.bulk_rounds = c->bulk_rounds;
    A.crit_items = c->crit_items;
    if (c->prof_mask & 16) {  // the phase trace of this step: [starts (+ launch start)][ends][last starts][first ends][tasks]
        const size_t M = STEP_MAX_PHASES, nst = M + 1;
        if (!c->d_trace) CK(dalloc(&c->d_trace, nst + 3 * M + M / 2));
        unsigned long long* t = c->d_trace;
        CK(cudaMemsetAsync(t, 0xff, nst * sizeof(unsigned long long), c->s));
        CK(cudaMemsetAsync(t + nst, 0, 2 * M * sizeof(unsigned long long), c->s));
        CK(cudaMemsetAsync(t + nst + 2 * M, 0xff, M * sizeof(unsigned long long), c->s));
        CK(cudaMemsetAsync(t + nst + 3 * M, 0, (M / 2) * sizeof(unsigned long long), c->s));
        A.tr_start = t;
        A.tr_end = t + nst;
        A.tr_start2 = t + nst + M;
        A.tr_end1 = t + nst + 2 * M;
        A.tr_tasks = (int*)(t + nst + 3 * M);
        c->trace_g = k;
    }
    const int e = launch_step(c->storage, P, A, c->step_grid, c->step_T, c->step_smem, c->s);
    if (e != 0) return fail(c, SBOT_ERR_CUDA, std::string("persistent step launch: ") + cudaGetErrorString((cudaError_t)e));
    c->launch_n++;
    *ran = steps;
    return SBOT_OK;
}

sbot_status check_device_error(sbot_ctx* c) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (e == 0) return SBOT_OK;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s));
    std::string m = "device reported:";
    if (e & ERRB_STENCIL) m += " a marker stencil left the finest interior cells;";
    if (e & ERRB_PATCH) m += " the marker patch exceeded its capacity;";
    if (e & ERRB_NOSOURCE) m += " an interior cell found no streaming source;";
    if (e & ERRB_HALO) m += " a coalescence found no fine halo cell;";
    if (e & ERRB_SCHED) m += " the step kernel's phase bookkeeping overflowed;";
    if (e & ERRB_TIMEOUT)
        return fail(c, SBOT_ERR_TIMEOUT, m + " a bounded device wait (a bulk copy or a step dependency) gave up");
    if (e & ERRB_NONFINITE) return fail(c, SBOT_ERR_NONFINITE, m + " non-finite populations");
    return fail(c, SBOT_ERR_STATE, m);
}

// Before its first step an instance's pre-collision state lives in the buffer
// its post-collision state will not use: f[1 - par[l]].  After stepping, the
// same buffer holds the post-collision state of the previous step, from which
// the current pre-collision state is pulled.
void* pre_buf(sbot_ctx* c, int l) { return c->f[1 - c->par[l]]; }

// between coarse steps, the next finer level's buffer holding the halo values
// the last sub-steps streamed (what the coarse pull merges), or none
const void* fine_buf(sbot_ctx* c, const Inst& I, int l) { return l + 1 < I.m ? c->f[c->par[l + 1]] : nullptr; }

// t = 0: the IBM on the pre-collision state, then the first collision
sbot_status finalize_inst(sbot_ctx* c, int ii) {
    Inst& I = c->inst[ii];
    if (I.finalized) return SBOT_OK;
    DevPool P = pool_view(c);
    const int fin = I.m - 1;
    if (I.has_body) {
        const int one[2] = {ii, 1};  // an instance list of one entry, and its length
        TRY(upload(c, c->d_one, one, sizeof one));
        launch_ibm(c->storage, P, c->d_one, c->d_one + 1, 1, pre_buf(c, fin), fin, 1, I.ibm_smem, c->s);
        c->launch_n++;
        CK(cudaGetLastError());
    }
    for (int l = 0; l < I.m; l++) {
        launch_collide_init(c->storage, P, int_part(I, l), I.int_n[l], pre_buf(c, l), c->f[c->par[l]], l, c->s);
        c->launch_n += I.int_n[l] > 0;
    }
    CK(cudaGetLastError());
    I.finalized = true;
    return SBOT_OK;
}

sbot_status finalize_all(sbot_ctx* c) {
    for (size_t ii = 0; ii < c->inst.size(); ii++)
        if (c->inst[ii].live && !c->inst[ii].finalized) TRY(finalize_inst(c, (int)ii));
    return SBOT_OK;
}

Inst* selected(sbot_ctx* c) {
    if (c->sel < 0 || c->sel >= (int)c->inst.size() || !c->inst[c->sel].live) return nullptr;
    return &c->inst[c->sel];
}

sbot_status level_ok(sbot_ctx* c, Inst* I, int level) {
    if (!I) return fail(c, SBOT_ERR_STATE, "no live instance selected");
    if (level < 0 || level >= I->m) return fail(c, SBOT_ERR_ARG, "level out of range");
    return SBOT_OK;
}

sbot_status upload_dense_pre(sbot_ctx* c, Inst& I, int level, const double* host, int planes, int from_fields) {
    int nx = I.d.nx0 << level, ny = I.d.ny0 << level;
    long long plane = (long long)nx * ny;
    double* d = nullptr;
    CK(dalloc(&d, (size_t)planes * plane));
    cudaError_t e = cudaMemcpyAsync(d, host, (size_t)planes * plane * sizeof(double), cudaMemcpyHostToDevice, c->s);
    if (e == cudaSuccess) {
        DevPool P = pool_view(c);
        launch_set_pre(c->storage, P, int_part(I, level), I.int_n[level], pre_buf(c, level), nx, d, plane, from_fields,
                       c->s);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(c->s);
    dfree(d);
    CK(e);
    CK(e2);
    return SBOT_OK;
}

// the initial state of instance ii: the equilibrium at (rho0, u_in)
sbot_status reset_state(sbot_ctx* c, int ii) {
    Inst& I = c->inst[ii];
    DevPool P = pool_view(c);
    for (int l = 0; l < I.m; l++)
        launch_set_pre(c->storage, P, int_part(I, l), I.int_n[l], pre_buf(c, l), 0, nullptr, 0, 1, c->s);
    CK(cudaGetLastError());
    InstState z{};
    z.pose_k0 = -1;
    TRY(upload(c, c->d_ist + ii, &z, sizeof(InstState)));
    I.finalized = false;
    I.coarse_step = 0;
    I.forces_read = 0;
    return SBOT_OK;
}

// dense export of a level of instance I: mode 0 populations, mode 1 fields
sbot_status export_level(sbot_ctx* c, Inst& I, int level, int mode, std::vector<double>& out) {
    int nx = I.d.nx0 << level, ny = I.d.ny0 << level;
    long long plane = (long long)nx * ny;
    int planes = mode == 0 ? 9 : 3;
    double* d = nullptr;
    CK(dalloc(&d, (size_t)planes * plane));
    out.resize((size_t)planes * plane);
    cudaError_t e = cudaMemsetAsync(d, 0, (size_t)planes * plane * sizeof(double), c->s);
    if (e == cudaSuccess) {
        DevPool P = pool_view(c);
        launch_export(c->storage, P, int_part(I, level), I.int_n[level], pre_buf(c, level), fine_buf(c, I, level), level,
                      I.coarse_step == 0 ? 1 : 0, nx, d, plane, mode, c->s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), d, out.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s);
    cudaError_t e2 = cudaStreamSynchronize(c->s);
    dfree(d);
    CK(e);
    CK(e2);
    return check_device_error(c);
}

sbot_status validate_desc(const sbot_domain_desc* d, std::string& why) {
    if (!d) return why = "null description", SBOT_ERR_ARG;
    if (d->levels < 1 || d->levels > SBOT_MAXLEV) return why = "levels must be 1..8", SBOT_ERR_ARG;
    if (d->block != 8 && d->block != 16 && d->block != 32) return why = "block must be 8, 16 or 32", SBOT_ERR_ARG;
    if (d->nx0 <= 0 || d->ny0 <= 0 || d->nx0 % d->block || d->ny0 % d->block)
        return why = "nx0, ny0 must be positive multiples of block", SBOT_ERR_ARG;
    for (int i = 0; i < 4; i++)
        if (d->bc[i] < 0 || d->bc[i] > 4) return why = "bad boundary kind", SBOT_ERR_ARG;
    if (d->solid_kind < 0 || d->solid_kind > 2) return why = "solid_kind must be 0, 1 or 2", SBOT_ERR_ARG;
    if (d->solid_kind == 1 && !(d->solid[2] > 0)) return why = "a solid circle needs a positive radius", SBOT_ERR_ARG;
    if (d->solid_kind != 0 && d->retag) return why = "a solid needs a static refinement (retag 0)", SBOT_ERR_ARG;
    if ((d->bc[0] == 0) != (d->bc[1] == 0) || (d->bc[2] == 0) != (d->bc[3] == 0))
        return why = "opposite sides must both be periodic or both not", SBOT_ERR_ARG;
    if (!(d->tau_finest > 0.5)) return why = "tau must exceed 1/2", SBOT_ERR_ARG;
    if (d->storage < 0 || d->storage > 3) return why = "bad storage kind", SBOT_ERR_ARG;
    if (d->n_boxes < 0 || (d->n_boxes > 0 && !d->boxes)) return why = "bad refinement boxes", SBOT_ERR_ARG;
    if (d->collision < 0 || d->collision > 2) return why = "collision must be 0 (BGK), 1 (MRT) or 2 (LES)", SBOT_ERR_ARG;
    if (!(d->les_cs >= 0 && d->les_cs < 1)) return why = "the Smagorinsky constant must lie in [0, 1)", SBOT_ERR_ARG;
    for (int k = 0; k < 3; k++)
        if (!(d->mrt_rates[k] >= 0 && d->mrt_rates[k] < 2)) return why = "MRT rates must lie in [0, 2)", SBOT_ERR_ARG;
    long long cells = (long long)d->nx0 * d->ny0 << (2 * (d->levels - 1));
    if (cells > (1LL << 36)) return why = "domain too large", SBOT_ERR_ARG;
    return SBOT_OK;
}

void free_inst_device(Inst& I) {
    dfree(I.d_latmap);
    dfree(I.d_int);
    dfree(I.d_qx);
    dfree(I.d_qy);
    dfree(I.d_patch);
    dfree(I.d_hist);
    dfree(I.d_pose);
    I.d_pose = nullptr;
    dfree(I.d_ibmcache);
    I.d_ibmcache = nullptr;
    dfree(I.d_fterm);
    I.d_fterm = nullptr;
    I.d_latmap = nullptr;
    I.d_int = nullptr;
    I.d_qx = I.d_qy = nullptr;
    I.d_patch = nullptr;
    I.d_hist = nullptr;
    I.latmap_n = 0;
    I.int_cap = 0;
}

long long bytes_in_use(const sbot_ctx* c) {
    long long used = (long long)(c->cap - (long long)c->free_slots.size()) * 2 * (long long)slot_bytes(c);
    for (auto& I : c->inst)
        if (I.live) used += I.extra_bytes + I.latmap_n * 4 + I.int_cap * 4;
    return used;
}

// instance ii from its descriptions (no slots yet)
sbot_status setup_inst(sbot_ctx* c, int ii, const sbot_domain_desc* desc, const sbot_body_desc* body) {
    Inst& I = c->inst[ii];
    I = Inst();
    I.d = *desc;
    I.d.boxes = nullptr;
    for (int i = 0; i < desc->n_boxes; i++)
        I.static_boxes.push_back({desc->boxes[i].level, desc->boxes[i].x0, desc->boxes[i].y0, desc->boxes[i].x1,
                                  desc->boxes[i].y1});
    I.d.n_boxes = 0;
    I.m = desc->levels;
    InstParams& ip = I.ip;
    ip.m = I.m;
    ip.nx0 = desc->nx0;
    ip.ny0 = desc->ny0;
    for (int i = 0; i < 4; i++) ip.bc[i] = desc->bc[i];
    ip.periodic_x = desc->bc[SIDE_W] == BCK_PERIODIC;
    ip.periodic_y = desc->bc[SIDE_S] == BCK_PERIODIC;
    for (int l = 0; l < I.m; l++)  // acoustic scaling (Eq. 9 per level): nu halves with every finer level
        ip.tau[l] = 0.5 + (desc->tau_finest - 0.5) / (double)(1 << (I.m - 1 - l));
    ip.rho0 = desc->rho0;
    ip.uin_x = desc->u_in[0];
    ip.uin_y = desc->u_in[1];
    {
        // 16-bit storage holds f - f^eq(rho0, u_in) (Eq. 7): its shift from the
        // compute form f - w_q, in FP64 then rounded once
        static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        static const double wq[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
        const bool half = c->storage == SBOT_F16DEV || c->storage == SBOT_BF16DEV;
        const double uu = ip.uin_x * ip.uin_x + ip.uin_y * ip.uin_y;
        for (int q = 0; q < 9; q++) {
            const double cu = ex[q] * ip.uin_x + ey[q] * ip.uin_y;
            const double d = wq[q] * ((ip.rho0 - 1.0) + ip.rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
            ip.dref[q] = half ? (float)d : 0.0f;
        }
        ip.dref_on = 0;
        for (int q = 0; q < 9; q++) ip.dref_on |= ip.dref[q] != 0.0f;
    }
    ip.K = desc->ibm_iters > 0 ? desc->ibm_iters : 5;
    for (int k = 0; k < 4; k++) {
        ip.uwall[k][0] = desc->wall_velocity[2 * k];
        ip.uwall[k][1] = desc->wall_velocity[2 * k + 1];
    }
    ip.les_cs = desc->les_cs > 0 ? desc->les_cs : 0.17;
    ip.solid = desc->solid_kind;
    for (int k = 0; k < 3; k++) ip.sol[k] = desc->solid[k];
    const double mrt_default[3] = {1.64, 1.54, 1.9};
    for (int k = 0; k < 3; k++) ip.mrt_s[k] = desc->mrt_rates[k] > 0 ? desc->mrt_rates[k] : mrt_default[k];
    if (!body) return SBOT_OK;
    if (desc->solid_kind != 0) return fail(c, SBOT_ERR_ARG, "an instance holds an IBM body or a solid, not both");
    HostBody& hb = I.body;
    if (!host_body_from_desc(body, hb)) return fail(c, SBOT_ERR_ARG, "bad body description");
    double R = 0;
    for (int j = 0; j < hb.n; j++) R = std::max(R, std::hypot(hb.qx[j] - hb.pivot[0], hb.qy[j] - hb.pivot[1]));
    int side = (int)std::ceil(2 * R) + 6;
    int cap = side * side;
    size_t smem = ibm_smem_bytes(c->storage, cap, hb.n);
    if (smem > ibm_smem_limit(c->storage))
        return fail(c, SBOT_ERR_ARG, "body too large for the one-block IBM kernel");
    I.ibm_smem = smem;
    I.has_body = true;
    ip.has_body = 1;
    ip.n_markers = hb.n;
    ip.ds = hb.ds;
    ip.pivot[0] = hb.pivot[0];
    ip.pivot[1] = hb.pivot[1];
    ip.motion = hb.motion;
    ip.x0[0] = hb.x0[0];
    ip.x0[1] = hb.x0[1];
    ip.alpha_mean = hb.alpha_mean;
    ip.alpha_amp = hb.alpha_amp;
    ip.period = hb.period;
    ip.phase = hb.phase;
    ip.heave_amp = hb.heave_amp;
    ip.beta = hb.beta;
    ip.cos_mean = std::cos(hb.alpha_mean);
    ip.sin_mean = std::sin(hb.alpha_mean);
    ip.cos_beta = std::cos(hb.beta);
    ip.sin_beta = std::sin(hb.beta);
    ip.ramp_as = hb.ramp_as;
    ip.ramp_rate = hb.ramp_rate;
    ip.ramp_t1 = hb.ramp_t1;
    ip.t_ref = hb.t_ref;
    ip.asym_xi = hb.asym_xi;
    ip.accel_frac = hb.accel_frac;
    ip.patch_cap = cap;
    const size_t cbytes = c->storage == 0 ? 8 : 4;
    CK(dalloc(&I.d_qx, hb.n));
    CK(dalloc(&I.d_qy, hb.n));
    CK(cudaMalloc(&I.d_patch, 2 * (size_t)cap * cbytes));
    CK(dalloc(&I.d_hist, (size_t)3 * SBOT_HIST_CAP));
    ip.fterm_n = 1 << (I.m - 1);
    CK(cudaMalloc(&I.d_fterm, (size_t)ip.fterm_n * 3 * hb.n * cbytes));
    ip.fterm = I.d_fterm;
    TRY(upload(c, I.d_qx, hb.qx.data(), hb.n * sizeof(double)));
    TRY(upload(c, I.d_qy, hb.qy.data(), hb.n * sizeof(double)));
    ip.qx = I.d_qx;
    ip.qy = I.d_qy;
    ip.patch = I.d_patch;
    ip.hist = I.d_hist;
    I.extra_bytes = (long long)hb.n * 16 + 2LL * cap * (long long)cbytes + 24LL * SBOT_HIST_CAP +
                    3LL * ip.fterm_n * hb.n * (long long)cbytes;
    // the stored IBM geometry: one entry for a static body, one per finest
    // step of a coarse step for a moving body (entries stamped -1: none valid)
    const size_t cb = ibm_cache_bytes(c->storage, cap, hb.n);
    const int entries = hb.motion == 0 ? 1 : 1 << (I.m - 1);
    CK(cudaMalloc(&I.d_ibmcache, cb * entries));
    CK(cudaMemsetAsync(I.d_ibmcache, 0xff, cb * entries, c->s));
    ip.ibm_cache = I.d_ibmcache;
    ip.ibm_cache_stride = (long long)cb;
    I.extra_bytes += (long long)(cb * entries);
    if (hb.motion != 0) {
        ip.pose_n = (1 << (I.m - 1)) + 1;
        CK(dalloc(&I.d_pose, (size_t)4 * ip.pose_n));
        ip.pose_tab = I.d_pose;
        I.extra_bytes += 32LL * ip.pose_n;
    }
    return SBOT_OK;
}

// release instance ii: its slots leave the lists, its device buffers are freed
// (after the queued work that may read them)
void drop_inst(sbot_ctx* c, int ii) {
    Inst& I = c->inst[ii];
    if (c->s) cudaStreamSynchronize(c->s);
    for (int sl : I.slot_of)
        if (sl >= 0 && sl < c->cap && c->h_type[sl] != ST_FREE) free_slot(c, sl);
    if (c->lpos[LK_IBM][ii] >= 0) list_remove(c, gl_of(I.m, I.m - 1), LK_IBM, ii, I.ip.patch_cap);
    // marked lattice-map entries name this instance's map, which goes now
    const int lat_arr = A_LAT + ii;
    c->dirty.erase(std::remove_if(c->dirty.begin(), c->dirty.end(), [&](const Dirty& d) { return d.arr == lat_arr; }),
                   c->dirty.end());
    free_inst_device(I);
    I = Inst();
}

sbot_status create_ctx(int max_instances, int block, int storage, long long budget, void* stream, sbot_ctx** out) {
    sbot_ctx* c = new sbot_ctx();
    cudaGetDevice(&c->device);
    c->s = (cudaStream_t)stream;
    if (!c->s) {
        if (cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return SBOT_ERR_CUDA;
        }
        c->own_stream = true;
    }
    c->storage = storage;
    c->B = block;
    c->words = (block * block + 31) / 32;
    c->budget = budget;
    c->inst.resize(max_instances);
    c->lpos[LK_IBM].assign(max_instances, -1);
    auto bail = [&](sbot_status e) {
        cudaGetLastError();
        sbot_destroy(c);
        return e;
    };
    if (cudaEventCreateWithFlags(&c->ev_gfork, cudaEventDisableTiming) != cudaSuccess) return bail(SBOT_ERR_CUDA);
    for (int i = 0; i < 2; i++)
        if (cudaEventCreateWithFlags(&c->arena[i].done, cudaEventDisableTiming) != cudaSuccess)
            return bail(SBOT_ERR_CUDA);
    if (dalloc(&c->d_ip, (size_t)max_instances) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (dalloc(&c->d_ist, (size_t)max_instances) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (dalloc(&c->d_err, 1) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (dalloc(&c->d_out3, 3) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (dalloc(&c->d_one, 2) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (dalloc(&c->d_counts, (size_t)NLISTS) != cudaSuccess) return bail(SBOT_ERR_OOM);
    if (cudaMemsetAsync(c->d_err, 0, sizeof(int), c->s) != cudaSuccess) return bail(SBOT_ERR_CUDA);
    if (cudaMemsetAsync(c->d_ist, 0, sizeof(InstState) * max_instances, c->s) != cudaSuccess)
        return bail(SBOT_ERR_CUDA);
    if (cudaMemsetAsync(c->d_ip, 0, sizeof(InstParams) * max_instances, c->s) != cudaSuccess)
        return bail(SBOT_ERR_CUDA);
    if (cudaMemsetAsync(c->d_counts, 0, sizeof(int) * NLISTS, c->s) != cudaSuccess)
        return bail(SBOT_ERR_CUDA);
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return bail(SBOT_ERR_CUDA);
    *out = c;
    return SBOT_OK;
}

// Admission by device footprint: the slots the instance needs at its first
// coarse step (half as many again when its refined region moves), its body
// buffers and its lattice maps must fit next to what the live instances hold.
sbot_status check_budget(sbot_ctx* c, const Inst& I) {
    if (c->budget <= 0) return SBOT_OK;
    TopoSpec ts = topo_spec(I, c->B);
    window_boxes(I, 0, ts.boxes);
    BlockStates bs;
    const char* why = nullptr;
    if (!plan_blocks(ts, bs, &why)) return fail(c, SBOT_ERR_STATE, why);
    std::vector<PlannedBlock> pbs;
    plan_slots(ts, bs, pbs);
    long long lat = 0;
    for (int l = 0; l < I.m; l++) lat += (long long)bs.nbx[l] * bs.nby[l] * 4;
    double envelope = (I.d.retag && I.has_body) ? 1.5 : 1.0;
    long long need = (long long)((double)pbs.size() * envelope) * 2 * (long long)slot_bytes(c) + I.extra_bytes + lat;
    if (bytes_in_use(c) + need > c->budget)
        return fail(c, SBOT_ERR_OOM, "admission refused: the instance does not fit the device-memory budget");
    return SBOT_OK;
}

// instance ii (free) from its descriptions: plan, take slots, set the initial state
sbot_status admit(sbot_ctx* c, int ii, const sbot_domain_desc* desc, const sbot_body_desc* body) {
    // one collision kind per context: the kernels are specialised on it
    bool any_live = false;
    for (size_t i = 0; i < c->inst.size(); i++) any_live |= c->inst[i].live && (int)i != ii;
    if (any_live && desc->collision != c->coll)
        return fail(c, SBOT_ERR_ARG, "the instance's collision kind must be the batch's");
    if (!any_live && desc->collision != c->coll) {
        c->coll = desc->collision;
        c->cap_version++;  // the step graphs pick kernel variants at capture
    }
    sbot_status st = setup_inst(c, ii, desc, body);
    if (st == SBOT_OK) st = check_budget(c, c->inst[ii]);
    if (st != SBOT_OK) {
        CK(cudaStreamSynchronize(c->s));
        free_inst_device(c->inst[ii]);
        c->inst[ii] = Inst();
        return st;
    }
    Inst& I = c->inst[ii];
    I.live = true;
    if (I.ip.dref_on && !c->shift_seen) {  // the step graphs pick the 8-cell kernel's shift variant at capture
        c->shift_seen = true;
        c->cap_version++;
    }
    if (I.ip.solid != 0) c->cap_version++;  // the step graphs switch to the fused kernel with solid links
    st = build_topology(c, ii, 0, false);
    if (st == SBOT_OK) {
        if (I.has_body) list_add(c, gl_of(I.m, I.m - 1), LK_IBM, ii, I.ip.patch_cap);
        st = refresh_groups(c);
        if (st == SBOT_OK) st = flush(c);
    }
    if (st == SBOT_OK) st = reset_state(c, ii);
    if (st == SBOT_OK) st = end_frame(c);
    if (st != SBOT_OK) {
        std::string m = c->err;
        drop_inst(c, ii);
        refresh_groups(c);
        flush(c);
        c->err = m;
    }
    return st;
}

// cell updates of one coarse step of instance I (interior cells x substeps)
int64_t cell_updates(const sbot_ctx* c, const Inst& I) {
    int64_t cu = 0;
    for (int l = 0; l < I.m; l++) cu += ((int64_t)I.int_n[l] * c->B * c->B) << l;
    return cu;
}

// partial sums of mass and momentum of instance I (one per thread block),
// then their fixed-order sum into out3_dev
sbot_status checksum_into(sbot_ctx* c, Inst& I, double* partials, double* out3_dev) {
    DevPool P = pool_view(c);
    int off = 0;
    const int direct = I.coarse_step == 0 ? 1 : 0;
    for (int l = 0; l < I.m; l++) {
        const int nb = checksum_blocks(I.int_n[l], c->B);
        const double area = (double)(1LL << (2 * (I.m - 1 - l)));
        if (I.int_n[l] > 0)
            launch_checksum_partials(c->storage, P, int_part(I, l), I.int_n[l], pre_buf(c, l), fine_buf(c, I, l), l, direct,
                                     area,
                                     partials + 3 * off, nb, c->s);
        else
            CK(cudaMemsetAsync(partials + 3 * off, 0, 3 * nb * sizeof(double), c->s));
        off += nb;
    }
    launch_reduce_partials(partials, off, out3_dev, c->d_err, c->s);
    CK(cudaGetLastError());
    return SBOT_OK;
}

int checksum_total(const sbot_ctx* c, const Inst& I) {
    int total = 0;
    for (int l = 0; l < I.m; l++) total += checksum_blocks(I.int_n[l], c->B);
    return total;
}

}  // namespace

extern "C" {

sbot_status sbot_create_domain(const sbot_domain_desc* desc, void* cuda_stream, sbot_ctx_t* out) {
    std::string why;
    if (!out) return SBOT_ERR_ARG;
    *out = nullptr;
    sbot_status st = validate_desc(desc, why);
    if (st != SBOT_OK) return st;
    sbot_ctx* c = nullptr;
    st = create_ctx(1, desc->block, desc->storage, 0, cuda_stream, &c);
    if (st != SBOT_OK) return st;
    st = admit(c, 0, desc, nullptr);
    if (st != SBOT_OK) {
        sbot_destroy(c);
        return st;
    }
    *out = c;
    return SBOT_OK;
}

sbot_status sbot_set_body_kinematics(sbot_ctx_t c, const sbot_body_desc* b) {
    if (!c || !b) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    if (!I) return fail(c, SBOT_ERR_STATE, "no live instance selected");
    if (I->coarse_step > 0) return fail(c, SBOT_ERR_STATE, "set the body before stepping");
    HostBody probe;
    if (!host_body_from_desc(b, probe)) return fail(c, SBOT_ERR_ARG, "bad body description");
    // re-admit the instance with the body: the refinement follows it and the state restarts
    sbot_domain_desc d = I->d;
    std::vector<sbot_box> boxes;
    for (const RefBox& r : I->static_boxes) boxes.push_back({r.level, r.x0, r.y0, r.x1, r.y1});
    d.n_boxes = (int)boxes.size();
    d.boxes = boxes.empty() ? nullptr : boxes.data();
    const int ii = c->sel;
    drop_inst(c, ii);
    return admit(c, ii, &d, b);
}

sbot_status sbot_set_fields(sbot_ctx_t c, int level, const double* rho, const double* ux, const double* uy) {
    if (!c || !rho || !ux || !uy) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    if (I->finalized) return fail(c, SBOT_ERR_STATE, "initial state can only be set before the first step");
    size_t plane = (size_t)(I->d.nx0 << level) * (I->d.ny0 << level);
    std::vector<double> tmp(3 * plane);
    std::memcpy(tmp.data(), rho, plane * sizeof(double));
    std::memcpy(tmp.data() + plane, ux, plane * sizeof(double));
    std::memcpy(tmp.data() + 2 * plane, uy, plane * sizeof(double));
    return upload_dense_pre(c, *I, level, tmp.data(), 3, 1);
}

sbot_status sbot_set_populations(sbot_ctx_t c, int level, const double* f) {
    if (!c || !f) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    if (I->finalized) return fail(c, SBOT_ERR_STATE, "initial state can only be set before the first step");
    return upload_dense_pre(c, *I, level, f, 9, 0);
}

sbot_status sbot_step(sbot_ctx_t c, int n) {
    if (!c || n < 0) return SBOT_ERR_ARG;
    TRY(finalize_all(c));
    if (c->groups == 0) return SBOT_OK;  // no live instance
    for (int k = 0; k < n;) {
        // re-tag every instance whose moving body has moved its refinement
        for (size_t ii = 0; ii < c->inst.size(); ii++) {
            Inst& I = c->inst[ii];
            if (I.live && I.d.retag && I.has_body && I.body.motion != 0 && I.coarse_step > 0)
                TRY(build_topology(c, (int)ii, I.coarse_step, true));
        }
        TRY(flush(c));
        // one CUDA graph per parity of level 0 (level 0 flips its buffers once
        // per coarse step, every finer level an even number of times); it reads
        // the list lengths on the device, so it is recaptured only when a
        // capacity, the pool or the depth changes
        const int g = c->par[0];
        int done = 0;
        TRY(step_persistent(c, n - k, &done));
        const bool ran = done > 0;
        if (!ran && (!c->gexec[g] || c->graph_version[g] != c->cap_version || c->graph_mask[g] != c->prof_mask)) {
            CK(cudaStreamSynchronize(c->s));
            drop_graph(c, g);
            cudaGraph_t gr = nullptr;
            c->capturing = true;
            c->pending.clear();
            CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
            advance_all(c);
            cudaError_t ce = cudaStreamEndCapture(c->s, &gr);
            c->capturing = false;
            c->graph_recs[g] = c->pending;
            c->pending.clear();
            CK(ce);
            size_t nn = 0;
            c->graph_kernels[g] = 0;
            if (cudaGraphGetNodes(gr, nullptr, &nn) == cudaSuccess && nn > 0) {
                std::vector<cudaGraphNode_t> nodes(nn);
                if (cudaGraphGetNodes(gr, nodes.data(), &nn) == cudaSuccess)
                    for (size_t i = 0; i < nn; i++) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                            c->graph_kernels[g]++;
                    }
            }
            cudaError_t ie = cudaGraphInstantiate(&c->gexec[g], gr, 0);
            cudaGraphDestroy(gr);
            CK(ie);
            c->graph_version[g] = c->cap_version;
            c->graph_mask[g] = c->prof_mask;
        }
        if (!ran) {
            CK(cudaGraphLaunch(c->gexec[g], c->s));
            c->launch_n += c->graph_kernels[g];
        }
        if (!ran && c->prof_mask) account(c, c->graph_recs[g]);
        const int steps = ran ? done : 1;
        c->par[0] ^= steps & 1;
        for (auto& I : c->inst)
            if (I.live) I.coarse_step += steps;
        k += steps;
        TRY(end_frame(c));
    }
    CK(cudaGetLastError());
    return SBOT_OK;
}

sbot_status sbot_batch_step(sbot_ctx_t c, int n) { return sbot_step(c, n); }

sbot_status sbot_set_profiling(sbot_ctx_t c, int mask) {
    if (!c || mask < 0 || mask > 31) return SBOT_ERR_ARG;
    CK(cudaStreamSynchronize(c->s));
    c->prof_mask = mask;
    c->launch_n = 0;
    if (mask)
        for (int k = 0; k < 4; k++) {
            c->prof_n[k] = 0;
            c->prof_ms[k] = 0;
            c->prof_bytes[k] = 0;
        }
    return SBOT_OK;
}

sbot_status sbot_set_tuning(sbot_ctx_t c, int what, int64_t value) {
    if (!c) return SBOT_ERR_ARG;
    if (what == SBOT_TUNE_VECTOR_MIN_CELLS) {
        if (value == c->vec_min_cells) return SBOT_OK;
        c->vec_min_cells = value;
    } else if (what == SBOT_TUNE_STAGED) {
        if (value != 0 && value != 1) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_STAGED takes 0 or 1");
        if (value == c->staged) return SBOT_OK;
        c->staged = (int)value;
    } else if (what == SBOT_TUNE_PDL) {
        if (value != 0 && value != 1) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_PDL takes 0 or 1");
        if (value == c->pdl) return SBOT_OK;
        c->pdl = (int)value;
    } else if (what == SBOT_TUNE_PERSISTENT) {
        if (value != 0 && value != 1) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_PERSISTENT takes 0 or 1");
        if (value == c->persist) return SBOT_OK;
        c->persist = (int)value;
    } else if (what == SBOT_TUNE_STEP_THREADS) {
        if (value != 0 && value != 256 && value != 768)
            return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_STEP_THREADS takes 0, 256 or 768");
        if (value == c->step_threads) return SBOT_OK;
        c->step_threads = (int)value;
    } else if (what == SBOT_TUNE_SPIN_NS) {
        if (value < 0) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_SPIN_NS must be >= 0");
        c->spin_ns = value;
        return SBOT_OK;  // a launch argument: nothing to rebuild
    } else if (what == SBOT_TUNE_IBM_THREADS) {
        if (value != 256 && value != 512 && value != 768 && value != 1024)
            return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_IBM_THREADS takes 256, 512, 768 or 1024");
        if (value == c->ibm_threads) return SBOT_OK;
        c->ibm_threads = (int)value;
    } else if (what == SBOT_TUNE_BULK_ROUNDS) {
        if (value < 1 || value > 64) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_BULK_ROUNDS takes 1..64");
        c->bulk_rounds = (int)value;
        return SBOT_OK;
    } else if (what == SBOT_TUNE_STEPS_PER_LAUNCH) {
        if (value < 1 || value > 16) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_STEPS_PER_LAUNCH takes 1..16");
        c->steps_per_launch = (int)value;
        return SBOT_OK;  // the list is rebuilt at the next launch that needs it
    } else if (what == SBOT_TUNE_VEC_WAVES) {
        if (value < -1 || value > 64) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_VEC_WAVES takes -1..64");
        if (value <= 0) value = 0;
        if (value == c->vec_waves) return SBOT_OK;
        c->vec_waves = (int)value;
    } else if (what == SBOT_TUNE_CRIT_BLOCKS) {
        if (value < 0 || value > 64) return fail(c, SBOT_ERR_ARG, "SBOT_TUNE_CRIT_BLOCKS takes 0..64");
        c->crit_items = (int)value;
        return SBOT_OK;  // a launch argument: nothing to rebuild
    } else {
        return fail(c, SBOT_ERR_ARG, "unknown tuning parameter");
    }
    c->cap_version++;  // the step graphs pick kernel variants at capture
    return SBOT_OK;
}

sbot_status sbot_get_tuning(sbot_ctx_t c, int what, int64_t* value) {
    if (!c || !value) return SBOT_ERR_ARG;
    if (what == SBOT_TUNE_VECTOR_MIN_CELLS)
        *value = c->vec_min_cells;
    else if (what == SBOT_TUNE_STAGED)
        *value = c->staged;
    else if (what == SBOT_TUNE_PDL)
        *value = c->pdl;
    else if (what == SBOT_TUNE_PERSISTENT)
        *value = c->persist;
    else if (what == SBOT_TUNE_STEP_THREADS)
        *value = c->step_threads;
    else if (what == SBOT_TUNE_SPIN_NS)
        *value = c->spin_ns;
    else if (what == SBOT_TUNE_BULK_ROUNDS)
        *value = c->bulk_rounds;
    else if (what == SBOT_TUNE_IBM_THREADS)
        *value = c->ibm_threads;
    else if (what == SBOT_TUNE_CRIT_BLOCKS)
        *value = c->crit_items;
    else if (what == SBOT_TUNE_STEPS_PER_LAUNCH)
        *value = c->steps_per_launch;
    else if (what == SBOT_TUNE_VEC_WAVES)
        *value = c->vec_waves;
    else
        return fail(c, SBOT_ERR_ARG, "unknown tuning parameter");
    return SBOT_OK;
}

sbot_status sbot_get_step_trace(sbot_ctx_t c, int* n_inout, int* kind, int* level, int* bulk, int* tasks,
                                double* us4) {
    if (!c || !n_inout || *n_inout < 0) return SBOT_ERR_ARG;
    const int g = c->trace_g;
    if (g < 0 || !c->d_trace) return fail(c, SBOT_ERR_STATE, "no traced persistent step");
    const int n = c->nph[g];
    if (*n_inout < n) {
        *n_inout = n;
        return fail(c, SBOT_ERR_ARG, "trace arrays too small");
    }
    const size_t M = STEP_MAX_PHASES, nst = M + 1;
    std::vector<unsigned long long> t(nst + 3 * M + M / 2);  // as allocated
    std::vector<StepPhase> ph((size_t)n);
    CK(cudaMemcpyAsync(t.data(), c->d_trace, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(ph.data(), c->d_ph[g], ph.size() * sizeof(StepPhase), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    const unsigned long long t0 = t[M];
    const int* cnt = (const int*)(t.data() + nst + 3 * M);
    auto us = [&](unsigned long long v) { return 1e-3 * (double)(long long)(v - t0); };
    for (int p = 0; p < n; p++) {
        if (kind) kind[p] = ph[p].kind;
        if (level) level[p] = ph[p].level;
        if (bulk) bulk[p] = ph[p].bulk;
        if (tasks) tasks[p] = cnt[p];
        const bool ran = cnt[p] > 0 && t[p] != ~0ULL;
        if (us4) {
            us4[4 * p + 0] = ran ? us(t[p]) : -1.0;                  // first task start
            us4[4 * p + 1] = ran ? us(t[nst + M + p]) : -1.0;        // last task start
            us4[4 * p + 2] = ran ? us(t[nst + 2 * M + p]) : -1.0;    // first task end
            us4[4 * p + 3] = ran ? us(t[nst + p]) : -1.0;            // last task end
        }
    }
    *n_inout = n;
    return check_device_error(c);
}

sbot_status sbot_get_profile(sbot_ctx_t c, int kind, int64_t* launches, double* ms, double* bytes) {
    if (!c || kind < 0 || kind > 4) return SBOT_ERR_ARG;
    if (kind == 4) {  // kernels launched by sbot_step, counted whether or not profiling is on
        if (launches) *launches = c->launch_n;
        if (ms) *ms = 0;
        if (bytes) *bytes = 0;
        return SBOT_OK;
    }
    if (launches) *launches = c->prof_n[kind];
    if (ms) *ms = c->prof_ms[kind];
    if (bytes) *bytes = c->prof_bytes[kind];
    return SBOT_OK;
}

sbot_status sbot_get_forces(sbot_ctx_t c, double* fx, double* fy, double* mz, int* n_inout) {
    if (!c || !n_inout || *n_inout < 0) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    if (!I) return fail(c, SBOT_ERR_STATE, "no live instance selected");
    if (!I->has_body) {
        *n_inout = 0;
        return SBOT_OK;
    }
    CK(cudaStreamSynchronize(c->s));
    TRY(check_device_error(c));
    long long upto = I->coarse_step << (I->m - 1);  // forces of finest steps k < canonical time
    long long avail = upto - I->forces_read;
    if (avail > SBOT_HIST_CAP) {
        I->forces_read = upto - SBOT_HIST_CAP;
        *n_inout = 0;
        return fail(c, SBOT_ERR_STATE, "force history overflowed; read forces more often");
    }
    int cnt = (int)std::min<long long>(avail, *n_inout);
    if (cnt > 0) {
        // the ring holds entry k at k mod capacity: at most two contiguous pieces
        std::vector<double> h((size_t)3 * cnt);
        long long k0 = I->forces_read % SBOT_HIST_CAP;
        long long first = std::min<long long>(cnt, SBOT_HIST_CAP - k0);
        CK(cudaMemcpyAsync(h.data(), I->d_hist + 3 * k0, (size_t)3 * first * sizeof(double), cudaMemcpyDeviceToHost,
                           c->s));
        if (first < cnt)
            CK(cudaMemcpyAsync(h.data() + 3 * first, I->d_hist, (size_t)3 * (cnt - first) * sizeof(double),
                               cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        for (int i = 0; i < cnt; i++) {
            if (fx) fx[i] = h[3 * i];
            if (fy) fy[i] = h[3 * i + 1];
            if (mz) mz[i] = h[3 * i + 2];
        }
    }
    I->forces_read += cnt;
    *n_inout = cnt;
    return SBOT_OK;
}

sbot_status sbot_get_fields(sbot_ctx_t c, int level, double* rho, double* ux, double* uy, int64_t* n_inout) {
    if (!c || !n_inout) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    int64_t plane = (int64_t)(I->d.nx0 << level) * (I->d.ny0 << level);
    if (*n_inout < plane) {
        *n_inout = plane;
        return fail(c, SBOT_ERR_ARG, "output arrays too small");
    }
    std::vector<double> out;
    TRY(export_level(c, *I, level, 1, out));
    if (rho) std::memcpy(rho, out.data(), plane * sizeof(double));
    if (ux) std::memcpy(ux, out.data() + plane, plane * sizeof(double));
    if (uy) std::memcpy(uy, out.data() + 2 * plane, plane * sizeof(double));
    *n_inout = plane;
    return SBOT_OK;
}

sbot_status sbot_get_populations(sbot_ctx_t c, int level, double* f, int64_t* n_inout) {
    if (!c || !n_inout || !f) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    int64_t n = (int64_t)9 * (I->d.nx0 << level) * (I->d.ny0 << level);
    if (*n_inout < n) {
        *n_inout = n;
        return fail(c, SBOT_ERR_ARG, "output array too small");
    }
    std::vector<double> out;
    TRY(export_level(c, *I, level, 0, out));
    std::memcpy(f, out.data(), n * sizeof(double));
    *n_inout = n;
    return SBOT_OK;
}

sbot_status sbot_get_celltypes(sbot_ctx_t c, int level, uint8_t* types, int64_t* n_inout) {
    if (!c || !n_inout || !types) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    std::vector<uint8_t> t;
    cell_types(I->ts, I->bs, level, t);
    if (level == I->m - 1 && I->ip.solid != 0) {  // solid cells (reading R15)
        const int nxl = I->ip.nx0 << level, nyl = I->ip.ny0 << level;
        for (int y = 0; y < nyl; y++)
            for (int x = 0; x < nxl; x++)
                if (t[(size_t)y * nxl + x] == ST_INT && host_in_solid(I->ip, x + 0.5, y + 0.5))
                    t[(size_t)y * nxl + x] = 4;
    }
    if (*n_inout < (int64_t)t.size()) {
        *n_inout = (int64_t)t.size();
        return fail(c, SBOT_ERR_ARG, "output array too small");
    }
    std::memcpy(types, t.data(), t.size());
    *n_inout = (int64_t)t.size();
    return SBOT_OK;
}

sbot_status sbot_get_topology(sbot_ctx_t c, int level, uint8_t* states, int* n_inout) {
    if (!c || !n_inout || !states) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    const std::vector<uint8_t>& s = I->bs.s[level];
    if (*n_inout < (int)s.size()) {
        *n_inout = (int)s.size();
        return fail(c, SBOT_ERR_ARG, "output array too small");
    }
    std::memcpy(states, s.data(), s.size());
    *n_inout = (int)s.size();
    return SBOT_OK;
}

sbot_status sbot_get_checksum(sbot_ctx_t c, double out3[3]) {
    if (!c || !out3) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    if (!I) return fail(c, SBOT_ERR_STATE, "no live instance selected");
    int total = checksum_total(c, *I);
    if (total > c->partials_cap) {
        CK(cudaStreamSynchronize(c->s));
        dfree(c->d_partials);
        c->d_partials = nullptr;
        c->partials_cap = 0;
        CK(dalloc(&c->d_partials, (size_t)3 * total));
        c->partials_cap = total;
    }
    TRY(checksum_into(c, *I, c->d_partials, c->d_out3));
    CK(cudaMemcpyAsync(out3, c->d_out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return check_device_error(c);
}

// Same result as sbot_get_checksum, but allocates nothing: the partial sums
// go to the library's static device scratch instead of a buffer that
// sbot_get_checksum allocates on its first call.
sbot_status sbot_get_checksum_noalloc(sbot_ctx_t c, double out3[3]) {
    if (!c || !out3) return SBOT_ERR_ARG;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != c->device) return fail(c, SBOT_ERR_STATE, "make the context's device current first");
    Inst* I = selected(c);
    if (!I) return fail(c, SBOT_ERR_STATE, "no live instance selected");
    int total = checksum_total(c, *I);
    if (total > SBOT_NOALLOC_MAX_PARTIALS)
        return fail(c, SBOT_ERR_ARG,
                    "sbot_get_checksum_noalloc: this domain needs " + std::to_string(total) +
                        " partial sums; the static scratch holds " + std::to_string(SBOT_NOALLOC_MAX_PARTIALS) +
                        " (use sbot_get_checksum)");
    double* scratch = noalloc_scratch();
    if (!scratch) return fail(c, SBOT_ERR_CUDA, "cannot look up the static scratch on this device");
    double* res = scratch + 3 * SBOT_NOALLOC_MAX_PARTIALS;
    TRY(checksum_into(c, *I, scratch, res));
    CK(cudaMemcpyAsync(out3, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return check_device_error(c);
}

sbot_status sbot_get_level_info(sbot_ctx_t c, int level, int* nx, int* ny, int64_t* n_interior) {
    if (!c) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    TRY(level_ok(c, I, level));
    if (nx) *nx = I->d.nx0 << level;
    if (ny) *ny = I->d.ny0 << level;
    if (n_interior) *n_interior = (int64_t)I->int_n[level] * c->B * c->B;
    return SBOT_OK;
}

sbot_status sbot_get_work(sbot_ctx_t c, int64_t* cell_updates_out, int64_t* fine_equivalent) {
    if (!c) return SBOT_ERR_ARG;
    Inst* I = selected(c);
    if (!I) return fail(c, SBOT_ERR_STATE, "no live instance selected");
    if (cell_updates_out) *cell_updates_out = cell_updates(c, *I);
    if (fine_equivalent) *fine_equivalent = ((int64_t)I->d.nx0 * I->d.ny0 << (2 * (I->m - 1))) << (I->m - 1);
    return SBOT_OK;
}

sbot_status sbot_plan_blocks(const sbot_domain_desc* desc, const sbot_body_desc* body, int64_t coarse_step,
                             int level, uint8_t* states, int* n_inout) {
    std::string why;
    if (!n_inout || !states || validate_desc(desc, why) != SBOT_OK) return SBOT_ERR_ARG;
    if (level < 0 || level >= desc->levels) return SBOT_ERR_ARG;
    Inst I;
    I.d = *desc;
    I.m = desc->levels;
    for (int i = 0; i < desc->n_boxes; i++)
        I.static_boxes.push_back({desc->boxes[i].level, desc->boxes[i].x0, desc->boxes[i].y0, desc->boxes[i].x1,
                                  desc->boxes[i].y1});
    if (body) {
        if (!host_body_from_desc(body, I.body)) return SBOT_ERR_ARG;
        I.has_body = true;
    }
    TopoSpec ts = topo_spec(I, desc->block);
    window_boxes(I, coarse_step, ts.boxes);
    BlockStates bs;
    const char* w = nullptr;
    if (!plan_blocks(ts, bs, &w)) return SBOT_ERR_STATE;
    if (*n_inout < (int)bs.s[level].size()) {
        *n_inout = (int)bs.s[level].size();
        return SBOT_ERR_ARG;
    }
    std::memcpy(states, bs.s[level].data(), bs.s[level].size());
    *n_inout = (int)bs.s[level].size();
    return SBOT_OK;
}

// ---------------------------------------------------------------------------
// batches: many instances in one context, stepped together
// ---------------------------------------------------------------------------

sbot_status sbot_batch_create(int max_instances, int block, int storage, int64_t hbm_budget_bytes, void* cuda_stream,
                              sbot_ctx_t* out) {
    if (!out) return SBOT_ERR_ARG;
    *out = nullptr;
    if (max_instances < 1 || max_instances > SBOT_MAX_INSTANCES || (block != 8 && block != 16 && block != 32) ||
        storage < 0 || storage > 3 || hbm_budget_bytes < 0)
        return SBOT_ERR_ARG;
    sbot_status st = create_ctx(max_instances, block, storage, hbm_budget_bytes, cuda_stream, out);
    // many instances keep the GPU busy from several streams: blocks scheduled
    // early to wait for their predecessor would only hold SMs the others need.
    // The per-phase graphs are the default here: on uneven batches whose
    // bodies need the IBM's large shared memory they measured faster than
    // the persistent kernel (one large thread block per SM), which the
    // autotuner still tries
    if (st == SBOT_OK) {
        (*out)->pdl = 0;
        (*out)->persist = 0;
    }
    return st;
}

sbot_status sbot_batch_admit(sbot_ctx_t c, const sbot_domain_desc* desc, const sbot_body_desc* body, int* slot) {
    if (!c || !desc || !slot) return SBOT_ERR_ARG;
    *slot = -1;
    std::string why;
    if (validate_desc(desc, why) != SBOT_OK) return fail(c, SBOT_ERR_ARG, why);
    if (desc->block != c->B || desc->storage != c->storage)
        return fail(c, SBOT_ERR_ARG, "the instance's block size and storage must be the batch's");
    int ii = -1;
    for (size_t i = 0; i < c->inst.size() && ii < 0; i++)
        if (!c->inst[i].live) ii = (int)i;
    if (ii < 0) return fail(c, SBOT_ERR_OOM, "admission refused: every instance slot is in use");
    TRY(admit(c, ii, desc, body));
    *slot = ii;
    return SBOT_OK;
}

sbot_status sbot_batch_retire(sbot_ctx_t c, int slot) {
    if (!c) return SBOT_ERR_ARG;
    if (slot < 0 || slot >= (int)c->inst.size() || !c->inst[slot].live)
        return fail(c, SBOT_ERR_ARG, "no live instance in that slot");
    drop_inst(c, slot);
    TRY(refresh_groups(c));
    TRY(flush(c));
    return end_frame(c);
}

sbot_status sbot_batch_select(sbot_ctx_t c, int slot) {
    if (!c) return SBOT_ERR_ARG;
    if (slot < 0 || slot >= (int)c->inst.size() || !c->inst[slot].live)
        return fail(c, SBOT_ERR_ARG, "no live instance in that slot");
    c->sel = slot;
    return SBOT_OK;
}

sbot_status sbot_batch_info(sbot_ctx_t c, int* live, int64_t* bytes, int64_t* cell_updates_per_step,
                            int64_t* coarse_steps_of_selected) {
    if (!c) return SBOT_ERR_ARG;
    int n = 0;
    int64_t cu = 0;
    for (auto& I : c->inst) {
        if (!I.live) continue;
        n++;
        cu += cell_updates(c, I);
    }
    if (live) *live = n;
    if (bytes) *bytes = bytes_in_use(c);
    if (cell_updates_per_step) *cell_updates_per_step = cu;
    if (coarse_steps_of_selected) {
        Inst* I = selected(c);
        *coarse_steps_of_selected = I ? I->coarse_step : -1;
    }
    return SBOT_OK;
}

sbot_status sbot_destroy(sbot_ctx_t c) {
    if (!c) return SBOT_OK;
    if (c->s) cudaStreamSynchronize(c->s);
    for (int i = 0; i < 2; i++) dfree(c->f[i]);
    void* ps[] = {c->d_nbr,    c->d_inst,  c->d_level, c->d_type,   c->d_ox,       c->d_oy,   c->d_flags,
                  c->d_parent, c->d_child, c->d_mask,  c->d_ip,     c->d_ist,      c->d_err,  c->d_lists,
                  c->d_counts, c->d_jobs,  c->d_out3,  c->d_one,    c->d_partials, c->d_recs,
                  c->d_ph[0],  c->d_ph[1], c->d_ph[2], c->d_ph[3], c->d_ctl, c->d_trace};
    for (void* p : ps) dfree(p);
    for (auto& I : c->inst) free_inst_device(I);
    for (int g = 0; g < 2; g++) drop_graph(c, g);
    for (int i = 0; i < 2; i++) {
        if (c->arena[i].host) cudaFreeHost(c->arena[i].host);
        if (c->arena[i].done) cudaEventDestroy(c->arena[i].done);
    }
    for (int i = 0; i < NGL; i++) {
        if (c->side[i]) cudaStreamSynchronize(c->side[i]);
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
        if (c->ev_fork[i]) cudaEventDestroy(c->ev_fork[i]);
        if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
    }
    for (int g = 0; g < SBOT_MAXLEV; g++) {
        if (c->gstream[g]) cudaStreamSynchronize(c->gstream[g]);
        if (c->gstream[g]) cudaStreamDestroy(c->gstream[g]);
        if (c->ev_gjoin[g]) cudaEventDestroy(c->ev_gjoin[g]);
        if (c->pstream[g]) cudaStreamSynchronize(c->pstream[g]);
        if (c->pstream[g]) cudaStreamDestroy(c->pstream[g]);
        if (c->ev_pose[g]) cudaEventDestroy(c->ev_pose[g]);
        if (c->ev_ibm_last[g]) cudaEventDestroy(c->ev_ibm_last[g]);
        if (c->ev_fsum[g]) cudaEventDestroy(c->ev_fsum[g]);
    }
    if (c->ev_gfork) cudaEventDestroy(c->ev_gfork);
    if (c->own_stream) cudaStreamDestroy(c->s);
    delete c;
    return SBOT_OK;
}

const char* sbot_last_error(sbot_ctx_t c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
