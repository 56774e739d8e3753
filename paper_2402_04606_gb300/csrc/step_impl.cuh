// The persistent step kernel: one launch runs one coarse step (Algorithm 1 of
// arXiv 2402.04606, unrolled over every level of every live instance) as a
// list of phases built by the host (api.cpp, build_step_phases):
//   PH_POSE   the poses of the coarse step of the moving bodies (Sec. 3.4-3.6)
//   PH_GEOM   the IBM geometry of one finest step of the moving bodies
//   PH_C2F    coarse-to-fine copy into the two halo layers (Sec. 2.4 step 2) at
//             the start of the coarse step; later copies are done by the coarse
//             sweep that produces the values (its cells next to the finer region)
//   PH_FUSED  pull streaming + boundary rules + collision of a work list of
//             blocks (Eqs. 3-10; the fine-to-coarse merge of Sec. 2.4 step 6
//             inside the coarse pull)
//   PH_IBM    multi-direct forcing of the bodies on their finest level (Sec. 2.2)
//   PH_FSUM   the FP64 force and moment sums of the coarse step (Eq. 16)
// Every phase is cut into tasks of one thread block.  A phase may start once
// every task of the phases it depends on has finished: each phase has a
// counter of finished tasks, raised by one reduction with release semantics
// after each task's writes; a block that wants to run a phase reads its
// dependencies' counters (relaxed loads, all at once) and, once every one is
// full, fences with acquire semantics before the task reads.  A phase with no
// work and no dependency is finished from the start; one with no work but
// with dependencies gets one empty task, so that it finishes after them.
//
// Scheduling.  Critical phases form one list in a topological order; bulk
// phases (level-0 blocks with no dependency inside the step, most of the
// cells of a large instance) form a queue of their own.  Warp 0 of a thread
// block looks at a window of critical phases after the first one that still
// has tasks to hand out and takes a task of one whose dependencies have
// finished; else it takes a bulk task; only when the bulk queue is empty does
// it take the first critical task not yet taken and wait for its
// dependencies.  Every phase depends only on earlier critical phases, a
// waiting block holds a task of the first phase with tasks left, and all
// thread blocks are resident at once (cooperative launch), so the earliest
// unfinished task can always run: the step completes.  Each wait is still
// bounded (spin_ns of device time): past it the thread block raises
// ERRB_TIMEOUT and the abort flag, and every block leaves at its next
// decision, so a broken schedule returns an error instead of hanging the
// device.
//
// Reads of buffers that other thread blocks wrote earlier in the launch use
// plain loads (no read-only cache path): the acquire fence after the
// dependency counters orders them after those writes.
#pragma once
#include "lbm_device.cuh"

namespace {

enum { STEP_EXIT = 0, STEP_RUN = 1 };

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class S>
__device__ __forceinline__ S* step_buf(const StepArgs& A, int i) {
    return i < 0 ? nullptr : (S*)(i == 0 ? A.f0 : A.f1);
}

// list items per task of a fused phase: the vector mapping covers one block
// per B * B / CPT threads (CPT cells per thread), the scalar one B * B cells
// per item over the thread block
template <class S, int B>
__device__ __forceinline__ bool fused_vec(const StepArgs& A, const StepPhase& ph, int n, int coll) {
    return B >= 16 && !(coll & COLL_SOLID) && ph.arg == 0 && A.vec_min_cells >= 0 &&
           (long long)n * B * B >= A.vec_min_cells;
}

template <class S, int B>
__device__ __forceinline__ int fused_items(bool vec, int T) {
    constexpr int CPT = sizeof(S) == 2 ? 8 : 4;
    return vec ? T / (B * B / CPT) : (T >= B * B ? T / (B * B) : 1);
}

// list items per round (per) and rounds per task of fused phase ph with n
// items: a bulk task, and a critical one whose phase would otherwise hand
// out more than 8 tasks per thread block (a whole level of a large grid, as
// in the later steps of a launch), take bulk_rounds thread-block fillings;
// another critical one at most crit_items items (so that a short sweep other
// phases wait for spreads over more SMs)
template <class S, int B>
__device__ __forceinline__ void task_shape(const StepArgs& A, const StepPhase& ph, int n, bool vec, int T, int& per,
                                           int& rounds) {
    per = fused_items<S, B>(vec, T);
    rounds = 1;
    if (ph.bulk || (long long)n > 8LL * per * gridDim.x) {
        rounds = A.bulk_rounds;
        return;
    }
    if (A.crit_items > 0 && A.crit_items < per) per = A.crit_items;
}

// tasks of phase p at this launch (from the device list lengths)
template <class S, int B>
__device__ int step_ntasks(const DevPool& P, const StepArgs& A, const StepPhase& ph, int T) {
    const int n = A.counts[ph.count_idx];
    if (n <= 0) return 0;
    switch (ph.kind) {
    case PH_FUSED: {
        int per, rounds;
        task_shape<S, B>(A, ph, n, fused_vec<S, B>(A, ph, n, P.coll), T, per, rounds);
        return (n + per * rounds - 1) / (per * rounds);
    }
    case PH_C2F: {
        const int per = T >= B * B ? T / (B * B) : 1;
        return (n + per - 1) / per;
    }
    case PH_FSUM: return n * ph.arg;
    default: return n;  // one body per task
    }
}

// the scalar mapping of a fused or copy phase: items [i0, i0 + k) of the list,
// B * B cells each, spread over the thread block's threads
template <class F>
__device__ __forceinline__ void for_cells(int n, int i0, int k, int BB, F&& fn) {
    const int cells = k * BB;
    for (int c = threadIdx.x; c < cells; c += blockDim.x) {
        const int item = i0 + c / BB;
        if (item < n) fn(item, c % BB);
    }
}

// the most list items a scalar task of a critical sweep holds (T / (B * B)
// for B >= 8)
#define STEP_META_MAX (STEP_MAX_THREADS / 64)

// A fused phase's task.  gate(): see step_task.  A critical task on the
// scalar mapping first reads its blocks' data (slot tables, neighbours and
// their types, children) into shared memory, which it may do before the
// phases it depends on have finished: after the gate only the population
// and force loads remain on its path.
template <class S, class C, int B, int COLL, class G>
__device__ void step_fused(const DevPool& P, const StepArgs& A, const StepPhase& ph, int local, G& gate) {
    __shared__ SlotMeta meta[STEP_META_MAX];
    const int n = A.counts[ph.count_idx];
    const int* list = A.lists + ph.list_off;
    const S* fin = step_buf<S>(A, ph.fin);
    S* fout = step_buf<S>(A, ph.fout);
    const S* ffine = step_buf<S>(A, ph.ffine);
    S* fhalo = ph.fold ? step_buf<S>(A, ph.ffine) : nullptr;  // the coarse-to-fine copy rides on this sweep
    const int T = blockDim.x;
    const bool vec = fused_vec<S, B>(A, ph, n, P.coll);
    int per, rounds;
    task_shape<S, B>(A, ph, n, vec, T, per, rounds);
    if (!ph.bulk && rounds == 1 && !vec && per <= STEP_META_MAX && per <= T / 32) {
        const int i0 = local * per, ne = min(n, i0 + per), w = threadIdx.x >> 5;
        if (i0 + w < ne) load_meta(P, list[i0 + w], meta[w]);
        if (!gate(true)) return;
        for_cells(ne, i0, per, B * B, [&](int item, int cell) {
            const SlotMeta& m = meta[item - i0];
            fused_cell<S, C, COLL, false, MetaS>(P, MetaS{&m}, fin, fout, ffine, m.type, P.inst[m.inst], ph.level,
                                                 cell % B, cell / B, ph.allow_force != 0, fhalo);
        });
        return;
    }
    if (!gate(false)) return;
    for (int r = 0; r < rounds; r++) {
        const int i0 = (local * rounds + r) * per;
        if (i0 >= n) break;
        const int ne = min(n, i0 + per);  // this round's items end here
        if constexpr (B >= 16) {
            if (vec) {
                if constexpr (sizeof(S) == 2)
                    fused_v8_task<S, C, B, COLL, false, true>(P, list, ne, i0, fin, fout, ffine, ph.level,
                                                              ph.allow_force, fhalo);
                else
                    fused_v4_task<S, C, B, COLL, false>(P, list, ne, i0, fin, fout, ffine, ph.level, ph.allow_force,
                                                        fhalo);
                continue;
            }
        }
        for_cells(ne, i0, per, B * B, [&](int item, int cell) {
            const int slot = list[item];
            fused_cell<S, C, COLL, false>(P, fin, fout, ffine, slot, P.slot_type[slot], P.inst[P.slot_inst[slot]],
                                          ph.level, cell % B, cell / B, ph.allow_force != 0, fhalo);
        });
    }
}

// One task of phase ph.  gate(prologue) is called exactly once by the whole
// thread block: it waits, when the task was taken before the phases it
// depends on had finished, for them; the task reads nothing they write
// before it.  prologue: the task wrote shared memory before it (a barrier
// is then due even when there is nothing to wait for).  It returns false
// when the launch is aborting (the task then stops).
template <class S, class C, int B, int COLL, class G>
__device__ void step_task(const DevPool& P, const StepArgs& A, const StepPhase& ph, int local, unsigned char* smraw,
                          IbmShared& sh, G& gate) {
    const int* list = A.lists + ph.list_off;
    if (A.counts[ph.count_idx] <= 0) {  // the empty task of a phase with no work
        gate(false);
        return;
    }
    switch (ph.kind) {
    case PH_FUSED: step_fused<S, C, B, COLL>(P, A, ph, local, gate); break;
    case PH_IBM: ibm_run<S, C>(P, list[local], step_buf<S>(A, ph.fin), ph.level, 0, 1, smraw, sh, gate); break;
    default: {
        if (!gate(false)) return;
        switch (ph.kind) {
        case PH_C2F: {
            const int n = A.counts[ph.count_idx], k = blockDim.x >= B * B ? blockDim.x / (B * B) : 1;
            const S* fc = step_buf<S>(A, ph.fin);
            S* ff = step_buf<S>(A, ph.fout);
            for_cells(n, local * k, k, B * B, [&](int item, int cell) { c2f_cell<S>(P, list[item], cell, fc, ff); });
            break;
        }
        case PH_GEOM: ibm_geom_run<C>(P, list[local], ph.arg, smraw, sh); break;
        case PH_POSE: pose_run(P, list[local]); break;
        case PH_FSUM: force_sum_run<C>(P, list[local / ph.arg], local % ph.arg, sh.red); break;
        default: break;
        }
    }
    }
}

// the last phase whose first task index (exclusive prefix `first`) is at most t
__device__ __forceinline__ int phase_of(const int* first, int nph, int t) {
    int lo = 0, hi = nph - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int ld_relaxed(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ void step_abort(const DevPool& P, const StepArgs& A, int bit) {
    atomicOr(P.err, bit);
    atomicExch(&A.ctl->abort, 1);
}

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The dependencies of every phase, copied to shared memory at the start of
// the launch (the phase table does not change during it).
struct StepDeps {
    int n[STEP_MAX_PHASES];
    unsigned short d[STEP_MAX_PHASES][8];
};

// One thread: has every phase that q depends on finished all its tasks?
// Relaxed loads, issued together: a screen; a yes is confirmed by
// deps_acquire before the task runs.
__device__ __forceinline__ bool deps_screen(const StepArgs& A, const StepDeps& D, int q, const int* ntask) {
    const int nd = D.n[q];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (k < nd) {
            const int d = D.d[q][k];
            ok &= ld_relaxed_gpu(&A.ctl->done[d]) >= ntask[d];
        }
    }
    return ok;
}

// Warp 0, all lanes: the same question with acquire loads, lane k reading
// dependency k (one round trip); after a yes, the writes of those phases are
// visible to the warp and, through the barrier that follows, to the block.
__device__ __forceinline__ bool deps_acquire(const StepArgs& A, const StepDeps& D, int q, const int* ntask) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < D.n[q]) {
        const int d = D.d[q][lane];
        ok = ld_acquire(&A.ctl->done[d]) >= ntask[d];
    }
    return __all_sync(0xffffffffu, ok);
}

// Warp 0, all lanes: wait until every dependency of phase q has finished,
// bounded by A.spin_ns of device time; false when the launch is aborting (by
// this wait or another)
__device__ bool wait_deps(const DevPool& P, const StepArgs& A, const StepDeps& D, int q, const int* ntask) {
    const unsigned long long t0 = global_ns();
    for (unsigned ns = 16;; ns = ns < 64 ? 2 * ns : ns) {  // short naps: each poll is an L2 round trip anyway
        if (deps_acquire(A, D, q, ntask)) return true;
        int stop = 0;
        if ((threadIdx.x & 31) == 0) {
            if (ld_relaxed(&A.ctl->abort)) {
                stop = 1;
            } else if ((long long)(global_ns() - t0) >= A.spin_ns) {
                step_abort(P, A, ERRB_TIMEOUT);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        __nanosleep(ns);
    }
}

template <class S, class C, int B, int COLL>
__global__ void __launch_bounds__(sizeof(S) == 8 ? 256 : STEP_MAX_THREADS) k_step(const __grid_constant__ DevPool P, const __grid_constant__ StepArgs A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ IbmShared sh;
    __shared__ int ntask[STEP_MAX_PHASES];   // tasks of each phase at this launch
    __shared__ StepDeps deps;                // dependencies of each phase
    __shared__ int crit[STEP_MAX_PHASES];    // the critical phases with tasks, in list order
    __shared__ int cpos[STEP_MAX_PHASES];    // (scratch: their positions)
    __shared__ int bfirst[STEP_MAX_PHASES];  // first task of each phase in the bulk queue
    __shared__ int wtot[32];
    // the scheduler's state lives in shared memory, so that no register is
    // held across a task (the vector sweep needs all of them)
    __shared__ int s_cmd, s_phase, s_local, s_last, s_ncp, s_nbulk, s_bulk_left;
    __shared__ int s_wait, s_go;  // the claimed critical phase to wait for (-1: none), the wait's outcome
    const int tid = threadIdx.x, nph = A.nph;
    StepCtl* ctl = A.ctl;
    constexpr unsigned FULL = 0xffffffffu;

    // task counts from this launch's list lengths (a critical phase with no
    // work but with dependencies gets one empty task, so that the phases after
    // it wait for its dependencies); the critical phases that have tasks,
    // compacted in order; the bulk queue's prefix sums
    for (int p = tid; p < nph; p += blockDim.x) {
        const StepPhase& ph = A.ph[p];
        int nt = step_ntasks<S, B>(P, A, ph, blockDim.x);
        if (nt == 0 && !ph.bulk && ph.ndep > 0) nt = 1;
        ntask[p] = nt;
        deps.n[p] = ph.ndep;
        for (int k = 0; k < ph.ndep; k++) deps.d[p][k] = (unsigned short)ph.dep[k];
        cpos[p] = (!ph.bulk && nt > 0) ? 1 : 0;
        bfirst[p] = ph.bulk ? nt : 0;
    }
    __syncthreads();
    {
        const int ncp = block_scan_inplace(cpos, nph, wtot);
        const int nbulk = block_scan_inplace(bfirst, nph, wtot);
        if (tid == 0) {
            s_ncp = ncp;
            s_nbulk = nbulk;
            s_bulk_left = nbulk > 0;
        }
    }
    for (int p = tid; p < nph; p += blockDim.x)
        if (!A.ph[p].bulk && ntask[p] > 0) crit[cpos[p]] = p;
    __syncthreads();
    if (A.tr_start && tid == 0) atomicMin(&A.tr_start[STEP_MAX_PHASES], global_ns());

    for (;;) {
        if (threadIdx.x < 32) {  // warp 0 decides
            const int lane = threadIdx.x, ncp = s_ncp, nbulk = s_nbulk;
            int cmd = STEP_EXIT, p = -1, local = 0;
            int wq = -1;  // a claimed critical phase: its dependencies are read with acquire before it runs
            if (!ld_relaxed(&ctl->abort)) {
                bool got = false;
                // 1. a task of a critical phase whose dependencies have
                //    finished, in a window after the first one with tasks
                //    left to take
                const int h = ld_relaxed(&ctl->head);
                for (int base = h; !got && base < ncp && base < h + 64; base += 32) {
                    const int i = base + lane;
                    const int q = i < ncp ? crit[i] : -1;
                    const bool avail = q >= 0 && ld_relaxed(&ctl->taken[q]) < ntask[q];
                    const bool rdy = avail && deps_screen(A, deps, q, ntask);
                    if (base == h) {  // phases that have nothing left to take leave the window for good
                        const unsigned av = __ballot_sync(FULL, avail);
                        const int nh = av ? base + __ffs(av) - 1 : min(base + 32, ncp);
                        if (lane == 0 && nh > h) atomicMax(&ctl->head, nh);
                    }
                    unsigned m = __ballot_sync(FULL, rdy);
                    while (m && !got) {
                        const int qq = __shfl_sync(FULL, q, __ffs(m) - 1);
                        int t = 0;
                        if (lane == 0) t = atomicAdd(&ctl->taken[qq], 1);
                        t = __shfl_sync(FULL, t, 0);
                        if (t < ntask[qq]) {
                            got = true;
                            p = qq;
                            local = t;
                            wq = qq;
                        }
                        m &= m - 1;
                    }
                }
                // 2. else a bulk task (no dependency)
                if (!got && s_bulk_left) {
                    int b = 0;
                    if (lane == 0) b = atomicAdd(&ctl->bulk_next, 1);
                    b = __shfl_sync(FULL, b, 0);
                    if (b < nbulk) {
                        got = true;
                        p = phase_of(bfirst, nph, b);
                        local = b - bfirst[p];
                        cmd = STEP_RUN;
                    } else if (lane == 0) {
                        s_bulk_left = 0;
                    }
                }
                // 3. else the first critical task not yet taken, waiting for
                //    its dependencies (every phase before it in the order has
                //    all its tasks taken)
                if (!got) {
                    if (lane == 0) {
                        for (int i = ld_relaxed(&ctl->head); i < ncp; i++) {
                            const int q = crit[i];
                            if (ld_relaxed(&ctl->taken[q]) >= ntask[q]) continue;
                            const int t = atomicAdd(&ctl->taken[q], 1);
                            if (t < ntask[q]) {
                                p = q;
                                local = t;
                                break;
                            }
                        }
                    }
                    p = __shfl_sync(FULL, p, 0);
                    local = __shfl_sync(FULL, local, 0);
                    wq = p;
                }
                if (wq >= 0) cmd = STEP_RUN;
            }
            if (lane == 0) {
                s_cmd = cmd;
                s_phase = p;
                s_local = local;
                s_wait = wq;
                s_go = 1;
            }
        }
        __syncthreads();
        if (s_cmd != STEP_RUN) break;
        // the task's gate: a claimed critical task waits here (warp 0, with
        // acquire loads) for the phases it depends on, after whatever part
        // of the task may run before them
        auto gate = [&](bool prologue = true) -> bool {
            if (!prologue && s_wait < 0) {  // nothing to wait for, nothing to publish
                if (threadIdx.x == 0 && A.tr_start) {
                    const unsigned long long t = global_ns();
                    atomicMin(&A.tr_start[s_phase], t);
                    atomicMax(&A.tr_start2[s_phase], t);
                }
                return true;
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                const int q = s_wait;
                const bool ok = q < 0 || wait_deps(P, A, deps, q, ntask);
                if (threadIdx.x == 0) {
                    s_go = ok;
                    if (ok && A.tr_start) {
                        const unsigned long long t = global_ns();
                        atomicMin(&A.tr_start[s_phase], t);
                        atomicMax(&A.tr_start2[s_phase], t);
                    }
                }
            }
            __syncthreads();
            return s_go != 0;
        };
        step_task<S, C, B, COLL>(P, A, A.ph[s_phase], s_local, smraw, sh, gate);
        __syncthreads();  // the task's writes, then its count (a release: the
                          // barrier orders every thread's writes before it)
        if (threadIdx.x == 0 && s_go) {
            const int p = s_phase;
            if (A.tr_start) {  // the task's end, before it is counted
                const unsigned long long t = global_ns();
                atomicMax(&A.tr_end[p], t);
                atomicMin(&A.tr_end1[p], t);
                atomicAdd(&A.tr_tasks[p], 1);
            }
            red_release_add(&ctl->done[p], 1);
        }
    }
    // the last thread block to leave zeroes the control block for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&ctl->exited, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int p = threadIdx.x; p < nph; p += blockDim.x) {
            ctl->taken[p] = 0;
            ctl->done[p] = 0;
        }
        if (threadIdx.x == 0) {
            ctl->head = 0;
            ctl->bulk_next = 0;
            ctl->abort = 0;
            ctl->exited = 0;
        }
    }
}

template <class S, class C, int B, int COLL>
cudaError_t launch_step_k(const DevPool& P, const StepArgs& A, int grid, int threads, size_t smem, cudaStream_t s) {
    auto kern = k_step<S, C, B, COLL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;  // every thread block resident at once
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P, A);
}

template <class S, class C, int B, int COLL>
int occupancy_k(int threads, size_t smem, size_t* static_smem) {
    auto kern = k_step<S, C, B, COLL>;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
    if (static_smem) *static_smem = fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

// the kernel of the context's block size and collision kind, one storage type
template <class S, class C>
int launch_step_s(const DevPool& P, const StepArgs& A, int grid, int threads, size_t smem, cudaStream_t s) {
    const int k = P.coll & 15;
    cudaError_t e = cudaErrorInvalidValue;
    if (P.B == 8)
        e = k == 1 ? launch_step_k<S, C, 8, 1>(P, A, grid, threads, smem, s)
                   : (k == 2 ? launch_step_k<S, C, 8, 2>(P, A, grid, threads, smem, s)
                             : launch_step_k<S, C, 8, 0>(P, A, grid, threads, smem, s));
    else if (P.B == 16)
        e = k == 1 ? launch_step_k<S, C, 16, 1>(P, A, grid, threads, smem, s)
                   : (k == 2 ? launch_step_k<S, C, 16, 2>(P, A, grid, threads, smem, s)
                             : launch_step_k<S, C, 16, 0>(P, A, grid, threads, smem, s));
    else if (P.B == 32)
        e = k == 1 ? launch_step_k<S, C, 32, 1>(P, A, grid, threads, smem, s)
                   : (k == 2 ? launch_step_k<S, C, 32, 2>(P, A, grid, threads, smem, s)
                             : launch_step_k<S, C, 32, 0>(P, A, grid, threads, smem, s));
    return (int)e;
}

template <class S, class C>
int step_occupancy_s(int B, int coll, int threads, size_t smem, size_t* static_smem) {
    const int k = coll & 15;
    if (B == 8)
        return k == 1 ? occupancy_k<S, C, 8, 1>(threads, smem, static_smem)
                      : (k == 2 ? occupancy_k<S, C, 8, 2>(threads, smem, static_smem)
                                : occupancy_k<S, C, 8, 0>(threads, smem, static_smem));
    if (B == 16)
        return k == 1 ? occupancy_k<S, C, 16, 1>(threads, smem, static_smem)
                      : (k == 2 ? occupancy_k<S, C, 16, 2>(threads, smem, static_smem)
                                : occupancy_k<S, C, 16, 0>(threads, smem, static_smem));
    if (B == 32)
        return k == 1 ? occupancy_k<S, C, 32, 1>(threads, smem, static_smem)
                      : (k == 2 ? occupancy_k<S, C, 32, 2>(threads, smem, static_smem)
                                : occupancy_k<S, C, 32, 0>(threads, smem, static_smem));
    return 0;
}

}  // namespace
