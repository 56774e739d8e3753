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
// every task of the phases it depends on has finished: a per-phase counter of
// finished tasks, raised with release semantics after the task's writes and
// read with acquire semantics before the dependent task reads.
//
// Scheduling.  Critical phases form one list in a topological order; bulk
// phases (level-0 blocks with no dependency inside the step, most of the
// cells of a large instance) form a queue of their own.  A phase is ready
// once every phase it depends on has completed: the thread block that
// finishes a phase's last task counts it off for each phase that waits for
// it (a phase without tasks completes as soon as it is ready).  Warp 0 of a
// thread block looks at a window of critical phases after the first one that
// still has tasks to hand out and takes a task of a ready one; else it takes
// a bulk task; only when the bulk queue is empty does it take the first
// critical task not yet taken and wait for its phase.  Every phase depends
// only on earlier critical phases, a waiting block holds a task of the first
// phase with tasks left, and all thread blocks are resident at once
// (cooperative launch), so the earliest unfinished task can always run: the
// step completes.  Each wait is still bounded (spin_ns of device time): past
// it the thread block raises ERRB_TIMEOUT and the abort flag, and every
// block leaves at its next decision, so a broken schedule returns an error
// instead of hanging the device.
//
// Reads of buffers that other thread blocks wrote earlier in the launch use
// plain loads (no read-only cache path): the acquire on the dependency
// counter orders them after those writes.
#pragma once
#include "lbm_device.cuh"

namespace {

enum { STEP_EXIT = 0, STEP_RUN = 1 };

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

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

// tasks of phase p at this launch (from the device list lengths)
template <class S, int B>
__device__ int step_ntasks(const DevPool& P, const StepArgs& A, const StepPhase& ph, int T) {
    const int n = A.counts[ph.count_idx];
    if (n <= 0) return 0;
    switch (ph.kind) {
    case PH_FUSED: {
        const int per = fused_items<S, B>(fused_vec<S, B>(A, ph, n, P.coll), T) * (ph.bulk ? A.bulk_rounds : 1);
        return (n + per - 1) / per;
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

template <class S, class C, int B, int COLL>
__device__ void step_fused(const DevPool& P, const StepArgs& A, const StepPhase& ph, int local) {
    const int n = A.counts[ph.count_idx];
    const int* list = A.lists + ph.list_off;
    const S* fin = step_buf<S>(A, ph.fin);
    S* fout = step_buf<S>(A, ph.fout);
    const S* ffine = step_buf<S>(A, ph.ffine);
    S* fhalo = ph.fold ? step_buf<S>(A, ph.ffine) : nullptr;  // the coarse-to-fine copy rides on this sweep
    const int T = blockDim.x, rounds = ph.bulk ? A.bulk_rounds : 1;
    const bool vec = fused_vec<S, B>(A, ph, n, P.coll);
    const int per = fused_items<S, B>(vec, T);
    for (int r = 0; r < rounds; r++) {
        const int i0 = (local * rounds + r) * per;
        if (i0 >= n) break;
        if constexpr (B >= 16) {
            if (vec) {
                if constexpr (sizeof(S) == 2)
                    fused_v8_task<S, C, B, COLL, false>(P, list, n, i0, fin, fout, ffine, ph.level, ph.allow_force,
                                                        fhalo);
                else
                    fused_v4_task<S, C, B, COLL, false>(P, list, n, i0, fin, fout, ffine, ph.level, ph.allow_force,
                                                        fhalo);
                continue;
            }
        }
        for_cells(n, i0, per, B * B, [&](int item, int cell) {
            const int slot = list[item];
            fused_cell<S, C, COLL, false>(P, fin, fout, ffine, slot, P.slot_type[slot], P.inst[P.slot_inst[slot]],
                                          ph.level, cell % B, cell / B, ph.allow_force != 0, fhalo);
        });
    }
}

template <class S, class C, int B, int COLL>
__device__ void step_task(const DevPool& P, const StepArgs& A, const StepPhase& ph, int local, unsigned char* smraw,
                          IbmShared& sh) {
    const int* list = A.lists + ph.list_off;
    switch (ph.kind) {
    case PH_FUSED: step_fused<S, C, B, COLL>(P, A, ph, local); break;
    case PH_C2F: {
        const int n = A.counts[ph.count_idx], k = blockDim.x >= B * B ? blockDim.x / (B * B) : 1;
        const S* fc = step_buf<S>(A, ph.fin);
        S* ff = step_buf<S>(A, ph.fout);
        for_cells(n, local * k, k, B * B, [&](int item, int cell) { c2f_cell<S>(P, list[item], cell, fc, ff); });
        break;
    }
    case PH_IBM: ibm_run<S, C>(P, list[local], step_buf<S>(A, ph.fin), ph.level, 0, 1, smraw, sh); break;
    case PH_GEOM: ibm_geom_run<C>(P, list[local], ph.arg, smraw, sh); break;
    case PH_POSE: pose_run(P, list[local]); break;
    case PH_FSUM: force_sum_run<C>(P, list[local / ph.arg], local % ph.arg, sh.red); break;
    default: break;
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

__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void step_abort(const DevPool& P, const StepArgs& A, int bit) {
    atomicOr(P.err, bit);
    atomicExch(&A.ctl->abort, 1);
}

// Phase p has completed: count it off for the phases that wait for it, and
// complete in turn every one of them that has no task and is now ready.
// One thread.
__device__ __noinline__ void step_complete(const DevPool& P, const StepArgs& A, int p, const int* ntask) {
    int stack[32];
    int top = 0;
    stack[top++] = p;
    while (top > 0) {
        const StepPhase& ph = A.ph[stack[--top]];
        for (int k = 0; k < ph.nsucc; k++) {
            const int r = ph.succ[k];
            const int now = atom_add_acq_rel(&A.ctl->ready[r], 1) + 1;
            if (now == A.ph[r].ndep && ntask[r] == 0) {
                if (top < 32)
                    stack[top++] = r;
                else
                    step_abort(P, A, ERRB_SCHED);
            }
        }
    }
}

// one thread: wait until phase p is ready, bounded by A.spin_ns of device
// time; false when the launch is aborting (by this wait or another)
__device__ bool wait_ready(const DevPool& P, const StepArgs& A, int p, int ndep) {
    const unsigned long long t0 = global_ns();
    for (unsigned ns = 32;; ns = ns < 256 ? 2 * ns : ns) {
        if (ld_acquire(&A.ctl->ready[p]) >= ndep) return true;
        if (ld_relaxed(&A.ctl->abort)) return false;
        if ((long long)(global_ns() - t0) >= A.spin_ns) {
            step_abort(P, A, ERRB_TIMEOUT);
            return false;
        }
        __nanosleep(ns);
    }
}

template <class S, class C, int B, int COLL>
__global__ void __launch_bounds__(sizeof(S) == 8 ? 256 : STEP_MAX_THREADS) k_step(DevPool P, StepArgs A) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ IbmShared sh;
    __shared__ int ntask[STEP_MAX_PHASES];   // tasks of each phase at this launch
    __shared__ int ndep[STEP_MAX_PHASES];    // dependencies of each phase
    __shared__ int crit[STEP_MAX_PHASES];    // the critical phases with tasks, in list order
    __shared__ int cpos[STEP_MAX_PHASES];    // (scratch: their positions)
    __shared__ int bfirst[STEP_MAX_PHASES];  // first task of each phase in the bulk queue
    __shared__ int wtot[32];
    // the scheduler's state lives in shared memory, so that no register is
    // held across a task (the vector sweep needs all of them)
    __shared__ int s_cmd, s_phase, s_local, s_last, s_ncp, s_nbulk, s_bulk_left;
    const int tid = threadIdx.x, nph = A.nph;
    StepCtl* ctl = A.ctl;
    constexpr unsigned FULL = 0xffffffffu;

    // task counts from this launch's list lengths; the critical phases that
    // have tasks, compacted in order; the bulk queue's prefix sums
    for (int p = tid; p < nph; p += blockDim.x) {
        const StepPhase& ph = A.ph[p];
        const int nt = step_ntasks<S, B>(P, A, ph, blockDim.x);
        ntask[p] = nt;
        ndep[p] = ph.ndep;
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
    // phases with neither a task nor a dependency are complete from the start
    if (blockIdx.x == 0 && tid == 0)
        for (int p = 0; p < nph; p++)
            if (ntask[p] == 0 && ndep[p] == 0) step_complete(P, A, p, ntask);
    if (A.tr_start && tid == 0) atomicMin(&A.tr_start[STEP_MAX_PHASES], global_ns());

    for (;;) {
        if (threadIdx.x < 32) {  // warp 0 decides
            const int lane = threadIdx.x, ncp = s_ncp, nbulk = s_nbulk;
            int cmd = STEP_EXIT, p = -1, local = 0;
            if (!ld_relaxed(&ctl->abort)) {
                bool got = false;
                // 1. a task of a critical phase that is ready, in a window
                //    after the first one with tasks left to take
                const int h = ld_relaxed(&ctl->head);
                for (int base = h; !got && base < ncp && base < h + 64; base += 32) {
                    const int i = base + lane;
                    const int q = i < ncp ? crit[i] : -1;
                    const bool avail = q >= 0 && ld_relaxed(&ctl->taken[q]) < ntask[q];
                    const bool rdy = avail && ld_acquire(&ctl->ready[q]) >= ndep[q];
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
                            cmd = STEP_RUN;
                        }
                        m &= m - 1;
                    }
                }
                // 2. else a bulk task
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
                // 3. else the first critical task not yet taken, waiting for it
                //    (every phase before it in the order has all its tasks taken)
                if (!got && lane == 0) {
                    for (int i = ld_relaxed(&ctl->head); i < ncp; i++) {
                        const int q = crit[i];
                        if (ld_relaxed(&ctl->taken[q]) >= ntask[q]) continue;
                        const int t = atomicAdd(&ctl->taken[q], 1);
                        if (t < ntask[q]) {
                            p = q;
                            local = t;
                            if (wait_ready(P, A, q, ndep[q])) cmd = STEP_RUN;
                            break;
                        }
                    }
                }
            }
            if (lane == 0) {
                s_cmd = cmd;
                s_phase = p;
                s_local = local;
            }
        }
        __syncthreads();
        if (s_cmd != STEP_RUN) break;
        if (A.tr_start && threadIdx.x == 0) {
            const unsigned long long t = global_ns();
            atomicMin(&A.tr_start[s_phase], t);
            atomicMax(&A.tr_start2[s_phase], t);
        }
        step_task<S, C, B, COLL>(P, A, A.ph[s_phase], s_local, smraw, sh);
        __syncthreads();  // the task's writes, then its completion
        if (threadIdx.x == 0) {
            const int p = s_phase;
            __threadfence();
            const int d = atom_add_acq_rel(&ctl->done[p], 1) + 1;
            if (d == ntask[p]) step_complete(P, A, p, ntask);
            if (A.tr_start) {
                const unsigned long long t = global_ns();
                atomicMax(&A.tr_end[p], t);
                atomicMin(&A.tr_end1[p], t);
                atomicAdd(&A.tr_tasks[p], 1);
            }
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
            ctl->ready[p] = 0;
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
