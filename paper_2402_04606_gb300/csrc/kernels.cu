// CUDA kernels (sm_103a) of the lattice-Boltzmann / immersed-boundary /
// block-refinement time step of arXiv 2402.04606.
//
// Kernels
//   k_fused        pull streaming (Eq. 10) + boundary rules + moments (Eq. 8) +
//                  BGK collision with Guo forcing (Eqs. 3, 6, 7) on the leaf
//                  blocks of one level; on fine-side halo blocks the same pull
//                  without collision (Sec. 2.4 steps 3 and 5); the MRT and LES
//                  collisions (Sec. 2.1) as variants.
//   k_fused_v4     the same for large lists, 4 cells per thread (FP32, FP64);
//   k_fused_v8     8 cells per thread (FP16, BF16); k_fused_tma the variant
//                  staged in shared memory by bulk copies.
//   k_c2f          coarse-to-fine copy into the two halo layers (Sec. 2.4 step 2).
//   merge_fine     fine-to-coarse merge of the halo layers (Sec. 2.4 step 6),
//                  evaluated inside the coarse pull (no kernel of its own).
//   k_ibm          multi-direct-forcing immersed boundary on the finest level
//                  (Sec. 2.2, Eqs. 11-16), one thread block per body;
//                  k_ibm_geom its geometry for moving bodies, k_force_sum the
//                  Eq. 16 sums of a coarse step, k_pose the body poses.
//   k_export / k_set_pre / k_checksum   state in and out.
//
// All arithmetic on the populations is done here; the host only plans.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <climits>
#include <type_traits>

#include "lbm_device.cuh"

namespace {

// fused stream + collide on one level, one thread per cell (any block size;
// used for 8 x 8 blocks and for blocks next to the finer region).  fhalo
// (may be null): the finer level's buffer (the one ffine points to) whose
// halo cells the cells next to the finer region fill with their
// post-collision values, the coarse-to-fine copy of the next sub-step.
template <class S, class C, int COLL, bool SOLID>
__global__ void __launch_bounds__(1024) k_fused(const __grid_constant__ DevPool P, const int* __restrict__ list, const int* __restrict__ pn,
                                                const S* __restrict__ fin, S* __restrict__ fout, const S* ffine,
                                                int level, int allow_force, S* fhalo) {
    pdl_enter();
    int item = blockIdx.x;
    if (item >= *pn) return;
    const int B = P.B;
    int slot = list[item];
    int cell = threadIdx.x;
    fused_cell<S, C, COLL, SOLID>(P, fin, fout, ffine, slot, P.slot_type[slot], P.inst[P.slot_inst[slot]], level,
                                  cell % B, cell / B, allow_force != 0, fhalo);
}

// (the LES variants spill at the 80 registers that 3 blocks per SM leave;
// at 2 blocks per SM they fit in 112 registers but measured slower on the
// 8192^2 sweep, 3.12 against 3.89 TB/s, so they keep 3)
template <class S, class C, int B, int COLL>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 1 : 3)
    k_fused_v4(const __grid_constant__ DevPool P, const int* __restrict__ list, const int* __restrict__ pn, const S* __restrict__ fin,
               S* __restrict__ fout, const S* __restrict__ ffine, int level, int allow_force) {
    pdl_enter();
    constexpr int SPC = 256 / (B * B / 4);
    const int n = *pn;
    for (int i0 = blockIdx.x * SPC; i0 < n; i0 += gridDim.x * SPC) {  // grid stride (vec_grid)
        fused_v4_task<S, C, B, COLL, true>(P, list, n, i0, fin, fout, ffine, level, allow_force);
        __syncthreads();  // the task's neighbour table is rewritten by the next one
    }
}

// Thread blocks of a vector-kernel launch: at most `waves` waves of resident
// blocks (3 per SM, SBOT_TUNE_VEC_WAVES, default 8), each walking the list
// with a grid stride; waves <= 0: one block per list group.  Fewer,
// longer-lived blocks than one per list group measured faster on the 8192^2
// sweep (FP32 0.82 -> 0.85, BF16 0.71 -> 0.75 of the measured copy
// bandwidth): less block launch and tail per sweep.
unsigned vec_grid(unsigned want, int waves) {
    static int sms = 0;
    if (waves <= 0) return want;
    if (sms == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            return want;
        }
        sms = n;
    }
    const unsigned cap = (unsigned)sms * 3u * (unsigned)waves;
    return want < cap ? want : cap;
}

// SH: some instance of the context stores a shifted 16-bit state (COLL_SHIFT)
template <class S, class C, int B, int COLL, bool SH>
__global__ void __launch_bounds__(256, 3)
    k_fused_v8(const __grid_constant__ DevPool P, const int* __restrict__ list, const int* __restrict__ pn, const S* __restrict__ fin,
               S* __restrict__ fout, const S* __restrict__ ffine, int level, int allow_force) {
    pdl_enter();
    constexpr int SPC = 256 / (B * B / 8);
    const int n = *pn;
    for (int i0 = blockIdx.x * SPC; i0 < n; i0 += gridDim.x * SPC) {  // grid stride (vec_grid)
        fused_v8_task<S, C, B, COLL, true, SH>(P, list, n, i0, fin, fout, ffine, level, allow_force);
        __syncthreads();  // the task's neighbour table is rewritten by the next one
    }
}

// collision only, on pre-collision populations (the state at t = 0)
template <class S, class C, int COLL>
__global__ void __launch_bounds__(1024) k_collide_init(const __grid_constant__ DevPool P, const int* __restrict__ list, int n,
                                                       const S* __restrict__ fpre, S* __restrict__ fpost, int level) {
    int item = blockIdx.x;
    if (item >= n) return;
    const int B = P.B, BB = B * B;
    int slot = list[item];
    int cell = threadIdx.x;
    const InstParams& ip = P.inst[P.slot_inst[slot]];
    C f[9];
#pragma unroll
    for (int q = 0; q < 9; q++) f[q] = Sto<S>::template ld<C>(fpre, ((size_t)slot * 9 + q) * BB + cell, q, ip.dref);
    C Fx = 0, Fy = 0;
    int gx = P.slot_ox[slot] + cell % B, gy = P.slot_oy[slot] + cell / B;
    if (ip.has_body && level == ip.m - 1) patch_force<C>(P, ip, gx, gy, Fx, Fy);
    collide_k<COLL, C, true, DevTrait<S>::value, sizeof(S) == 4>(f, (C)1 / (C)ip.tau[level], Fx, Fy, ip);
#pragma unroll
    for (int q = 0; q < 9; q++) Sto<S>::template st<C>(fpost, ((size_t)slot * 9 + q) * BB + cell, q, f[q], ip.dref);
}

template <class S>
__global__ void __launch_bounds__(1024) k_c2f(const __grid_constant__ DevPool P, const int* __restrict__ list, const int* __restrict__ pn,
                                              const S* __restrict__ fc, S* __restrict__ ff) {
    pdl_enter();
    int item = blockIdx.x;
    if (item >= *pn) return;
    c2f_cell<S>(P, list[item], threadIdx.x, fc, ff);
}

// ---------------------------------------------------------------------------
// Fused stream + collide with the block's populations staged in shared memory
// by the tensor memory accelerator's bulk copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy completing on `bar` (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 4 consecutive values of one population plane from shared memory, as compute type
template <class S, class C>
struct Vec4s;
template <class C>
struct Vec4s<float, C> {
    static __device__ __forceinline__ void ld(const float* p, C* v) {
        float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
};
template <class C>
struct Vec4s<double, C> {
    static __device__ __forceinline__ void ld(const double* p, C* v) {
        double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
};
template <class C>
struct Vec4s<__half, C> {
    static __device__ __forceinline__ void ld(const __half* p, C* v) {
        uint2 t = *reinterpret_cast<const uint2*>(p);
        float2 a = __half22float2(*reinterpret_cast<__half2*>(&t.x));
        float2 b = __half22float2(*reinterpret_cast<__half2*>(&t.y));
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
};
template <class C>
struct Vec4s<__nv_bfloat16, C> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16* p, C* v) {
        uint2 t = *reinterpret_cast<const uint2*>(p);
        float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&t.x));
        float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&t.y));
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
};

// Shared memory of one block in k_fused_tma, in elements of S: its 9
// population planes (bulk copies), the neighbour rows that the y-shifted
// populations pull (bulk copies: the bottom block's last row for c_y = +1,
// the top block's first row for c_y = -1), the neighbour columns of the
// x-shifted populations and the 4 diagonal corners (plain loads).
template <int B>
struct TmaSlot {
    static constexpr int BB = B * B;
    static constexpr int planes = 0, rows = 9 * BB, cols = rows + 9 * B, corner = cols + 9 * B;
    static constexpr int elems = corner + 16;  // a multiple of 16 bytes for every storage type
};
#define TMA_SPIN_LIMIT (1 << 22)  // polls of the copy barrier before the launch reports ERRB_TIMEOUT

template <class S, class C, int B, int COLL>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 1 : (sizeof(S) == 4 ? 3 : 4))
    k_fused_tma(const __grid_constant__ DevPool P, const int* __restrict__ list, const int* __restrict__ pn, const S* __restrict__ fin,
                S* __restrict__ fout, const S* __restrict__ ffine, int level, int allow_force) {
    pdl_enter();
    constexpr int BB = B * B, TPS = BB / 4, SPC = 256 / TPS, TPR = B / 4;
    using L = TmaSlot<B>;
    extern __shared__ __align__(128) unsigned char smraw[];
    S* sm = reinterpret_cast<S*>(smraw);
    __shared__ int nb[SPC][9];
    __shared__ int fast[SPC];
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x, ls = tid / TPS, t = tid % TPS;
    const int item = blockIdx.x * SPC + ls;
    const int n = *pn;
    if (t < 9) nb[ls][t] = item < n ? P.nbr[list[item] * 9 + t] : -1;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    // the staged path: an interior block off the domain sides, without a
    // neighbour in the finer region, with all 8 neighbours present
    if (t == 0) {
        int ok = 0;
        if (item < n) {
            const int s0 = nb[ls][4];
            ok = P.slot_type[s0] == ST_INT && !(P.slot_flags[s0] & (SLOTF_EDGE | SLOTF_MAILBOX | SLOTF_SOLID));
            for (int k = 0; k < 9; k++) ok = ok && nb[ls][k] >= 0;
        }
        fast[ls] = ok;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t bytes = 0;
        for (int j = 0; j < SPC; j++)
            if (fast[j]) bytes += (uint32_t)((9 * BB + 6 * B) * sizeof(S));
        mbar_expect_tx(&bar, bytes);
        for (int j = 0; j < SPC; j++) {
            if (!fast[j]) continue;
            S* base = sm + j * L::elems;
            const size_t s0 = (size_t)nb[j][4];
#pragma unroll 1
            for (int q = 0; q < 9; q++)
                bulk_g2s(base + L::planes + q * BB, fin + (s0 * 9 + q) * BB, (uint32_t)(BB * sizeof(S)), &bar);
            const size_t sb = (size_t)nb[j][1], stp = (size_t)nb[j][7];  // bottom and top neighbours
#pragma unroll 1
            for (int k = 0; k < 3; k++) {
                const int qu = k == 0 ? 2 : (k == 1 ? 5 : 6);  // c_y = +1: last row of the bottom block
                const int qd = k == 0 ? 4 : (k == 1 ? 7 : 8);  // c_y = -1: first row of the top block
                bulk_g2s(base + L::rows + qu * B, fin + (sb * 9 + qu) * BB + (B - 1) * B, (uint32_t)(B * sizeof(S)),
                         &bar);
                bulk_g2s(base + L::rows + qd * B, fin + (stp * 9 + qd) * BB, (uint32_t)(B * sizeof(S)), &bar);
            }
        }
    }
    if (fast[ls]) {
        S* base = sm + ls * L::elems;
        for (int e = t; e < 6 * B + 4; e += TPS) {
            if (e < 6 * B) {
                // c_x = +1 (q 1, 5, 8): last column of the left block; c_x = -1 (q 3, 6, 7): first of the right
                const int k = e / B, r = e % B;
                const int q = k == 0 ? 1 : (k == 1 ? 5 : (k == 2 ? 8 : (k == 3 ? 3 : (k == 4 ? 6 : 7))));
                const size_t ns = (size_t)(k < 3 ? nb[ls][3] : nb[ls][5]);
                base[L::cols + q * B + r] = fin[(ns * 9 + q) * BB + r * B + (k < 3 ? B - 1 : 0)];
            } else {
                // the diagonal populations' corner sources
                const int q = 5 + (e - 6 * B);
                const int k = q == 5 ? 0 : (q == 6 ? 2 : (q == 7 ? 8 : 6));
                const int cx = (q == 5 || q == 8) ? B - 1 : 0, cy = (q == 5 || q == 6) ? B - 1 : 0;
                base[L::corner + q] = fin[((size_t)nb[ls][k] * 9 + q) * BB + cy * B + cx];
            }
        }
    }
    // the bulk copies (bounded wait: a copy that never lands is reported, not waited for forever)
    bool landed = false;
    for (int it = 0; it < TMA_SPIN_LIMIT && !landed; it++) landed = mbar_try_wait(&bar, 0);
    if (!landed) {
        if (tid == 0) atomicOr(P.err, ERRB_TIMEOUT);
        for (int it = 0; it < TMA_SPIN_LIMIT && !landed; it++) landed = mbar_try_wait(&bar, 0);
    }
    __syncthreads();
    if (item >= n || !landed) return;
    const int slot = nb[ls][4];
    const int type = P.slot_type[slot];
    const InstParams& ip = P.inst[P.slot_inst[slot]];
    const int y = t / TPR, x0 = (t % TPR) * 4;
    if (!fast[ls]) {
        for (int i = 0; i < 4; i++)
            fused_cell<S, C, COLL, false>(P, fin, fout, ffine, slot, type, ip, level, x0 + i, y, allow_force != 0);
        return;
    }
    const S* base = sm + ls * L::elems;
    C f[9][4];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const int cx = CXq(q), cy = CYq(q);
        const int sy = y - cy;
        const bool inside = sy >= 0 && sy < B;
        C v[4];
        Vec4s<S, C>::ld(inside ? base + L::planes + q * BB + sy * B + x0 : base + L::rows + q * B + x0, v);
        if (cx == 0) {
#pragma unroll
            for (int i = 0; i < 4; i++) f[q][i] = v[i];
        } else if (cx == 1) {
            C left = __shfl_up_sync(0xffffffffu, v[3], 1, TPR);
            if (x0 == 0) left = Sto<S>::template ldr<C>(base, inside ? L::cols + q * B + sy : L::corner + q);
            f[q][0] = left, f[q][1] = v[0], f[q][2] = v[1], f[q][3] = v[2];
        } else {
            C right = __shfl_down_sync(0xffffffffu, v[0], 1, TPR);
            if (x0 + 4 == B) right = Sto<S>::template ldr<C>(base, inside ? L::cols + q * B + sy : L::corner + q);
            f[q][0] = v[1], f[q][1] = v[2], f[q][2] = v[3], f[q][3] = right;
        }
    }
    const C om = (C)1 / (C)ip.tau[level];
    const int gx0 = P.slot_ox[slot] + x0, gy = P.slot_oy[slot] + y;
    bool force = false;
    if (allow_force && ip.has_body && level == ip.m - 1) {  // block meets the IBM force patch?
        const InstState& st = P.ist[P.slot_inst[slot]];
        int bx = P.slot_ox[slot], by = P.slot_oy[slot];
        force = bx < st.patch_x0 + st.patch_w && st.patch_x0 < bx + B && by < st.patch_y0 + st.patch_h &&
                st.patch_y0 < by + B;
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        C g[9];
#pragma unroll
        for (int q = 0; q < 9; q++) g[q] = f[q][i] + dshift<S, C>(ip.dref, q);  // compute form
        C Fx = 0, Fy = 0;
        if (force) {
            patch_force<C>(P, ip, gx0 + i, gy, Fx, Fy);
            collide_k<COLL, C, true, DevTrait<S>::value, sizeof(S) == 4>(g, om, Fx, Fy, ip);
        } else {
            collide_k<COLL, C, false, DevTrait<S>::value, sizeof(S) == 4>(g, om, (C)0, (C)0, ip);
        }
#pragma unroll
        for (int q = 0; q < 9; q++) f[q][i] = g[q] - dshift<S, C>(ip.dref, q);  // storage form
    }
#pragma unroll
    for (int q = 0; q < 9; q++) Vec4<S, C>::st(fout + ((size_t)slot * 9 + q) * BB + y * B + x0, q, f[q]);
}

__global__ void __launch_bounds__(128) k_pose(const __grid_constant__ DevPool P, const int* __restrict__ ilist, const int* __restrict__ pn) {
    pdl_enter();
    const int item = blockIdx.x;
    if (item >= *pn) return;
    pose_run(P, ilist[item]);
}

template <class C>
__global__ void __launch_bounds__(IBM_THREADS) k_ibm_geom(const __grid_constant__ DevPool P, const int* __restrict__ ilist,
                                                          const int* __restrict__ pn) {
    pdl_enter();
    const int item = blockIdx.x;
    if (item >= *pn) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ IbmShared sh;
    ibm_geom_run<C>(P, ilist[item], blockIdx.y, smraw, sh);
}

template <class S, class C>
__global__ void __launch_bounds__(IBM_THREADS) k_ibm(const __grid_constant__ DevPool P, const int* __restrict__ ilist,
                                                     const int* __restrict__ pn, const S* __restrict__ fin,
                                                     int level, int direct, int deferred) {
    pdl_enter();
    const int item = blockIdx.x;
    if (item >= *pn) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ IbmShared sh;
    ibm_run<S, C>(P, ilist[item], fin, level, direct, deferred, smraw, sh, [] { return true; });
}

template <class C>
__global__ void __launch_bounds__(IBM_THREADS) k_force_sum(const __grid_constant__ DevPool P, const int* __restrict__ ilist,
                                                           const int* __restrict__ pn) {
    pdl_enter();
    const int item = blockIdx.x;
    if (item >= *pn) return;
    __shared__ double red[3][32];
    force_sum_run<C>(P, ilist[item], blockIdx.y, red);
}

// ---------------------------------------------------------------------------
// canonical (pre-collision) state out, initial state in, checksums
// ---------------------------------------------------------------------------
// mode 0: populations [9][ny][nx]; mode 1: rho, sum c f / rho as [3][ny][nx]
template <class S, class C>
__global__ void __launch_bounds__(1024) k_export(const __grid_constant__ DevPool P, const int* __restrict__ list, int n,
                                                 const S* __restrict__ f, const S* __restrict__ ffine, int level,
                                                 int direct, int nx, double* __restrict__ dense, long long plane,
                                                 int mode) {
    int item = blockIdx.x;
    if (item >= n) return;
    const int B = P.B;
    int slot = list[item];
    int cell = threadIdx.x;
    int x = cell % B, y = cell / B;
    const InstParams& ip = P.inst[P.slot_inst[slot]];
    int gx = P.slot_ox[slot] + x, gy = P.slot_oy[slot] + y;
    bool inl = (P.slot_flags[slot] & SLOTF_EDGE) && inlet_cell<C>(ip, level, gx, gy);
    // moments in FP64 from the storage form (deviations keep their precision)
    double r = 0.0, jx = 0.0, jy = 0.0;
    C vs[9];
#pragma unroll
    for (int q = 0; q < 9; q++)
        vs[q] = direct ? Sto<S>::template ld<C>(f, ((size_t)slot * 9 + q) * B * B + cell, q, ip.dref)
                       : pull_int<S, C>(P, f, ffine, (P.slot_flags[slot] & SLOTF_MAILBOX) != 0, slot, ip, level, x, y, q);
    if (!direct && (P.slot_flags[slot] & SLOTF_SOLID)) solid_links<S, C>(P, f, slot, ip, level, x, y, vs);
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const C v = vs[q];
        double dv = (double)v;
        if (inl && !direct) dv = (double)feq<C>(q, (C)ip.rho0, (C)ip.uin_x, (C)ip.uin_y) - wdev<S>(q);
        if (mode == 0) {
            dense[q * plane + (long long)gy * nx + gx] = dv + wdev<S>(q);
        } else {
            r += dv;
            jx += CXq(q) * dv;
            jy += CYq(q) * dv;
        }
    }
    if (mode == 1) {
        if (DevTrait<S>::value) r += 1.0;
        long long g = (long long)gy * nx + gx;
        dense[g] = r;
        dense[plane + g] = jx / r;
        dense[2 * plane + g] = jy / r;
    }
}

template <class S, class C>
__global__ void __launch_bounds__(1024) k_set_pre(const __grid_constant__ DevPool P, const int* __restrict__ list, int n, S* __restrict__ f,
                                                  int nx, const double* __restrict__ dense, long long plane,
                                                  int from_fields) {
    int item = blockIdx.x;
    if (item >= n) return;
    const int B = P.B;
    int slot = list[item];
    int cell = threadIdx.x;
    long long g = (long long)(P.slot_oy[slot] + cell / B) * nx + (P.slot_ox[slot] + cell % B);
    if (dense == nullptr) {  // the domain's uniform initial state (rho0, u_in)
        const InstParams& ip = P.inst[P.slot_inst[slot]];
#pragma unroll
        for (int q = 0; q < 9; q++)
            Sto<S>::template st<C>(f, ((size_t)slot * 9 + q) * B * B + cell, q,
                                   feq_s<S, C>(q, (C)ip.rho0, (C)ip.uin_x, (C)ip.uin_y), ip.dref);
    } else if (from_fields) {
        const InstParams& ip = P.inst[P.slot_inst[slot]];
        C r = (C)dense[g], u = (C)dense[plane + g], v = (C)dense[2 * plane + g];
#pragma unroll
        for (int q = 0; q < 9; q++)
            Sto<S>::template st<C>(f, ((size_t)slot * 9 + q) * B * B + cell, q, feq_s<S, C>(q, r, u, v), ip.dref);
    } else {
        const InstParams& ip = P.inst[P.slot_inst[slot]];
#pragma unroll
        for (int q = 0; q < 9; q++)
            Sto<S>::template st<C>(f, ((size_t)slot * 9 + q) * B * B + cell, q,
                                   (C)(dense[q * plane + g] - wdev<S>(q)), ip.dref);
    }
}

// per-thread-block partial sums of mass and momentum (FP64), written in
// block order; a single block then adds the partials in index order, so the
// result does not depend on scheduling
template <class S, class C>
__global__ void __launch_bounds__(256) k_checksum_partials(const __grid_constant__ DevPool P, const int* __restrict__ list, int n,
                                                           const S* __restrict__ f, const S* __restrict__ ffine,
                                                           int level, int direct, double weight,
                                                           double* __restrict__ partials) {
    __shared__ double red[32];
    const int B = P.B, BB = B * B;
    double m = 0.0, px = 0.0, py = 0.0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)n * BB;
         idx += (long long)gridDim.x * blockDim.x) {
        int slot = list[idx / BB];
        int cell = (int)(idx % BB);
        int x = cell % B, y = cell / B;
        const InstParams& ip = P.inst[P.slot_inst[slot]];
        int gx = P.slot_ox[slot] + x, gy = P.slot_oy[slot] + y;
        bool inl = !direct && (P.slot_flags[slot] & SLOTF_EDGE) && inlet_cell<C>(ip, level, gx, gy);
        const bool near_solid = (P.slot_flags[slot] & SLOTF_SOLID) != 0;
        if (near_solid && in_solid(ip, gx + 0.5, gy + 0.5)) continue;  // solid cells hold no fluid
        C vs[9];
        for (int q = 0; q < 9; q++)
            vs[q] = direct ? Sto<S>::template ld<C>(f, ((size_t)slot * 9 + q) * BB + cell, q, ip.dref)
                           : pull_int<S, C>(P, f, ffine, (P.slot_flags[slot] & SLOTF_MAILBOX) != 0, slot, ip, level,
                                            x, y, q);
        if (!direct && near_solid) solid_links<S, C>(P, f, slot, ip, level, x, y, vs);
        for (int q = 0; q < 9; q++) {
            const C v = vs[q];
            double full = (double)v + wdev<S>(q);  // full population, added in FP64
            if (inl) full = (double)feq<C>(q, (C)ip.rho0, (C)ip.uin_x, (C)ip.uin_y);
            double dv = weight * full;
            m += dv;
            px += CXq(q) * dv;
            py += CYq(q) * dv;
        }
    }
    m = block_sum<C>(m, red);
    px = block_sum<C>(px, red);
    py = block_sum<C>(py, red);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = m;
        partials[3 * blockIdx.x + 1] = px;
        partials[3 * blockIdx.x + 2] = py;
    }
}

__global__ void k_reduce_partials(const double* __restrict__ partials, int n, double* __restrict__ out3,
                                  int* __restrict__ err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = 0.0, px = 0.0, py = 0.0;
    for (int i = 0; i < n; i++) {
        m += partials[3 * i];
        px += partials[3 * i + 1];
        py += partials[3 * i + 2];
    }
    out3[0] = m;
    out3[1] = px;
    out3[2] = py;
    if (!isfinite(m) || !isfinite(px) || !isfinite(py)) atomicOr(err, ERRB_NONFINITE);
}

// re-tag transfer (post-collision state, reading R5).  job = (dst, kind, s0,
// s1, s2, s3, source buffer, destination buffer): kind 0 copies, into every cell of the new block, the covering
// cell of the coarser old block s0 that lies s1 levels up; kind 1 sets every
// cell to the mean of its 4 children in the old finer blocks s0..s3 (the
// quadrants (0,0), (1,0), (0,1), (1,1) of the new block).
template <class S, class C>
__global__ void __launch_bounds__(1024) k_retag(const __grid_constant__ DevPool P, const int* __restrict__ jobs, int n, S* f0, S* f1) {
    int item = blockIdx.x;
    if (item >= n) return;
    const int B = P.B, BB = B * B;
    const int* jb = jobs + RETAG_JOB_INTS * item;
    int dst = jb[0], kind = jb[1];
    const S* fsrc = jb[6] ? f1 : f0;
    S* fdst = jb[7] ? f1 : f0;
    int cell = threadIdx.x;
    int x = cell % B, y = cell / B;
    // the destination's origin comes with the job (its table entry may not be
    // written yet); the sources are old interior blocks with valid entries
    int gx = jb[8] + x, gy = jb[9] + y;
    if (kind == 0) {
        int src = jb[2], up = jb[3];
        int sx = (gx >> up) - P.slot_ox[src], sy = (gy >> up) - P.slot_oy[src];
#pragma unroll
        for (int q = 0; q < 9; q++) fdst[((size_t)dst * 9 + q) * BB + cell] = fsrc[((size_t)src * 9 + q) * BB + sy * B + sx];
    } else {
        int quad = (y >= B / 2 ? 2 : 0) + (x >= B / 2 ? 1 : 0);
        int src = jb[2 + quad];
        int lx = 2 * gx - P.slot_ox[src], ly = 2 * gy - P.slot_oy[src];
#pragma unroll
        for (int q = 0; q < 9; q++) {
            size_t base = ((size_t)src * 9 + q) * BB;
            C v = Sto<S>::template ldr<C>(fsrc, base + ly * B + lx);  // a mean of stored values
            v += Sto<S>::template ldr<C>(fsrc, base + ly * B + lx + 1);
            v += Sto<S>::template ldr<C>(fsrc, base + (ly + 1) * B + lx);
            v += Sto<S>::template ldr<C>(fsrc, base + (ly + 1) * B + lx + 1);
            Sto<S>::template str<C>(fdst, ((size_t)dst * 9 + q) * BB + cell, (C)0.25 * v);
        }
    }
}

// host table updates: each record names one int of a device table and its new value
__global__ void __launch_bounds__(256) k_scatter(const ScatterRec* __restrict__ recs, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ScatterRec r = recs[i];
        *r.dst = r.value;
    }
}

template <class F>
void dispatch(int storage, F&& fn) {
    switch (storage) {
    case 0: fn((double*)nullptr, (double*)nullptr); break;
    case 1: fn((float*)nullptr, (float*)nullptr); break;
    case 2: fn((__half*)nullptr, (float*)nullptr); break;
    default: fn((__nv_bfloat16*)nullptr, (float*)nullptr); break;
    }
}

}  // namespace

int storage_bytes(int storage) { return storage == 0 ? 8 : (storage == 1 ? 4 : 2); }

template <class S, class C, int B, int COLL>
void launch_tma(const DevPool& P, const int* list, const int* pn, int cap, const void* fin, void* fout,
                const void* ffine, int level, sbot_stream_t s, int allow_force) {
    constexpr int SPC = 256 / (B * B / 4);
    const size_t smem = (size_t)SPC * TmaSlot<B>::elems * sizeof(S);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_fused_tma<S, C, B, COLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
    }
    launch_k(P.pdl, k_fused_tma<S, C, B, COLL>, dim3((cap + SPC - 1) / SPC), dim3(256), smem, s, P, list, pn,
             (const S*)fin, (S*)fout, (const S*)ffine, level, allow_force);
}

template <class S, class C, int COLL>
void launch_fused_k(const DevPool& P, const int* list, const int* pn, int n, int n_hint, long long vec_min_cells,
                    int staged, const void* fin, void* fout, const void* ffine, int level, sbot_stream_t s,
                    int allow_force, void* fhalo) {
    if (P.coll & COLL_SOLID) {  // a context holding a solid runs the scalar kernel with the solid links
        launch_k(P.pdl, k_fused<S, C, COLL, true>, dim3(n), dim3(P.B * P.B), 0, s, P, list, pn, (const S*)fin,
                 (S*)fout, (const S*)ffine, level, allow_force, (S*)fhalo);
        return;
    }
    // the vector kernel needs enough blocks to fill the GPU: small launches
    // are latency-bound and run faster with one thread per cell (and so does
    // a launch that also fills the finer level's halo)
    const bool big = fhalo == nullptr && vec_min_cells >= 0 && (long long)n_hint * P.B * P.B >= vec_min_cells;
    if (big && staged && P.B == 16)
        launch_tma<S, C, 16, COLL>(P, list, pn, n, fin, fout, ffine, level, s, allow_force);
    else if (big && staged && P.B == 32)
        launch_tma<S, C, 32, COLL>(P, list, pn, n, fin, fout, ffine, level, s, allow_force);
    else if (big && (P.B == 16 || P.B == 32)) {
        if constexpr (sizeof(S) == 2) {  // 16-bit storage: 8 cells per thread
            const bool sh = (P.coll & COLL_SHIFT) != 0;
            if (P.B == 16)
                launch_k(P.pdl, sh ? k_fused_v8<S, C, 16, COLL, true> : k_fused_v8<S, C, 16, COLL, false>,
                         dim3(vec_grid((n + 7) / 8, P.vec_waves)), dim3(256), 0, s, P, list, pn, (const S*)fin, (S*)fout, (const S*)ffine,
                         level, allow_force);
            else
                launch_k(P.pdl, sh ? k_fused_v8<S, C, 32, COLL, true> : k_fused_v8<S, C, 32, COLL, false>,
                         dim3(vec_grid((n + 1) / 2, P.vec_waves)), dim3(256), 0, s, P, list, pn, (const S*)fin, (S*)fout, (const S*)ffine,
                         level, allow_force);
        } else {  // FP32 and FP64: 4 cells per thread
            if (P.B == 16)
                launch_k(P.pdl, k_fused_v4<S, C, 16, COLL>, dim3(vec_grid((n + 3) / 4, P.vec_waves)), dim3(256), 0, s, P, list, pn,
                         (const S*)fin, (S*)fout, (const S*)ffine, level, allow_force);
            else
                launch_k(P.pdl, k_fused_v4<S, C, 32, COLL>, dim3(vec_grid(n, P.vec_waves)), dim3(256), 0, s, P, list, pn, (const S*)fin,
                         (S*)fout, (const S*)ffine, level, allow_force);
        }
    }
    else
        launch_k(P.pdl, k_fused<S, C, COLL, false>, dim3(n), dim3(P.B * P.B), 0, s, P, list, pn, (const S*)fin,
                 (S*)fout, (const S*)ffine, level, allow_force, (S*)fhalo);
}

void launch_fused(int storage, const DevPool& P, const int* list, const int* pn, int cap, int n_hint,
                  long long vec_min_cells, int staged, const void* fin, void* fout, const void* ffine, int level,
                  sbot_stream_t s, int allow_force, void* fhalo) {
    if (cap <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        if ((P.coll & 15) == 1)
            launch_fused_k<S, C, 1>(P, list, pn, cap, n_hint, vec_min_cells, staged, fin, fout, ffine, level, s,
                                    allow_force, fhalo);
        else if ((P.coll & 15) == 2)
            launch_fused_k<S, C, 2>(P, list, pn, cap, n_hint, vec_min_cells, staged, fin, fout, ffine, level, s,
                                    allow_force, fhalo);
        else
            launch_fused_k<S, C, 0>(P, list, pn, cap, n_hint, vec_min_cells, staged, fin, fout, ffine, level, s,
                                    allow_force, fhalo);
    });
}

void launch_collide_init(int storage, const DevPool& P, const int* list, int n, const void* fpre, void* fpost,
                         int level, sbot_stream_t s) {
    if (n <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        if ((P.coll & 15) == 1)
            k_collide_init<S, C, 1><<<n, P.B * P.B, 0, s>>>(P, list, n, (const S*)fpre, (S*)fpost, level);
        else if ((P.coll & 15) == 2)
            k_collide_init<S, C, 2><<<n, P.B * P.B, 0, s>>>(P, list, n, (const S*)fpre, (S*)fpost, level);
        else
            k_collide_init<S, C, 0><<<n, P.B * P.B, 0, s>>>(P, list, n, (const S*)fpre, (S*)fpost, level);
    });
}

void launch_c2f(int storage, const DevPool& P, const int* list, const int* pn, int cap, const void* fcoarse,
                void* ffine, sbot_stream_t s) {
    if (cap <= 0) return;
    dispatch(storage, [&](auto* sp, auto*) {
        using S = std::remove_pointer_t<decltype(sp)>;
        launch_k(P.pdl, k_c2f<S>, dim3(cap), dim3(P.B * P.B), 0, s, P, list, pn, (const S*)fcoarse, (S*)ffine);
    });
}

static size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

size_t ibm_cache_bytes(int storage, int patch_cap, int n_markers) {
    // the first regions of k_ibm's shared memory (up to the list weights) and the header
    const size_t c = storage == 0 ? 8 : 4, n = (size_t)n_markers, cap = (size_t)patch_cap;
    const size_t ncap = cap < 8 * n + 64 ? cap : 8 * n + 64;
    const size_t ent = storage == 0 ? 16 : 8;  // sizeof(IbmEnt<C>)
    return al16(IBM_MAXB * IBM_MAXB * 9 * 4) + 2 * al16(n * 4) + al16(8 * n * c) + al16(4 * n * c) +
           al16(16 * n * 2) + al16(ncap * 4) + al16((ncap + 1) * 4) + al16(16 * n * ent) + sizeof(IbmCacheHead);
}

size_t ibm_smem_bytes(int storage, int patch_cap, int n_markers) {
    // the carve order of k_ibm, each region rounded up to 16 bytes
    const size_t c = storage == 0 ? 8 : 4, n = (size_t)n_markers, cap = (size_t)patch_cap;
    const size_t ncap = cap < 8 * n + 64 ? cap : 8 * n + 64, W = (cap + 31) / 32 + 1;
    return ibm_cache_bytes(storage, patch_cap, n_markers) - sizeof(IbmCacheHead) + al16(n * c) + 2 * al16(2 * n * c) +
           al16(W * 4) + al16((W + 1) * 4) + al16(ncap * 4) + al16(4 * ncap * c) + 2 * al16(ncap * c);
}

size_t ibm_smem_limit(int storage) {
    // the device's opt-in shared memory per block less k_ibm's static shared memory
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || optin <= 0)
        return 220 * 1024;
    size_t stat = 0;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        cudaFuncAttributes fa{};
        stat = cudaFuncGetAttributes(&fa, k_ibm<S, C>) == cudaSuccess ? fa.sharedSizeBytes : 4096;
    });
    return (size_t)optin > stat ? (size_t)optin - stat : 0;
}

void launch_pose(const DevPool& P, const int* inst_list, const int* pn, int cap, sbot_stream_t s) {
    if (cap <= 0) return;
    launch_k(P.pdl, k_pose, dim3(cap), dim3(128), 0, s, P, inst_list, pn);
}

void launch_ibm_geom(int storage, const DevPool& P, const int* inst_list, const int* pn, int cap, int steps,
                     size_t smem, sbot_stream_t s) {
    if (cap <= 0 || steps <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using C = std::remove_pointer_t<decltype(cp)>;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_ibm_geom<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ibm_smem_limit(storage));
            attr_set = true;
        }
        launch_k(P.pdl, k_ibm_geom<C>, dim3(cap, steps), dim3(IBM_THREADS), smem, s, P, inst_list, pn);
    });
}

void launch_force_sum(int storage, const DevPool& P, const int* inst_list, const int* pn, int cap, int steps,
                      sbot_stream_t s) {
    if (cap <= 0 || steps <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using C = std::remove_pointer_t<decltype(cp)>;
        launch_k(P.pdl, k_force_sum<C>, dim3(cap, steps), dim3(IBM_THREADS), 0, s, P, inst_list, pn);
    });
}

void launch_ibm(int storage, const DevPool& P, const int* inst_list, const int* pn, int cap, const void* f,
                int level, int direct, size_t smem, sbot_stream_t s, int deferred, int threads) {
    if (cap <= 0) return;
    const int n = cap;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_ibm<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)ibm_smem_limit(storage));
            attr_set = true;
        }
        launch_k(P.pdl, k_ibm<S, C>, dim3(n), dim3(threads > 0 && threads <= IBM_THREADS ? threads : IBM_THREADS),
                 smem, s, P, inst_list, pn, (const S*)f, level, direct, deferred);
    });
}

void launch_export(int storage, const DevPool& P, const int* list, int n, const void* f, const void* ffine, int level,
                   int direct, int nx, double* dense, long long plane, int mode, sbot_stream_t s) {
    if (n <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        k_export<S, C><<<n, P.B * P.B, 0, s>>>(P, list, n, (const S*)f, (const S*)ffine, level, direct, nx, dense,
                                               plane, mode);
    });
}

void launch_set_pre(int storage, const DevPool& P, const int* list, int n, void* f, int nx, const double* dense,
                    long long plane, int from_fields, sbot_stream_t s) {
    if (n <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        k_set_pre<S, C><<<n, P.B * P.B, 0, s>>>(P, list, n, (S*)f, nx, dense, plane, from_fields);
    });
}

int checksum_blocks(int n_slots, int B) {
    long long cells = (long long)n_slots * B * B;
    long long b = (cells + 255) / 256;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

void launch_checksum_partials(int storage, const DevPool& P, const int* list, int n, const void* f, const void* ffine,
                              int level, int direct, double weight, double* partials, int nblocks, sbot_stream_t s) {
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        k_checksum_partials<S, C><<<nblocks, 256, 0, s>>>(P, list, n, (const S*)f, (const S*)ffine, level, direct,
                                                          weight, partials);
    });
}

void launch_reduce_partials(const double* partials, int n, double* out3, int* err, sbot_stream_t s) {
    k_reduce_partials<<<1, 32, 0, s>>>(partials, n, out3, err);
}

// Scratch of the allocation-free checksum (sbot_get_checksum_noalloc): the
// partial sums of up to SBOT_NOALLOC_MAX_PARTIALS thread blocks (3 doubles
// each) followed by the 3 results.  Every GPU that loads this library holds
// it (98,328 bytes) until the process exits.  In host code the name is only a
// host-side stand-in: kernels get the device address looked up below.
static __device__ __align__(256) double g_noalloc_scratch[3 * SBOT_NOALLOC_MAX_PARTIALS + 3];

// Device address of the scratch array in the current device's context,
// looked up on every call (a cached address would go stale if the context
// were destroyed and created again, e.g. after cudaDeviceReset).  The first
// lookup on a device may load this library's module there.  Returns nullptr
// when the lookup fails.
double* noalloc_scratch() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (double*)p;
}

void launch_retag(int storage, const DevPool& P, const int* jobs, int n, void* f0, void* f1, sbot_stream_t s) {
    if (n <= 0) return;
    dispatch(storage, [&](auto* sp, auto* cp) {
        using S = std::remove_pointer_t<decltype(sp)>;
        using C = std::remove_pointer_t<decltype(cp)>;
        k_retag<S, C><<<n, P.B * P.B, 0, s>>>(P, jobs, n, (S*)f0, (S*)f1);
    });
}

void launch_scatter(const ScatterRec* recs, int n, sbot_stream_t s) {
    if (n <= 0) return;
    int blocks = (n + 255) / 256;
    k_scatter<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(recs, n);
}


// the persistent step kernel of each storage kind (step_<kind>.cu)
int launch_step_f64(const DevPool&, const StepArgs&, int, int, size_t, sbot_stream_t);
int launch_step_f32(const DevPool&, const StepArgs&, int, int, size_t, sbot_stream_t);
int launch_step_f16(const DevPool&, const StepArgs&, int, int, size_t, sbot_stream_t);
int launch_step_bf16(const DevPool&, const StepArgs&, int, int, size_t, sbot_stream_t);
int step_occupancy_f64(int, int, int, size_t, size_t*);
int step_occupancy_f32(int, int, int, size_t, size_t*);
int step_occupancy_f16(int, int, int, size_t, size_t*);
int step_occupancy_bf16(int, int, int, size_t, size_t*);

int launch_step(int storage, const DevPool& P, const StepArgs& A, int grid, int threads, size_t smem,
                sbot_stream_t s) {
    switch (storage) {
    case 0: return launch_step_f64(P, A, grid, threads, smem, s);
    case 1: return launch_step_f32(P, A, grid, threads, smem, s);
    case 2: return launch_step_f16(P, A, grid, threads, smem, s);
    default: return launch_step_bf16(P, A, grid, threads, smem, s);
    }
}

int step_occupancy(int storage, int B, int coll, int threads, size_t smem, size_t* static_smem) {
    switch (storage) {
    case 0: return step_occupancy_f64(B, coll, threads, smem, static_smem);
    case 1: return step_occupancy_f32(B, coll, threads, smem, static_smem);
    case 2: return step_occupancy_f16(B, coll, threads, smem, static_smem);
    default: return step_occupancy_bf16(B, coll, threads, smem, static_smem);
    }
}
