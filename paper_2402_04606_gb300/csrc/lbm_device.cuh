// Device code of the lattice-Boltzmann / immersed-boundary / block-refinement
// time step of arXiv 2402.04606, shared by the per-phase kernels
// (kernels.cu) and the persistent step kernel (step_impl.cuh): the lattice
// and its storage forms, the collisions, the pulls with their boundary and
// interface rules, the fused per-cell and per-block updates, the
// coarse-to-fine copy, and the immersed boundary's pose, geometry,
// multi-direct forcing and force sums.  Everything is in an unnamed
// namespace: each translation unit that includes it has its own copy.
//
// Pointer parameters carry no __restrict__ here: the persistent kernel reads,
// within one launch, buffers that other thread blocks wrote earlier in it.
// The per-phase kernels mark their own parameters.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <climits>
#include <type_traits>

#include "kinematics.h"
#include "sbot_internal.h"

#define STEP_MAX_THREADS 768  // largest thread block of the persistent step kernel

namespace {


// Programmatic dependent launch: wait until the kernel this one depends on
// (the previous one on the stream, when launched with the attribute) has
// finished and its writes are visible, then let the next kernel be scheduled.
// Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch with the programmatic-stream-serialization attribute when `pdl`
template <typename... KArgs, typename... Args>
void launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// ---------------------------------------------------------------------------
// lattice (Eq. 1) and weights (text after Eq. 7)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ constexpr int CXq(int q) {
    return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int CYq(int q) {
    return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
}
template <class C>
__device__ __forceinline__ constexpr C Wq(int q) {
    return q == 0 ? C(4.0 / 9.0) : (q < 5 ? C(1.0 / 9.0) : C(1.0 / 36.0));
}
// w_q x with the weight as a two-term constant in FP32 (w_q = hi + lo, hi the
// nearest float, lo the float nearest the remainder): fma(x, hi, x lo) is
// w_q x to about one rounding.  The nearest floats to 4/9, 1/9 and 1/36 all
// exceed them by 2^-27 of themselves, so with plain products the odd part of
// a deviation equilibrium carries the momentum of the moments times
// (1 + 2^-27); the collision adds that excess at every cell and step with the
// same sign, and the velocity drifts linearly with the number of steps (a
// third of the 3e-4 error of a Taylor-Green vortex at tau = 0.52 after 10,000
// steps; the biased reciprocal in moments9 is the rest); the even part's
// excess shows as a slow drift of the mass.  FP64 takes the plain product.
__host__ __device__ __forceinline__ constexpr float WloF(int q) {
    return q == 0 ? (float)(4.0 / 9.0 - (double)(float)(4.0 / 9.0))
                  : (q < 5 ? (float)(1.0 / 9.0 - (double)(float)(1.0 / 9.0))
                           : (float)(1.0 / 36.0 - (double)(float)(1.0 / 36.0)));
}
template <class C>
__device__ __forceinline__ C wmul(int q, C x) {
    if constexpr (sizeof(C) == 4)
        return __fmaf_rn(x, Wq<float>(q), x * WloF(q));
    else
        return Wq<C>(q) * x;
}
// x / 6 likewise (the MRT basis's momentum rows): fl(1/6) exceeds 1/6 by
// 2.98e-8 of itself, which would add that fraction of the momentum per step
template <class C>
__device__ __forceinline__ C div6(C x) {
    if constexpr (sizeof(C) == 4)
        return __fmaf_rn(x, (float)(1.0 / 6.0), x * (float)(1.0 / 6.0 - (double)(float)(1.0 / 6.0)));
    else
        return x * ((C)1 / (C)6);
}

// a b + c rounded once
template <class C>
__device__ __forceinline__ C fmac(C a, C b, C c) {
    if constexpr (sizeof(C) == 4)
        return __fmaf_rn(a, b, c);
    else
        return fma(a, b, c);
}

// direction with c_x (c_y) reversed
__device__ __forceinline__ int flipX(int q) {
    const int t[9] = {0, 3, 2, 1, 4, 6, 5, 8, 7};
    return t[q];
}
__device__ __forceinline__ int flipY(int q) {
    const int t[9] = {0, 1, 4, 3, 2, 8, 7, 6, 5};
    return t[q];
}

// ---------------------------------------------------------------------------
// storage: FP64 holds f; the FP32 arithmetic of the other kinds works on the
// deviation f - w_q ("zero-centred" populations, the compute form), so
// rounding is relative to O(u) quantities instead of O(w).  FP32 stores that
// deviation; FP16 and BF16 store f - feq_q(rho0, u_in) of the instance, the
// compute form less a per-instance shift (Sto below).  Population values in
// registers are in the compute form, except where a copy or a mean moves
// stored values as they are.
// ---------------------------------------------------------------------------
template <class S>
struct DevTrait {
    static constexpr bool value = true;
};
template <>
struct DevTrait<double> {
    static constexpr bool value = false;
};
template <class S, class C>
__device__ __forceinline__ constexpr C shift(int q) {
    return DevTrait<S>::value ? Wq<C>(q) : (C)0;
}

// the shift of the deviation kinds in FP64, exactly w_q: the value added when
// populations leave the storage form (export, checksum) and subtracted when
// they enter it from FP64 (the deviation arithmetic is relative to w_q itself,
// not to its rounding in the compute type)
template <class S>
__device__ __forceinline__ double wdev(int q) {
    return DevTrait<S>::value ? Wq<double>(q) : 0.0;
}

// Storage access.  ld / st convert between the storage form and the compute
// form (f - w_q for the deviation kinds, f for FP64); ldr / str move the
// stored value as it is (copies and means of stored values).  16-bit storage
// holds f - feq_q(rho0, u_in) of the instance, the compute form less dr[q]
// (dr: the instance's nine shifts, InstParams::dref): a flow close to its
// free stream then stores small values, which the 8 or 11 mantissa bits keep
// to a small absolute error.  32- and 64-bit storage ignore dr.
template <class S>
struct Sto;
template <>
struct Sto<double> {
    template <class C>
    static __device__ __forceinline__ C ld(const double* p, size_t i, int, const float*) { return (C)p[i]; }
    template <class C>
    static __device__ __forceinline__ void st(double* p, size_t i, int, C v, const float*) { p[i] = (double)v; }
    template <class C>
    static __device__ __forceinline__ C ldr(const double* p, size_t i) { return (C)p[i]; }
    template <class C>
    static __device__ __forceinline__ void str(double* p, size_t i, C v) { p[i] = (double)v; }
};
template <>
struct Sto<float> {
    template <class C>
    static __device__ __forceinline__ C ld(const float* p, size_t i, int, const float*) { return (C)p[i]; }
    template <class C>
    static __device__ __forceinline__ void st(float* p, size_t i, int, C v, const float*) { p[i] = (float)v; }
    template <class C>
    static __device__ __forceinline__ C ldr(const float* p, size_t i) { return (C)p[i]; }
    template <class C>
    static __device__ __forceinline__ void str(float* p, size_t i, C v) { p[i] = (float)v; }
};
template <>
struct Sto<__half> {
    template <class C>
    static __device__ __forceinline__ C ldr(const __half* p, size_t i) { return (C)__half2float(p[i]); }
    template <class C>
    static __device__ __forceinline__ void str(__half* p, size_t i, C v) { p[i] = __float2half_rn((float)v); }
    template <class C>
    static __device__ __forceinline__ C ld(const __half* p, size_t i, int q, const float* dr) {
        return ldr<C>(p, i) + (C)dr[q];
    }
    template <class C>
    static __device__ __forceinline__ void st(__half* p, size_t i, int q, C v, const float* dr) {
        str<C>(p, i, v - (C)dr[q]);
    }
};
template <>
struct Sto<__nv_bfloat16> {
    template <class C>
    static __device__ __forceinline__ C ldr(const __nv_bfloat16* p, size_t i) { return (C)__bfloat162float(p[i]); }
    template <class C>
    static __device__ __forceinline__ void str(__nv_bfloat16* p, size_t i, C v) {
        p[i] = __float2bfloat16_rn((float)v);
    }
    template <class C>
    static __device__ __forceinline__ C ld(const __nv_bfloat16* p, size_t i, int q, const float* dr) {
        return ldr<C>(p, i) + (C)dr[q];
    }
    template <class C>
    static __device__ __forceinline__ void st(__nv_bfloat16* p, size_t i, int q, C v, const float* dr) {
        str<C>(p, i, v - (C)dr[q]);
    }
};
// the shift between the compute form and the storage form of direction q
template <class S, class C>
__device__ __forceinline__ C dshift(const float* dr, int q) {
    return sizeof(S) == 2 ? (C)dr[q] : (C)0;
}

// ---------------------------------------------------------------------------
// single-cell arithmetic (Sec. 2.1), constants of c_s^2 = 1/3 folded in
// ---------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ C feq(int q, C rho, C ux, C uy) {
    C cu = (C)CXq(q) * ux + (C)CYq(q) * uy;
    C uu = ux * ux + uy * uy;
    return Wq<C>(q) * rho * ((C)1 + (C)3 * cu + (C)4.5 * cu * cu - (C)1.5 * uu);
}

// Eq. 7 in storage form (minus w_q for the deviation kinds)
template <class S, class C>
__device__ __forceinline__ C feq_s(int q, C rho, C ux, C uy) {
    return feq<C>(q, rho, ux, uy) - shift<S, C>(q);
}

// Eq. 7, Eq. 3, Eq. 6 -- in place on f[9], given the moments: rho (drho =
// rho - 1 in deviation storage, else unused) and the half-force velocity u
// of Eq. 8.  Opposite directions q, q' (c_q' = -c_q) share the even part of
// f^eq and of the Guo term; only the odd part changes sign.  FORCE = false
// drops the Guo term (F = 0, e.g. every block outside the IBM patch).
template <class C, bool FORCE, bool DEV, bool SPLITW = true, bool NEQ = false>
__device__ __forceinline__ void bgk_update(C* f, C om, C Fx, C Fy, C rho, C drho, C ux, C uy) {
    // DEV: f holds f - w_q, and f^eq - w_q = w_q (drho + rho X); the odd part
    // (the equilibrium's momentum) takes its weight through wmul.
    // NEQ (32-bit storage): the even part takes its weight through wmul too
    // (with plain weights a periodic box gained 5e-7 of its mass in 10,000
    // steps, against 1e-8), and Eq. 6 is evaluated as f^eq + (1 - omega)
    // (f - f^eq): f - f^eq is small and nearly exact, so the one rounding is
    // of the result alone.  The form (1 - omega) f + omega f^eq rounds two
    // O(f) terms (a periodic box lost 7e-6 of its momentum in 10,000 steps,
    // against 4e-8).  16-bit storage rounds far more than either on its own,
    // and its kernels have no registers to spare for these forms.
    const C base = (DEV ? (C)0 : (C)1) - (C)1.5 * (ux * ux + uy * uy);
    const C om1 = (C)1 - om;
    const C gf = (C)1 - (C)0.5 * om;
    const C uF = FORCE ? ux * Fx + uy * Fy : (C)0;
    // rest population
    {
        C fe = NEQ ? wmul<C>(0, drho + rho * base) : Wq<C>(0) * (drho + rho * base);
        C Fi = FORCE ? Wq<C>(0) * gf * ((C)-3 * uF) : (C)0;
        f[0] = NEQ ? fmac<C>(om1, f[0] - fe, fe) + Fi : om1 * f[0] + om * fe + Fi;
    }
    // pairs (1,3), (2,4), (5,7), (6,8)
#pragma unroll
    for (int p = 0; p < 4; p++) {
        const int a = p < 2 ? 1 + p : 5 + (p - 2);
        const int b = p < 2 ? 3 + p : 7 + (p - 2);
        const C cu = (C)CXq(a) * ux + (C)CYq(a) * uy;
        const C ev = NEQ ? wmul<C>(a, drho + rho * (base + (C)4.5 * cu * cu))
                         : Wq<C>(a) * (drho + rho * (base + (C)4.5 * cu * cu));
        C od;
        if constexpr (DEV && SPLITW)
            od = wmul<C>(a, rho * (C)3 * cu);
        else
            od = Wq<C>(a) * rho * (C)3 * cu;
        C Fa = 0, Fb = 0;
        if (FORCE) {
            const C cF = (C)CXq(a) * Fx + (C)CYq(a) * Fy;
            const C gw = Wq<C>(a) * gf;
            const C e2 = gw * ((C)9 * cu * cF - (C)3 * uF);
            const C o2 = gw * (C)3 * cF;
            Fa = e2 + o2;
            Fb = e2 - o2;
        }
        if constexpr (NEQ) {
            const C ea = ev + od, eb = ev - od;
            f[a] = fmac<C>(om1, f[a] - ea, ea) + Fa;
            f[b] = fmac<C>(om1, f[b] - eb, eb) + Fb;
        } else {
            f[a] = om1 * f[a] + om * (ev + od) + Fa;
            f[b] = om1 * f[b] + om * (ev - od) + Fb;
        }
    }
}

// Eq. 8: density and half-force velocity of f[9] (storage form).
// DEV: u = a / rho is taken as a - a (drho / rho), a = j + F / 2.  The
// product a * fl(1 / rho) is biased: for rho = 1 + d the nearest float to
// 1 / rho is 1 - d rounded on the grid near 1, about d^2 below the exact
// reciprocal at most cells, which takes momentum out of every collision; the
// correction term carries its rounding at O(d) of the velocity and the one
// fma rounds the result once.
template <class C, bool FORCE, bool DEV>
__device__ __forceinline__ void moments9(const C* f, C Fx, C Fy, C& rho, C& drho, C& ux, C& uy) {
    if constexpr (DEV) {
        C srho = 0, ax = 0, ay = 0;
#pragma unroll
        for (int q = 0; q < 9; q++) {
            srho += f[q];
            ax += (C)CXq(q) * f[q];
            ay += (C)CYq(q) * f[q];
        }
        if (FORCE) {
            ax += (C)0.5 * Fx;
            ay += (C)0.5 * Fy;
        }
        rho = (C)1 + srho;
        drho = srho;
        const C t = srho * ((C)1 / rho);
        ux = fmac<C>(-ax, t, ax);
        uy = fmac<C>(-ay, t, ay);
    } else {
        C srho = 0, jx = 0, jy = 0;
#pragma unroll
        for (int q = 0; q < 9; q++) {
            srho += f[q];
            jx += (C)CXq(q) * f[q];
            jy += (C)CYq(q) * f[q];
        }
        rho = srho;
        drho = (C)0;
        const C irho = (C)1 / rho;
        ux = FORCE ? (jx + (C)0.5 * Fx) * irho : jx * irho;
        uy = FORCE ? (jy + (C)0.5 * Fy) * irho : jy * irho;
    }
}

// Eq. 8 (half-force velocity), Eq. 7, Eq. 3, Eq. 6 -- in place on f[9].
template <class C, bool FORCE, bool DEV, bool NEQ = false>
__device__ __forceinline__ void collide9f(C* f, C om, C Fx, C Fy) {
    C rho, drho, ux, uy;
    moments9<C, FORCE, DEV>(f, Fx, Fy, rho, drho, ux, uy);
    bgk_update<C, FORCE, DEV, true, NEQ>(f, om, Fx, Fy, rho, drho, ux, uy);
}

// The MRT option of Sec. 2.1, in place on f[9]: the D2Q9 moment basis
// (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy), whose rows are orthogonal
// with squared norms 9, 36, 36, 6, 12, 6, 12, 4, 4.  The equilibrium moments
// of Eq. 7 are rho (-2 + 3 u^2), rho (1 - 3 u^2), -rho u (heat fluxes),
// rho (ux^2 - uy^2), rho ux uy; the moments of the Guo term (Eq. 3 without
// its prefactor) are 6 u.F, -6 u.F, F, -F, 2 (ux Fx - uy Fy), ux Fy + uy Fx,
// added with (1 - s/2).  The conserved moments gain F exactly; e, eps, q
// relax at se, seps, sq and the stresses at snu = 1 / tau.  DEV: f holds
// f - w_q, whose moments are those of f less (1, -2, 1, 0, ...); its
// momentum rows are formed with div6 (the momentum moments are carried, not
// recomputed from u, so the reciprocal's rounding does not reach them).
template <class C, bool FORCE, bool DEV>
__device__ __forceinline__ void collide9m(C* f, C snu, C Fx, C Fy, C se, C seps, C sq) {
    const C sa = f[1] + f[2] + f[3] + f[4], sd = f[5] + f[6] + f[7] + f[8];
    const C ax = f[1] - f[3], ay = f[2] - f[4];
    const C dx = f[5] - f[6] - f[7] + f[8], dy = f[5] + f[6] - f[7] - f[8];
    const C m0 = f[0] + sa + sd;
    C m1 = (C)-4 * f[0] - sa + (C)2 * sd;
    C m2 = (C)4 * f[0] - (C)2 * sa + sd;
    C m3 = ax + dx, m4 = (C)-2 * ax + dx;
    C m5 = ay + dy, m6 = (C)-2 * ay + dy;
    C m7 = (f[1] + f[3]) - (f[2] + f[4]);
    C m8 = (f[5] + f[7]) - (f[6] + f[8]);
    const C rho = DEV ? (C)1 + m0 : m0;
    const C irho = (C)1 / rho;
    const C ux = FORCE ? (m3 + (C)0.5 * Fx) * irho : m3 * irho;
    const C uy = FORCE ? (m5 + (C)0.5 * Fy) * irho : m5 * irho;
    const C ru2 = (C)3 * rho * (ux * ux + uy * uy);
    const C ee = (C)-2 * m0 + ru2;  // e_eq in storage form (DEV: -2 drho + 3 rho u^2)
    const C pe = m0 - ru2;          // eps_eq likewise
    m1 += se * (ee - m1);
    m2 += seps * (pe - m2);
    m4 += sq * (-rho * ux - m4);
    m6 += sq * (-rho * uy - m6);
    m7 += snu * (rho * (ux * ux - uy * uy) - m7);
    m8 += snu * (rho * ux * uy - m8);
    if (FORCE) {
        const C uF = ux * Fx + uy * Fy;
        m1 += ((C)1 - (C)0.5 * se) * (C)6 * uF;
        m2 -= ((C)1 - (C)0.5 * seps) * (C)6 * uF;
        m3 += Fx;
        m5 += Fy;
        m4 -= ((C)1 - (C)0.5 * sq) * Fx;
        m6 -= ((C)1 - (C)0.5 * sq) * Fy;
        m7 += ((C)1 - (C)0.5 * snu) * (C)2 * (ux * Fx - uy * Fy);
        m8 += ((C)1 - (C)0.5 * snu) * (ux * Fy + uy * Fx);
    }
    // f = M^T diag(1 / norm) m
    const C n0 = m0 * ((C)1 / (C)9), n1 = m1 * ((C)1 / (C)36), n2 = m2 * ((C)1 / (C)36);
    const C n3 = DEV ? div6<C>(m3) : m3 * ((C)1 / (C)6), n4 = m4 * ((C)1 / (C)12);
    const C n5 = DEV ? div6<C>(m5) : m5 * ((C)1 / (C)6), n6 = m6 * ((C)1 / (C)12);
    const C n7 = m7 * (C)0.25, n8 = m8 * (C)0.25;
    const C axis = n0 - n1 - (C)2 * n2, diag = n0 + (C)2 * n1 + n2;
    f[0] = n0 - (C)4 * n1 + (C)4 * n2;
    f[1] = axis + n3 - (C)2 * n4 + n7;
    f[3] = axis - n3 + (C)2 * n4 + n7;
    f[2] = axis + n5 - (C)2 * n6 - n7;
    f[4] = axis - n5 + (C)2 * n6 - n7;
    const C xp = n3 + n4, yp = n5 + n6;
    f[5] = diag + xp + yp + n8;
    f[6] = diag - xp + yp - n8;
    f[7] = diag - xp - yp + n8;
    f[8] = diag + xp - yp - n8;
}

// The LES option of Sec. 2.1: BGK at tau_e = tau + 3 nu_t with the
// Smagorinsky viscosity nu_t = cs^2 |S| in the level's units, |S| = 3 Q /
// (2 rho tau_e) from the non-equilibrium stress Pi_ab = sum c_a c_b (f - f^eq)
// (Q = sqrt(2 Pi:Pi)): tau_e = (tau + sqrt(tau^2 + 18 cs^2 Q / rho)) / 2.
template <class C, bool FORCE, bool DEV>
__device__ __forceinline__ void collide9s(C* f, C om, C Fx, C Fy, C cs) {
    // Pi - Pi^eq from the second moments: the D2Q9 equilibrium of Eq. 7 has
    // sum c_a c_b f^eq = rho / 3 delta_ab + rho u_a u_b exactly (less 1/3
    // delta_ab for the deviations f - w_q, whose weights sum c c w to it)
    const C sd = f[5] + f[6] + f[7] + f[8];
    C pxx = f[1] + f[3] + sd, pyy = f[2] + f[4] + sd, pxy = f[5] - f[6] + f[7] - f[8];
    C rho, drho, ux, uy;
    moments9<C, FORCE, DEV>(f, Fx, Fy, rho, drho, ux, uy);
    const C p0 = (DEV ? drho : rho) * ((C)1 / (C)3);
    pxx -= p0 + rho * ux * ux;
    pyy -= p0 + rho * uy * uy;
    pxy -= rho * ux * uy;
    C ome;
    if constexpr (sizeof(C) == 4) {
        // tau_e = tau + dT, dT = (X / 2) / (sqrt(tau^2 + X) + tau), X = 18 cs^2
        // Q / rho, and 1 / tau_e = omega - omega a / (1 + a), a = omega dT: the
        // same tau_e without the cancellation of the printed form, and omega
        // itself wherever Q = 0.  Only the eddy part takes the approximate
        // reciprocal square root and divisions (no slow paths, so no registers
        // held for them).
        const float q2 = 2.0f * (pxx * pxx + pyy * pyy + 2.0f * pxy * pxy);
        const float Q = q2 > 0.0f ? q2 * rsqrtf(q2) : 0.0f;
        const float tau = __fdividef(1.0f, om);
        const float X = __fdividef(18.0f * cs * cs * Q, rho);
        const float d = tau * tau + X;
        const float dT = __fdividef(0.5f * X, d * rsqrtf(d) + tau);
        const float a = om * dT;
        ome = __fmaf_rn(-om, __fdividef(a, 1.0f + a), om);
    } else {
        const C tau = (C)1 / om;
        const C Q = sqrt((C)2 * (pxx * pxx + pyy * pyy + (C)2 * pxy * pxy));
        const C te = (C)0.5 * (tau + sqrt(tau * tau + (C)18 * cs * cs * Q / rho));
        ome = (C)1 / te;
    }
    bgk_update<C, FORCE, DEV, false>(f, ome, Fx, Fy, rho, drho, ux, uy);  // the moments of the same f
}

// the collision of the context's kind: COLL 0 BGK (Eq. 6), 1 MRT, 2 LES.
// NEQ: the relaxation form of 32-bit storage (bgk_update).
template <int COLL, class C, bool FORCE, bool DEV, bool NEQ = false>
__device__ __forceinline__ void collide_k(C* f, C om, C Fx, C Fy, const InstParams& ip) {
    if constexpr (COLL == 1)
        collide9m<C, FORCE, DEV>(f, om, Fx, Fy, (C)ip.mrt_s[0], (C)ip.mrt_s[1], (C)ip.mrt_s[2]);
    else if constexpr (COLL == 2)
        collide9s<C, FORCE, DEV>(f, om, Fx, Fy, (C)ip.les_cs);
    else
        collide9f<C, FORCE, DEV, NEQ>(f, om, Fx, Fy);
}

// Eq. 14
template <class C>
__device__ __forceinline__ C phi4(C r) {
    C a = r < (C)0 ? -r : r;
    if (a <= (C)1) return (C)0.125 * ((C)3 - (C)2 * a + sqrt((C)1 + (C)4 * a - (C)4 * a * a));
    if (a <= (C)2) return (C)0.125 * ((C)5 - (C)2 * a - sqrt((C)-7 + (C)12 * a - (C)4 * a * a));
    return (C)0;
}

__device__ __forceinline__ bool mask_bit(const DevPool& P, int slot, int cell) {
    return (P.slot_mask[(size_t)slot * P.mask_words + (cell >> 5)] >> (cell & 31)) & 1u;
}

__device__ __forceinline__ int wrapi(int v, int n) { return ((v % n) + n) % n; }

// Where a sweep finds the per-block data of the slot it updates: the pool's
// tables (MetaG), or a copy in shared memory (MetaS over a SlotMeta), which a
// task of the persistent step kernel reads before it waits for the phases it
// depends on (none of this data changes during a step).  Both give the same
// values, so the arithmetic is the same either way.
struct SlotMeta {
    int slot, type, flags, inst, ox, oy;
    int nb[9], nbt[9];        // neighbour slots (-1: none) and their types
    int child[4], childt[4];  // quarter children on the next level (-1: none) and their types
};
struct MetaG {
    const DevPool& P;
    int s;
    __device__ __forceinline__ int slot() const { return s; }
    __device__ __forceinline__ int flags() const { return P.slot_flags[s]; }
    __device__ __forceinline__ int ox() const { return P.slot_ox[s]; }
    __device__ __forceinline__ int oy() const { return P.slot_oy[s]; }
    __device__ __forceinline__ int nb(int k) const { return P.nbr[s * 9 + k]; }
    __device__ __forceinline__ int nbt(int, int ns) const { return P.slot_type[ns]; }
    __device__ __forceinline__ int child(int k) const { return P.slot_child[s * 4 + k]; }
    __device__ __forceinline__ int childt(int, int c) const { return P.slot_type[c]; }
};
struct MetaS {
    const SlotMeta* m;
    __device__ __forceinline__ int slot() const { return m->slot; }
    __device__ __forceinline__ int flags() const { return m->flags; }
    __device__ __forceinline__ int ox() const { return m->ox; }
    __device__ __forceinline__ int oy() const { return m->oy; }
    __device__ __forceinline__ int nb(int k) const { return m->nb[k]; }
    __device__ __forceinline__ int nbt(int k, int) const { return m->nbt[k]; }
    __device__ __forceinline__ int child(int k) const { return m->child[k]; }
    __device__ __forceinline__ int childt(int k, int) const { return m->childt[k]; }
};

// one warp: the data of `slot` into m (two dependent rounds of loads)
__device__ __forceinline__ void load_meta(const DevPool& P, int slot, SlotMeta& m) {
    const int lane = threadIdx.x & 31;
    if (lane < 9) {
        const int ns = P.nbr[slot * 9 + lane];
        m.nb[lane] = ns;
        m.nbt[lane] = ns >= 0 ? P.slot_type[ns] : -1;
    } else if (lane < 13) {
        const int c = P.slot_child[slot * 4 + lane - 9];
        m.child[lane - 9] = c;
        m.childt[lane - 9] = c >= 0 ? P.slot_type[c] : -1;
    } else if (lane == 13) {
        m.slot = slot;
        m.type = P.slot_type[slot];
    } else if (lane == 14) {
        m.flags = P.slot_flags[slot];
    } else if (lane == 15) {
        m.inst = P.slot_inst[slot];
    } else if (lane == 16) {
        m.ox = P.slot_ox[slot];
    } else if (lane == 17) {
        m.oy = P.slot_oy[slot];
    }
}

__device__ __forceinline__ int lat_slot(const DevPool& P, const InstParams& ip, int level, int gx, int gy) {
    int nxl = ip.nx0 << level, nyl = ip.ny0 << level;
    if (gx < 0 || gy < 0 || gx >= nxl || gy >= nyl) return -1;
    return ip.latmap[ip.latmap_off[level] + (long long)(gy / P.B) * ip.nbx[level] + gx / P.B];
}

// Half-way bounce-back from a wall side (reading R15): the population that
// left cell (ox, oy) toward the wall returns reversed, plus the momentum of
// the moving wall, 2 w_q rho0 (c_q . u_w) / c_s^2 (the same on deviations:
// opposite directions share w_q).
template <class S, class C>
__device__ C wall_bounce(const DevPool& P, const S* fin, const InstParams& ip, int level, int ox, int oy, int q,
                         int side) {
    const int s = lat_slot(P, ip, level, ox, oy);
    if (s < 0) {
        atomicOr(P.err, ERRB_NOSOURCE);
        return (C)0;
    }
    const int o = flipX(flipY(q)), B = P.B;
    const C a = Sto<S>::template ld<C>(fin, ((size_t)s * 9 + o) * B * B + (oy - P.slot_oy[s]) * B + (ox - P.slot_ox[s]), o,
                                       ip.dref);
    const double mw = 6.0 * Wq<double>(q) * ip.rho0 * (CXq(q) * ip.uwall[side][0] + CYq(q) * ip.uwall[side][1]);
    return a + (C)mw;
}

// Pull from outside the domain (non-periodic side), reading R2: the y-side
// rule first, then the x-side rule; periodic axes wrap.  (gx, gy) is the
// source of direction q; the cell pulling is (gx, gy) + c_q.
template <class S, class C>
__device__ __noinline__ C pull_boundary(const DevPool& P, const S* fin, const InstParams& ip, int level, int gx,
                                        int gy, int q) {
    const int ox = gx + CXq(q), oy = gy + CYq(q);
    int nxl = ip.nx0 << level, nyl = ip.ny0 << level;
    if (ip.periodic_y) gy = wrapi(gy, nyl);
    if (ip.periodic_x) gx = wrapi(gx, nxl);
    if (gy < 0 || gy >= nyl) {
        int side = gy < 0 ? SIDE_S : SIDE_N;
        int edge = gy < 0 ? 0 : nyl - 1;
        int k = ip.bc[side];
        if (k == BCK_INLET) return feq_s<S, C>(q, (C)ip.rho0, (C)ip.uin_x, (C)ip.uin_y);
        if (k == BCK_WALL) return wall_bounce<S, C>(P, fin, ip, level, ox, oy, q, side);
        gy = edge;
        if (k == BCK_SYMMETRY) q = flipY(q);
    }
    if (gx < 0 || gx >= nxl) {
        int side = gx < 0 ? SIDE_W : SIDE_E;
        int edge = gx < 0 ? 0 : nxl - 1;
        int k = ip.bc[side];
        if (k == BCK_INLET) return feq_s<S, C>(q, (C)ip.rho0, (C)ip.uin_x, (C)ip.uin_y);
        if (k == BCK_WALL) return wall_bounce<S, C>(P, fin, ip, level, ox, oy, q, side);
        gx = edge;
        if (k == BCK_SYMMETRY) q = flipX(q);
    }
    int s = lat_slot(P, ip, level, gx, gy);
    if (s < 0) {
        atomicOr(P.err, ERRB_NOSOURCE);
        return (C)0;
    }
    int B = P.B;
    return Sto<S>::template ld<C>(fin, ((size_t)s * 9 + q) * B * B + (gy - P.slot_oy[s]) * B + (gx - P.slot_ox[s]), q,
                                  ip.dref);
}

// The volumetric merge (Sec. 2.4 step 6, reading R3c): population q of
// coarse interior cell (x, y) of `slot`, streaming in from the finer region,
// is the mean of q over the 4 fine halo cells inside that cell (in its
// block's quarter child on the next level, after the two fine sub-steps).
template <class S, class C, class M>
__device__ __noinline__ C merge_fine(const DevPool& P, M mt, const S* ffine, const float* dr, int x, int y, int q) {
    const int B = P.B, BB = B * B;
    const int lx2 = 2 * x, ly2 = 2 * y;
    const int qx = lx2 >= B ? 1 : 0, qy = ly2 >= B ? 1 : 0;
    const int fslot = mt.child(qy * 2 + qx);
    if (ffine == nullptr || fslot < 0 || mt.childt(qy * 2 + qx, fslot) != ST_GF) {
        atomicOr(P.err, ERRB_HALO);
        return (C)0;
    }
    const int lx = lx2 - qx * B, ly = ly2 - qy * B;
    const size_t base = ((size_t)fslot * 9 + q) * BB;
    C s = Sto<S>::template ldr<C>(ffine, base + ly * B + lx);
    s += Sto<S>::template ldr<C>(ffine, base + ly * B + lx + 1);
    s += Sto<S>::template ldr<C>(ffine, base + (ly + 1) * B + lx);
    s += Sto<S>::template ldr<C>(ffine, base + (ly + 1) * B + lx + 1);
    return (C)0.25 * s + dshift<S, C>(dr, q);  // the mean of stored values, in compute form
}

// Eq. 10 for interior cell (x, y) of the slot mt describes, direction q.
// `mailbox`: the block has a neighbour inside the finer region
// (SLOTF_MAILBOX), whose populations come from the fine level (ffine)
// through merge_fine.
template <class S, class C, class M>
__device__ __forceinline__ C pull_int(const DevPool& P, M mt, const S* fin, const S* ffine, bool mailbox,
                                      const InstParams& ip, int level, int x, int y, int q) {
    const int B = P.B;
    int sx = x - CXq(q), sy = y - CYq(q);
    int dx = sx < 0 ? -1 : (sx >= B ? 1 : 0);
    int dy = sy < 0 ? -1 : (sy >= B ? 1 : 0);
    const int k = (dy + 1) * 3 + (dx + 1);
    int ns = mt.nb(k);
    if (ns >= 0) {
        if (mailbox && mt.nbt(k, ns) == ST_GC) return merge_fine<S, C, M>(P, mt, ffine, ip.dref, x, y, q);
        return Sto<S>::template ld<C>(fin, ((size_t)ns * 9 + q) * B * B + (sy - dy * B) * B + (sx - dx * B), q,
                                      ip.dref);
    }
    return pull_boundary<S, C>(P, fin, ip, level, mt.ox() + sx, mt.oy() + sy, q);
}
template <class S, class C>
__device__ __forceinline__ C pull_int(const DevPool& P, const S* fin, const S* ffine, bool mailbox, int slot,
                                      const InstParams& ip, int level, int x, int y, int q) {
    return pull_int<S, C, MetaG>(P, MetaG{P, slot}, fin, ffine, mailbox, ip, level, x, y, q);
}

// Reading R15: a solid obstacle on the finest level, kind 1 a circle, kind 2
// the half-plane y < y0; cell centres at (x + 1/2, y + 1/2)
__device__ __forceinline__ bool in_solid(const InstParams& ip, double px, double py) {
    if (ip.solid == 1) {
        const double dx = px - ip.sol[0], dy = py - ip.sol[1];
        return dx * dx + dy * dy < ip.sol[2] * ip.sol[2];
    }
    if (ip.solid == 2) return py < ip.sol[0];
    return false;
}

// the fraction of the link from (px, py) along (ex, ey) that lies outside
// the solid (the start outside, the end inside)
__device__ __forceinline__ double link_outside(const InstParams& ip, double px, double py, double ex, double ey) {
    if (ip.solid == 2) return (py - ip.sol[0]) / -ey;
    const double ax = px - ip.sol[0], ay = py - ip.sol[1];
    const double a = ex * ex + ey * ey, b = ax * ex + ay * ey, c = ax * ax + ay * ay - ip.sol[2] * ip.sol[2];
    return (-b - sqrt(b * b - a * c)) / a;
}

// Linearly interpolated bounce-back (reading R15) on the values f[9] just
// pulled into cell (x, y) of a block near the solid: every direction q whose
// source x - c_q is solid becomes, with t the fraction of that link outside
// the solid and o = opposite(q),
//   t < 1/2:  2t f*_o(x) + (1 - 2t) f*_o(x + c_q)  (x + c_q fluid: its f*_o is
//             the value pulled for direction o),
//   else:     f*_o(x) / 2t + (1 - 1/2t) f*_q(x).
// Returns false when the cell itself is solid (it is left as it is).
template <class S, class C>
__device__ __noinline__ bool solid_links(const DevPool& P, const S* fin, int slot, const InstParams& ip,
                                         int level, int x, int y, C* f) {
    const int B = P.B;
    const int gx = P.slot_ox[slot] + x, gy = P.slot_oy[slot] + y;
    const double px = gx + 0.5, py = gy + 0.5;
    if (in_solid(ip, px, py)) return false;
    C g[9];
#pragma unroll
    for (int q = 0; q < 9; q++) g[q] = f[q];
    const size_t own = (size_t)slot * 9 * B * B + (size_t)y * B + x;
    const int nxl = ip.nx0 << level, nyl = ip.ny0 << level;
    for (int q = 1; q < 9; q++) {
        const int cx = CXq(q), cy = CYq(q);
        if (!in_solid(ip, px - cx, py - cy)) continue;
        const int o = flipX(flipY(q));
        const double t = link_outside(ip, px, py, (double)-cx, (double)-cy);
        const C a = Sto<S>::template ld<C>(fin, own + (size_t)o * B * B, o, ip.dref);
        const int fx = gx + cx, fy = gy + cy;
        const bool far_fluid = (ip.periodic_x || (fx >= 0 && fx < nxl)) && (ip.periodic_y || (fy >= 0 && fy < nyl)) &&
                               !in_solid(ip, px + cx, py + cy);
        if (t < 0.5 && far_fluid) {
            f[q] = (C)(2.0 * t) * a + (C)(1.0 - 2.0 * t) * g[o];
        } else {
            const C b = Sto<S>::template ld<C>(fin, own + (size_t)q * B * B, q, ip.dref);
            f[q] = a / (C)(2.0 * t) + (C)(1.0 - 1.0 / (2.0 * t)) * b;
        }
    }
    return true;
}

template <class C>
__device__ __forceinline__ bool inlet_cell(const InstParams& ip, int level, int gx, int gy) {
    int nxl = ip.nx0 << level, nyl = ip.ny0 << level;
    return (gx == 0 && ip.bc[SIDE_W] == BCK_INLET) || (gx == nxl - 1 && ip.bc[SIDE_E] == BCK_INLET) ||
           (gy == 0 && ip.bc[SIDE_S] == BCK_INLET) || (gy == nyl - 1 && ip.bc[SIDE_N] == BCK_INLET);
}

template <class C>
__device__ __forceinline__ void patch_force(const DevPool& P, const InstParams& ip, int gx, int gy, C& Fx, C& Fy) {
    const InstState& st = P.ist[&ip - P.inst];
    int px = gx - st.patch_x0, py = gy - st.patch_y0;
    if (px >= 0 && py >= 0 && px < st.patch_w && py < st.patch_h) {
        const C* F = (const C*)ip.patch;
        int c = py * st.patch_w + px;
        Fx = F[c];
        Fy = F[ip.patch_cap + c];
    }
}

// ---------------------------------------------------------------------------
// fused stream + collide on one level
// ---------------------------------------------------------------------------
// one cell of the fused step, scalar path: halo cells stream without
// collision (Sec. 2.4 steps 3, 5); interior cells pull (Eq. 10 + boundary
// rules), take the IBM force, and collide (Eqs. 3, 6-8)
// fhalo (non-null): the finer level's buffer whose halo cells inside this
// level's blocks receive the post-collision populations of the coarse cell
// that contains them (the coarse-to-fine copy of Sec. 2.4 step 2, done by the
// cell that owns the values, right after the merge read the same halo cells)
template <class S, class C, int COLL, bool SOLID, class M>
__device__ __forceinline__ void fused_cell(const DevPool& P, M mt, const S* fin, S* fout, const S* ffine, int type,
                                           const InstParams& ip, int level, int x, int y, bool allow_force,
                                           S* fhalo = nullptr) {
    const int B = P.B, BB = B * B;
    const int cell = y * B + x;
    const int slot = mt.slot();
    if (type == ST_GF) {
        if (!mask_bit(P, slot, cell)) return;
#pragma unroll
        for (int q = 0; q < 9; q++) {
            int sx = x - CXq(q), sy = y - CYq(q);
            int dx = sx < 0 ? -1 : (sx >= B ? 1 : 0);
            int dy = sy < 0 ? -1 : (sy >= B ? 1 : 0);
            const int k = (dy + 1) * 3 + (dx + 1);
            int ns = mt.nb(k);
            int lc = (sy - dy * B) * B + (sx - dx * B);
            bool ok = false;
            if (ns >= 0) {
                int t = mt.nbt(k, ns);
                ok = (t == ST_INT) || (t == ST_GF && mask_bit(P, ns, lc));
            }
            size_t src = ok ? ((size_t)ns * 9 + q) * BB + lc : ((size_t)slot * 9 + q) * BB + cell;
            fout[((size_t)slot * 9 + q) * BB + cell] = fin[src];
        }
        return;
    }
    C f[9];
    const int flags = mt.flags();
    const bool mailbox = (flags & SLOTF_MAILBOX) != 0;
#pragma unroll
    for (int q = 0; q < 9; q++) f[q] = pull_int<S, C, M>(P, mt, fin, ffine, mailbox, ip, level, x, y, q);
    if constexpr (SOLID) {  // only in contexts holding a solid: the code costs every kernel that contains it
        if ((flags & SLOTF_SOLID) && !solid_links<S, C>(P, fin, slot, ip, level, x, y, f)) return;
    }
    C Fx = 0, Fy = 0;
    int gx = mt.ox() + x, gy = mt.oy() + y;
    if ((flags & SLOTF_EDGE) && inlet_cell<C>(ip, level, gx, gy)) {
#pragma unroll
        for (int q = 0; q < 9; q++) f[q] = feq_s<S, C>(q, (C)ip.rho0, (C)ip.uin_x, (C)ip.uin_y);
    } else if (allow_force && ip.has_body && level == ip.m - 1) {
        patch_force<C>(P, ip, gx, gy, Fx, Fy);
    }
    collide_k<COLL, C, true, DevTrait<S>::value, sizeof(S) == 4>(f, (C)1 / (C)ip.tau[level], Fx, Fy, ip);
#pragma unroll
    for (int q = 0; q < 9; q++) Sto<S>::template st<C>(fout, ((size_t)slot * 9 + q) * BB + cell, q, f[q], ip.dref);
    if (fhalo != nullptr && mailbox) {
        const int qx = 2 * x >= B ? 1 : 0, qy = 2 * y >= B ? 1 : 0;
        const int fs = mt.child(qy * 2 + qx);
        if (fs >= 0 && mt.childt(qy * 2 + qx, fs) == ST_GF) {
            const int lx = 2 * x - qx * B, ly = 2 * y - qy * B;
            S v[9];
#pragma unroll
            for (int q = 0; q < 9; q++) Sto<S>::template st<C>(v, q, q, f[q], ip.dref);  // as stored in fout
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int fc = (ly + (k >> 1)) * B + lx + (k & 1);
                if (!mask_bit(P, fs, fc)) continue;
#pragma unroll
                for (int q = 0; q < 9; q++) fhalo[((size_t)fs * 9 + q) * BB + fc] = v[q];
            }
        }
    }
}
template <class S, class C, int COLL, bool SOLID>
__device__ __forceinline__ void fused_cell(const DevPool& P, const S* fin, S* fout, const S* ffine, int slot, int type,
                                           const InstParams& ip, int level, int x, int y, bool allow_force,
                                           S* fhalo = nullptr) {
    fused_cell<S, C, COLL, SOLID, MetaG>(P, MetaG{P, slot}, fin, fout, ffine, type, ip, level, x, y, allow_force,
                                         fhalo);
}

// 4 consecutive values of one population plane, as compute type
template <class S, class C>
struct Vec4;
template <class C>
struct Vec4<float, C> {
    template <bool NC>
    static __device__ __forceinline__ float4 raw(const float* p) {
        return NC ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    }
    static __device__ __forceinline__ void unpack(float4 t, C* v) { v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w; }
    template <bool NC>
    static __device__ __forceinline__ void ld(const float* p, int, C* v) {
        float4 t = raw<NC>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float* p, int, const C* v) {
        *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    }
};
template <class C>
struct Vec4<double, C> {
    template <bool NC>
    static __device__ __forceinline__ void ld(const double* p, int, C* v) {
        const double2* p2 = reinterpret_cast<const double2*>(p);
        double2 a = NC ? __ldg(p2) : p2[0], b = NC ? __ldg(p2 + 1) : p2[1];
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
    static __device__ __forceinline__ void st(double* p, int, const C* v) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};
template <class C>
struct Vec4<__half, C> {
    static __device__ __forceinline__ void st(__half* p, int, const C* v) {
        __half2 a = __floats2half2_rn((float)v[0], (float)v[1]);
        __half2 b = __floats2half2_rn((float)v[2], (float)v[3]);
        uint2 t;
        t.x = *reinterpret_cast<unsigned*>(&a);
        t.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = t;
    }
};
template <class C>
struct Vec4<__nv_bfloat16, C> {
    static __device__ __forceinline__ void st(__nv_bfloat16* p, int, const C* v) {
        __nv_bfloat162 a = __floats2bfloat162_rn((float)v[0], (float)v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn((float)v[2], (float)v[3]);
        uint2 t;
        t.x = *reinterpret_cast<unsigned*>(&a);
        t.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = t;
    }
};
// one 16-byte load: through the read-only path when the data cannot change
// during the launch (NC), else a plain load
template <bool NC>
__device__ __forceinline__ uint4 ld_u4(const uint4* p) {
    return NC ? __ldg(p) : *p;
}

// Fused stream + collide for FP32 and FP64 storage (16-bit storage takes the
// 8-cell kernel below), 4 x-consecutive cells per thread (B = 16 or 32):
// every population plane is read with one 16-byte-class load per thread; the
// +-x shift of Eq. 10 comes from the neighbouring lane by a shuffle, and only
// the first/last lane of a row loads its edge cell from the west/east block.
// Neighbour slots are cached in shared memory.  Halo blocks and blocks on a
// non-periodic side (per warp: a warp never spans two blocks) take the scalar
// path above.
// The kernel's work for the list items item0, item0 + 1, ... (one per
// B * B / 4 threads of the thread block; items from n on are skipped).
// NC: the input buffer does not change during the launch (loads may take the
// read-only path).  Contains a block-wide barrier.
template <class S, class C, int B, int COLL, bool NC>
__device__ __forceinline__ void fused_v4_task(const DevPool& P, const int* list, int n, int item0, const S* fin, S* fout,
                                              const S* ffine, int level, int allow_force, S* fhalo = nullptr) {
    static_assert(sizeof(S) >= 4, "16-bit storage takes the 8-cell kernel");
    constexpr int BB = B * B, TPS = BB / 4, TPR = B / 4;
    __shared__ int nb[STEP_MAX_THREADS / TPS][9];
    const int ls = threadIdx.x / TPS, t = threadIdx.x % TPS;
    const int item = item0 + ls;
    if (t < 9) nb[ls][t] = item < n ? P.nbr[list[item] * 9 + t] : -1;
    __syncthreads();
    if (item >= n) return;
    const int slot = nb[ls][4];
    const int type = P.slot_type[slot];
    const InstParams& ip = P.inst[P.slot_inst[slot]];
    const int y = t / TPR, x0 = (t % TPR) * 4;
    if (type != ST_INT || (P.slot_flags[slot] & (SLOTF_EDGE | SLOTF_MAILBOX | SLOTF_SOLID))) {
        for (int i = 0; i < 4; i++)
            fused_cell<S, C, COLL, false>(P, fin, fout, ffine, slot, type, ip, level, x0 + i, y, allow_force != 0,
                                          fhalo);
        return;
    }
    C f[9][4];
    if constexpr (sizeof(S) == 4) {
        // FP32: the nine rows and the edge columns are all requested before
        // any is unpacked or shuffled, so that every load of the thread is in
        // flight at once (the kernel is memory-latency bound); 3 blocks per
        // SM hold its 36 row registers without spilling
        float4 raw[9];
        C edge[9];
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const int cx = CXq(q), cy = CYq(q);
            const int sy = y - cy;
            const int vy = sy < 0 ? 0 : (sy >= B ? 2 : 1);
            const int ry = sy + (vy == 0 ? B : (vy == 2 ? -B : 0));
            const size_t rowoff = (size_t)q * BB + ry * B;
            raw[q] = Vec4<S, C>::template raw<NC>(fin + (size_t)nb[ls][vy * 3 + 1] * 9 * BB + rowoff + x0);
            edge[q] = (C)0;
            if (cx == 1 && x0 == 0)
                edge[q] = Sto<S>::template ldr<C>(fin, (size_t)nb[ls][vy * 3 + 0] * 9 * BB + rowoff + (B - 1));
            if (cx == -1 && x0 + 4 == B)
                edge[q] = Sto<S>::template ldr<C>(fin, (size_t)nb[ls][vy * 3 + 2] * 9 * BB + rowoff);
        }
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const int cx = CXq(q);
            C v[4];
            Vec4<S, C>::unpack(raw[q], v);
            if (cx == 0) {
#pragma unroll
                for (int i = 0; i < 4; i++) f[q][i] = v[i];
            } else if (cx == 1) {
                C left = __shfl_up_sync(0xffffffffu, v[3], 1, TPR);
                if (x0 == 0) left = edge[q];
                f[q][0] = left, f[q][1] = v[0], f[q][2] = v[1], f[q][3] = v[2];
            } else {
                C right = __shfl_down_sync(0xffffffffu, v[0], 1, TPR);
                if (x0 + 4 == B) right = edge[q];
                f[q][0] = v[1], f[q][1] = v[2], f[q][2] = v[3], f[q][3] = right;
            }
        }
    } else {
#pragma unroll
    for (int q = 0; q < 9; q++) {
        constexpr int dummy = 0;
        (void)dummy;
        const int cx = CXq(q), cy = CYq(q);
        const int sy = y - cy;
        const int vy = sy < 0 ? 0 : (sy >= B ? 2 : 1);
        const int ry = sy + (vy == 0 ? B : (vy == 2 ? -B : 0));
        const size_t rowoff = (size_t)q * BB + ry * B;
        const int rs = nb[ls][vy * 3 + 1];
        C v[4];
        Vec4<S, C>::template ld<NC>(fin + (size_t)rs * 9 * BB + rowoff + x0, q, v);
        if (cx == 0) {
#pragma unroll
            for (int i = 0; i < 4; i++) f[q][i] = v[i];
        } else if (cx == 1) {
            C left = __shfl_up_sync(0xffffffffu, v[3], 1, TPR);
            if (x0 == 0) left = Sto<S>::template ldr<C>(fin, (size_t)nb[ls][vy * 3 + 0] * 9 * BB + rowoff + (B - 1));
            f[q][0] = left, f[q][1] = v[0], f[q][2] = v[1], f[q][3] = v[2];
        } else {
            C right = __shfl_down_sync(0xffffffffu, v[0], 1, TPR);
            if (x0 + 4 == B) right = Sto<S>::template ldr<C>(fin, (size_t)nb[ls][vy * 3 + 2] * 9 * BB + rowoff);
            f[q][0] = v[1], f[q][1] = v[2], f[q][2] = v[3], f[q][3] = right;
        }
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
    if (force) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            C g[9];
#pragma unroll
            for (int q = 0; q < 9; q++) g[q] = f[q][i];
            C Fx = 0, Fy = 0;
            patch_force<C>(P, ip, gx0 + i, gy, Fx, Fy);
            collide_k<COLL, C, true, DevTrait<S>::value, sizeof(S) == 4>(g, om, Fx, Fy, ip);
#pragma unroll
            for (int q = 0; q < 9; q++) f[q][i] = g[q];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            C g[9];
#pragma unroll
            for (int q = 0; q < 9; q++) g[q] = f[q][i];
            collide_k<COLL, C, false, DevTrait<S>::value, sizeof(S) == 4>(g, om, (C)0, (C)0, ip);
#pragma unroll
            for (int q = 0; q < 9; q++) f[q][i] = g[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 9; q++) Vec4<S, C>::st(fout + ((size_t)slot * 9 + q) * BB + y * B + x0, q, f[q]);
}
// Two 16-bit values packed in one 32-bit word (the lower address in the low
// half), to and from the compute type; the rounding is that of the 4-cell
// kernel's stores.
template <class S>
struct Pair16;
template <>
struct Pair16<__half> {
    static __device__ __forceinline__ float lo(unsigned w) {
        return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu)));
    }
    static __device__ __forceinline__ float hi(unsigned w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<unsigned*>(&h);
    }
};
template <>
struct Pair16<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(unsigned w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<unsigned*>(&h);
    }
};
// value k (0..7) of a packed row of eight
template <class S>
__device__ __forceinline__ float el8(const uint4& r, int k) {
    const unsigned w = k < 2 ? r.x : (k < 4 ? r.y : (k < 6 ? r.z : r.w));
    return (k & 1) ? Pair16<S>::hi(w) : Pair16<S>::lo(w);
}
// Fused stream + collide for 16-bit storage, 8 x-consecutive cells per thread
// (B = 16 or 32): each population plane is one 16-byte load per thread, so the
// thread has as many bytes in flight as the FP32 kernel above with the same
// 36 row registers; the values stay packed until their cell is collided and
// the results are packed again pair by pair.  The +-x shift of Eq. 10 takes
// the neighbouring lane's end value by a shuffle, the first/last lane of a row
// its edge value from the west/east block.  The arithmetic and rounding per
// cell are those of the 4-cell kernel, so the results equal it bit for bit.
// The kernel's work for the list items item0, item0 + 1, ... (one per
// B * B / 8 threads; n and NC as for fused_v4_task).  Contains a block-wide
// barrier.
template <class S, class C, int B, int COLL, bool NC, bool SH>
__device__ __forceinline__ void fused_v8_task(const DevPool& P, const int* list, int n, int item0, const S* fin, S* fout,
                                              const S* ffine, int level, int allow_force, S* fhalo = nullptr) {
    static_assert(sizeof(S) == 2, "the 8-cell kernel is for 16-bit storage");
    constexpr int BB = B * B, TPS = BB / 8, TPR = B / 8;
    __shared__ int nb[STEP_MAX_THREADS / TPS][9];
    const int ls = threadIdx.x / TPS, t = threadIdx.x % TPS;
    const int item = item0 + ls;
    if (t < 9) nb[ls][t] = item < n ? P.nbr[list[item] * 9 + t] : -1;
    __syncthreads();
    if (item >= n) return;
    const int slot = nb[ls][4];
    const int type = P.slot_type[slot];
    const InstParams& ip = P.inst[P.slot_inst[slot]];
    const int y = t / TPR, x0 = (t % TPR) * 8;
    if (type != ST_INT || (P.slot_flags[slot] & (SLOTF_EDGE | SLOTF_MAILBOX | SLOTF_SOLID))) {
        for (int i = 0; i < 8; i++)
            fused_cell<S, C, COLL, false>(P, fin, fout, ffine, slot, type, ip, level, x0 + i, y, allow_force != 0,
                                          fhalo);
        return;
    }
    // all nine rows and the edge values requested before any is used
    uint4 raw[9];
    C edge[9];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const int cx = CXq(q), cy = CYq(q);
        const int sy = y - cy;
        const int vy = sy < 0 ? 0 : (sy >= B ? 2 : 1);
        const int ry = sy + (vy == 0 ? B : (vy == 2 ? -B : 0));
        const size_t rowoff = (size_t)q * BB + ry * B;
        raw[q] = ld_u4<NC>(reinterpret_cast<const uint4*>(fin + (size_t)nb[ls][vy * 3 + 1] * 9 * BB + rowoff + x0));
        edge[q] = (C)0;
        if (cx == 1 && x0 == 0)
            edge[q] = Sto<S>::template ldr<C>(fin, (size_t)nb[ls][vy * 3 + 0] * 9 * BB + rowoff + (B - 1));
        if (cx == -1 && x0 + 8 == B)
            edge[q] = Sto<S>::template ldr<C>(fin, (size_t)nb[ls][vy * 3 + 2] * 9 * BB + rowoff);
    }
    // the value each shifted plane pulls from beyond this thread's eight cells
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const int cx = CXq(q);
        if (cx == 1) {
            const C left = Pair16<S>::hi(__shfl_up_sync(0xffffffffu, raw[q].w, 1, TPR));
            if (x0 != 0) edge[q] = left;
        } else if (cx == -1) {
            const C right = Pair16<S>::lo(__shfl_down_sync(0xffffffffu, raw[q].x, 1, TPR));
            if (x0 + 8 != B) edge[q] = right;
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
    unsigned ow[9][4];
    // SH: values move between the storage and the compute form by the
    // instance's shift (its nine values take registers the kernel is short
    // of, so contexts whose instances all have a zero shift launch SH = false)
    auto shift = [&](int q) { return SH ? (C)ip.dref[q] : (C)0; };
    auto cells = [&](auto with_force) {
        constexpr bool F = decltype(with_force)::value;
        C prev[9];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            C g[9];
#pragma unroll
            for (int q = 0; q < 9; q++) {
                const int src = i - CXq(q);  // Eq. 10: pull from x - c_q
                g[q] = (src < 0 || src > 7) ? edge[q] : el8<S>(raw[q], src);
                if constexpr (SH) g[q] += shift(q);  // compute form
            }
            C Fx = 0, Fy = 0;
            if constexpr (F) patch_force<C>(P, ip, gx0 + i, gy, Fx, Fy);
            collide_k<COLL, C, F, DevTrait<S>::value, sizeof(S) == 4>(g, om, Fx, Fy, ip);
#pragma unroll
            for (int q = 0; q < 9; q++) {
                const C sq = SH ? g[q] - shift(q) : g[q];  // storage form
                if (i & 1)
                    ow[q][i >> 1] = Pair16<S>::pack((float)prev[q], (float)sq);
                else
                    prev[q] = sq;
            }
        }
    };
    if (force)
        cells(std::true_type{});
    else
        cells(std::false_type{});
#pragma unroll
    for (int q = 0; q < 9; q++)
        *reinterpret_cast<uint4*>(fout + ((size_t)slot * 9 + q) * BB + y * B + x0) =
            make_uint4(ow[q][0], ow[q][1], ow[q][2], ow[q][3]);
}
// ---------------------------------------------------------------------------
// Sec. 2.4 step 2: every fine halo cell gets the post-collision populations of
// the coarse cell that contains it
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void c2f_cell(const DevPool& P, int slot, int cell, const S* fc, S* ff) {
    const int B = P.B, BB = B * B;
    if (!mask_bit(P, slot, cell)) return;
    int parent = P.slot_parent[slot];
    if (parent < 0) {
        atomicOr(P.err, ERRB_HALO);
        return;
    }
    int gx = P.slot_ox[slot] + cell % B, gy = P.slot_oy[slot] + cell / B;
    int cx = (gx >> 1) - P.slot_ox[parent], cy = (gy >> 1) - P.slot_oy[parent];
#pragma unroll
    for (int q = 0; q < 9; q++)
        ff[((size_t)slot * 9 + q) * BB + cell] = fc[((size_t)parent * 9 + q) * BB + cy * B + cx];
}

// ---------------------------------------------------------------------------
// Sec. 2.2 + Sec. 3.6: body pose, markers, multi-direct forcing, body force
// ---------------------------------------------------------------------------
__device__ __forceinline__ void marker_at(const DevPool& P, const InstParams& ip, int j, double cx, double cy,
                                          double ca, double sa, double& rx, double& ry) {
    double px = ip.qx[j] - ip.pivot[0];
    double py = ip.qy[j] - ip.pivot[1];
    rx = cx + ip.pivot[0] + ca * px - sa * py;
    ry = cy + ip.pivot[1] + sa * px + ca * py;
}

__device__ __forceinline__ int stencil0(double r) {
    double v = floor(r - 0.5) - 1.0;
    return (v > -1.0e9 && v < 1.0e9) ? (int)v : (v > 0 ? 1000000000 : -1000000000);  // NaN maps to -1e9
}

#define IBM_MAXB 16                  // blocks per side of the marker box held in the slot table

template <class C>
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    return s;  // valid in thread 0
}

// carve `n` elements of T out of shared memory at `p`, 16-byte aligned
template <class T>
__device__ __forceinline__ T* carve(unsigned char*& p, long long n) {
    T* r = reinterpret_cast<T*>(p);
    p += ((size_t)n * sizeof(T) + 15) & ~(size_t)15;
    return r;
}

// Exclusive prefix sum of a[0..n) in place by the whole block; returns the
// total.  wtot: 32 ints of shared scratch.
__device__ int block_scan_inplace(int* a, int n, int* wtot) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
    const int per = (n + nt - 1) / nt, i0 = tid * per, i1 = min(n, i0 + per);
    int sum = 0;
    for (int i = i0; i < i1; i++) sum += a[i];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();  // wtot may still be read by a previous call
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int v = lane < nwarp ? wtot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wtot[lane] = v;
    }
    __syncthreads();
    int base = (wid > 0 ? wtot[wid - 1] : 0) + x - sum;
    for (int i = i0; i < i1; i++) {
        const int c = a[i];
        a[i] = base;
        base += c;
    }
    const int total = wtot[nwarp - 1];
    __syncthreads();
    return total;
}

// Sec. 3.4-3.6 kinematics of one body at finest time t: centre and cos, sin
// of the pitch angle (the stroke-plane angle's cos and sin come from the host)
__device__ __forceinline__ void pose_at(const InstParams& ip, double t, double* out) {
    double al = ip.alpha_mean, h = 0.0;
    if (ip.motion == 1 || ip.motion == 2)
        al = ip.alpha_mean - ip.alpha_amp * sin(2.0 * M_PI * t / ip.period + ip.phase);
    if (ip.motion == 3)
        al = ip.alpha_mean - sbot_kin::ramp_alpha(ip.alpha_amp, ip.ramp_as, ip.ramp_rate, ip.ramp_t1, t / ip.t_ref);
    if (ip.motion == 4)
        al = ip.alpha_mean - sbot_kin::triangle_alpha(ip.alpha_amp, ip.asym_xi, ip.accel_frac, ip.period,
                                                      t + ip.phase * ip.period / (2.0 * M_PI));
    if (ip.motion == 2) h = 0.5 * ip.heave_amp * cos(2.0 * M_PI * t / ip.period);
    double sa, ca;
    sincos(al, &sa, &ca);
    out[0] = ip.x0[0] + h * ip.cos_beta;
    out[1] = ip.x0[1] + h * ip.sin_beta;
    out[2] = ca;
    out[3] = sa;
}
// the poses of the coarse step starting at the body's current finest time,
// one thread per time, so that the IBM launches of the step read them
// instead of evaluating the kinematics one after another
__device__ void pose_run(const DevPool& P, int inst) {
    const InstParams& ip = P.inst[inst];
    if (ip.motion == 0 || ip.pose_tab == nullptr) return;
    InstState* st = &P.ist[inst];
    const long long k0 = st->fine_step;
    for (int i = threadIdx.x; i < ip.pose_n; i += blockDim.x) pose_at(ip, (double)(k0 + i), ip.pose_tab + 4 * i);
    if (threadIdx.x == 0) st->pose_k0 = k0;
}
// The IBM of Sec. 2.2, one thread block per body.  It works on the union of
// the marker stencils only (a bitmap over the markers' bounding box,
// compacted by a prefix sum), and gives every stencil cell the list of the
// markers that cover it, sorted by marker index.  Each of the K iterations is
// then two gathers without atomics: per marker, Eq. 12 over its 16 cells and
// Eq. 11; per cell, Eq. 15 over its markers (in ascending marker order, the
// order of a plain loop over markers) and the half-force correction of
// Eq. 8.  Every sum runs in a fixed order, so results do not depend on
// thread scheduling.
//
// The geometry (stencils, kernel weights, moment arms, desired velocities,
// compact cells, lists, block slots) depends only on the body's pose and on
// the topology of the coarse step, so it is computed off the critical path
// and stored: a static body's by its first IBM launch, a moving body's for
// every finest step of the coarse step at once by k_ibm_geom on the pose
// stream.  k_ibm loads the stored copy and computes the geometry itself only
// when no stored copy belongs to its step.
//
// Shared memory, carved in this order (ibm_smem_bytes sizes it); the first
// part, up to the lists, is what a stored geometry holds after its header:
// the slot table of the box blocks; per marker its stencil origin ([N] x and
// y), its 4 + 4 kernel weights ([N][8]), its desired velocity and moment arm
// ([N] records of 4), the compact indices of its 16 stencil cells ([N][16]);
// per stencil cell its box index and the start of its marker list; the lists
// as (marker * 16 + stencil position, kernel weight) records.  Then: per
// marker the interpolated density, the force and the force increment (pairs);
// the bitmap with per-word prefix counts; list fill cursors; per stencil cell
// the velocity being corrected and the force (records of 4), rho and
// 1/(2 rho).  Records are read and written whole (vector accesses), so each
// iteration issues about half the shared-memory instructions of one array
// per component.
#define IBM_THREADS 1024

struct IbmCacheHead {  // the first bytes of a stored IBM geometry
    long long stamp;   // moving bodies: the finest time the geometry belongs to
    int valid, px0, py0, w, h, ncell, table, pnbx, pnby, pbx0, pby0, pad[3];
};
static_assert(sizeof(IbmCacheHead) % 16 == 0, "the stored geometry follows its header at 16-byte alignment");

template <class C>
struct alignas(2 * sizeof(C)) IbmV2 {
    C x, y;
};
template <class C>
struct alignas(16) IbmV4 {
    C x, y, z, w;
};
template <class C>
struct alignas(sizeof(C) == 8 ? 16 : 8) IbmEnt {  // a list entry: marker * 16 + stencil position, weight
    int m16;
    C w;
};

template <class C>
struct IbmSmem {
    int* pslot;
    int *ox, *oy;
    C* wph;               // [N][8]: phi_x[0..3], phi_y[0..3]
    IbmV4<C>* mk;         // [N]: u^d x, u^d y, arm x, arm y
    uint16_t* cidx;       // [N][16]
    int *ccell, *cst;
    IbmEnt<C>* ent;       // [16 N]
    size_t cache_bytes;   // the part a stored geometry holds
    C* rj;
    IbmV2<C> *F, *dF;     // [N]
    unsigned* bits;
    int *wpre, *ccur;
    IbmV4<C>* cs;         // [ncap]: u x, u y, F x, F y
    C *crho, *cinv;
};

template <class C>
__device__ __forceinline__ IbmSmem<C> ibm_carve(unsigned char* smraw, int N, int ncap, int W) {
    IbmSmem<C> m;
    unsigned char* sp = smraw;
    m.pslot = carve<int>(sp, IBM_MAXB * IBM_MAXB * 9);
    m.ox = carve<int>(sp, N);
    m.oy = carve<int>(sp, N);
    m.wph = carve<C>(sp, 8LL * N);
    m.mk = carve<IbmV4<C>>(sp, N);
    m.cidx = carve<uint16_t>(sp, 16LL * N);
    m.ccell = carve<int>(sp, ncap);
    m.cst = carve<int>(sp, ncap + 1);
    m.ent = carve<IbmEnt<C>>(sp, 16LL * N);
    m.cache_bytes = (size_t)(sp - smraw);
    m.rj = carve<C>(sp, N);
    m.F = carve<IbmV2<C>>(sp, N);
    m.dF = carve<IbmV2<C>>(sp, N);
    m.bits = carve<unsigned>(sp, W);
    m.wpre = carve<int>(sp, W + 1);
    m.ccur = carve<int>(sp, ncap);
    m.cs = carve<IbmV4<C>>(sp, ncap);
    m.crho = carve<C>(sp, ncap);
    m.cinv = carve<C>(sp, ncap);
    return m;
}

// stencil cells: markers about one cell apart (Sec. 2.2) add 4-5 new cells
// each; 8 per marker allows spacings up to about two cells (more is an
// ERRB_PATCH report)
__device__ __forceinline__ int ibm_ncap(int cap, int N) { return min(cap, 8 * N + 64); }

// The geometry of one body on `level` at the pose pose[0..3] (centre, cos,
// sin at time k), with the desired marker velocities of Eq. 11 toward
// pose[4..7] (time k + 1; zero for a static body), into the stored part of
// shared memory and `hd`.  Called by the whole block; returns false, for all
// threads, when the stencils do not fit the force patch (reported as
// ERRB_PATCH).
template <class C>
__device__ bool ibm_geometry(const DevPool& P, const InstParams& ip, int level, const double* pose, bool still,
                             const IbmSmem<C>& m, IbmCacheHead& hd, int* bb, int* wtot) {
    const int B = P.B, N = ip.n_markers, cap = ip.patch_cap, tid = threadIdx.x, nt = blockDim.x;
    const int ncap = ibm_ncap(cap, N), W = (cap + 31) / 32 + 1;
    if (tid == 0) {
        bb[0] = INT_MAX;
        bb[1] = INT_MAX;
        bb[2] = INT_MIN;
        bb[3] = INT_MIN;
    }
    __syncthreads();
    // markers: positions, desired velocities, stencils, kernel weights (Eq. 14)
    for (int j = tid; j < N; j += nt) {
        double rx, ry;
        marker_at(P, ip, j, pose[0], pose[1], pose[2], pose[3], rx, ry);
        IbmV4<C> mj;
        if (still) {
            mj.x = 0;
            mj.y = 0;
        } else {
            double rx1, ry1;
            marker_at(P, ip, j, pose[4], pose[5], pose[6], pose[7], rx1, ry1);
            mj.x = (C)(rx1 - rx);  // Sec. 2.2: u^d = (r(t + dt) - r(t)) / dt
            mj.y = (C)(ry1 - ry);
        }
        mj.z = (C)(rx - (pose[0] + ip.pivot[0]));  // arm of the moment about the pivot
        mj.w = (C)(ry - (pose[1] + ip.pivot[1]));
        m.mk[j] = mj;
        const int i0 = stencil0(rx), j0 = stencil0(ry);
        m.ox[j] = i0;
        m.oy[j] = j0;
        const C fx = (C)(rx - (double)i0 - 0.5), fy = (C)(ry - (double)j0 - 0.5);  // in [1, 2)
#pragma unroll
        for (int a = 0; a < 4; a++) {
            m.wph[8 * j + a] = phi4<C>((C)a - fx);
            m.wph[8 * j + 4 + a] = phi4<C>((C)a - fy);
        }
        atomicMin(&bb[0], i0);
        atomicMin(&bb[1], j0);
        atomicMax(&bb[2], i0 + 3);
        atomicMax(&bb[3], j0 + 3);
    }
    __syncthreads();
    const int px0 = bb[0], py0 = bb[1];
    const long long wl = (long long)bb[2] - bb[0] + 1, hl = (long long)bb[3] - bb[1] + 1;
    if (wl <= 0 || hl <= 0 || wl > 65536 || hl > 65536 || wl * hl > cap) {  // also catches NaN positions
        if (tid == 0) atomicOr(P.err, ERRB_PATCH);
        return false;
    }
    const int w = (int)wl, h = (int)hl;
    // slots of the blocks under the box and of their 3x3 neighbourhoods,
    // resolved once (when the box spans at most IBM_MAXB x IBM_MAXB blocks)
    const int pbx0 = px0 >= 0 ? px0 / B : -1, pby0 = py0 >= 0 ? py0 / B : -1;
    const int pnbx = (px0 + w - 1) / B - pbx0 + 1, pnby = (py0 + h - 1) / B - pby0 + 1;
    const bool table = px0 >= 0 && py0 >= 0 && pnbx <= IBM_MAXB && pnby <= IBM_MAXB;
    if (table) {
        for (int e = tid; e < pnbx * pnby * 9; e += nt) {
            int b = e / 9, kk = e % 9;
            int sl = lat_slot(P, ip, level, (pbx0 + b % pnbx) * B, (pby0 + b / pnbx) * B);
            m.pslot[b * 9 + kk] =
                (sl >= 0 && P.slot_type[sl] == ST_INT) ? P.nbr[sl * 9 + kk] : (kk == 4 ? -1 : -2);
        }
    }
    for (int i = tid; i < W; i += nt) m.bits[i] = 0u;
    for (int i = tid; i <= ncap; i += nt) m.cst[i] = 0;
    __syncthreads();
    // the union of the marker stencils as a bitmap over the box
    for (int t = tid; t < 16 * N; t += nt) {
        const int j = t >> 4, s = t & 15;
        const int c = (m.oy[j] - py0 + (s >> 2)) * w + (m.ox[j] - px0 + (s & 3));
        atomicOr(&m.bits[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
    for (int i = tid; i < W; i += nt) m.wpre[i] = __popc(m.bits[i]);
    __syncthreads();
    // compact index of a stencil cell = the set bits before it
    const int ncell = block_scan_inplace(m.wpre, W, wtot);
    if (ncell > ncap) {
        if (tid == 0) atomicOr(P.err, ERRB_PATCH);
        return false;
    }
    for (int i = tid; i < W; i += nt) {
        unsigned b = m.bits[i];
        int r = m.wpre[i];
        while (b) {
            m.ccell[r++] = i * 32 + (__ffs(b) - 1);
            b &= b - 1;
        }
    }
    for (int t = tid; t < 16 * N; t += nt) {
        const int j = t >> 4, s = t & 15;
        const int c = (m.oy[j] - py0 + (s >> 2)) * w + (m.ox[j] - px0 + (s & 3));
        const int ci = m.wpre[c >> 5] + __popc(m.bits[c >> 5] & ((1u << (c & 31)) - 1u));
        m.cidx[16 * j + s] = (uint16_t)ci;
        atomicAdd(&m.cst[ci], 1);
    }
    __syncthreads();
    // each cell's list of covering markers: starts, a fill, then marker order
    block_scan_inplace(m.cst, ncell + 1, wtot);
    for (int i = tid; i < ncell; i += nt) m.ccur[i] = m.cst[i];
    __syncthreads();
    for (int t = tid; t < 16 * N; t += nt)  // t = marker * 16 + stencil position
        m.ent[atomicAdd(&m.ccur[m.cidx[t]], 1)].m16 = t;
    __syncthreads();
    for (int ci = tid; ci < ncell; ci += nt) {
        const int b0 = m.cst[ci], b1 = m.cst[ci + 1];
        for (int i = b0 + 1; i < b1; i++) {  // insertion sort of the cell's few entries
            const int v = m.ent[i].m16;
            int q = i - 1;
            while (q >= b0 && m.ent[q].m16 > v) {
                m.ent[q + 1].m16 = m.ent[q].m16;
                q--;
            }
            m.ent[q + 1].m16 = v;
        }
        for (int e = b0; e < b1; e++) {
            const int j = m.ent[e].m16 >> 4, sc = m.ent[e].m16 & 15;
            m.ent[e].w = m.wph[8 * j + (sc & 3)] * m.wph[8 * j + 4 + (sc >> 2)];
        }
    }
    if (tid == 0) {
        hd.stamp = -1;
        hd.valid = 1, hd.px0 = px0, hd.py0 = py0, hd.w = w, hd.h = h, hd.ncell = ncell;
        hd.table = table ? 1 : 0, hd.pnbx = pnbx, hd.pnby = pnby, hd.pbx0 = pbx0, hd.pby0 = pby0;
    }
    __syncthreads();
    return true;
}

// a stored geometry: the header, then the first cache_bytes of shared memory
// (called by the whole block; the stamp is written last, with release
// semantics after every thread's copy, so that a reader that sees it with
// acquire semantics finds the whole entry)
__device__ __forceinline__ void ibm_store(IbmCacheHead* dst, const IbmCacheHead& hd, const unsigned char* smraw,
                                          size_t cache_bytes, long long stamp) {
    const uint4* s = (const uint4*)smraw;
    uint4* d = (uint4*)(dst + 1);
    for (size_t i = threadIdx.x; i < cache_bytes / 16; i += blockDim.x) d[i] = s[i];
    if (threadIdx.x == 0) {
        IbmCacheHead h = hd;
        h.stamp = -1;
        *dst = h;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(&dst->stamp), "l"(stamp) : "memory");
    }
}

__device__ __forceinline__ long long ld_acquire_s64(const long long* p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void ibm_load(const IbmCacheHead* src, IbmCacheHead& hd, unsigned char* smraw,
                                         size_t cache_bytes) {
    if (threadIdx.x < (int)(sizeof(IbmCacheHead) / 4)) ((int*)&hd)[threadIdx.x] = ((const int*)src)[threadIdx.x];
    const uint4* s = (const uint4*)(src + 1);
    uint4* d = (uint4*)smraw;
    for (size_t i = threadIdx.x; i < cache_bytes / 16; i += blockDim.x) d[i] = s[i];
}

// Eq. 16 and the moment about the pivot from per-marker terms (F_j ds and
// (r_j - r_p) x F_j ds in the compute type): an FP64 sum in a fixed order
// (markers strided over the block's threads, then lanes, then warps) into
// out3 by thread 0.  Called by the whole block.
template <class C, class Terms>
__device__ void ibm_force_sum(int N, Terms terms, double (*red)[32], double* out3) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    double fx = 0.0, fy = 0.0, mz = 0.0;
    const int nw = min(nt, N + 31) >> 5;  // warps that hold markers
    for (int j = tid; j < N; j += nt) {
        C a, b, mm;
        terms(j, a, b, mm);
        fx -= (double)a;
        fy -= (double)b;
        mz -= (double)mm;
    }
    if (wid < nw) {
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_down_sync(0xffffffffu, fx, o);
            fy += __shfl_down_sync(0xffffffffu, fy, o);
            mz += __shfl_down_sync(0xffffffffu, mz, o);
        }
    }
    if (lane == 0 && wid < nw) {
        red[0][wid] = fx;
        red[1][wid] = fy;
        red[2][wid] = mz;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0, b2 = 0, c2 = 0;
        for (int i = 0; i < nw; i++) {
            a += red[0][i];
            b2 += red[1][i];
            c2 += red[2][i];
        }
        out3[0] = a;
        out3[1] = b2;
        out3[2] = c2;
    }
}
// the fixed-size shared memory of the IBM and geometry steps
struct IbmShared {
    int bb[4];
    double pose[8];
    double red[3][32];
    int wtot[32];
    IbmCacheHead head;
};

// The geometry of every finest step of the coarse step of the moving bodies
// in the list, one block per (body, step), from the pose table k_pose wrote
// just before on the same stream: entry i of the body's store is the
// geometry at time pose_k0 + i.
template <class C>
__device__ void ibm_geom_run(const DevPool& P, int inst, int i, unsigned char* smraw, IbmShared& sh) {
    const InstParams& ip = P.inst[inst];
    const InstState* st = &P.ist[inst];
    if (ip.motion == 0 || ip.ibm_cache == nullptr || ip.pose_tab == nullptr || i + 1 >= ip.pose_n) return;
    const long long k0 = st->pose_k0;
    if (k0 < 0) return;
    const int N = ip.n_markers, ncap = ibm_ncap(ip.patch_cap, N), W = (ip.patch_cap + 31) / 32 + 1;
    const IbmSmem<C> m = ibm_carve<C>(smraw, N, ncap, W);
    int* const bb = sh.bb;
    double* const pose = sh.pose;
    int* const wtot = sh.wtot;
    IbmCacheHead& head = sh.head;
    if (threadIdx.x < 8) pose[threadIdx.x] = ip.pose_tab[4 * i + threadIdx.x];
    __syncthreads();
    IbmCacheHead* e = (IbmCacheHead*)((unsigned char*)ip.ibm_cache + (size_t)i * ip.ibm_cache_stride);
    if (!ibm_geometry<C>(P, ip, ip.m - 1, pose, false, m, head, bb, wtot)) {
        if (threadIdx.x == 0) e->stamp = -1;
        return;
    }
    ibm_store(e, head, smraw, m.cache_bytes, k0 + i);
}
// One body's IBM step (k_ibm runs one per thread block); smraw is the
// block's dynamic shared memory (ibm_smem_bytes), sh its fixed part.
// gate(): called once by the whole block, after the part that may run before
// the step's earlier phases have finished (the load of a stored geometry)
// and before the first read of their results; false: stop (the launch is
// aborting).
template <class S, class C, class G>
__device__ void ibm_run(const DevPool& P, int inst, const S* fin, int level, int direct, int deferred,
                        unsigned char* smraw, IbmShared& sh, G&& gate) {
    const InstParams& ip = P.inst[inst];
    InstState* st = &P.ist[inst];
    const int B = P.B;
    const int N = ip.n_markers, cap = ip.patch_cap, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int ncap = ibm_ncap(cap, N), W = (cap + 31) / 32 + 1;

    const IbmSmem<C> m = ibm_carve<C>(smraw, N, ncap, W);
    int* const pslot = m.pslot;
    IbmV2<C>* const F = m.F;
    int* const bb = sh.bb;
    double* const pose = sh.pose;
    double(*const red)[32] = sh.red;
    int* const wtot = sh.wtot;
    IbmCacheHead& head = sh.head;

    const bool still = ip.motion == 0;
    // the stored geometry of finest step kk, if any: a static body's after
    // its first launch, a moving body's from the geometry step (flag and
    // stamp read with acquire semantics: the entry is complete when seen)
    auto find_stored = [&](long long kk) -> const IbmCacheHead* {
        if (ip.ibm_cache == nullptr) return nullptr;
        if (still) return ld_acquire_s32(&st->ibm_cached) != 0 ? (const IbmCacheHead*)ip.ibm_cache : nullptr;
        const long long k0 = st->pose_k0, i = kk - k0;
        if (k0 < 0 || i < 0 || i + 1 >= ip.pose_n) return nullptr;
        const IbmCacheHead* e =
            (const IbmCacheHead*)((const unsigned char*)ip.ibm_cache + (size_t)i * ip.ibm_cache_stride);
        return ld_acquire_s64(&e->stamp) == kk ? e : nullptr;
    };
    // before the gate: the step counter may still be the previous step's
    // (its IBM may not have finished); the geometry loaded for it is kept
    // only if it is the one of the step found after the gate
    const long long kp = *(volatile const long long*)&st->fine_step;
    const IbmCacheHead* pre = find_stored(kp);
    if (pre != nullptr) ibm_load(pre, head, smraw, m.cache_bytes);
    if (!gate()) return;
    const long long k = st->fine_step;
    const IbmCacheHead* stored = find_stored(k);
    if (stored != nullptr) {
        if (!(stored == pre && (still || k == kp))) ibm_load(stored, head, smraw, m.cache_bytes);
    } else {
        // pose at t = k and t = k + 1 (Sec. 3.4-3.6): from the coarse step's
        // pose table, else computed here (for motions 1 and 2 with the
        // transcendental functions of the two times on different lanes)
        const long long pi0 = k - st->pose_k0;
        const bool tab =
            !still && ip.pose_tab != nullptr && st->pose_k0 >= 0 && pi0 >= 0 && pi0 + 1 < ip.pose_n;
        if (wid == 0) {
            if (tab) {
                if (lane < 8) pose[lane] = ip.pose_tab[4 * pi0 + lane];
            } else if (still) {
                if (lane == 0) {
                    pose[0] = pose[4] = ip.x0[0];
                    pose[1] = pose[5] = ip.x0[1];
                    pose[2] = pose[6] = ip.cos_mean;
                    pose[3] = pose[7] = ip.sin_mean;
                }
            } else if (ip.motion >= 3) {
                if (lane < 2) pose_at(ip, (double)(k + lane), pose + 4 * lane);
            } else {
                double v = 0.0;
                if (lane < 4) {
                    const double t = (double)(k + (lane & 1));
                    v = lane < 2 ? sin(2.0 * M_PI * t / ip.period + ip.phase) : cos(2.0 * M_PI * t / ip.period);
                }
                const double sn = __shfl_sync(0xffffffffu, v, lane & 1);
                const double cs = __shfl_sync(0xffffffffu, v, 2 + (lane & 1));
                if (lane < 2) {
                    const double al = ip.alpha_mean - ip.alpha_amp * sn;
                    const double hh = ip.motion == 2 ? 0.5 * ip.heave_amp * cs : 0.0;
                    double sa, ca;
                    sincos(al, &sa, &ca);
                    pose[4 * lane + 0] = ip.x0[0] + hh * ip.cos_beta;
                    pose[4 * lane + 1] = ip.x0[1] + hh * ip.sin_beta;
                    pose[4 * lane + 2] = ca;
                    pose[4 * lane + 3] = sa;
                }
            }
        }
        __syncthreads();
        if (!ibm_geometry<C>(P, ip, level, pose, still, m, head, bb, wtot)) return;
    }
    for (int j = tid; j < N; j += nt) F[j] = IbmV2<C>{(C)0, (C)0};
    __syncthreads();
    const int px0 = head.px0, py0 = head.py0, w = head.w, h = head.h, ncell = head.ncell;
    const bool table = head.table != 0;
    const int pnbx = head.pnbx, pbx0 = head.pbx0, pby0 = head.pby0;
    const int wh = w * h;
    const int* const ccell = m.ccell;
    const int* const cst = m.cst;
    const IbmEnt<C>* const ent = m.ent;
    const uint16_t* const cidx = m.cidx;
    const C* const wph = m.wph;
    const IbmV4<C>* const mk = m.mk;
    C* const rj = m.rj;
    IbmV2<C>* const dF = m.dF;
    IbmV4<C>* const cs = m.cs;
    C* const crho = m.crho;
    C* const cinv = m.cinv;
    // uncorrected moments of the pre-collision state on the stencil cells (Sec. 2.2 after Eq. 11)
    for (int ci = tid; ci < ncell; ci += nt) {
        const int c = ccell[ci];
        const int gx = px0 + c % w, gy = py0 + c / w;
        C r = 1, jx = 0, jy = 0;
        const int bi = table ? (gy / B - pby0) * pnbx + (gx / B - pbx0) : 0;
        if (table && pslot[bi * 9 + 4] >= 0) {
            const int x = gx % B, y = gy % B;
            r = 0;  // deviations: rho = 1 + the sum, the 1 added last (the sum keeps its low bits)
            bool ok = true;
#pragma unroll
            for (int q = 0; q < 9; q++) {
                C v;
                if (direct) {
                    v = Sto<S>::template ld<C>(fin, ((size_t)pslot[bi * 9 + 4] * 9 + q) * B * B + y * B + x, q,
                                               ip.dref);
                } else {
                    const int sx = x - CXq(q), sy = y - CYq(q);
                    const int dx = sx < 0 ? -1 : (sx >= B ? 1 : 0), dy = sy < 0 ? -1 : (sy >= B ? 1 : 0);
                    const int ns = pslot[bi * 9 + (dy + 1) * 3 + dx + 1];
                    ok &= ns >= 0;
                    v = ns >= 0 ? Sto<S>::template ld<C>(
                                      fin, ((size_t)ns * 9 + q) * B * B + (sy - dy * B) * B + (sx - dx * B), q,
                                      ip.dref)
                                : (C)0;
                }
                r += v;
                jx += (C)CXq(q) * v;
                jy += (C)CYq(q) * v;
            }
            if (DevTrait<S>::value) r += (C)1;
            if (!ok) {
                atomicOr(P.err, ERRB_STENCIL);
                r = 1;
            }
        } else if (!table) {
            const int slot = lat_slot(P, ip, level, gx, gy);
            if (slot < 0 || P.slot_type[slot] != ST_INT) {
                atomicOr(P.err, ERRB_STENCIL);
            } else {
                const int x = gx - P.slot_ox[slot], y = gy - P.slot_oy[slot];
                r = 0;
#pragma unroll
                for (int q = 0; q < 9; q++) {
                    C v = direct ? Sto<S>::template ld<C>(fin, ((size_t)slot * 9 + q) * B * B + y * B + x, q, ip.dref)
                                 : pull_int<S, C>(P, fin, nullptr, false, slot, ip, level, x, y, q);
                    r += v;
                    jx += (C)CXq(q) * v;
                    jy += (C)CYq(q) * v;
                }
                if (DevTrait<S>::value) r += (C)1;
            }
        } else {
            atomicOr(P.err, ERRB_STENCIL);
        }
        crho[ci] = r;
        cinv[ci] = (C)1 / ((C)2 * r);
        cs[ci] = IbmV4<C>{jx / r, jy / r, (C)0, (C)0};
    }
    __syncthreads();
    const C ds = (C)ip.ds;
    // K iterations: per marker Eq. 12 over its 16 cells and Eq. 11; per cell
    // Eq. 15 over its markers and the correction of Eq. 8
    const int K = ip.K;
    for (int it = 0; it < K; it++) {
        for (int j = tid; j < N; j += nt) {
            C u = 0, v = 0, r = 0;
            const IbmV4<C> wx = *(const IbmV4<C>*)(wph + 8 * j), wy = *(const IbmV4<C>*)(wph + 8 * j + 4);
            const C wxa[4] = {wx.x, wx.y, wx.z, wx.w}, wya[4] = {wy.x, wy.y, wy.z, wy.w};
            const uint4 i0 = *(const uint4*)(cidx + 16 * j), i1 = *(const uint4*)(cidx + 16 * j + 8);
            const unsigned iw[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
            for (int s16 = 0; s16 < 16; s16++) {
                const int ci = (iw[s16 >> 1] >> (16 * (s16 & 1))) & 0xffffu;
                const C d = wxa[s16 & 3] * wya[s16 >> 2];
                const IbmV2<C> cu = *(const IbmV2<C>*)(cs + ci);
                u += cu.x * d;
                v += cu.y * d;
                if (it == 0) r += crho[ci] * d;
            }
            if (it == 0) rj[j] = r;
            const C rr = it == 0 ? r : rj[j];
            const IbmV4<C> mj = mk[j];
            const C ax = (C)2 * rr * (mj.x - u);  // Eq. 11, dt = 1
            const C ay = (C)2 * rr * (mj.y - v);
            dF[j] = IbmV2<C>{ax, ay};
            IbmV2<C> fj = F[j];
            fj.x += ax;
            fj.y += ay;
            F[j] = fj;
        }
        __syncthreads();
        for (int ci = tid; ci < ncell; ci += nt) {
            C sx = 0, sy = 0;
            const int b1 = cst[ci + 1];
            for (int e = cst[ci]; e < b1; e++) {
                const IbmEnt<C> en = ent[e];
                const IbmV2<C> d = dF[en.m16 >> 4];
                sx += en.w * d.x;
                sy += en.w * d.y;
            }
            sx *= ds;  // Eq. 15
            sy *= ds;
            IbmV4<C> c = cs[ci];
            const C iv = cinv[ci];
            c.z += sx;
            c.w += sy;
            c.x += sx * iv;
            c.y += sy * iv;
            cs[ci] = c;
        }
        __syncthreads();
    }
    // the force field: zero on the box, the accumulated force on the stencil
    // cells (a static body with a stored geometry writes the same cells as the
    // launch that stored it, whose zeros the rest of the box still holds)
    C* gF = (C*)ip.patch;
    if (!(still && stored != nullptr)) {
        for (int c = tid; c < wh; c += nt) {
            gF[c] = 0;
            gF[cap + c] = 0;
        }
        __syncthreads();
    }
    for (int ci = tid; ci < ncell; ci += nt) {
        const int c = ccell[ci];
        gF[c] = cs[ci].z;
        gF[cap + c] = cs[ci].w;
    }
    // a static body keeps its geometry for the next launches
    if (still && ip.ibm_cache != nullptr && stored == nullptr)
        ibm_store((IbmCacheHead*)ip.ibm_cache, head, smraw, m.cache_bytes, -1);
    // Eq. 16 and the moment about the pivot: per-marker terms in the compute
    // type; inside the step graph they are stored and summed for the whole
    // coarse step by k_force_sum, off the critical path (FP64 runs at a small
    // fraction of the FP32 rate); the first IBM (outside the graph) sums here
    auto terms = [&](int j, C& a, C& b, C& mm) {
        const IbmV2<C> fj = F[j];
        const IbmV4<C> mj = mk[j];
        a = fj.x * ds;
        b = fj.y * ds;
        mm = (mj.z * fj.y - mj.w * fj.x) * ds;
    };
    const bool store_cache = still && ip.ibm_cache != nullptr && stored == nullptr;
    if (deferred) {
        C* out = (C*)ip.fterm + (size_t)(k % ip.fterm_n) * 3 * N;
        for (int j = tid; j < N; j += nt) {
            C a, b, mm;
            terms(j, a, b, mm);
            out[j] = a;
            out[N + j] = b;
            out[2 * N + j] = mm;
        }
        if (store_cache) __syncthreads();  // the cache writes before the flag below
    } else {
        ibm_force_sum<C>(N, terms, red, ip.hist + 3 * (k % SBOT_HIST_CAP));
    }
    if (tid == 0) {
        st->patch_x0 = px0;
        st->patch_y0 = py0;
        st->patch_w = w;
        st->patch_h = h;
        st->fine_step = k + 1;
        if (store_cache) {
            __threadfence();
            st->ibm_cached = 1;
        }
    }
}
// The force and moment of Eq. 16 for every finest step of the coarse step
// just run, one block per (body, step), from the terms k_ibm stored: the
// same FP64 sum in the same order as inside k_ibm.
template <class C>
__device__ void force_sum_run(const DevPool& P, int inst, int i, double (*red)[32]) {
    const InstParams& ip = P.inst[inst];
    const int nf = ip.fterm_n, N = ip.n_markers;
    if (i >= nf) return;
    const long long k = P.ist[inst].fine_step - nf + i;  // the steps of this coarse step
    if (k < 0) return;
    const C* in = (const C*)ip.fterm + (size_t)(k % nf) * 3 * N;
    auto terms = [&](int j, C& a, C& b, C& mm) {
        a = in[j];
        b = in[N + j];
        mm = in[2 * N + j];
    };
    ibm_force_sum<C>(N, terms, red, ip.hist + 3 * (k % SBOT_HIST_CAP));
}
}  // namespace
