/*
 * sbot_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the
 * lattice-Boltzmann / immersed-boundary / block-refinement method of
 * Nguyen & Duong, "SBoTFlow" (arXiv 2402.04606).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two agree only because
 * both follow the paper.
 *
 * Representation (deliberately unlike the GPU library): every refinement
 * level l is one DENSE array covering the whole domain at that level's
 * resolution, with a per-cell type map telling which cells take part.
 * Loops are plain per-cell loops in the order the paper states the steps.
 *
 * Paper passages followed (section / equation / algorithm of the paper):
 *   lattice D2Q9 ........................ Sec. 2.1, Eq. 1
 *   BGK collision with forcing .......... Sec. 2.1, Eq. 2 and Eq. 6
 *   Guo forcing term .................... Sec. 2.1, Eq. 3 (moment conditions Eqs. 4-5)
 *   equilibrium ......................... Sec. 2.1, Eq. 7
 *   moments with half-force shift ....... Sec. 2.1, Eq. 8
 *   viscosity / relaxation time ......... Sec. 2.1, Eq. 9
 *   streaming ........................... Sec. 2.1, Eq. 10
 *   IBM: desired velocity, boundary force Sec. 2.2, Eq. 11
 *   IBM: interpolation, delta, kernel ... Sec. 2.2, Eqs. 12-14
 *   IBM: spreading, body force .......... Sec. 2.2, Eqs. 15-16
 *   MRT collision option ................ Sec. 2.1 after Eq. 9 (reading R14)
 *   walls and solids, bounce-back ....... Sec. 2.1 after Eq. 10 (reading R15)
 *   LES (Smagorinsky) option ............ Sec. 2.1 after Eq. 9 (reading R16)
 *   multi-direct forcing (iteration) .... Sec. 1 (Breugem's scheme, named only)
 *   block refinement, 2:1 balance ....... Sec. 2.3, Sec. 2.4
 *   coarse/fine interface steps (1)-(6) . Sec. 2.4, Fig. 3 description
 *   recursive sub-cycled time step ...... Algorithm 1
 *   pitch-up ramp kinematics ............ Sec. 3.4, Eqs. 20-21
 *   asymmetric triangular pitching ...... Sec. 3.5, Eqs. 22-24
 *   flapping kinematics ................. Sec. 3.6, Eqs. 25-27
 *
 * Readings where the paper is silent or ambiguous:
 *   R1 tau per level: acoustic scaling, tau_l = 1/2 + (tau_finest - 1/2) / 2^(m-1-l).
 *   R2 domain boundaries: periodic = wrap; equilibrium inlet = the boundary
 *      column is reset to f^eq(rho0, u_in) after streaming; open outlet =
 *      unknown populations copied from the neighbouring interior cell
 *      (zero gradient); symmetry = half-way specular mirror (the virtual cell
 *      beyond the wall is the boundary cell with the normal velocity
 *      component reflected).  At a corner the y-side rule is applied first,
 *      then the x-side rule.
 *   R3 coarse/fine interface (Sec. 2.4 steps (1)-(6) and Algorithm 1), fine
 *      side: 2 halo layers of fine cells inside the coarser leaf; C2F copies
 *      the coarse post-collision populations of the containing coarse cell
 *      into every fine halo cell (piecewise constant); fine streaming also
 *      updates halo cells, which pull where a source exists and otherwise
 *      keep their value; halo cells are never collided (PreStreamingStep
 *      keeps them).
 *   R3c coarse side (default, the volumetric scheme of Rohde et al. that the
 *      paper adopts): F2C merges the two fine halo layers into the coarse
 *      grid -- every coarse interior population whose streaming source lies
 *      in the finer region is set to the mean of that population over the
 *      4 fine halo cells inside the coarse cell.  No rescaling.
 *   R3a coarse side, alternative (iface = 0): one coarse ghost layer inside
 *      the finer region holds the mean of the 4 fine post-stream cells, is
 *      collided with the coarse tau and is pulled by the coarse interior.
 *      Kept only as the documented alternative: it does not converge for
 *      diffusion-dominated flow (the tests show it).
 *   R3b interface rescaling (option for R3a, off by default): the non-equilibrium
 *      part f - f^eq is rescaled when populations change level (Dupuis and
 *      Chopard), so the viscous stress is continuous across the interface:
 *      coarse post-collision -> fine ghost: x (tau_f - 1) / (2 (tau_c - 1));
 *      mean of fine post-stream -> coarse ghost: x 2 tau_c / tau_f.
 *      Not used with R3c, whose volumetric transfer needs none.
 *   R4 IBM: runs only on the finest level; rho in Eq. 11 is the
 *      interpolated density; Delta s_b = perimeter / N; the desired velocity
 *      is the forward difference of marker positions over one finest step;
 *      the multi-direct-forcing loop repeats K times: interpolate, force
 *      increment, spread, correct the velocity (u += dF / 2 rho).
 *   R5 re-tagging (moving refinement) is not in the paper: evaluated once
 *      per coarse step, on the post-collision state; a new cell keeps its
 *      value if it existed at the same level, else copies the covering
 *      coarser cell, else averages its 4 children (recursively).
 *   R10 pitch-up ramp (Eqs. 20-21): the maximum of G is taken as its supremum
 *      2 a_s (t2* - t1*), the value G reaches after the ramp; log cosh is
 *      evaluated as |x| + log1p(exp(-2|x|)) - log 2 (the same number without
 *      overflow); t* = t / t_ref, t_ref = c / U in finest steps; the body
 *      angle is alpha_mean - alpha(t), about a pivot at the leading edge.
 *   R11 asymmetric triangular pitch (Eqs. 22-24, printed garbled): peak
 *      +alpha_0 at t2 = xi T / 2, trough -alpha_0 at t5 = T - xi T / 2, each
 *      corner smoothed over t_a = 0.15 T on both sides (t1 = t2 - t_a,
 *      t3 = t2 + t_a, t4 = t5 - t_a, t6 = t5 + t_a); every quartic has
 *      2 t_a^3 in its first denominator, which makes the angle C2 and
 *      periodic (the printed 2 t_2^3 breaks continuity); pivot at the
 *      quarter chord.
 *   R12 body shapes (Secs. 3.4-3.5): the flat plate is a rectangle with
 *      markers at exact equal arc length from (a, 0) counter-clockwise; the
 *      NACA 0018 section uses the four-digit half-thickness polynomial with
 *      the closed-trailing-edge last coefficient, markers at equal arc length
 *      along x = a cos(theta) as for the ellipse.
 *   R14 MRT (named with a citation only): the D2Q9 moment basis of Lallemand
 *      and Luo (rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy); equilibrium
 *      moments M f^eq of Eq. 7; Guo forcing in moment space (I - S/2) M Fbar,
 *      Fbar = Eq. 3 without its prefactor; the stress moments relax at
 *      1/tau_l (the viscosity of Eq. 9), e, epsilon and q at fixed rates.
 *      With every rate 1/tau it is the BGK collision of Eq. 6.
 *   R15 walls and solids (interpolated bounce-back, formulas left to the
 *      cited work): a wall side is half-way bounce-back,
 *      f_i(x) = f*_opp(i)(x) + 2 w_i rho0 (c_i . u_w) / c_s^2; a solid
 *      (circle or half-plane) on the finest level makes the cells whose
 *      centres lie inside it solid, and a population whose source is solid
 *      takes the linear interpolation of Bouzidi, Firdaouss and Lallemand at
 *      the exact link fraction t: 2t f*_opp(x) + (1 - 2t) f*_opp(x + c_i) for
 *      t < 1/2, else f*_opp(x) / 2t + (1 - 1/2t) f*_i(x).
 *   R16 LES (named with a citation only): Smagorinsky, BGK with forcing at
 *      tau_e = tau_l + 3 nu_t, nu_t = C_s^2 |S| in the level's own units,
 *      |S| from the non-equilibrium stress Pi = sum c c (f - f^eq) with
 *      Q = sqrt(2 Pi:Pi), so tau_e = (tau_l + sqrt(tau_l^2 + 18 C_s^2 Q / rho)) / 2.
 *
 * Pins (tests/test_oracle_*.py, run without a GPU): moment identities of
 * Eq. 7 and Eqs. 3-5, conservation, streaming shifts, boundary fixed points,
 * the Taylor-Green decay and its second order at the parameters of
 * Sec. 3.1, the kernel's closed forms and discrete moments, IBM against
 * brute-force loops and the closed-form multi-direct-forcing contraction,
 * Eq. 16's force and moment by the fluid's momentum and angular momentum,
 * refinement fixed points, bitwise equality of a fully refined run, interface
 * convergence orders, re-tag round trips, the four motions (Eqs. 20-27:
 * ramp, triangle, sinusoidal pitch, pitch plus tilted-stroke heave) and
 * the shapes against closed forms and their properties,
 * MRT and LES reductions and decay rates, exact Couette flow with walls.
 * The cylinder's force statistics are held to the values of Table 1 on the
 * GPU path, which the parity tests hold to this oracle.
 * Parity unpinned: the force values of the wing, plate, NACA and cavity
 * cases (the paper prints no values for them); there the oracle is checked
 * only through the pins of its parts and its agreement with the GPU path.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define NQ 9
#define MAXLEV 8

/* Sec. 2.1, Eq. 1: discrete velocities in the paper's order. */
static const int CX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Sec. 2.1, text after Eq. 7: weights. */
static const double WQ[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s = 1/sqrt(3) */

enum { T_NONE = 0, T_INT = 1, T_GF = 2, T_GC = 3, T_SOLID = 4 };
enum { BC_PERIODIC = 0, BC_INLET = 1, BC_OUTLET = 2, BC_SYMMETRY = 3, BC_WALL = 4 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

/* direction with the x (resp. y) component of c reversed */
static int flip_x(int i) {
    for (int k = 0; k < NQ; k++)
        if (CX[k] == -CX[i] && CY[k] == CY[i]) return k;
    return -1;
}
static int flip_y(int i) {
    for (int k = 0; k < NQ; k++)
        if (CX[k] == CX[i] && CY[k] == -CY[i]) return k;
    return -1;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1 single-cell formulas                                       */
/* ------------------------------------------------------------------ */

/* Eq. 7 */
double orc_feq(int i, double rho, double ux, double uy) {
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WQ[i] * rho * (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 3 */
double orc_guo(int i, double tau, double ux, double uy, double Fx, double Fy) {
    double cF = CX[i] * Fx + CY[i] * Fy;
    double cu = CX[i] * ux + CY[i] * uy;
    double uF = ux * Fx + uy * Fy;
    return WQ[i] * (1.0 - 1.0 / (2.0 * tau)) * (cF / CS2 + cu * cF / (CS2 * CS2) - uF / CS2);
}

/* Eq. 8, then Eq. 6 on one cell.  f: 9 pre-collision values, fs: 9 outputs. */
void orc_collide_cell(const double* f, double tau, double Fx, double Fy, double* fs) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NQ; i++) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double ux = jx / rho + Fx / (2.0 * rho);
    double uy = jy / rho + Fy / (2.0 * rho);
    for (int i = 0; i < NQ; i++) {
        double feq = orc_feq(i, rho, ux, uy);
        fs[i] = f[i] - (f[i] - feq) / tau + orc_guo(i, tau, ux, uy, Fx, Fy);
    }
}

/* Multiple-relaxation-time collision (the MRT option of Sec. 2.1, citing Du
 * et al.; reading R14): the D2Q9 moment basis of Lallemand and Luo, each row
 * a polynomial in the lattice velocity c_i,
 *   rho: 1, e: -4 + 3|c|^2, eps: 4 - 21/2 |c|^2 + 9/2 |c|^4, j_x: c_x,
 *   q_x: (-5 + 3|c|^2) c_x, j_y: c_y, q_y: (-5 + 3|c|^2) c_y,
 *   p_xx: c_x^2 - c_y^2, p_xy: c_x c_y,
 * written row by row into M[9][9].  Its rows are orthogonal, so
 * M^-1 = M^T diag(1 / |row|^2). */
void orc_mrt_matrix(double* M) {
    for (int i = 0; i < NQ; i++) {
        double cx = CX[i], cy = CY[i], c2 = cx * cx + cy * cy;
        M[0 * NQ + i] = 1.0;
        M[1 * NQ + i] = -4.0 + 3.0 * c2;
        M[2 * NQ + i] = 4.0 - 10.5 * c2 + 4.5 * c2 * c2;
        M[3 * NQ + i] = cx;
        M[4 * NQ + i] = (-5.0 + 3.0 * c2) * cx;
        M[5 * NQ + i] = cy;
        M[6 * NQ + i] = (-5.0 + 3.0 * c2) * cy;
        M[7 * NQ + i] = cx * cx - cy * cy;
        M[8 * NQ + i] = cx * cy;
    }
}

/* MRT collision with Guo forcing in moment space, on one cell:
 *   m = M f, m_eq = M f^eq(rho, u) (Eq. 7 with Eq. 8's u),
 *   Fb_i = w_i (3 (c_i - u) + 9 (c_i . u) c_i) . F   (Eq. 3 without its factor),
 *   m* = m - S (m - m_eq) + (I - S / 2) M Fb,   f* = M^-1 m*,
 * S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, s_nu, s_nu), s_nu = 1 / tau (the
 * viscosity of Eq. 9), s3 = {s_e, s_eps, s_q}.  With every rate 1 / tau this
 * is the BGK collision of Eq. 6 with Eq. 3. */
void orc_collide_cell_mrt(const double* f, double tau, const double* s3, double Fx, double Fy, double* fs) {
    double M[NQ * NQ];
    orc_mrt_matrix(M);
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NQ; i++) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double ux = jx / rho + Fx / (2.0 * rho);
    double uy = jy / rho + Fy / (2.0 * rho);
    double feq[NQ], Fb[NQ];
    for (int i = 0; i < NQ; i++) {
        feq[i] = orc_feq(i, rho, ux, uy);
        double cu = CX[i] * ux + CY[i] * uy;
        Fb[i] = WQ[i] * (3.0 * ((CX[i] - ux) * Fx + (CY[i] - uy) * Fy) + 9.0 * cu * (CX[i] * Fx + CY[i] * Fy));
    }
    double S[NQ] = {0.0, s3[0], s3[1], 0.0, s3[2], 0.0, s3[2], 1.0 / tau, 1.0 / tau};
    double ms[NQ];
    for (int k = 0; k < NQ; k++) {
        double m = 0.0, me = 0.0, mf = 0.0;
        for (int i = 0; i < NQ; i++) {
            m += M[k * NQ + i] * f[i];
            me += M[k * NQ + i] * feq[i];
            mf += M[k * NQ + i] * Fb[i];
        }
        ms[k] = m - S[k] * (m - me) + (1.0 - 0.5 * S[k]) * mf;
    }
    for (int i = 0; i < NQ; i++) {
        double v = 0.0;
        for (int k = 0; k < NQ; k++) {
            double nk = 0.0;
            for (int j = 0; j < NQ; j++) nk += M[k * NQ + j] * M[k * NQ + j];
            v += M[k * NQ + i] * ms[k] / nk;
        }
        fs[i] = v;
    }
}

/* Large-eddy option (the LES of Sec. 2.1 after Eq. 9; reading R16): BGK
 * (Eq. 6 with Eq. 3) at a local relaxation time tau_e = tau + 3 nu_t, the
 * Smagorinsky eddy viscosity nu_t = (C_s Delta)^2 |S| in the units of the
 * level (Delta = 1), with the strain rate read from the non-equilibrium
 * stress Pi_ab = sum_i c_ia c_ib (f_i - f^eq_i): |S| = 3 Q / (2 rho tau_e),
 * Q = sqrt(2 Pi_ab Pi_ab).  The two relations give the positive root of
 * tau_e^2 - tau tau_e - 9 C_s^2 Q / (2 rho) = 0. */
double orc_les_tau(const double* f, double tau, double cs, double Fx, double Fy) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NQ; i++) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double ux = jx / rho + Fx / (2.0 * rho);
    double uy = jy / rho + Fy / (2.0 * rho);
    double pxx = 0.0, pyy = 0.0, pxy = 0.0;
    for (int i = 0; i < NQ; i++) {
        double ne = f[i] - orc_feq(i, rho, ux, uy);
        pxx += CX[i] * CX[i] * ne;
        pyy += CY[i] * CY[i] * ne;
        pxy += CX[i] * CY[i] * ne;
    }
    double Q = sqrt(2.0 * (pxx * pxx + pyy * pyy + 2.0 * pxy * pxy));
    return 0.5 * (tau + sqrt(tau * tau + 18.0 * cs * cs * Q / rho));
}

void orc_collide_cell_les(const double* f, double tau, double cs, double Fx, double Fy, double* fs) {
    orc_collide_cell(f, orc_les_tau(f, tau, cs, Fx, Fy), Fx, Fy, fs);
}

/* f^eq(rho, u) + beta (f - f^eq(rho, u)), rho and u the moments of f (Eq. 8, F = 0) */
void orc_rescale_neq(const double* f, double beta, double* out) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NQ; i++) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double ux = jx / rho, uy = jy / rho;
    for (int i = 0; i < NQ; i++) {
        double feq = orc_feq(i, rho, ux, uy);
        out[i] = feq + beta * (f[i] - feq);
    }
}

/* Eq. 14: Peskin's 4-point kernel, r in lattice units (Delta x = 1). */
double orc_phi(double r) {
    double a = fabs(r);
    if (a <= 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
    if (a <= 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: the multi-direct-forcing IBM operator on one dense grid.  */
/* ------------------------------------------------------------------ */

/* Cell (i, j) of the grid has its centre at (i + 1/2, j + 1/2).  The 4 cells
 * of the stencil of a marker at x = r are i0 .. i0+3, i0 = floor(r - 1/2) - 1,
 * which are exactly the cells with |i + 1/2 - r| <= 2 (support of Eq. 14). */
static int stencil_origin(double r) { return (int)floor(r - 0.5) - 1; }

/*
 * Multi-direct forcing on a dense nx * ny grid (reading R4):
 *   F_x = 0, F_j = 0;
 *   repeat K times:
 *     u_j   = sum_x u_x D(x - r_j) dx^2,  rho_j likewise     (Eq. 12, Eq. 13)
 *     dF_j  = 2 rho_j (u^d_j - u_j) / dt                       (Eq. 11)
 *     dF_x  = sum_j dF_j D(x - r_j) ds_j                        (Eq. 15)
 *     u_x  += dF_x / (2 rho_x);  F_x += dF_x;  F_j += dF_j
 * ux, uy enter as the uncorrected velocity and leave corrected.
 * Returns 0, or -1 when a stencil leaves the grid.
 */
int orc_ibm_mdf(int nx, int ny, const double* rho, double* ux, double* uy, int n,
                const double* rx, const double* ry, const double* udx, const double* udy,
                const double* ds, int K, double* Fx, double* Fy, double* Fjx, double* Fjy) {
    size_t ncell = (size_t)nx * ny;
    double* dFx = (double*)calloc(ncell, sizeof(double));
    double* dFy = (double*)calloc(ncell, sizeof(double));
    double* dFjx = (double*)calloc((size_t)n, sizeof(double));
    double* dFjy = (double*)calloc((size_t)n, sizeof(double));
    int rc = 0;
    for (size_t c = 0; c < ncell; c++) Fx[c] = Fy[c] = 0.0;
    for (int j = 0; j < n; j++) Fjx[j] = Fjy[j] = 0.0;
    for (int j = 0; j < n; j++) {
        int i0 = stencil_origin(rx[j]), j0 = stencil_origin(ry[j]);
        if (i0 < 0 || j0 < 0 || i0 + 3 >= nx || j0 + 3 >= ny) rc = -1;
    }
    if (rc != 0) goto done;
    for (int k = 0; k < K; k++) {
        /* interpolation of the current (partly corrected) velocity, Eq. 12 */
        for (int j = 0; j < n; j++) {
            int i0 = stencil_origin(rx[j]), j0 = stencil_origin(ry[j]);
            double uj = 0.0, vj = 0.0, rj = 0.0;
            for (int b = 0; b < 4; b++) {
                for (int a = 0; a < 4; a++) {
                    int ci = i0 + a, cj = j0 + b;
                    double d = orc_phi(ci + 0.5 - rx[j]) * orc_phi(cj + 0.5 - ry[j]);
                    size_t c = (size_t)cj * nx + ci;
                    uj += ux[c] * d;
                    vj += uy[c] * d;
                    rj += rho[c] * d;
                }
            }
            /* Eq. 11 with dt = 1 */
            dFjx[j] = 2.0 * rj * (udx[j] - uj);
            dFjy[j] = 2.0 * rj * (udy[j] - vj);
        }
        /* spreading, Eq. 15 */
        for (size_t c = 0; c < ncell; c++) dFx[c] = dFy[c] = 0.0;
        for (int j = 0; j < n; j++) {
            int i0 = stencil_origin(rx[j]), j0 = stencil_origin(ry[j]);
            for (int b = 0; b < 4; b++) {
                for (int a = 0; a < 4; a++) {
                    int ci = i0 + a, cj = j0 + b;
                    double d = orc_phi(ci + 0.5 - rx[j]) * orc_phi(cj + 0.5 - ry[j]);
                    size_t c = (size_t)cj * nx + ci;
                    dFx[c] += dFjx[j] * d * ds[j];
                    dFy[c] += dFjy[j] * d * ds[j];
                }
            }
        }
        /* velocity correction (half-force shift of Eq. 8) and accumulation */
        for (size_t c = 0; c < ncell; c++) {
            if (dFx[c] == 0.0 && dFy[c] == 0.0) continue;
            ux[c] += dFx[c] / (2.0 * rho[c]);
            uy[c] += dFy[c] / (2.0 * rho[c]);
            Fx[c] += dFx[c];
            Fy[c] += dFy[c];
        }
        for (int j = 0; j < n; j++) {
            Fjx[j] += dFjx[j];
            Fjy[j] += dFjy[j];
        }
    }
done:
    free(dFx);
    free(dFy);
    free(dFjx);
    free(dFjy);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Body geometry and kinematics                                        */
/* ------------------------------------------------------------------ */

/* Markers at equal arc length on an ellipse x = a cos(t), y = b sin(t):
 * the perimeter is the length of the M-gon through t_k = 2 pi k / M,
 * M = 64 n; marker j sits at arc length j * P / n, found by linear
 * interpolation of t inside the polygon segment containing it.  A circle
 * (a == b) gives t_j = 2 pi j / n exactly.  Returns P. */
double orc_place_markers(double a, double b, int n, double* qx, double* qy) {
    if (a == b) {
        for (int j = 0; j < n; j++) {
            double t = 2.0 * M_PI * (double)j / (double)n;
            qx[j] = a * cos(t);
            qy[j] = a * sin(t);
        }
        return 2.0 * M_PI * a;
    }
    int M = 64 * n;
    double* s = (double*)malloc((size_t)(M + 1) * sizeof(double));
    s[0] = 0.0;
    for (int k = 0; k < M; k++) {
        double t0 = 2.0 * M_PI * (double)k / (double)M;
        double t1 = 2.0 * M_PI * (double)(k + 1) / (double)M;
        double dx = a * cos(t1) - a * cos(t0), dy = b * sin(t1) - b * sin(t0);
        s[k + 1] = s[k] + sqrt(dx * dx + dy * dy);
    }
    double P = s[M];
    int k = 0;
    for (int j = 0; j < n; j++) {
        double target = P * (double)j / (double)n;
        while (k < M - 1 && s[k + 1] <= target) k++;
        double frac = (target - s[k]) / (s[k + 1] - s[k]);
        double t = 2.0 * M_PI * ((double)k + frac) / (double)M;
        qx[j] = a * cos(t);
        qy[j] = b * sin(t);
    }
    free(s);
    return P;
}

/* Markers at equal arc length on a rectangle (a flat plate with square
 * edges, Sec. 3.4) of half-sides a (x) and b (y): the perimeter 4a + 4b is
 * walked counter-clockwise from (a, 0).  Exact; returns the perimeter. */
static double place_rectangle(double a, double b, int n, double* qx, double* qy) {
    double P = 4.0 * a + 4.0 * b;
    for (int j = 0; j < n; j++) {
        double s = P * (double)j / (double)n;
        double x, y;
        if (s < b) {
            x = a, y = s;
        } else if (s < b + 2.0 * a) {
            x = a - (s - b), y = b;
        } else if (s < 3.0 * b + 2.0 * a) {
            x = -a, y = b - (s - b - 2.0 * a);
        } else if (s < 3.0 * b + 4.0 * a) {
            x = -a + (s - 3.0 * b - 2.0 * a), y = -b;
        } else {
            x = a, y = -b + (s - 3.0 * b - 4.0 * a);
        }
        qx[j] = x;
        qy[j] = y;
    }
    return P;
}

/* Half-thickness of a symmetric NACA four-digit section (the airfoil of
 * Sec. 3.5) at chordwise position xc in [0, 1], thickness ratio t, chord 1,
 * with the closed-trailing-edge last coefficient (reading R12). */
static double naca_half_thickness(double t, double xc) {
    return 5.0 * t * (0.2969 * sqrt(xc) - 0.1260 * xc - 0.3516 * xc * xc + 0.2843 * xc * xc * xc -
                      0.1036 * xc * xc * xc * xc);
}

/* Markers at equal arc length on that airfoil, chord 2a along x from the
 * leading edge at -a to the trailing edge at +a, maximum half-thickness
 * about b (thickness ratio b / a).  The curve is x = a cos(th),
 * y = +-y_t((1 + cos th) / 2) (upper surface for 0 < th < pi), and the
 * markers are placed on its M-gon, M = 64 n, through th_k = 2 pi k / M as
 * for the ellipse.  Returns the polygon's perimeter. */
static double place_naca(double a, double b, int n, double* qx, double* qy) {
    const double t = b / a, c = 2.0 * a;
    int M = 64 * n;
    double* s = (double*)malloc((size_t)(M + 1) * sizeof(double));
    double px = a, py = 0.0;
    s[0] = 0.0;
    for (int k = 0; k < M; k++) {
        double th = 2.0 * M_PI * (double)(k + 1) / (double)M;
        double x = a * cos(th);
        double yt = c * naca_half_thickness(t, 0.5 * (1.0 + cos(th)));
        double y = sin(th) >= 0.0 ? yt : -yt;
        if (k + 1 == M) x = a, y = 0.0;
        s[k + 1] = s[k] + sqrt((x - px) * (x - px) + (y - py) * (y - py));
        px = x, py = y;
    }
    double P = s[M];
    int k = 0;
    for (int j = 0; j < n; j++) {
        double target = P * (double)j / (double)n;
        while (k < M - 1 && s[k + 1] <= target) k++;
        double frac = (target - s[k]) / (s[k + 1] - s[k]);
        double th = 2.0 * M_PI * ((double)k + frac) / (double)M;
        double yt = c * naca_half_thickness(t, 0.5 * (1.0 + cos(th)));
        qx[j] = a * cos(th);
        qy[j] = sin(th) >= 0.0 ? yt : -yt;
    }
    free(s);
    return P;
}

/* Markers of a body of the given kind: 0 circle, 1 ellipse, 2 rectangle
 * (flat plate), 3 symmetric NACA four-digit airfoil. */
double orc_place_markers_kind(int kind, double a, double b, int n, double* qx, double* qy) {
    if (kind == 2) return place_rectangle(a, b, n, qx, qy);
    if (kind == 3) return place_naca(a, b, n, qx, qy);
    return orc_place_markers(a, kind == 0 ? a : b, n, qx, qy);
}

/* log cosh x written as |x| + log(1 + e^(-2|x|)) - log 2, the same number
 * without the overflow of cosh at large |x| */
static double log_cosh(double x) {
    double ax = fabs(x);
    return ax + log1p(exp(-2.0 * ax)) - log(2.0);
}

/* Sec. 3.4, Eqs. 20-21: pitch angle of the smoothed pitch-up ramp at
 * nondimensional time ts (t U / c),
 *   G(ts) = log[cosh(a_s (ts - t1)) / cosh(a_s (ts - t2))] - a_s (t1 - t2),
 *   t2 = t1 + A / (2 K),   alpha = A G / max G,
 * with max G taken as its supremum 2 a_s (t2 - t1), the value G tends to
 * after the ramp (reading R10). */
double orc_ramp_alpha(double A, double as, double K, double t1, double ts) {
    double t2 = t1 + A / (2.0 * K);
    double G = log_cosh(as * (ts - t1)) - log_cosh(as * (ts - t2)) - as * (t1 - t2);
    double Gmax = 2.0 * as * (t2 - t1);
    return A * G / Gmax;
}

/* Sec. 3.5, Eqs. 22-24: the smoothed asymmetric triangular pitch of
 * amplitude a0, period T, asymmetry xi and corner time t_a = acc T, at time t
 * (reduced to [0, T)).  Reading R11 of the garbled printed form: the peak is
 * at t2 = xi T / 2 and the trough at t5 = T - xi T / 2, each corner is
 * smoothed over t_a on both sides (t1 = t2 - t_a, t3 = t2 + t_a,
 * t4 = t5 - t_a, t6 = t5 + t_a), and the quartic pieces all carry 2 t_a^3
 * in their first denominator (the printed 2 t_2^3 of two of them would break
 * the continuity with the linear pieces). */
double orc_triangle_alpha(double a0, double xi, double acc, double T, double t) {
    double tt = t - T * floor(t / T);
    double ta = acc * T;
    double ad1 = 2.0 * a0 / (xi * T - ta);          /* Eq. 23 */
    double ad2 = -2.0 * a0 / ((1.0 - xi) * T - ta); /* Eq. 24 */
    double t2 = 0.5 * xi * T, t5 = T - 0.5 * xi * T;
    double t1 = t2 - ta, t3 = t2 + ta, t4 = t5 - ta, t6 = t5 + ta;
    double ta2 = ta * ta, ta3 = ta2 * ta;
    if (tt < t1) return ad1 * tt;
    if (tt < t2) {
        double u = tt - t2;
        return ad1 / (2.0 * ta3) * u * u * u * u + ad1 / ta2 * u * u * u + a0;
    }
    if (tt < t3) {
        double u = tt - t2;
        return -ad2 / (2.0 * ta3) * u * u * u * u + ad2 / ta2 * u * u * u + a0;
    }
    if (tt < t4) return ad2 * (tt - t4) - ad2 * ta / 2.0 - a0;
    if (tt < t5) {
        double u = tt - t5;
        return ad2 / (2.0 * ta3) * u * u * u * u + ad2 / ta2 * u * u * u - a0;
    }
    if (tt < t6) {
        double u = tt - t5;
        return -ad1 / (2.0 * ta3) * u * u * u * u + ad1 / ta2 * u * u * u - a0;
    }
    return ad1 * (tt - T);
}

typedef struct {
    int present;
    int n;
    double* qx; /* body-frame marker coordinates (relative to the body centre) */
    double* qy;
    double ds; /* Delta s_b = perimeter / n (reading R4) */
    double pivot[2];
    int motion; /* 0 static, 1 pitching, 2 flapping (pitch + heave), 3 pitch-up ramp, 4 triangular pitching */
    double x0[2], alpha_mean, alpha_amp, period, phase, heave_amp, beta;
    double ramp_as, ramp_rate, ramp_t1, t_ref; /* motion 3: a_s, K, t1*, finest steps per unit of t* */
    double xi, acc;                            /* motion 4: asymmetry and corner time / T */
    int K;
    double* hist; /* (Fx, Fy, Mz) per finest step, Eq. 16 and its moment */
    long hist_n, hist_cap;
} Body;

/* Sec. 3.6, Eqs. 25-27, with time in finest steps and the pitch amplitude a
 * parameter (the paper's value is pi/4):
 *   alpha(t) = alpha_mean - alpha_amp sin(2 pi t / T + phase)
 *   x_c(t)   = (A0 / 2) cos(2 pi t / T) cos(beta),  y_c likewise with sin(beta)
 * The body is rotated by alpha about its pivot (body frame), the centre is
 * x0 + (x_c, y_c).  motion 0 keeps alpha = alpha_mean, motion 1 omits the heave.
 * motion 3 (Sec. 3.4) and motion 4 (Sec. 3.5) turn the body by
 * alpha_mean - alpha_pitch(t) about the fixed centre, alpha_pitch from
 * orc_ramp_alpha at t / t_ref, or from orc_triangle_alpha at
 * t + phase T / (2 pi). */
static void body_pose(const Body* bd, double t, double* cx, double* cy, double* alpha) {
    double al = bd->alpha_mean, hx = 0.0, hy = 0.0;
    if (bd->motion == 1 || bd->motion == 2)
        al = bd->alpha_mean - bd->alpha_amp * sin(2.0 * M_PI * t / bd->period + bd->phase);
    if (bd->motion == 3)
        al = bd->alpha_mean - orc_ramp_alpha(bd->alpha_amp, bd->ramp_as, bd->ramp_rate, bd->ramp_t1, t / bd->t_ref);
    if (bd->motion == 4)
        al = bd->alpha_mean - orc_triangle_alpha(bd->alpha_amp, bd->xi, bd->acc, bd->period,
                                                 t + bd->phase * bd->period / (2.0 * M_PI));
    if (bd->motion == 2) {
        double h = 0.5 * bd->heave_amp * cos(2.0 * M_PI * t / bd->period);
        hx = h * cos(bd->beta);
        hy = h * sin(bd->beta);
    }
    *cx = bd->x0[0] + hx;
    *cy = bd->x0[1] + hy;
    *alpha = al;
}

static void marker_positions(const Body* bd, double t, double* rx, double* ry) {
    double cx, cy, al;
    body_pose(bd, t, &cx, &cy, &al);
    double c = cos(al), s = sin(al);
    for (int j = 0; j < bd->n; j++) {
        double px = bd->qx[j] - bd->pivot[0], py = bd->qy[j] - bd->pivot[1];
        rx[j] = cx + bd->pivot[0] + c * px - s * py;
        ry[j] = cy + bd->pivot[1] + s * px + c * py;
    }
}

/* ------------------------------------------------------------------ */
/* Domain                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny;   /* cells of this level over the whole domain */
    int nbx, nby; /* block lattice of this level */
    int h;        /* cell size in finest units */
    double tau;
    unsigned char* bstate; /* [nby*nbx] 0 absent (inside a coarser leaf), 1 leaf, 2 refined */
    unsigned char* type;   /* [ny*nx] T_NONE / T_INT / T_GF / T_GC */
    double* f;             /* [9][ny][nx] post-stream (pre-collision) values */
    double* fs;            /* [9][ny][nx] post-collision values */
    double* tmp;           /* [9][ny][nx] streaming target */
    double* Fx;            /* [ny*nx] body force density (finest level only) */
    double* Fy;
} Lev;

typedef struct {
    int m, B, nx0, ny0;
    int bc[4];
    double tau_f, rho0, uin[2];
    Lev lev[MAXLEV];
    Body body;
    long fine_step;   /* number of finest-level collisions performed */
    long coarse_step; /* number of completed coarse steps */
    int retag, retag_pending;
    int rescale; /* reading R3b */
    int coll;    /* 0 BGK (Eq. 6), 1 MRT (reading R14), 2 LES (reading R16; C_s in mrt_s[0]) */
    double mrt_s[3];
    double uwall[4][2]; /* BC_WALL sides: wall velocity (reading R15) */
    int solid;          /* solid obstacle on the finest level: 0 none, 1 circle, 2 half-plane y < y0 */
    double sol[3];      /* circle: centre x, y, radius; half-plane: y0 (finest units) */
    int iface;   /* 0: overlapping coarse ghost layer (R3); 1: volumetric coalescence (R3c) */
    double margin[MAXLEV], wake[MAXLEV];
    int nbox;
    double* boxes; /* nbox * 5: level, x0, y0, x1, y1 (finest units) */
    int err;
    char msg[256];
} Dom;

#define IDX(L, x, y) ((size_t)(y) * (size_t)(L)->nx + (size_t)(x))
#define FQ(L, arr, i, x, y) ((L)->arr[(size_t)(i) * (size_t)(L)->nx * (size_t)(L)->ny + IDX(L, x, y)])

static void set_err(Dom* d, const char* m) {
    if (!d->err) {
        d->err = 1;
        snprintf(d->msg, sizeof d->msg, "%s", m);
    }
}

static int periodic_x(const Dom* d) { return d->bc[SIDE_W] == BC_PERIODIC; }
static int periodic_y(const Dom* d) { return d->bc[SIDE_S] == BC_PERIODIC; }

Dom* orc_create(int nx0, int ny0, int levels, int block, const int* bc, double tau_finest, double rho0,
                double uin_x, double uin_y) {
    if (levels < 1 || levels > MAXLEV || block < 2 || nx0 % block || ny0 % block) return NULL;
    if ((bc[SIDE_W] == BC_PERIODIC) != (bc[SIDE_E] == BC_PERIODIC)) return NULL;
    if ((bc[SIDE_S] == BC_PERIODIC) != (bc[SIDE_N] == BC_PERIODIC)) return NULL;
    Dom* d = (Dom*)calloc(1, sizeof(Dom));
    d->m = levels;
    d->B = block;
    d->nx0 = nx0;
    d->ny0 = ny0;
    for (int s = 0; s < 4; s++) d->bc[s] = bc[s];
    d->tau_f = tau_finest;
    d->rho0 = rho0;
    d->uin[0] = uin_x;
    d->uin[1] = uin_y;
    d->rescale = 0;
    d->iface = 1;
    for (int l = 0; l < levels; l++) {
        Lev* L = &d->lev[l];
        L->nx = nx0 << l;
        L->ny = ny0 << l;
        L->nbx = L->nx / block;
        L->nby = L->ny / block;
        L->h = 1 << (levels - 1 - l);
        /* reading R1 (acoustic scaling): nu_l = nu_finest / 2^(m-1-l), Eq. 9 */
        L->tau = 0.5 + (tau_finest - 0.5) / (double)L->h;
        size_t nc = (size_t)L->nx * L->ny;
        L->bstate = (unsigned char*)calloc((size_t)L->nbx * L->nby, 1);
        L->type = (unsigned char*)calloc(nc, 1);
        L->f = (double*)calloc(nc * NQ, sizeof(double));
        L->fs = (double*)calloc(nc * NQ, sizeof(double));
        L->tmp = (double*)calloc(nc * NQ, sizeof(double));
        L->Fx = (double*)calloc(nc, sizeof(double));
        L->Fy = (double*)calloc(nc, sizeof(double));
        if (!L->bstate || !L->type || !L->f || !L->fs || !L->tmp || !L->Fx || !L->Fy) return NULL;
    }
    return d;
}

void orc_destroy(Dom* d) {
    if (!d) return;
    for (int l = 0; l < d->m; l++) {
        Lev* L = &d->lev[l];
        free(L->bstate);
        free(L->type);
        free(L->f);
        free(L->fs);
        free(L->tmp);
        free(L->Fx);
        free(L->Fy);
    }
    free(d->body.qx);
    free(d->body.qy);
    free(d->body.hist);
    free(d->boxes);
    free(d);
}

const char* orc_error(Dom* d) { return d->err ? d->msg : ""; }
int orc_level_dims(Dom* d, int l, int* nx, int* ny) {
    if (l < 0 || l >= d->m) return -1;
    *nx = d->lev[l].nx;
    *ny = d->lev[l].ny;
    return 0;
}
double orc_level_tau(Dom* d, int l) { return d->lev[l].tau; }

int orc_set_rescale(Dom* d, int on) {
    d->rescale = on;
    return 0;
}
int orc_set_iface(Dom* d, int mode) {
    d->iface = mode;
    return 0;
}

/* scale factors of reading R3b between level lc and lc + 1 */
static double beta_c2f(Dom* d, int lc) {
    double tc = d->lev[lc].tau, tf = d->lev[lc + 1].tau;
    return d->rescale ? (tf - 1.0) / (2.0 * (tc - 1.0)) : 1.0;
}
static double beta_f2c(Dom* d, int lc) {
    double tc = d->lev[lc].tau, tf = d->lev[lc + 1].tau;
    return d->rescale ? 2.0 * tc / tf : 1.0;
}

int orc_add_box(Dom* d, int level, double x0, double y0, double x1, double y1) {
    d->boxes = (double*)realloc(d->boxes, (size_t)(d->nbox + 1) * 5 * sizeof(double));
    double* b = d->boxes + 5 * d->nbox;
    b[0] = level;
    b[1] = x0;
    b[2] = y0;
    b[3] = x1;
    b[4] = y1;
    d->nbox++;
    return 0;
}

/* margins (finest units) of the body-following refinement, index = level 1..m-1 */
int orc_set_refine_margins(Dom* d, const double* margin, const double* wake, int retag) {
    for (int l = 0; l < MAXLEV; l++) {
        d->margin[l] = margin[l];
        d->wake[l] = wake[l];
    }
    d->retag = retag;
    return 0;
}

int orc_set_body(Dom* d, double a, double b, int n, const double* pivot, int motion, const double* x0,
                 double alpha_mean, double alpha_amp, double period, double phase, double heave_amp,
                 double beta, int K) {
    Body* bd = &d->body;
    free(bd->qx);
    free(bd->qy);
    bd->present = 1;
    bd->n = n;
    bd->qx = (double*)malloc((size_t)n * sizeof(double));
    bd->qy = (double*)malloc((size_t)n * sizeof(double));
    double P = orc_place_markers(a, b, n, bd->qx, bd->qy);
    bd->ds = P / (double)n;
    bd->pivot[0] = pivot[0];
    bd->pivot[1] = pivot[1];
    bd->motion = motion;
    bd->x0[0] = x0[0];
    bd->x0[1] = x0[1];
    bd->alpha_mean = alpha_mean;
    bd->alpha_amp = alpha_amp;
    bd->period = period;
    bd->phase = phase;
    bd->heave_amp = heave_amp;
    bd->beta = beta;
    bd->K = K;
    return 0;
}

/* Body shape and the parameters of motions 3 and 4, after orc_set_body:
 * extra = {a_s, K, t1*, t_ref, xi, t_a / T}. */
/* Reading R15: walls and solid obstacles with bounce-back (the boundary
 * family of Sec. 2.1 after Eq. 10, whose formulas the paper leaves to its
 * reference; the half-way and linearly interpolated forms of Bouzidi et al.). */
int orc_set_walls(Dom* d, const double* uwall8) {
    for (int s = 0; s < 4; s++) {
        d->uwall[s][0] = uwall8[2 * s];
        d->uwall[s][1] = uwall8[2 * s + 1];
    }
    return 0;
}

int orc_set_solid(Dom* d, int kind, const double* prm) {
    if (kind < 0 || kind > 2) return -1;
    d->solid = kind;
    for (int k = 0; k < 3; k++) d->sol[k] = prm[k];
    return 0;
}

/* is the point (px, py) (finest units) inside the solid? */
static int in_solid(const Dom* d, double px, double py) {
    if (d->solid == 1) {
        double dx = px - d->sol[0], dy = py - d->sol[1];
        return dx * dx + dy * dy < d->sol[2] * d->sol[2];
    }
    if (d->solid == 2) return py < d->sol[0];
    return 0;
}

/* fraction t in (0, 1] of the link from the centre (px, py) along (ex, ey)
 * (one lattice vector of the finest level) at which it meets the solid's
 * surface; the start lies outside, the end inside */
static double wall_fraction(const Dom* d, double px, double py, double ex, double ey) {
    if (d->solid == 2) return (py - d->sol[0]) / (-ey);
    double ax = px - d->sol[0], ay = py - d->sol[1];
    double A = ex * ex + ey * ey, Bh = ax * ex + ay * ey, Cc = ax * ax + ay * ay - d->sol[2] * d->sol[2];
    return (-Bh - sqrt(Bh * Bh - A * Cc)) / A; /* the smaller root: the entry point */
}

double orc_wall_fraction(Dom* d, double px, double py, double ex, double ey) {
    return wall_fraction(d, px, py, ex, ey);
}
int orc_in_solid(Dom* d, double px, double py) { return in_solid(d, px, py); }

/* collision kind: 0 BGK, 1 MRT with rates s3 = {s_e, s_eps, s_q}, 2 LES
 * with the Smagorinsky constant s3[0] */
int orc_set_collision(Dom* d, int kind, const double* s3) {
    if (kind < 0 || kind > 2) return -1;
    d->coll = kind;
    for (int k = 0; k < 3; k++) d->mrt_s[k] = s3[k];
    return 0;
}

int orc_set_body_ext(Dom* d, int kind, double a, double b, const double* extra) {
    Body* bd = &d->body;
    if (!bd->present || kind < 0 || kind > 3) return -1;
    bd->ds = orc_place_markers_kind(kind, a, b, bd->n, bd->qx, bd->qy) / (double)bd->n;
    bd->ramp_as = extra[0];
    bd->ramp_rate = extra[1];
    bd->ramp_t1 = extra[2];
    bd->t_ref = extra[3];
    bd->xi = extra[4];
    bd->acc = extra[5];
    return 0;
}

/* centre and rotation angle of the body at finest time t */
int orc_body_pose(Dom* d, double t, double* out3) {
    if (!d->body.present) return -1;
    body_pose(&d->body, t, &out3[0], &out3[1], &out3[2]);
    return 0;
}

int orc_body_markers(Dom* d, long fine_step, double* rx, double* ry) {
    if (!d->body.present) return -1;
    marker_positions(&d->body, (double)fine_step, rx, ry);
    return d->body.n;
}
double orc_body_ds(Dom* d) { return d->body.ds; }

/* ------------------------------------------------------------------ */
/* Topology: Sec. 2.3 (square blocks, levels 0..m-1) and Sec. 2.4      */
/* (level jump of at most one between adjacent blocks, two halo layers)*/
/* ------------------------------------------------------------------ */

/* The region that must be at level >= L: the open rectangle around the body's
 * marker bounding box over the finest steps of the coarse step [n, n+1],
 * widened by margin[L] on every side and by wake[L] on the +x side. */
static int body_box(Dom* d, int L, double* x0, double* y0, double* x1, double* y1) {
    Body* bd = &d->body;
    if (!bd->present || d->margin[L] <= 0.0) return 0;
    long nf = 1L << (d->m - 1);
    long k0 = d->coarse_step * nf;
    double* rx = (double*)malloc((size_t)bd->n * sizeof(double));
    double* ry = (double*)malloc((size_t)bd->n * sizeof(double));
    double mnx = 1e300, mny = 1e300, mxx = -1e300, mxy = -1e300;
    for (long k = k0; k <= k0 + nf; k++) {
        marker_positions(bd, (double)k, rx, ry);
        for (int j = 0; j < bd->n; j++) {
            if (rx[j] < mnx) mnx = rx[j];
            if (rx[j] > mxx) mxx = rx[j];
            if (ry[j] < mny) mny = ry[j];
            if (ry[j] > mxy) mxy = ry[j];
        }
    }
    free(rx);
    free(ry);
    *x0 = mnx - d->margin[L];
    *x1 = mxx + d->margin[L] + d->wake[L];
    *y0 = mny - d->margin[L];
    *y1 = mxy + d->margin[L];
    return 1;
}

static int rect_hits_block(double x0, double y0, double x1, double y1, double bx0, double by0, double bx1,
                           double by1) {
    return bx0 < x1 && x0 < bx1 && by0 < y1 && y0 < by1;
}

/* does the level-l block (bx, by) intersect a region that requires level >= l+1 ? */
static int needs_refine(Dom* d, int l, int bx, int by) {
    double w = (double)d->B * d->lev[l].h;
    double X0 = bx * w, X1 = (bx + 1) * w, Y0 = by * w, Y1 = (by + 1) * w;
    for (int k = 0; k < d->nbox; k++) {
        double* b = d->boxes + 5 * k;
        if ((int)b[0] >= l + 1 && rect_hits_block(b[1], b[2], b[3], b[4], X0, Y0, X1, Y1)) return 1;
    }
    for (int L = l + 1; L < d->m; L++) {
        double x0, y0, x1, y1;
        if (body_box(d, L, &x0, &y0, &x1, &y1) && rect_hits_block(x0, y0, x1, y1, X0, Y0, X1, Y1)) return 1;
    }
    return 0;
}

static void refine_block(Dom* d, int l, int bx, int by) {
    Lev* L = &d->lev[l];
    Lev* C = &d->lev[l + 1];
    L->bstate[(size_t)by * L->nbx + bx] = 2;
    for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) C->bstate[(size_t)(2 * by + b) * C->nbx + 2 * bx + a] = 1;
}

/* wrap (periodic) or reject a lattice coordinate; returns 0 when outside */
static int wrap_coord(int v, int n, int periodic, int* out) {
    if (v >= 0 && v < n) {
        *out = v;
        return 1;
    }
    if (!periodic) return 0;
    *out = ((v % n) + n) % n;
    return 1;
}

static void build_blocks(Dom* d) {
    for (int l = 0; l < d->m; l++) memset(d->lev[l].bstate, 0, (size_t)d->lev[l].nbx * d->lev[l].nby);
    Lev* L0 = &d->lev[0];
    memset(L0->bstate, 1, (size_t)L0->nbx * L0->nby);
    for (int l = 0; l + 1 < d->m; l++) {
        Lev* L = &d->lev[l];
        for (int by = 0; by < L->nby; by++)
            for (int bx = 0; bx < L->nbx; bx++)
                if (L->bstate[(size_t)by * L->nbx + bx] == 1 && needs_refine(d, l, bx, by)) refine_block(d, l, bx, by);
    }
    /* 2:1 balance over faces and corners: a leaf of level l must not touch a
     * refined level-(l+1) block (that would put a level >= l+2 leaf next to it) */
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int l = 0; l + 2 < d->m; l++) {
            Lev* L = &d->lev[l];
            Lev* C = &d->lev[l + 1];
            for (int by = 0; by < L->nby; by++) {
                for (int bx = 0; bx < L->nbx; bx++) {
                    if (L->bstate[(size_t)by * L->nbx + bx] != 1) continue;
                    int hit = 0;
                    for (int y = 2 * by - 1; y <= 2 * by + 2 && !hit; y++) {
                        for (int x = 2 * bx - 1; x <= 2 * bx + 2 && !hit; x++) {
                            if (x >= 2 * bx && x <= 2 * bx + 1 && y >= 2 * by && y <= 2 * by + 1) continue;
                            int wx, wy;
                            if (!wrap_coord(x, C->nbx, periodic_x(d), &wx)) continue;
                            if (!wrap_coord(y, C->nby, periodic_y(d), &wy)) continue;
                            if (C->bstate[(size_t)wy * C->nbx + wx] == 2) hit = 1;
                        }
                    }
                    if (hit) {
                        refine_block(d, l, bx, by);
                        changed = 1;
                    }
                }
            }
        }
    }
}

/* Cell types of every level (Sec. 2.4: two halo layers on the fine side;
 * reading R3: one ghost layer on the coarse side). */
static void build_types(Dom* d) {
    for (int l = 0; l < d->m; l++) {
        Lev* L = &d->lev[l];
        for (int y = 0; y < L->ny; y++) {
            for (int x = 0; x < L->nx; x++) {
                int bs = L->bstate[(size_t)(y / d->B) * L->nbx + x / d->B];
                L->type[IDX(L, x, y)] = (bs == 1) ? T_INT : T_NONE;
            }
        }
        for (int y = 0; y < L->ny; y++) {
            for (int x = 0; x < L->nx; x++) {
                int bs = L->bstate[(size_t)(y / d->B) * L->nbx + x / d->B];
                if (bs == 1) continue;
                int reach = (bs == 2) ? 1 : 2; /* coarse-side ghost: 1 layer; fine-side: 2 */
                int near = 0;
                for (int dy = -reach; dy <= reach && !near; dy++) {
                    for (int dx = -reach; dx <= reach && !near; dx++) {
                        int wx, wy;
                        if (!wrap_coord(x + dx, L->nx, periodic_x(d), &wx)) continue;
                        if (!wrap_coord(y + dy, L->ny, periodic_y(d), &wy)) continue;
                        int ws = L->bstate[(size_t)(wy / d->B) * L->nbx + wx / d->B];
                        if (ws == 1) near = 1;
                    }
                }
                if (near) L->type[IDX(L, x, y)] = (bs == 2) ? T_GC : T_GF;
            }
        }
    }
    /* solid cells: finest interior cells whose centre lies inside the solid */
    if (d->solid) {
        Lev* L = &d->lev[d->m - 1];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++)
                if (L->type[IDX(L, x, y)] == T_INT && in_solid(d, x + 0.5, y + 0.5)) L->type[IDX(L, x, y)] = T_SOLID;
    }
}

/* refinement must stay clear of non-periodic domain sides */
static int check_topology(Dom* d) {
    for (int l = 1; l < d->m; l++) {
        Lev* L = &d->lev[l];
        for (int by = 0; by < L->nby; by++) {
            for (int bx = 0; bx < L->nbx; bx++) {
                if (L->bstate[(size_t)by * L->nbx + bx] == 0) continue;
                if (!periodic_x(d) && (bx == 0 || bx == L->nbx - 1)) return -1;
                if (!periodic_y(d) && (by == 0 || by == L->nby - 1)) return -1;
            }
        }
    }
    return 0;
}

/* every cell within two cells of a solid cell must be a finest interior or
 * solid cell (the interpolated bounce-back reads two cells from the wall) */
static int check_solid(Dom* d) {
    if (!d->solid) return 0;
    if (d->retag) return -1;
    Lev* L = &d->lev[d->m - 1];
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            if (!in_solid(d, x + 0.5, y + 0.5)) continue;
            for (int dy = -2; dy <= 2; dy++)
                for (int dx = -2; dx <= 2; dx++) {
                    int wx = x + dx, wy = y + dy;
                    if (!wrap_coord(wx, L->nx, periodic_x(d), &wx) || !wrap_coord(wy, L->ny, periodic_y(d), &wy)) {
                        if (d->solid == 1) return -1; /* a circle must keep clear of the sides */
                        continue;
                    }
                    int t = L->type[IDX(L, wx, wy)];
                    if (t != T_INT && t != T_SOLID) return -1;
                }
        }
    return 0;
}

int orc_build(Dom* d) {
    build_blocks(d);
    build_types(d);
    if (check_topology(d)) {
        set_err(d, "refinement touches a non-periodic domain side");
        return -1;
    }
    if (check_solid(d)) {
        set_err(d, "the solid must lie in the finest interior, two cells clear, with a static refinement");
        return -1;
    }
    return 0;
}

int orc_get_types(Dom* d, int l, unsigned char* out) {
    Lev* L = &d->lev[l];
    memcpy(out, L->type, (size_t)L->nx * L->ny);
    return 0;
}
int orc_get_blocks(Dom* d, int l, unsigned char* out) {
    Lev* L = &d->lev[l];
    memcpy(out, L->bstate, (size_t)L->nbx * L->nby);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Initial state                                                       */
/* ------------------------------------------------------------------ */

/* f = f^eq(rho, u) (Eq. 7) on the interior cells of level l; dense inputs */
int orc_set_fields(Dom* d, int l, const double* rho, const double* ux, const double* uy) {
    Lev* L = &d->lev[l];
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = IDX(L, x, y);
            if (L->type[c] != T_INT) continue;
            for (int i = 0; i < NQ; i++) FQ(L, f, i, x, y) = orc_feq(i, rho[c], ux[c], uy[c]);
        }
    return 0;
}

/* raw pre-collision populations, dense [9][ny][nx]; only interior cells used */
int orc_set_populations(Dom* d, int l, const double* f) {
    Lev* L = &d->lev[l];
    size_t nc = (size_t)L->nx * L->ny;
    for (int i = 0; i < NQ; i++)
        for (size_t c = 0; c < nc; c++)
            if (L->type[c] == T_INT) L->f[i * nc + c] = f[i * nc + c];
    return 0;
}

static void f2c(Dom* d, int lf, int lc);

/* coarse-side ghost cells start as the mean of their children (reading R3) */
int orc_finalize_init(Dom* d) {
    if (d->iface == 0)
        for (int l = d->m - 2; l >= 0; l--) f2c(d, l + 1, l);
    d->retag_pending = 0;
    return d->err ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Level operations of Algorithm 1                                     */
/* ------------------------------------------------------------------ */

/* UpdateVelocity: IBM on the finest level (reading R4), no-op elsewhere */
static void update_velocity(Dom* d, int l) {
    Lev* L = &d->lev[l];
    if (l != d->m - 1 || !d->body.present) return;
    Body* bd = &d->body;
    size_t nc = (size_t)L->nx * L->ny;
    double* rho = (double*)calloc(nc, sizeof(double));
    double* ux = (double*)calloc(nc, sizeof(double));
    double* uy = (double*)calloc(nc, sizeof(double));
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = IDX(L, x, y);
            if (L->type[c] != T_INT) continue;
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < NQ; i++) {
                double v = FQ(L, f, i, x, y);
                r += v;
                jx += CX[i] * v;
                jy += CY[i] * v;
            }
            rho[c] = r;
            ux[c] = jx / r; /* uncorrected velocity, Sec. 2.2 text after Eq. 11 */
            uy[c] = jy / r;
        }
    int n = bd->n;
    double* rx = (double*)malloc((size_t)n * sizeof(double));
    double* ry = (double*)malloc((size_t)n * sizeof(double));
    double* rx1 = (double*)malloc((size_t)n * sizeof(double));
    double* ry1 = (double*)malloc((size_t)n * sizeof(double));
    double* udx = (double*)malloc((size_t)n * sizeof(double));
    double* udy = (double*)malloc((size_t)n * sizeof(double));
    double* dsj = (double*)malloc((size_t)n * sizeof(double));
    double* Fjx = (double*)malloc((size_t)n * sizeof(double));
    double* Fjy = (double*)malloc((size_t)n * sizeof(double));
    long k = d->fine_step;
    marker_positions(bd, (double)k, rx, ry);
    marker_positions(bd, (double)(k + 1), rx1, ry1);
    for (int j = 0; j < n; j++) {
        /* Sec. 2.2: u^d = (r(t + dt) - r(t)) / dt with dt one finest step */
        udx[j] = rx1[j] - rx[j];
        udy[j] = ry1[j] - ry[j];
        dsj[j] = bd->ds;
        int i0 = stencil_origin(rx[j]), j0 = stencil_origin(ry[j]);
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) {
                int ci = i0 + a, cj = j0 + b;
                if (ci < 0 || cj < 0 || ci >= L->nx || cj >= L->ny || L->type[IDX(L, ci, cj)] != T_INT)
                    set_err(d, "a marker stencil leaves the finest interior cells");
            }
    }
    if (!d->err && orc_ibm_mdf(L->nx, L->ny, rho, ux, uy, n, rx, ry, udx, udy, dsj, bd->K, L->Fx, L->Fy, Fjx, Fjy))
        set_err(d, "IBM stencil outside the grid");
    /* Eq. 16: F_s = - sum_j F_j ds; moment about the pivot likewise */
    double cx, cy, al;
    body_pose(bd, (double)k, &cx, &cy, &al);
    double px = cx + bd->pivot[0], py = cy + bd->pivot[1];
    double FX = 0.0, FY = 0.0, MZ = 0.0;
    for (int j = 0; j < n; j++) {
        FX -= Fjx[j] * dsj[j];
        FY -= Fjy[j] * dsj[j];
        MZ -= ((rx[j] - px) * Fjy[j] - (ry[j] - py) * Fjx[j]) * dsj[j];
    }
    if (bd->hist_n + 1 > bd->hist_cap) {
        bd->hist_cap = bd->hist_cap ? 2 * bd->hist_cap : 1024;
        bd->hist = (double*)realloc(bd->hist, (size_t)bd->hist_cap * 3 * sizeof(double));
    }
    bd->hist[3 * bd->hist_n + 0] = FX;
    bd->hist[3 * bd->hist_n + 1] = FY;
    bd->hist[3 * bd->hist_n + 2] = MZ;
    bd->hist_n++;
    free(rho);
    free(ux);
    free(uy);
    free(rx);
    free(ry);
    free(rx1);
    free(ry1);
    free(udx);
    free(udy);
    free(dsj);
    free(Fjx);
    free(Fjy);
}

/* CollisionStep: interior and coarse-side ghost cells (Eq. 6 with Eq. 3) */
static void collide(Dom* d, int l) {
    Lev* L = &d->lev[l];
    int finest = (l == d->m - 1);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = IDX(L, x, y);
            int t = L->type[c];
            if (t != T_INT && (t != T_GC || d->iface == 1)) continue;
            double f[NQ], fs[NQ];
            for (int i = 0; i < NQ; i++) f[i] = FQ(L, f, i, x, y);
            double Fx = (finest && t == T_INT) ? L->Fx[c] : 0.0;
            double Fy = (finest && t == T_INT) ? L->Fy[c] : 0.0;
            if (d->coll == 1)
                orc_collide_cell_mrt(f, L->tau, d->mrt_s, Fx, Fy, fs);
            else if (d->coll == 2)
                orc_collide_cell_les(f, L->tau, d->mrt_s[0], Fx, Fy, fs);
            else
                orc_collide_cell(f, L->tau, Fx, Fy, fs);
            for (int i = 0; i < NQ; i++) FQ(L, fs, i, x, y) = fs[i];
        }
    if (finest) d->fine_step++;
}

/* value pulled into cell (x, y), direction i: Eq. 10 plus reading R2 at the
 * domain sides and reading R3 for ghost cells */
/* half-way bounce-back from a wall side (reading R15): the population that
 * left (x, y) toward the wall comes back reversed, with the momentum of the
 * moving wall, 2 w_i rho0 (c_i . u_w) / c_s^2 */
static double bounce_wall(Dom* d, Lev* L, int x, int y, int i, int side) {
    int o = flip_x(flip_y(i));
    return FQ(L, fs, o, x, y) + 2.0 * WQ[i] * d->rho0 * (CX[i] * d->uwall[side][0] + CY[i] * d->uwall[side][1]) / CS2;
}

/* linearly interpolated bounce-back (reading R15) into fluid cell (x, y) of
 * the finest level, direction i, whose source x - c_i is solid: with t the
 * fraction of the link x -> x - c_i outside the solid,
 *   t < 1/2:  f_i = 2t f*_o(x) + (1 - 2t) f*_o(x + c_i)
 *   t >= 1/2: f_i = f*_o(x) / (2t) + (1 - 1/(2t)) f*_i(x)
 * (o = opposite of i; the first form needs x + c_i to be a fluid cell, else
 * the second is used) */
static double bounce_solid(Dom* d, Lev* L, int x, int y, int i) {
    int o = flip_x(flip_y(i));
    double t = wall_fraction(d, x + 0.5, y + 0.5, -CX[i], -CY[i]);
    double a = FQ(L, fs, o, x, y);
    if (t < 0.5) {
        int nx2, ny2;
        if (wrap_coord(x + CX[i], L->nx, periodic_x(d), &nx2) && wrap_coord(y + CY[i], L->ny, periodic_y(d), &ny2) &&
            L->type[IDX(L, nx2, ny2)] == T_INT)
            return 2.0 * t * a + (1.0 - 2.0 * t) * FQ(L, fs, o, nx2, ny2);
    }
    return a / (2.0 * t) + (1.0 - 1.0 / (2.0 * t)) * FQ(L, fs, i, x, y);
}

static double pull(Dom* d, int l, int x, int y, int i) {
    Lev* L = &d->lev[l];
    int q = i;
    int sx = x - CX[i], sy = y - CY[i];
    if (periodic_x(d)) sx = ((sx % L->nx) + L->nx) % L->nx;
    if (periodic_y(d)) sy = ((sy % L->ny) + L->ny) % L->ny;
    if (sy < 0 || sy >= L->ny) {
        int side = (sy < 0) ? SIDE_S : SIDE_N;
        int edge = (sy < 0) ? 0 : L->ny - 1;
        switch (d->bc[side]) {
        case BC_SYMMETRY: sy = edge; q = flip_y(q); break;
        case BC_OUTLET: sy = edge; break;
        case BC_INLET: return orc_feq(q, d->rho0, d->uin[0], d->uin[1]);
        case BC_WALL: return bounce_wall(d, L, x, y, i, side);
        }
    }
    if (sx < 0 || sx >= L->nx) {
        int side = (sx < 0) ? SIDE_W : SIDE_E;
        int edge = (sx < 0) ? 0 : L->nx - 1;
        switch (d->bc[side]) {
        case BC_SYMMETRY: sx = edge; q = flip_x(q); break;
        case BC_OUTLET: sx = edge; break;
        case BC_INLET: return orc_feq(q, d->rho0, d->uin[0], d->uin[1]);
        case BC_WALL: return bounce_wall(d, L, x, y, i, side);
        }
    }
    int t = L->type[IDX(L, sx, sy)];
    if (t == T_SOLID) {
        if (L->type[IDX(L, x, y)] == T_INT && q == i) return bounce_solid(d, L, x, y, i);
        set_err(d, "a solid cell is the streaming source of a non-interior cell");
        return 0.0;
    }
    if (t == T_GC && d->iface == 1) return 0.0; /* filled by the coalescence */
    if (t == T_INT || t == T_GC) return FQ(L, fs, q, sx, sy);
    if (t == T_GF) return FQ(L, f, q, sx, sy); /* ghost values are never collided */
    if (L->type[IDX(L, x, y)] == T_GF) return FQ(L, f, i, x, y); /* no source: keep */
    set_err(d, "an interior cell has no streaming source");
    return 0.0;
}

/* StreamingStep + BoundaryConditionStep on level l */
static void stream_bc(Dom* d, int l) {
    Lev* L = &d->lev[l];
#pragma omp parallel for schedule(static)
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            int t = L->type[IDX(L, x, y)];
            if (t != T_INT && t != T_GF) continue;
            for (int i = 0; i < NQ; i++) FQ(L, tmp, i, x, y) = pull(d, l, x, y, i);
        }
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            int t = L->type[IDX(L, x, y)];
            if (t != T_INT && t != T_GF) continue;
            for (int i = 0; i < NQ; i++) FQ(L, f, i, x, y) = FQ(L, tmp, i, x, y);
        }
    /* equilibrium inlet: the boundary column is reset (reading R2) */
    for (int s = 0; s < 4; s++) {
        if (d->bc[s] != BC_INLET) continue;
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                int on = (s == SIDE_W && x == 0) || (s == SIDE_E && x == L->nx - 1) || (s == SIDE_S && y == 0) ||
                         (s == SIDE_N && y == L->ny - 1);
                if (!on || L->type[IDX(L, x, y)] != T_INT) continue;
                for (int i = 0; i < NQ; i++) FQ(L, f, i, x, y) = orc_feq(i, d->rho0, d->uin[0], d->uin[1]);
            }
    }
}

/* CoarseToFineCommunication (Sec. 2.4 step 2, reading R3) */
static void c2f(Dom* d, int lc, int lf) {
    Lev* C = &d->lev[lc];
    Lev* F = &d->lev[lf];
    for (int y = 0; y < F->ny; y++)
        for (int x = 0; x < F->nx; x++) {
            if (F->type[IDX(F, x, y)] != T_GF) continue;
            int px = x / 2, py = y / 2;
            if (C->type[IDX(C, px, py)] != T_INT) {
                set_err(d, "fine ghost cell without an interior coarse parent");
                continue;
            }
            double src[NQ], out[NQ];
            for (int i = 0; i < NQ; i++) src[i] = FQ(C, fs, i, px, py);
            orc_rescale_neq(src, beta_c2f(d, lc), out);
            for (int i = 0; i < NQ; i++) FQ(F, f, i, x, y) = out[i];
        }
}

/* FineToCoarseCommunication, volumetric reading R3c: every coarse interior
 * population whose streaming source lies in the finer region becomes the
 * mean of that population over the 4 fine halo cells inside the coarse cell */
static void f2c_volumetric(Dom* d, int lf, int lc) {
    Lev* C = &d->lev[lc];
    Lev* F = &d->lev[lf];
    for (int y = 0; y < C->ny; y++)
        for (int x = 0; x < C->nx; x++) {
            if (C->type[IDX(C, x, y)] != T_INT) continue;
            for (int i = 0; i < NQ; i++) {
                int sx = x - CX[i], sy = y - CY[i];
                if (!wrap_coord(sx, C->nx, periodic_x(d), &sx) || !wrap_coord(sy, C->ny, periodic_y(d), &sy))
                    continue;
                if (C->type[IDX(C, sx, sy)] != T_GC) continue;
                double m = 0.0;
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++) {
                        if (F->type[IDX(F, 2 * x + a, 2 * y + b)] != T_GF) set_err(d, "coalescence without halo");
                        m += FQ(F, f, i, 2 * x + a, 2 * y + b);
                    }
                FQ(C, f, i, x, y) = 0.25 * m;
            }
        }
}

/* FineToCoarseCommunication (Sec. 2.4 step 6, reading R3) */
static void f2c(Dom* d, int lf, int lc) {
    Lev* C = &d->lev[lc];
    Lev* F = &d->lev[lf];
    if (d->iface == 1) {
        f2c_volumetric(d, lf, lc);
        return;
    }
    for (int y = 0; y < C->ny; y++)
        for (int x = 0; x < C->nx; x++) {
            if (C->type[IDX(C, x, y)] != T_GC) continue;
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++)
                    if (F->type[IDX(F, 2 * x + a, 2 * y + b)] != T_INT)
                        set_err(d, "coarse ghost cell whose children are not interior");
            double mean[NQ], out[NQ];
            for (int i = 0; i < NQ; i++)
                mean[i] = 0.25 * (FQ(F, f, i, 2 * x, 2 * y) + FQ(F, f, i, 2 * x + 1, 2 * y) +
                                  FQ(F, f, i, 2 * x, 2 * y + 1) + FQ(F, f, i, 2 * x + 1, 2 * y + 1));
            orc_rescale_neq(mean, beta_f2c(d, lc), out);
            for (int i = 0; i < NQ; i++) FQ(C, f, i, x, y) = out[i];
        }
}

/* ------------------------------------------------------------------ */
/* Re-tagging (reading R5)                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    unsigned char* type[MAXLEV];
    unsigned char* bstate[MAXLEV];
    double* fs[MAXLEV];
} OldState;

/* post-collision populations of (l, x, y) in the old topology (reading R5,
 * with the rescaling of reading R3b when values change level: a copy from
 * the coarser level maps f - f^eq by (tau_f - 1) / (2 (tau_c - 1)) per level,
 * a mean of 4 finer values by the inverse) */
static void old_values(Dom* d, OldState* o, int l, int x, int y, double* out) {
    Lev* L = &d->lev[l];
    size_t nc = (size_t)L->nx * L->ny;
    size_t c = IDX(L, x, y);
    int t = o->type[l][c];
    if (t == T_INT || (t == T_GC && d->iface == 0)) {
        for (int i = 0; i < NQ; i++) out[i] = o->fs[l][(size_t)i * nc + c];
        return;
    }
    int bs = o->bstate[l][(size_t)(y / d->B) * L->nbx + x / d->B];
    if (bs == 0) { /* inside a coarser leaf: copy the covering coarser cell */
        int ll = l, xx = x, yy = y;
        while (ll > 0) {
            ll--;
            xx /= 2;
            yy /= 2;
            Lev* P = &d->lev[ll];
            size_t pc = IDX(P, xx, yy);
            if (o->type[ll][pc] == T_INT) {
                double v[NQ];
                for (int i = 0; i < NQ; i++) v[i] = o->fs[ll][(size_t)i * P->nx * P->ny + pc];
                for (int lv = ll; lv < l; lv++) {
                    orc_rescale_neq(v, beta_c2f(d, lv), out);
                    for (int i = 0; i < NQ; i++) v[i] = out[i];
                }
                for (int i = 0; i < NQ; i++) out[i] = v[i];
                return;
            }
        }
        set_err(d, "re-tag: no covering coarser cell");
        for (int i = 0; i < NQ; i++) out[i] = 0.0;
        return;
    }
    if (l + 1 >= d->m) {
        set_err(d, "re-tag: refined finest block");
        for (int i = 0; i < NQ; i++) out[i] = 0.0;
        return;
    }
    double mean[NQ] = {0}, kid[NQ];
    for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) {
            old_values(d, o, l + 1, 2 * x + a, 2 * y + b, kid);
            for (int i = 0; i < NQ; i++) mean[i] += kid[i];
        }
    for (int i = 0; i < NQ; i++) mean[i] *= 0.25;
    orc_rescale_neq(mean, 1.0 / beta_c2f(d, l), out);
}

static void retag(Dom* d) {
    OldState o;
    for (int l = 0; l < d->m; l++) {
        Lev* L = &d->lev[l];
        size_t nc = (size_t)L->nx * L->ny;
        o.type[l] = (unsigned char*)malloc(nc);
        o.bstate[l] = (unsigned char*)malloc((size_t)L->nbx * L->nby);
        o.fs[l] = (double*)malloc(nc * NQ * sizeof(double));
        memcpy(o.type[l], L->type, nc);
        memcpy(o.bstate[l], L->bstate, (size_t)L->nbx * L->nby);
        memcpy(o.fs[l], L->fs, nc * NQ * sizeof(double));
    }
    if (orc_build(d) == 0) {
        for (int l = 0; l < d->m; l++) {
            Lev* L = &d->lev[l];
            for (int y = 0; y < L->ny; y++)
                for (int x = 0; x < L->nx; x++) {
                    int t = L->type[IDX(L, x, y)];
                    if (t != T_INT && (t != T_GC || d->iface == 1)) continue;
                    double v[NQ];
                    old_values(d, &o, l, x, y, v);
                    for (int i = 0; i < NQ; i++) FQ(L, fs, i, x, y) = v[i];
                }
        }
    }
    for (int l = 0; l < d->m; l++) {
        free(o.type[l]);
        free(o.bstate[l]);
        free(o.fs[l]);
    }
}

/* apply only the value transfer of a re-tag to a given new block layout
 * (used by the round-trip tests): the domain's blocks are replaced by the
 * caller's, for every level, and values are carried over as in retag(). */
int orc_retag_to(Dom* d, const unsigned char* const* new_bstate) {
    OldState o;
    for (int l = 0; l < d->m; l++) {
        Lev* L = &d->lev[l];
        size_t nc = (size_t)L->nx * L->ny;
        o.type[l] = (unsigned char*)malloc(nc);
        o.bstate[l] = (unsigned char*)malloc((size_t)L->nbx * L->nby);
        o.fs[l] = (double*)malloc(nc * NQ * sizeof(double));
        memcpy(o.type[l], L->type, nc);
        memcpy(o.bstate[l], L->bstate, (size_t)L->nbx * L->nby);
        memcpy(o.fs[l], L->fs, nc * NQ * sizeof(double));
        memcpy(L->bstate, new_bstate[l], (size_t)L->nbx * L->nby);
    }
    build_types(d);
    for (int l = 0; l < d->m; l++) {
        Lev* L = &d->lev[l];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                int t = L->type[IDX(L, x, y)];
                if (t != T_INT && (t != T_GC || d->iface == 1)) continue;
                double v[NQ];
                old_values(d, &o, l, x, y, v);
                for (int i = 0; i < NQ; i++) FQ(L, fs, i, x, y) = v[i];
            }
    }
    for (int l = 0; l < d->m; l++) {
        free(o.type[l]);
        free(o.bstate[l]);
        free(o.fs[l]);
    }
    return d->err ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: SynchronousNonUniformTimeStep(l)                       */
/* ------------------------------------------------------------------ */

static void step_level(Dom* d, int l) {
    int finest = d->m - 1;
    update_velocity(d, l);
    collide(d, l);
    if (l == finest && d->retag_pending) { /* all levels are post-collision here */
        retag(d);
        d->retag_pending = 0;
    }
    if (l != finest) step_level(d, l + 1);
    if (l != 0) c2f(d, l - 1, l);
    /* SameLevelCommunication: nothing to exchange on a dense array */
    stream_bc(d, l);
    if (l != finest) f2c(d, l + 1, l);
    if (l == 0) return;
    update_velocity(d, l);
    collide(d, l);
    if (l != finest) step_level(d, l + 1);
    /* PreStreamingStep: the fine ghost layers are not collided (reading R3) */
    stream_bc(d, l);
    if (l != finest) f2c(d, l + 1, l);
}

/* advance n coarse steps; returns 0 or -1 (see orc_error) */
int orc_step(Dom* d, int n) {
    for (int s = 0; s < n && !d->err; s++) {
        d->retag_pending = (d->retag && d->coarse_step > 0);
        step_level(d, 0);
        d->coarse_step++;
    }
    return d->err ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Outputs                                                             */
/* ------------------------------------------------------------------ */

/* canonical pre-collision populations of level l, dense [9][ny][nx];
 * cells that are not interior are written as 0 */
int orc_get_populations(Dom* d, int l, double* out) {
    Lev* L = &d->lev[l];
    size_t nc = (size_t)L->nx * L->ny;
    for (int i = 0; i < NQ; i++)
        for (size_t c = 0; c < nc; c++) out[i * nc + c] = (L->type[c] == T_INT) ? L->f[i * nc + c] : 0.0;
    return 0;
}

/* post-collision populations (all types that hold them), dense [9][ny][nx] */
int orc_get_post(Dom* d, int l, double* out) {
    Lev* L = &d->lev[l];
    memcpy(out, L->fs, (size_t)L->nx * L->ny * NQ * sizeof(double));
    return 0;
}

/* rho and the uncorrected velocity sum_i c_i f_i / rho (Eq. 8 without F) */
int orc_get_fields(Dom* d, int l, double* rho, double* ux, double* uy) {
    Lev* L = &d->lev[l];
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = IDX(L, x, y);
            if (L->type[c] != T_INT) {
                rho[c] = ux[c] = uy[c] = 0.0;
                continue;
            }
            double r = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < NQ; i++) {
                double v = FQ(L, f, i, x, y);
                r += v;
                jx += CX[i] * v;
                jy += CY[i] * v;
            }
            rho[c] = r;
            ux[c] = jx / r;
            uy[c] = jy / r;
        }
    return 0;
}

/* mass and momentum of the canonical state, in finest-cell area units */
int orc_checksum(Dom* d, double* out3) {
    double M = 0.0, PX = 0.0, PY = 0.0;
    for (int l = 0; l < d->m; l++) {
        Lev* L = &d->lev[l];
        double area = (double)L->h * (double)L->h;
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                if (L->type[IDX(L, x, y)] != T_INT) continue;
                for (int i = 0; i < NQ; i++) {
                    double v = FQ(L, f, i, x, y);
                    M += area * v;
                    PX += area * CX[i] * v;
                    PY += area * CY[i] * v;
                }
            }
    }
    out3[0] = M;
    out3[1] = PX;
    out3[2] = PY;
    return 0;
}

/* force history: (Fx, Fy, Mz) per finest step; returns the number copied */
long orc_get_forces(Dom* d, double* out, long cap) {
    long n = d->body.hist_n < cap ? d->body.hist_n : cap;
    if (n > 0) memcpy(out, d->body.hist, (size_t)n * 3 * sizeof(double));
    return n;
}

long orc_fine_step(Dom* d) { return d->fine_step; }
long orc_coarse_step(Dom* d) { return d->coarse_step; }
