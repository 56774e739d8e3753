"""Seeded synthetic workloads shaped like the paper's test cases.

This module holds workload *parameters* only: grid sizes, boundary kinds,
body geometry and kinematics, Reynolds numbers, seeds, arrival times and the
Taylor-Green initial fields.  It holds none of the method's arithmetic
(no equilibria, collisions, streaming, kernels, interpolation or spreading):
both the CUDA library and the CPU oracle receive these numbers and do their
own work.

Workloads (the paper measures on no external data set; every input here is
generated from the parameters below):
  tgv        Taylor-Green vortex (Sec. 3.1), single level, periodic
  cylinder   flow past a circular cylinder (Sec. 3.3), W inlet / E outlet /
             symmetric N,S sides, static body, block refinement around it
  cylinder_table1
             the same at the sizes of the paper's Table 1 study (D = 128
             finest cells, 4 levels, U = 0.1, Re 100 / 300 / 550)
  wing       2D ellipse wing with sinusoidal pitch and a tilted-stroke heave
             (Sec. 3.6, Eqs. 25-27), periodic domain, refinement that follows
             the body
  pitch_up   flat plate (rectangle) pitching up about its leading edge with
             the smoothed ramp of Sec. 3.4 (Eqs. 20-21), inlet / outlet /
             symmetric sides, refinement that follows the body
  cavity     lid-driven square cavity with a central cylinder (Sec. 3.2),
             walls by bounce-back, the cylinder by interpolated bounce-back
             or by the IBM
  pitching_airfoil
             symmetric NACA section in smoothed asymmetric triangular pitch
             (Sec. 3.5, Eqs. 22-24), same domain kind
  batch      many uneven cylinder / wing instances drawn from a seed
  serving    Poisson arrivals of such instances
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

BC_PERIODIC, BC_INLET, BC_OUTLET, BC_SYMMETRY, BC_WALL = 0, 1, 2, 3, 4
F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
CS2 = 1.0 / 3.0  # lattice speed of sound squared (Sec. 2.1), used for the TGV initial density


@dataclass
class BodySpec:
    kind: int = 0  # 0 circle, 1 ellipse, 2 rectangle (flat plate), 3 symmetric NACA 00xx
    a: float = 20.0  # semi-axes (half chord, half thickness) in finest cells
    b: float = 20.0
    n_markers: int = 126
    pivot: tuple = (0.0, 0.0)  # body frame, relative to the centre
    motion: int = 0  # 0 static, 1 pitching, 2 flapping (pitch + heave), 3 pitch-up ramp, 4 triangular pitching
    x0: tuple = (0.0, 0.0)  # centre, finest units
    alpha_mean: float = 0.0
    alpha_amp: float = 0.0
    period: float = 1.0  # finest steps
    phase: float = 0.0
    heave_amp: float = 0.0  # A0 (the centre moves by A0/2)
    beta: float = 0.0  # stroke-plane angle
    K: int = 5  # multi-direct-forcing iterations
    u_ref: float = 0.05
    l_ref: float = 40.0
    ramp_as: float = 11.0  # motion 3 (Sec. 3.4): a_s, pitch rate K, t1*, finest steps per unit of t* = t U / c
    ramp_rate: float = 0.2
    ramp_t1: float = 1.0
    t_ref: float = 1.0
    xi: float = 0.5  # motion 4 (Sec. 3.5): asymmetry, corner time / period
    acc: float = 0.15


@dataclass
class DomainSpec:
    name: str
    nx0: int
    ny0: int
    levels: int = 1
    block: int = 16
    bc: tuple = (BC_PERIODIC,) * 4  # W, E, S, N
    tau_finest: float = 0.8
    rho0: float = 1.0
    u_in: tuple = (0.0, 0.0)
    storage: int = F64
    boxes: list = field(default_factory=list)  # (level, x0, y0, x1, y1), finest units
    margin: tuple = (0.0,) * 8  # per level: body-box dilation, finest units
    wake: tuple = (0.0,) * 8  # per level: extra +x extension
    retag: int = 0
    body: BodySpec | None = None
    steps: int = 100  # coarse steps of the workload
    init: str = "uniform"  # "uniform" (rho0, u_in) or "tgv"
    tgv_u0: float = 0.0
    tgv_offset: float = 0.0  # 0: x = i (nodes), 0.5: cell centres
    collision: int = 0  # 0 BGK (Eq. 6), 1 MRT, 2 LES (Sec. 2.1)
    mrt_rates: tuple = (1.64, 1.54, 1.9)  # MRT relaxation rates of e, eps, q
    les_cs: float = 0.17  # Smagorinsky constant of the LES collision (collision 2)
    uwall: tuple = (0.0,) * 8  # velocity (x, y) of each wall side W, E, S, N
    solid: tuple = (0, 0.0, 0.0, 0.0)  # (kind, ...): 1 circle (cx, cy, R), 2 half-plane y < y0

    @property
    def finest_nx(self) -> int:
        return self.nx0 << (self.levels - 1)

    @property
    def finest_ny(self) -> int:
        return self.ny0 << (self.levels - 1)

    def cells_per_level_domain(self):
        return [(self.nx0 << l) * (self.ny0 << l) for l in range(self.levels)]


def tau_from_re(u_ref: float, l_ref: float, re: float) -> float:
    """tau of the finest level from Re = U L / nu and nu = cs^2 (tau - 1/2) (Eq. 9)."""
    return 0.5 + (u_ref * l_ref / re) / CS2


def _round_up(v: float, m: int) -> int:
    return int(math.ceil(v / m) * m)


# ---------------------------------------------------------------------------
# Taylor-Green vortex (Sec. 3.1)
# ---------------------------------------------------------------------------

def tgv_fields(nx: int, ny: int, h: float, u0: float, wavelength: float, rho0: float = 1.0,
               offset: float = 0.0, t: float = 0.0, nu: float = 0.0):
    """rho, ux, uy of the Taylor-Green vortex at positions ((i+offset) h, (j+offset) h).

    u = -u0 cos(kx) sin(ky) e^{-2 nu k^2 t}, v = u0 sin(kx) cos(ky) e^{-2 nu k^2 t},
    p = -rho0 u0^2 / 4 (cos 2kx + cos 2ky) e^{-4 nu k^2 t},  rho = rho0 + p / cs^2.
    (The paper prints sin(2 pi y) in p and t_d = 1/(2 pi^2 nu); the form above
    is the standard solution that its velocity field belongs to.)
    """
    k = 2.0 * math.pi / wavelength
    x = (np.arange(nx) + offset) * h
    y = (np.arange(ny) + offset) * h
    X, Y = np.meshgrid(x, y)
    dec = math.exp(-2.0 * nu * k * k * t)
    ux = -u0 * np.cos(k * X) * np.sin(k * Y) * dec
    uy = u0 * np.sin(k * X) * np.cos(k * Y) * dec
    p = -rho0 * u0 * u0 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y)) * dec * dec
    rho = rho0 + p / CS2
    return rho, ux, uy


def initial_fields(spec: "DomainSpec", level: int):
    """rho, ux, uy of a workload's initial state on level `level`'s dense
    grid [ny_l][nx_l]: the Taylor-Green fields for a TGV spec, else the
    uniform state (rho0, u_in)."""
    nx, ny = spec.nx0 << level, spec.ny0 << level
    h = 1 << (spec.levels - 1 - level)
    if spec.init == "tgv":
        return tgv_fields(nx, ny, h, spec.tgv_u0, spec.finest_nx, spec.rho0, spec.tgv_offset)
    rho = np.full((ny, nx), spec.rho0)
    return rho, np.full((ny, nx), spec.u_in[0]), np.full((ny, nx), spec.u_in[1])


def random_fields(nx: int, ny: int, seed: int, amp_u: float = 0.02, amp_rho: float = 0.01, modes: int = 4):
    """Smooth random periodic rho, ux, uy (a few Fourier modes), seeded."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) / nx
    y = np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for amp, base in ((amp_rho, 1.0), (amp_u, 0.0), (amp_u, 0.0)):
        fld = np.full((ny, nx), base)
        for _ in range(modes):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * math.pi, size=2)
            fld = fld + amp / modes * rng.uniform(-1, 1) * np.cos(2 * math.pi * kx * X + ph[0]) * np.cos(
                2 * math.pi * ky * Y + ph[1])
        out.append(np.ascontiguousarray(fld))
    return out


# ---------------------------------------------------------------------------
# presets
# ---------------------------------------------------------------------------

def tgv(n: int = 128, tau: float = 0.8, u0: float = 0.02, steps: int = 1000, storage: int = F64,
        block: int = 16) -> DomainSpec:
    """Taylor-Green vortex, D2Q9 BGK, single level, n x n periodic."""
    return DomainSpec(name=f"tgv{n}", nx0=n, ny0=n, levels=1, block=block, tau_finest=tau, storage=storage,
                      steps=steps, init="tgv", tgv_u0=u0, tgv_offset=0.0)


def cylinder(D: int = 40, levels: int = 3, re: float = 100.0, u: float = 0.05, n_markers: int = 126,
             K: int = 5, storage: int = F32, block: int = 16, lx: float = 30.0, ly: float = 15.0,
             periods: float = 20.0, xc: float = 8.0) -> DomainSpec:
    """Flow past a circular cylinder: D finest cells, coarsest grid lx*D x ly*D
    (rounded up to whole blocks), equilibrium inlet W, open outlet E, symmetric
    N/S, refinement boxes around the body with a downstream wake extension."""
    h0 = 1 << (levels - 1)
    nx0 = _round_up(lx * D / h0, block)
    ny0 = _round_up(ly * D / h0, block)
    cx, cy = xc * D, ny0 * h0 / 2.0
    margin = [0.0] * 8
    wake = [0.0] * 8
    for l in range(1, levels):
        depth = levels - 1 - l  # 0 at the finest level
        margin[l] = 0.6 * D * (2 ** depth) + 8.0
        wake[l] = 3.0 * D * (2 ** depth)
    body = BodySpec(kind=0, a=D / 2.0, b=D / 2.0, n_markers=n_markers, motion=0, x0=(cx, cy), K=K, u_ref=u,
                    l_ref=float(D))
    St = 0.165
    period_fine = D / (St * u)
    steps = int(math.ceil(periods * period_fine / h0))
    return DomainSpec(name=f"cylinder_D{D}_m{levels}", nx0=nx0, ny0=ny0, levels=levels, block=block,
                      bc=(BC_INLET, BC_OUTLET, BC_SYMMETRY, BC_SYMMETRY), tau_finest=tau_from_re(u, D, re),
                      rho0=1.0, u_in=(u, 0.0), storage=storage, margin=tuple(margin), wake=tuple(wake), retag=0,
                      body=body, steps=steps)


def cylinder_table1(re: float = 300.0, D: int = 128, levels: int = 4, u: float = 0.1, storage: int = F32,
                    block: int = 16, lx: float = 150.0, ly: float = 100.0, xc: float = 50.0,
                    periods: float = 20.0) -> DomainSpec:
    """The stationary-cylinder study of Sec. 3.3 (Table 1, Re 100 / 300 /
    550): four levels with the finest spacing D / 128, free stream U = 0.1,
    markers one finest cell apart, a 100 D x 150 D domain (reading: 150 D
    streamwise, 100 D across, the cylinder 50 D from the inlet).  A static
    body: the IBM reuses its stored stencil geometry every step."""
    spec = cylinder(D=D, levels=levels, re=re, u=u, n_markers=int(round(math.pi * D)), storage=storage,
                    block=block, lx=lx, ly=ly, periods=periods, xc=xc)
    spec.name = f"cylinder_table1_Re{int(re)}_D{D}_m{levels}"
    return spec


def wing(c: int = 64, levels: int = 4, re: float = 157.0, amp_deg: float = 45.0, u_ref: float = 0.05,
         n_markers: int = 200, K: int = 5, storage: int = F32, block: int = 16, domain_chords: float = 50.0,
         periods: float = 1.0, thickness: float = 0.12, beta_deg: float = 60.0, heave_chords: float = 2.5,
         alpha_mean: float = math.pi / 2.0) -> DomainSpec:
    """Flapping ellipse wing (Sec. 3.6 kinematics): chord c finest cells,
    periodic square domain of domain_chords * c, refinement that follows the body."""
    h0 = 1 << (levels - 1)
    n0 = _round_up(domain_chords * c / h0, block)
    A0 = heave_chords * c
    # Sec. 3.6: T = 2.5 pi in units of c / U_ref; with A0 = 2.5 c the peak heave
    # speed pi A0 / T then equals U_ref
    T = 2.5 * math.pi * c / u_ref
    margin = [0.0] * 8
    wake = [0.0] * 8
    for l in range(1, levels):
        depth = levels - 1 - l
        margin[l] = 12.0 * (2 ** depth) + 6.0
    centre = n0 * h0 / 2.0
    body = BodySpec(kind=1, a=c / 2.0, b=thickness * c / 2.0, n_markers=n_markers, motion=2, x0=(centre, centre),
                    alpha_mean=alpha_mean, alpha_amp=math.radians(amp_deg), period=T, phase=0.0, heave_amp=A0,
                    beta=math.radians(beta_deg), K=K, u_ref=u_ref, l_ref=float(c))
    steps = int(math.ceil(periods * T / h0))
    return DomainSpec(name=f"wing_c{c}_m{levels}", nx0=n0, ny0=n0, levels=levels, block=block,
                      bc=(BC_PERIODIC,) * 4, tau_finest=tau_from_re(u_ref, c, re), rho0=1.0, u_in=(0.0, 0.0),
                      storage=storage, margin=tuple(margin), wake=tuple(wake), retag=1, body=body, steps=steps)


def _pitch_domain(name, c, levels, re, u, block, storage, lx, ly, x_le, body, steps, margin_c, wake_c):
    """Inlet W, open outlet E, symmetric N/S, coarsest grid lx c x ly c
    rounded to blocks (lx streamwise: reading of the paper's 40 x 70 chord
    domain of Sec. 3.4), body-following refinement."""
    h0 = 1 << (levels - 1)
    nx0 = _round_up(lx * c / h0, block)
    ny0 = _round_up(ly * c / h0, block)
    body.x0 = (x_le * c + body.a, ny0 * h0 / 2.0)
    margin = [0.0] * 8
    wake = [0.0] * 8
    for l in range(1, levels):
        depth = levels - 1 - l
        margin[l] = margin_c * c * (2 ** depth) + 8.0
        wake[l] = wake_c * c * (2 ** depth)
    return DomainSpec(name=name, nx0=nx0, ny0=ny0, levels=levels, block=block,
                      bc=(BC_INLET, BC_OUTLET, BC_SYMMETRY, BC_SYMMETRY), tau_finest=tau_from_re(u, c, re),
                      rho0=1.0, u_in=(u, 0.0), storage=storage, margin=tuple(margin), wake=tuple(wake), retag=1,
                      body=body, steps=steps)


def pitch_up(c: int = 64, levels: int = 3, re: float = 1000.0, u: float = 0.05, thickness: float = 0.023,
             amp: float = math.pi / 2.0, a_s: float = 11.0, rate: float = 0.2, t1: float = 1.0, t_end: float = 5.0,
             K: int = 5, storage: int = F32, block: int = 16, lx: float = 70.0, ly: float = 40.0,
             x_le: float = 20.0) -> DomainSpec:
    """Flat plate with square edges (Sec. 3.4): chord c finest cells,
    thickness 2.3 % of c, pitched up by ``amp`` about its leading edge with
    the smoothed ramp (Eqs. 20-21, a_s = 11, K = 0.2, t1* = 1), run to
    t* = t U / c = t_end.  Markers about one cell apart."""
    a, b = c / 2.0, thickness * c / 2.0
    n = max(8, int(round(4.0 * (a + b))))
    body = BodySpec(kind=2, a=a, b=b, n_markers=n, pivot=(-a, 0.0), motion=3, alpha_mean=0.0, alpha_amp=amp,
                    K=K, u_ref=u, l_ref=float(c), ramp_as=a_s, ramp_rate=rate, ramp_t1=t1, t_ref=c / u)
    h0 = 1 << (levels - 1)
    steps = int(math.ceil(t_end * c / u / h0))
    return _pitch_domain(f"pitch_up_c{c}_m{levels}", c, levels, re, u, block, storage, lx, ly, x_le, body, steps,
                         margin_c=0.25, wake_c=1.0)


def pitching_airfoil(c: int = 64, levels: int = 3, re: float = 1000.0, u: float = 0.05, thickness: float = 0.18,
                     k: float = 0.22, amp_deg: float = 64.0, xi: float = 0.5, acc: float = 0.15,
                     periods: float = 1.0, K: int = 5, storage: int = F32, block: int = 16, lx: float = 70.0,
                     ly: float = 40.0, x_le: float = 20.0, n_markers: int | None = None) -> DomainSpec:
    """Symmetric NACA section (NACA 0018 by default) in smoothed asymmetric
    triangular pitch (Sec. 3.5, Eqs. 22-24) about its quarter chord
    (reading), reduced frequency k = pi f c / U, so the period is
    T = pi c / (k U) finest steps; corner time 0.15 T."""
    a, b = c / 2.0, thickness * c / 2.0
    T = math.pi * c / (k * u)
    n = n_markers or max(8, int(round(2.08 * c)))  # perimeter of a 12-18 % section is about 2.05-2.08 c
    body = BodySpec(kind=3, a=a, b=b, n_markers=n, pivot=(-a / 2.0, 0.0), motion=4, alpha_mean=0.0,
                    alpha_amp=math.radians(amp_deg), period=T, phase=0.0, K=K, u_ref=u, l_ref=float(c), xi=xi,
                    acc=acc)
    h0 = 1 << (levels - 1)
    steps = int(math.ceil(periods * T / h0))
    return _pitch_domain(f"pitching_naca_c{c}_m{levels}", c, levels, re, u, block, storage, lx, ly, x_le, body,
                         steps, margin_c=0.25, wake_c=1.0)


def batch(n_instances: int = 64, seed: int = 0, storage: int = BF16DEV, block: int = 16, scale: float = 1.0):
    """Uneven cylinder / wing instances: coarsest nx in {256..2048} (times scale),
    ny = nx/2, 2-4 levels, Re ~ U[50, 400], pitch amplitude ~ U[16, 64] degrees."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        nx = int(rng.choice([256, 512, 1024, 2048]))
        levels = int(rng.choice([2, 3, 4]))
        kind = int(rng.integers(0, 2))
        re = float(rng.uniform(50.0, 400.0))
        amp = float(rng.uniform(16.0, 64.0))
        nxs = max(4 * block, _round_up(nx * scale, block))
        nys = max(4 * block, _round_up(nxs / 2, block))
        h0 = 1 << (levels - 1)
        if kind == 0:
            D = 40
            spec = cylinder(D=D, levels=levels, re=re, storage=storage, block=block, periods=1.0)
            spec = replace(spec, nx0=nxs, ny0=nys,
                           body=replace(spec.body, x0=(min(8.0 * D, 0.25 * nxs * h0), nys * h0 / 2.0)))
        else:
            c = 64
            spec = wing(c=c, levels=levels, re=re, amp_deg=amp, storage=storage, block=block, periods=1.0)
            spec = replace(spec, nx0=nxs, ny0=nys, body=replace(spec.body, x0=(nxs * h0 / 2.0, nys * h0 / 2.0)))
        spec.name = f"batch{k}_{'cyl' if kind == 0 else 'wing'}_{nxs}x{nys}_m{levels}"
        out.append(spec)
    return out


def cavity(L: int = 304, re: float = 100.0, u_lid: float = 0.05, d_frac: float = 0.4, mode: str = "bounce",
           storage: int = F32, block: int = 16, levels: int = 1, steps: int = 20000,
           n_markers: int | None = None) -> DomainSpec:
    """Lid-driven square cavity with a circular cylinder at its centre
    (Sec. 3.2): side L finest cells (the paper's 300 rounded to whole blocks),
    walls at rest on W, E, S, the lid N moving at u_lid, cylinder diameter
    d_frac L, Re = u_lid L / nu.  mode "bounce": the cylinder is a solid with
    interpolated bounce-back; "ibm": the cylinder is a static IBM body with
    markers about one cell apart (the comparison the paper makes)."""
    h0 = 1 << (levels - 1)
    n0 = _round_up(L / h0, block)
    side = n0 * h0
    c = side / 2.0
    R = d_frac * side / 2.0
    spec = DomainSpec(name=f"cavity_{mode}_L{side}_Re{int(re)}", nx0=n0, ny0=n0, levels=levels, block=block,
                      bc=(BC_WALL,) * 4, tau_finest=tau_from_re(u_lid, side, re), rho0=1.0, storage=storage,
                      uwall=(0.0,) * 6 + (u_lid, 0.0), steps=steps)
    if levels > 1:
        spec.boxes = [(levels - 1, c - R - 12.0, c - R - 12.0, c + R + 12.0, c + R + 12.0)]
    if mode == "bounce":
        spec.solid = (1, c, c, R)
    else:
        n = n_markers or int(round(2.0 * math.pi * R))
        spec.body = BodySpec(kind=0, a=R, b=R, n_markers=n, motion=0, x0=(c, c), u_ref=u_lid, l_ref=2.0 * R)
    return spec


def with_mrt(spec: DomainSpec, rates: tuple = (1.64, 1.54, 1.9)) -> DomainSpec:
    """``spec`` with the MRT collision (Sec. 2.1) in place of BGK."""
    return replace(spec, collision=1, mrt_rates=tuple(rates), boxes=list(spec.boxes),
                   body=replace(spec.body) if spec.body is not None else None)


def with_les(spec: DomainSpec, cs: float = 0.17) -> DomainSpec:
    """``spec`` with the LES collision (Sec. 2.1, Smagorinsky constant cs)."""
    return replace(spec, collision=2, les_cs=cs, boxes=list(spec.boxes),
                   body=replace(spec.body) if spec.body is not None else None)


def replace_storage(spec: DomainSpec, storage: int, block: int | None = None) -> DomainSpec:
    """A copy of ``spec`` with another population storage (the block size
    must stay the spec's: grids are whole blocks)."""
    if block is not None and block != spec.block:
        raise ValueError(f"{spec.name}: block {spec.block}, requested {block}")
    return replace(spec, storage=storage, boxes=list(spec.boxes),
                   body=replace(spec.body) if spec.body is not None else None)


def serving_arrivals(n_requests: int = 64, rate_per_s: float = 20.0, seed: int = 1):
    """Poisson arrival times (seconds) and the request mix, seeded."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    return np.cumsum(gaps), batch(n_requests, seed=seed + 1000)
