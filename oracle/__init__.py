"""FP64 CPU oracle of the SBoTFlow time step (arXiv 2402.04606).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product library
never imports, links or calls anything here, and nothing here imports the
product library.

The arithmetic lives in ``sbot_oracle.c`` (plain per-cell loops over dense
per-level arrays, one function per step of the paper).  This module compiles
it with gcc (``build()``) and wraps it with ctypes.  Array conventions: level
``l`` is a dense ``ny_l x nx_l`` grid (``nx_l = nx0 * 2**l``); populations are
``[9, ny_l, nx_l]`` float64 in the paper's direction order (Eq. 1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbot_oracle.c")
_LIBS = {False: os.path.join(_HERE, "libsbot_oracle.so"), True: os.path.join(_HERE, "libsbot_oracle_omp.so")}

T_NONE, T_INT, T_GF, T_GC, T_SOLID = 0, 1, 2, 3, 4
BC_PERIODIC, BC_INLET, BC_OUTLET, BC_SYMMETRY, BC_WALL = 0, 1, 2, 3, 4


def build(openmp: bool = False, force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so x86 and Arm agree)."""
    out = _LIBS[openmp]
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
           "-D_DEFAULT_SOURCE", "-o", out + ".tmp", _SRC, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)
    return out


_lib_cache: dict = {}


def lib(openmp: bool = False):
    if openmp in _lib_cache:
        return _lib_cache[openmp]
    L = C.CDLL(build(openmp))
    d, i, p, v, l = C.c_double, C.c_int, C.c_void_p, None, C.c_long
    dp = C.POINTER(C.c_double)
    sig = {
        "orc_feq": (d, [i, d, d, d]),
        "orc_guo": (d, [i, d, d, d, d, d]),
        "orc_collide_cell": (v, [dp, d, d, d, dp]),
        "orc_phi": (d, [d]),
        "orc_ibm_mdf": (i, [i, i, dp, dp, dp, i, dp, dp, dp, dp, dp, i, dp, dp, dp, dp]),
        "orc_place_markers": (d, [d, d, i, dp, dp]),
        "orc_create": (p, [i, i, i, i, C.POINTER(C.c_int), d, d, d, d]),
        "orc_destroy": (v, [p]),
        "orc_error": (C.c_char_p, [p]),
        "orc_level_dims": (i, [p, i, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "orc_level_tau": (d, [p, i]),
        "orc_add_box": (i, [p, i, d, d, d, d]),
        "orc_set_rescale": (i, [p, i]),
        "orc_set_iface": (i, [p, i]),
        "orc_rescale_neq": (v, [dp, d, dp]),
        "orc_set_refine_margins": (i, [p, dp, dp, i]),
        "orc_set_body": (i, [p, d, d, i, dp, i, dp, d, d, d, d, d, d, i]),
        "orc_body_markers": (i, [p, l, dp, dp]),
        "orc_set_body_ext": (i, [p, i, d, d, dp]),
        "orc_set_collision": (i, [p, i, dp]),
        "orc_set_walls": (i, [p, dp]),
        "orc_set_solid": (i, [p, i, dp]),
        "orc_wall_fraction": (d, [p, d, d, d, d]),
        "orc_in_solid": (i, [p, d, d]),
        "orc_mrt_matrix": (v, [dp]),
        "orc_collide_cell_mrt": (v, [dp, d, dp, d, d, dp]),
        "orc_collide_cell_les": (v, [dp, d, d, d, d, dp]),
        "orc_les_tau": (d, [dp, d, d, d, d]),
        "orc_body_pose": (i, [p, d, dp]),
        "orc_place_markers_kind": (d, [i, d, d, i, dp, dp]),
        "orc_ramp_alpha": (d, [d, d, d, d, d]),
        "orc_triangle_alpha": (d, [d, d, d, d, d]),
        "orc_body_ds": (d, [p]),
        "orc_build": (i, [p]),
        "orc_get_types": (i, [p, i, C.POINTER(C.c_ubyte)]),
        "orc_get_blocks": (i, [p, i, C.POINTER(C.c_ubyte)]),
        "orc_set_fields": (i, [p, i, dp, dp, dp]),
        "orc_set_populations": (i, [p, i, dp]),
        "orc_finalize_init": (i, [p]),
        "orc_retag_to": (i, [p, C.POINTER(C.POINTER(C.c_ubyte))]),
        "orc_step": (i, [p, i]),
        "orc_get_populations": (i, [p, i, dp]),
        "orc_get_post": (i, [p, i, dp]),
        "orc_get_fields": (i, [p, i, dp, dp, dp]),
        "orc_checksum": (i, [p, dp]),
        "orc_get_forces": (l, [p, dp, l]),
        "orc_fine_step": (l, [p]),
        "orc_coarse_step": (l, [p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib_cache[openmp] = L
    return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------------------
# single-cell formulas (Sec. 2.1) and the IBM operator (Sec. 2.2)
# ---------------------------------------------------------------------------

def feq(i: int, rho: float, ux: float, uy: float) -> float:
    return lib().orc_feq(i, rho, ux, uy)


def guo(i: int, tau: float, ux: float, uy: float, Fx: float, Fy: float) -> float:
    return lib().orc_guo(i, tau, ux, uy, Fx, Fy)


def collide_cell(f, tau: float, Fx: float = 0.0, Fy: float = 0.0) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_collide_cell(_dp(f), tau, Fx, Fy, _dp(out))
    return out


def mrt_matrix() -> np.ndarray:
    """The 9 x 9 moment matrix of the MRT collision (rows rho, e, eps, j_x,
    q_x, j_y, q_y, p_xx, p_xy)."""
    M = np.zeros(81)
    lib().orc_mrt_matrix(_dp(M))
    return M.reshape(9, 9)


def collide_cell_mrt(f, tau: float, s3, Fx: float = 0.0, Fy: float = 0.0) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    s = np.ascontiguousarray(s3, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_collide_cell_mrt(_dp(f), tau, _dp(s), Fx, Fy, _dp(out))
    return out


def collide_cell_les(f, tau: float, cs: float, Fx: float = 0.0, Fy: float = 0.0) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_collide_cell_les(_dp(f), tau, cs, Fx, Fy, _dp(out))
    return out


def phi(r: float) -> float:
    return lib().orc_phi(float(r))


def place_markers(a: float, b: float, n: int, kind: int | None = None):
    """Body-frame markers at equal arc length and the perimeter: kind 0
    circle, 1 ellipse (the default picks 0 or 1 from a == b), 2 rectangle,
    3 symmetric NACA four-digit airfoil."""
    qx, qy = np.zeros(n), np.zeros(n)
    if kind is None:
        P = lib().orc_place_markers(a, b, n, _dp(qx), _dp(qy))
    else:
        P = lib().orc_place_markers_kind(int(kind), a, b, n, _dp(qx), _dp(qy))
    return qx, qy, P


def ramp_alpha(A: float, a_s: float, K: float, t1: float, ts: float) -> float:
    """Pitch angle of the smoothed pitch-up ramp (Sec. 3.4, Eqs. 20-21)."""
    return lib().orc_ramp_alpha(A, a_s, K, t1, float(ts))


def triangle_alpha(a0: float, xi: float, acc: float, T: float, t: float) -> float:
    """Smoothed asymmetric triangular pitch angle (Sec. 3.5, Eqs. 22-24)."""
    return lib().orc_triangle_alpha(a0, xi, acc, T, float(t))


def ibm_mdf(rho, ux, uy, rx, ry, udx, udy, ds, K):
    """Multi-direct forcing on a dense grid; returns (ux, uy, Fx, Fy, Fjx, Fjy)."""
    rho = np.ascontiguousarray(rho, np.float64)
    ny, nx = rho.shape
    ux = np.array(ux, np.float64, copy=True, order="C")
    uy = np.array(uy, np.float64, copy=True, order="C")
    n = len(rx)
    arrs = [np.ascontiguousarray(a, np.float64) for a in (rx, ry, udx, udy)]
    ds = np.ascontiguousarray(np.broadcast_to(np.asarray(ds, np.float64), (n,)))
    Fx, Fy = np.zeros_like(rho), np.zeros_like(rho)
    Fjx, Fjy = np.zeros(n), np.zeros(n)
    rc = lib().orc_ibm_mdf(nx, ny, _dp(rho), _dp(ux), _dp(uy), n, *[_dp(a) for a in arrs], _dp(ds), int(K),
                           _dp(Fx), _dp(Fy), _dp(Fjx), _dp(Fjy))
    if rc != 0:
        raise ValueError("IBM stencil outside the grid")
    return ux, uy, Fx, Fy, Fjx, Fjy


# ---------------------------------------------------------------------------
# a whole domain
# ---------------------------------------------------------------------------

@dataclass
class Body:
    a: float
    b: float
    n_markers: int
    pivot: tuple = (0.0, 0.0)
    motion: int = 0
    x0: tuple = (0.0, 0.0)
    alpha_mean: float = 0.0
    alpha_amp: float = 0.0
    period: float = 1.0
    phase: float = 0.0
    heave_amp: float = 0.0
    beta: float = 0.0
    K: int = 5
    kind: int | None = None  # None: circle or ellipse from a == b; 2 rectangle; 3 NACA 00xx
    ramp_as: float = 11.0  # motion 3 (Sec. 3.4): a_s, pitch rate K, t1*, finest steps per unit of t*
    ramp_rate: float = 0.2
    ramp_t1: float = 1.0
    t_ref: float = 1.0
    xi: float = 0.5  # motion 4 (Sec. 3.5): asymmetry, corner time / period
    acc: float = 0.15


@dataclass
class Domain:
    nx0: int
    ny0: int
    levels: int = 1
    block: int = 16
    bc: tuple = (BC_PERIODIC,) * 4  # W, E, S, N
    tau_finest: float = 0.8
    rho0: float = 1.0
    u_in: tuple = (0.0, 0.0)
    boxes: list = field(default_factory=list)  # (level, x0, y0, x1, y1) finest units
    margin: tuple = (0.0,) * 8  # per level, body-following refinement
    wake: tuple = (0.0,) * 8
    retag: int = 0
    rescale: int = 0  # reading R3b: f^neq rescaling at level changes (only meaningful with iface=0)
    iface: int = 1  # 1 volumetric coalescence (R3c, default), 0 overlapping coarse ghost layer (R3a)
    coll: int = 0  # 0 BGK (Eq. 6), 1 MRT, 2 LES (Smagorinsky constant in mrt_s[0])
    mrt_s: tuple = (1.64, 1.54, 1.9)  # s_e, s_eps, s_q of the MRT collision
    uwall: tuple = (0.0,) * 8  # per side W, E, S, N: velocity (x, y) of a wall side
    solid: tuple = (0, 0.0, 0.0, 0.0)  # kind (0 none, 1 circle cx cy R, 2 half-plane y < y0), parameters


class Oracle:
    """One domain of the FP64 oracle."""

    def __init__(self, dom: Domain, body: Body | None = None, openmp: bool = False):
        self.L = lib(openmp)
        self.dom = dom
        bc = (C.c_int * 4)(*dom.bc)
        self.h = self.L.orc_create(dom.nx0, dom.ny0, dom.levels, dom.block, bc, dom.tau_finest, dom.rho0,
                                   dom.u_in[0], dom.u_in[1])
        if not self.h:
            raise ValueError("oracle: invalid domain description")
        self.L.orc_set_rescale(self.h, int(dom.rescale))
        self.L.orc_set_iface(self.h, int(dom.iface))
        if self.L.orc_set_collision(self.h, int(dom.coll), _dp(np.array(dom.mrt_s, np.float64))) != 0:
            raise ValueError("oracle: bad collision kind")
        self.L.orc_set_walls(self.h, _dp(np.array(dom.uwall, np.float64)))
        if self.L.orc_set_solid(self.h, int(dom.solid[0]), _dp(np.array(dom.solid[1:4], np.float64))) != 0:
            raise ValueError("oracle: bad solid kind")
        for (lv, x0, y0, x1, y1) in dom.boxes:
            self.L.orc_add_box(self.h, int(lv), x0, y0, x1, y1)
        mg = np.ascontiguousarray(np.array(list(dom.margin) + [0.0] * (8 - len(dom.margin)), np.float64)[:8])
        wk = np.ascontiguousarray(np.array(list(dom.wake) + [0.0] * (8 - len(dom.wake)), np.float64)[:8])
        self.L.orc_set_refine_margins(self.h, _dp(mg), _dp(wk), int(dom.retag))
        self.body = body
        if body is not None:
            pv = np.array(body.pivot, np.float64)
            x0 = np.array(body.x0, np.float64)
            self.L.orc_set_body(self.h, body.a, body.b, body.n_markers, _dp(pv), body.motion, _dp(x0),
                                body.alpha_mean, body.alpha_amp, body.period, body.phase, body.heave_amp,
                                body.beta, body.K)
            if body.kind is not None or body.motion >= 3:
                kind = body.kind if body.kind is not None else (0 if body.a == body.b else 1)
                ext = np.array([body.ramp_as, body.ramp_rate, body.ramp_t1, body.t_ref, body.xi, body.acc],
                               np.float64)
                if self.L.orc_set_body_ext(self.h, int(kind), body.a, body.b, _dp(ext)) != 0:
                    raise ValueError("oracle: invalid body kind")
        self._check(self.L.orc_build(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_destroy(self.h)
            self.h = None

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError("oracle: " + self.L.orc_error(self.h).decode())

    # geometry ---------------------------------------------------------------
    def dims(self, level: int):
        nx, ny = C.c_int(), C.c_int()
        self.L.orc_level_dims(self.h, level, C.byref(nx), C.byref(ny))
        return nx.value, ny.value

    def tau(self, level: int) -> float:
        return self.L.orc_level_tau(self.h, level)

    def types(self, level: int) -> np.ndarray:
        nx, ny = self.dims(level)
        out = np.zeros((ny, nx), np.uint8)
        self.L.orc_get_types(self.h, level, out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return out

    def blocks(self, level: int) -> np.ndarray:
        nx, ny = self.dims(level)
        B = self.dom.block
        out = np.zeros((ny // B, nx // B), np.uint8)
        self.L.orc_get_blocks(self.h, level, out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return out

    def markers(self, fine_step: int):
        n = self.body.n_markers
        rx, ry = np.zeros(n), np.zeros(n)
        self.L.orc_body_markers(self.h, fine_step, _dp(rx), _dp(ry))
        return rx, ry

    def ds(self) -> float:
        return self.L.orc_body_ds(self.h)

    def wall_fraction(self, px: float, py: float, ex: float, ey: float) -> float:
        """fraction of the link (px, py) -> (px + ex, py + ey) outside the solid"""
        return self.L.orc_wall_fraction(self.h, px, py, ex, ey)

    def in_solid(self, px: float, py: float) -> bool:
        return bool(self.L.orc_in_solid(self.h, px, py))

    def pose(self, t: float):
        """(centre x, centre y, rotation angle) of the body at finest time t."""
        out = np.zeros(3)
        self.L.orc_body_pose(self.h, float(t), _dp(out))
        return out

    # state ------------------------------------------------------------------
    def set_fields(self, level, rho, ux, uy):
        nx, ny = self.dims(level)
        a = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (ny, nx))) for v in (rho, ux, uy)]
        self.L.orc_set_fields(self.h, level, *[_dp(x) for x in a])

    def set_populations(self, level, f):
        f = np.ascontiguousarray(f, np.float64)
        self.L.orc_set_populations(self.h, level, _dp(f))

    def finalize_init(self):
        self._check(self.L.orc_finalize_init(self.h))

    def retag_to(self, new_blocks: list):
        arrs = [np.ascontiguousarray(b, np.uint8) for b in new_blocks]
        ptrs = (C.POINTER(C.c_ubyte) * len(arrs))(*[a.ctypes.data_as(C.POINTER(C.c_ubyte)) for a in arrs])
        self._check(self.L.orc_retag_to(self.h, ptrs))

    def step(self, n: int = 1):
        self._check(self.L.orc_step(self.h, int(n)))

    def populations(self, level: int) -> np.ndarray:
        nx, ny = self.dims(level)
        out = np.zeros((9, ny, nx))
        self.L.orc_get_populations(self.h, level, _dp(out))
        return out

    def post_collision(self, level: int) -> np.ndarray:
        nx, ny = self.dims(level)
        out = np.zeros((9, ny, nx))
        self.L.orc_get_post(self.h, level, _dp(out))
        return out

    def fields(self, level: int):
        nx, ny = self.dims(level)
        rho, ux, uy = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
        self.L.orc_get_fields(self.h, level, _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def checksum(self) -> np.ndarray:
        out = np.zeros(3)
        self.L.orc_checksum(self.h, _dp(out))
        return out

    def forces(self) -> np.ndarray:
        cap = max(1, int(self.L.orc_fine_step(self.h)) + 1)
        out = np.zeros((cap, 3))
        n = self.L.orc_get_forces(self.h, _dp(out), cap)
        return out[:n].copy()

    @property
    def fine_step(self) -> int:
        return int(self.L.orc_fine_step(self.h))

    @property
    def coarse_step(self) -> int:
        return int(self.L.orc_coarse_step(self.h))
