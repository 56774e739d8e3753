"""ctypes binding of the C ABI in include/sbot.h -- argument marshalling only.

Every computation runs in the CUDA kernels of ``libsbot.so``; this module
converts numpy arrays and dataclasses to the ABI's plain pointers and
structs.  There is no CPU fallback: without the built library or without a
CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsbot.so")
HEADER = os.path.join(_HERE, "..", "include", "sbot.h")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_STATE = range(7)
TUNE_VECTOR_MIN_CELLS = 0
TUNE_STAGED = 1
TUNE_PDL = 2
TUNE_PERSISTENT = 3
TUNE_STEP_THREADS = 4
TUNE_SPIN_NS = 5
TUNE_BULK_ROUNDS = 6
TUNE_IBM_THREADS = 7
TUNE_CRIT_BLOCKS = 8
TUNE_STEPS_PER_LAUNCH = 9
TUNE_VEC_WAVES = 10
STEP_MAX_PHASES = 512
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_NONFINITE", 6: "ERR_STATE"}


class SbotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sbot_box(C.Structure):
    _fields_ = [("level", C.c_int), ("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double),
                ("y1", C.c_double)]


class sbot_domain_desc(C.Structure):
    _fields_ = [("nx0", C.c_int), ("ny0", C.c_int), ("levels", C.c_int), ("block", C.c_int),
                ("bc", C.c_int * 4), ("tau_finest", C.c_double), ("rho0", C.c_double), ("u_in", C.c_double * 2),
                ("storage", C.c_int), ("ibm_iters", C.c_int), ("retag", C.c_int),
                ("refine_margin", C.c_double * 8), ("refine_wake", C.c_double * 8), ("n_boxes", C.c_int),
                ("boxes", C.POINTER(sbot_box)), ("collision", C.c_int), ("mrt_rates", C.c_double * 3),
                ("les_cs", C.c_double),
                ("wall_velocity", C.c_double * 8), ("solid_kind", C.c_int), ("solid", C.c_double * 3)]


class sbot_body_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("b", C.c_double), ("n_markers", C.c_int),
                ("pivot", C.c_double * 2), ("motion", C.c_int), ("x0", C.c_double * 2),
                ("alpha_mean", C.c_double), ("alpha_amp", C.c_double), ("period", C.c_double),
                ("phase", C.c_double), ("heave_amp", C.c_double), ("stroke_beta", C.c_double),
                ("u_ref", C.c_double), ("l_ref", C.c_double),
                ("ramp_as", C.c_double), ("ramp_rate", C.c_double), ("ramp_t1", C.c_double), ("t_ref", C.c_double),
                ("asym_xi", C.c_double), ("accel_frac", C.c_double)]


_lib = None


def header_functions() -> list:
    """Names of every function the ABI header declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:sbot_status|const char\*)\s+(sbot_\w+)\s*\(", text, re.M)))


def load():
    """Load the in-tree library (build it first with ``build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"the CUDA library is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    i, d, p, i64 = C.c_int, C.c_double, C.c_void_p, C.c_int64
    dp, u8p, ip, i64p = C.POINTER(C.c_double), C.POINTER(C.c_uint8), C.POINTER(C.c_int), C.POINTER(C.c_int64)
    sig = {
        "sbot_create_domain": [C.POINTER(sbot_domain_desc), p, C.POINTER(p)],
        "sbot_set_body_kinematics": [p, C.POINTER(sbot_body_desc)],
        "sbot_set_fields": [p, i, dp, dp, dp],
        "sbot_set_populations": [p, i, dp],
        "sbot_step": [p, i],
        "sbot_get_forces": [p, dp, dp, dp, ip],
        "sbot_get_fields": [p, i, dp, dp, dp, i64p],
        "sbot_get_populations": [p, i, dp, i64p],
        "sbot_get_celltypes": [p, i, u8p, i64p],
        "sbot_get_topology": [p, i, u8p, ip],
        "sbot_get_checksum": [p, dp],
        "sbot_get_checksum_noalloc": [p, dp],
        "sbot_get_level_info": [p, i, ip, ip, i64p],
        "sbot_get_work": [p, i64p, i64p],
        "sbot_plan_blocks": [C.POINTER(sbot_domain_desc), C.POINTER(sbot_body_desc), i64, i, u8p, ip],
        "sbot_set_profiling": [p, i],
        "sbot_get_profile": [p, i, i64p, dp, dp],
        "sbot_get_step_trace": [p, ip, ip, ip, ip, ip, dp],
        "sbot_destroy": [p],
        "sbot_batch_create": [i, i, i, i64, p, C.POINTER(p)],
        "sbot_batch_admit": [p, C.POINTER(sbot_domain_desc), C.POINTER(sbot_body_desc), ip],
        "sbot_batch_retire": [p, i],
        "sbot_batch_step": [p, i],
        "sbot_batch_select": [p, i],
        "sbot_batch_info": [p, ip, i64p, i64p, i64p],
        "sbot_set_tuning": [p, i, i64],
        "sbot_get_tuning": [p, i, i64p],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.sbot_last_error.argtypes = [p]
    L.sbot_last_error.restype = C.c_char_p
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def domain_desc(spec: wl.DomainSpec):
    boxes = (sbot_box * max(1, len(spec.boxes)))()
    for k, (lv, x0, y0, x1, y1) in enumerate(spec.boxes):
        boxes[k] = sbot_box(int(lv), x0, y0, x1, y1)
    d = sbot_domain_desc()
    d.nx0, d.ny0, d.levels, d.block = spec.nx0, spec.ny0, spec.levels, spec.block
    for k in range(4):
        d.bc[k] = int(spec.bc[k])
    d.tau_finest, d.rho0 = spec.tau_finest, spec.rho0
    d.u_in[0], d.u_in[1] = spec.u_in
    d.storage = int(spec.storage)
    d.ibm_iters = spec.body.K if spec.body is not None else 5
    d.retag = int(spec.retag)
    for k in range(8):
        d.refine_margin[k] = spec.margin[k] if k < len(spec.margin) else 0.0
        d.refine_wake[k] = spec.wake[k] if k < len(spec.wake) else 0.0
    d.n_boxes = len(spec.boxes)
    d.boxes = C.cast(boxes, C.POINTER(sbot_box))
    d.collision = int(spec.collision)
    for k in range(3):
        d.mrt_rates[k] = spec.mrt_rates[k]
    d.les_cs = spec.les_cs
    for k in range(8):
        d.wall_velocity[k] = spec.uwall[k]
    d.solid_kind = int(spec.solid[0])
    for k in range(3):
        d.solid[k] = spec.solid[1 + k]
    return d, boxes


def body_desc(b: wl.BodySpec):
    o = sbot_body_desc()
    o.kind, o.a, o.b, o.n_markers = b.kind, b.a, b.b, b.n_markers
    o.pivot[0], o.pivot[1] = b.pivot
    o.motion = b.motion
    o.x0[0], o.x0[1] = b.x0
    o.alpha_mean, o.alpha_amp, o.period, o.phase = b.alpha_mean, b.alpha_amp, b.period, b.phase
    o.heave_amp, o.stroke_beta, o.u_ref, o.l_ref = b.heave_amp, b.beta, b.u_ref, b.l_ref
    o.ramp_as, o.ramp_rate, o.ramp_t1, o.t_ref = b.ramp_as, b.ramp_rate, b.ramp_t1, b.t_ref
    o.asym_xi, o.accel_frac = b.xi, b.acc
    return o


def plan_blocks(spec: wl.DomainSpec, level: int, coarse_step: int = 0) -> np.ndarray:
    """Host-only topology plan of the library (no GPU needed)."""
    L = load()
    d, keep = domain_desc(spec)
    bd = body_desc(spec.body) if spec.body is not None else None
    nbx = (spec.nx0 << level) // spec.block
    nby = (spec.ny0 << level) // spec.block
    out = np.zeros((nby, nbx), np.uint8)
    n = C.c_int(out.size)
    rc = L.sbot_plan_blocks(C.byref(d), C.byref(bd) if bd is not None else None, coarse_step, level,
                            out.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(n))
    if rc != OK:
        raise SbotError(rc, "sbot_plan_blocks failed")
    return out


class _InstanceCalls:
    """Calls that address one instance of a context (see the header's
    per-instance calls); subclasses say which instance by ``_select``."""

    L = None
    h = None
    spec = None

    def _select(self):
        pass

    def _check(self, rc):
        if rc != OK:
            raise SbotError(rc, self.L.sbot_last_error(self.h).decode())

    def dims(self, level: int):
        self._select()
        nx, ny, ni = C.c_int(), C.c_int(), C.c_int64()
        self._check(self.L.sbot_get_level_info(self.h, level, C.byref(nx), C.byref(ny), C.byref(ni)))
        return nx.value, ny.value

    def n_interior(self, level: int) -> int:
        self._select()
        nx, ny, ni = C.c_int(), C.c_int(), C.c_int64()
        self._check(self.L.sbot_get_level_info(self.h, level, C.byref(nx), C.byref(ny), C.byref(ni)))
        return ni.value

    def work(self):
        self._select()
        a, b = C.c_int64(), C.c_int64()
        self._check(self.L.sbot_get_work(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_fields(self, level, rho, ux, uy):
        self._select()
        nx, ny = self.dims(level)
        a = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, np.float64), (ny, nx))) for v in (rho, ux, uy)]
        self._check(self.L.sbot_set_fields(self.h, level, *[_dp(x) for x in a]))

    def set_populations(self, level, f):
        self._select()
        f = np.ascontiguousarray(f, np.float64)
        self._check(self.L.sbot_set_populations(self.h, level, _dp(f)))

    def populations(self, level: int) -> np.ndarray:
        self._select()
        nx, ny = self.dims(level)
        out = np.zeros((9, ny, nx))
        n = C.c_int64(out.size)
        self._check(self.L.sbot_get_populations(self.h, level, _dp(out), C.byref(n)))
        return out

    def fields(self, level: int):
        self._select()
        nx, ny = self.dims(level)
        rho, ux, uy = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
        n = C.c_int64(nx * ny)
        self._check(self.L.sbot_get_fields(self.h, level, _dp(rho), _dp(ux), _dp(uy), C.byref(n)))
        return rho, ux, uy

    def types(self, level: int) -> np.ndarray:
        self._select()
        nx, ny = self.dims(level)
        out = np.zeros((ny, nx), np.uint8)
        n = C.c_int64(out.size)
        self._check(self.L.sbot_get_celltypes(self.h, level, out.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(n)))
        return out

    def blocks(self, level: int) -> np.ndarray:
        self._select()
        nx, ny = self.dims(level)
        B = self.spec.block
        out = np.zeros((ny // B, nx // B), np.uint8)
        n = C.c_int(out.size)
        self._check(self.L.sbot_get_topology(self.h, level, out.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(n)))
        return out

    def checksum(self) -> np.ndarray:
        self._select()
        out = np.zeros(3)
        self._check(self.L.sbot_get_checksum(self.h, _dp(out)))
        return out

    def checksum_noalloc(self) -> np.ndarray:
        """sbot_get_checksum without device allocation (static scratch)."""
        self._select()
        out = np.zeros(3)
        self._check(self.L.sbot_get_checksum_noalloc(self.h, _dp(out)))
        return out

    def forces(self, cap: int = 1 << 20) -> np.ndarray:
        self._select()
        fx, fy, mz = np.zeros(cap), np.zeros(cap), np.zeros(cap)
        n = C.c_int(cap)
        self._check(self.L.sbot_get_forces(self.h, _dp(fx), _dp(fy), _dp(mz), C.byref(n)))
        k = n.value
        return np.stack([fx[:k], fy[:k], mz[:k]], axis=1)


PHASE_KINDS = ("pose", "ibm_geometry", "c2f_copy", "sweep", "ibm", "force_sums")


def _step_trace(obj) -> list:
    n = C.c_int(STEP_MAX_PHASES)
    arrs = [np.zeros(STEP_MAX_PHASES, np.int32) for _ in range(4)]
    us4 = np.zeros(4 * STEP_MAX_PHASES)
    ptrs = [a.ctypes.data_as(C.POINTER(C.c_int)) for a in arrs]
    obj._check(obj.L.sbot_get_step_trace(obj.h, C.byref(n), *ptrs, _dp(us4)))
    k = n.value
    return [{"kind": PHASE_KINDS[arrs[0][i]], "level": int(arrs[1][i]), "bulk": int(arrs[2][i]),
             "tasks": int(arrs[3][i]), "start_us": float(us4[4 * i]), "last_start_us": float(us4[4 * i + 1]),
             "first_end_us": float(us4[4 * i + 2]), "end_us": float(us4[4 * i + 3])} for i in range(k)]


class Domain(_InstanceCalls):
    """One simulation instance on the GPU (wraps an sbot_ctx_t)."""

    def __init__(self, spec: wl.DomainSpec, stream=None):
        import torch  # device and stream plumbing only

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the library has no CPU path")
        self.L = load()
        self.spec = spec
        if stream is None:
            # a dedicated stream: the legacy default stream cannot be captured into CUDA graphs
            stream = torch.cuda.Stream()
        self.stream = stream
        handle = getattr(stream, "cuda_stream", stream)
        d, self._boxes = domain_desc(spec)
        h = C.c_void_p()
        rc = self.L.sbot_create_domain(C.byref(d), C.c_void_p(handle), C.byref(h))
        if rc != OK:
            raise SbotError(rc, "sbot_create_domain failed")
        self.h = h
        if spec.body is not None:
            self._check(self.L.sbot_set_body_kinematics(self.h, C.byref(body_desc(spec.body))))

    def close(self):
        if getattr(self, "h", None):
            self.L.sbot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._check(self.L.sbot_step(self.h, int(n)))

    def sync(self):
        """wait for the work queued on the instance's stream"""
        self.stream.synchronize()

    def set_profiling(self, mask: int):
        self._check(self.L.sbot_set_profiling(self.h, int(mask)))

    def profile(self, kind: int):
        n, ms, b = C.c_int64(), C.c_double(), C.c_double()
        self._check(self.L.sbot_get_profile(self.h, kind, C.byref(n), C.byref(ms), C.byref(b)))
        return n.value, ms.value, b.value

    def set_tuning(self, what: int, value: int):
        self._check(self.L.sbot_set_tuning(self.h, int(what), int(value)))

    def tuning(self, what: int) -> int:
        v = C.c_int64()
        self._check(self.L.sbot_get_tuning(self.h, int(what), C.byref(v)))
        return v.value

    def step_trace(self) -> list:
        """phases of the last traced persistent step (profiling mask bit 16)"""
        return _step_trace(self)


class Batch:
    """Many instances stepped together (sbot_batch_*): one launch per phase
    of the time step covers the blocks of every live instance."""

    def __init__(self, max_instances: int, block: int = 16, storage: int = wl.F32, budget_bytes: int = 0,
                 stream=None):
        import torch  # device and stream plumbing only

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the library has no CPU path")
        self.L = load()
        self.block, self.storage = block, storage
        self.stream = stream if stream is not None else torch.cuda.Stream()
        handle = getattr(self.stream, "cuda_stream", self.stream)
        h = C.c_void_p()
        rc = self.L.sbot_batch_create(int(max_instances), int(block), int(storage), int(budget_bytes),
                                      C.c_void_p(handle), C.byref(h))
        if rc != OK:
            raise SbotError(rc, "sbot_batch_create failed")
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise SbotError(rc, self.L.sbot_last_error(self.h).decode())

    def admit(self, spec: wl.DomainSpec) -> "BatchInstance":
        """Admit ``spec`` (its block and storage must be the batch's);
        raises SbotError with status ERR_OOM when it does not fit."""
        d, keep = domain_desc(spec)
        bd = body_desc(spec.body) if spec.body is not None else None
        slot = C.c_int(-1)
        self._check(self.L.sbot_batch_admit(self.h, C.byref(d), C.byref(bd) if bd is not None else None,
                                            C.byref(slot)))
        return BatchInstance(self, slot.value, spec)

    def retire(self, inst: "BatchInstance"):
        self._check(self.L.sbot_batch_retire(self.h, inst.slot))
        inst.slot = -1

    def step(self, n: int = 1):
        self._check(self.L.sbot_batch_step(self.h, int(n)))

    def info(self) -> dict:
        live, b, cu, st = C.c_int(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.L.sbot_batch_info(self.h, C.byref(live), C.byref(b), C.byref(cu), C.byref(st)))
        return {"live": live.value, "bytes": b.value, "cell_updates_per_step": cu.value}

    def set_profiling(self, mask: int):
        self._check(self.L.sbot_set_profiling(self.h, int(mask)))

    def profile(self, kind: int):
        n, ms, b = C.c_int64(), C.c_double(), C.c_double()
        self._check(self.L.sbot_get_profile(self.h, kind, C.byref(n), C.byref(ms), C.byref(b)))
        return n.value, ms.value, b.value

    def set_tuning(self, what: int, value: int):
        self._check(self.L.sbot_set_tuning(self.h, int(what), int(value)))

    def tuning(self, what: int) -> int:
        v = C.c_int64()
        self._check(self.L.sbot_get_tuning(self.h, int(what), C.byref(v)))
        return v.value

    def step_trace(self) -> list:
        """phases of the last traced persistent step (profiling mask bit 16)"""
        return _step_trace(self)

    def close(self):
        if getattr(self, "h", None):
            self.L.sbot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchInstance(_InstanceCalls):
    """One instance of a Batch: the per-instance calls select it first."""

    def __init__(self, batch: Batch, slot: int, spec: wl.DomainSpec):
        self.batch, self.slot, self.spec = batch, slot, spec
        self.L, self.h = batch.L, batch.h

    def _select(self):
        if self.slot < 0:
            raise RuntimeError("this instance was retired")
        self._check(self.L.sbot_batch_select(self.h, self.slot))

    def _check(self, rc):
        if rc != OK:
            raise SbotError(rc, self.L.sbot_last_error(self.h).decode())

    def coarse_steps(self) -> int:
        self._select()
        live, b, cu, st = C.c_int(), C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.L.sbot_batch_info(self.h, C.byref(live), C.byref(b), C.byref(cu), C.byref(st)))
        return st.value
