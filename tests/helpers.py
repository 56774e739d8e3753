"""Glue between workload specs and the two implementations (tests only)."""
from __future__ import annotations

import numpy as np

import oracle as orc
from paper_2402_04606_gb300 import workloads as wl
from paper_2402_04606_gb300.workloads import initial_fields  # noqa: F401  (re-exported for the tests)


def oracle_from_spec(spec: wl.DomainSpec, openmp: bool = False) -> orc.Oracle:
    dom = orc.Domain(nx0=spec.nx0, ny0=spec.ny0, levels=spec.levels, block=spec.block, bc=tuple(spec.bc),
                     tau_finest=spec.tau_finest, rho0=spec.rho0, u_in=tuple(spec.u_in), boxes=list(spec.boxes),
                     margin=tuple(spec.margin), wake=tuple(spec.wake), retag=spec.retag, coll=spec.collision,
                     mrt_s=(spec.les_cs, 0.0, 0.0) if spec.collision == 2 else tuple(spec.mrt_rates),
                     uwall=tuple(spec.uwall), solid=tuple(spec.solid))
    body = None
    if spec.body is not None:
        b = spec.body
        body = orc.Body(a=b.a, b=b.b, n_markers=b.n_markers, pivot=tuple(b.pivot), motion=b.motion,
                        x0=tuple(b.x0), alpha_mean=b.alpha_mean, alpha_amp=b.alpha_amp, period=b.period,
                        phase=b.phase, heave_amp=b.heave_amp, beta=b.beta, K=b.K,
                        kind=b.kind if b.kind >= 2 else None, ramp_as=b.ramp_as, ramp_rate=b.ramp_rate,
                        ramp_t1=b.ramp_t1, t_ref=b.t_ref, xi=b.xi, acc=b.acc)
    return orc.Oracle(dom, body, openmp=openmp)


def init_oracle(o: orc.Oracle, spec: wl.DomainSpec):
    for l in range(spec.levels):
        o.set_fields(l, *initial_fields(spec, l))
    o.finalize_init()
    return o


def rel_l2(a, b, mask=None):
    a = np.asarray(a)
    b = np.asarray(b)
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def small_pitch_specs():
    """A flat plate in a fast pitch-up ramp and a NACA section in triangular
    pitch, small enough for the oracle (Sec. 3.4, Sec. 3.5)."""
    p = wl.pitch_up(c=16, levels=3, block=8, lx=14.0, ly=12.0, x_le=5.0)
    p.body.t_ref = 48.0  # the ramp within the first coarse steps (trailing edge at up to 0.13 per step)
    p.body.ramp_t1 = 0.25
    a = wl.pitching_airfoil(c=16, levels=3, block=8, lx=14.0, ly=12.0, x_le=5.0, amp_deg=40.0)
    a.body.period = 480.0
    return [p, a]
