"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 storage -- relative L2 of the populations <= 1e-12 after
the stated number of steps (all levels); FP32 storage -- relative L2 of the
velocity <= 1e-5 (arithmetic in FP32: ~1e-7 per step, growing slowly with the
number of steps).  Integer work (topology, cell kinds) is compared exactly.
"""
import math

import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl
from tests.helpers import init_oracle, oracle_from_spec, rel_l2, small_pitch_specs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_U = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()


def gpu_domain(spec):
    from paper_2402_04606_gb300.native import Domain

    from tests.helpers import initial_fields

    g = Domain(spec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    return g


def compare_populations(g, o, levels, tol):
    for l in range(levels):
        t = o.types(l)
        assert np.array_equal(g.types(l), t), f"cell kinds differ on level {l}"
        mask = t == 1
        if not mask.any():
            continue
        fg, fo = g.populations(l), o.populations(l)
        err = rel_l2(fg[:, mask], fo[:, mask])
        assert err <= tol, f"level {l}: rel L2 {err:.3e} > {tol}"


def compare_forces(fg, fo, radius):
    # force and moment histories; the tolerance scales with the force level.
    # The GPU runs the K iterations of Eq. 11 as gathers over per-marker
    # stencils and per-cell marker lists (the oracle's arithmetic in another
    # rounding order), and Eq. 16 sums marker forces that largely cancel, so
    # round-off of 1e-16 reaches ~1e-12 of the force scale (the moment of a
    # symmetric body is zero up to round-off of r - r_pivot)
    assert fg.shape == fo.shape
    assert np.isfinite(fo).all()
    scale = np.abs(fo[:, :2]).max()
    np.testing.assert_allclose(fg[:, :2], fo[:, :2], rtol=1e-10, atol=1e-11 * scale)
    np.testing.assert_allclose(fg[:, 2], fo[:, 2], rtol=1e-10, atol=1e-11 * scale * radius)


def velocity_error(g, o, levels):
    num = den = 0.0
    for l in range(levels):
        mask = o.types(l) == 1
        _, ug, vg = g.fields(l)
        _, uo, vo = o.fields(l)
        num += (((ug - uo) ** 2 + (vg - vo) ** 2)[mask]).sum()
        den += ((uo ** 2 + vo ** 2)[mask]).sum()
    return math.sqrt(num / den)


@pytest.mark.parametrize("n,block", [(128, 16), (96, 8), (64, 32)])
def test_tgv_fp64_matches_oracle(n, block):
    spec = wl.tgv(n=n, block=block, steps=100)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    # the state at t = 0 comes back as set (each side evaluates Eq. 7 itself)
    np.testing.assert_allclose(g.populations(0), o.populations(0), rtol=1e-15, atol=0)
    o.step(100)
    g.step(100)
    compare_populations(g, o, 1, TOL64)
    cg, co = g.checksum(), o.checksum()
    assert abs(cg[0] - co[0]) / co[0] < 1e-13
    assert np.allclose(cg[1:], co[1:], atol=1e-12 * co[0])


def test_ragged_rectangle_fp64():
    spec = wl.DomainSpec("rect", 48, 24, levels=1, block=8, tau_finest=0.6)
    rng = np.random.default_rng(2)
    rho, ux, uy = wl.random_fields(48, 24, seed=9)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux, uy)
    o.finalize_init()
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    g.set_fields(0, rho, ux, uy)
    o.step(37)
    g.step(37)
    compare_populations(g, o, 1, TOL64)


def test_single_block_periodic_domain():
    spec = wl.DomainSpec("one", 8, 8, levels=1, block=8, tau_finest=0.9)
    rho, ux, uy = wl.random_fields(8, 8, seed=4)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux, uy)
    o.finalize_init()
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    g.set_fields(0, rho, ux, uy)
    o.step(20)
    g.step(20)
    compare_populations(g, o, 1, TOL64)


def test_boundaries_fp64():
    # equilibrium inlet W, open outlet E, symmetry S/N, with a perturbed interior
    spec = wl.DomainSpec("bc", 64, 32, levels=1, block=16, bc=(1, 2, 3, 3), tau_finest=0.6, u_in=(0.05, 0.0))
    rho, ux, uy = wl.random_fields(64, 32, seed=6)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux + 0.05, uy)
    o.finalize_init()
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    g.set_fields(0, rho, ux + 0.05, uy)
    o.step(80)
    g.step(80)
    compare_populations(g, o, 1, TOL64)


@pytest.mark.parametrize("levels,block", [(2, 8), (3, 8), (3, 16)])
def test_refined_periodic_fp64(levels, block):
    n0 = 32
    nf = n0 << (levels - 1)
    boxes = [(1, nf * 0.2, nf * 0.25, nf * 0.7, nf * 0.6)]
    if levels == 3:
        boxes.append((2, nf * 0.35, nf * 0.38, nf * 0.52, nf * 0.5))
    spec = wl.DomainSpec("ref", n0, n0, levels=levels, block=block, tau_finest=0.7, boxes=boxes)
    o = oracle_from_spec(spec)
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    for l in range(levels):
        nx, ny = o.dims(l)
        h = 1 << (levels - 1 - l)
        f = wl.tgv_fields(nx, ny, float(h), 0.03, nf, offset=0.5)
        o.set_fields(l, *f)
        g.set_fields(l, *f)
    o.finalize_init()
    o.step(30)
    g.step(30)
    compare_populations(g, o, levels, TOL64)
    cg, co = g.checksum(), o.checksum()
    assert abs(cg[0] - co[0]) / co[0] < 1e-13


def test_cylinder_fp64_small():
    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=100.0)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(60)
    g.step(60)
    compare_populations(g, o, 3, TOL64)
    fg, fo = g.forces(), o.forces()
    assert fg.shape == fo.shape == (60 * 4, 3)
    compare_forces(fg, fo, spec.body.a)


def test_wing_retag_fp64_small():
    # pitching (+-45 deg) and heaving wing, fast enough that the refined region
    # moves within the test, slow enough to stay subsonic (peak speed ~0.1)
    spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=wl.F64,
                   heave_chords=1.0)
    spec.body.period = 400.0
    spec.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    b0 = [g.blocks(l) for l in range(3)]
    o.step(50)
    g.step(50)
    assert any(not np.array_equal(g.blocks(l), b0[l]) for l in range(3)), "the refined region did not move"
    for l in range(3):
        assert np.array_equal(g.blocks(l), o.blocks(l))
    compare_populations(g, o, 3, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


@pytest.mark.parametrize("which", [0, 1], ids=["pitch_up_plate", "triangle_pitch_naca"])
def test_pitch_motions_fp64(which):
    """A flat plate (rectangle markers) in the pitch-up ramp of Sec. 3.4 and a
    NACA section in the triangular pitch of Sec. 3.5, with the refined
    region following the body: populations and forces against the oracle.
    The force bound adds the rounding of the prescribed angle (host and
    device libraries may round log1p, exp, sin, cos one ulp apart), which
    moves each marker's Eq. 11 velocity by up to 2 ulp(|x0|)."""
    spec = wl.replace_storage(small_pitch_specs()[which], wl.F64)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    b0 = [g.blocks(l) for l in range(3)]
    o.step(20)
    g.step(20)
    assert any(not np.array_equal(g.blocks(l), b0[l]) for l in range(3)), "the refined region did not move"
    for l in range(3):
        assert np.array_equal(g.blocks(l), o.blocks(l))
    compare_populations(g, o, 3, TOL64)
    fg, fo = g.forces(), o.forces()
    assert fg.shape == fo.shape and np.isfinite(fo).all()
    b = spec.body
    scale = np.abs(fo[:, :2]).max()
    ds = o.ds()
    atol = max(1e-11 * scale, 4.0 * b.n_markers * ds * np.spacing(max(abs(b.x0[0]), abs(b.x0[1]))))
    np.testing.assert_allclose(fg[:, :2], fo[:, :2], rtol=1e-10, atol=atol)
    np.testing.assert_allclose(fg[:, 2], fo[:, 2], rtol=1e-10, atol=atol * 2 * b.a)


def test_large_body_ibm_fp32():
    """A cylinder of D = 128 finest cells and 402 markers (the Table 1 body
    of Sec. 3.3), whose one-block IBM needs nearly all of the shared memory a
    block can have: FP32 storage against the FP64 oracle."""
    spec = wl.cylinder(D=128, levels=2, re=300.0, u=0.1, n_markers=402, block=16, storage=wl.F32, lx=12.0,
                       ly=6.0, xc=3.0)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(20)
    g.step(20)
    assert velocity_error(g, o, 2) <= TOL32_U
    fo, fg = o.forces(), g.forces()
    np.testing.assert_allclose(fg[:, :2], fo[:, :2], rtol=0, atol=1e-4 * np.abs(fo[:, :2]).max())


def test_fp32_velocity_tolerance():
    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(100)
    g.step(100)
    err = velocity_error(g, o, 3)
    assert err <= TOL32_U, err


def test_fields_and_populations_agree_with_each_other():
    spec = wl.tgv(n=32, block=16)
    g = gpu_domain(spec)
    g.step(5)
    f = g.populations(0)
    rho, ux, uy = g.fields(0)
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    np.testing.assert_allclose(rho, f.sum(0), rtol=1e-14)
    np.testing.assert_allclose(ux, (cx[:, None, None] * f).sum(0) / f.sum(0), rtol=1e-12, atol=1e-16)


# ---------------------------------------------------------------------------
# launches of at least 2^19 cells take the vectorised kernel (4 cells per
# thread); the cases below cover it, including the IBM force patch
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("block", [16, 32])
def test_large_grid_vector_kernel_fp64(block):
    spec = wl.DomainSpec("big", 1024, 512, levels=1, block=block, tau_finest=0.7)
    rho, ux, uy = wl.random_fields(1024, 512, seed=12)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux, uy)
    o.finalize_init()
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    g.set_fields(0, rho, ux, uy)
    o.step(12)
    g.step(12)
    compare_populations(g, o, 1, TOL64)


def test_large_single_level_cylinder_vector_kernel_fp64():
    spec = wl.cylinder(D=10, levels=1, block=16, storage=wl.F64, re=100.0, lx=102.4, ly=51.2, xc=20.0)
    assert spec.nx0 * spec.ny0 >= 1 << 19
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(15)
    g.step(15)
    compare_populations(g, o, 1, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


@pytest.mark.parametrize("storage,tol", [(wl.F32, 1e-5), (wl.BF16DEV, 2e-3), (wl.F16DEV, 5e-4)])
def test_large_grid_reduced_storage(storage, tol):
    # velocity error of reduced-precision storage against the FP64 oracle
    spec = wl.DomainSpec("bigr", 1024, 512, levels=1, block=16, tau_finest=0.7, storage=storage)
    rho, ux, uy = wl.random_fields(1024, 512, seed=13)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux, uy)
    o.finalize_init()
    from paper_2402_04606_gb300.native import Domain

    g = Domain(spec)
    g.set_fields(0, rho, ux, uy)
    o.step(20)
    g.step(20)
    err = velocity_error(g, o, 1)
    assert err <= tol, err


# The 16-bit target is 2e-3.  16-bit storage holds the deviation from the
# instance's free-stream equilibrium, so the cylinder's far field stores small
# values: FP16 and BF16 both meet the target (with the deviation from w_q,
# BF16's 8 mantissa bits gave 6.2e-3 here).  The bound at the target stays
# an expected failure if it is ever missed, with the level checked below it.
@pytest.mark.parametrize("storage,measured", [(wl.BF16DEV, 2e-3), (wl.F16DEV, 2e-3)])
def test_refined_cylinder_16bit_storage(storage, measured):
    spec = wl.cylinder(D=10, levels=3, block=8, storage=storage, re=100.0)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    o.step(100)
    g.step(100)
    err = velocity_error(g, o, 3)
    assert err <= measured, err
    if err > 2e-3:
        pytest.xfail(f"velocity L2 {err:.2e} misses the 16-bit target 2e-3")


def test_vector_and_scalar_kernels_agree_fp64():
    # the tuning knob picks the kernel variant; both follow the oracle
    from paper_2402_04606_gb300.native import TUNE_VECTOR_MIN_CELLS, Domain

    spec = wl.DomainSpec("knob", 256, 128, levels=1, block=16, tau_finest=0.7)
    rho, ux, uy = wl.random_fields(256, 128, seed=21)
    out = []
    for v in (-1, 0):
        g = Domain(spec)
        g.set_tuning(TUNE_VECTOR_MIN_CELLS, v)
        assert g.tuning(TUNE_VECTOR_MIN_CELLS) == v
        g.set_fields(0, rho, ux, uy)
        g.step(10)
        out.append(g.populations(0))
        g.close()
    assert rel_l2(out[0], out[1]) <= 1e-14


def test_autotuner_picks_a_measured_configuration():
    from paper_2402_04606_gb300 import autotune as at

    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    r = at.tune([spec], steps=5, warmup=2)
    assert r["best"] in r["trials"] and r["best"]["ms_per_step"] > 0
    assert r["best"]["ms_per_step"] == min(t["ms_per_step"] for t in r["trials"])
    assert {t["block"] for t in r["trials"]} <= set(at.block_candidates([spec]))


@pytest.mark.parametrize("block", [16, 32])
def test_staged_kernel_fp64_and_equal_to_vector_kernel(block):
    # the variant that stages blocks in shared memory with bulk copies: FP64
    # against the oracle, and bit for bit equal to the vector kernel in FP32
    from paper_2402_04606_gb300.native import TUNE_STAGED, TUNE_VECTOR_MIN_CELLS, Domain

    spec = wl.DomainSpec("staged", 512, 256, levels=1, block=block, tau_finest=0.7)
    rho, ux, uy = wl.random_fields(512, 256, seed=31)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux, uy)
    o.finalize_init()
    o.step(8)
    g = Domain(spec)
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
    g.set_tuning(TUNE_STAGED, 1)
    g.set_fields(0, rho, ux, uy)
    g.step(8)
    compare_populations(g, o, 1, TOL64)
    g.close()
    out = []
    for staged in (0, 1):
        g = Domain(wl.replace_storage(spec, wl.F32))
        g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
        g.set_tuning(TUNE_STAGED, staged)
        g.set_fields(0, rho, ux, uy)
        g.step(8)
        out.append(g.populations(0))
        g.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("storage", [wl.BF16DEV, wl.F16DEV])
@pytest.mark.parametrize("block", [16, 32])
def test_16bit_vector_kernel_equals_staged_kernel(storage, block):
    # 16-bit storage takes the 8-cell vector kernel; the staged kernel does
    # the same arithmetic per cell with the same rounding, so the two agree
    # bit for bit
    from paper_2402_04606_gb300.native import TUNE_STAGED, TUNE_VECTOR_MIN_CELLS, Domain

    spec = wl.replace_storage(wl.DomainSpec("v8", 512, 256, levels=1, block=block, tau_finest=0.7), storage)
    rho, ux, uy = wl.random_fields(512, 256, seed=41)
    out = []
    for staged in (0, 1):
        g = Domain(spec)
        g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
        g.set_tuning(TUNE_STAGED, staged)
        g.set_fields(0, rho, ux, uy)
        g.step(8)
        out.append(g.populations(0))
        g.close()
    assert np.isfinite(out[0]).all()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("coll", ["mrt", "les"])
def test_16bit_vector_kernel_other_collisions_against_oracle(coll):
    # the MRT and LES collisions through the 8-cell kernel, FP16 deviations
    # against the FP64 oracle (the oracle with its deviations rounded to FP16
    # after every step departs from itself by 1.7e-4 (MRT) and 2.9e-4 (LES)
    # here)
    from paper_2402_04606_gb300.native import TUNE_VECTOR_MIN_CELLS, Domain

    spec = wl.DomainSpec("v8c", 512, 256, levels=1, block=16, tau_finest=0.505 if coll == "les" else 0.7)
    spec = wl.with_mrt(spec, (1.2, 1.1, 1.3)) if coll == "mrt" else wl.with_les(spec, 0.17)
    rho, ux, uy = wl.random_fields(512, 256, seed=43)
    o = oracle_from_spec(spec)
    o.set_fields(0, rho, ux, uy)
    o.finalize_init()
    o.step(8)
    g = Domain(wl.replace_storage(spec, wl.F16DEV))
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
    g.set_fields(0, rho, ux, uy)
    g.step(8)
    err = velocity_error(g, o, 1)
    g.close()
    assert err <= 5e-3, err


def test_16bit_vector_kernel_refined_cylinder_equals_staged():
    # every level of a refined cylinder in BF16 through the vector path: the
    # IBM force patch, the interface blocks and the domain sides
    from paper_2402_04606_gb300.native import TUNE_STAGED, TUNE_VECTOR_MIN_CELLS

    spec = wl.cylinder(D=10, levels=3, block=16, storage=wl.BF16DEV, re=100.0, lx=40, ly=20, xc=12)
    runs = []
    for staged in (0, 1):
        g = gpu_domain(spec)
        g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
        g.set_tuning(TUNE_STAGED, staged)
        g.step(30)
        runs.append(([g.populations(l) for l in range(3)], g.forces()))
        g.close()
    for l in range(3):
        assert np.array_equal(runs[0][0][l], runs[1][0][l])
    assert np.array_equal(runs[0][1], runs[1][1]) and np.abs(runs[0][1][:, 0]).max() > 0


def test_staged_kernel_refined_cylinder_fp64():
    # staged launches on every level of a refined cylinder with its IBM patch
    from paper_2402_04606_gb300.native import TUNE_STAGED, TUNE_VECTOR_MIN_CELLS

    # blocks of 16 need room between the refinement and the sides
    spec = wl.cylinder(D=10, levels=3, block=16, storage=wl.F64, re=100.0, lx=40, ly=20, xc=12)
    o = init_oracle(oracle_from_spec(spec), spec)
    g = gpu_domain(spec)
    g.set_tuning(TUNE_VECTOR_MIN_CELLS, 0)
    g.set_tuning(TUNE_STAGED, 1)
    o.step(30)
    g.step(30)
    compare_populations(g, o, 3, TOL64)
    compare_forces(g.forces(), o.forces(), spec.body.a)


@pytest.mark.parametrize("which", ["cylinder", "wing"])
def test_dependent_launch_changes_nothing(which):
    """Programmatic dependent launch (SBOT_TUNE_PDL) only changes when kernels
    are scheduled: populations and forces equal bit for bit with it off."""
    from paper_2402_04606_gb300.native import TUNE_PDL, TUNE_PERSISTENT

    if which == "cylinder":
        spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    else:
        spec = wl.wing(c=16, levels=3, re=100.0, n_markers=50, block=8, domain_chords=8.0, storage=wl.F32,
                       heave_chords=1.0)
        spec.body.period = 400.0
        spec.margin = (0.0, 14.0, 6.0) + (0.0,) * 5
    runs = []
    for pdl in (0, 1):
        g = gpu_domain(spec)
        g.set_tuning(TUNE_PERSISTENT, 0)  # the per-phase graphs, where the launches are
        g.set_tuning(TUNE_PDL, pdl)
        assert g.tuning(TUNE_PDL) == pdl
        g.step(30)
        runs.append(([g.populations(l) for l in range(3)], g.forces()))
        g.close()
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(runs[0][1], runs[1][1])
