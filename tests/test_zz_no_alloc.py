"""sbot_get_checksum_noalloc: the checksum entry point for callers that cannot
allocate device memory (device memory owned by another allocator, or loops
that must not pay for cudaMalloc's device-wide synchronisation).  It must give
the same mass and momentum as sbot_get_checksum, which allocates its
partial-sum buffer, on consecutive calls that share the static scratch.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2402_04606_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def domain():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_04606_gb300 import build

    build.build()
    from paper_2402_04606_gb300.native import Domain
    from paper_2402_04606_gb300.workloads import initial_fields

    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=100.0)
    g = Domain(spec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    yield g
    g.close()


def _fresh_domain(spec):
    from paper_2402_04606_gb300.native import Domain

    return Domain(spec)


def same(a, b):
    # the tolerance of the checksum comparisons in the parity tests
    assert abs(a[0] - b[0]) / abs(b[0]) < 1e-13
    np.testing.assert_allclose(a[1:], b[1:], rtol=1e-13, atol=1e-12 * abs(b[0]))


def test_noalloc_checksum_matches_allocating_one_on_consecutive_calls(domain):
    g = domain
    g.step(6)
    ref = g.checksum()
    first = g.checksum_noalloc()
    second = g.checksum_noalloc()
    assert np.isfinite(first).all()
    same(first, ref)
    same(second, ref)
    # the state moves on; the shared scratch keeps the last call's partial sums
    g.step(5)
    ref2 = g.checksum()
    third = g.checksum_noalloc()
    fourth = g.checksum_noalloc()
    same(third, ref2)
    same(fourth, ref2)
    assert not np.array_equal(ref2, ref)


def test_noalloc_first_call_allocates_no_device_memory():
    """The first allocation-free call on a new context leaves the device's
    free memory unchanged (cudaMemGetInfo before and after)."""
    import torch

    from paper_2402_04606_gb300.workloads import initial_fields

    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F32, re=100.0)
    g = _fresh_domain(spec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    g.step(2)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    out = g.checksum_noalloc()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    g.close()
    assert np.isfinite(out).all()
    assert free1 == free0


def test_noalloc_rejects_domains_beyond_its_scratch():
    """A domain needing more than 4096 partial sums (one per 256 interior
    cells of a level, at most 1024 per level) is refused with SBOT_ERR_ARG;
    the allocating checksum still serves it."""
    from paper_2402_04606_gb300.native import ERR_ARG, SbotError

    # five levels, each with at least 1024 interior blocks of 16 x 16 cells:
    # nested boxes 512, 2048, 4096, 8192 finest cells wide around the centre
    h0, n0 = 16, 1024
    c = n0 * h0 / 2.0
    boxes = [(4, c - 256, c - 256, c + 256, c + 256), (3, c - 1024, c - 1024, c + 1024, c + 1024),
             (2, c - 2048, c - 2048, c + 2048, c + 2048), (1, c - 4096, c - 4096, c + 4096, c + 4096)]
    spec = wl.DomainSpec(name="five_levels", nx0=n0, ny0=n0, levels=5, block=16, storage=wl.F32, boxes=boxes)
    g = _fresh_domain(spec)
    try:
        n = [g.n_interior(l) // 256 for l in range(5)]
        assert sum(min(1024, k) for k in n) > 4096, n
        with pytest.raises(SbotError) as e:
            g.checksum_noalloc()
        assert e.value.status == ERR_ARG
        m = g.checksum()  # the uniform state at rest: mass = finest-cell area, no momentum
        assert abs(m[0] - (n0 * h0) ** 2) <= 1e-9 * (n0 * h0) ** 2
    finally:
        g.close()
