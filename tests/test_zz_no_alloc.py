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
    from tests.helpers import initial_fields

    spec = wl.cylinder(D=10, levels=3, block=8, storage=wl.F64, re=100.0)
    g = Domain(spec)
    for l in range(spec.levels):
        g.set_fields(l, *initial_fields(spec, l))
    yield g
    g.close()


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
