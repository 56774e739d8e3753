"""Block-size candidates of the autotuner (host only: the planner, no GPU)."""
from paper_2402_04606_gb300 import autotune as at
from paper_2402_04606_gb300 import workloads as wl


def test_candidates_divide_the_grid():
    cyl = wl.cylinder(D=40, levels=3)  # coarsest 304 x 160: 8 and 16 divide it, 32 does not
    assert at.block_candidates([cyl]) == [8, 16]
    tgv = wl.tgv(n=256)
    assert at.block_candidates([tgv]) == [8, 16, 32]


def test_with_block_keeps_the_grid_and_copies():
    cyl = wl.cylinder(D=40, levels=3)
    c8 = at.with_block(cyl, 8)
    assert (c8.block, c8.nx0, c8.ny0) == (8, cyl.nx0, cyl.ny0)
    assert c8.body is not cyl.body and c8.body == cyl.body
