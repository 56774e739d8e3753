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


def test_search_order_and_choice_with_a_cost_model():
    """The tuner's search with a cost model in place of device timing: block
    sizes at the default threshold, then every threshold at the best size,
    the staged variant, dependent launch, the IBM's threads per body, the
    vector kernel's waves of blocks, then
    the persistent kernel's shapes, task sizes and steps per launch, each on
    the best so far; the model's
    minimum is returned with all its knobs, and the best of each step form."""
    from paper_2402_04606_gb300 import autotune as at

    calls = []

    def model(specs, block, vec, storage, steps, warmup, stream, **k):
        calls.append((block, vec, k["staged"], k["pdl"], k["ibm_threads"], k["persistent"], k["step_threads"],
                      k["bulk_rounds"], k["crit_blocks"], k["steps_per_launch"], k["vec_waves"]))
        return (1.0 + abs(block - 16) / 8 + (0.0 if vec == 1 << 16 else 0.1) + 0.05 * k["staged"] - 0.02 * k["pdl"]
                - (0.01 if k["ibm_threads"] == 512 else 0.0) - 0.03 * k["persistent"] * (k["step_threads"] == 768)
                - 0.004 * (k["crit_blocks"] == 2) + 0.001 * (k["steps_per_launch"] == 16)
                - 0.002 * (k["vec_waves"] == 0))

    spec = wl.cylinder(D=40, levels=3)
    cands = at.block_candidates([spec])
    assert cands == [8, 16]
    r = at.tune([spec], timer=model)
    expect = [(b, 1 << 19, 0, 0, 1024, 0, 0, 8, 0, 8, 8) for b in cands]
    expect += [(16, v, 0, 0, 1024, 0, 0, 8, 0, 8, 8) for v in at.VEC_THRESHOLDS if v != 1 << 19]
    expect += [(16, 1 << 16, 1, 0, 1024, 0, 0, 8, 0, 8, 8), (16, 1 << 16, 0, 1, 1024, 0, 0, 8, 0, 8, 8)]
    expect += [(16, 1 << 16, 0, 1, 256, 0, 0, 8, 0, 8, 8), (16, 1 << 16, 0, 1, 512, 0, 0, 8, 0, 8, 8)]
    expect += [(16, 1 << 16, 0, 1, 512, 0, 0, 8, 0, 8, 0), (16, 1 << 16, 0, 1, 512, 0, 0, 8, 0, 8, 2)]
    expect += [(16, v, 0, 1, 512, 1, 0, 8, 0, 8, 0) for v in sorted({1 << 19, 1 << 16, -1})]
    expect += [(16, 1 << 16, 0, 1, 512, 1, 768, 8, 0, 8, 0), (16, 1 << 16, 0, 1, 512, 1, 0, 1, 0, 8, 0),
               (16, 1 << 16, 0, 1, 512, 1, 0, 16, 0, 8, 0)]
    expect += [(16, 1 << 16, 0, 1, 512, 1, 768, 8, 1, 8, 0), (16, 1 << 16, 0, 1, 512, 1, 768, 8, 2, 8, 0)]
    expect += [(16, 1 << 16, 0, 1, 512, 1, 768, 8, 2, 16, 0)]
    assert calls == expect
    best = r["best"]
    assert (best["block"], best["vec_min_cells"], best["staged"], best["pdl"], best["ibm_threads"], best["persistent"],
            best["step_threads"], best["crit_blocks"]) == (16, 1 << 16, 0, 1, 512, 1, 768, 2)
    assert best["ms_per_step"] == min(t["ms_per_step"] for t in r["trials"])
    assert len(r["trials"]) == len(expect)
    assert at.best_of_form(r, 1) == best
    g = at.best_of_form(r, 0)
    assert g["persistent"] == 0 and (g["vec_min_cells"], g["pdl"], g["ibm_threads"]) == (1 << 16, 1, 512)
