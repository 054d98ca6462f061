"""The op-counting build of the oracle (oracle/opcount.cpp), which gives the
benchmark its algorithmic work: it runs the oracle's own arithmetic in
double with a counting scalar type, so it must take the oracle's substep
sequence (LI) and accepted steps (NR) exactly, and its counts must add up
cell by cell."""
import numpy as np

import inputs
import oracle

YR = inputs.YR


def test_counted_li_takes_the_oracles_substeps():
    c = inputs.cells_uniform(48, seed=11)
    r = oracle.opcount(c, 1e3 * YR, 1.0)
    ref = oracle.li_step(c, 1e3 * YR, 1.0)
    assert r["substeps"] == int(ref["n_sub"].astype(np.int64).sum())
    assert r["per_substep"]["flops"] > 1000 and r["per_substep"]["transcendentals"] > 10


def test_counted_nr_takes_the_oracles_steps():
    c = inputs.cells_uniform(48, seed=12)
    r = oracle.opcount(c, 1e3 * YR, 1.0, method="nr")
    ref = oracle.nr_step(c, 1e3 * YR, 1.0)
    assert r["substeps"] == int(ref["n_sub"].astype(np.int64).sum())
    assert r["per_cell"]["flops"] > 0


def test_counts_add_up_over_cells_and_sections():
    c = inputs.cells_uniform(40, seed=13)
    a = inputs.subset(c, np.arange(0, 20))
    b = inputs.subset(c, np.arange(20, 40))
    for m in ("li", "nr"):
        rc, ra, rb = (oracle.opcount(x, 1e3 * YR, 10.0, method=m) for x in (c, a, b))
        assert rc["substeps"] == ra["substeps"] + rb["substeps"]
        for sec in rc["counts"]:
            for op, v in rc["counts"][sec].items():
                assert v == ra["counts"][sec][op] + rb["counts"][sec][op], (m, sec, op)
        tot = sum(v["add"] + v["mul"] + v["div"] + 2 * v["fma"] for v in rc["counts"].values())
        assert abs(tot / rc["cells"] - rc["per_cell"]["flops"]) <= 1e-9 * tot
