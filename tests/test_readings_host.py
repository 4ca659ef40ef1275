"""Host side of the BP-reading runs and of the Table 2 comparison (no GPU):
the lattice maps the readings build match the oracle's, and the Table 2
constants and statistics match the paper's table."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2212_06985_gb300 import readings, threshold

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("L", [2, 3, 5])
def test_face_edges_match_the_oracle(L):
    fe = readings.face_edges(L)
    for f in range(3 * L ** 3):
        assert fe[f].tolist() == oracle.face_edges(L, f).tolist()


def test_measurement_graph_adds_one_degree_one_variable_per_check():
    L = 3
    n = 3 * L ** 3
    cptr, cvar = readings.measurement_graph(L)
    ref_ptr, ref_var = oracle.toric_tanner(L)
    assert cptr.tolist() == (5 * np.arange(n + 1)).tolist()
    rows = cvar.reshape(n, 5)
    assert np.array_equal(rows[:, :4].reshape(-1), ref_var)
    assert rows[:, 4].tolist() == list(range(n, 2 * n))
    # every measurement variable sits in exactly one check, every qubit in four
    deg = np.bincount(cvar, minlength=2 * n)
    assert (deg[:n] == 4).all() and (deg[n:] == 1).all()


def test_table2_constants_equal_the_golden_file():
    with open(os.path.join(HERE, "golden", "table2_correlations.json")) as f:
        g = json.load(f)
    assert threshold.TABLE2_PAPER == g["counts"]
    assert sum(g["counts"].values()) == g["runs"] == threshold.TABLE2_SETUP["runs"]
    assert (g["L"], g["p"], g["cycles"]) == (threshold.TABLE2_SETUP["L"], threshold.TABLE2_SETUP["p"],
                                             threshold.TABLE2_SETUP["T"])


def test_pattern_counts_map_mask_bits_to_qubits():
    c = [0] * 8
    c[1], c[2], c[4], c[7] = 5, 6, 7, 8            # qubit 0 alone, qubit 1 alone, qubit 2 alone, all three
    pat = threshold.pattern_counts(c)
    assert (pat["100"], pat["010"], pat["001"], pat["111"]) == (5, 6, 7, 8)
    assert threshold.by_weight(pat) == [0, 18, 0, 8]


def test_table2_comparison_accepts_the_paper_and_rejects_no_failures():
    pytest.importorskip("scipy")
    paper = threshold.TABLE2_PAPER
    c = [0] * 8
    for k, v in paper.items():
        c[int(k[0]) | int(k[1]) << 1 | int(k[2]) << 2] = v
    same = threshold.table2_compare(c)
    assert same["all"]["p_value"] > 0.99 and same["failed"]["p_value"] > 0.99
    none = threshold.table2_compare([1000, 0, 0, 0, 0, 0, 0, 0])
    assert none["all"]["p_value"] < 1e-10 and none["failed"] is None
    # independent failures at the paper's single-qubit rate put too little weight on 2 and 3 qubits
    f = 0.128
    indep = [int(round(1000 * (f ** k) * ((1 - f) ** (3 - k)))) for k in range(4)]
    cc = [indep[0], indep[1] // 3, indep[1] // 3, indep[2] // 3, indep[1] // 3, indep[2] // 3, indep[2] // 3, indep[3]]
    assert threshold.table2_compare(cc)["failed"]["p_value"] < 1e-3


def test_reading_names():
    assert readings.READINGS == ("restart", "warm", "halfiter", "measdecide")
    with pytest.raises(ValueError):
        readings.run_stepwise(4, 0.05, 0.05, 64, 1, 1, 2, "", 0, reading="sideways")
