"""The values the paper prints (fixtures under tests/golden, each citing its table or section)
against the code that restates them.

table1_h2_single_card.txt (Table 1): its speedup columns are the quotients of its time columns
within the rounding of the printed digits, which checks the transcription; the bench's context
quote carries the same chemistry times.
per_species_network.txt (Section 2): the per-species networks' widths against the trainer's, and
the rule that inert species get no network against the oracle's increments over the training
states' distribution."""
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def _half_ulp(tok):
    """Half a unit in the last printed digit of a decimal token."""
    return 0.5 * 10.0 ** -(len(tok.split(".")[1]) if "." in tok else 0)


def _quotient_bounds(num, den):
    a, b = float(num), float(den)
    ha, hb = _half_ulp(num), _half_ulp(den)
    return (a - ha) / (b + hb), (a + ha) / (b - hb)


def test_table1_speedups_are_the_quotients_of_the_printed_times():
    rows = _rows("table1_h2_single_card.txt")
    assert [int(r[0]) for r in rows] == [32, 64, 128]
    for r in rows:
        assert len(r) == 10
        for cpu, gpu, sp in ((1, 2, 3), (4, 5, 6), (7, 8, 9)):
            lo, hi = _quotient_bounds(r[cpu], r[gpu])
            h = _half_ulp(r[sp])
            assert lo - h <= float(r[sp]) <= hi + h, (r[0], r[cpu], r[gpu], r[sp])


def test_table1_sum_is_chemistry_plus_fluid():
    """The sum column covers the chemistry and fluid columns; what else it holds is under 0.02 %
    of the step on the CPU side and within the rounding on the GPU side."""
    for r in _rows("table1_h2_single_card.txt"):
        for tot, chem, fluid in ((1, 4, 7), (2, 5, 8)):
            h = _half_ulp(r[tot]) + _half_ulp(r[chem]) + _half_ulp(r[fluid])
            rest = float(r[tot]) - float(r[chem]) - float(r[fluid])
            assert -h <= rest <= 2e-4 * float(r[tot]) + h, r


def test_bench_quotes_table1_as_printed():
    import bench
    ctx = bench.paper_context()
    for r in _rows("table1_h2_single_card.txt"):
        side = int(r[0])
        row = ctx["rows"][f"{side}^3"]
        assert bench.PAPER_TABLE1_CHEMISTRY_S[side] == (float(r[4]), float(r[5]))
        lo, hi = _quotient_bounds(r[4], r[5])
        assert lo <= row["chemistry_speedup"] <= hi
        assert row["gpu_dnn_cell_updates_per_s"] == pytest.approx(side ** 3 / float(r[5]), rel=1e-15)
    # the largest mesh: 2^21 cells in 0.41 s, about 5.1 M cells/s for the paper's DNN chemistry
    assert ctx["rows"]["128^3"]["gpu_dnn_cell_updates_per_s"] == pytest.approx(5.115e6, rel=1e-3)


def _network_fixture():
    return {r[0]: r[1:] for r in _rows("per_species_network.txt")}


def test_per_species_network_shape_is_the_papers():
    from paper_2312_13513_gb300 import train
    g = _network_fixture()
    assert tuple(int(w) for w in g["hidden"]) == train.PER_SPECIES_HIDDEN
    assert g["outputs_per_network"] == ["1"] and g["activation"] == ["gelu"] and g["optimizer"] == ["adam"]
    assert g["inputs"] == ["T", "p", "Y"]


def test_inert_species_get_no_network():
    """On the training states' distribution the oracle leaves the inert species (N2 of the H2/air
    mechanism, in no reaction) bitwise unchanged over dt, while every other species moves; the
    statistics rule then gives a network to each species but N2."""
    from oracle import OracleMech
    from paper_2312_13513_gb300 import train
    from synth.mechanism import h2_mechanism
    from synth.states import flamelet_samples, load_table
    assert _network_fixture()["inert_species_networks"] == ["0"]
    mech = h2_mechanism()
    om = OracleMech(mech)
    f = flamelet_samples(load_table("h2_flamelet.npz"), 256, 5, front_fraction=0.5)
    T1, Y1, status, _ = om.advance(f["T"], f["p"], f["Y"], 5e-7)
    assert np.all(status == 0)
    dY = Y1 - f["Y"]
    inert = np.all(dY == 0.0, axis=1)
    n2 = mech.species.index("N2")
    assert inert[n2] and inert.sum() == 1
    # the training statistics' rule: zero in every state -> y_std = 0, otherwise the deviation
    y_std = np.where(inert, 0.0, dY.std(axis=1))
    species = train.networked_species(y_std)
    assert species == [k for k in range(mech.ns) if k != n2] and len(species) == mech.ns - 1
