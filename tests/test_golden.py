"""The paper's printed values (tests/golden/, each file citing its source) against the copies the
code quotes: the fingering comparison in bench.py reports the paper's Table 1 t* beside its own."""
import os

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


def test_table1_characteristic_times():
    rows = _rows("table1_characteristic_times.txt")
    assert len(rows) == 3
    assert {h: (det, sto) for h, det, sto in rows} == bench.FING_T_STAR_PAPER
