"""The paper values stored in tests/golden/ checked against the derived numbers the
paper prints beside them (percent changes, improvement factors, spreads), so that a
mistyped digit in a stored value fails here rather than in a device test.  CPU only."""
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

import paper_scale as PS  # noqa: E402


def _spread(vals):
    vals = list(vals)
    return 100.0 * (max(vals) - min(vals)) / (sum(vals) / len(vals))


# Table II: Delta_MDF % and Delta_DFC % columns, per (Re, kernel)
TABLE2_DELTAS = {(20, "hat"): (0.04, 0.32), (20, "P4"): (-0.29, -0.09), (40, "hat"): (-0.24, 0.51),
                 (40, "P4"): (-0.81, -0.35), (100, "hat"): (-0.83, 1.40), (100, "P4"): (-2.19, -0.89),
                 (200, "hat"): (0.82, 4.94), (200, "P4"): (3.28, 3.91)}
# Table III: DF -> MDF and DF -> DFC improvement factors
TABLE3_FACTORS = {(20, "hat"): (10.0, 3.0), (20, "P4"): (124.9, 89.1), (40, "hat"): (8.2, 2.6),
                  (40, "P4"): (80.1, 58.1), (100, "hat"): (7.5, 2.1), (100, "P4"): (55.3, 35.3),
                  (200, "hat"): (8.3, 2.4), (200, "P4"): (68.1, 40.8)}


def test_table2_and_table3_values_match_printed_ratios():
    t = PS.paper_tables()
    assert len(t) == 8
    for key, (dm, dd) in TABLE2_DELTAS.items():
        cd = t[key]["cd"]
        assert 100.0 * (cd["MDF"] / cd["DF"] - 1.0) == pytest.approx(dm, abs=0.006), key
        assert 100.0 * (cd["DFC"] / cd["DF"] - 1.0) == pytest.approx(dd, abs=0.006), key
    for key, (fm, fd) in TABLE3_FACTORS.items():
        sl = t[key]["slip"]
        assert sl["DF"] / sl["MDF"] == pytest.approx(fm, rel=0.01), key
        assert sl["DF"] / sl["DFC"] == pytest.approx(fd, rel=0.03), key


def test_table4_values_match_printed_spreads():
    printed = {(1.01, "P4"): 0.19, (1.01, "hat"): 0.24, (1.1, "P4"): 0.57, (1.1, "hat"): 0.64,
               (1.5, "P4"): 0.85, (1.5, "hat"): 0.88}
    t4 = PS.paper_table4()
    assert len(t4) == 6
    for key, sp in printed.items():
        assert _spread(t4[key].values()) == pytest.approx(sp, abs=0.006), key


def test_table_b4_values_match_printed_spreads():
    printed = {(100, "hat", "DF"): 0.94, (100, "P4", "DF"): 0.59, (100, "hat", "MDF"): 0.93,
               (100, "P4", "MDF"): 0.65, (100, "hat", "DFC"): 0.24, (100, "P4", "DFC"): 0.21,
               (200, "hat", "DF"): 0.91, (200, "P4", "DF"): 0.60, (200, "hat", "MDF"): 0.33,
               (200, "P4", "MDF"): 0.10, (200, "hat", "DFC"): 0.11, (200, "P4", "DFC"): 0.27}
    t6 = PS.paper_table6()
    t2 = PS.paper_tables()
    for (re, kern, sch), sp in printed.items():
        row = t6[("a", re, kern, sch)]
        assert _spread(row.values()) == pytest.approx(sp, abs=0.006), (re, kern, sch)
        assert row["BGK"] == t2[(re, kern)]["cd"][sch]          # the BGK column is Table II
    assert t6[("b", "heavy")]["BGK"] == PS.paper_table5()[("DF", "B-2")][0]
    assert t6[("b", "light")]["BGK"] == PS.paper_table5()[("DF", "B-2")][1]


def test_wake_values_match_printed_gaps():
    """Table C.3: the light particle's gap between B-2 and A, (eh - none) / none,
    is +19.60 % for DF and +12.30 % for DFC; Table V: -2.16 % and -13.78 % for the
    A arm of DF relative to the reference 276.61 / 231.41."""
    t5 = PS.paper_table5()
    for sch, gap in (("DF", 19.60), ("MDF", 21.51), ("DFC", 12.30)):
        eh, none = t5[(sch, "B-2")][1], t5[(sch, "A")][1]
        assert 100.0 * (eh / none - 1.0) == pytest.approx(gap, abs=0.01), sch
    # App. C, Sec. C.2: heavy spread |eh - none| / mean and light deficit (none - eh) / eh
    for sch, spread, deficit in (("DF", 2.55, -16.39), ("MDF", 2.99, -17.71), ("DFC", 2.87, -10.95)):
        (h_eh, l_eh), (h_no, l_no) = t5[(sch, "B-2")], t5[(sch, "A")]
        assert 100.0 * abs(h_eh - h_no) / (0.5 * (h_eh + h_no)) == pytest.approx(spread, abs=0.01), sch
        assert 100.0 * (l_no - l_eh) / l_eh == pytest.approx(deficit, abs=0.01), sch
    assert 100.0 * (t5[("DF", "A")][0] / 276.61 - 1.0) == pytest.approx(-2.16, abs=0.01)
    assert 100.0 * (t5[("DF", "A")][1] / 231.41 - 1.0) == pytest.approx(-13.78, abs=0.01)
