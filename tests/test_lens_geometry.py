"""The lens analysis used by the spreading-lens checks, pinned to the paper's
printed analytical values and to exact geometry."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import workloads as W
from lens_geometry import measure_lens, neumann

GOLDEN = json.loads((Path(__file__).parent / "golden" / "table2_lens_analytic.json").read_text())


@pytest.mark.parametrize("row", GOLDEN["rows"])
def test_neumann_closed_form_reproduces_table2(row):
    # paper labels: 1 = lens, 2 = upper, 3 = lower; neumann() takes
    # (upper|lower, lens|upper, lens|lower)
    g12, g13, g23 = row["ratio"]
    th_up, th_lo, d = neumann(g23, g12, g13, math.pi * 30 ** 2)
    assert abs(th_up - row["theta1_deg"]) < 0.01
    assert abs(th_lo - row["theta2_deg"]) < 0.01
    assert abs(d - row["d"]) < 0.03        # the paper rounds d to two decimals of its own quadrature


def test_measurement_of_the_initial_circle():
    """Eq. 56 initial lens: a circle of radius 40 cut by the flat interface
    through its centre -- two half-discs: 90 degree caps and chord 80."""
    phi = W.liquid_lens(512, 256, 40.0, 4.0, 256.0, 128.0)
    th_up, th_lo, d = measure_lens(*phi)
    assert abs(th_up - 90) < 1.0 and abs(th_lo - 90) < 1.0
    assert abs(d - 80) < 0.5
