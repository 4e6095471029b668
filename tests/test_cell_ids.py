"""april_cell_ids (CPU): the Hilbert id of the grid cell holding a lattice
point, by the two-levels-a-step table the filter's triage also uses, equals
the oracle's curve (Sec. 3.2, pinned in test_oracle_pins.py) at every order,
on an offset grid, with points outside the grid mapped to UINT64_MAX."""
import numpy as np
import pytest

import oracle
from paper_2307_01716_gb300 import april as A


@pytest.mark.parametrize("order", range(1, 17))
def test_cell_ids_equal_the_oracle_curve(order):
    rng = np.random.default_rng(order)
    ox, oy, lc = 5, -7, 3
    side = (1 << order) << lc
    m = side // 20 + 1  # a margin outside the grid on every side
    x = rng.integers(ox - m, ox + side + m, 4000)
    y = rng.integers(oy - m, oy + side + m, 4000)
    ids = A.april_cell_ids(A.grid(order, ox, oy, lc), x, y)
    cx, cy = np.floor_divide(x - ox, 1 << lc), np.floor_divide(y - oy, 1 << lc)
    inside = (cx >= 0) & (cy >= 0) & (cx < (1 << order)) & (cy < (1 << order))
    assert inside.sum() > 3000 and (~inside).sum() > 0
    assert np.array_equal(ids[inside], oracle.hilbert(order, cx[inside], cy[inside]).astype(np.uint64))
    assert (ids[~inside] == np.uint64(2 ** 64 - 1)).all()
