"""The parity tests' host-side helpers, on the CPU: the one-triangle coverage used to sort
out snapping differences agrees with the oracle's raster rule."""
import numpy as np

import oracle
from gpu_common import coverage, edge_band


def test_coverage_matches_the_oracle_raster_rule():
    rng = np.random.default_rng(11)
    W, H = 48, 40
    n_cov = 0
    for k in range(400):
        t = np.zeros(1, oracle.TRI_DTYPE)
        if k % 3 == 0:   # vertices on the pixel-centre lattice and half-pixel positions
            t["X"] = 16 * rng.integers(-4, W + 4, 3) + 8 * rng.integers(0, 2, 3)
            t["Y"] = 16 * rng.integers(-4, H + 4, 3) + 8 * rng.integers(0, 2, 3)
        elif k % 3 == 1:  # slivers
            x0, y0 = rng.integers(0, 16 * W), rng.integers(0, 16 * H)
            dx, dy = rng.integers(-300, 300, 2)
            t["X"] = [x0, x0 + dx, x0 + dx + rng.integers(-2, 3)]
            t["Y"] = [y0, y0 + dy, y0 + dy + rng.integers(-2, 3)]
        else:
            t["X"] = rng.integers(-200, 16 * W + 200, 3)
            t["Y"] = rng.integers(-200, 16 * H + 200, 3)
        area = (int(t["X"][0, 1]) - int(t["X"][0, 0])) * (int(t["Y"][0, 2]) - int(t["Y"][0, 0])) - \
            (int(t["X"][0, 2]) - int(t["X"][0, 0])) * (int(t["Y"][0, 1]) - int(t["Y"][0, 0]))
        if area > 0:  # the oracle rasterises front faces (negative area, y down)
            t["X"] = t["X"][:, [0, 2, 1]]
            t["Y"] = t["Y"][:, [0, 2, 1]]
        t["d"] = 0.5
        t["prim"] = 12
        want = oracle.raster(t, W, H, False, 12, 12).key != 0
        got = np.zeros((H, W), bool)
        cv = coverage(t[0], W, H)
        if cv is not None:
            j0, i0, m = cv
            got[j0:j0 + m.shape[0], i0:i0 + m.shape[1]] = m
        assert np.array_equal(got, want), (t["X"], t["Y"])
        n_cov += int(cv is not None)
    assert n_cov > 100


def test_edge_band_is_the_boundary_ring():
    """A 3 x 4 rectangle at rows 3..5, columns 4..7: the band is the 5 x 6 ring around and on
    its boundary (rows 2..6, columns 3..8) minus the pixels whose 3 x 3 neighbourhood lies
    inside it (row 4, columns 5..6)."""
    m = np.zeros((5, 6), bool)
    m[1:4, 1:5] = True
    band = edge_band((2, 3, m), 20, 20)
    want = np.zeros((20, 20), bool)
    want[2:7, 3:9] = True
    want[4, 5:7] = False
    assert np.array_equal(band, want)


def test_centre_depth_of_a_right_triangle():
    """The deepest covered centre of a right triangle with legs along the axes from (0, 0)
    lies min(x, y, (L - x - y) / sqrt 2) units inside; a 1-unit sliver's centres are all
    within a unit of an edge."""
    from gpu_common import max_centre_depth_units
    t = np.zeros(1, oracle.TRI_DTYPE)[0]
    L = 160
    t["X"] = [0, L, 0]
    t["Y"] = [0, 0, L]
    cv = coverage(t, 16, 16)
    jj, ii = np.nonzero(cv[2])
    x, y = 16.0 * (ii + cv[1]) + 8, 16.0 * (jj + cv[0]) + 8
    want = np.minimum(np.minimum(x, y), (L - x - y) / np.sqrt(2)).max()
    assert abs(max_centre_depth_units(t, cv) - want) < 1e-9
    s = np.zeros(1, oracle.TRI_DTYPE)[0]
    s["X"] = [320, 272, 271]
    s["Y"] = [1032, 1032, 1033]
    assert max_centre_depth_units(s, coverage(s, 128, 128)) <= 1.0
