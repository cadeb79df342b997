"""Pins of the oracle's sky-count map: bin edges, one count per bin of a grid of
bin centres, the 30-second window, events without direction."""
import numpy as np

import oracle


def test_bin_edges_and_invalid_values():
    v = np.array([-2.56, np.nextafter(np.float32(-2.56), np.float32(-3)), 0.0, 0.02, 2.5599, 2.56, 7.0, np.nan],
                 np.float32)
    assert oracle.sky_bin(v).tolist() == [0, -1, 128, 129, 255, -1, -1, -1]


def test_grid_of_bin_centres_fills_every_bin_once():
    c = (np.arange(256) + 0.5) * 0.02 - 2.56
    X, Y = np.meshgrid(c, c)
    m = oracle.skymap(X.ravel(), Y.ravel(), np.ones(X.size, bool), np.zeros(X.size, np.int64), 0)
    assert (m == 1).all()
    # row index is y: a single event at (x, y) = (-2.55, 2.55) lands in [255, 0]
    m = oracle.skymap([-2.55], [2.55], [True], [0], 0)
    assert m[255, 0] == 1 and m.sum() == 1


def test_thirty_second_window_and_missing_directions():
    x = np.zeros(6)
    secs = np.array([70, 71, 99, 100, 101, 100])
    has = np.array([True, True, True, True, True, False])
    m = oracle.skymap(x, x, has, secs, 100)
    assert m.sum() == 3            # seconds 71, 99, 100 count; 70 is 30 s old, 101 is in the future
    assert m[128, 128] == 3
