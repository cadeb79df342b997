"""Pins of the oracle's tailcut cleaning: exhaustive enumeration on tiny cameras.

Every charge assignment over 4 levels (including values exactly at the
thresholds) of a 7-pixel hexagonal camera (4^7 images) and a 3x3 square camera
(4^9 images) is cleaned by the oracle and compared with the set definition
written as adjacency-matrix algebra over the whole enumeration at once.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def adjacency(nb):
    P = nb.shape[0]
    A = np.zeros((P, P), np.int64)
    for i in range(P):
        for j in nb[i]:
            if j >= 0:
                A[i, j] = 1
    return A


def reference_masks(Q, A, hi, lo, core_nb):
    above = (Q >= hi).astype(np.int64)
    core = above.astype(bool)
    if core_nb:
        core &= (above @ A.T) > 0
    boundary = (Q >= lo) & ((core.astype(np.int64) @ A.T) > 0)
    return (core | boundary).astype(np.uint8)


def enumerate_all(P, levels):
    return np.array(list(itertools.product(levels, repeat=P)), np.float32)


@pytest.mark.parametrize("core_nb", [0, 1])
def test_hex7_exhaustive(core_nb):
    xy, nb = synth.lattice("hex", 7, 0.1)
    A = adjacency(nb)
    assert A.sum(1).tolist() == [6, 3, 3, 3, 3, 3, 3]       # centre + first ring
    assert (A == A.T).all()
    hi, lo = 10.0, 5.0
    Q = enumerate_all(7, [2.0, 5.0, 7.5, 10.0])
    ref = reference_masks(Q, A, hi, lo, core_nb)
    got = np.stack([oracle.clean(q, nb, hi, lo, core_nb) for q in Q])
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("core_nb", [0, 1])
def test_square3x3_exhaustive(core_nb):
    xy, nb = synth.lattice("grid", 9, 0.1)
    A = adjacency(nb)
    assert A.sum(1).tolist() == [2, 3, 2, 3, 4, 3, 2, 3, 2]
    hi, lo = 8.0, 4.0
    Q = enumerate_all(9, [0.0, 4.0, 6.0, 8.0])
    ref = reference_masks(Q, A, hi, lo, core_nb)
    got = np.stack([oracle.clean(q, nb, hi, lo, core_nb) for q in Q])
    np.testing.assert_array_equal(got, ref)


def test_hand_worked_square():
    xy, nb = synth.lattice("grid", 9, 0.1)
    # pixel 4 is the centre; 3 and 5 are its left/right neighbours; 0 is a corner
    q = np.zeros(9, np.float32)
    q[4] = 10
    assert oracle.clean(q, nb, 10, 5, 0).tolist() == [0, 0, 0, 0, 1, 0, 0, 0, 0]
    assert oracle.clean(q, nb, 10, 5, 1).tolist() == [0] * 9        # isolated core removed
    q[5] = 10
    q[3] = 5
    q[0] = 9                                                         # not adjacent to a core
    assert oracle.clean(q, nb, 10, 5, 1).tolist() == [0, 0, 0, 1, 1, 1, 0, 0, 0]
    q[3] = np.nextafter(np.float32(5), np.float32(0))                # just below t_lo
    assert oracle.clean(q, nb, 10, 5, 1).tolist() == [0, 0, 0, 0, 1, 1, 0, 0, 0]


def test_monotonicity_and_containment_on_real_camera():
    cam = synth.camera(1)
    rng = np.random.default_rng(7)
    q = rng.exponential(3.0, cam.n_pix).astype(np.float32)
    m1 = oracle.clean(q, cam.nb, 8, 4, 1)
    m2 = oracle.clean(q, cam.nb, 8, 5, 1)
    m0 = oracle.clean(q, cam.nb, 8, 4, 0)
    assert (m2 <= m1).all()                 # raising t_lo only removes pixels
    assert (m1 <= m0).all()                 # the neighbour test only removes cores
    assert (q[m1 == 1] >= 4).all()
    assert m1.sum() > 0


def test_camera_neighbour_lists_are_symmetric():
    for c in range(4):
        cam = synth.camera(c)
        A = adjacency(cam.nb)
        assert (A == A.T).all()
        d = np.linalg.norm(cam.xy[:, None, :] - cam.xy[None, :, :], axis=-1) if cam.n_pix <= 256 else None
        if d is not None:
            close = (np.abs(d - cam.pitch) < 1e-4) & (d > 0)
            np.testing.assert_array_equal(close, A.astype(bool))
