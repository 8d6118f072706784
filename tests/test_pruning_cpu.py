"""The live-ghost definition of dead-ghost elimination (Sec. IV-C), pinned by
closed-form counts for star and box stencils."""
import numpy as np
import pytest

from paper_2605_14780_gb300 import bc
from pruning import live_cells


def _blk2(n0, n1, h):
    return {"n": (n0, n1, 1), "h": (h, h, 0)}


@pytest.mark.parametrize("n0,n1", [(5, 7), (16, 3), (1, 1)])
def test_star_radius_one_keeps_the_first_face_layer(n0, n1):
    m = live_cells(_blk2(n0, n1, 2), bc.star_stencil(2, 1))
    assert m.sum() == 2 * n0 + 2 * n1
    # depth-1 cells next to the data, nothing at depth 2 or on the corners
    assert not m[0, 0, :].any() and not m[0, :, 0].any()
    assert m[0, 1, 2:2 + n0].all() and m[0, 2:2 + n1, 1].all()


@pytest.mark.parametrize("n0,n1", [(5, 7), (9, 2)])
def test_box_radius_one_adds_the_diagonal_corners(n0, n1):
    m = live_cells(_blk2(n0, n1, 2), bc.box_stencil(2, 1))
    assert m.sum() == 2 * n0 + 2 * n1 + 4


@pytest.mark.parametrize("r", [1, 2, 3])
def test_star_radius_r_keeps_r_layers(r):
    n0, n1 = 11, 6
    m = live_cells(_blk2(n0, n1, 3), bc.star_stencil(2, r))
    assert m.sum() == r * (2 * n0 + 2 * n1)


def test_hpcg_seven_and_27_points():
    blk = {"n": (12, 9, 7), "h": (1, 1, 1)}
    assert live_cells(blk, bc.star_stencil(3, 1)).sum() == 2 * (12 * 9 + 12 * 7 + 9 * 7)
    # the 27-point stencil reads every ghost cell of an h = 1 frame
    assert live_cells(blk, bc.box_stencil(3, 1)).sum() == 14 * 11 * 9 - 12 * 9 * 7


def test_stencil_helpers():
    assert len(bc.star_stencil(2, 1)) == 5 and len(bc.star_stencil(3, 2)) == 13
    assert len(bc.box_stencil(2, 1)) == 9 and len(bc.box_stencil(3, 1)) == 27
    assert (0, 0, 0) in map(tuple, bc.box_stencil(3, 2))


def test_one_sided_stencil():
    """The single offset (+1, 0, 0) reads only the first ghost column on the
    high-x side."""
    blk = _blk2(4, 3, 2)
    m = live_cells(blk, np.array([(1, 0, 0)]))
    assert m.sum() == 3
    assert m[0, 2:5, 6].all()
