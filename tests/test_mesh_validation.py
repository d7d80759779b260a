"""Host checks of a coarse mesh (sgdg_validate_mesh; sgdg_create runs the
same checks before it touches a device), CPU only.

Every mesh the workloads build passes.  Meshes with a planted defect are
refused with SGDG_EINVAL and a message naming the check: a box with lo >= hi,
a vertex outside the box or not finite, two vertices at one point, a cell
index out of range, a cell of zero volume, a duplicated cell (overlap), a
missing cell (hole), a hanging vertex (a face of one cell inside the box),
and periodic sides whose vertices do not match."""
import numpy as np
import pytest

import paper_2204_05988_gb300 as P
import sgdg_workloads as W

EINVAL = 1


def _refused(mesh, words):
    with pytest.raises(P.SgdgError) as e:
        P.validate_mesh(mesh)
    assert e.value.code == EINVAL
    assert words in str(e.value), str(e.value)


def _mesh(coords, cells, lo, hi, periodic=None):
    coords = np.asarray(coords, dtype=np.float64)
    d = coords.shape[1]
    return W.CoarseMesh(coords=coords, cells=np.asarray(cells, dtype=np.int32), lo=tuple(lo), hi=tuple(hi),
                        periodic=tuple(periodic or [False] * d))


@pytest.mark.parametrize("mesh", [
    W.interval_mesh(0.0, 1.0, 4), W.interval_mesh(0.0, 1.0, 4, periodic=True), W.interval_mesh(-6.0, 6.0, 8),
    W.square_mesh(0.0, 1.0, 2), W.square_mesh(-1.0, 1.0, 4, periodic=True), W.square_mesh(0.0, 4 * np.pi, 2, True),
    W.cube_mesh(0.0, 1.0, 1), W.cube_mesh(-1.0, 1.0, 2), W.cube_mesh(0.0, 1.0, 2, periodic=True)],
    ids=lambda m: f"d{m.dim}_{len(m.cells)}cells{'_per' if any(m.periodic) else ''}")
def test_workload_meshes_pass(mesh):
    P.validate_mesh(mesh)


def test_every_workload_problem_mesh_passes():
    for prob in (W.free_streaming_1d(L=1), W.transport_2d(L=1), W.landau_4d(L=1), W.transport_3d(L=1),
                 W.periodic_advection_1d(L=1), W.inflow_manufactured_2d(L=1), W.time_dependent_2d(L=1)):
        P.validate_mesh(prob.mesh_x)
        P.validate_mesh(prob.mesh_v)


def test_box_and_vertices():
    _refused(_mesh([[0.0], [1.0]], [[0, 1]], [1.0], [0.0]), "lo < hi")
    _refused(_mesh([[0.0], [1.5]], [[0, 1]], [0.0], [1.0]), "outside its box")
    _refused(_mesh([[0.0], [np.nan]], [[0, 1]], [0.0], [1.0]), "outside its box")
    _refused(_mesh([[0.0], [0.5], [0.5], [1.0]], [[0, 1], [2, 3]], [0.0], [1.0]), "share their coordinates")


def test_cells():
    sq = [[0, 0], [1, 0], [0, 1], [1, 1]]
    _refused(_mesh(sq, [[0, 1, 3], [0, 3, 4]], [0, 0], [1, 1]), "out of range")
    _refused(_mesh(sq, [[0, 1, 3], [0, 3, -1]], [0, 0], [1, 1]), "out of range")
    _refused(_mesh(sq, [[0, 1, 3], [0, 3, 3]], [0, 0], [1, 1]), "zero volume")
    _refused(_mesh(sq, [[0, 1, 3], [0, 3, 2], [0, 1, 3]], [0, 0], [1, 1]), "do not tile the box")
    _refused(_mesh(sq, [[0, 1, 3]], [0, 0], [1, 1]), "do not tile the box")


def test_hanging_vertex_is_refused():
    # the square's lower-right triangle is split through the midpoint of the
    # diagonal, the upper-left one is not: the diagonal is a face of one cell
    # inside the box
    coords = [[0, 0], [1, 0], [0, 1], [1, 1], [0.5, 0.5]]
    cells = [[0, 1, 4], [1, 3, 4], [0, 3, 2]]
    _refused(_mesh(coords, cells, [0, 0], [1, 1]), "not on a side of its box")


def test_periodic_sides_must_match():
    coords = [[0, 0], [1, 0], [1, 1], [0, 1], [0, 0.5]]
    cells = [[0, 1, 4], [4, 1, 2], [4, 2, 3]]
    P.validate_mesh(_mesh(coords, cells, [0, 0], [1, 1]))                 # a valid non-periodic mesh
    P.validate_mesh(_mesh(coords, cells, [0, 0], [1, 1], [False, True]))  # y sides match
    _refused(_mesh(coords, cells, [0, 0], [1, 1], [True, False]), "periodic axis")


def test_create_refuses_before_any_device_call():
    """sgdg_create returns EINVAL for a bad mesh without touching a device
    (this runs on hosts without one)."""
    prob = W.free_streaming_1d(L=1)
    prob.mesh_v = _mesh([[-1.0], [0.0], [0.0], [1.0]], [[0, 1], [2, 3]], [-1.0], [1.0])
    with pytest.raises(P.SgdgError) as e:
        P.Solver(prob)
    assert e.value.code == EINVAL and "mesh_v" in str(e.value)
