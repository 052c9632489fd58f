"""Oracle pins for the static geometry fields (Sec. 2.2).

NN(x) of Eq. nearest_solid_neighbors, the wall set used by the wetting step,
the solid normal of Eq. normal_vector_solid on shapes whose normal is known in
closed form, and the reactive surface area of Eq. surface_area_reactive.
"""
import numpy as np

from oracle import cglbm as O


def test_flat_wall_normal_points_into_solid():
    solid = np.zeros((12, 5, 6), bool)
    solid[0:3] = True                       # solid below z = 3
    g = O.Geometry(solid=solid, bc_z=1)     # clamped z: the solid continues below z = 0
    wall = g.wall
    assert wall[3].all() and not wall[4:].any() and not wall[:3].any()
    ns = g.ns[:, 3]
    assert np.allclose(ns[2], -1.0) and np.allclose(ns[:2], 0.0)
    assert (g.nn[3] == 1).all() and (g.nn[4:] == 0).all()
    # reactive surface area A_r = sum r NN (Eq. surface_area_reactive), r = 1 on wall layers
    assert (g.reactive * g.nn).sum() == 5 * 6


def test_corner_normal_is_diagonal():
    """Inside a square-corner solid the normal at the corner node is along the bisector."""
    solid = np.zeros((1, 16, 16), bool)
    solid[0, :6, :] = True
    solid[0, :, :6] = True
    g = O.Geometry(solid=solid, bc_z=0)
    n = g.ns[:, 0, 6, 6]
    assert np.allclose(n, [-1 / np.sqrt(2), -1 / np.sqrt(2), 0.0], atol=1e-12)


def test_sphere_normal_is_radial():
    n = 24
    c = (n - 1) / 2
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    solid = r < 7.0
    g = O.Geometry(solid=solid, bc_z=0)
    idx = np.nonzero(g.wall)
    radial = np.stack([(c - x)[idx], (c - y)[idx], (c - z)[idx]]) / r[idx]   # towards the solid centre
    cos = (g.ns[:, idx[0], idx[1], idx[2]] * radial).sum(axis=0)
    assert cos.min() > 0.97       # eighth-order stencil: close to radial at every wall node
    assert np.median(cos) > 0.985


def test_nn_counts_hand_mask():
    solid = np.zeros((3, 3, 3), bool)
    solid[1, 1, 0] = solid[1, 1, 2] = solid[1, 0, 1] = True
    g = O.Geometry(solid=solid, bc_z=1)
    assert g.nn[1, 1, 1] == 3
    # periodic: node (z=1, y=1, x=1) sees both x-solids; (z=1, y=2, x=0) sees one (y-1)
    g2 = O.Geometry(solid=solid, bc_z=0)
    assert g2.nn[1, 2, 0] == 1 and g2.nn[1, 1, 1] == 3 and g2.nn[0, 1, 1] == 0
    assert g2.solid_bnd[1, 1, 0] and g2.solid_bnd.sum() == 3
