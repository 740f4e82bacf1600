"""The seeded input recipes: the square-cylinder mesh (Sec. 4.3) and the body
face ids, checked against the numbers the recipe fixes (cell counts, the
square's extent and faces, the alignment with four multigrid levels, the
quadrature rule, the rear-region initial state)."""
import math

import numpy as np
import pytest

from paper_1704_03151_gb300 import workloads as wl


def test_square_cylinder_recipe():
    c = wl.square_cylinder()
    assert (c["nx"], c["ny"]) == (160, 120)
    solid = np.asarray(c["solid"]).reshape(120, 160).astype(bool)
    assert solid.sum() == 32 * 24 and (~solid).sum() == 18432
    x, y = np.asarray(c["x_nodes"]), np.asarray(c["y_nodes"])
    assert x[0] == pytest.approx(-7.5) and x[-1] == pytest.approx(7.5)
    assert y[0] == pytest.approx(-7.5) and y[-1] == pytest.approx(7.5)
    assert np.all(np.diff(x) > 0) and np.all(np.diff(y) > 0)
    # the square is the unit square at the centre
    cols = np.where(solid.any(axis=0))[0]
    rows = np.where(solid.any(axis=1))[0]
    assert x[cols[0]] == pytest.approx(-0.5) and x[cols[-1] + 1] == pytest.approx(0.5)
    assert y[rows[0]] == pytest.approx(-0.5) and y[rows[-1] + 1] == pytest.approx(0.5)
    # wall faces: 24 on each vertical side, 32 on each horizontal side
    fbx = np.asarray(c["face_bc_x"]).reshape(120, 161)
    fby = np.asarray(c["face_bc_y"]).reshape(121, 160)
    assert (fbx == 0).sum() == 48 and (fby == 0).sum() == 64
    assert np.all(fbx[:, 0] == 1) and np.all(fbx[:, -1] == 2)       # inflow farfield, outflow
    assert np.all(fby[0, :] == 1) and np.all(fby[-1, :] == 1)
    # Ma 5 freestream with gamma 5/3 and R = 1/2
    assert c["bcs"][1]["u"] == pytest.approx(5.0 * math.sqrt(5.0 / 6.0))
    assert c["vgrid"]["rule"] == wl.TRAPEZOID and c["vgrid"]["nu"] == 89
    # the body fills whole cells of the three coarser levels
    cc = c
    for _ in range(3):
        cc = wl.coarsen_case(cc)
    assert np.asarray(cc["solid"]).sum() == 4 * 3


def test_rear_region_initial_state():
    c = wl.square_cylinder()
    rho, u, v, t = wl.initial_fields(c)
    xc = 0.5 * (np.asarray(c["x_nodes"])[1:] + np.asarray(c["x_nodes"])[:-1])
    rear = np.broadcast_to(xc[None, :] > 0.5, (c["ny"], c["nx"])).ravel()
    assert np.all(rho[rear] == 0.1) and np.all(u[rear] == 0.0)
    assert np.all(rho[~rear] == 1.0) and np.all(u[~rear] == c["init"]["u"])
    assert np.all(t == 1.0) and np.all(v == 0.0)


def test_body_face_ids_mark_exactly_the_fluid_solid_faces():
    solid = np.zeros((6, 8), dtype=np.uint8)
    solid[2:4, 3:6] = 1
    fbx, fby = wl.edge_face_ids(8, 6, 0, 1, 2, 3)
    fbx, fby = wl.body_face_ids(solid, fbx, fby, 9)
    fbx = fbx.reshape(6, 9)
    fby = fby.reshape(7, 8)
    assert (fbx == 9).sum() == 4 and (fby == 9).sum() == 6
    assert fbx[2, 4] == -1 and fby[3, 4] == -1                       # faces inside the body
    assert np.all(fbx[:, 0] == 0) and np.all(fby[0, :] == 2)         # edges untouched
