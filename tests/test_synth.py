"""The seeded input generators: deterministic, connected free space, walks stay on free cells."""
import math

import numpy as np

from synth import fields, floorplan, scan, trajectory, workloads


def test_maps_are_deterministic_and_connected():
    a, b = floorplan.rooms_map(0), floorplan.rooms_map(0)
    assert np.array_equal(a, b) and floorplan.free_components(a) == 1
    o = floorplan.office_map(1, size=512)
    assert floorplan.free_components(o) == 1
    assert 0.02 < o.mean() < 0.5
    assert o[0].all() and o[:, -1].all()


def test_rooms_map_box_fraction():
    occ = floorplan.rooms_map(0)
    walls = floorplan.rooms_map(0, box_frac=0.0)
    boxes = int(occ.sum()) - int(walls.sum())
    assert boxes >= 0.05 * int((walls == 0).sum())


def test_walk_stays_free_and_odometry_composes():
    wl = workloads.get("rooms64")
    occ = workloads.make_map(wl)
    walk = workloads.make_walk(wl, occ)
    c = wl["cell"]
    for x, y, _ in walk.poses:
        assert occ[int(y // c), int(x // c)] == 0
    x, y, th = walk.poses[0]
    for (u, v, w) in walk.odom_true:
        x, y = x + math.cos(th) * u - math.sin(th) * v, y + math.sin(th) * u + math.cos(th) * v
        th += w
    assert np.allclose([x, y, th], walk.poses[-1], atol=1e-9)
    assert np.abs(walk.odom - walk.odom_true).max() > 0


def test_scan_ranges_and_dropouts():
    occ = floorplan.rooms_map(0)
    z = scan.simulate_scan(occ, 0.1, (3.25, 3.25, 0.0), seed=0, r_max=10.0)
    assert z.dtype == np.float32 and z.shape == (360,)
    assert (z >= 0).all() and (z <= 10.0).all()
    clean = scan.simulate_scan(occ, 0.1, (3.25, 3.25, 0.0), seed=0, noise_sigma=0, dropout=0)
    assert clean.max() < 6.5                       # the grid is 6.4 m wide


def test_fields_are_seeded():
    occ = floorplan.rooms_map(0)
    a = fields.belief_like(occ, 4, 1)
    assert np.array_equal(a, fields.belief_like(occ, 4, 1))
    assert abs(a.sum() - 1) < 1e-12 and (a[:, occ != 0] == 0).all()
