"""Seeded 3-D geometry generator (sphere packs): links and gamma.

gamma is the fraction of the segment x_f -> x_f - c_i that lies in fluid
(the distance ratio of Sec. 3.B); for a sphere it is where the segment
meets the surface, which the test checks point by point."""
import numpy as np

from paper_2012_14707_gb300 import cases


def _nearest_distance(points, centres, dims):
    d = np.abs(points[:, None, :] - centres[None, :, :])
    d = np.minimum(d, dims - d)
    return np.sqrt((d * d).sum(axis=2))  # [points, spheres]


def test_sphere_pack_links_and_gamma():
    c = cases.sphere_pack3d(40, 32, 24, seed=3, porosity=0.85, r_range=(2.5, 5.0))
    nz, ny, nx = c.solid.shape
    dims = np.array([nx, ny, nz], np.float64)
    assert abs(c.n_fluid / c.solid.size - 0.85) < 0.03
    # every (fluid node, direction) whose upstream neighbour is solid is a link, once
    xs = np.arange(nx)[None, None, :]
    ys = np.arange(ny)[None, :, None]
    zs = np.arange(nz)[:, None, None]
    want = 0
    for i in range(1, 19):
        up = c.solid[(zs - cases.C3[i, 2]) % nz, (ys - cases.C3[i, 1]) % ny,
                     (xs - cases.C3[i, 0]) % nx]
        want += int(((c.solid == 0) & (up != 0)).sum())
    assert c.n_links == want
    key = ((c.link_z.astype(np.int64) * ny + c.link_y) * nx + c.link_x) * 19 + c.link_dir
    assert np.unique(key).shape[0] == c.n_links
    assert (c.solid[c.link_z, c.link_y, c.link_x] == 0).all()
    assert ((c.link_q > 0) & (c.link_q <= 1)).all()
    # the wall point x_f - gamma c_i is on a sphere's surface, and the part
    # of the segment before it is outside every sphere
    centres, radii = c.meta["centres"], c.meta["radii"]
    x = np.stack([c.link_x, c.link_y, c.link_z], axis=1).astype(np.float64)
    d = -cases.C3[c.link_dir].astype(np.float64)
    g = c.link_q[:, None]
    on = _nearest_distance(x + g * d, centres, dims) - radii[None, :]
    assert np.abs(on).min(axis=1).max() < 1e-9
    for frac in (0.25, 0.5, 0.9):
        before = _nearest_distance(x + frac * g * d, centres, dims) - radii[None, :]
        assert before.min(axis=1).min() > 0.0
