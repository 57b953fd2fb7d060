"""The seeded input recipes that are more than a random draw: the NLPP
quadrature batch (icosahedron rule, rotations, points on the spheres about
the ions)."""
import numpy as np

from paper_1708_02645_gb300 import inputs


def test_icosahedron_rule_integrates_low_degree_harmonics():
    d = inputs.icosahedron_directions()
    assert d.shape == (12, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    # antipodal pairs: the rule integrates every odd polynomial to zero
    assert all(np.isclose((d @ (-v)).max(), 1.0) for v in d)   # -v is a vertex too
    assert np.allclose(d.sum(axis=0), 0.0)
    # mean of x_i x_j over the sphere is delta_ij / 3; the 12-point rule is
    # exact up to degree 5
    assert np.allclose(d.T @ d / 12.0, np.eye(3) / 3.0)
    assert np.isclose(np.mean(d[:, 0] ** 4), 1.0 / 5.0)
    assert np.isclose(np.mean(d[:, 0] ** 2 * d[:, 1] ** 2), 1.0 / 15.0)


def test_rotations_are_proper_and_orthonormal():
    r = inputs.random_rotations(11, 64)
    assert np.allclose(np.einsum("nij,nkj->nik", r, r), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(r), 1.0)


def test_nlpp_points_lie_on_spheres_about_the_ions():
    cfg = inputs.NlppConfig(walkers=4, electrons=500, seed=99)
    pts, row_of = cfg.make_points()
    assert pts.dtype == np.float32 and row_of.dtype == np.int32
    assert len(pts) == len(row_of) and len(pts) % 12 == 0 and len(pts) > 0
    assert pts.min() >= 0.0 and pts.max() < 1.0
    e = inputs.uniform_positions(cfg.n_electrons, cfg.seed).astype(np.float64)
    a = float(cfg.ion_edge)
    for k in range(0, len(pts), 12):
        el = int(row_of[k])
        assert np.all(row_of[k:k + 12] == el)
        ion = np.round(e[el] * a) / a
        r = np.linalg.norm(e[el] - ion)
        assert r < cfg.r_cut
        # minimum-image distance of each point from the ion equals r
        dq = pts[k:k + 12].astype(np.float64) - ion
        dq -= np.round(dq)
        assert np.allclose(np.linalg.norm(dq, axis=1), r, atol=1e-6)
    # every electron within the cut-off is present, and no other
    ion = np.round(e * a) / a
    near = np.nonzero(np.linalg.norm(e - ion, axis=1) < cfg.r_cut)[0]
    assert np.array_equal(np.unique(row_of), near)
