"""The seeded input recipes: the counter-based generator against its
published outputs, and the recipes that are more than a random draw (the
NLPP quadrature batch: icosahedron rule, rotations, points on the spheres
about the ions)."""
import numpy as np

from paper_1708_02645_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) from state 0: the
    # well-known first outputs of the reference implementation
    assert [int(x) for x in inputs.splitmix64(0, 4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    # counter based: a stream drawn from an offset is the tail of the full one
    full = inputs.splitmix64(12345, 64)
    assert np.array_equal(inputs.splitmix64(12345, 40, offset=24), full[24:])


def test_uniform_and_normal_streams():
    u = inputs.uniform01(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 5e-3
    z = inputs.normal(8, 200001)
    assert len(z) == 200001
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2
    p = inputs.uniform_positions(1000, 9)
    assert p.dtype == np.float32 and p.min() >= 0.0 and p.max() < 1.0
    # multiples of 2^-24: exact in FP32
    assert np.array_equal(p.astype(np.float64) * 2.0 ** 24, np.round(p.astype(np.float64) * 2.0 ** 24))


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
