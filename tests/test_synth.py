"""The seeded input generators against the recipes their docstrings state (no GPU).

Both the oracle's tests and the CUDA path's draw their inputs from these
generators, so a generator that drifted from its recipe (points off the
surface, a non-uniform area density, cells in another order) would change every
workload without failing a parity test.  Each check here is independent of the
generator's own code: closed forms, brute force, or a numerical integral.
"""
import numpy as np
import pytest

from paper_1210_7292_gb300 import synth


def test_same_seed_same_draw_other_seed_other_draw():
    for fn in (lambda s: synth.uniform_cube(500, s), lambda s: synth.sphere_surface(500, s),
               lambda s: synth.ellipsoid_surface(500, seed=s)):
        p1, q1 = fn(11)
        p2, q2 = fn(11)
        p3, _ = fn(12)
        assert np.array_equal(p1, p2) and np.array_equal(q1, q2)
        assert not np.array_equal(p1, p3)
    assert np.array_equal(synth.gaussian_vectors(7, 9, 5), synth.gaussian_vectors(7, 9, 5))
    assert synth.batched_tree_specs(seed=4) == synth.batched_tree_specs(seed=4)


def test_uniform_cube_bounds_and_moments():
    n = 100_000
    pts, q = synth.uniform_cube(n, seed=1)
    assert pts.shape == (n, 3) and q.shape == (n,)
    assert pts.min() >= -1.0 and pts.max() < 1.0 and np.abs(q).max() <= 1.0
    # U(-1, 1): mean 0, variance 1/3; five standard errors
    assert np.all(np.abs(pts.mean(axis=0)) < 5 * np.sqrt(1 / 3 / n))
    assert np.all(np.abs(pts.var(axis=0) - 1 / 3) < 5 * np.sqrt(4 / 45 / n))


def test_sphere_surface_radius_and_isotropy():
    n, r = 100_000, 0.999
    pts, q = synth.sphere_surface(n, seed=2)
    assert np.allclose(np.linalg.norm(pts, axis=1), r, rtol=0, atol=1e-12)
    # uniform on the sphere: every coordinate has mean 0 and second moment r^2 / 3,
    # and z / r is U(-1, 1) (Archimedes' hat-box theorem)
    assert np.all(np.abs(pts.mean(axis=0)) < 5 * r / np.sqrt(3 * n))
    assert np.all(np.abs((pts ** 2).mean(axis=0) - r * r / 3) < 5 * r * r * np.sqrt(4 / 45 / n))
    counts, _ = np.histogram(pts[:, 2] / r, bins=10, range=(-1.0, 1.0))
    assert np.all(np.abs(counts - n / 10) < 5 * np.sqrt(n / 10))
    assert abs(q.mean()) < 5 / np.sqrt(n) and abs(q.var() - 1) < 5 * np.sqrt(2 / n)


def _ellipsoid_cap_fraction(a, b, c, t):
    """Area of {z > c t} on the ellipsoid over its whole area.  The cap is the graph of
    z = c sqrt(1 - (x/a)^2 - (y/b)^2) over an ellipse; with x = a r cos th, y = b r sin th its
    area element is a b r sqrt(1 + (c r / s)^2 (cos^2 th / a^2 + sin^2 th / b^2)) dr dth,
    s = sqrt(1 - r^2).  The whole area is 4 pi a b c R_G(1/a^2, 1/b^2, 1/c^2) (Carlson)."""
    integrate = pytest.importorskip("scipy.integrate")
    special = pytest.importorskip("scipy.special")

    def dA(r, th):
        s2 = 1.0 - r * r
        return a * b * r * np.sqrt(1.0 + (c * c * r * r / s2) * (np.cos(th) ** 2 / a ** 2 + np.sin(th) ** 2 / b ** 2))

    cap, _ = integrate.dblquad(dA, 0.0, 2 * np.pi, 0.0, np.sqrt(1.0 - t * t))
    whole = 4 * np.pi * a * b * c * special.elliprg(1 / a ** 2, 1 / b ** 2, 1 / c ** 2)
    return cap / whole


def test_ellipsoid_surface_on_surface_and_area_uniform():
    n, axes = 200_000, (1.0, 0.5, 0.25)
    pts, q = synth.ellipsoid_surface(n, axes, seed=7)
    a, b, c = axes
    assert pts.shape == (n, 3) and q.shape == (n,)
    # on the ellipsoid scaled by 0.999, so inside the cube [-1, 1]^3
    lhs = (pts[:, 0] / a) ** 2 + (pts[:, 1] / b) ** 2 + (pts[:, 2] / c) ** 2
    assert np.allclose(lhs, 0.999 ** 2, rtol=0, atol=1e-12)
    assert np.abs(pts).max() < 1.0
    # area-uniform: the share of points on a cap equals the cap's share of the area.  For
    # these axes the caps z > c/2 hold 31.5 % of the area; the plain sphere map would put
    # 25 % of the points there, so the check tells the two apart by about 60 standard errors.
    for t, sign in ((0.5, 1), (0.5, -1), (0.8, 1)):
        want = _ellipsoid_cap_fraction(a, b, c, t)
        got = np.mean(sign * pts[:, 2] / 0.999 > c * t)
        assert abs(got - want) < 5 * np.sqrt(want * (1 - want) / n), (t, sign, got, want)
    # the same along x (the long axis), where the area is thin: the caps x > a/2
    swapped = _ellipsoid_cap_fraction(c, b, a, 0.5)
    got = np.mean(pts[:, 0] / 0.999 > a * 0.5)
    assert abs(got - swapped) < 5 * np.sqrt(swapped * (1 - swapped) / n)


def test_gaussian_vectors_shape_dtype_and_moments():
    w = synth.gaussian_vectors(400, 125, seed=3, dtype=np.float32)
    assert w.shape == (400, 125) and w.dtype == np.float32
    n = w.size
    assert abs(float(w.mean())) < 5 / np.sqrt(n) and abs(float(w.var()) - 1) < 5 * np.sqrt(2 / n)
    # the float32 draw is the float64 draw rounded
    assert np.array_equal(w, synth.gaussian_vectors(400, 125, seed=3).astype(np.float32))


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_full_grid_order(level):
    g = synth.full_grid(level)
    n = 1 << level
    assert g.shape == (n ** 3, 3) and g.dtype == np.int32 and g.flags["C_CONTIGUOUS"]
    for row, (i, j, k) in enumerate(g.tolist()):
        assert (i, j, k) == (row % n, (row // n) % n, row // (n * n))


def test_occupied_cells_against_brute_force():
    pts, _ = synth.uniform_cube(3000, seed=9)
    pts = np.concatenate([pts, [[-1.0, -1.0, -1.0], [0.9999999, 0.9999999, 0.9999999], [0.0, 0.0, 0.0]]])
    for level in (0, 1, 2, 3, 4):
        n = 1 << level
        w = 2.0 / n
        want = set()
        for x, y, z in pts.tolist():
            want.add(tuple(min(n - 1, max(0, int(np.floor((v + 1.0) / w)))) for v in (x, y, z)))
        cells = synth.occupied_cells(pts, level)
        assert cells.dtype == np.int32 and cells.flags["C_CONTIGUOUS"]
        got = [tuple(r) for r in cells.tolist()]
        assert set(got) == want and len(got) == len(want)
        # x fastest: ascending linear index i + n j + n^2 k
        lin = [i + n * j + n * n * k for i, j, k in got]
        assert lin == sorted(lin)


def test_batched_tree_specs_recipe():
    specs = synth.batched_tree_specs(64, seed=4)
    assert len(specs) == 64
    ells = set()
    for i, s in enumerate(specs):
        assert 10_000 <= s["n"] <= 1_000_000
        assert s["geometry"] == ("cube" if i % 2 == 0 else "sphere")
        # leaf level: log_8(N / 64) rounded, clamped to [3, 6]
        assert s["leaf_level"] == min(6, max(3, int(round(np.log(s["n"] / 64.0) / np.log(8.0)))))
        assert s["ell"] in (4, 5, 6)
        ells.add(s["ell"])
        pts, _ = synth.tree_points(dict(s, n=50))
        if s["geometry"] == "sphere":
            assert np.allclose(np.linalg.norm(pts, axis=1), 0.999, atol=1e-12)
        else:
            assert np.abs(pts).max() <= 1.0
    assert ells == {4, 5, 6}
    assert len({s["seed"] for s in specs}) == 64
