"""The seeded input generator against its stated recipe, by brute force on a 2,000-atom glass:
periodic cube at density 0.06 per cubic Angstrom, no two atoms closer than 2.2 Angstrom (minimum image),
a bond for exactly every pair closer than 3.5 Angstrom, 64 % type A, masses by type, lognormal spring
constants (median 1, sigma 0.3), Morton-ordered atoms, bit-identical repeats.  The generator holds no
arithmetic of the method; these tests only fix what the inputs are."""
import numpy as np
import pytest

import glassgen

N = 2000


@pytest.fixture(scope="module")
def glass():
    return glassgen.generate(N, 4)


def _min_image(pos, box):
    d = pos[None, :, :] - pos[:, None, :]
    d -= box * np.round(d / box)
    return d


def test_box_density_and_composition(glass):
    g = glass
    assert g.box == pytest.approx((N / 0.06) ** (1.0 / 3.0), rel=1e-12)
    assert np.all((g.pos >= 0.0) & (g.pos < g.box))
    assert int(np.sum(g.types == 0)) == round(0.64 * N)
    assert np.all(g.mass[g.types == 0] == 63.546) and np.all(g.mass[g.types == 1] == 91.224)


def test_minimum_distance_and_bond_set(glass):
    g = glass
    d = _min_image(g.pos, g.box)
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    iu = np.triu_indices(N, 1)
    assert r[iu].min() >= 2.2
    want = {(int(i), int(j)) for i, j in zip(*iu) if r[i, j] < 3.5}
    got = set(zip(g.bi.tolist(), g.bj.tolist()))
    assert np.all(g.bi < g.bj)
    assert len(got) == g.n_bonds  # no duplicate bonds
    assert got == want
    # unit vectors from bi to bj under the minimum image
    dv = d[g.bi, g.bj]
    assert np.allclose(g.rhat, dv / np.linalg.norm(dv, axis=1)[:, None], atol=1e-14)
    # about 10 neighbours an atom (the recipe's 11.3 blocks a BSR row, with the diagonal)
    assert 9.5 < 2.0 * g.n_bonds / N < 11.5


def test_spring_constants_lognormal(glass):
    lk = np.log(glass.k)
    m = lk.size
    assert abs(np.median(lk)) < 4 * 0.3 * 1.2533 / np.sqrt(m)
    assert abs(lk.std() - 0.3) < 5 * 0.3 / np.sqrt(2 * m)


def test_morton_order_gives_locality(glass):
    """Bonded atoms are close in index as well as in space: the Morton order of 3.5 Angstrom cells."""
    g = glass
    gap = np.abs(g.bj - g.bi)
    assert np.median(gap) < N / 20
    plain = glassgen.generate(N, 4, spatial_sort=False)
    assert np.median(gap) < 0.25 * np.median(np.abs(plain.bj - plain.bi))


def test_generator_is_deterministic(glass):
    h = glassgen.generate(N, 4)
    for f in ("pos", "mass", "types", "bi", "bj", "k", "rhat"):
        assert np.array_equal(getattr(glass, f), getattr(h, f)), f
    other = glassgen.generate(N, 5)
    assert not np.array_equal(glass.pos, other.pos)
