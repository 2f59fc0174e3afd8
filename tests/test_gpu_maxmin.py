"""The maxmin ordering on the device (vecchia_maxmin_order) against the CPU ordering of the
same definition (workloads.maxmin_order: grid and lazy max-heap, itself pinned against the
brute-force definition): first point nearest the centroid, then the point farthest from the
chosen set, ties to the lowest index.  The orders must be identical.  The one place the
two may legitimately part is the first point, when two locations are equally near the
centroid to within the rounding of the centroid's sums; the tests check for that case
instead of comparing the rest."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def _check(x):
    ref = workloads.maxmin_order(x)
    got = vg.vecchia_maxmin_order(torch.as_tensor(x, device="cuda:0")).cpu().numpy()
    assert sorted(got.tolist()) == list(range(len(x)))          # a permutation
    if got[0] != ref[0]:
        cen = x.mean(axis=0)
        da = ((x[got[0]] - cen) ** 2).sum()
        db = ((x[ref[0]] - cen) ** 2).sum()
        assert abs(da - db) <= 1e-12 * max(da, db, 1e-300), (got[0], ref[0], da, db)
        pytest.skip("first points tie to within the centroid's rounding")
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, "first difference at position %d of %d" % (bad[0], len(x))


@pytest.mark.parametrize("n,d,seed", [(1, 2, 0), (2, 2, 1), (3, 1, 2), (257, 2, 3), (5000, 2, 4),
                                      (4000, 1, 5), (6000, 3, 6), (20011, 2, 7)])
def test_uniform_matches_cpu_ordering(n, d, seed):
    _check(np.random.default_rng(seed).uniform(size=(n, d)))


def test_clustered_and_anisotropic_extents():
    rng = np.random.default_rng(11)
    c = rng.uniform(size=(20, 2))
    x = np.concatenate([cc + 0.01 * rng.normal(size=(400, 2)) for cc in c])
    x[:, 1] *= 0.05                     # a thin strip: most cells of a square grid empty
    _check(x)


def test_lattice_with_exact_ties():
    # a regular lattice: many distances tie exactly, so the lowest-index rule decides, and
    # more candidates tie at the largest distance than the device's candidate pool holds
    g = np.arange(90, dtype=np.float64)
    x = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    _check(x)
    _check(x[np.random.default_rng(12).permutation(len(x))])


def test_duplicate_locations():
    rng = np.random.default_rng(13)
    x = rng.uniform(size=(3000, 2))
    x = np.concatenate([x, x[:1500], x[:10]])      # exact duplicates come last, by index
    _check(x)


@pytest.mark.slow
def test_full_size_uniform_and_swath():
    _check(np.random.default_rng(1002).uniform(size=(100000, 2)))
    rng = np.random.default_rng(1003)
    locs = workloads.swath_locations(rng)
    _check(locs / np.array([5.0, 5.0, 2.0]))
