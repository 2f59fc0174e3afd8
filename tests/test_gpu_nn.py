"""Ordered nearest neighbours on the device, bit-exact against the CPU search of the same
definition (workloads/prep.c, pinned against brute force): uniform, clustered and lattice
points (many exact distance ties, broken by the lower index), d = 1, 2, 3, m = 0, m > n,
a single point, and the full 1.2 M-point space-time swath."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def _gpu_nn(L, m):
    NN = vg.vecchia_ordered_nn(torch.as_tensor(np.ascontiguousarray(L), dtype=torch.float64,
                                               device="cuda:0"), m)
    torch.cuda.synchronize()
    return NN.cpu().numpy()


def _ordered(L):
    return L[workloads.maxmin_order(L)]


@pytest.mark.parametrize("n,d,m,seed", [
    (5000, 2, 30, 1), (20000, 2, 10, 2), (3000, 1, 8, 3), (6000, 3, 20, 4), (700, 2, 60, 5),
    (2500, 2, 80, 6)])
def test_uniform_points(n, d, m, seed):
    L = _ordered(np.random.default_rng(seed).uniform(size=(n, d)))
    assert np.array_equal(_gpu_nn(L, m), workloads.ordered_nn(L, m))


def test_clustered_points():
    rng = np.random.default_rng(7)
    centres = rng.uniform(size=(12, 2))
    L = np.concatenate([c + 0.01 * rng.standard_normal((800, 2)) for c in centres])
    L = _ordered(np.concatenate([L, rng.uniform(size=(500, 2))]))
    assert np.array_equal(_gpu_nn(L, 25), workloads.ordered_nn(L, 25))


def test_lattice_ties_go_to_the_lower_index():
    g = np.arange(60, dtype=np.float64)
    L = _ordered(np.array([(a, b) for a in g for b in g]))
    got = _gpu_nn(L, 12)
    assert np.array_equal(got, workloads.ordered_nn(L, 12))
    assert np.array_equal(got[:400], workloads.ordered_nn(L[:400], 12, brute=True))


def test_edge_cases():
    L = _ordered(np.random.default_rng(8).uniform(size=(50, 2)))
    assert np.array_equal(_gpu_nn(L, 0), np.arange(50, dtype=np.int32)[:, None])
    assert np.array_equal(_gpu_nn(L, 70), workloads.ordered_nn(L, 70))    # m > n: -1 padding
    assert np.array_equal(_gpu_nn(L[:1], 5), np.array([[0, -1, -1, -1, -1, -1]], np.int32))
    same = np.zeros((40, 2))                                                 # coincident points
    assert np.array_equal(_gpu_nn(same, 6), workloads.ordered_nn(same, 6))


@pytest.mark.slow
def test_full_size_swath():
    # the workload's neighbours are searched on the coordinates scaled by the ranges
    w = workloads.cfg_swath_1m2()
    scaled = w.locs / np.array([w.theta_true[1], w.theta_true[1], w.theta_true[2]])
    assert np.array_equal(_gpu_nn(scaled, w.m), w.NN)
