"""The library's host builder of grouped-conditioning blocks (vecchia_group_blocks, no GPU
needed) against the oracle's, bit for bit, and its argument errors."""
import numpy as np
import pytest

import workloads
from oracle import grouped as og

vg = pytest.importorskip("paper_2407_02740_gb300")


@pytest.mark.parametrize("n,m,g,seed", [(3000, 30, 8, 1), (500, 10, 3, 2), (200, 5, 40, 3)])
def test_blocks_match_oracle(n, m, g, seed):
    w, goff = workloads.grouped_field(n, 1, [1.0, 0.1, 1.0, 0.05], m, g, seed=seed, m_sim=10)
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, goff)
    o_off, o_idx, o_nm = og.group_blocks(w.NN, goff)
    assert np.array_equal(off, o_off) and np.array_equal(idx, o_idx) and np.array_equal(nm, o_nm)
    assert kmax == int(np.diff(off).max())


def test_singletons_and_one_group():
    w, _ = workloads.grouped_field(300, 1, [1.0, 0.1, 1.0, 0.05], 8, 4, seed=4, m_sim=8)
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, np.arange(w.n + 1))
    assert np.all(nm == 1) and kmax == 9
    for i in (0, 5, 299):      # block i = i's neighbours ascending, then i
        nb = sorted(int(j) for j in w.NN[i, 1:] if j >= 0)
        assert list(idx[off[i]:off[i + 1]]) == nb + [i]
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, [0, w.n])
    assert list(idx) == list(range(w.n)) and nm[0] == w.n and kmax == w.n


def test_bad_arguments():
    w, goff = workloads.grouped_field(200, 1, [1.0, 0.1, 1.0, 0.05], 8, 4, seed=5, m_sim=8)
    for bad in ([0, 50, 50, 200], [0, 100], [1, 200], [0, 120, 100, 200]):
        with pytest.raises(vg.VecchiaError):
            vg.vecchia_group_blocks(w.NN, bad)
    NN = w.NN.copy()
    NN[40, 2] = 41                          # a neighbour that does not precede its row
    with pytest.raises(vg.VecchiaError):
        vg.vecchia_group_blocks(NN, goff)
    NN = w.NN.copy()
    NN[3, 4:] = -1                          # row 3 has 3 neighbours: pad, then a neighbour
    NN[3, 5] = 0
    with pytest.raises(vg.VecchiaError):
        vg.vecchia_group_blocks(NN, goff)


@pytest.mark.parametrize("nclass", [1, 2, 3, 5])
def test_group_classes_partition_the_groups(nclass):
    w, goff = workloads.grouped_field(3000, 1, [1.0, 0.1, 1.0, 0.05], 30, 8, seed=6, m_sim=10)
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, goff)
    gorder, coff, ckmax = vg.vecchia_group_classes(off, nclass)
    ng = len(off) - 1
    assert sorted(gorder.tolist()) == list(range(ng)) and coff[0] == 0 and coff[-1] == ng
    size = np.diff(off)
    lo = 0
    for c in range(nclass):
        grp = gorder[coff[c]:coff[c + 1]]
        if len(grp) == 0:
            assert ckmax[c] == 0
            continue
        sz = size[grp]                                        # larger blocks first,
        assert np.all(np.diff(sz) <= 0)                       # then ascending index
        assert np.all((np.diff(sz) < 0) | (np.diff(grp) > 0))
        assert size[grp].max() == ckmax[c] and size[grp].min() > lo
        lo = ckmax[c]
    assert ckmax.max() == kmax
    if nclass == 1:
        assert coff[1] == ng
    # more classes never cost more (sum of groups x largest size^2)
    cost = sum((coff[c + 1] - coff[c]) * int(ckmax[c]) ** 2 for c in range(nclass))
    assert cost <= ng * kmax ** 2


def test_group_classes_errors_and_single_group():
    off = np.array([0, 12], dtype=np.int64)
    gorder, coff, ckmax = vg.vecchia_group_classes(off, 4)
    assert list(gorder) == [0] and list(coff) == [0, 1, 1, 1, 1] and list(ckmax) == [12, 0, 0, 0]
    for nclass in (0, 17):
        with pytest.raises(vg.VecchiaError):
            vg.vecchia_group_classes(off, nclass)
    with pytest.raises(vg.VecchiaError):
        vg.vecchia_group_classes(np.array([0, 5, 5, 9], dtype=np.int64), 2)   # an empty block


@pytest.mark.parametrize("seed", range(6))
def test_group_classes_minimise_the_stated_cost(seed):
    # brute force over every split of the distinct block sizes into at most nclass ranges
    import itertools
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, 82, size=int(rng.integers(3, 40)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    nclass = int(rng.integers(1, 4))
    gorder, coff, ckmax = vg.vecchia_group_classes(off, nclass)
    got = sum((coff[c + 1] - coff[c]) * int(ckmax[c]) ** 2 for c in range(nclass))
    vals = np.unique(sizes)
    best = None
    for k in range(1, min(nclass, len(vals)) + 1):
        for cuts in itertools.combinations(range(1, len(vals)), k - 1):
            bounds = list(cuts) + [len(vals)]
            lo, cost = 0, 0
            for b in bounds:
                top = vals[b - 1]
                cost += int(np.sum((sizes > (vals[lo - 1] if lo else 0)) & (sizes <= top))) * int(top) ** 2
                lo = b
            best = cost if best is None else min(best, cost)
    assert got == best
