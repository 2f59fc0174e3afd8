"""Semivariogram features on the device against the oracle's definition: bin counts
bit-exact (same FP64 lag arithmetic and bin decisions on both sides), bin sums to 1e-12
relative (FP64, different summation order), FP32 features to 2 ulp; several fields,
d = 2 and 3, no NNarray pairs, no random pairs, 64 bins; and run-to-run determinism."""
import numpy as np
import pytest

import workloads
from oracle import features as of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=torch.device("cuda:0"))


def _case(n, d, m, nf, npairs, seed):
    rng = np.random.default_rng(seed)
    L = rng.uniform(size=(n, d))
    L = L[workloads.maxmin_order(L)]
    NN = workloads.ordered_nn(L, m) if m > 0 else np.arange(n, dtype=np.int32)[:, None]
    Y = rng.standard_normal((nf, n)) * rng.uniform(0.5, 3, (nf, 1)) + rng.uniform(-2, 2, (nf, 1))
    # smooth the fields a little so that the bins differ
    Y += np.sin(6 * L[:, 0])[None, :]
    R = rng.integers(0, 2**32, size=(npairs, 2), dtype=np.uint64).astype(np.uint32)
    return L, NN, Y, R


def _run(L, NN, Y, R, e2):
    return vg.vecchia_fields_variogram(_dev(L, torch.float64), _dev(NN, torch.int32),
                                       _dev(Y, torch.float64), _dev(R.view(np.int32), torch.int32),
                                       _dev(e2, torch.float64), raw=True)


@pytest.mark.parametrize("n,d,m,nf,npairs,nbins", [
    (3000, 2, 30, 4, 2**18, 32),
    (1500, 3, 10, 3, 50000, 64),
    (2000, 2, 0, 2, 100000, 32),     # random pairs only
    (2500, 2, 20, 2, 0, 16),         # NNarray pairs only
])
def test_features_match_oracle(n, d, m, nf, npairs, nbins):
    L, NN, Y, R = _case(n, d, m, nf, npairs, seed=n + d + m)
    e2 = of.log_edges2(nbins)
    f, s, c = _run(L, NN, Y, R, e2)
    torch.cuda.synchronize()
    f, s, c = f.cpu().numpy(), s.cpu().numpy(), c.cpu().numpy()
    for b in range(nf):
        fo, so, co = of.features(L, NN, Y[b], R, e2)
        assert np.array_equal(c[b], co)
        assert np.allclose(s[b], so, rtol=1e-12, atol=0)
        fo32 = fo.astype(np.float32)
        assert np.all(np.abs(f[b] - fo32) <= 2 * np.spacing(np.abs(fo32)))


def test_features_are_deterministic_and_fill_empty_bins():
    L, NN, Y, R = _case(1200, 2, 8, 3, 20000, seed=9)
    # bins far beyond the domain's largest lag stay empty and copy the last filled bin
    e2 = np.geomspace(0.001, 5.0, 41) ** 2
    a = _run(L, NN, Y, R, e2)
    b = _run(L, NN, Y, R, e2)
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    f, _, c = (t.cpu().numpy() for t in a)
    assert np.any(c[0] == 0)
    for k in range(3):
        fo, _, _ = of.features(L, NN, Y[k], R, e2)
        assert np.allclose(f[k], fo.astype(np.float32), rtol=3e-7)
