"""The allocation-free entry point (vecchia_loglik_grad_info_noalloc), through the C ABI.

It serves callers that cannot allocate device memory when they need a likelihood value
(GPU memory owned by another allocator or held to a fixed budget, loops that cannot take
an allocation's synchronisation).  It must give the same results as the handle-based
vecchia_loglik_grad_info on the same inputs, call after call, although every call reuses
the library's one static scratch array.  This file is collected last so that a failure
here comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import workloads
import paper_2407_02740_gb300 as vg

TOL = 1e-10
VEC_ERR_UNSUPPORTED = 7


def _close(a, b, q, p):
    ra, rb = vg.unpack(a, q, p), vg.unpack(b, q, p)
    assert abs(ra["loglik"] - rb["loglik"]) <= TOL * abs(rb["loglik"])
    scale = max(np.linalg.norm(rb["grad"]), np.sqrt(np.trace(rb["info"])))
    assert np.linalg.norm(ra["grad"] - rb["grad"]) <= TOL * scale
    assert np.linalg.norm(ra["info"] - rb["info"]) <= TOL * np.linalg.norm(rb["info"])
    assert np.linalg.norm(ra["betahat"] - rb["betahat"]) <= TOL * (np.linalg.norm(rb["betahat"]) + 1)


def test_noalloc_rejects_the_mixed_path_before_any_cuda_call():
    # only the FP64 path is offered; the check comes before the device is touched, so it
    # runs on a host without a GPU (the pointers are never dereferenced)
    lib = vg.lib()
    P = ctypes.c_void_p
    dummy = P(256)
    st = lib.vecchia_loglik_grad_info_noalloc(dummy, dummy, dummy, dummy, 100, 2, 1, 10, dummy,
                                              vg.EXP_ISO, 1, None, dummy, dummy)
    assert st == VEC_ERR_UNSUPPORTED
    assert b"VEC_FP64" in lib.vecchia_last_error()


@pytest.mark.gpu
def test_noalloc_rejects_a_plan_larger_than_its_scratch():
    # one range per coordinate with d = 20 and p = 8 has a 1243-double record; with at
    # least one block per SM the partial sums exceed the 131072 doubles of the scratch
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    n, d, p, m = 64, 20, 8, 4
    rng = np.random.default_rng(3)
    locs = torch.tensor(rng.normal(size=(n, d)), device=dev)
    y = torch.tensor(rng.normal(size=n), device=dev)
    X = torch.ones((n, p), dtype=torch.float64, device=dev)
    NN = torch.full((n, m + 1), -1, dtype=torch.int32, device=dev)
    NN[:, 0] = torch.arange(n, dtype=torch.int32, device=dev)
    th = torch.ones(d + 2, dtype=torch.float64, device=dev)
    with pytest.raises(vg.VecchiaError) as ei:
        vg.vecchia_loglik_grad_info_noalloc(locs, y, X, NN, th, vg.EXP_ANISO)
    assert ei.value.code == VEC_ERR_UNSUPPORTED
    assert "partial sums" in str(ei.value)


@pytest.mark.gpu
@pytest.mark.parametrize("covfun,theta,p,m", [
    (vg.MATERN_ISO, [2.0, 0.05, 1.5, 0.05], 3, 30),
    (vg.EXP_ISO, [1.0, 0.1, 0.01], 1, 10),
])
def test_noalloc_matches_handle_entry_point_on_two_calls(covfun, theta, p, m):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    w = workloads.make_field(3001, covfun, theta, m, p=p, seed=12, sim="sequential",
                             beta=np.linspace(1.0, -0.5, p), m_sim=m + 5)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    args = (t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64),
            t(w.NN, torch.int32))
    q = len(theta)
    th1 = t(theta, torch.float64)
    th2 = t(np.array(theta) * np.array([1.3, 0.8] + [1.1] * (q - 2)), torch.float64)
    h = vg.Handle(0)
    try:
        for th in (th1, th2):  # two calls in a row, different parameters
            ref, rst = vg.vecchia_loglik_grad_info(*args, th, covfun, handle=h)
            out, st = vg.vecchia_loglik_grad_info_noalloc(*args, th, covfun)
            torch.cuda.synchronize()
            assert int(rst[0]) == 0 and int(st[0]) == 0 and int(st[1]) == -1
            _close(out, ref, q, w.p)
    finally:
        h.close()
