"""Pins for the oracle's covariance functions (Sec. 4.3 Eq. 6; Matern family).

Each value is checked against something other than the oracle itself: closed forms,
scipy's modified Bessel function, mpmath at 30 digits, or finite differences.
"""
import numpy as np
import pytest
import scipy.special as sp

import oracle

EXP, MAT, ST = oracle.EXP_ISO, oracle.MATERN_ISO, oracle.EXP_SPACETIME


def _pairs(rs, d=2):
    la = np.zeros((len(rs), d))
    lb = np.zeros((len(rs), d))
    lb[:, 0] = rs
    return la, lb


def matern_scipy(nu, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    pos = x > 0
    out[pos] = 2.0 ** (1 - nu) / sp.gamma(nu) * x[pos] ** nu * sp.kv(nu, x[pos])
    return out


def test_digamma_matches_scipy():
    xs = [0.05, 0.1, 0.5, 0.999, 1.0, 1.5, 2.3, 7.0, 19.9, 20.0]
    for x in xs:
        assert abs(oracle.digamma(x) - sp.digamma(x)) <= 2e-15 * max(1.0, abs(sp.digamma(x)))


def test_exponential_closed_form():
    theta = np.array([1.7, 0.23, 0.04])
    rs = np.array([0.0, 1e-9, 0.01, 0.1, 0.5, 3.0])
    la, lb = _pairs(rs)
    same = np.zeros(len(rs), dtype=np.int32)
    same[0] = 1
    C, dC = oracle.cov_pairs(EXP, theta, la, lb, same)
    x = rs / theta[1]
    Cref = theta[0] * np.exp(-x) + same * theta[0] * theta[2]
    assert np.allclose(C, Cref, rtol=1e-15, atol=0)
    assert np.allclose(dC[:, 0], np.exp(-x) + same * theta[2], rtol=1e-15)
    assert np.allclose(dC[:, 1], theta[0] * np.exp(-x) * rs / theta[1] ** 2, rtol=1e-14, atol=0)
    assert np.allclose(dC[:, 2], same * theta[0], rtol=0, atol=0)


@pytest.mark.parametrize("nu,closed,dclosed", [
    (0.5, lambda x: np.exp(-x), lambda x: -np.exp(-x)),
    (1.5, lambda x: (1 + x) * np.exp(-x), lambda x: -x * np.exp(-x)),
    (2.5, lambda x: (1 + x + x * x / 3) * np.exp(-x), lambda x: -(x / 3) * (1 + x) * np.exp(-x)),
])
def test_matern_half_integer_closed_forms(nu, closed, dclosed):
    rho = 0.07
    rs = np.array([1e-7, 1e-4, 0.003, 0.02, 0.07, 0.3, 1.0, 2.5])
    la, lb = _pairs(rs)
    theta = np.array([1.3, rho, nu, 0.02])
    C, dC = oracle.cov_pairs(MAT, theta, la, lb, np.zeros(len(rs), np.int32))
    x = rs / rho
    assert np.allclose(C, theta[0] * closed(x), rtol=1e-13, atol=1e-300)
    # d/drho of closed(r/rho) = closed'(x) * (-x/rho)
    assert np.allclose(dC[:, 1], theta[0] * dclosed(x) * (-x / rho), rtol=1e-13, atol=1e-300)


def test_matern_general_nu_matches_scipy_kv():
    xs = np.array([1e-6, 1e-3, 0.05, 0.3, 1.0, 2.0, 5.0, 12.0, 30.0])
    for nu in [0.05, 0.3, 0.999, 1.0, 1.0001, 1.5, 2.2, 3.0, 7.5, 20.0]:
        rho = 0.5
        la, lb = _pairs(xs * rho)
        theta = np.array([1.0, rho, nu, 0.1])
        C, dC = oracle.cov_pairs(MAT, theta, la, lb, np.zeros(len(xs), np.int32))
        ref = matern_scipy(nu, xs)
        mask = ref > 1e-250
        assert np.allclose(C[mask], ref[mask], rtol=2e-13, atol=0), nu
        # rho-derivative: rho dM/drho = 2^(1-nu)/Gamma(nu) x^(nu+1) K_{nu-1}(x)
        dref = 2.0 ** (1 - nu) / sp.gamma(nu) * xs ** (nu + 1) * sp.kv(nu - 1, xs) / rho
        m2 = dref > 1e-250
        assert np.allclose(dC[m2, 1], dref[m2], rtol=2e-12, atol=0), nu


def test_matern_nu_derivative_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30

    def M(nu, x):
        return 2 ** (1 - nu) / mpmath.gamma(nu) * x ** nu * mpmath.besselk(nu, x)

    rho = 1.0
    for nu in [0.05, 0.5, 1.0, 1.5, 2.71, 8.0]:
        for x in [1e-4, 0.01, 0.2, 1.0, 4.0, 15.0]:
            ref = float(mpmath.diff(lambda v: M(v, mpmath.mpf(x)), mpmath.mpf(nu)))
            la, lb = _pairs(np.array([x * rho]))
            _, dC = oracle.cov_pairs(MAT, np.array([1.0, rho, nu, 0.1]), la, lb,
                                     np.zeros(1, np.int32))
            # absolute accuracy relative to the O(1) scale of the Matern function
            assert abs(dC[0, 2] - ref) <= 1e-14 + 1e-12 * abs(ref), (nu, x, dC[0, 2], ref)


def test_matern_nugget_and_diagonal():
    theta = np.array([2.0, 0.1, 1.2, 0.05])
    la = np.zeros((1, 2))
    C, dC = oracle.cov_pairs(MAT, theta, la, la, np.ones(1, np.int32))
    assert C[0] == pytest.approx(2.0 * 1.05, rel=1e-15)
    assert dC[0, 0] == pytest.approx(1.05, rel=1e-15)
    assert dC[0, 1] == 0.0 and dC[0, 2] == 0.0
    assert dC[0, 3] == pytest.approx(2.0, rel=1e-15)


def test_spacetime_values_and_fd_derivatives():
    theta = np.array([1.1, 5.0, 2.0, 0.1])
    rng = np.random.default_rng(7)
    la = rng.uniform(0, 20, size=(12, 3))
    lb = la + rng.normal(0, 4, size=(12, 3))
    lb[0] = la[0]  # coincident pair (off-diagonal)
    same = np.zeros(12, np.int32)
    C, dC = oracle.cov_pairs(ST, theta, la, lb, same)
    D = np.sqrt(((la[:, :2] - lb[:, :2]) ** 2).sum(1) / 25.0 + (la[:, 2] - lb[:, 2]) ** 2 / 4.0)
    assert np.allclose(C, 1.1 * np.exp(-D), rtol=1e-14)
    for j in (1, 2):
        h = 1e-6 * theta[j]
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        Cp, _ = oracle.cov_pairs(ST, tp, la, lb, same)
        Cm, _ = oracle.cov_pairs(ST, tm, la, lb, same)
        fd = (Cp - Cm) / (2 * h)
        assert np.allclose(dC[:, j], fd, rtol=1e-7, atol=1e-12)
    assert dC[0, 1] == 0.0 and dC[0, 2] == 0.0


ANI = oracle.EXP_ANISO


def test_anisotropic_values_and_fd_derivatives():
    d = 5
    theta = np.array([1.4, 0.3, 0.7, 1.1, 2.5, 0.45, 0.08])
    rng = np.random.default_rng(11)
    la = rng.uniform(0, 2, size=(15, d))
    lb = la + rng.normal(0, 0.5, size=(15, d))
    lb[0] = la[0]                                      # coincident pair (off-diagonal)
    same = np.zeros(15, np.int32)
    C, dC = oracle.cov_pairs(ANI, theta, la, lb, same)
    D = np.sqrt((((la - lb) / theta[1:-1]) ** 2).sum(1))
    assert np.allclose(C, 1.4 * np.exp(-D), rtol=1e-14)
    assert np.allclose(dC[:, 0], np.exp(-D), rtol=1e-14)
    for j in range(1, d + 1):
        h = 1e-6 * theta[j]
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (oracle.cov_pairs(ANI, tp, la, lb, same)[0]
              - oracle.cov_pairs(ANI, tm, la, lb, same)[0]) / (2 * h)
        # central-difference rounding: ~1e-16 C / h absolute
        assert np.allclose(dC[:, j], fd, rtol=1e-7, atol=1e-9)
    assert np.all(dC[0, 1:] == 0.0) and np.all(dC[:, d + 1] == 0.0)
    # the diagonal: nugget sigma2 tau2, d/dsigma2 = 1 + tau2, d/dtau2 = sigma2
    C, dC = oracle.cov_pairs(ANI, theta, la[:1], la[:1], np.ones(1, np.int32))
    assert C[0] == pytest.approx(1.4 * 1.08, rel=1e-15)
    assert dC[0, 0] == pytest.approx(1.08, rel=1e-15) and dC[0, d + 1] == pytest.approx(1.4)


def test_anisotropic_reduces_to_isotropic_and_spacetime():
    rng = np.random.default_rng(12)
    la, lb = rng.uniform(size=(20, 3)), rng.uniform(size=(20, 3))
    same = np.zeros(20, np.int32)
    # equal ranges: the isotropic exponential; the range derivatives sum to d C/d rho
    Ca, dCa = oracle.cov_pairs(ANI, np.array([1.2, 0.3, 0.3, 0.3, 0.05]), la, lb, same)
    Ci, dCi = oracle.cov_pairs(EXP, np.array([1.2, 0.3, 0.05]), la, lb, same)
    assert np.allclose(Ca, Ci, rtol=1e-14)
    assert np.allclose(dCa[:, 1:4].sum(1), dCi[:, 1], rtol=1e-13)
    # rho_1 = rho_2: the space-time exponential (space = first two coordinates)
    Ca, dCa = oracle.cov_pairs(ANI, np.array([0.9, 0.4, 0.4, 0.7, 0.1]), la, lb, same)
    Cs, dCs = oracle.cov_pairs(ST, np.array([0.9, 0.4, 0.7, 0.1]), la, lb, same)
    assert np.allclose(Ca, Cs, rtol=1e-14)
    assert np.allclose(dCa[:, 1] + dCa[:, 2], dCs[:, 1], rtol=1e-13)
    assert np.allclose(dCa[:, 3], dCs[:, 2], rtol=1e-13)


def test_anisotropic_parameter_count():
    assert oracle.nparms(ANI, 18) == 20
    assert oracle._load().orc_nparms_d(ANI, 18) == 20       # noqa: SLF001
    assert oracle._load().orc_nparms_d(ANI, 21) == -1       # noqa: SLF001
    assert oracle._load().orc_nparms(ANI) == -1             # noqa: SLF001
    with pytest.raises(ValueError):
        oracle.nparms(ANI, 21)
    la = np.zeros((1, 4))
    with pytest.raises(oracle.OracleError):
        oracle.cov_pairs(ANI, np.array([1.0, 0.1, -0.2, 0.1, 0.3, 0.01]), la, la,
                         np.ones(1, np.int32))


def test_invalid_parameters_rejected():
    la = np.zeros((1, 2))
    with pytest.raises(oracle.OracleError):
        oracle.cov_pairs(EXP, np.array([1.0, -0.1, 0.01]), la, la, np.ones(1, np.int32))
    with pytest.raises(oracle.OracleError):
        oracle.cov_pairs(MAT, np.array([1.0, 0.1, 25.0, 0.01]), la, la, np.ones(1, np.int32))
