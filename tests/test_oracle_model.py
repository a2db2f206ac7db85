"""Pins of the oracle's model arithmetic: profiles, integrators, reflection
and the coarse/fine coupling (CPU only).

Each test checks the oracle against something other than its own formula:
a finite-difference derivative, special values of the profiles, numbers the
paper prints, exact discrete moments of the linear constant-coefficient
recurrences, the paper's algebraic form of the reflected step, and the exact
fine/coarse agreement that the O-step coupling implies.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ----------------------------------------------------------------------------- profiles
def test_dsigma2_dz_matches_finite_difference():
    p = O.make_params(W.BL600)
    H = p.H
    for z in np.linspace(0.01 * H, 0.99 * H, 37):
        d = 1e-4
        f1 = O.coefficients(p, z + d)[1]
        f0 = O.coefficients(p, z - d)[1]
        fd = (f1 - f0) / (2 * d)
        assert O.coefficients(p, z)[2] == pytest.approx(fd, rel=1e-6)


def test_regularised_profile_is_frozen_outside_band():
    p = O.make_params(W.BL600)
    H, eps = p.H, p.eps_reg_frac * p.H
    lo = O.coefficients(p, eps)
    hi = O.coefficients(p, H - eps)
    for z in (0.0, 0.3 * eps, 0.99 * eps):
        c = O.coefficients(p, z)
        assert np.allclose(c[[0, 1, 3, 4]], lo[[0, 1, 3, 4]], rtol=0, atol=0)
        assert c[2] == 0.0          # derivative of the frozen profile
    for z in (H, H - 0.5 * eps):
        c = O.coefficients(p, z)
        assert np.allclose(c[[0, 1, 3, 4]], hi[[0, 1, 3, 4]], rtol=0, atol=0)
        assert c[2] == 0.0
    # the alternative reading keeps the band-edge derivative
    p1 = O.make_params(W.BL600, drift_outside=1)
    assert O.coefficients(p1, 0.5 * eps)[2] == pytest.approx(O.coefficients(p1, eps)[2])


def test_profile_special_values():
    # sigma_U at 1 - z/H = 1/16 is kappa u* / 8 ((1/16)^(3/4) = 1/8)
    p = O.make_params(W.PAPER)
    z = 1.0 - 1.0 / 16.0
    assert O.coefficients(p, z)[0] == pytest.approx(1.3 * 0.2 / 8.0, rel=1e-14)
    # surface-layer limit of tau = 0.5 z / sigma_U with sigma_U -> 1.3 u*
    # (the form the paper takes from Wilson 2009, Section 2)
    z = 0.02
    tau = 1.0 / O.coefficients(p, z)[3]
    assert tau == pytest.approx(0.5 * z / (1.3 * 0.2), rel=0.02)
    # sigma^2 = 2 sigma_U^2 / tau
    c = O.coefficients(p, 0.3)
    assert c[4] ** 2 == pytest.approx(2 * c[1] * c[3], rel=1e-14)


def test_tau_at_regularisation_height_matches_paper():
    p = O.make_params(W.PAPER)          # nondimensional: t_ref = 1000 s
    tau_s = 1000.0 / O.coefficients(p, p.eps_reg_frac)[3]
    g = GOLDEN["tau_at_eps_reg_seconds"]["value"]
    assert 0.9 * g < tau_s <= g         # "does not exceed 20 s"


def test_se_stability_bound_matches_paper_M0_270():
    p = O.make_params(W.PAPER, eps_reg_frac=1e-3)
    lam_max = O.coefficients(p, 1e-3)[3]
    M0 = GOLDEN["se_stable_M0_eps_reg_0.001"]["M0"]
    assert lam_max / M0 < 2.0           # h lambda < 2: stable
    assert lam_max / 250 > 2.0          # a rounder, smaller M0 would not be


def test_bl600_se_stability_level():
    p = O.make_params(W.BL600)
    lam_max = O.coefficients(p, 0.0)[3]
    h6 = p.T / (8 << 6)
    h5 = p.T / (8 << 5)
    assert lam_max * h6 < 2.0 <= lam_max * h5


# ------------------------------------------------------------------------ integrators
def _const_params(**kw):
    # eps_reg = H/2 freezes sigma_U and tau at their mid-height values, so
    # lambda and sigma are constants and d sigma_U^2/dz = 0 away from z = H/2.
    d = dict(W.BL600, H=1000.0, eps_reg_frac=0.5, c_f=15.0, f_coriolis=1e-2, z0=300.0,
             w0=0.3, w0_mode=0, T=20.0, M0=16, level_min=0)
    d.update(kw)
    return O.make_params(d)


def _linear_moments(A, B, x0, M):
    mean = np.array(x0, dtype=float)
    cov = np.zeros((2, 2))
    for _ in range(M):
        mean = A @ mean
        cov = A @ cov @ A.T + np.outer(B, B)
    return mean, cov


@pytest.mark.parametrize("integ", [O.SE, O.GL, O.BAOAB])
def test_constant_coefficient_discrete_moments(integ):
    p = _const_params()
    M = p.M0
    h = p.T / M
    c = O.coefficients(p, 300.0)
    sig_u, lam, sig = c[0], c[3], c[4]
    assert c[2] == 0.0
    if integ == O.SE:
        a = 1 - lam * h
        A = np.array([[1.0, h * a], [0.0, a]])
        B = np.array([h * sig * math.sqrt(h), sig * math.sqrt(h)])
    else:
        e = math.exp(-lam * h)
        cn = sig_u * math.sqrt(1 - e * e)
        if integ == O.GL:
            A = np.array([[1.0, h * e], [0.0, e]])
            B = np.array([h * cn, cn])
        else:
            A = np.array([[1.0, h / 2 + h / 2 * e], [0.0, e]])
            B = np.array([h / 2 * cn, cn])
    mean, cov = _linear_moments(A, B, [p.z0, p.w0], M)
    N = 40000
    zs, bad = O.paths(p, integ, 0, N, 0, 5)
    assert bad.sum() == 0
    X, U = zs[:, 0], zs[:, 1]
    assert abs(X.mean() - mean[0]) < 4 * math.sqrt(cov[0, 0] / N)
    assert abs(U.mean() - mean[1]) < 4 * math.sqrt(cov[1, 1] / N)
    assert abs(X.var() - cov[0, 0]) < 4 * cov[0, 0] * math.sqrt(2.0 / N)
    assert abs(U.var() - cov[1, 1]) < 4 * cov[1, 1] * math.sqrt(2.0 / N)
    cxu = np.mean((X - X.mean()) * (U - U.mean()))
    assert abs(cxu - cov[0, 1]) < 5 * math.sqrt(cov[0, 0] * cov[1, 1] / N)


def test_gl_ou_velocity_is_exact_in_h():
    # With constant coefficients the O-step is the exact OU transition, so the
    # GL velocity variance at T does not depend on h: sigma_U^2 (1 - e^{-2 lam T}).
    for M0 in (4, 64):
        p = _const_params(M0=M0)
        c = O.coefficients(p, 300.0)
        exact = c[1] * (1 - math.exp(-2 * c[3] * p.T))
        N = 30000
        zs, _ = O.paths(p, O.GL, 0, N, 0, 11)
        U = zs[:, 1]
        mean_exact = p.w0 * math.exp(-c[3] * p.T)
        assert abs(U.mean() - mean_exact) < 4 * math.sqrt(exact / N)
        assert abs(U.var() - exact) < 4 * exact * math.sqrt(2.0 / N)


# ------------------------------------------------------------------------- reflection
@pytest.mark.parametrize("integ", [O.SE, O.GL])
def test_reflected_step_matches_paper_form(integ):
    # Eq. (reflected_equation): X_{n+1} = s (X_n + s U_{n+1} h) with
    # s = S_{n+1} S_n; here checked on traces with many reflections.
    p = O.make_params(W.BL600, z0=3.0)
    M = 64
    h = p.T / M
    seen = 0
    for i in range(40):
        r = O.path(p, integ, 3, i, 3, trace=True)
        tf = r["trace_f"]
        assert np.all(tf[:, 0] >= 0) and np.all(tf[:, 0] <= p.H)
        assert np.all(np.abs(tf[:, 2]) == 1)
        for n in range(M):
            Xn, Sn = tf[n, 0], tf[n, 2]
            X1, U1, S1 = tf[n + 1]
            s = S1 * Sn
            assert X1 == pytest.approx(s * (Xn + s * U1 * h), abs=1e-9 * p.H)
            seen += s < 0
        # parity equals (-1)^(number of reflections)
        assert tf[-1, 2] == (-1) ** r["refl_f"]
    assert seen > 20


@pytest.mark.parametrize("integ", [O.GL, O.BAOAB])
def test_coupling_keeps_fine_and_coarse_speed_equal_with_walls(integ):
    # Constant lambda, sigma and no drift: in the extended variables the fine
    # pair of O-steps and the coarse O-step of 2h coincide (Eq.
    # SymEulerCoupled), so |U_f(t_2k)| = |U_c(t_k)| through any number of
    # reflections when the coarse normal carries the S factors of Eq.
    # (splitting_coupled_treatment), and not with the naive S = 1.
    base = dict(H=5.0, z0=1.0, w0=-0.3, T=60.0, M0=64)
    p = _const_params(**base)
    pn = _const_params(coupling=1, **base)
    differ = 0
    naive_bad = 0
    for i in range(30):
        r = O.path(p, integ, 1, i, 9, trace=True)
        tf, tc = r["trace_f"], r["trace_c"]
        assert np.allclose(np.abs(tf[::2, 1]), np.abs(tc[:, 1]), rtol=1e-9, atol=1e-12)
        differ += int(np.any(tf[::2, 2] != tc[:, 2]))
        rn = O.path(pn, integ, 1, i, 9, trace=True)
        naive_bad += int(not np.allclose(np.abs(rn["trace_f"][::2, 1]),
                                         np.abs(rn["trace_c"][:, 1]), rtol=1e-6))
    assert differ >= 10       # parities did differ, so the S factors mattered
    assert naive_bad >= 10


def test_divergence_is_flagged_on_unstable_se_level():
    p = O.make_params(W.bl600(O.SE, level_min=0))
    s = O.level_sums(p, O.SE, 2, 2000, 0, 1)
    assert s["n_nonfinite"] > 0
    assert s["n"] + s["n_nonfinite"] == 2000
