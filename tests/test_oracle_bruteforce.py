"""Third, independent evaluation of tiny cases (CPU only).

A pure-Python float64 restatement of the paper's equations -- its own Philox,
Box-Muller, profiles, the three integrators, the reflections and the coupled
coarse increments -- is compared step by step with the traces the C oracle
prints, for 8 path pairs of 16 fine steps.  It catches slips of the C code
(an index, a sign, a swapped argument) that a statistical test would miss.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

MASK = 0xFFFFFFFF


def philox(ctr, key):
    c = list(ctr)
    k0, k1 = key
    for _ in range(10):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK, p1 & MASK, ((p0 >> 32) ^ c[3] ^ k1) & MASK, p0 & MASK]
        k0 = (k0 + 0x9E3779B9) & MASK
        k1 = (k1 + 0xBB67AE85) & MASK
    return c


def words(p, level, i, block, seed):
    return philox([block, i & MASK, ((i >> 32) ^ (level << 24)) & MASK, p["stream_id"]],
                  [seed & MASK, (seed >> 32) & MASK])


def unif(p, x):
    if p["uniform_map"] == 0:
        return ((x >> 9) + 0.5) / 2.0 ** 23
    return (x + 0.5) / 2.0 ** 32


def bm(ua, ub):
    r = math.sqrt(-2 * math.log(ua))
    return r * math.cos(2 * math.pi * ub), r * math.sin(2 * math.pi * ub)


def coef(p, X):
    H = p["H"]
    e = p["eps_reg_frac"] * H
    Xc = min(max(X, e), H - e)
    su = p["kappa_sigma"] * p["u_star"] * (1 - Xc / H) ** 0.75
    tau = p["kappa_tau"] * Xc / su / (1 + p["c_f"] * p["f_coriolis"] * Xc / p["u_star"])
    lam = 1 / tau
    sig = math.sqrt(2 * su * su / tau)
    if e <= X <= H - e:
        d = -1.5 * (p["kappa_sigma"] * p["u_star"]) ** 2 * math.sqrt(1 - X / H) / H
    else:
        d = 0.0
    return su, lam, sig, d


def dvdx(c, U):
    su, _, _, d = c
    return -0.5 * (1 + U * U / (su * su)) * d


def fold(p, X, U, S):
    H = p["H"]
    while X < 0 or X > H:
        if not abs(X) <= 1e3 * H:
            raise FloatingPointError("path diverged")
        X = -X if X < 0 else 2 * H - X
        U, S = -U, -S
    return X, U, S


def step(p, integ, st, h, get_xi, half=None):
    """One step; get_xi(S, lam) returns the normal given the parity and the
    O-step lambda at the noise time; half (a list) receives BAOAB's state
    after its first half-step."""
    X, U, S = st
    if integ == 0:
        c = coef(p, X)
        xi = get_xi(S, c[1])
        U = (1 - c[1] * h) * U - dvdx(c, U) * h + c[2] * math.sqrt(h) * xi
        X = X + U * h
        return fold(p, X, U, S)
    if integ == 1:
        c = coef(p, X)
        xi = get_xi(S, c[1])
        e = math.exp(-c[1] * h)
        Us = e * U + c[2] * math.sqrt(-math.expm1(-2 * c[1] * h) / (2 * c[1])) * xi
        U = Us - dvdx(c, Us) * h
        X = X + U * h
        return fold(p, X, U, S)
    c = coef(p, X)
    U = U - dvdx(c, U) * h / 2
    X = X + U * h / 2
    X, U, S = fold(p, X, U, S)
    if half is not None:
        half.append((X, U, S))
    c = coef(p, X)
    xi = get_xi(S, c[1])
    e = math.exp(-c[1] * h)
    U = e * U + c[2] * math.sqrt(-math.expm1(-2 * c[1] * h) / (2 * c[1])) * xi
    X = X + U * h / 2
    X, U, S = fold(p, X, U, S)
    c = coef(p, X)
    U = U - dvdx(c, U) * h / 2
    return X, U, S


def pair(p, integ, level, i, seed, halves=None):
    M = p["M0"] << level
    hf, hc = ([], []) if halves is None else halves
    h = p["T"] / M
    x = words(p, level, i, 0xFFFFFFFF, seed)
    X0, U0 = p["z0"], p["w0"]
    if p["w0_mode"] >= 1:
        xa, _ = bm(unif(p, x[0]), unif(p, x[1]))
        if p["w0_mode"] == 2:
            X0 = p["H"] * unif(p, x[2])
        U0 = coef(p, X0)[0] * xa
    xi = []
    for b in range((M + 3) // 4):
        w = words(p, level, i, b, seed)
        xi += list(bm(unif(p, w[0]), unif(p, w[1]))) + list(bm(unif(p, w[2]), unif(p, w[3])))
    f = (X0, U0, 1)
    c = (X0, U0, 1)
    tf, tc = [f], [c]
    for k in range(M // 2):
        rec = {}

        def g(n):
            def get(S, lam):
                rec[n] = (S, lam)
                return xi[n]
            return get
        f = step(p, integ, f, h, g(2 * k), hf)
        tf.append(f)
        f = step(p, integ, f, h, g(2 * k + 1), hf)
        tf.append(f)
        (Sa, lam_a), (Sb, _) = rec[2 * k], rec[2 * k + 1]

        def gc(S, lam):
            Sc, sa, sb = (S, Sa, Sb) if p["coupling"] == 0 else (1, 1, 1)
            if integ == 0:
                return Sc / math.sqrt(2) * (sa * xi[2 * k] + sb * xi[2 * k + 1])
            e = math.exp(-lam_a * h)
            return Sc * (e * sa * xi[2 * k] + sb * xi[2 * k + 1]) / math.sqrt(e * e + 1)
        c = step(p, integ, c, 2 * h, gc, hc)
        tc.append(c)
    return np.array(tf), np.array(tc)


CASES = [
    (dict(W.BL600, M0=8, z0=2.0), 1),
    (dict(W.PAPER, M0=8), 1),
    (dict(W.BL600, M0=8, w0_mode=2, uniform_map=0), 1),
    (dict(W.PAPER, M0=8, coupling=1, z0=0.004), 1),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("integ", [0, 1, 2])
def test_oracle_trace_equals_python_restatement(case, integ):
    d, level = CASES[case]
    d = dict(d)
    d.setdefault("uniform_map", 1)
    if integ == 0 and d["H"] > 1.0:
        d["M0"] = 384        # SE is stable on BL600 only with h < 2.3 s
    p = O.make_params(d)
    d["H"] = p.H
    for i in range(8):
        r = O.path(p, integ, level, i + 1000, 123456789012, trace=True)
        tf, tc = pair(d, integ, level, i + 1000, 123456789012)
        assert np.allclose(r["trace_f"], tf, rtol=1e-11, atol=1e-12 * d["H"]), i
        assert np.allclose(r["trace_c"], tc, rtol=1e-11, atol=1e-12 * d["H"]), i


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_baoab_half_steps_equal_python_restatement(case):
    # the rows after the first half of each BAOAB step (the fold after the
    # first A half-step, where the step's noise enters)
    d, level = CASES[case]
    d = dict(d)
    d.setdefault("uniform_map", 1)
    p = O.make_params(d)
    d["H"] = p.H
    for i in range(8):
        r = O.path_half(p, 2, level, i + 1000, 123456789012)
        hf, hc = [], []
        tf, tc = pair(d, 2, level, i + 1000, 123456789012, (hf, hc))
        assert np.allclose(r["half_f"], np.array(hf), rtol=1e-11, atol=1e-12 * d["H"]), i
        assert np.allclose(r["half_c"], np.array(hc), rtol=1e-11, atol=1e-12 * d["H"]), i
        assert r["zf"] == pytest.approx(tf[-1][0], rel=1e-11, abs=1e-12 * d["H"])
    with pytest.raises(ValueError):
        O.path_half(p, 1, level, 0, 1)
