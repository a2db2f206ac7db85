"""Pins of the oracle's adaptive, non-nested timestepping (CPU only),
Section 7.2 (Eqs. adaptive h, AdaptivityIncrementEuler and
AdaptivityIncrementSplitting) and Section 7.3 of the paper.

* A pure-Python restatement that forms each step's increment from the
  explicit sums of the two equations (the oracle accumulates them step by
  step) reproduces the oracle's path pairs and step counts.
* Where no step is ever shortened the scheme is the uniform one: the SE pair
  equals the uniform SE pair, the GL fine path the uniform GL fine path.
* The step rule keeps h_n lambda(X_n) <= h lambda(X_adapt), so SE is stable
  on a level where uniform SE diverges.
* The coarse path of level l has the law of the fine path of level l - 1
  (position moments and step counts), which is what keeps the telescoping
  sum unbiased.
* Section 7.3's findings in its scenario (X_adapt = 0.05): Var[Y_l] decays
  like h_l^2 with the reflection-aware increments (not with all S = 1),
  adaptivity lowers Var[Y_l] at a given h_l, the SE bias falls about 6x and
  the GL bias grows about 3x.
* The step rule that the library uses, a shortened step rounded down to a
  1024th of h, against the paper's min(h, lambda(X_adapt) / lambda(X_n) h)
  (the oracle's adapt_q = 30: a 2^-30 of h, 1e-9 relative to the exact
  rule): E[Y_l] and Var[Y_l] agree within 3 standard errors on levels 2..5
  of the Section 7.3 scenario, for SE and GL.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W
from test_oracle_bruteforce import bm, coef, dvdx, fold, unif, words

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
TICK_BITS = 40


def _init(p, level, i, seed):
    x = words(p, level, i, 0xFFFFFFFF, seed)
    X0, U0 = p["z0"], p["w0"]
    if p["w0_mode"] >= 1:
        xa, _ = bm(unif(p, x[0]), unif(p, x[1]))
        if p["w0_mode"] == 2:
            X0 = p["H"] * unif(p, x[2])
        U0 = coef(p, X0)[0] * xa
    return X0, U0


def adaptive_pair(p, integ, level, i, seed):
    """The adaptive pair written from the equations: the merged grid is built
    as the paths advance, every step keeps the list of (d_j, xi_j, S_j^(f))
    of the intervals inside it, and the increment is the explicit sum."""
    coupled = level > p["level_min"]
    lam_a = coef(p, p["z_adapt"])[1]
    sec = (p["T"] / p["M0"]) / 2.0 ** TICK_BITS
    T_ticks = p["M0"] << TICK_BITS
    cache = {}

    def xi(j):
        b = j // 4
        if b not in cache:
            w = words(p, level, i, b, seed)
            cache[b] = bm(unif(p, w[0]), unif(p, w[1])) + bm(unif(p, w[2]), unif(p, w[3]))
        return cache[b][j % 4]

    X0, U0 = _init(p, level, i, seed)
    paths = {"f": dict(X=X0, U=U0, S=1, hmax=1 << (TICK_BITS - level), steps=0),
             "c": dict(X=X0, U=U0, S=1, hmax=2 << (TICK_BITS - level), steps=0)}

    def begin(P, t):
        c = coef(p, P["X"])
        H, e = p["H"], p["eps_reg_frac"] * p["H"]
        n = P["hmax"]
        if min(max(P["X"], e), H - e) < p["z_adapt"]:      # lambda(X_n) > lambda(X_adapt)
            Q = 1 << (p.get("adapt_q") or 10)
            k = min(max(math.floor(Q * (lam_a / c[1])), 1), Q)
            n = k * (P["hmax"] // Q)
        n = min(n, T_ticks - t)
        P.update(c=c, n=n, end=t + n, ivals=[])

    def finish(P, Sx):
        su, lam, sig, _ = P["c"]
        h = P["n"] * sec
        ds = [d for d, _, _ in P["ivals"]]
        if integ == O.SE:
            dW = Sx * sum(w * x * math.sqrt(d) for d, x, w in P["ivals"])
            U1 = (1 - lam * h) * P["U"] - dvdx(P["c"], P["U"]) * h + sig * dW
        else:
            A = Sx * sum(w * x * math.sqrt(-math.expm1(-2 * lam * d) / (2 * lam))
                         * math.exp(-lam * sum(ds[k + 1:]))
                         for k, (d, x, w) in enumerate(P["ivals"]))
            Us = math.exp(-lam * h) * P["U"] + sig * A
            U1 = Us - dvdx(P["c"], Us) * h
        X1 = P["X"] + U1 * h
        P["X"], P["U"], P["S"] = fold(p, X1, U1, P["S"])
        P["steps"] += 1

    f, c = paths["f"], paths["c"]
    begin(f, 0)
    if coupled:
        begin(c, 0)
    t, j = 0, 0
    while t < T_ticks:
        t_next = min(f["end"], c["end"]) if coupled else f["end"]
        d = (t_next - t) * sec
        x = xi(j)
        j += 1
        Sf = f["S"] if p["coupling"] == 0 else 1
        f["ivals"].append((d, x, 1))
        if coupled:
            c["ivals"].append((d, x, Sf))
        t = t_next
        if t == f["end"]:
            finish(f, 1)
            if t < T_ticks:
                begin(f, t)
        if coupled and t == c["end"]:
            finish(c, c["S"] if p["coupling"] == 0 else 1)
            if t < T_ticks:
                begin(c, t)
    return (f["X"], f["U"], c["X"] if coupled else 0.0, c["U"] if coupled else 0.0,
            f["steps"], c["steps"] if coupled else 0)


def _dict(d, **kw):
    d = dict(d, **kw)
    d.setdefault("uniform_map", 1)
    p = O.make_params(d)
    d["H"] = p.H
    return d, p


CASES = [
    (O.SE, dict(W.bl600(O.SE), z_adapt=30.0), 7),
    (O.GL, dict(W.bl600(O.GL), z_adapt=30.0), 2),
    (O.SE, dict(W.PAPER, z_adapt=0.05), 1),
    (O.GL, dict(W.PAPER, z_adapt=0.05, coupling=1), 1),
    (O.GL, dict(W.PAPER, z_adapt=0.05, z0=0.004, uniform_map=0), 0),
    (O.SE, dict(W.PAPER, z_adapt=0.05, adapt_q=30), 2),     # the unquantized step rule
    (O.GL, dict(W.PAPER, z_adapt=0.05, adapt_q=30), 3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_adaptive_pair_equals_python_restatement(case):
    integ, d, level = CASES[case]
    d, p = _dict(d)
    for i in range(6):
        r = O.path(p, integ, level, i + 77, 987654321)
        zf, wf, zc, wc, nf, nc = adaptive_pair(d, integ, level, i + 77, 987654321)
        assert r["nonfinite"] == 0
        assert (r["steps_f"], r["steps_c"]) == (nf, nc), i
        got = np.array([r["zf"], r["wf"], r["zc"], r["wc"]])
        assert np.allclose(got, [zf, wf, zc, wc], rtol=1e-11, atol=1e-12 * d["H"]), (i, got)


@pytest.mark.parametrize("integ", [O.SE, O.GL])
def test_no_shortened_step_is_the_uniform_scheme(integ):
    # X_adapt at the regularisation height: lambda(X_adapt) = lambda_max, so
    # the ratio is >= 1 everywhere and every step is h (2h on the coarse path)
    base = W.bl600(integ) if integ == O.GL else W.bl600(O.SE)
    p_u = O.make_params(base)
    p_a = O.make_params(base, z_adapt=base["eps_reg_frac"] * 600.0)
    lm = base["level_min"]
    for level in (lm, lm + 2):
        M = 8 << level
        zs_u, bad_u = O.paths(p_u, integ, level, 40, 5, 3)
        zs_a, bad_a, steps, _ = O.paths(p_a, integ, level, 40, 5, 3, extra=True)
        assert bad_u.sum() == 0 and bad_a.sum() == 0
        assert np.all(steps[:, 0] == M)
        assert np.all(steps[:, 1] == (M // 2 if level > lm else 0))
        cols = [0, 1, 2, 3] if integ == O.SE else [0, 1]
        assert np.allclose(zs_a[:, cols], zs_u[:, cols], rtol=1e-10, atol=1e-10), level


def _lambda(p, z):
    return O.coefficients(p, z)[3]


def test_step_rule_makes_se_stable():
    # level 2 of the 600 m layer on a hierarchy from level 0: the coarse step
    # is 2h = 37.5 s against 2 / lambda_max = 2.3 s, and uniform SE diverges
    d = W.bl600(O.SE, level_min=0)
    p_u = O.make_params(d)
    level = 2
    hc = 2 * d["T"] / (8 << level)
    assert hc * _lambda(p_u, 0.0) > 2
    # X_adapt with 2h lambda(X_adapt) = 1 (lambda decreases with height)
    lo, hi = 1.0, 300.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if hc * _lambda(p_u, mid) > 1 else (lo, mid)
    p_a = O.make_params(d, z_adapt=hi)
    s_u = O.level_sums(p_u, O.SE, level, 2000, 0, 1)
    s_a = O.level_sums(p_a, O.SE, level, 2000, 0, 1)
    assert s_u["n_nonfinite"] > 0
    assert s_a["n_nonfinite"] == 0
    zs, bad = O.paths(p_a, O.SE, level, 2000, 0, 1)
    sigma_max = O.coefficients(p_a, 0.0)[0]
    assert np.abs(zs[:, [1, 3]]).max() < 6 * sigma_max      # no amplified velocities
    # adaptive levels cost more steps than M + M/2 per pair, uniform exactly that
    M = 8 << level
    assert s_u["path_steps"] == 2000 * (M + M // 2)
    assert s_a["path_steps"] > 2000 * (M + M // 2)


@pytest.mark.parametrize("integ", [O.SE, O.GL])
def test_coarse_path_has_the_law_of_the_coarser_fine_path(integ):
    p = O.make_params(dict(W.PAPER, z_adapt=0.05))
    N = 30000
    zs3, b3, st3, _ = O.paths(p, integ, 3, N, 0, 21, extra=True)
    zs2, b2, st2, _ = O.paths(p, integ, 2, N, 10 ** 6, 21, extra=True)
    assert b3.sum() == 0 and b2.sum() == 0
    for k, (a, b) in enumerate([(zs3[:, 2], zs2[:, 0]), (zs3[:, 2] ** 2, zs2[:, 0] ** 2),
                                (st3[:, 1].astype(float), st2[:, 0].astype(float))]):
        se = math.sqrt(a.var() / N + b.var() / N)
        assert abs(a.mean() - b.mean()) < 4 * se, (k, a.mean(), b.mean(), se)
    # and the pair is strongly coupled: |z_f - z_c| is far below the spread of z
    assert np.abs(zs3[:, 0] - zs3[:, 2]).mean() < 0.1 * zs3[:, 0].std()


def _level_stats(p, integ, level, N, seed):
    s = O.level_sums(p, integ, level, N, 0, seed)
    n = s["n"]
    m = s["sum"][0][0] / n
    return m, s["sum"][0][1] / n - m * m, math.sqrt((s["sum"][0][1] / n - m * m) / n)


@pytest.mark.parametrize("integ", [O.SE, O.GL])
def test_variance_decays_like_h_squared_with_the_reflection_aware_increments(integ):
    za = GOLDEN["adaptive_bias_ratio"]["X_adapt"]
    N = 20000
    aware = O.make_params(dict(W.PAPER, z_adapt=za))
    naive = O.make_params(dict(W.PAPER, z_adapt=za, coupling=1))
    uniform = O.make_params(dict(W.PAPER))
    Va = [_level_stats(aware, integ, l, N, 3)[1] for l in (3, 4)]
    Vn = [_level_stats(naive, integ, l, N, 3)[1] for l in (3, 4)]
    Vu = _level_stats(uniform, integ, 4, N, 3)[1]
    assert Va[0] / Va[1] > 3.0, Va          # beta ~ 2: a factor ~4 per level
    assert Vn[0] / Vn[1] < 2.0, Vn          # beta < 1 with all S = 1
    assert Va[1] < Vu                       # adaptivity lowers Var[Y_l] at this h_l


def test_bias_ratios_of_section_7_3():
    g = GOLDEN["adaptive_bias_ratio"]
    N = 100000
    out = {}
    for integ in (O.SE, O.GL):
        mu, _, su = _level_stats(O.make_params(dict(W.PAPER)), integ, 3, N, 5)
        ma, _, sa = _level_stats(O.make_params(dict(W.PAPER, z_adapt=g["X_adapt"])), integ, 3, N, 5)
        # E[Y_3] estimates the bias of level 2 (weak order 1)
        assert abs(mu) > 5 * su and abs(ma) > 5 * sa
        out[integ] = (abs(mu), abs(ma))
    se_ratio = out[O.SE][0] / out[O.SE][1]
    gl_ratio = out[O.GL][1] / out[O.GL][0]
    # paper: about 6x smaller for SE, about 3x larger for GL
    assert g["SE_uniform_over_adaptive"] / 2 < se_ratio < g["SE_uniform_over_adaptive"] * 2
    assert g["GL_adaptive_over_uniform"] / 2 < gl_ratio < g["GL_adaptive_over_uniform"] * 2


def test_estimate_uses_the_measured_cost():
    p = O.make_params(dict(W.PAPER, z_adapt=0.05, n_init=4000, L_max=8))
    r = O.estimate(p, O.SE, 1e-3, seed=9)
    assert r["converged"] == 1 and r["n_nonfinite"] == 0
    uniform_cost = sum(n * ((40 << l) * 3 // 2 if l > 0 else 40) for l, n in enumerate(r["N"]))
    assert r["total_path_steps"] > uniform_cost
    assert abs(r["estimate"][0] - GOLDEN["mean_position"]["value"]) < 3e-3


def test_adaptive_parameters_are_checked():
    with pytest.raises(ValueError):
        O.make_params(dict(W.PAPER, z_adapt=-0.1))
    with pytest.raises(ValueError):
        O.make_params(dict(W.PAPER, z_adapt=2.0))         # above H
    p = O.make_params(dict(W.PAPER, z_adapt=0.05))
    with pytest.raises(ValueError):
        O.path(p, O.BAOAB, 1, 0, 1)                        # Section 7.2 covers SE and GL


def _batched_stats(p, integ, level, n_batch, batches, seed):
    """Mean and variance of Y_l over batches of consecutive pairs, with the
    standard error of each from the spread of the batch estimates."""
    ms, vs = [], []
    for b in range(batches):
        s = O.level_sums(p, integ, level, n_batch, b * n_batch, seed)
        n = s["n"]
        m = s["sum"][0][0] / n
        ms.append(m)
        vs.append((s["sum"][0][1] - n * m * m) / (n - 1))
    ms, vs = np.array(ms), np.array(vs)
    return (ms.mean(), ms.std(ddof=1) / math.sqrt(batches), vs.mean(),
            vs.std(ddof=1) / math.sqrt(batches))


@pytest.mark.parametrize("integ", [O.SE, O.GL])
def test_quantized_step_rule_matches_the_exact_rule(integ):
    # Section 7.2, Eq. (adaptive h), in the Section 7.3 scenario: the two
    # rules draw the same normals per merged interval but their grids part
    # after the first shortened step, so the comparison is statistical.
    za = GOLDEN["adaptive_bias_ratio"]["X_adapt"]
    quant = O.make_params(dict(W.PAPER, z_adapt=za))
    exact = O.make_params(dict(W.PAPER, z_adapt=za, adapt_q=30))
    for level in (2, 3, 4, 5):
        n_batch = 8000 if level <= 3 else 3000
        mq, smq, vq, svq = _batched_stats(quant, integ, level, n_batch, 8, 17)
        me, sme, ve, sve = _batched_stats(exact, integ, level, n_batch, 8, 17)
        assert abs(mq - me) <= 3 * math.hypot(smq, sme), (level, mq, me, smq, sme)
        assert abs(vq - ve) <= 3 * math.hypot(svq, sve), (level, vq, ve, svq, sve)
