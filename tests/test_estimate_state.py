"""The checkpointable host-driven estimator (CPU part): argument checks,
the state's exact JSON round trip, the result of a given state, and the
complete state's no-op pass -- all host logic, no device work."""
import ctypes as C
import json
import math
import random

import pytest

import paper_1612_07717_gb300 as G


def _begin(eps=0.5, integ=G.BAOAB, **kw):
    p = G.make_params(**kw)
    st = G.EstimateState()
    rc = G.lib().mlmc_estimate_begin(eps, integ, C.byref(p), 7, C.byref(st))
    return rc, p, st


def test_begin_checks_its_arguments():
    assert _begin(eps=0.0)[0] == G.EINVAL
    assert _begin(eps=-1.0)[0] == G.EINVAL
    assert _begin(integ=3)[0] == G.EINVAL
    assert _begin(L_max=1, level_min=0)[0] == G.EINVAL
    assert _begin(n_init=1)[0] == G.EINVAL
    rc, p, st = _begin(level_min=2, L_max=9)
    assert rc == G.OK
    assert (st.L, st.phase, st.converged, st.passes, st.seed, st.integrator) == (2, 0, 0, 0, 7, G.BAOAB)
    assert st.eps == 0.5 and all(x == 0 for x in st.n_done)


def _filled(seed=3):
    rng = random.Random(seed)
    e = G.Estimation.__new__(G.Estimation)
    st = G.EstimateState()
    st.eps, st.seed, st.integrator, st.L, st.phase = 1.0 / 3.0, 2 ** 63 + 5, 1, 6, 1
    st.seconds, st.passes = math.pi * 1e-3, 11
    for l in range(G.MAX_LEVELS):
        st.n_done[l] = rng.getrandbits(64)
        st.n[l] = rng.getrandbits(40)
        st.n_nonfinite[l] = rng.getrandbits(8)
        st.path_steps[l] = rng.getrandbits(60)
        for q in range(2):
            for k in range(6):
                st.sum[l][q][k] = rng.uniform(-1e6, 1e6) * 10.0 ** rng.randint(-300, 300)
    e.state = st
    return e


def test_state_round_trips_through_json_exactly():
    a = _filled()
    text = json.dumps(a.state_dict())
    b = G.Estimation.__new__(G.Estimation)
    b.load_state_dict(json.loads(text))
    assert bytes(a.state) == bytes(b.state)


def test_result_of_a_state():
    p = G.make_params(level_min=0, L_max=6)
    st = G.EstimateState()
    st.L, st.phase, st.converged = 2, 2, 1
    data = {0: (1000, [50.0, 30.0]), 1: (400, [-2.0, 1.5]), 2: (100, [0.25, 0.2])}
    for l, (n, (m1, m2)) in data.items():
        st.n[l] = n
        st.path_steps[l] = n * 10
        st.sum[l][0][0], st.sum[l][0][1] = m1, m2
        st.sum[l][1][0], st.sum[l][1][1] = m1 / 2, m2 / 4
    r = G.Result()
    rc = G.lib().mlmc_estimate_result(C.byref(st), C.byref(p), C.byref(r))
    assert rc == G.OK
    est = sum(m1 / n for n, (m1, _) in data.values())
    var = sum(max((m2 - m1 * m1 / n) / (n - 1), 0.0) / n for n, (m1, m2) in data.values())
    assert r.estimate[0] == pytest.approx(est, rel=1e-15)
    assert r.est_variance[0] == pytest.approx(var, rel=1e-15)
    assert r.L == 2 and r.converged == 1 and r.total_path_steps == 15000
    st.n_nonfinite[1] = 3
    assert G.lib().mlmc_estimate_result(C.byref(st), C.byref(p), C.byref(r)) == G.ENONFINITE
    st.n_nonfinite[1] = 0
    st.converged = 0
    assert G.lib().mlmc_estimate_result(C.byref(st), C.byref(p), C.byref(r)) == G.ENOTCONV


def test_a_complete_state_needs_no_device():
    p = G.make_params()
    st = G.EstimateState()
    st.L, st.phase = p.level_min + 2, 2
    # phase 2: the pass returns at once (no workspace, no stream touched)
    assert G.lib().mlmc_estimate_pass(C.byref(st), C.byref(p), None, 0, None) == 1
    st.phase = 7
    assert G.lib().mlmc_estimate_pass(C.byref(st), C.byref(p), None, 0, None) == G.EINVAL


def test_rates_recover_known_decay():
    L = 8
    r = dict(mean_y=[5.0] + [3.0 * 2.0 ** (-1.0 * l) for l in range(1, L + 1)],
             V=[7.0] + [0.5 * 2.0 ** (-2.0 * l) for l in range(1, L + 1)])
    got = G.rates(r)
    assert got["alpha"] == pytest.approx(1.0, abs=1e-12)
    assert got["beta"] == pytest.approx(2.0, abs=1e-12)
    # level_min shifts the level index, not the slope; too few levels give None
    assert G.rates(r, level_min=6)["beta"] == pytest.approx(2.0, abs=1e-12)
    assert G.rates(dict(mean_y=[1.0, 0.5], V=[1.0, 0.25]))["alpha"] is None
