"""The benchmark's error-versus-oracle bookkeeping (host logic, no GPU): the
oracle trajectory it builds and the max-abs errors it reports for a form.
A form whose rows and sampled entries are the oracle's own reports zero; a
planted deviation in one column or one entry is reported at its size."""
import numpy as np

import bench
import workloads as W


def _fake_form(cfg, rows, psis, first, steps, rng):
    ii = rng.integers(0, cfg.N, 500)
    jj = rng.integers(0, cfg.N, 500)
    psi = psis[first + steps]
    return {"obs": rows[first:first + steps + 1].copy(), "first": first, "steps": steps,
            "sample": (ii, jj, psi[ii] * psi[jj].conj())}


def test_error_of_the_oracle_itself_is_zero_and_planted_errors_show(oracle):
    cfg = W.config_n8()
    rows, psis, per_step = bench._oracle_trajectories(cfg, [5, 3, 7])
    assert rows.shape == (8, 2 * cfg.n + 5) and set(psis) == {0, 3, 5, 7} and per_step > 0
    # the trajectory is the oracle's propagate, row for row
    _, ref = oracle.propagate(cfg.n, cfg.g, cfg.omega_a, cfg.omega_c, cfg.dt, 7, W.all_excited_state(cfg.n))
    assert np.array_equal(rows, ref)
    rng = np.random.default_rng(0)
    f = _fake_form(cfg, rows, psis, 3, 4, rng)
    e = bench._error_vs_oracle(f, cfg.n, rows, psis)
    assert e["steps"] == "3..7"
    for k in ("populations", "mean_photons", "photon_number_probabilities", "rho_sampled"):
        assert e[k] == 0.0, k
    n = cfg.n
    f["obs"][2, 1] += 3e-6            # P_2 after step 5
    f["obs"][4, n] -= 2e-7            # <p> after step 7
    f["obs"][1, n + 1 + 3] += 5e-8    # P(3) after step 4
    f["sample"][2][17] += 4e-6j
    e = bench._error_vs_oracle(f, n, rows, psis)
    assert abs(e["populations"] - 3e-6) < 1e-12
    assert abs(e["mean_photons"] - 2e-7) < 1e-12
    assert abs(e["photon_number_probabilities"] - 5e-8) < 1e-12
    assert abs(e["rho_sampled"] - 4e-6) < 1e-12


def test_dicke_route_of_the_n8_workload(oracle):
    """c1 has equal couplings: the bench's second route for P(m), the Dicke
    tridiagonal evolved exactly, agrees with the full-space oracle to 1e-12 and
    reports a planted P(m) deviation; unequal couplings have no such route."""
    cfg = W.config_n8()
    rows, psis, _ = bench._oracle_trajectories(cfg, [6])
    dicke = bench._dicke_pm(cfg, 6)
    n = cfg.n
    assert dicke.shape == (7, n + 1)
    assert np.max(np.abs(dicke - rows[:, n + 1:2 * n + 2])) < 1e-12
    rng = np.random.default_rng(1)
    f = _fake_form(cfg, rows, psis, 2, 4, rng)
    f["obs"][3, n + 1 + 5] -= 7e-8      # P(5) after step 5
    e = bench._error_vs_oracle(f, n, rows, psis, dicke)
    assert abs(e["photon_number_probabilities_vs_dicke"] - 7e-8) < 1e-11
    assert bench._dicke_pm(W.config_n12(), 3) is None
