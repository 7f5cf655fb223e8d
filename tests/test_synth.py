"""The seeded input generator follows its stated recipe (no GPU).

Checked on draws large enough for the statistics to be tight:
  * h: diagonal in [-3, 2), off-diagonal normal with standard deviation 0.05, symmetric;
  * L^J: symmetric; amplitude exp(-J / tau) exp(-|m - n| / 6) * scale on a standard normal,
    so log E|L^J_mn| falls linearly in J (slope -1 / tau) and in |m - n| (slope -1 / 6);
  * the same seed gives the same draw, another seed another draw;
  * RHF output: canonical (diagonal) Fock matrix, aufbau occupation (every occupied orbital
    energy below every virtual one), ERIs g = sum_J L^J L^J positive semidefinite;
  * levels nested, CCSD at the highest occupied and lowest virtual orbitals;
  * the workload table: tau = N_J / 5 and scale = 0.5 / sqrt(tau);
  * the serving mix: sizes, Cholesky counts, active fractions and the two request kinds in
    their stated ranges and proportions, one stream per request, exponential arrival gaps
    at the stated rate.
"""
import math

import numpy as np
import pytest

from synth.generator import (CONFIGS, SystemSpec, default_scale, draw_model_hamiltonian, level_map, make_system,
                             serving_arrivals, serving_request_spec)


def test_one_electron_matrix():
    ham = draw_model_hamiltonian(400, 2, 10.0, seed=3)
    h = ham.h
    assert np.array_equal(h, h.T)
    d = np.diag(h)
    assert d.min() >= -3.0 and d.max() < 2.0
    assert abs(d.mean() - (-0.5)) < 0.15          # U[-3, 2] has mean -0.5, sd 1.44 / sqrt(400)
    off = h[np.triu_indices(400, 1)]
    assert abs(off.std() - 0.05) < 0.002 and abs(off.mean()) < 0.002


def test_cholesky_vectors_decay_as_stated():
    n, nj, tau, scale = 60, 120, 30.0, 0.7
    L = draw_model_hamiltonian(n, nj, tau, seed=5, scale=scale).L
    assert np.array_equal(L, L.transpose(0, 2, 1))
    # decay in J: mean |L| over each J against exp(-J / tau) (E|z| = sqrt(2 / pi))
    band = np.exp(-np.abs(np.subtract.outer(np.arange(n), np.arange(n))) / 6.0)
    iu = np.triu_indices(n)
    ratio = np.abs(L[:, iu[0], iu[1]]) / band[iu][None, :]
    per_J = ratio.mean(axis=1) / (scale * math.sqrt(2.0 / math.pi))
    slope = np.polyfit(np.arange(nj), np.log(per_J), 1)[0]
    assert abs(slope - (-1.0 / tau)) < 0.1 / tau
    # decay across the band: mean |L| over each distance |m - n| against exp(-|m-n| / 6)
    dist = np.abs(iu[0] - iu[1])
    w = np.exp(np.arange(nj) / tau)[:, None]
    norm = np.abs(L[:, iu[0], iu[1]]) * w
    per_d = np.array([norm[:, dist == k].mean() for k in range(20)])
    slope_d = np.polyfit(np.arange(20), np.log(per_d), 1)[0]
    assert abs(slope_d - (-1.0 / 6.0)) < 0.02


def test_seeded_and_reproducible():
    a = draw_model_hamiltonian(20, 5, 4.0, seed=9)
    b = draw_model_hamiltonian(20, 5, 4.0, seed=9)
    c = draw_model_hamiltonian(20, 5, 4.0, seed=10)
    assert np.array_equal(a.h, b.h) and np.array_equal(a.L, b.L)
    assert not np.array_equal(a.L, c.L)


@pytest.fixture(scope="module")
def small():
    return make_system(CONFIGS["small"])


def test_rhf_output_is_canonical_with_aufbau(small):
    F, eps, no = small.fock, small.eps, small.spec.n_occ
    assert np.abs(F - np.diag(np.diag(F))).max() < 1e-8
    assert np.allclose(np.diag(F), eps, atol=1e-10)
    assert eps[:no].max() < eps[no:].min()
    assert small.rhf_gradient < 1e-8
    n = small.spec.n_mo
    g = np.einsum("Jpq,Jrs->pqrs", small.L, small.L).reshape(n * n, n * n)
    w = np.linalg.eigvalsh(0.5 * (g + g.T))
    assert w.min() > -1e-10 * w.max()


def test_levels_nested_and_placed():
    lev = level_map(8, 40, 6, 30, 3, 12)
    assert list(lev[:2]) == [0, 0] and list(lev[2:5]) == [1, 1, 1] and list(lev[5:8]) == [2, 2, 2]
    assert list(lev[8:20]) == [2] * 12 and list(lev[20:38]) == [1] * 18 and list(lev[38:]) == [0] * 10


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_workload_table(name):
    s = CONFIGS[name]
    assert isinstance(s, SystemSpec)
    assert s.tau == s.n_chol / 5.0 and s.scale == default_scale(s.tau) == 0.5 / math.sqrt(s.tau)
    assert 0 <= s.t_occ <= s.s_occ <= s.n_occ and 0 <= s.t_vir <= s.s_vir <= s.n_vir


def test_serving_mix_recipe():
    specs = [serving_request_spec(r) for r in range(256)]
    kinds = [k for _, k, _ in specs]
    for s, k, f in specs:
        assert 20 <= s.n_occ <= 80 and 150 <= s.n_vir <= 600
        assert s.n_chol == 5 * (s.n_occ + s.n_vir) and s.tau == s.n_chol / 5.0
        assert 0.1 <= f < 0.3 and s.n_roots == 4
        assert s.s_occ == max(1, round(f * s.n_occ)) and s.s_vir == max(1, round(f * s.n_vir))
        if k == "ccs_ccsd":
            assert (s.t_occ, s.t_vir) == (s.s_occ, s.s_vir)
        else:
            assert (s.t_occ, s.t_vir) == (0, 0)
    # both kinds about equally often (binomial(256, 1/2): sd 8)
    assert abs(kinds.count("mlcc2") - 128) < 40
    occ = np.array([s.n_occ for s, _, _ in specs])
    assert abs(occ.mean() - 50.0) < 4.0       # U{20..80}: mean 50, sd 17.6 / sqrt(256)
    # request r depends on its own seed only
    assert serving_request_spec(17)[0] == specs[17][0]
    assert serving_request_spec(0, seed_base=1)[0].n_occ == specs[1][0].n_occ


def test_serving_arrivals():
    t = serving_arrivals(4096, rate=20.0)
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 0.05) < 0.004    # mean 1 / rate, sd 0.05 / sqrt(4095)
    assert abs(np.median(gaps) - 0.05 * math.log(2)) < 0.004
    assert np.array_equal(serving_arrivals(10), serving_arrivals(10))
