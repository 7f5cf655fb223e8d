"""Pins of the left-eigenvector oracle (oracle/left.py), against the definition of the
Jacobian (the complex-step sigma) rather than the dense matrix they are built from:

  * the adjoint identity <rho(l), c> = <l, A c> for random admissible l and c, with A c
    from sigma directly;
  * the left problem has the right problem's eigenvalues (the Davidson roots of A);
  * left and right eigenvectors of different roots are orthogonal in the inner product, and
    each left vector solves rho(l) = omega l.
"""
import numpy as np
import pytest

from oracle import left as oleft
from oracle.davidson import excited_states
from oracle.mlcc import MLCCSystem, sigma, solve_ground_state
from test_oracle_pins import PARTITIONS
from tiny_systems import tiny


def _ip(a1, a2, b1, b2):
    return float(np.sum(a1 * b1) + np.sum(a2 * b2))


def _rand(sys, rng):
    c1 = rng.standard_normal((sys.nv, sys.no))
    c2 = rng.standard_normal(sys.doubles_shape())
    return c1, c2 + c2.transpose(2, 3, 0, 1)


@pytest.mark.parametrize("name", ["cc2", "mlcc2_ccs_outer", "three_level", "ccs_ccsd", "ccsd"])
def test_left_transformation_is_the_adjoint(name):
    t = tiny()
    lev = np.array(dict(PARTITIONS)[name], dtype=np.int8)
    o = MLCCSystem(t.L, t.F, t.k, lev)
    gs = solve_ground_state(o)
    parts = oleft.dense(o, gs)
    rng = np.random.default_rng(1)
    for _ in range(3):
        l1, l2 = _rand(o, rng)
        c1, c2 = _rand(o, rng)
        r1, r2 = oleft.left_transform(o, gs, l1, l2, parts)
        s1, s2 = sigma(o, gs.t1, gs.x2, c1, c2)
        lhs, rhs = _ip(r1, r2, c1, c2), _ip(l1, l2, s1, s2)
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))
        assert np.abs(r2 - r2.transpose(2, 3, 0, 1)).max() == 0.0


@pytest.mark.parametrize("name", ["cc2", "mlcc2_ccs_outer", "three_level"])
def test_left_eigenpairs(name):
    t = tiny()
    lev = np.array(dict(PARTITIONS)[name], dtype=np.int8)
    o = MLCCSystem(t.L, t.F, t.k, lev)
    gs = solve_ground_state(o)
    parts = oleft.dense(o, gs)
    w, lefts, rights = oleft.left_eigenpairs(o, gs, 3, parts)
    es = excited_states(o, gs, 3, res_tol=1e-10)
    assert np.abs(w - es.omega).max() < 1e-9
    for k in range(3):
        r1, r2 = oleft.left_transform(o, gs, *lefts[k], parts)
        assert np.abs(r1 - w[k] * lefts[k][0]).max() < 1e-9
        assert np.abs(r2 - w[k] * lefts[k][1]).max() < 1e-9
        for m in range(3):
            ov = _ip(*lefts[k], *rights[m])
            assert abs(ov - (1.0 if k == m else 0.0)) < 1e-9
