"""The ground-state ladder from undressed integrals (Sec. 2.1 T1 dressing; Appendix A ladder).

The T1 dressing (1 - t1) L (1 + t1) changes only the virtual rows of the virtual-virtual
block, L~_ac = L_ac - sum_K t_aK L_Kc (K over every occupied orbital). Expanding
g~_acbd = sum_J L~_ac L~_bd in the ladder term gives

  sum_cd g~_acbd t_cidj = sum_cd g_acbd t_cidj - sum_K t_aK U_Kbij - sum_L t_bL U_Laji
                          + sum_KL t_aK t_bL W_KLij,
  U_Kbij = sum_cd g_Kcbd t_cidj,   W_KLij = sum_cd g_KcLd t_cidj,

which the library evaluates as one GEMM against the stacked undressed rows
[(ab) | (Kb) | (KL)] x (cd) and three small contractions. Checked here on the host
against the oracle's direct form: the dressed integrals from oracle.mlcc.t1_transform
and the ladder contracted from them. The layout follows the library's (row blocks of
the stacked operand, [(cd)][(ij)] doubles), so that an index or sign slip in that
layout fails the test.
"""
import numpy as np
import pytest

from oracle.mlcc import MLCCSystem, t1_transform
from tests.tiny_systems import tiny


def _ladder_direct(L_t, v, t):
    L_ac = L_t[:, v][:, :, v]
    g = np.einsum("Kac,Kbd->acbd", L_ac, L_ac)
    return np.einsum("acbd,cidj->aibj", g, t)


def _ladder_undressed(L, no, v, t1v, t):
    """The library's evaluation order, written out with numpy."""
    tv, to = t.shape[0], t.shape[1]
    L_ac = L[:, v][:, :, v]
    L_Kc = L[:, :no][:, :, v]
    A1 = np.einsum("Jac,Jbd->abcd", L_ac, L_ac).reshape(tv * tv, tv * tv)
    A2 = np.einsum("JKc,Jbd->Kbcd", L_Kc, L_ac).reshape(no * tv, tv * tv)
    A3 = np.einsum("JKc,JLd->KLcd", L_Kc, L_Kc).reshape(no * no, tv * tv)
    A = np.vstack([A1, A2, A3])
    tcd = np.einsum("cidj->cdij", t).reshape(tv * tv, to * to)
    W = A @ tcd
    om = np.einsum("abij->aibj", W[:tv * tv].reshape(tv, tv, to, to))
    Y = (t1v @ W[tv * tv:tv * tv + no * tv].reshape(no, tv * to * to)).reshape(tv, tv, to, to)
    om = om - np.einsum("abij->aibj", Y) - np.einsum("baji->aibj", Y)
    Z = (t1v @ W[tv * tv + no * tv:].reshape(no, no * to * to)).reshape(tv, no, to * to)
    Q = np.stack([t1v @ Z[a] for a in range(tv)]).reshape(tv, tv, to, to)
    return om + np.einsum("abij->aibj", Q)


LEVELS = {
    # 7 orbitals, 2 occupied: 2 = CCSD-active, 1 = CC2-active, 0 = CCS
    "ccsd": [2] * 7,
    "three_level": [2, 1, 2, 2, 1, 1, 0],
    "ccs_ccsd": [2, 0, 2, 2, 0, 0, 0],
}


@pytest.mark.parametrize("name", sorted(LEVELS))
def test_undressed_ladder_equals_the_dressed_one(name):
    s = tiny()
    sys = MLCCSystem(s.L, s.F, s.k, np.array(LEVELS[name]))
    o, v = sys.tbox()
    if len(o) == 0 or len(v) == 0:
        pytest.skip("no CCSD level")
    rng = np.random.default_rng(7)
    t1 = 0.1 * rng.standard_normal((sys.nv, sys.no))
    tv, to = len(v), len(o)
    t = 0.1 * rng.standard_normal((tv, to, tv, to))
    t = t + t.transpose(2, 3, 0, 1)          # pair symmetry of the doubles
    L_t = t1_transform(sys.L, t1, sys.no)
    ref = _ladder_direct(L_t, v, t)
    got = _ladder_undressed(sys.L, sys.no, v, t1[np.asarray(v) - sys.no], t)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # without the t1 terms the expansion is not the dressed ladder (the test can fail)
    bare = _ladder_undressed(sys.L, sys.no, v, 0.0 * t1[np.asarray(v) - sys.no], t)
    assert np.max(np.abs(bare - ref)) > 1e-6
