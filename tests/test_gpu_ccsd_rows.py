"""The CCSD rows of sigma (the tangent of the MLCCSD doubles residual, Appendix A Eq.
sigma_mlccsd) where its contractions are large enough to leave the small-GEMM path: a
CCSD block of 10 occupied / 60 virtual orbitals, so the ladder sum_cd g~_acbd c_cidj
(2 t_v^4 t_o^2 = 2.6e9 flop) and the other block contractions run on the tcgen05 tensor
cores in MLCC_FP64E and BF16X3 (everything at or above 2e8 flop). Every element of sigma,
in binary64, MLCC_FP64E and BF16X3, against the oracle's sigma (the complex-step derivative
of its residual), for an MLCCSD system (CC2 the rest) and a three-level one (CCS outer).
"""
import numpy as np
import pytest

from gpu_helpers import Layout
from oracle.mlcc import MLCCSystem, sigma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2006_05226_gb300 import mlcc
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = mlcc.Context(0)
    yield c
    c.close()


def _system(kind):
    from synth.generator import SystemSpec, default_scale, make_system
    if kind == "mlccsd":
        spec = SystemSpec("ccsd_rows", 12, 90, 300, 60.0, 12, 90, 10, 60, 3, 7, default_scale(60.0))
    else:
        spec = SystemSpec("ccsd_rows3", 13, 91, 300, 60.0, 11, 71, 10, 60, 3, 8, default_scale(60.0))
    return make_system(spec)


@pytest.mark.parametrize("kind", ["mlccsd", "three_level"])
def test_ccsd_rows_on_the_tensor_cores(ctx, kind):
    from paper_2006_05226_gb300 import mlcc
    s = _system(kind)
    no = s.spec.n_occ
    o = MLCCSystem(s.L, s.fock, no, s.level)
    g = mlcc.System(ctx, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"), no, s.level)
    assert g.dims.t_occ == 10 and g.dims.t_vir == 60
    lay = Layout(g, o)
    rng = np.random.default_rng(31)
    t1 = 0.02 * rng.standard_normal((o.nv, o.no))
    x2 = 0.02 * rng.standard_normal(o.doubles_shape())
    x2 = x2 + x2.transpose(2, 3, 0, 1)
    g.jacobian_prepare(torch.as_tensor(lay.t1(t1), device="cuda"), torch.as_tensor(lay.x2(x2).ravel(), device="cuda"))
    cs, refs = [], []
    for k in range(2):
        c1 = rng.standard_normal((o.nv, o.no))
        c2 = rng.standard_normal(o.doubles_shape())
        c2 = c2 + c2.transpose(2, 3, 0, 1)
        s1, s2 = sigma(o, t1, x2, c1, c2)
        cs.append(lay.vec(c1, c2))
        refs.append(lay.vec(s1, s2))
    c = torch.as_tensor(np.stack(cs), device="cuda")
    ref = np.stack(refs)
    n1 = o.nv * o.no
    so, sv = g.dims.s_occ, g.dims.s_vir
    box = np.zeros((sv, so, sv, so), bool)
    box[:60, :10, :60, :10] = True
    for prec, tol in ((mlcc.MLCC_FP64, 1e-10), (mlcc.MLCC_FP64E, 1e-10), (mlcc.MLCC_BF16X3, 2e-5)):
        out = g.sigma(c, precision=prec).cpu().numpy()
        for k in range(2):
            scale = float(np.abs(ref[k]).max())
            err = np.abs(out[k] - ref[k])
            # the CCSD rows on their own, and the whole vector
            rows = err[n1:].reshape(sv, so, sv, so)[box]
            assert rows.max() <= tol * scale, (prec, k, float(rows.max()), scale)
            assert err.max() <= tol * scale, (prec, k, float(err.max()), scale)
    g.close()
