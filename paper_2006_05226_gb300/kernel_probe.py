"""Runs the Jacobian transformation of one synthetic system for kernel profiling.

A system with the Cholesky-rank GEMM shapes of the benchmark workload scaled down so
that the device holds a few GB: builds the system, prepares the Jacobian at seeded small
amplitudes (no ground-state solve), and evaluates sigma-vectors in the chosen precision
inside a cudaProfilerStart/Stop range (profile with --profile-from-start off).

  python -m paper_2006_05226_gb300.kernel_probe [--occ 40] [--vir 150] [--chol 1500]
         [--precision 2] [--nsigma 1]
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--occ", type=int, default=40)
    ap.add_argument("--vir", type=int, default=150)
    ap.add_argument("--chol", type=int, default=1500)
    ap.add_argument("--ccsd-occ", type=int, default=10)
    ap.add_argument("--ccsd-vir", type=int, default=60)
    ap.add_argument("--precision", type=int, default=2)
    ap.add_argument("--nsigma", type=int, default=1)
    a = ap.parse_args()
    import numpy as np
    import torch
    from paper_2006_05226_gb300 import mlcc
    from synth.generator import SystemSpec, default_scale, make_system
    tau = a.chol / 5.0
    spec = SystemSpec("probe", a.occ, a.vir, a.chol, tau, a.occ, a.vir, a.ccsd_occ, a.ccsd_vir,
                      4, 0, default_scale(tau))
    s = make_system(spec, rhf_tol=1e-8)
    ctx = mlcc.Context(0)
    g = mlcc.System(ctx, torch.as_tensor(s.L, device="cuda"), torch.as_tensor(s.fock, device="cuda"),
                    a.occ, s.level)
    d = g.dims
    rng = np.random.default_rng(0)
    t1 = torch.as_tensor(0.01 * rng.standard_normal(d.n_singles), device="cuda")
    m = d.s_vir * d.s_occ
    x2 = 0.01 * rng.standard_normal((m, m))
    x2 = torch.as_tensor((x2 + x2.T).ravel(), device="cuda")
    g.jacobian_prepare(t1, x2)
    c = rng.standard_normal(d.vector_len)
    c2 = c[d.n_singles:].reshape(m, m)
    c[d.n_singles:] = (c2 + c2.T).ravel()
    c = torch.as_tensor(c, device="cuda").reshape(1, -1)
    g.sigma(c, precision=a.precision)      # warm: operand caches, kernel attributes
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    for _ in range(a.nsigma):
        g.sigma(c, precision=a.precision)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    g.close()
    ctx.close()
    print(f"kernel_probe ok: vector_len {d.vector_len}, precision {a.precision}, {a.nsigma} sigma")


if __name__ == "__main__":
    main()
