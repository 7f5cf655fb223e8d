"""The serving loop through the C ABI (mlcc_server_create / mlcc_submit / mlcc_poll):
independent whole solves of different sizes and partitions, admitted into slots that run
concurrently on their own streams. Each request's result in the mix equals the same solve
run alone (mlcc_solve on one context), in binary64 and on the mixed path; the requests
overlapped; the footprint the server admits by bounds the device memory one solve takes;
over-budget requests are rejected and queued ones can be cancelled.
Collected after the other GPU tests, so that a failure here cannot hide their results.
"""
import threading

import numpy as np
import pytest

from tiny_systems import tiny

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# identical kernels and launch shapes alone and in the mix; the tolerance is the binary64
# parity bound of the energies
TOL = 1e-10


@pytest.fixture(scope="module")
def problems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from synth import CONFIGS, make_system
    from synth.generator import SystemSpec, default_scale
    small = make_system(CONFIGS["small"])
    ragged = make_system(SystemSpec("ragged", 6, 31, 29, 5.8, 5, 21, 2, 7, 3, 4, default_scale(5.8)))
    t = tiny()
    out = [(small.L, small.fock, small.spec.n_occ, small.level),
           (ragged.L, ragged.fock, ragged.spec.n_occ, ragged.level),
           (t.L, t.F, t.k, np.array([1, 2, 2, 2, 1, 1, 0], dtype=np.int8))]
    return [tuple(np.ascontiguousarray(a) for a in p[:2]) + (p[2], np.asarray(p[3], np.int8)) for p in out]


def _opts(mixed):
    from paper_2006_05226_gb300 import mlcc
    if mixed:
        return mlcc.default_options(n_roots=3, precision=mlcc.MLCC_BF16X3, gs_precision=mlcc.MLCC_BF16X3,
                                    refine_fp64=1000, refine_precision=mlcc.MLCC_FP64E, lowp_res_tol=1e-3)
    return mlcc.default_options(n_roots=3)


@pytest.mark.parametrize("mixed", [False, True])
def test_each_result_in_the_mix_equals_the_solve_alone(problems, mixed):
    from paper_2006_05226_gb300 import mlcc
    opts = _opts(mixed)
    ctx = mlcc.Context(0)
    alone = []
    for L, F, no, lev in problems:
        sol = mlcc.solve(ctx, L, F, no, lev, opts)
        alone.append((sol.gs.e_corr, sol.omega))
    ctx.close()
    srv = mlcc.Server(0, n_slots=3)
    order = [0, 1, 2, 0, 2, 1]                      # more requests than slots
    tickets = [srv.submit(*problems[k], opts=opts) for k in order]
    results = [srv.poll(t) for t in tickets]
    info = srv.stats()
    srv.close()
    for k, (res, w) in zip(order, results):
        assert res.status == 0, mlcc.STATUS.get(res.status)
        assert res.attempts == 1 and 0 <= res.slot < 3
        assert res.t_submit <= res.t_start <= res.t_finish
        assert abs(res.gs.e_corr - alone[k][0]) <= TOL
        assert np.abs(w - alone[k][1]).max() <= TOL
    assert info.finished == len(order) and info.running == 0 and info.waiting == 0
    assert info.peak_running >= 2                   # admitted requests ran together
    assert info.peak_bytes <= info.budget_bytes


def test_footprint_bounds_the_device_memory_of_a_solve(problems):
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = problems[0]
    for mixed in (False, True):
        opts = _opts(mixed)
        fp = mlcc.solve_footprint(F.shape[0], no, L.shape[0], lev, opts)
        ctx = mlcc.Context(0)
        mlcc.solve(ctx, L, F, no, lev, opts)        # kernels loaded before the measurement
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        low = [free0]
        stop = threading.Event()

        def sample():
            while not stop.is_set():
                low[0] = min(low[0], torch.cuda.mem_get_info()[0])

        th = threading.Thread(target=sample)
        th.start()
        try:
            mlcc.solve(ctx, L, F, no, lev, opts)
        finally:
            stop.set()
            th.join()
        ctx.close()
        used = free0 - low[0]
        assert used <= fp, (mixed, used, fp)


def test_rejection_and_cancellation(problems):
    from paper_2006_05226_gb300 import mlcc
    L, F, no, lev = problems[2]
    fp = mlcc.solve_footprint(F.shape[0], no, L.shape[0], lev)
    srv = mlcc.Server(0, n_slots=1, budget_bytes=fp - 1)
    with pytest.raises(mlcc.MLCCError) as e:
        srv.submit(L, F, no, lev)
    assert e.value.status == mlcc.MLCC_E_REJECTED
    srv.close()
    big = problems[0]
    fp_big = mlcc.solve_footprint(big[1].shape[0], big[2], big[0].shape[0], big[3])
    srv = mlcc.Server(0, n_slots=1, budget_bytes=4 * max(fp, fp_big))
    first = srv.submit(*big)                        # occupies the only slot for a while
    queued = [srv.submit(L, F, no, lev) for _ in range(3)]
    srv.cancel(queued[-1])
    results = [srv.poll(t) for t in [first] + queued]
    assert [r[0].status for r in results] == [0, 0, 0, mlcc.MLCC_E_CANCELLED]
    assert results[-1][0].slot == -1
    srv.close()


def test_problem_queries(problems):
    from paper_2006_05226_gb300 import mlcc
    for L, F, no, lev in problems:
        n, nj = F.shape[0], L.shape[0]
        so = int(np.sum(lev[:no] >= 1))
        sv = int(np.sum(lev[no:] >= 1))
        assert mlcc.vector_len(n, no, nj, lev) == (n - no) * no + (so * sv) ** 2
        ctx = mlcc.Context(0)
        h = mlcc.solve(ctx, L, F, no, lev, _opts(False))
        d = mlcc.solve_device(ctx, torch.as_tensor(L, device="cuda"), torch.as_tensor(F, device="cuda"),
                              no, lev, _opts(False))
        gs_h, w_h, gs_d, w_d = h.gs, h.omega, d.gs, d.omega
        ctx.close()
        assert gs_d.e_corr == gs_h.e_corr and np.array_equal(w_d, w_h)


@pytest.mark.parametrize("mixed", [False, True])
def test_sigma_graph_replay_equals_the_eager_solve(problems, mixed):
    """mlcc_options.sigma_graph: the Davidson's Jacobian transformations replayed from CUDA
    graphs give bitwise the eager solve's roots and vectors, with the same sigma count, and
    the graphs stand for fewer host launches per sigma (the library counts their kernels)."""
    from paper_2006_05226_gb300 import mlcc
    for L, F, no, lev in problems:
        ctx = mlcc.Context(0)
        res = []
        for graph in (0, 1):
            o = _opts(mixed)
            o.sigma_graph = graph
            res.append(mlcc.solve(ctx, L, F, no, lev, o, vectors=True))
        ctx.close()
        a, b = res
        assert np.array_equal(a.omega, b.omega) and np.array_equal(a.r, b.r)
        assert a.es.n_sigma == b.es.n_sigma and a.gs.e_corr == b.gs.e_corr
