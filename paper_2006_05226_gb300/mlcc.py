"""Thin Python binding of libmlcc (include/mlcc.h): argument marshalling only.

Every step of the method runs inside libmlcc.so; this module only moves pointers and
sizes across the C ABI. torch provides device memory and streams. The library works on
its own CUDA stream; calls order it after torch's current stream and order torch's
current stream after it, so tensors can be used on either side without races.
"""
import atexit
import ctypes
import os
import weakref
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int8, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlcc.so")

# enum values of include/mlcc.h (tests/test_library.py checks them against the header)
MLCC_FP64, MLCC_BF16, MLCC_BF16X3, MLCC_BF16X6, MLCC_FP64E = 0, 1, 2, 3, 4
MLCC_LEVEL_CCS, MLCC_LEVEL_CC2, MLCC_LEVEL_CCSD = 0, 1, 2
MLCC_OK = 0
MLCC_E_ARG = -1
MLCC_E_OOM = -2
MLCC_E_GS_NOCONV = -3
MLCC_E_ES_NOCONV = -4
MLCC_E_COMPLEX_ROOT = -5
MLCC_E_NAN = -6
MLCC_E_TIMEOUT = -7
MLCC_E_CUDA = -8
MLCC_E_STATE = -9
MLCC_E_REJECTED = -10
MLCC_E_CANCELLED = -11
MLCC_PENDING = 1
STATUS = {v: k for k, v in dict(globals()).items()
          if k.startswith("MLCC_") and (k.startswith("MLCC_E_") or k in ("MLCC_OK", "MLCC_PENDING"))}

# every symbol include/mlcc.h declares
EXPORTS = ["mlcc_default_options", "mlcc_sigma_left", "mlcc_excited_states_left", "mlcc_mo_screening", "mlcc_cholesky_decompose", "mlcc_cholesky_mo_vectors", "mlcc_sigma_partial", "mlcc_cnto", "mlcc_ctx_create", "mlcc_ctx_create_budget", "mlcc_orbitals", "mlcc_ctx_destroy", "mlcc_ctx_stream",
           "mlcc_last_error", "mlcc_kernel_timing", "mlcc_kernel_time", "mlcc_system_create",
           "mlcc_system_destroy", "mlcc_system_info", "mlcc_orbital_order", "mlcc_t1_transform",
           "mlcc_fock_t1", "mlcc_omega", "mlcc_ground_state", "mlcc_jacobian_prepare",
           "mlcc_sigma", "mlcc_excited_states", "mlcc_solve", "mlcc_launch_count",
           "mlcc_fock_t1_noalloc", "mlcc_gemm", "mlcc_solve_device", "mlcc_vector_len",
           "mlcc_solve_footprint", "mlcc_server_create", "mlcc_server_destroy", "mlcc_submit",
           "mlcc_poll", "mlcc_cancel", "mlcc_server_stats", "mlcc_sigma_eff", "mlcc_fold_window",
           "mlcc_excited_states_folded"]


class mlcc_problem(ctypes.Structure):
    _fields_ = [("n_mo", c_int32), ("n_occ", c_int32), ("n_chol", c_int32),
                ("level", POINTER(c_int8))]


class mlcc_dims(ctypes.Structure):
    _fields_ = [("n_occ", c_int32), ("n_vir", c_int32), ("s_occ", c_int32), ("s_vir", c_int32),
                ("t_occ", c_int32), ("t_vir", c_int32), ("n_singles", c_int64),
                ("n_doubles", c_int64), ("vector_len", c_int64), ("workspace_bytes", c_int64)]


class mlcc_options(ctypes.Structure):
    _fields_ = [("n_roots", c_int32), ("max_gs_iter", c_int32), ("max_es_iter", c_int32),
                ("diis_dim", c_int32), ("max_subspace", c_int32), ("precision", c_int32),
                ("refine_fp64", c_int32), ("gs_precision", c_int32), ("gs_tol", c_double),
                ("gs_energy_tol", c_double), ("es_res_tol", c_double),
                ("es_omega_tol", c_double), ("lowp_res_tol", c_double),
                ("refine_precision", c_int32), ("sigma_graph", c_int32)]


class mlcc_gs_info(ctypes.Structure):
    _fields_ = [("e_hf", c_double), ("e_corr", c_double), ("omega_norm", c_double),
                ("iterations", c_int32), ("converged", c_int32)]


class mlcc_es_info(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("n_sigma", c_int32), ("n_sigma_lowp", c_int32),
                ("converged", c_int32), ("complex_pair", c_int32), ("fp64_sweeps", c_int32),
                ("max_residual", c_double)]


class mlcc_request_result(ctypes.Structure):
    _fields_ = [("status", c_int32), ("slot", c_int32), ("attempts", c_int32), ("n_roots", c_int32),
                ("footprint_bytes", c_int64), ("t_submit", c_double), ("t_start", c_double),
                ("t_finish", c_double), ("gs", mlcc_gs_info), ("es", mlcc_es_info)]


class mlcc_server_info(ctypes.Structure):
    _fields_ = [("n_slots", c_int32), ("running", c_int32), ("waiting", c_int32),
                ("peak_running", c_int32), ("budget_bytes", c_int64), ("in_use_bytes", c_int64),
                ("peak_bytes", c_int64), ("submitted", c_int64), ("finished", c_int64),
                ("cancelled", c_int64), ("retried", c_int64)]


class mlcc_result(ctypes.Structure):
    _fields_ = [("gs", mlcc_gs_info), ("es", mlcc_es_info), ("omega", POINTER(c_double)),
                ("residual", POINTER(c_double)), ("t1", c_void_p), ("x2", c_void_p), ("r", c_void_p),
                ("perm", POINTER(c_int32)), ("orbitals", POINTER(c_double))]


class mlcc_cnto_result(ctypes.Structure):
    _fields_ = [("omega", POINTER(c_double)), ("m", POINTER(c_double)), ("n", POINTER(c_double)),
                ("occ_values", POINTER(c_double)), ("occ_vectors", POINTER(c_double)),
                ("vir_values", POINTER(c_double)), ("vir_vectors", POINTER(c_double)),
                ("n_occ_active", c_int32), ("n_vir_active", c_int32), ("block_rows", c_int32),
                ("reserved", c_int32)]


class MLCCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_live_contexts = weakref.WeakSet()


def load():
    """Loads libmlcc.so from the package directory; fails loudly if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    D = POINTER(c_double)
    sig = {
        "mlcc_default_options": (None, [POINTER(mlcc_options)]),
        "mlcc_ctx_create": (c_int, [c_int, POINTER(c_void_p)]),
        "mlcc_ctx_create_budget": (c_int, [c_int, c_int64, POINTER(c_void_p)]),
        "mlcc_orbitals": (c_int, [P, D]),
        "mlcc_mo_screening": (c_int, [P, c_int32, c_int32, P, P]),
        "mlcc_cholesky_decompose": (c_int, [P, c_int64, P, P, c_double, c_int32, POINTER(c_int32), P, P,
                                            POINTER(c_int32)]),
        "mlcc_cholesky_mo_vectors": (c_int, [P, c_int32, c_int32, P, POINTER(c_int32), c_int32, P, P]),
        "mlcc_cnto": (c_int, [P, c_int32, c_int32, c_int32, P, P, c_int32, c_int32, POINTER(mlcc_cnto_result)]),
        "mlcc_ctx_destroy": (None, [P]),
        "mlcc_ctx_stream": (c_void_p, [P]),
        "mlcc_last_error": (c_char_p, []),
        "mlcc_kernel_timing": (None, [P, c_int]),
        "mlcc_kernel_time": (c_int, [P, c_char_p, POINTER(c_int64), D, D]),
        "mlcc_launch_count": (c_int64, []),
        "mlcc_fock_t1_noalloc": (c_int, [c_int32, c_int32, c_int32, P, P, P, P, P, P]),
        "mlcc_gemm": (c_int, [P, c_int32, c_int32, c_int64, c_int64, c_int64, c_double, P, c_int64,
                              P, c_int64, c_double, P, c_int64, c_int32]),
        "mlcc_system_create": (c_int, [P, POINTER(mlcc_problem), P, P, POINTER(c_void_p)]),
        "mlcc_system_destroy": (None, [P]),
        "mlcc_system_info": (c_int, [P, POINTER(mlcc_dims)]),
        "mlcc_orbital_order": (c_int, [P, POINTER(c_int32)]),
        "mlcc_t1_transform": (c_int, [P, P, P]),
        "mlcc_fock_t1": (c_int, [P, P, P]),
        "mlcc_omega": (c_int, [P, P, P, P, P, P]),
        "mlcc_ground_state": (c_int, [P, POINTER(mlcc_options), P, P, POINTER(mlcc_gs_info)]),
        "mlcc_jacobian_prepare": (c_int, [P, P, P]),
        "mlcc_sigma": (c_int, [P, c_int32, P, P, c_int32]),
        "mlcc_sigma_partial": (c_int, [P, c_int32, c_int32, c_int32, c_int32, P, P, c_int32]),
        "mlcc_sigma_left": (c_int, [P, c_int32, P, P, c_int32]),
        "mlcc_excited_states_left": (c_int, [P, POINTER(mlcc_options), D, P, P, POINTER(mlcc_es_info)]),
        "mlcc_excited_states": (c_int, [P, POINTER(mlcc_options), D, P, POINTER(mlcc_es_info)]),
        "mlcc_solve": (c_int, [P, POINTER(mlcc_problem), P, P, POINTER(mlcc_options), POINTER(mlcc_result)]),
        "mlcc_solve_device": (c_int, [P, POINTER(mlcc_problem), P, P, POINTER(mlcc_options),
                                      POINTER(mlcc_result)]),
        "mlcc_vector_len": (c_int64, [POINTER(mlcc_problem)]),
        "mlcc_sigma_eff": (c_int, [P, c_int32, D, P, P, P, c_int32]),
        "mlcc_fold_window": (c_int, [P, D]),
        "mlcc_excited_states_folded": (c_int, [P, POINTER(mlcc_options), D, P, POINTER(mlcc_es_info)]),
        "mlcc_solve_footprint": (c_int, [POINTER(mlcc_problem), POINTER(mlcc_options), POINTER(c_int64)]),
        "mlcc_server_create": (c_int, [c_int, c_int32, c_int64, POINTER(c_void_p)]),
        "mlcc_server_destroy": (None, [P]),
        "mlcc_submit": (c_int, [P, POINTER(mlcc_problem), P, P, POINTER(mlcc_options), POINTER(ctypes.c_uint64)]),
        "mlcc_poll": (c_int, [P, ctypes.c_uint64, c_int64, POINTER(mlcc_request_result), D]),
        "mlcc_cancel": (c_int, [P, ctypes.c_uint64]),
        "mlcc_server_stats": (c_int, [P, POINTER(mlcc_server_info)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise MLCCError(status, load().mlcc_last_error().decode())


def launch_count():
    """Kernels libmlcc has launched in this process."""
    return int(load().mlcc_launch_count())


def fock_t1_noalloc(chol, fock, n_occ, t1, lt_out, ft_out, stream=None):
    """mlcc_fock_t1_noalloc on caller-owned device tensors (caller orbital order); the
    library allocates nothing. stream: a torch CUDA stream (default: the current one)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(load().mlcc_fock_t1_noalloc(fock.shape[0], n_occ, chol.shape[0], _ptr(chol), _ptr(fock),
                                       _ptr(t1), _ptr(lt_out), _ptr(ft_out), c_void_p(st.cuda_stream)))


def default_options(**kw):
    o = mlcc_options()
    load().mlcc_default_options(byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    return c_void_p(t.data_ptr()) if t is not None else None


class Context:
    """mlcc_ctx: one device, one stream; budget_bytes > 0 caps the device memory its systems
    and whole solves may hold (mlcc_ctx_create_budget)."""

    def __init__(self, device=0, budget_bytes=0):
        import torch
        self._torch = torch
        h = c_void_p()
        _check(load().mlcc_ctx_create_budget(device, int(budget_bytes), byref(h)))
        self.handle = h
        self.device = device
        self.stream = torch.cuda.ExternalStream(load().mlcc_ctx_stream(h), device=f"cuda:{device}")
        self.systems = weakref.WeakSet()
        _live_contexts.add(self)

    def before(self, *tensors):
        # the library stream waits for torch's stream; after() makes torch's stream wait
        # for the library, so tensors freed afterwards on torch's stream are safe to reuse
        self.stream.wait_stream(self._torch.cuda.current_stream(self.device))

    def after(self):
        self._torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def kernel_timing(self, enable):
        load().mlcc_kernel_timing(self.handle, 1 if enable else 0)

    def kernel_time(self, family="rank_gemm_tc"):
        n, ms, fl = c_int64(), c_double(), c_double()
        _check(load().mlcc_kernel_time(self.handle, family.encode(), byref(n), byref(ms), byref(fl)))
        return n.value, ms.value, fl.value

    def gemm(self, a, b, c, alpha=1.0, beta=0.0, trans_a=False, trans_b=False,
             precision=MLCC_FP64):
        """mlcc_gemm on contiguous row-major float64 device tensors:
        c = alpha op(a) op(b) + beta c."""
        M, N = c.shape
        K = a.shape[0] if trans_a else a.shape[1]
        self.before()
        _check(load().mlcc_gemm(self.handle, int(trans_a), int(trans_b), M, N, K, alpha, _ptr(a),
                                a.shape[1], _ptr(b), b.shape[1], beta, _ptr(c), c.shape[1],
                                precision))
        self.after()
        return c

    def close(self):
        if self.handle:
            for sysobj in list(self.systems):
                sysobj.close()
            self._torch.cuda.synchronize(self.device)
            load().mlcc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@atexit.register
def _close_all():
    for c in list(_live_contexts):
        try:
            c.close()
        except Exception:
            pass


class System:
    """mlcc_system: device copy of one problem (chol [n_chol, n, n], fock [n, n])."""

    def __init__(self, ctx, chol, fock, n_occ, level):
        torch = ctx._torch
        assert chol.dtype == torch.float64 and fock.dtype == torch.float64
        assert chol.is_cuda and fock.is_cuda and chol.is_contiguous() and fock.is_contiguous()
        self.ctx = ctx
        self.level = np.ascontiguousarray(np.asarray(level, dtype=np.int8))
        prob = mlcc_problem(fock.shape[0], n_occ, chol.shape[0],
                            self.level.ctypes.data_as(POINTER(c_int8)))
        h = c_void_p()
        ctx.before(chol, fock)
        _check(load().mlcc_system_create(ctx.handle, byref(prob), _ptr(chol), _ptr(fock), byref(h)))
        self.handle = h
        ctx.systems.add(self)
        d = mlcc_dims()
        _check(load().mlcc_system_info(h, byref(d)))
        self.dims = d
        perm = (c_int32 * fock.shape[0])()
        _check(load().mlcc_orbital_order(h, perm))
        self.perm = np.array(perm[:], dtype=np.int64)
        self.n, self.no = fock.shape[0], n_occ
        self.nv = self.n - n_occ
        self.n_chol = chol.shape[0]

    def orbitals(self):
        """mlcc_orbitals: [n, n] with column k the system's orbital k in the caller's orbitals."""
        c = np.zeros((self.n, self.n))
        _check(load().mlcc_orbitals(self.handle, c.ctypes.data_as(POINTER(c_double))))
        return c

    def _new(self, *shape):
        return self.ctx._torch.empty(*shape, dtype=self.ctx._torch.float64,
                                     device=f"cuda:{self.ctx.device}")

    def t1_transform(self, t1):
        out = self._new(self.n_chol, self.n, self.n)
        self.ctx.before(t1, out)
        _check(load().mlcc_t1_transform(self.handle, _ptr(t1), _ptr(out)))
        self.ctx.after()
        return out

    def fock_t1(self, t1):
        out = self._new(self.n, self.n)
        self.ctx.before(t1, out)
        _check(load().mlcc_fock_t1(self.handle, _ptr(t1), _ptr(out)))
        self.ctx.after()
        return out

    def omega(self, t1, x2):
        om1 = self._new(self.dims.n_singles)
        om2 = self._new(max(self.dims.n_doubles, 1))
        e = self._new(1)
        self.ctx.before(t1, x2, om1, om2, e)
        _check(load().mlcc_omega(self.handle, _ptr(t1), _ptr(x2), _ptr(om1), _ptr(om2), _ptr(e)))
        self.ctx.after()
        return om1, om2[: self.dims.n_doubles], e

    def ground_state(self, opts=None):
        opts = opts or default_options()
        t1 = self._new(self.dims.n_singles)
        x2 = self._new(max(self.dims.n_doubles, 1))
        info = mlcc_gs_info()
        self.ctx.before(t1, x2)
        st = load().mlcc_ground_state(self.handle, byref(opts), _ptr(t1), _ptr(x2), byref(info))
        self.ctx.after()
        _check(st)
        return t1, x2[: self.dims.n_doubles], info

    def sigma_eff(self, c, omega, precision=MLCC_FP64, derivative=False):
        """mlcc_sigma_eff: A_eff(omega_k) c_k (singles and P_T rows) and, if derivative,
        the singles of dA_eff/domega c_k. c: [n_vec, vector_len]; omega: n_vec floats."""
        c = c.reshape(-1, self.dims.vector_len)
        n_vec = c.shape[0]
        w = (c_double * max(1, n_vec))(*[float(x) for x in np.atleast_1d(omega)])
        out = self._new(n_vec, self.dims.vector_len)
        dout = self._new(n_vec, self.dims.n_singles) if derivative else None
        self.ctx.before(c, out)
        _check(load().mlcc_sigma_eff(self.handle, n_vec, w, _ptr(c), _ptr(out), _ptr(dout), precision))
        self.ctx.after()
        return (out, dout) if derivative else out

    def excited_states_folded(self, opts=None, want_vectors=True):
        """mlcc_excited_states_folded: (omega array, unfolded vectors or None, mlcc_es_info)."""
        opts = opts or default_options()
        w = (c_double * opts.n_roots)()
        R = self._new(opts.n_roots, self.dims.vector_len) if want_vectors else None
        info = mlcc_es_info()
        self.ctx.before()
        st = load().mlcc_excited_states_folded(self.handle, byref(opts), w, _ptr(R), byref(info))
        self.ctx.after()
        _check(st)
        return np.array(w[:]), R, info

    def fold_window(self):
        w = c_double(0.0)
        _check(load().mlcc_fold_window(self.handle, byref(w)))
        return w.value

    def jacobian_prepare(self, t1, x2):
        self.ctx.before(t1, x2)
        _check(load().mlcc_jacobian_prepare(self.handle, _ptr(t1), _ptr(x2)))
        self.ctx.after()

    def sigma(self, c, precision=MLCC_FP64):
        c = c.reshape(-1, self.dims.vector_len)
        out = self._new(c.shape[0], self.dims.vector_len)
        self.ctx.before(c, out)
        _check(load().mlcc_sigma(self.handle, c.shape[0], _ptr(c), _ptr(out), precision))
        self.ctx.after()
        return out

    def sigma_partial(self, c, j_begin, j_end, with_rest, precision=MLCC_FP64):
        """mlcc_sigma_partial: the part of sigma over the Cholesky vectors [j_begin, j_end),
        plus the terms that do not sum over them when with_rest."""
        c = c.reshape(-1, self.dims.vector_len)
        out = self._new(c.shape[0], self.dims.vector_len)
        self.ctx.before(c, out)
        _check(load().mlcc_sigma_partial(self.handle, int(j_begin), int(j_end), int(bool(with_rest)), c.shape[0],
                                         _ptr(c), _ptr(out), precision))
        self.ctx.after()
        return out

    def sigma_sharded(self, c, rank, world, precision=MLCC_FP64, group=None):
        """sigma split over `world` ranks by Cholesky index (shard_range), summed with one
        torch.distributed all-reduce: on the device under NCCL, through host memory under
        gloo. Rank 0 adds the terms that do not sum over J."""
        return sharded_sum(lambda j0, j1, rest: self.sigma_partial(c, j0, j1, rest, precision),
                           self.n_chol, rank, world, group)

    def sigma_left(self, l, precision=MLCC_FP64):
        """mlcc_sigma_left: rho = A^T l for [n_vec, vector_len] symmetric-doubles vectors."""
        l = l.reshape(-1, self.dims.vector_len)
        out = self._new(l.shape[0], self.dims.vector_len)
        self.ctx.before(l, out)
        _check(load().mlcc_sigma_left(self.handle, l.shape[0], _ptr(l), _ptr(out), precision))
        self.ctx.after()
        return out

    def excited_states_left(self, opts=None, right=None):
        """mlcc_excited_states_left: (omega, left vectors [n_roots, vector_len], info); with
        `right` ([n_roots, vector_len] device tensor) the pairs are made biorthonormal."""
        opts = opts or default_options()
        w = (c_double * opts.n_roots)()
        Lv = self._new(opts.n_roots, self.dims.vector_len)
        info = mlcc_es_info()
        self.ctx.before()
        st = load().mlcc_excited_states_left(self.handle, byref(opts), w, _ptr(Lv), _ptr(right), byref(info))
        self.ctx.after()
        _check(st)
        return np.array(w[:]), Lv, info

    def excited_states(self, opts=None, want_vectors=True):
        opts = opts or default_options()
        w = (c_double * opts.n_roots)()
        R = self._new(opts.n_roots, self.dims.vector_len) if want_vectors else None
        info = mlcc_es_info()
        self.ctx.before(R)
        st = load().mlcc_excited_states(self.handle, byref(opts), w, _ptr(R), byref(info))
        self.ctx.after()
        _check(st)
        return np.array(w[:]), R, info

    def close(self):
        if self.handle and self.ctx.handle:
            load().mlcc_system_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solution:
    """What a whole solve returned: gs (mlcc_gs_info), es (mlcc_es_info), omega and residual
    (numpy, per root), and t1, x2, r, perm, orbitals where asked for (else None): numpy
    arrays from solve(), torch device tensors (t1, x2, r) from solve_device()."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _dims_of(n_mo, n_occ, level):
    lev = np.asarray(level)
    so = int(np.sum(lev[:n_occ] >= MLCC_LEVEL_CC2))
    sv = int(np.sum(lev[n_occ:] >= MLCC_LEVEL_CC2))
    n1 = (n_mo - n_occ) * n_occ
    return n1, (so * sv) ** 2


def _solve(entry, ctx, chol, fock, n_occ, level, opts, t1, x2, vectors, orbitals, alloc):
    opts = opts or default_options()
    n_mo = fock.shape[0]
    prob, lev = _problem(n_mo, n_occ, chol.shape[0], level)
    n1, nd = _dims_of(n_mo, n_occ, lev)
    w = np.zeros(opts.n_roots)
    rs = np.zeros(opts.n_roots)
    out = {"t1": alloc(n1) if t1 else None, "x2": alloc(max(nd, 1)) if x2 else None,
           "r": alloc(opts.n_roots * (n1 + nd)) if vectors else None}
    perm = np.zeros(n_mo, dtype=np.int32)
    orb = np.zeros((n_mo, n_mo)) if orbitals else None
    res = mlcc_result()
    res.omega = w.ctypes.data_as(POINTER(c_double))
    res.residual = rs.ctypes.data_as(POINTER(c_double))
    addr = (lambda a: None if a is None else (a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()))
    res.t1, res.x2, res.r = addr(out["t1"]), addr(out["x2"]), addr(out["r"])
    res.perm = perm.ctypes.data_as(POINTER(c_int32))
    res.orbitals = orb.ctypes.data_as(POINTER(c_double)) if orb is not None else None
    st = entry(res, prob)
    _check(st)
    if out["x2"] is not None:
        out["x2"] = out["x2"][:nd]
    if out["r"] is not None:
        out["r"] = out["r"].reshape(opts.n_roots, n1 + nd)
    return Solution(gs=res.gs, es=res.es, omega=w, residual=rs, perm=perm.astype(np.int64),
                    orbitals=orb, **out)


def solve(ctx, chol_host, fock_host, n_occ, level, opts=None, t1=False, x2=False, vectors=False,
          orbitals=False):
    """mlcc_solve from host arrays (copies them to the device inside the call). t1, x2,
    vectors, orbitals: also return those (host numpy arrays)."""
    chol_host = np.ascontiguousarray(chol_host, dtype=np.float64)
    fock_host = np.ascontiguousarray(fock_host, dtype=np.float64)
    o = opts or default_options()
    return _solve(lambda res, prob: load().mlcc_solve(ctx.handle, byref(prob), c_void_p(chol_host.ctypes.data),
                                                      c_void_p(fock_host.ctypes.data), byref(o), byref(res)),
                  ctx, chol_host, fock_host, n_occ, level, o, t1, x2, vectors, orbitals,
                  lambda n: np.zeros(n))


def _problem(n_mo, n_occ, n_chol, level):
    """(mlcc_problem, the int8 level array it points into: keep both alive together)."""
    level = np.ascontiguousarray(np.asarray(level, dtype=np.int8))
    return mlcc_problem(n_mo, n_occ, n_chol, level.ctypes.data_as(POINTER(c_int8))), level


def solve_device(ctx, chol, fock, n_occ, level, opts=None, t1=False, x2=False, vectors=False,
                 orbitals=False):
    """mlcc_solve_device on float64 CUDA tensors (borrowed for the call); t1, x2 and the
    vectors come back as device tensors."""
    o = opts or default_options()
    torch = ctx._torch

    def entry(res, prob):
        ctx.before()
        st = load().mlcc_solve_device(ctx.handle, byref(prob), _ptr(chol), _ptr(fock), byref(o), byref(res))
        ctx.after()
        return st

    return _solve(entry, ctx, chol, fock, n_occ, level, o, t1, x2, vectors, orbitals,
                  lambda n: torch.zeros(n, dtype=torch.float64, device=f"cuda:{ctx.device}"))


def cnto(ctx, chol, fock, n_occ, n_states, n_occ_active, n_vir_active=0, precision=MLCC_FP64, block_rows=0):
    """mlcc_cnto on float64 CUDA tensors (canonical orbitals): a Solution with omega, m, n,
    occ_values, occ_vectors, vir_values, vir_vectors (numpy) and the active counts."""
    n_mo = fock.shape[0]
    nv = n_mo - n_occ
    out = {"omega": np.zeros(n_states), "m": np.zeros((n_occ, n_occ)), "n": np.zeros((nv, nv)),
           "occ_values": np.zeros(n_occ), "occ_vectors": np.zeros((n_occ, n_occ)),
           "vir_values": np.zeros(nv), "vir_vectors": np.zeros((nv, nv))}
    res = mlcc_cnto_result()
    for k, a in out.items():
        setattr(res, k, a.ctypes.data_as(POINTER(c_double)))
    res.n_occ_active, res.n_vir_active, res.block_rows = n_occ_active, n_vir_active, block_rows
    ctx.before()
    st = load().mlcc_cnto(ctx.handle, n_mo, n_occ, chol.shape[0], _ptr(chol), _ptr(fock), n_states, precision,
                          byref(res))
    ctx.after()
    _check(st)
    return Solution(n_occ_active=res.n_occ_active, n_vir_active=res.n_vir_active, **out)


def mo_screening(ctx, c_active):
    """mlcc_mo_screening: the weights nu_a nu_b [n_ao * n_ao] of the screened diagonal."""
    n_ao, n_act = c_active.shape
    w = ctx._torch.empty(n_ao * n_ao, dtype=ctx._torch.float64, device=f"cuda:{ctx.device}")
    ctx.before()
    _check(load().mlcc_mo_screening(ctx.handle, n_ao, n_act, _ptr(c_active), _ptr(w)))
    ctx.after()
    return w


def cholesky_decompose(ctx, g, tau, max_vectors=None, w=None):
    """mlcc_cholesky_decompose of the [n_pairs, n_pairs] device matrix g: (pivots list,
    L [n_pairs, n_vectors] device tensor, final diagonal [n_pairs] device tensor)."""
    torch = ctx._torch
    m = g.shape[0]
    mv = m if max_vectors is None else int(max_vectors)
    L = torch.zeros(m, mv, dtype=torch.float64, device=f"cuda:{ctx.device}")
    D = torch.empty(m, dtype=torch.float64, device=f"cuda:{ctx.device}")
    piv = (c_int32 * mv)()
    nvec = c_int32(0)
    ctx.before()
    _check(load().mlcc_cholesky_decompose(ctx.handle, m, _ptr(g), _ptr(w), float(tau), mv, piv, _ptr(L), _ptr(D),
                                          byref(nvec)))
    ctx.after()
    return list(piv[:nvec.value]), L[:, :nvec.value], D


def cholesky_mo_vectors(ctx, g, pivots, C):
    """mlcc_cholesky_mo_vectors (Algorithm 1): [n_vectors, n_mo, n_mo] device tensor."""
    torch = ctx._torch
    n_ao, n_mo = C.shape
    piv = (c_int32 * len(pivots))(*pivots)
    out = torch.empty(len(pivots), n_mo, n_mo, dtype=torch.float64, device=f"cuda:{ctx.device}")
    ctx.before()
    _check(load().mlcc_cholesky_mo_vectors(ctx.handle, n_ao, n_mo, _ptr(g), piv, len(pivots), _ptr(C), _ptr(out)))
    ctx.after()
    return out


def shard_range(n_chol, rank, world):
    """[j_begin, j_end) of Cholesky vectors for one of `world` ranks: contiguous, in rank
    order, sizes differing by at most one (the first n_chol % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world or world > n_chol:
        raise ValueError("need 0 <= rank < world <= n_chol")
    q, r = divmod(int(n_chol), int(world))
    j0 = rank * q + min(rank, r)
    return j0, j0 + q + (1 if rank < r else 0)


def sharded_sum(partial, n_chol, rank, world, group=None):
    """The sum over ranks of partial(j_begin, j_end, with_rest) (a torch tensor) for this
    rank's shard_range, with_rest on rank 0 only: one torch.distributed all-reduce, on the
    device under NCCL and through host memory under gloo."""
    j0, j1 = shard_range(n_chol, rank, world)
    part = partial(j0, j1, rank == 0)
    if world == 1:
        return part
    import torch.distributed as dist
    if dist.get_backend(group) == "nccl" or part.device.type == "cpu":
        dist.all_reduce(part, group=group)
        return part
    host = part.cpu()
    dist.all_reduce(host, group=group)
    return host.to(part.device)


def vector_len(n_mo, n_occ, n_chol, level):
    """mlcc_vector_len: Davidson vector length of a problem (-1 if invalid)."""
    prob, lev = _problem(n_mo, n_occ, n_chol, level)
    return int(load().mlcc_vector_len(byref(prob)))


def solve_footprint(n_mo, n_occ, n_chol, level, opts=None):
    """mlcc_solve_footprint: device bytes mlcc_solve of the problem holds at its peak."""
    opts = opts or default_options()
    prob, lev = _problem(n_mo, n_occ, n_chol, level)
    b = c_int64(0)
    _check(load().mlcc_solve_footprint(byref(prob), byref(opts), byref(b)))
    return int(b.value)


class Server:
    """mlcc_server: whole solves submitted as requests, admitted by footprint into slots.

    submit() keeps the host arrays of each request alive until its result is polled."""

    def __init__(self, device=0, n_slots=4, budget_bytes=0):
        h = c_void_p()
        _check(load().mlcc_server_create(device, n_slots, budget_bytes, byref(h)))
        self.handle = h
        self._held = {}

    def submit(self, chol_host, fock_host, n_occ, level, opts=None):
        chol_host = np.ascontiguousarray(chol_host, dtype=np.float64)
        fock_host = np.ascontiguousarray(fock_host, dtype=np.float64)
        opts = opts or default_options()
        prob, lev = _problem(fock_host.shape[0], n_occ, chol_host.shape[0], level)
        t = ctypes.c_uint64(0)
        _check(load().mlcc_submit(self.handle, byref(prob), c_void_p(chol_host.ctypes.data),
                                  c_void_p(fock_host.ctypes.data), byref(opts), byref(t)))
        self._held[t.value] = (chol_host, fock_host, opts.n_roots)
        return t.value

    def poll(self, ticket, wait_ms=-1):
        """(mlcc_request_result, omega array) once finished, None while pending."""
        n_roots = self._held[ticket][2] if ticket in self._held else 1
        res = mlcc_request_result()
        w = (c_double * max(1, n_roots))()
        st = load().mlcc_poll(self.handle, ticket, wait_ms, byref(res), w)
        if st == MLCC_PENDING:
            return None
        _check(st)
        self._held.pop(ticket, None)
        return res, np.array(w[:res.n_roots])

    def cancel(self, ticket):
        _check(load().mlcc_cancel(self.handle, ticket))

    def stats(self):
        info = mlcc_server_info()
        _check(load().mlcc_server_stats(self.handle, byref(info)))
        return info

    def close(self):
        if self.handle:
            load().mlcc_server_destroy(self.handle)
        self.handle = None
        self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
