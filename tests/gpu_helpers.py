"""Index maps between the oracle's layout and libmlcc's level-ordered layout (test helper)."""
import numpy as np


class Layout:
    """Maps oracle arrays (caller orbital order) to the library's internal order."""

    def __init__(self, gsys, osys):
        no = gsys.no
        perm = gsys.perm
        self.po = perm[:no]                   # internal occ -> caller occ
        self.pv = perm[no:] - no              # internal vir -> caller vir
        pos_o = {int(u): k for k, u in enumerate(osys.os)}
        pos_v = {int(u): k for k, u in enumerate(osys.vs)}
        so, sv = gsys.dims.s_occ, gsys.dims.s_vir
        self.lo = np.array([pos_o[int(u)] for u in self.po[:so]], dtype=np.int64)
        self.lv = np.array([pos_v[int(u)] for u in self.pv[:sv]], dtype=np.int64)
        self.perm = perm
        self.n1 = gsys.nv * no
        self.dshape = (sv, so, sv, so)

    # oracle -> library
    def t1(self, t1):
        return np.ascontiguousarray(t1[np.ix_(self.pv, self.po)])

    def x2(self, x2):
        return np.ascontiguousarray(x2[np.ix_(self.lv, self.lo, self.lv, self.lo)])

    def vec(self, c1, c2):
        return np.concatenate([self.t1(c1).ravel(), self.x2(c2).ravel()])

    def mo(self, M):
        """[.., n, n] caller order -> internal order."""
        p = self.perm
        return M[..., p[:, None], p[None, :]]

    # library -> oracle
    def t1_back(self, g, shape):
        out = np.empty(shape)
        out[np.ix_(self.pv, self.po)] = np.asarray(g).reshape(len(self.pv), len(self.po))
        return out

    def x2_back(self, g, shape):
        out = np.zeros(shape)
        out[np.ix_(self.lv, self.lo, self.lv, self.lo)] = np.asarray(g).reshape(self.dshape)
        return out
