"""Oracle-side reference objects for the GPU parity tests (test infrastructure)."""

import functools

import numpy as np

import workload as W
from oracle import collocation as C, fd as F, geometry as Geo, gmres as G


class Ref:
    """Oracle view of one problem: spaces, map, collocation points, FD, and (for
    sizes where it is affordable) the assembled A_C."""

    def __init__(self, d, n_elem, p, geometry="annulus", r0=1.0, r1=2.0, assemble=True,
                 wind=None):
        self.d, self.n_elem, self.p = d, n_elem, p
        self.wind = None if wind is None else np.asarray(wind, dtype=np.float64)
        self.fmap = Geo.make_map(geometry, d, r0, r1)
        self.spaces = [C.Space1D(n_elem, p) for _ in range(d)]
        self.n = self.spaces[0].n
        self.N = self.n ** d
        self.points = C.physical_points(self.fmap, [s.tau for s in self.spaces])
        self.fd = F.FD(self.spaces, self.wind)
        self.A = (C.assemble_collocation(self.spaces, self.fmap, self.wind) if assemble
                  else None)
        self.r0, self.r1 = r0, r1

    def P_apply(self, s):
        """P s through the Kronecker form (eq. colloc2D / colloc3D)."""
        out = np.zeros(self.N)
        shape = tuple([self.n] * self.d)
        for l in range(self.d):
            w = 0.0 if self.wind is None else self.wind[l]
            mats = [C.wind_factor(self.spaces[j], w) if j == l else self.spaces[j].M
                    for j in range(self.d)]
            out += F.kron_apply(mats, s, shape)
        return out

    def rows(self, idx):
        return C.collocation_rows(self.spaces, self.fmap, idx, self.wind)

    def gmres(self, b, M="fd", tol=1e-8, max_iter=200, flexible=False):
        Mop = self.fd if M == "fd" else None
        return G.gmres(self.A, b, M=Mop, tol=tol, max_iter=max_iter, flexible=flexible)

    def manufactured_rhs(self, sigma=0.0, seed=0):
        return W.perturb(W.manufactured_f(self.points, self.r0, self.r1), sigma, seed)


@functools.lru_cache(maxsize=32)
def ref(d, n_elem, p, geometry="annulus", r0=1.0, r1=2.0, assemble=True, wind=None):
    """``wind``: None or a tuple of d floats (hashable, for the cache)."""
    return Ref(d, n_elem, p, geometry, r0, r1, assemble, wind)
