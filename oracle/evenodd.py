"""Even-odd (Schur complement) preconditioned clover-Wilson operator (oracle).

Ordering the sites even-first, M = [[A_ee, -kappa D_eo], [-kappa D_oe, A_oo]],
where D_eo maps odd-site fields to even sites and D_oe the reverse.  Solving
M (x_e, x_o) = (b, 0) on the even sites reduces to

    Mhat x_e = b,   Mhat = A_ee - kappa^2 D_eo A_oo^-1 D_oe,
    x_o = kappa A_oo^-1 D_oe x_e,

the asymmetric Schur form (the paper, Sec. 1, names only the MILC clover
application; the form is a convention of this project).  Mhat^dag is written
from the adjoints of its factors: A_ee - kappa^2 D_oe^dag A_oo^-1 D_eo^dag.

Even/odd fields are arrays [V/2, 4, 3] (see ``lattice.split_eo``).
"""

import numpy as np

from . import dirac
from .lattice import split_eo, join_eo


class SchurOperator:
    """Mhat and Mhat^dag for fixed links U, kappa, c_sw and time boundary sign."""

    def __init__(self, U, kappa, csw, t_bc=-1.0):
        self.U = U
        self.kappa = kappa
        self.csw = csw
        self.t_bc = t_bc
        T, Z, Y, X = U.shape[:4]
        self.dims = (X, Y, Z, T)
        self.A = dirac.clover_term(U, kappa, csw)
        A_e, A_o = split_eo(self.A, self.dims)
        self.A_ee = A_e
        self.A_oo = A_o
        # site-by-site inverse of the 12 x 12 clover matrix (library primitive)
        self.A_oo_inv = np.linalg.inv(A_o)

    # hopping blocks --------------------------------------------------------
    def D_oe(self, x_e):
        return split_eo(dirac.hopping(self.U, join_eo(x_e, None, self.dims), self.t_bc), self.dims)[1]

    def D_eo(self, x_o):
        return split_eo(dirac.hopping(self.U, join_eo(None, x_o, self.dims), self.t_bc), self.dims)[0]

    def D_oe_dag(self, x_o):
        """(D_oe)^dag: odd -> even."""
        return split_eo(dirac.hopping_dagger(self.U, join_eo(None, x_o, self.dims), self.t_bc), self.dims)[0]

    def D_eo_dag(self, x_e):
        """(D_eo)^dag: even -> odd."""
        return split_eo(dirac.hopping_dagger(self.U, join_eo(x_e, None, self.dims), self.t_bc), self.dims)[1]

    # site matrices ---------------------------------------------------------
    @staticmethod
    def site(Am, v):
        return np.einsum('nij,nj->ni', Am, v.reshape(v.shape[0], 12)).reshape(v.shape)

    # operators -------------------------------------------------------------
    def Mhat(self, x_e):
        k2 = self.kappa ** 2
        t_o = self.site(self.A_oo_inv, self.D_oe(x_e))
        return self.site(self.A_ee, x_e) - k2 * self.D_eo(t_o)

    def Mhat_dag(self, x_e):
        k2 = self.kappa ** 2
        Ad_ee = dirac.dagger(self.A_ee)
        Ad_oo_inv = dirac.dagger(self.A_oo_inv)
        t_o = self.site(Ad_oo_inv, self.D_eo_dag(x_e))
        return self.site(Ad_ee, x_e) - k2 * self.D_oe_dag(t_o)

    def MdagM(self, x_e):
        return self.Mhat_dag(self.Mhat(x_e))

    def odd_solution(self, x_e):
        """x_o = kappa A_oo^-1 D_oe x_e (the odd half of the full solution for source (b, 0))."""
        return self.kappa * self.site(self.A_oo_inv, self.D_oe(x_e))
