"""Forward scattering solve (Sec. 2.1, Eq. 3-5): measured-data synthesis.

Solves (I - G_D diag(chi)) E_tot = E_inc per incidence, then J = chi E_tot and
E_sca = G_S J.  Dense LU for M <= dense_max, else BiCGSTAB/GMRES (SciPy, library
primitives) with the FFT-applied G_D, relative tolerance 1e-10.

Pinned by: the Mie series (tests/test_oracle_physics.py), reciprocity, and the
dense-vs-iterative agreement on small grids.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg as sla
from scipy.sparse import linalg as spla

from .green import Operators


def forward_solve(ops: Operators, chi: np.ndarray, dense_max: int = 1024, tol: float = 1e-10):
    """Return (J, E_tot, E_sca): [ni][ny][nx], [ni][ny][nx], [ni][nr] complex128."""
    p = ops.p
    m = p.m
    c = chi.reshape(-1).astype(np.complex128)
    Einc = ops.Einc.reshape(p.ni, m)
    if m <= dense_max:
        G = ops.GD if ops.GD is not None else Operators(p, dense_gd=True).GD
        A = np.eye(m, dtype=np.complex128) - G * c[None, :]
        Etot = sla.solve(A, Einc.T).T
    else:
        def mv(x):
            return x - ops.gd((c * x).reshape(p.ny, p.nx)).reshape(-1)
        A = spla.LinearOperator((m, m), matvec=mv, dtype=np.complex128)
        Etot = np.empty_like(Einc)
        for t in range(p.ni):
            x, info = spla.bicgstab(A, Einc[t], x0=Einc[t].copy(), rtol=tol, maxiter=5000)
            if info != 0:
                x, info = spla.gmres(A, Einc[t], x0=x, rtol=tol, restart=200, maxiter=200)
            if info != 0:
                raise RuntimeError(f"forward solve did not converge for incidence {t} (info={info})")
            Etot[t] = x
    J = c[None, :] * Etot
    Esca = J @ ops.GS.T
    return J.reshape(p.ni, p.ny, p.nx), Etot.reshape(p.ni, p.ny, p.nx), Esca
