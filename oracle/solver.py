"""Newton's method with load steps on tiny meshes, with direct linear solves (oracle;
test infrastructure only).

Section 2.1: Newton's method for F(u, du) = 0 with the tangent K(u; du, .) (Eq. DF);
Section 2.2: at every iterate the correction solves K(u; Du, phi_i) = -F(u, phi_i).
Here the linear systems are solved exactly (dense LU on the assembled matrices), which is
the plain definition the GPU's iterative solvers approximate.

Load stepping and Dirichlet lifting (a reading; the paper's own test applies tractions):
load step s of S prescribes g_s (u_z = -c s/S on z = 1 for the compression preset).  At
iterate u, d = g_s - u on the constrained set D (0 elsewhere); the correction solves
A du = b with b_f = -R_f(u) - (K(u) d)_f and b_D = d_D, A the constrained operator (identity
rows and columns on D); u += theta du with theta halved while det F <= 0 somewhere.  A step
converges when d = 0 and ||b|| <= rtol ||b_0||, b_0 the right-hand side of its first iterate.
"""
from __future__ import annotations

import numpy as np

from .fem import Operator
from .material import NonPositiveJacobian


def newton_load_steps(op: Operator, steps: int, compression: float, rtol: float = 1e-8,
                      max_iter: int = 20, first: int = 1, last: int | None = None,
                      u0: np.ndarray | None = None, max_backtracks: int = 8):
    mesh = op.mesh
    raw = Operator(mesh, op.mu, op.lam, bc=0, model=op.model, factors=op.factors)
    fixed = op.fixed
    u = np.zeros(mesh.n_dofs) if u0 is None else u0.copy()
    last = steps if last is None else last
    history = []
    for s in range(first, last + 1):
        g = mesh.prescribed_values(op.bc, -compression * s / steps)
        ref = None
        its = 0
        rel = None
        for it in range(max_iter + 1):
            R = op.residual(u)
            d = np.where(fixed, g - u, 0.0)
            b = -R
            if np.any(d != 0.0):
                b = b - raw.assemble(u) @ d
            b[fixed] = d[fixed]
            bn = np.linalg.norm(b)
            ref = bn if ref is None else ref
            rel = bn / ref if ref > 0 else 0.0
            its = it
            if not np.any(d != 0.0) and (bn <= rtol * ref or bn == 0.0):
                break
            if it == max_iter:
                raise RuntimeError(f"oracle Newton: load step {s} did not converge")
            du = np.linalg.solve(op.assemble(u), b)
            theta = 1.0
            for _ in range(max_backtracks + 1):
                trial = u + theta * du
                try:
                    op.residual(trial)
                    break
                except NonPositiveJacobian:
                    theta *= 0.5
            else:
                raise NonPositiveJacobian("oracle Newton: backtracking failed")
            u = trial
            if theta == 1.0:
                u[fixed] = g[fixed]
        history.append({"step": s, "newton_iters": its, "rel_residual": rel})
    return u, history
