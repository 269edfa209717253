"""Oracle: gradient of J = 1/2 |u_loc(theta) - u_obs|^2 for the ONE-PASS
localized gamblet solution u_loc (Algorithm 2 with exact patch solves,
Definition defb, and exact level solves, Alg. 2 lines 8 and 16), with respect
to the cell log-coefficients theta_c = log a_c of the Q1 problem of Sec. 5.1.

The paper differentiates nothing; this is reverse-mode differentiation of
the map theta -> A^(q)(theta) -> (localized setup) -> u_loc, written out
step by step in the paper's notation (dense float64, small grids).  With X-bar
the adjoint of a quantity X:

Solve (Alg. 2 lines 15, 8, 16, 17, 18 in reverse order)
  v^(1) = U^(1), v^(k) = R^(k,k-1) v^(k-1) + W^(k)T w^(k), u_loc = v^(q)
  vbar^(q) = u_loc - u_obs, vbar^(k-1) = R^(k-1,k) vbar^(k),
  Rbar^(k-1,k) += v^(k-1) vbar^(k)T, lambda^(k) = B^(k)-1 W^(k) vbar^(k),
  lambda^(1) = A^(1)-1 vbar^(1);  Abar^(1) = -lambda^(1) U^(1)T,
  Abar^(k) += W^T (-lambda^(k) w^(k)T) W;
  gbar^(1) = lambda^(1), gbar^(k) = W^T lambda^(k) + R^(k,k-1) gbar^(k-1),
  Rbar^(k-1,k) += gbar^(k-1) g^(k)T.
  (gbar^(q) = dJ/dg.)
Setup, k = 2..q (Alg. 2 lines 13, 12, 11, 7 in reverse order)
  Xbar = (Abar^(k-1) + Abar^(k-1)T)/2   (A^(k-1) is symmetrised after line 13)
  Abar^(k) += R^T Xbar R,  Rbar += 2 Xbar R A^(k)            (line 13)
  Dbar = W Rbar^T                                            (line 12)
  per patch i: mu_i = B_i^-1 Dbar[i^chi, i],  bbar_i = mu_i,
               Bbar[i^chi, i^chi] -= mu_i y_i^T              (line 11)
  Abar^(k) += W^T Bbar W - W^T bbar pibar                    (line 7 and the
                                                              patch right-hand
                                                              side)
Fine operator (Sec. 5.1): A^(q) = sum_c a_c K_c, so
  dJ/dtheta_c = a_c sum_{p,r corners of c} Abar^(q)_sym[p, r] K_ref[p, r].

Pins (tests/test_oracle_local_adjoint.py): central differences of the
one-pass map itself (also on a domain with holes), the exact-solution
adjoint when the patches cover the domain, dJ/dg = G_loc (u_loc - u_obs)
(G_loc is symmetric), and planted mistakes that the differences catch.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from workloads import cell_corner_dofs

from .local import gamblet_local_setup


def _dense(M):
    return M.toarray() if hasattr(M, "toarray") else np.asarray(M, dtype=np.float64)


def _spd_solve(M, b):
    if M.shape[0] == 0:
        return np.zeros(b.shape)
    return sla.cho_solve(sla.cho_factor(M, lower=True), b)


def one_pass(A, g, cells, q, rho, rule="euclid", construction="const2"):
    """Localized setup and one-pass solve with every intermediate kept.
    Returns (setup, fwd) with fwd = {g, w, U1, v, u}."""
    S = gamblet_local_setup(A, cells, q, rho, rule, construction)
    R, W, B, Am = S["R"], S["W"], S["B"], S["A"]
    gk = {q: np.asarray(g, dtype=np.float64)}
    for k in range(q, 1, -1):                          # Alg. 2 line 15
        gk[k - 1] = R[k] @ gk[k]
    w = {k: _spd_solve(_dense(B[k]), W[k] @ gk[k]) for k in range(2, q + 1)}
    U1 = _spd_solve(_dense(Am[1]), gk[1])              # line 16
    v = {1: U1}
    for k in range(2, q + 1):                          # lines 10, 17, 18
        v[k] = R[k].T @ v[k - 1] + W[k].T @ w[k]
    return S, {"g": gk, "w": w, "U1": U1, "v": v, "u": v[q]}


def cell_gradient(n, a, Abar_q, K_ref, cell_nodes=None):
    """dJ/dlog a_c = a_c sum_{p,r} Abar_sym[p, r] K_ref[p, r] over the
    unknown corners of each cell (cells row-major, as log_a.ravel();
    cell_nodes[c, p] = unknown of corner p or -1, default: every interior
    node of the n x n grid)."""
    X = 0.5 * (Abar_q + Abar_q.T)
    cd = cell_corner_dofs(n) if cell_nodes is None else np.asarray(cell_nodes)
    av = np.asarray(a, dtype=np.float64).ravel()
    out = np.zeros(n * n)
    for c in range(n * n):
        s = 0.0
        for p in range(4):
            if cd[c, p] < 0:
                continue
            for r in range(4):
                if cd[c, r] < 0:
                    continue
                s += X[cd[c, p], cd[c, r]] * K_ref[p, r]
        out[c] = av[c] * s
    return out


def gradient_one_pass(A, g, u_obs, n, a, K_ref, cells, q, rho, rule="euclid",
                      construction="const2", cell_nodes=None):
    """Returns dict with J, grad (dJ/dlog a per cell), u (the one-pass
    solution), dJ_dg, and the per-level adjoints Abar (dense) and Rbar."""
    S, f = one_pass(A, g, cells, q, rho, rule, construction)
    H = S["hier"]
    R = {k: _dense(S["R"][k]) for k in range(2, q + 1)}
    W = {k: _dense(S["W"][k]) for k in range(2, q + 1)}
    B = {k: _dense(S["B"][k]) for k in range(2, q + 1)}
    Ad = {k: _dense(S["A"][k]) for k in range(1, q + 1)}
    gk, w, U1, v = f["g"], f["w"], f["U1"], f["v"]
    ubar = f["u"] - np.asarray(u_obs, dtype=np.float64)
    J = 0.5 * float(ubar @ ubar)

    # ---- reverse of the one-pass solve
    Rbar = {k: np.zeros(R[k].shape) for k in range(2, q + 1)}
    Abar = {k: np.zeros(Ad[k].shape) for k in range(1, q + 1)}
    vbar = {q: ubar}
    for k in range(q, 1, -1):
        vbar[k - 1] = R[k] @ vbar[k]
        Rbar[k] += np.outer(v[k - 1], vbar[k])
    lam = {k: _spd_solve(B[k], W[k] @ vbar[k]) for k in range(2, q + 1)}
    lam1 = _spd_solve(Ad[1], vbar[1])
    Abar[1] += -np.outer(lam1, U1)
    for k in range(2, q + 1):
        Abar[k] += W[k].T @ (-np.outer(lam[k], w[k])) @ W[k]
    gbar = {1: lam1}
    for k in range(2, q + 1):
        Rbar[k] += np.outer(gbar[k - 1], gk[k])
        gbar[k] = W[k].T @ lam[k] + R[k].T @ gbar[k - 1]

    # ---- reverse of the localized setup, coarse to fine
    for k in range(2, q + 1):
        Xbar = 0.5 * (Abar[k - 1] + Abar[k - 1].T)
        Abar[k] += R[k].T @ Xbar @ R[k]
        Rbar[k] += 2.0 * Xbar @ R[k] @ Ad[k]
        Wk = W[k]
        pibar = _dense(H.pibar(k))
        Dbar = Wk @ Rbar[k].T                          # J^(k) x I^(k-1)
        rhs = -(Wk @ Ad[k] @ pibar.T)
        jpar = H.j_parent(k)
        nbrs = H.neighbours(k - 1, rho, rule)
        nkm1 = H.n(k - 1)
        Bbar = np.zeros(B[k].shape)
        rhsbar = np.zeros(rhs.shape)
        in_patch = np.zeros(nkm1, dtype=bool)
        for i in range(nkm1):
            in_patch[:] = False
            in_patch[nbrs[i]] = True
            chi = np.nonzero(in_patch[jpar])[0]
            if len(chi) == 0:
                continue
            Bp = B[k][np.ix_(chi, chi)]
            y = _spd_solve(Bp, rhs[chi, i])
            mu = _spd_solve(Bp, Dbar[chi, i])
            rhsbar[chi, i] += mu
            Bbar[np.ix_(chi, chi)] -= np.outer(mu, y)
        Abar[k] += Wk.T @ Bbar @ Wk - Wk.T @ rhsbar @ pibar

    grad = cell_gradient(n, a, Abar[q], K_ref, cell_nodes)
    return {"J": J, "grad": grad, "u": f["u"], "dJ_dg": gbar[q],
            "Abar": Abar, "Rbar": Rbar, "setup": S}
