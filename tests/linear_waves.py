"""Linear MHD waves for convergence tests (test helper).

Background of Gardiner & Stone (2008, J. Comput. Phys. 227, 4123): rho = 1,
p = 1/gamma (sound speed 1), B = (1, sqrt(2), 1/2), at rest (entropy mode:
v_x = 1); fast, Alfven and slow speeds 2, 1, 1/2.  A wave along +x is the
background plus amp * r * sin(2 pi x), r the right eigenvector (of the
conservative 7-variable system at fixed B_x) of the wave's eigenvalue.  The
eigenvectors come from a central finite-difference Jacobian of the flux
written out below (independent of the oracle and of the library) and
numpy's eigen-solver; the exact linear solution translates at the
eigenvalue.  Point values at cell centres; face by, bz equal the cell values
(no variation across y, z), bx = 1.
"""
import numpy as np

GAMMA = 5.0 / 3.0
MODES = {"fast": 6, "alfven": 5, "slow": 4, "entropy": 3}   # index in the sorted eigenvalues


def _flux7(X, bn, gamma):
    rho, mn, m1, m2, b1, b2, E = X
    u, v1, v2 = mn / rho, m1 / rho, m2 / rho
    bb = bn * bn + b1 * b1 + b2 * b2
    p = (gamma - 1) * (E - 0.5 * (mn * u + m1 * v1 + m2 * v2) - 0.5 * bb)
    pt = p + 0.5 * bb
    return np.array([mn, mn * u + pt - bn * bn, m1 * u - bn * b1, m2 * u - bn * b2,
                     u * b1 - v1 * bn, u * b2 - v2 * bn, (E + pt) * u - bn * (u * bn + v1 * b1 + v2 * b2)])


def background(mode, gamma=GAMMA):
    rho, p = 1.0, 1.0 / gamma
    u = 1.0 if mode == "entropy" else 0.0
    bn, b1, b2 = 1.0, np.sqrt(2.0), 0.5
    E = p / (gamma - 1) + 0.5 * rho * u * u + 0.5 * (bn * bn + b1 * b1 + b2 * b2)
    return np.array([rho, rho * u, 0.0, 0.0, b1, b2, E]), bn


def eigen(mode, gamma=GAMMA):
    X0, bn = background(mode, gamma)
    A = np.zeros((7, 7))
    for c in range(7):
        h = 1e-7 * max(1.0, abs(X0[c]))
        Xp, Xm = X0.copy(), X0.copy()
        Xp[c] += h
        Xm[c] -= h
        A[:, c] = (_flux7(Xp, bn, gamma) - _flux7(Xm, bn, gamma)) / (2 * h)
    lam, R = np.linalg.eig(A)
    order = np.argsort(lam.real)
    lam, R = lam.real[order], R.real[:, order]
    k = MODES[mode]
    r = R[:, k] / np.abs(R[:, k]).max()
    return lam[k], r


def state(N, mode, amp=1e-5, t=0.0, ny=1, gamma=GAMMA, offset=0.5):
    """(U[8, ny, ny, N], bx, by, bz, dx, lam) of the wave at time t, sampled
    at x = (i + offset)/N (offset 0: the points of grid N are every m-th
    point of grid m N, for self-convergence against a finer run)."""
    lam, r = eigen(mode, gamma)
    X0, bn = background(mode, gamma)
    x = (np.arange(N) + offset) / N
    X = X0[:, None] + amp * r[:, None] * np.sin(2 * np.pi * (x - lam * t))[None, :]
    shape = (ny, ny, N)
    U = np.empty((8,) + shape)
    for q, f in zip((0, 1, 2, 3, 5, 6, 7), range(7)):
        U[q] = np.broadcast_to(X[f], shape)
    U[4] = bn
    bx = np.full(shape, bn)
    by = U[5].copy()
    bz = U[6].copy()
    return U, bx, by, bz, 1.0 / N, lam


def l1_error(U, Uex):
    """Gardiner-Stone error: |(mean |dq| per variable)| over the variables."""
    d = np.abs(U - Uex).reshape(8, -1).mean(axis=1)
    return float(np.sqrt((d * d).sum()))
