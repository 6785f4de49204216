"""Deterministic solutions of the linearised RTA phonon BTE that pin the
Monte Carlo oracle (TEST INFRASTRUCTURE ONLY).

Every function here is a plain definition or a textbook solve, written with
numpy / scipy library primitives (the exponential integrals E_n come from
``scipy.special.expn``):

* ``kinetic_kappa``       bulk limit kappa = (1/3) sum_i C_i v_i^2 tau_i
* ``fuchs_sondheimer``    in-plane film reduction S(d/Lambda, p) per bin
* ``gray_slab_nystrom``   gray slab between black (isothermal) walls: the
                          integral equation for the local temperature with
                          the E1 kernel, solved by product integration; the
                          heat flux Psi = 1 - 2 int phi E2
* ``gray_slab_ordinates`` the same slab by discrete ordinates (independent)
* ``nongray_slab``        frequency-dependent slab between black walls: the
                          multi-group integral equation for the local
                          temperature (relaxation weights C_i / tau_i of
                          Eq. n_scatt), per-bin flux and energy temperature
* ``ballistic_transient`` the paper's Eq. Analytical_T (Sec. 5.1)
* ``gaussian_fourier``    long-time Fourier solution of a Gaussian hot spot
                          against an adiabatic plane (image method)
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import expn


def E(n: int, x):
    """Exponential integral E_n(x) for x >= 0, with E_n(0) = 1/(n-1) (n >= 2)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    zero = x <= 0.0
    if n >= 2:
        out[zero] = 1.0 / (n - 1)
    else:
        out[zero] = np.inf
    out[~zero] = expn(n, x[~zero])
    return out


def kinetic_kappa(C, v, tau) -> float:
    """Bulk RTA conductivity (1/3) sum_i C_i v_i^2 tau_i  (W/m/K)."""
    C, v, tau = (np.asarray(a, dtype=np.float64) for a in (C, v, tau))
    return float(np.sum(C * v * v * tau) / 3.0)


def fs_suppression(delta, p: float = 0.0, kmax: int = 4000):
    """Fuchs-Sondheimer S(delta, p) = 1 - 3(1-p)/(2 delta) int_1^inf (t^-3 - t^-5)
    (1 - e^{-delta t}) / (1 - p e^{-delta t}) dt, evaluated through the
    geometric series in p e^{-delta t} and int_1^inf t^-n e^{-a t} dt = E_n(a)."""
    delta = np.atleast_1d(np.asarray(delta, dtype=np.float64))
    acc = np.zeros_like(delta)
    pk = 1.0
    for k in range(kmax):
        a0 = k * delta
        a1 = (k + 1) * delta
        term = (E(3, a0) - E(5, a0)) - (E(3, a1) - E(5, a1))
        acc += pk * term
        pk *= p
        if pk < 1e-18:
            break
    return 1.0 - (3.0 * (1.0 - p) / (2.0 * delta)) * acc


def fuchs_sondheimer(C, v, tau, d: float, p: float = 0.0) -> float:
    """In-plane conductivity of a film of thickness d with wall specularity p:
    sum_i (1/3) C_i v_i^2 tau_i S(d / Lambda_i, p)."""
    C, v, tau = (np.asarray(a, dtype=np.float64) for a in (C, v, tau))
    lam = v * tau
    return float(np.sum(C * v * v * tau / 3.0 * fs_suppression(d / lam, p)))


def _hat_moments_E1(x_a, x_b):
    """For x in [x_a, x_b] (0 <= x_a < x_b): int E1(x) dx and int x E1(x) dx."""
    e2a, e2b = E(2, x_a), E(2, x_b)
    e3a, e3b = E(3, x_a), E(3, x_b)
    m0 = e2a - e2b
    m1 = x_a * e2a - x_b * e2b + e3a - e3b
    return m0, m1


def gray_slab_nystrom(tau0: float, n: int = 801):
    """Gray slab of optical thickness tau0 between black walls (hot at 0,
    cold at tau0).  phi(tau) = (T_loc - T_cold)/(T_hot - T_cold) solves
        phi(tau) = 1/2 [ E2(tau) + int_0^tau0 phi(t) E1(|tau - t|) dt ].
    phi is piecewise linear on n uniform nodes and the E1 kernel is integrated
    exactly against each hat function (product integration).
    Returns (nodes, phi, Psi) with Psi = q / (C v dT / 4) = 1 - 2 int phi E2."""
    t = np.linspace(0.0, tau0, n)
    h = t[1] - t[0]
    K = np.zeros((n, n))
    for i in range(n):
        ti = t[i]
        for side in (0, 1):
            # intervals [t_j, t_j+1] to the right (side 0) or left (side 1) of t_i
            if side == 0:
                js = np.arange(i, n - 1)
                xa = t[js] - ti
                xb = t[js + 1] - ti
                near, far = js, js + 1        # node at x_a, node at x_b
            else:
                js = np.arange(0, i)
                xa = ti - t[js + 1]
                xb = ti - t[js]
                near, far = js + 1, js
            if js.size == 0:
                continue
            m0, m1 = _hat_moments_E1(xa, xb)
            # hat at x_a: (x_b - x)/h ; hat at x_b: (x - x_a)/h
            w_near = (xb * m0 - m1) / h
            w_far = (m1 - xa * m0) / h
            np.add.at(K[i], near, w_near)
            np.add.at(K[i], far, w_far)
    A = np.eye(n) - 0.5 * K
    rhs = 0.5 * E(2, t)
    phi = np.linalg.solve(A, rhs)
    # int_0^tau0 phi(t) E2(t) dt with the same piecewise-linear phi
    xa, xb = t[:-1], t[1:]
    e3a, e3b, e4a, e4b = E(3, xa), E(3, xb), E(4, xa), E(4, xb)
    m0 = e3a - e3b
    m1 = xa * e3a - xb * e3b + e4a - e4b
    integ = np.sum(phi[:-1] * (xb * m0 - m1) / h + phi[1:] * (m1 - xa * m0) / h)
    return t, phi, 1.0 - 2.0 * integ


def _hat_weights(n_nodes: int, h: float, n: int):
    """Product-integration weights of the kernel E_n on a uniform grid of
    spacing h (optical units).  For the interval whose near end lies at
    distance m h and far end at (m + 1) h from the evaluation point, a[m] and
    b[m] are the weights of its near and far node in int f(t') E_n(|t' - s|) dt'
    with f linear on the interval (moments int E_n = -E_{n+1},
    int x E_n = -x E_{n+1} - E_{n+2})."""
    m = np.arange(n_nodes - 1, dtype=np.float64)
    xa, xb = m * h, (m + 1.0) * h
    ea1, eb1 = E(n + 1, xa), E(n + 1, xb)
    m0 = ea1 - eb1
    m1 = xa * ea1 - xb * eb1 + E(n + 2, xa) - E(n + 2, xb)
    return (xb * m0 - m1) / h, (m1 - xa * m0) / h


def _kernel_matrix(a, b):
    """K[i, k] = weight of node k in int f(t') E_n(|t' - t_i|) dt' over the
    whole grid, from the per-interval weights of _hat_weights."""
    n = a.shape[0] + 1
    ap, bp = np.append(a, 0.0), np.append(b, 0.0)
    i = np.arange(n)[:, None]
    k = np.arange(n)[None, :]
    o = np.abs(k - i)
    prev = bp[np.maximum(o - 1, 0)]
    K = np.where(k > i, ap[o] * (k <= n - 2) + prev, 0.0)
    K += np.where(k < i, ap[o] * (k >= 1) + prev, 0.0)
    K += np.where(k == i, a[0] * ((i <= n - 2).astype(np.float64) + (i >= 1)), 0.0)
    return K


def _side_rows(a, b, s: int):
    """Rows (right, left) of node weights in int_{t' > t_s} f E_n(t' - t_s) dt'
    and int_{t' < t_s} f E_n(t_s - t') dt'."""
    n = a.shape[0] + 1
    ap, bp = np.append(a, 0.0), np.append(b, 0.0)
    k = np.arange(n)
    o = np.abs(k - s)
    prev = bp[np.maximum(o - 1, 0)]
    right = np.where(k > s, ap[o] * (k <= n - 2) + prev, 0.0)
    right += np.where(k == s, a[0] * (s <= n - 2), 0.0)
    left = np.where(k < s, ap[o] * (k >= 1) + prev, 0.0)
    left += np.where(k == s, a[0] * (s >= 1), 0.0)
    return right, left


def nongray_slab(C, v, tau, L: float, dT_hot: float, dT_cold: float, n_cells: int,
                 n_nodes: int = 801, relax_weights=None) -> dict:
    """Frequency-dependent slab 0 <= z <= L between black walls (deviational
    temperatures dT_hot at z = 0, dT_cold at z = L), linearised RTA with one
    relaxation time per bin.

    With t = z / Lambda_i (Lambda_i = v_i tau_i) the pseudo-temperature of
    bin i (its energy density over C_i) is
        T_i(t) = 1/2 [dT_hot E2(t) + dT_cold E2(tau0_i - t)
                      + g_i int_0^tau0_i T_loc(t') E1(|t - t'|) dt']
    and the local temperature balances the relaxed energy,
        T_loc = sum_i w_i T_i,   w_i = (C_i / tau_i) / sum_j (C_j / tau_j).
    g_i = 1 when relaxed energy is re-emitted in proportion to C_i / tau_i
    (Eq. n_scatt); a re-emission law w'_i (relax_weights, normalised here)
    gives g_i = w'_i / w_i.  T_loc is piecewise linear on n_nodes uniform
    nodes and every kernel is integrated exactly against it (product
    integration); (n_nodes - 1) must be a multiple of n_cells.

    Returns the nodes z, T_loc at the nodes, the cell averages of the energy
    temperature sum_i C_i T_i / sum_i C_i ("T_cells", the track-length
    temperature of Eq. temp_steady), the slab-averaged flux of every bin
    (1/L) int q_i dz with q_i = (C_i v_i / 2)[dT_hot E3(t) - dT_cold E3(tau0 - t)
    + g_i int T_loc(t') sgn(t - t') E2(|t - t'|) dt'] ("q_bin", the per-bin
    flux of Eq. flux_x_steady), and their sum ("q")."""
    C, v, tau = (np.asarray(x, dtype=np.float64) for x in (C, v, tau))
    nb = C.shape[0]
    if (n_nodes - 1) % n_cells:
        raise ValueError("n_nodes - 1 must be a multiple of n_cells")
    lam = v * tau
    u = C / tau
    w = u / u.sum()
    wr = u if relax_weights is None else np.asarray(relax_weights, dtype=np.float64)
    g = (wr / wr.sum()) / w
    z = np.linspace(0.0, L, n_nodes)
    A = np.eye(n_nodes)
    rhs = np.zeros(n_nodes)
    groups = []
    for i in range(nb):
        tau0 = L / lam[i]
        h = tau0 / (n_nodes - 1)
        t = z / lam[i]
        a1, b1 = _hat_weights(n_nodes, h, 1)
        A -= (0.5 * w[i] * g[i]) * _kernel_matrix(a1, b1)
        rhs += (0.5 * w[i]) * (dT_hot * E(2, t) + dT_cold * E(2, tau0 - t))
        groups.append((tau0, h, t))
    f = np.linalg.solve(A, rhs)
    per = (n_nodes - 1) // n_cells
    edges = np.arange(0, n_nodes, per)
    T_bins = np.zeros((nb, n_cells))
    q_bin = np.zeros(nb)
    for i, (tau0, h, t) in enumerate(groups):
        a2, b2 = _hat_weights(n_nodes, h, 2)
        J = np.zeros(edges.shape[0])
        for c, s in enumerate(edges):
            r, l = _side_rows(a2, b2, int(s))
            J[c] = (r - l) @ f
        ta, tb = t[edges[:-1]], t[edges[1:]]
        inner = np.array([h * (0.5 * f[s] + f[s + 1:s + per].sum() + 0.5 * f[s + per]) for s in edges[:-1]])
        wall = dT_hot * (E(3, ta) - E(3, tb)) + dT_cold * (E(3, tau0 - tb) - E(3, tau0 - ta))
        T_bins[i] = (0.5 * wall + 0.5 * g[i] * (2.0 * inner + J[1:] - J[:-1])) / (tb - ta)
        a3, b3 = _hat_weights(n_nodes, h, 3)
        r0, _ = _side_rows(a3, b3, 0)
        _, lN = _side_rows(a3, b3, n_nodes - 1)
        vol = (r0 - lN) @ f
        q_bin[i] = C[i] * v[i] / (2.0 * tau0) * ((dT_hot - dT_cold) * (1.0 / 3.0 - E(4, tau0)) + g[i] * vol)
    T_cells = (C[:, None] * T_bins).sum(axis=0) / C.sum()
    return {"z": z, "T_loc": f, "T_cells": T_cells, "T_bins": T_bins, "q_bin": q_bin, "q": float(q_bin.sum())}


def nongray_slab_extrapolated(C, v, tau, L: float, dT_hot: float, dT_cold: float, n_cells: int,
                              relax_weights=None) -> dict:
    """nongray_slab on 401 and 801 nodes with Richardson extrapolation (O(h^2))."""
    r1 = nongray_slab(C, v, tau, L, dT_hot, dT_cold, n_cells, 401, relax_weights)
    r2 = nongray_slab(C, v, tau, L, dT_hot, dT_cold, n_cells, 801, relax_weights)
    out = dict(r2)
    for k in ("T_cells", "q_bin"):
        out[k] = r2[k] + (r2[k] - r1[k]) / 3.0
    out["q"] = float(out["q_bin"].sum())
    return out


def gray_slab_psi(tau0: float) -> float:
    """Psi(tau0) from two Nystrom grids with Richardson extrapolation (O(h^2))."""
    _, _, p1 = gray_slab_nystrom(tau0, 401)
    _, _, p2 = gray_slab_nystrom(tau0, 801)
    return p2 + (p2 - p1) / 3.0


def gray_slab_ordinates(tau0: float, n_mu: int = 32, n_cells: int = 400, tol: float = 1e-12):
    """Discrete ordinates for the same gray slab: double Gauss-Legendre
    directions on each hemisphere, step-characteristic sweeps with the
    isotropic source S = (1/2) sum_k w_k I_k, black walls I = 1 (hot) and 0,
    source iteration to convergence.  Returns (cell centres, phi, Psi)."""
    x, w = np.polynomial.legendre.leggauss(n_mu)
    mu = 0.5 * (x + 1.0)          # (0, 1)
    wm = 0.5 * w                  # weights on (0, 1), sum 1
    edges = np.linspace(0.0, tau0, n_cells + 1)
    dt = edges[1] - edges[0]
    S = np.full(n_cells, 0.5)
    a = np.exp(-dt / mu)
    b = 1.0 - a
    avg_coef = mu / dt * (1.0 - a)
    for _ in range(200000):
        Ip = np.zeros((n_mu, n_cells))   # forward (mu > 0) cell averages
        Im = np.zeros((n_mu, n_cells))
        I = np.ones(n_mu)
        for c in range(n_cells):
            Ip[:, c] = S[c] + (I - S[c]) * avg_coef
            I = I * a + S[c] * b
        I = np.zeros(n_mu)
        for c in range(n_cells - 1, -1, -1):
            Im[:, c] = S[c] + (I - S[c]) * avg_coef
            I = I * a + S[c] * b
        bwd_out = I
        S_new = 0.5 * (wm @ Ip + wm @ Im)
        if np.max(np.abs(S_new - S)) < tol:
            S = S_new
            break
        S = S_new
    # flux at the hot wall: q/(pi I1) = 2 * (int_0^1 I+ mu dmu - int_0^1 I- mu dmu)
    psi = 2.0 * (np.sum(wm * mu * 1.0) - np.sum(wm * mu * bwd_out))
    return 0.5 * (edges[1:] + edges[:-1]), S, psi


def ballistic_transient(z, t, L: float, v: float, dT_left: float, dT_right: float):
    """Eq. Analytical_T: purely ballistic 1-D temperature after the two walls
    are switched to dT_left (z=0) and dT_right (z=L) at t=0."""
    z = np.asarray(z, dtype=np.float64)
    a = 1.0 - z / (v * t)
    b = 1.0 - (L - z) / (v * t)
    return 0.5 * a * (a > 0) * dT_left + 0.5 * b * (b > 0) * dT_right


def gaussian_fourier(r2, t: float, sigma: float, dT: float, alpha: float):
    """Heat-equation solution for an initial Gaussian dT exp(-r^2/(2 sigma^2))
    in free space (equivalently: centred on an adiabatic plane, by images)."""
    s2 = sigma * sigma + 2.0 * alpha * t
    return dT * (sigma * sigma / s2) ** 1.5 * np.exp(-np.asarray(r2) / (2.0 * s2))
