"""Direction-independent G-Jones calibration (Sec. 5.1, Architectural View for Calibration),
written out in FP64 in the paper's order: Eq. VAvg, then Eq. CalUpdateDir and Eq. CalUpdateModel
iterated to the exit test |g^{k+1} - g^k| < delta.

TEST INFRASTRUCTURE ONLY (see the package header).

Readings where the paper is terse:
* Eq. VAvg sums V / M over the solution interval; the weighted form used here is
  X = sum w V conj(M) / sum w |M|^2 (the average of V / M weighted by w |M|^2, which is that ratio
  when V / M is constant), and its weight w_ij is sum w |M|^2.  Flagged samples (w <= 0) are skipped.
* Eq. CalUpdateDir sums over the baselines of antenna i with X_ij = conj(X_ji); all g_j are those
  of iteration k (Jacobi order); the exit test is the largest |g_i^{k+1} - g_i^k| over antennas.
* The solution is defined up to a common phase; the reference antenna's phase is removed at the
  end (g_i conj(g_ref) / |g_ref|).
* The parallel hands are pols 0 and P - 1; the iteration starts from g = 1.
"""
from __future__ import annotations

import numpy as np


def average(vis, model, weight, n_bl, sol_int, sol_chan):
    """Eq. VAvg: X [n_ts, n_fs, n_hands, n_bl] complex128 and its weights (float64)."""
    vis = np.asarray(vis, dtype=np.complex128)
    model = np.asarray(model, dtype=np.complex128)
    weight = np.asarray(weight, dtype=np.float64)
    R, C, P = vis.shape
    n_int = R // n_bl
    hands = [0] if P == 1 else [0, P - 1]
    n_ts, n_fs = -(-n_int // sol_int), -(-C // sol_chan)
    X = np.zeros((n_ts, n_fs, len(hands), n_bl), dtype=np.complex128)
    Wt = np.zeros((n_ts, n_fs, len(hands), n_bl), dtype=np.float64)
    v = vis.reshape(n_int, n_bl, C, P)
    m = model.reshape(n_int, n_bl, C, P)
    w = np.where(weight > 0, weight, 0.0).reshape(n_int, n_bl, C, P)
    for ts in range(n_ts):
        t0, t1 = ts * sol_int, min((ts + 1) * sol_int, n_int)
        for fs in range(n_fs):
            c0, c1 = fs * sol_chan, min((fs + 1) * sol_chan, C)
            for q, p in enumerate(hands):
                vv, mm, ww = v[t0:t1, :, c0:c1, p], m[t0:t1, :, c0:c1, p], w[t0:t1, :, c0:c1, p]
                num = (ww * vv * np.conj(mm)).sum(axis=(0, 2))
                den = (ww * np.abs(mm) ** 2).sum(axis=(0, 2))
                X[ts, fs, q] = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
                Wt[ts, fs, q] = den
    return X, Wt


def solve_gains(X, Wt, ant1, ant2, n_ant, alpha, delta, max_iter, ref_ant=0):
    """Eq. CalUpdateDir / Eq. CalUpdateModel for one (interval, hand): X, Wt [n_bl].
    Returns (gains [n_ant] complex128, iterations run)."""
    ant1 = np.asarray(ant1)
    ant2 = np.asarray(ant2)
    g = np.ones(n_ant, dtype=np.complex128)
    it = 0
    for it in range(1, max_iter + 1):
        num = np.zeros(n_ant, dtype=np.complex128)
        den = np.zeros(n_ant, dtype=np.float64)
        # antenna ant1 sees X_ij (j = ant2); antenna ant2 sees X_ji = conj(X_ij) (j = ant1)
        np.add.at(num, ant1, g[ant2] * X * Wt)
        np.add.at(den, ant1, np.abs(g[ant2]) ** 2 * Wt)
        np.add.at(num, ant2, g[ant1] * np.conj(X) * Wt)
        np.add.at(den, ant2, np.abs(g[ant1]) ** 2 * Wt)
        step = np.where(den > 0, num / np.where(den > 0, den, 1.0), g)
        g_new = np.where(den > 0, (1.0 - alpha) * g + alpha * step, g)
        change = np.abs(g_new - g).max()
        g = g_new
        if change < delta:
            break
    gr = g[ref_ant]
    if abs(gr) > 0:
        g = g * np.conj(gr) / abs(gr)
    return g, it


def gcal(vis, model, weight, ant1, ant2, n_ant, sol_int, sol_chan, alpha, delta, max_iter, ref_ant=0):
    """Whole solve: (gains [n_ts, n_fs, n_hands, n_ant], iterations [n_ts, n_fs, n_hands])."""
    n_bl = len(ant1)
    X, Wt = average(vis, model, weight, n_bl, sol_int, sol_chan)
    G = np.zeros(X.shape[:3] + (n_ant,), dtype=np.complex128)
    its = np.zeros(X.shape[:3], dtype=np.int32)
    for idx in np.ndindex(*X.shape[:3]):
        G[idx], its[idx] = solve_gains(X[idx], Wt[idx], ant1, ant2, n_ant, alpha, delta, max_iter, ref_ant)
    return G, its
