"""Exact references that pin the oracle (test infrastructure only).

Nothing here shares arithmetic with oracle.tnmc's builder or sampler: these
are brute-force or closed-form computations of the quantities the method
approximates (Sec. 2, eqs. ising, boltzmann, pf-ising).
"""
import math

import numpy as np
from scipy import integrate, special


def all_states(Ly, Lx):
    """All 2^n configurations, [2^n, Ly, Lx] int8; state k has s_site = +1 iff bit `site` of k."""
    n = Ly * Lx
    k = np.arange(2 ** n, dtype=np.int64)[:, None]
    bits = (k >> np.arange(n, dtype=np.int64)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8).reshape(-1, Ly, Lx)


def energy_loops(Jh, Jv, h, s):
    """H of one configuration by explicit loops over sites and bonds (eq. ising)."""
    Ly, Lx = s.shape
    E = 0.0
    for r in range(Ly):
        for c in range(Lx):
            E -= h[r][c] * s[r][c]
            if c + 1 < Lx:
                E -= Jh[r][c] * s[r][c] * s[r][c + 1]
            if r + 1 < Ly:
                E -= Jv[r][c] * s[r][c] * s[r + 1][c]
    return E


def boltzmann(Jh, Jv, h, beta):
    """(states, log Z, pi) by enumeration (eqs. boltzmann, pf-ising); n <= ~22."""
    h = np.asarray(h, dtype=np.float64)
    Ly, Lx = h.shape
    S = all_states(Ly, Lx).astype(np.float64)
    E = -(h[None] * S).sum(axis=(1, 2))
    if Lx > 1:
        E -= (np.asarray(Jh).reshape(Ly, Lx - 1)[None] * S[:, :, :-1] * S[:, :, 1:]).sum(axis=(1, 2))
    if Ly > 1:
        E -= (np.asarray(Jv).reshape(Ly - 1, Lx)[None] * S[:, :-1, :] * S[:, 1:, :]).sum(axis=(1, 2))
    a = -beta * E
    amax = a.max()
    logZ = amax + math.log(np.exp(a - amax).sum())
    return S.astype(np.int8), logZ, np.exp(a - logZ), E


def transfer_matrix(Jh, Jv, h, beta):
    """Row transfer matrix over 2^Lx row states (Lx <= 12).

    Returns log Z, <E>, <|m|> with m = sum s / n, by propagating the
    distribution over (row state, running magnetisation) and the running
    energy moment, rescaling per row.
    """
    h = np.asarray(h, dtype=np.float64)
    Ly, Lx = h.shape
    Jh = np.asarray(Jh, dtype=np.float64).reshape(Ly, max(Lx - 1, 0))
    Jv = np.asarray(Jv, dtype=np.float64).reshape(max(Ly - 1, 0), Lx)
    rows = all_states(1, Lx).reshape(-1, Lx).astype(np.float64)     # [2^Lx, Lx]
    mrow = rows.sum(axis=1).astype(np.int64)                          # row magnetisation
    n = Lx * Ly
    nm = 2 * n + 1                                                    # M in [-n, n]

    def row_energy(r):
        e = -(rows * h[r][None]).sum(axis=1)
        if Lx > 1:
            e -= (Jh[r][None] * rows[:, :-1] * rows[:, 1:]).sum(axis=1)
        return e

    e0 = row_energy(0)
    Z = np.zeros((rows.shape[0], nm))          # weight by (row state, M + n)
    Ez = np.zeros((rows.shape[0], nm))         # energy-weighted
    w0 = np.exp(-beta * e0)
    Z[np.arange(rows.shape[0]), mrow + n] = w0
    Ez[np.arange(rows.shape[0]), mrow + n] = w0 * e0
    logscale = 0.0
    for r in range(1, Ly):
        ev = -(rows[:, None, :] * rows[None, :, :] * Jv[r - 1][None, None, :]).sum(axis=2)   # [prev, new]
        er = row_energy(r)
        etot = ev + er[None, :]
        T = np.exp(-beta * etot)
        Zn = np.zeros_like(Z)
        En = np.zeros_like(Ez)
        for j in range(rows.shape[0]):
            sh = mrow[j]
            contribZ = T[:, j] @ Z                      # over previous row states
            contribE = T[:, j] @ Ez + (T[:, j] * etot[:, j]) @ Z
            if sh >= 0:
                Zn[j, sh:] = contribZ[:nm - sh]
                En[j, sh:] = contribE[:nm - sh]
            else:
                Zn[j, :nm + sh] = contribZ[-sh:]
                En[j, :nm + sh] = contribE[-sh:]
        s = Zn.max()
        Z, Ez = Zn / s, En / s
        logscale += math.log(s)
    Ztot = Z.sum()
    logZ = logscale + math.log(Ztot)
    Emean = Ez.sum() / Ztot
    M = np.arange(nm) - n
    absm = (Z.sum(axis=0) * np.abs(M)).sum() / Ztot / n
    return logZ, Emean, absm


def onsager_minus_beta_f(beta):
    """-beta f of the infinite square-lattice ferromagnet, J = 1 (Onsager 1944)."""
    c2 = math.cosh(2 * beta) ** 2
    s2 = math.sinh(2 * beta)

    def g(t2, t1):
        return math.log(c2 - s2 * (math.cos(t1) + math.cos(t2)))

    val, _ = integrate.dblquad(g, 0.0, math.pi, 0.0, math.pi, epsabs=1e-11, epsrel=1e-11)
    # the integrand is even in each angle: [0, 2pi]^2 integral = 4 x [0, pi]^2
    return math.log(2.0) + 4.0 * val / (8.0 * math.pi ** 2)


def onsager_energy_per_spin(beta):
    """u = -coth(2 beta) [1 + (2/pi)(2 tanh^2(2 beta) - 1) K(k)], k = 2 sinh / cosh^2."""
    k = 2 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    K = special.ellipk(k * k)
    return -(1 / math.tanh(2 * beta)) * (1 + (2 / math.pi) * (2 * math.tanh(2 * beta) ** 2 - 1) * K)


def yang_magnetisation(beta):
    """Spontaneous magnetisation (1 - sinh(2 beta)^-4)^(1/8) for beta > beta_c (Yang 1952)."""
    x = 1.0 - math.sinh(2 * beta) ** -4
    return x ** 0.125 if x > 0 else 0.0


BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))     # T_c = 2 / ln(1 + sqrt 2)


def independence_acceptance(pi, q):
    """Stationary acceptance of the independence sampler with proposal q.

    a = sum_{w, w'} min(pi(w) q(w'), pi(w') q(w)) = sum_i q_i [ r_i Q_ge(i) + S_lt(i) ]
    with r = pi / q, Q_ge(i) = sum_{r_j >= r_i} q_j, S_lt(i) = sum_{r_j < r_i} q_j r_j.
    States with q = 0 contribute nothing (they are never proposed).
    """
    pi = np.asarray(pi, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    keep = q > 0
    pi, q = pi[keep], q[keep]
    r = pi / q
    order = np.argsort(r, kind="stable")
    r, q = r[order], q[order]
    # ties: group equal r so that "r_j >= r_i" includes all of the group
    uniq, start = np.unique(r, return_index=True)
    q_cum = np.concatenate([[0.0], np.cumsum(q)])
    qr_cum = np.concatenate([[0.0], np.cumsum(q * r)])
    grp = np.searchsorted(uniq, r)
    first = start[grp]
    q_ge = q_cum[-1] - q_cum[first]
    s_lt = qr_cum[first]
    return float(np.sum(q * (r * q_ge + s_lt)))


def tv_distance(pi, q):
    """||pi - q||_TV = 1/2 sum |pi - q| (eq. tv)."""
    return 0.5 * float(np.abs(np.asarray(pi) - np.asarray(q)).sum())


def row_weight_vector(Jh, Jv, h, beta, r):
    """psi_r(sigma_r): the exact weight of row r's configurations, by enumeration.

    The Boltzmann weight of rows r..Ly-1 (their fields, horizontal bonds and the
    vertical bonds among them) summed over rows r+1..Ly-1 -- the quantity the
    boundary-MPS environment of row r stands for (App. A, eq. braket-top-tm-bot,
    read bottom-up), without the vertical bonds to row r-1.  Entry j holds the
    row configuration with s_c = +1 iff bit c of j.  Cost 2^(Lx (Ly - r)).
    """
    h = np.asarray(h, dtype=np.float64)
    Ly, Lx = h.shape
    Jh = np.asarray(Jh, dtype=np.float64).reshape(Ly, max(Lx - 1, 0))
    Jv = np.asarray(Jv, dtype=np.float64).reshape(max(Ly - 1, 0), Lx)
    _, logZ, pi, _ = boltzmann(Jh[r:], Jv[r:], h[r:], beta)
    # boltzmann() enumerates the sub-lattice of rows r.. with row r in the low Lx bits
    w = pi.reshape(-1, 1 << Lx).sum(axis=0)          # sum over the rows below
    return w * math.exp(logZ)


def schmidt_values(psi, Lx, c):
    """Singular values of psi reshaped to (sites c..Lx-1) x (sites 0..c-1), divided by
    their 2-norm: the Schmidt coefficients of the cut between sites c-1 and c."""
    S = np.linalg.svd(np.asarray(psi).reshape(1 << (Lx - c), 1 << c), compute_uv=False)
    return S / math.sqrt(float(np.sum(S * S)))
