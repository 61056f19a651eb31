"""Plain FP64 oracle of the TNMH proposal path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may use this
module.  Everything is written for clarity: numpy loops over rows and sites,
vectorised over samples; numpy's QR / SVD / matmul serve as library steps.

Conventions (Sec. 2, eq. ising):
  lattice Ly x Lx, open boundaries, site (r, c), row r = 0 is sampled first;
  Jh[r, c]  bond (r, c)-(r, c+1)   shape (Ly, Lx-1)
  Jv[r, c]  bond (r, c)-(r+1, c)   shape (Ly-1, Lx)
  h[r, c]   field                  shape (Ly, Lx)
  H = -sum h s - sum J s s;   physical index 0 <-> s = -1, 1 <-> s = +1.

Environment of row r (App. A, eq. braket-top-tm-bot, read bottom-up):
  env_r(sigma_r) approximates the Boltzmann weight of rows r..Ly-1 summed over
  rows r+1.., including row r's fields and horizontal bonds but not the
  vertical bonds to row r-1.  It is an MPS  M^(r)_c[a, sigma, b]  built as
    env_{Ly-1} = exact row weight,
    env_r      = T_chi[ D_r H_r V_r env_{r+1} ],
  V_r: sum over row r+1 with the vertical bond weights (no bond growth),
  D_r: fields, H_r: horizontal bonds as a bond-2 copy MPO (bond doubles),
  T_chi: "successive SVD" -- a left-to-right QR sweep, then a right-to-left
  SVD sweep keeping chi_c = min(chi, 2^c, 2^(Lx-c), 2^(Ly-r)) values.
The conditioned rows above are a product state (the fixed-spin tensors of
App. A are rank one), so sampling row r uses env_r with site factors
  f_c(sigma) = exp(beta Jv[r-1, c] s_{r-1, c} sigma).
Each site conditional is normalised, w_+ / (w_+ + w_-) (Sec. 2, eq.
pi-approx), after clamping negative weights at zero.
"""
import math

import numpy as np

from . import philox

SPIN = np.array([-1.0, 1.0])          # physical index -> spin value
F_BAD = 1                             # flag: non-positive / non-finite normaliser


def bond_dim(chi, Lx, Ly, r, c):
    """Static bond dimension of bond c (between sites c-1 and c) of env_r."""
    if c <= 0 or c >= Lx:
        return 1
    e = min(c, Lx - c, Ly - r, 30)
    return min(chi, 1 << e)


class Env:
    """Boundary-MPS row environments of one instance (all FP64)."""

    def __init__(self, Lx, Ly, beta, chi, Jh, Jv, h):
        self.Lx, self.Ly, self.beta, self.chi = Lx, Ly, beta, chi
        self.Jh, self.Jv, self.h = Jh, Jv, h
        self.M = [None] * Ly            # M[r][c]: array (chi_c, 2, chi_{c+1})
        self.log_scale = np.zeros(Ly)   # log of the factor removed while building row r
        self.log_lambda = np.zeros(Ly + 1)
        self.sv = {}                    # (r, c) -> kept singular values / 2-norm of all
        self.discarded = {}             # (r, c) -> discarded squared weight fraction
        self.logZ = float("nan")
        self.Mr = None                  # optional Mr[r][c][u]: right-sweep tensors (env_bf16)
        self.order = "raster"           # site order: "raster", or "snake" (odd rows right to left)


def _check_lattice(Jh, Jv, h):
    h = np.asarray(h, dtype=np.float64)
    Ly, Lx = h.shape
    Jh = np.asarray(Jh, dtype=np.float64).reshape(Ly, max(Lx - 1, 0))
    Jv = np.asarray(Jv, dtype=np.float64).reshape(max(Ly - 1, 0), Lx)
    return Jh, Jv, h, Lx, Ly


def apply_row_mpo(env_next, Jh, Jv, h, beta, r):
    """D_r H_r V_r env_{r+1} as an explicit MPS with doubled bonds.

    Left index of site c > 0 is (a, k) -> 2 a + k with k the copied spin
    index of site c-1; right index of site c < Lx-1 is (b, k') -> 2 b + k'.
    """
    Ly, Lx = h.shape
    P = []
    for c in range(Lx):
        if env_next is None:
            t = np.ones((1, 2, 1))
        else:
            W = np.exp(beta * Jv[r, c] * np.outer(SPIN, SPIN))     # W[sigma, sigma']
            t = np.einsum("ts,asb->atb", W, env_next[c])
        t = t * np.exp(beta * h[r, c] * SPIN)[None, :, None]
        Dl, _, Dr = t.shape
        if c > 0:
            G = np.exp(beta * Jh[r, c - 1] * np.outer(SPIN, SPIN))  # G[k, sigma]
            t = np.einsum("asb,ks->aksb", t, G).reshape(Dl * 2, 2, Dr)
            Dl *= 2
        if c < Lx - 1:
            t2 = np.zeros((Dl, 2, Dr, 2))
            for s in range(2):
                t2[:, s, :, s] = t[:, s, :]
            t = t2.reshape(Dl, 2, Dr * 2)
        P.append(t)
    return P


def truncate_row(P, chi, Lx, Ly, r, env=None):
    """T_chi: left-to-right QR sweep, then right-to-left SVD sweep (App. A).

    Returns (tensors, log of the removed scale).  Rescalings along the sweeps
    only move a positive factor into the returned log-scale.
    """
    P = list(P)
    logs = 0.0
    for c in range(Lx - 1):
        Dl, _, Dr = P[c].shape
        Q, R = np.linalg.qr(P[c].reshape(Dl * 2, Dr))
        P[c] = Q.reshape(Dl, 2, Q.shape[1])
        sc = np.abs(R).max()
        if not sc > 0:
            raise FloatingPointError("row %d: zero environment" % r)
        logs += math.log(sc)
        P[c + 1] = np.einsum("ij,jsk->isk", R / sc, P[c + 1])
    for c in range(Lx - 1, 0, -1):
        Dl, _, Dr = P[c].shape
        U, S, Vh = np.linalg.svd(P[c].reshape(Dl, 2 * Dr), full_matrices=False)
        k = bond_dim(chi, Lx, Ly, r, c)
        assert k <= S.size
        P[c] = Vh[:k].reshape(k, 2, Dr)
        if not S[0] > 0:
            raise FloatingPointError("row %d: zero environment" % r)
        if env is not None:
            tot = float(np.sum(S * S))
            env.sv[(r, c)] = S[:k] / math.sqrt(tot)
            env.discarded[(r, c)] = float(np.sum(S[k:] ** 2)) / tot
        logs += math.log(S[0])
        P[c - 1] = np.einsum("isj,jk->isk", P[c - 1], U[:, :k] * (S[:k] / S[0]))
    n0 = float(np.linalg.norm(P[0]))
    if not n0 > 0:
        raise FloatingPointError("row %d: zero environment" % r)
    P[0] = P[0] / n0
    logs += math.log(n0)
    return P, logs


def build_env(Jh, Jv, h, beta, chi):
    """All row environments, bottom-up (App. A, eq. braket-top-tm-bot)."""
    Jh, Jv, h, Lx, Ly = _check_lattice(Jh, Jv, h)
    env = Env(Lx, Ly, float(beta), int(chi), Jh, Jv, h)
    nxt = None
    for r in range(Ly - 1, -1, -1):
        P = apply_row_mpo(nxt, Jh, Jv, h, beta, r)
        env.M[r], env.log_scale[r] = truncate_row(P, chi, Lx, Ly, r, env)
        env.log_lambda[r] = env.log_lambda[r + 1] + env.log_scale[r]
        nxt = env.M[r]
    # Z~ = lambda_0 * sum_sigma env_0(sigma): row 0 has no field from above.
    v = np.ones(1)
    logv = 0.0
    for c in range(Lx):
        v = v @ (env.M[0][c][:, 0, :] + env.M[0][c][:, 1, :])
        m = np.abs(v).max()
        if m > 0:
            v = v / m
            logv += math.log(m)
    env.logZ = env.log_lambda[0] + logv + math.log(v[0]) if v[0] > 0 else float("nan")
    return env


def round_bf16(x):
    """Round FP64 values to the nearest bfloat16 (8 significant bits, ties to even)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, |m| in [0.5, 1)
    e = np.maximum(e, -125)                  # bfloat16 shares float32's exponent range
    return np.ldexp(np.round(np.ldexp(m, 8 + (np.frexp(x)[1] - e))), e - 8)


def split_bf16(x):
    """hi + lo with hi = bf16(x), lo = bf16(x - hi): x to about 16 significant bits."""
    hi = round_bf16(x)
    return hi + round_bf16(np.asarray(x, dtype=np.float64) - hi)


def field_combined(env, r, c):
    """Mt^(u)[a, b] = sum_sigma f_u(sigma) M^(r)_c[a, sigma, b] for u = -1, +1 (index 0, 1):
    the site tensor with the field of the spin above (value u) applied, f_u(sigma) =
    exp(beta Jv[r-1, c] u sigma), 1 on row 0.  The right-sweep recursion of one sample
    is R_c = Mt^(u) R_{c+1} with u its spin above (Sec. 2, eq. pi-approx; App. A: the
    rows above are a product state)."""
    M = env.M[r][c]
    if r == 0:
        t = M[:, 0, :] + M[:, 1, :]
        return np.stack([t, t])
    f = np.exp(env.beta * env.Jv[r - 1, c] * np.outer(SPIN, SPIN))       # f[u, sigma]
    return np.einsum("us,asb->uab", f, M)


def env_bf16(env):
    """The environment as the tensor-core contraction sees it: every entry of M (left
    sweep) and of the field-combined right-sweep tensors Mt^(u) (formed in FP64) replaced
    by its BF16 hi + lo pair."""
    out = Env(env.Lx, env.Ly, env.beta, env.chi, env.Jh, env.Jv, env.h)
    out.M = [[split_bf16(t) for t in row] for row in env.M]
    out.Mr = [[split_bf16(field_combined(env, r, c)) for c in range(env.Lx)] for r in range(env.Ly)]
    out.log_scale, out.log_lambda, out.logZ = env.log_scale, env.log_lambda, env.logZ
    return out


def _pow2_normalize(x):
    """Scale each row of x by the power of two that puts its max |x| in [1, 2)."""
    m = np.max(np.abs(x), axis=1)
    _, e = np.frexp(m)
    e = np.where(m > 0, e - 1, 0)
    return np.ldexp(x, -e[:, None])


def row_fields(env, spins, r):
    """f[b, c, idx] = exp(beta Jv[r-1, c] s_{r-1, c} SPIN[idx]); ones for r = 0."""
    B = spins.shape[0]
    if r == 0:
        return np.ones((B, env.Lx, 2))
    up = spins[:, r - 1, :].astype(np.float64)
    return np.exp(env.beta * (env.Jv[r - 1][None, :, None] * up[:, :, None]) * SPIN[None, None, :])


def threshold_plus(pplus, x):
    """Draw rule: s = +1 iff x < floor(p_+ 2^64) (always when p_+ >= 1)."""
    ge1 = pplus >= 1.0
    K = np.where(ge1, 0.0, np.floor(pplus * 2.0 ** 64)).astype(np.uint64)
    return ge1 | (x < K)


def run(env, B, seed=0, sample_offset=0, forced=None, keep=False, samples=None):
    """Sequential sampler (forced=None) or evaluator (forced spins [B, Ly, Lx]).

    Sample b uses Philox sample index sample_offset + b, or samples[b] when an
    explicit index array is given.  Returns (spins int8 [B, Ly, Lx], logq [B],
    energy [B], flags [B]) and, with keep=True, the per-row forward record
    used by the gradient.  A site whose normaliser w_+ + w_- is not positive or not
    finite is drawn with p = 1/2, adds log 1/2 to log q and sets the sample's flag:
    log q stays the log of the probability the sample was drawn with, so q is the
    exact law of the procedure and MH stays exact.
    """
    Lx, Ly = env.Lx, env.Ly
    spins = np.zeros((B, Ly, Lx), dtype=np.int8) if forced is None else np.asarray(forced, dtype=np.int8)
    logq = np.zeros(B)
    flags = np.zeros(B, dtype=np.int32)
    if samples is None:
        samples = np.uint64(sample_offset) + np.arange(B, dtype=np.uint64)
    else:
        samples = np.asarray(samples, dtype=np.uint64)
    record = []
    snake = getattr(env, "order", "raster") == "snake"
    if snake and (keep or env.Mr is not None):
        raise NotImplementedError("snake order: no gradient record and no field-combined right tensors")
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for r in range(Ly):
            f = row_fields(env, spins, r)
            # the row in sampling order: row r runs right to left in snake order when r is odd;
            # the reversed row is the same MPS read backwards (site tensors with their bonds swapped)
            cols = list(range(Lx - 1, -1, -1)) if (snake and r % 2 == 1) else list(range(Lx))
            rev = cols[0] != 0
            M = [env.M[r][c].transpose(2, 1, 0) if rev else env.M[r][c] for c in cols]
            f = f[:, cols, :]
            R = [None] * (Lx + 1)
            R[Lx] = np.ones((B, 1))
            up = (spins[:, r - 1, :] > 0).astype(np.int64) if r > 0 else np.zeros((B, Lx), dtype=np.int64)
            for c in range(Lx - 1, 0, -1):
                if env.Mr is None:
                    Y = np.einsum("asb,nb->nas", M[c], R[c + 1])
                    R[c] = _pow2_normalize(Y[:, :, 0] * f[:, c, 0:1] + Y[:, :, 1] * f[:, c, 1:2])
                else:
                    # the same recursion with the field-combined tensor of each sample's
                    # spin above, as given (the rounded tensors of env_bf16)
                    R[c] = _pow2_normalize(np.einsum("nab,nb->na", env.Mr[r][c][up[:, c]], R[c + 1]))
            Lam = [None] * (Lx + 1)
            Lam[0] = np.ones((B, 1))
            wraw = np.zeros((B, Lx, 2))
            for c in range(Lx):
                U = np.einsum("na,asb->nsb", Lam[c], M[c])
                wr = np.einsum("nsb,nb->ns", U, R[c + 1]) * f[:, c, :]
                wraw[:, c, :] = wr
                w = np.maximum(wr, 0.0)
                tot = w[:, 0] + w[:, 1]
                bad = ~(tot > 0) | ~np.isfinite(tot)
                pplus = np.where(bad, 0.5, w[:, 1] / tot)
                pminus = np.where(bad, 0.5, w[:, 0] / tot)
                col = cols[c]
                if forced is None:
                    x = philox.draw_words(seed, r * Lx + col, samples)
                    plus = threshold_plus(pplus, x)
                    spins[:, r, col] = np.where(plus, 1, -1)
                else:
                    plus = spins[:, r, col] > 0
                logq += np.log(np.where(plus, pplus, pminus))
                flags |= np.where(bad, F_BAD, 0).astype(np.int32)
                idx = plus.astype(np.int64)
                Lam[c + 1] = _pow2_normalize(U[np.arange(B), idx, :] * f[np.arange(B), c, idx][:, None])
            if keep:
                record.append((row_fields(env, spins, r), R, Lam, wraw))
    E = energy(env.Jh, env.Jv, env.h, spins)
    if keep:
        return spins, logq, E, flags, record
    return spins, logq, E, flags


def sample(env, B, seed=0, sample_offset=0, samples=None):
    """Draw B proposals from q = pi~ (Sec. 2, eqs. pi-approx, tns-prior)."""
    return run(env, B, seed, sample_offset, samples=samples)


def logq(env, spins):
    """Forced evaluation of log q for given configurations (App. A, last eq.)."""
    s = np.asarray(spins, dtype=np.int8)
    return run(env, s.shape[0], forced=s)


def energy(Jh, Jv, h, spins):
    """H(sigma) of eq. ising for a batch of configurations [B, Ly, Lx]."""
    s = np.asarray(spins, dtype=np.float64)
    E = -(np.asarray(h)[None] * s).sum(axis=(1, 2))
    if s.shape[2] > 1:
        E -= (np.asarray(Jh)[None] * s[:, :, :-1] * s[:, :, 1:]).sum(axis=(1, 2))
    if s.shape[1] > 1:
        E -= (np.asarray(Jv)[None] * s[:, :-1, :] * s[:, 1:, :]).sum(axis=(1, 2))
    return E


def init_chains(env, C, seed):
    """Random +-1 start (Algorithm 1, second step) with its log q and energy."""
    sp = philox.init_bits(seed, env.Lx * env.Ly, np.arange(C)).reshape(C, env.Ly, env.Lx)
    _, lq, E, _ = logq(env, sp)
    return sp, lq, E


def mh_accept(beta, lq_prop, E_prop, lq_cur, E_cur, u):
    """Metropolis-Hastings rule of eq. mh-acc with g(w'|w) = q(w') (eq. tns-prior).

    Delta = log pi(prop) q(cur) / (pi(cur) q(prop)) = a(prop) - a(cur) with
    a = -beta E - log q (each a rounded once, then the difference); accept iff the
    proposal is valid (finite log q) and u < exp(min(0, Delta)).

    A current state with log q = -inf lies outside the numerical support of q
    (only the random start of Algorithm 1 can be such a state: every later state
    is an accepted proposal, whose log q is finite).  Its ratio
    q(cur) pi(prop) / (q(prop) pi(cur)) is then read as +inf rather than 0, so the
    first valid proposal is accepted; with the literal 0 the chain could never
    leave its start.  The rule only changes the transient out of the start.
    """
    with np.errstate(invalid="ignore", over="ignore"):
        d = (-beta * E_prop - lq_prop) - (-beta * E_cur - lq_cur)
        ok = np.isfinite(lq_prop) & ~np.isnan(d)
        start = np.isneginf(lq_cur)
        return ok & (start | (u < np.exp(np.minimum(np.where(ok & ~start, d, 0.0), 0.0))))


def mh_scan(beta, C, T, prop_spins, prop_logq, prop_E, chain_spins, chain_logq, chain_E,
            seed, step_offset=0):
    """C chains, chain i consumes proposals i*T .. i*T+T-1 in order (Algorithm 1).

    Returns (accepted [C*T] bool, new chain spins, log q, energy).
    """
    chains = np.arange(C)
    acc = np.zeros(C * T, dtype=bool)
    lq = np.array(chain_logq, dtype=np.float64)
    E = np.array(chain_E, dtype=np.float64)
    last = np.full(C, -1)
    for j in range(T):
        t = chains * T + j
        u = philox.mh_uniform(seed, np.uint64(step_offset + j), chains)
        a = mh_accept(beta, prop_logq[t], prop_E[t], lq, E, u)
        acc[t] = a
        lq = np.where(a, prop_logq[t], lq)
        E = np.where(a, prop_E[t], E)
        last = np.where(a, t, last)
    sp = np.array(chain_spins, copy=True)
    for i in range(C):
        if last[i] >= 0:
            sp[i] = prop_spins[last[i]]
    return acc, sp, lq, E


def logq_grad(env, spins, weights):
    """Reverse-mode gradient of sum_b weights_b log q(spins_b) w.r.t. every M^(r)_c.

    Follows the forced evaluation step by step: per-site normalised, clamped
    conditionals, power-of-two rescalings treated as constants.  Samples with
    a flag or with q = 0 contribute nothing.  Returns (logq, grads) with grads
    shaped like env.M.
    """
    spins = np.asarray(spins, dtype=np.int8)
    B = spins.shape[0]
    _, lq, _, flags, rec = run(env, B, forced=spins, keep=True)
    wts = np.where(np.isfinite(lq) & (flags == 0), np.asarray(weights, dtype=np.float64), 0.0)
    Lx = env.Lx
    grads = []
    for r in range(env.Ly):
        M = env.M[r]
        f, R, Lam, wraw = rec[r]
        s_idx = (spins[:, r, :] > 0).astype(np.int64)
        G = [np.zeros_like(m) for m in M]
        Lbar = [np.zeros_like(Lam[c]) for c in range(Lx + 1)]
        Rbar = [np.zeros_like(R[c]) for c in range(Lx + 1)]
        ar = np.arange(B)
        # direct terms of each site's log w(s) - log(w_+ + w_-)
        for c in range(Lx):
            w = np.maximum(wraw[:, c, :], 0.0)
            tot = w[:, 0] + w[:, 1]
            ws = w[ar, s_idx[:, c]]
            safe = (wts != 0) & (ws > 0) & (tot > 0)
            gw = np.zeros((B, 2))
            inv_tot = np.where(safe, 1.0 / np.where(safe, tot, 1.0), 0.0)
            gw -= inv_tot[:, None]
            gw[ar, s_idx[:, c]] += np.where(safe, 1.0 / np.where(safe, ws, 1.0), 0.0)
            gw *= (wraw[:, c, :] > 0) * wts[:, None] * f[:, c, :]
            # w(sigma) = f sum_ab Lam[a] M[a, sigma, b] R[b]
            G[c] += np.einsum("ns,na,nb->asb", gw, Lam[c], R[c + 1])
            Lbar[c] += np.einsum("ns,asb,nb->na", gw, M[c], R[c + 1])
            Rbar[c + 1] += np.einsum("ns,na,asb->nb", gw, Lam[c], M[c])
        # left chain: Lam[c+1] = kappa f(s) Lam[c] M[:, s, :]
        for c in range(Lx - 1, -1, -1):
            U = np.einsum("na,asb->nsb", Lam[c], M[c])[ar, s_idx[:, c], :] * f[ar, c, s_idx[:, c]][:, None]
            kap = _ratio(Lam[c + 1], U)
            coef = kap * f[ar, c, s_idx[:, c]]
            Ms = M[c][:, s_idx[:, c], :]                       # (a, n, b)
            Lbar[c] += np.einsum("n,anb,nb->na", coef, Ms, Lbar[c + 1])
            for s in range(2):
                sel = (s_idx[:, c] == s) * coef
                G[c][:, s, :] += np.einsum("n,na,nb->ab", sel, Lam[c], Lbar[c + 1])
        # right chain: R[c] = kappa sum_sigma f(sigma) M[:, sigma, :] R[c+1]
        for c in range(1, Lx):
            Y = np.einsum("asb,nb->nas", M[c], R[c + 1])
            raw = Y[:, :, 0] * f[:, c, 0:1] + Y[:, :, 1] * f[:, c, 1:2]
            kap = _ratio(R[c], raw)
            Rbar[c + 1] += np.einsum("n,ns,asb,na->nb", kap, f[:, c, :], M[c], Rbar[c])
            G[c] += np.einsum("n,ns,na,nb->asb", kap, f[:, c, :], Rbar[c], R[c + 1])
        grads.append(G)
    return lq, grads


def _ratio(scaled, raw):
    """Per-sample power-of-two factor kappa with scaled = kappa * raw."""
    m_s = np.max(np.abs(scaled), axis=1)
    m_r = np.max(np.abs(raw), axis=1)
    return np.where(m_r > 0, m_s / np.where(m_r > 0, m_r, 1.0), 1.0)


def logq_at(env, spins, r, c, delta):
    """log q after adding `delta` to M^(r)_c (finite-difference helper)."""
    M0 = env.M[r][c]
    env.M[r][c] = M0 + delta
    try:
        _, lq, _, _ = logq(env, spins)
    finally:
        env.M[r][c] = M0
    return lq


def finite_diff_grad(env, spins, weights, r, c, h_rel=1e-6):
    """Central differences of sum_b weights_b log q_b w.r.t. every entry of M^(r)_c."""
    M0 = env.M[r][c]
    h = h_rel * max(np.abs(M0).max(), 1e-300)
    G = np.zeros_like(M0)
    w = np.asarray(weights, dtype=np.float64)
    for idx in np.ndindex(M0.shape):
        d = np.zeros_like(M0)
        d[idx] = h
        G[idx] = (np.dot(w, logq_at(env, spins, r, c, d)) - np.dot(w, logq_at(env, spins, r, c, -d))) / (2 * h)
    return G


# ---- single-spin-flip Metropolis sweeps and the link-overlap diagnostic (Sec. 3) ----

def local_field(Jh, Jv, h, spins):
    """h_i + sum_j J_ij s_j for every site of every configuration [C, Ly, Lx] (eq. ising:
    the energy change of flipping s_i is 2 s_i times it)."""
    s = np.asarray(spins, dtype=np.float64)
    Ly, Lx = s.shape[1:]
    Jh = np.asarray(Jh, dtype=np.float64).reshape(Ly, max(Lx - 1, 0))
    Jv = np.asarray(Jv, dtype=np.float64).reshape(max(Ly - 1, 0), Lx)
    f = np.broadcast_to(np.asarray(h, dtype=np.float64), s.shape).copy()
    if Lx > 1:
        f[:, :, :-1] += Jh[None] * s[:, :, 1:]     # right neighbour
        f[:, :, 1:] += Jh[None] * s[:, :, :-1]     # left neighbour
    if Ly > 1:
        f[:, :-1, :] += Jv[None] * s[:, 1:, :]     # neighbour below
        f[:, 1:, :] += Jv[None] * s[:, :-1, :]     # neighbour above
    return f


def metropolis_sweeps(Jh, Jv, h, beta, spins, seed, sweep_offset, sweeps, chain_ids):
    """`sweeps` checkerboard single-spin-flip Metropolis sweeps of each chain (the sweeps
    the paper intersperses between proposals, Sec. 3 "Equilibration").

    A sweep updates the sites with (r + c) even, then those with (r + c) odd; sites of
    one colour have no bond between them, so each is updated against the current
    values of the other colour.  Site i of chain `chain_ids[b]` in sweep
    sweep_offset + k flips iff u < exp(-beta dE), dE = 2 s_i (h_i + sum_j J_ij s_j),
    with u = philox.sweep_uniform(seed, i, chain, sweep).  Returns the new spins.
    """
    s = np.array(spins, dtype=np.int8, copy=True)
    C, Ly, Lx = s.shape
    chain_ids = np.asarray(chain_ids, dtype=np.uint64)
    rr, cc = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    site = (rr * Lx + cc).astype(np.uint64)
    for k in range(sweeps):
        sw = np.uint64((sweep_offset + k) & 0xFFFFFFFF)
        for colour in (0, 1):
            mask = ((rr + cc) & 1) == colour
            dE = 2.0 * s.astype(np.float64) * local_field(Jh, Jv, h, s)
            u = philox.sweep_uniform(seed, site[None, :, :], chain_ids[:, None, None], sw)
            with np.errstate(over="ignore"):
                flip = (u < np.exp(-beta * dE)) & mask[None]
            s = np.where(flip, -s, s).astype(np.int8)
    return s


def link_overlap(Jh, Jv, spins_a, spins_b):
    """sum over the bonds <ij> of s_i^a s_j^a s_i^b s_j^b for each replica pair (a, b)
    (the link overlap of Sec. 3, eq. Delta, for one pair of configurations).  Only the
    lattice's bonds count; J enters only through which bonds exist (all of them)."""
    a = np.asarray(spins_a, dtype=np.int64)
    b = np.asarray(spins_b, dtype=np.int64)
    q = np.zeros(a.shape[0])
    if a.shape[2] > 1:
        q += (a[:, :, :-1] * a[:, :, 1:] * b[:, :, :-1] * b[:, :, 1:]).sum(axis=(1, 2))
    if a.shape[1] > 1:
        q += (a[:, :-1, :] * a[:, 1:, :] * b[:, :-1, :] * b[:, 1:, :]).sum(axis=(1, 2))
    return q


def n_bonds(Lx, Ly):
    """|E| of the open-boundary Ly x Lx lattice."""
    return Ly * (Lx - 1) + (Ly - 1) * Lx


def delta_instance(beta, Lx, Ly, mean_energy, mean_link_overlap):
    """(1/|V|) <H> + (beta/|V|) (|E| - sum_<ij> <s_i s_j>^2) of one instance (Sec. 3, eq.
    Delta before the disorder average), from a thermal estimate of <H> and of the link
    overlap (the mean over replica pairs of link_overlap, which estimates sum <s_i s_j>^2)."""
    return (mean_energy + beta * (n_bonds(Lx, Ly) - mean_link_overlap)) / (Lx * Ly)


def delta_from_chains(beta, Lx, Ly, chain_spins, chain_energy):
    """delta_instance from the C chains of one instance: <H> is the mean of their energies,
    the link overlap the mean over the replica pairs (2k, 2k + 1)."""
    sp = np.asarray(chain_spins)
    q = link_overlap(None, None, sp[0::2], sp[1::2])
    return delta_instance(beta, Lx, Ly, float(np.mean(chain_energy)), float(np.mean(q)))


# ---- arbitrary boundary conditions by frozen lines (App. B) ----

def energy_periodic(Jh, Jv, h, spins, px, py):
    """H of eq. ising on an Ly x Lx lattice that may close in x (px) and/or y (py):
    Jh [Ly, Lx] bond (r, c)-(r, c+1 mod Lx) (the last column used only when px),
    Jv [Ly, Lx] bond (r, c)-(r+1 mod Ly, c) (the last row used only when py)."""
    s = np.asarray(spins, dtype=np.float64)
    E = -(np.asarray(h)[None] * s).sum(axis=(1, 2))
    Lx = s.shape[2]
    Ly = s.shape[1]
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    E -= (Jh[None, :, :Lx - 1] * s[:, :, :-1] * s[:, :, 1:]).sum(axis=(1, 2))
    if px:
        E -= (Jh[None, :, Lx - 1] * s[:, :, -1] * s[:, :, 0]).sum(axis=1)
    E -= (Jv[None, :Ly - 1, :] * s[:, :-1, :] * s[:, 1:, :]).sum(axis=(1, 2))
    if py:
        E -= (Jv[None, Ly - 1, :] * s[:, -1, :] * s[:, 0, :]).sum(axis=1)
    return E


def frozen_cut(Jh, Jv, h, spins, kr, kc, px, py):
    """The open-boundary instance left when column kc (if px) and row kr (if py) are frozen
    (App. B): the free rows are kr+1, ..., kr-1 (mod Ly) when py (all rows otherwise), the
    free columns likewise, in that order.  Bonds between free sites keep their couplings;
    a bond from a free site to a frozen one becomes a field J s_frozen on the free site.
    Returns (rows, cols, Jh_eff [ly, lx-1], Jv_eff [ly-1, lx], h_eff [C, ly, lx])."""
    s = np.asarray(spins, dtype=np.float64)
    C, Ly, Lx = s.shape
    rows = [(kr + 1 + i) % Ly for i in range(Ly - 1)] if py else list(range(Ly))
    cols = [(kc + 1 + j) % Lx for j in range(Lx - 1)] if px else list(range(Lx))
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    ly, lx = len(rows), len(cols)
    Jh_e = np.array([[Jh[r, cols[j]] for j in range(lx - 1)] for r in rows]).reshape(ly, max(lx - 1, 0))
    Jv_e = np.array([[Jv[rows[i], c] for c in cols] for i in range(ly - 1)]).reshape(max(ly - 1, 0), lx)
    h_e = np.broadcast_to(h[np.ix_(rows, cols)], (C, ly, lx)).copy()
    frozen_c = {kc} if px else set()
    frozen_r = {kr} if py else set()
    for i, r in enumerate(rows):
        for j, c in enumerate(cols):
            # the four neighbours of (r, c) on the closed lattice; bonds to frozen sites
            nbrs = []
            if px or c + 1 < Lx:
                nbrs.append((r, (c + 1) % Lx, Jh[r, c]))
            if px or c > 0:
                nbrs.append((r, (c - 1) % Lx, Jh[r, (c - 1) % Lx]))
            if py or r + 1 < Ly:
                nbrs.append(((r + 1) % Ly, c, Jv[r, c]))
            if py or r > 0:
                nbrs.append(((r - 1) % Ly, c, Jv[(r - 1) % Ly, c]))
            for rn, cn, J in nbrs:
                if rn in frozen_r or cn in frozen_c:
                    h_e[:, i, j] += J * s[:, rn, cn]
    return rows, cols, Jh_e, Jv_e, h_e


def frozen_line_step(Jh, Jv, h, beta, chi, chains, kr, kc, px, py, seed, step, T, instance_offset=0):
    """One move of Markov chains on a closed lattice (App. B): freeze the line(s), build the
    environment of each chain's open instance (its frozen spins enter as fields), draw T
    proposals of the free spins from it and run the MH scan against the chain's current
    free spins (whose log q is evaluated under the same environment).  The frozen spins
    do not change, so the free spins' conditional law pi(free | frozen) is the Boltzmann
    weight of the open instance and the move keeps pi invariant.

    Chain i is instance j = instance_offset + i: its proposals use sample indices
    (j << 40) + step T + t and its MH uniforms the step offsets (j << 40) + step T (chain 0
    of the instance).  Returns
    (new chain spins [C, Ly, Lx], accepted [C, T])."""
    sp = np.array(chains, dtype=np.int8, copy=True)
    C = sp.shape[0]
    rows, cols, Jh_e, Jv_e, h_e = frozen_cut(Jh, Jv, h, sp, kr, kc, px, py)
    acc = np.zeros((C, T), dtype=bool)
    # chains with the same frozen spins have the same open instance, hence one environment
    groups = {}
    for i in range(C):
        groups.setdefault(h_e[i].tobytes(), []).append(i)
    for members in groups.values():
        idx = np.array(members)
        env = build_env(Jh_e, Jv_e, h_e[idx[0]], beta, chi)
        off = ((idx + instance_offset).astype(np.uint64) << np.uint64(40)) + np.uint64(step * T)   # per chain
        psp, plq, pE, _ = sample(env, idx.size * T, seed=seed,
                                 samples=(off[:, None] + np.arange(T, dtype=np.uint64)[None, :]).ravel())
        cur = sp[idx][:, rows][:, :, cols]
        _, lq, E, _ = logq(env, cur)
        # the MH scan of each chain over its T proposals (chain 0 of its own instance)
        for j in range(T):
            t = np.arange(idx.size) * T + j
            u = philox.mh_uniform(seed, off + np.uint64(j), 0)
            a = mh_accept(beta, plq[t], pE[t], lq, E, u)
            acc[idx, j] = a
            lq = np.where(a, plq[t], lq)
            E = np.where(a, pE[t], E)
            cur = np.where(a[:, None, None], psp[t], cur)
        for k, i in enumerate(idx):
            sp[i][np.ix_(rows, cols)] = cur[k]
    return sp, acc


# ---- the bond-basis gauge of App. A (a builder variant that changes q) ----

def vertical_split(J, beta):
    """W = B T for the vertical bond weight W[s, s'] = exp(beta J s s') (App. A: each W is
    split by its SVD into a factor for each end).  W is symmetric with eigenvectors
    u_0 = (1, 1)/sqrt 2 and u_1 = (1, -1)/sqrt 2 (index 0 <-> s = -1) and eigenvalues
    2 cosh(beta J), 2 sinh(beta J); B[s, rho] = u_rho(s) sqrt|lambda_rho| and
    T[rho, s'] = sign(lambda_rho) sqrt|lambda_rho| u_rho(s').  Returns (B, T)."""
    lam = np.array([2.0 * math.cosh(beta * J), 2.0 * math.sinh(beta * J)])
    U = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)       # U[s, rho]
    root = np.sqrt(np.abs(lam))
    B = U * root[None, :]
    T = (np.sign(lam) * root)[:, None] * U.T
    return B, T


def row_tensors_bond(envb_next, Jh, Jv, h, beta, r):
    """D_r H_r V'_r env'_{r+1}: row r's site tensors (physical index: row r's spins) with the
    lower factor B of each vertical bond (r, r+1) applied to the bond-basis boundary MPS
    env'_{r+1} (physical index: the vertical bond).  Same index layout as apply_row_mpo."""
    Ly, Lx = h.shape
    P = []
    for c in range(Lx):
        if envb_next is None:
            t = np.ones((1, 2, 1))
        else:
            Bv, _ = vertical_split(Jv[r, c], beta)
            t = np.einsum("sp,apb->asb", Bv, envb_next[c])
        t = t * np.exp(beta * h[r, c] * SPIN)[None, :, None]
        Dl, _, Dr = t.shape
        if c > 0:
            G = np.exp(beta * Jh[r, c - 1] * np.outer(SPIN, SPIN))
            t = np.einsum("asb,ks->aksb", t, G).reshape(Dl * 2, 2, Dr)
            Dl *= 2
        if c < Lx - 1:
            t2 = np.zeros((Dl, 2, Dr, 2))
            for s in range(2):
                t2[:, s, :, s] = t[:, s, :]
            t = t2.reshape(Dl, 2, Dr * 2)
        P.append(t)
    return P


def build_env_bond(Jh, Jv, h, beta, chi):
    """Environments in the bond-basis gauge (App. A, eqs. pf_bond_description to
    pf_vertex_description): the boundary MPS carries the vertical bond indices, is built
    bottom-up as env'_r = T_chi[ T_{r-1} D_r H_r V'_r env'_{r+1} ] (T_{r-1}: the upper factor
    of the bonds between rows r-1 and r, applied on the physical leg before truncating),
    and row r is sampled from the untruncated M'_r = D_r H_r V'_r env'_{r+1} (bond up to 2 chi;
    the rows above enter through W(s_up, s) = sum_rho B(s_up, rho) T(rho, s) = f(s), as in the
    spin basis).  env.M holds the M'_r; log Z~ = sum_{r >= 1} log_scale[r] + log of the
    contraction of M'_0 over row 0's spins."""
    Jh, Jv, h, Lx, Ly = _check_lattice(Jh, Jv, h)
    env = Env(Lx, Ly, float(beta), int(chi), Jh, Jv, h)
    nxt = None
    for r in range(Ly - 1, -1, -1):
        P = row_tensors_bond(nxt, Jh, Jv, h, beta, r)
        env.M[r] = P
        if r > 0:
            X = []
            for c in range(Lx):
                _, Tv = vertical_split(Jv[r - 1, c], beta)
                X.append(np.einsum("ps,asb->apb", Tv, P[c]))
            nxt, env.log_scale[r] = truncate_row(X, chi, Lx, Ly, r, env)
    v = np.ones(1)
    logv = 0.0
    for c in range(Lx):
        v = v @ (env.M[0][c][:, 0, :] + env.M[0][c][:, 1, :])
        m = np.abs(v).max()
        if m > 0:
            v = v / m
            logv += math.log(m)
    env.logZ = float(np.sum(env.log_scale[1:])) + logv + math.log(v[0]) if v[0] > 0 else float("nan")
    return env


# ---- two-site variational compression (App. A: the alternative to successive SVD) ----

def _left_overlap(Lenv, Y, X):
    """<Y_0..Y_c | X_0..X_c> from <Y_0..Y_{c-1} | X_0..X_{c-1}>: [ay, ax] -> [by, bx]."""
    return np.einsum("ab,asc,bsd->cd", Lenv, Y, X)


def _right_overlap(Renv, Y, X):
    """<Y_c.. | X_c..> from <Y_{c+1}.. | X_{c+1}..>: [by, bx] -> [ay, ax]."""
    return np.einsum("asc,bsd,cd->ab", Y, X, Renv)


def _rescaled(T):
    m = float(np.abs(T).max())
    if not m > 0:
        raise FloatingPointError("zero overlap environment")
    return T / m, math.log(m)


def truncate_row_variational(P, chi, Lx, Ly, r, sweeps, env=None):
    """T_chi by two-site variational compression (App. A names it beside successive SVD).

    The row X = P (the exact MPO-MPS product) is approximated by an MPS Y with the
    static bond dims of bond_dim().  Start: the successive-SVD result (truncate_row).
    Then `sweeps` rounds, each a left-to-right and a right-to-left pass over the
    neighbour pairs (c, c+1).  At a pair, the sites outside it are isometries
    (left-orthonormal left of c, right-orthonormal right of c+1), so the Y closest
    to X in 2-norm with those sites fixed has the two-site tensor
        Theta = <Y_<c| X_c X_{c+1} |Y_>c+1>   (overlap environments, exact),
    and the best one of rank <= k at bond c+1 is its truncated SVD
    (Eckart-Young).  Going right, Y_c = U (left-orthonormal) and Y_{c+1} = S V^T;
    going left, Y_{c+1} = V^T and Y_c = U S.  No update increases ||X - Y||.

    The singular-value record of a bond is that of its last update (the final
    right-to-left pass).  Returns (tensors, log of the removed scale) like
    truncate_row: Y_0 carries unit norm, the other sites are right-orthonormal."""
    Y, logs = truncate_row(P, chi, Lx, Ly, r, env)
    if Lx < 2 or sweeps <= 0:
        return Y, logs
    X = list(P)
    # right environments of the start (Y_1.. right-orthonormal); log scales kept apart
    R = [None] * (Lx + 1)
    lR = np.zeros(Lx + 1)
    R[Lx] = np.ones((1, 1))
    for c in range(Lx - 1, 1, -1):
        R[c], s = _rescaled(_right_overlap(R[c + 1], Y[c], X[c]))
        lR[c] = lR[c + 1] + s
    L = [None] * (Lx + 1)
    lL = np.zeros(Lx + 1)
    L[0] = np.ones((1, 1))

    def theta(c):
        T = np.einsum("ab,bsx,xtd,ed->aste", L[c], X[c], X[c + 1], R[c + 2])
        a, _, _, e = T.shape
        return T.reshape(a * 2, 2 * e), a, e

    def split(c, going_right):
        Th, a, e = theta(c)
        U, S, Vh = np.linalg.svd(Th, full_matrices=False)
        k = bond_dim(chi, Lx, Ly, r, c + 1)
        if not S[0] > 0:
            raise FloatingPointError("row %d: zero environment" % r)
        if env is not None and not going_right:
            tot = float(np.sum(S * S))
            env.sv[(r, c + 1)] = S[:k] / math.sqrt(tot)
            env.discarded[(r, c + 1)] = float(np.sum(S[k:] ** 2)) / tot
        if going_right:
            Y[c] = U[:, :k].reshape(a, 2, k)
            Y[c + 1] = (S[:k, None] * Vh[:k]).reshape(k, 2, e)
        else:
            Y[c] = (U[:, :k] * S[None, :k]).reshape(a, 2, k)
            Y[c + 1] = Vh[:k].reshape(k, 2, e)
        return S[:k]

    for _ in range(sweeps):
        for c in range(Lx - 1):
            split(c, True)
            if c + 1 < Lx - 1:
                L[c + 1], s = _rescaled(_left_overlap(L[c], Y[c], X[c]))
                lL[c + 1] = lL[c] + s
        for c in range(Lx - 2, -1, -1):
            S = split(c, False)
            if c > 0:
                R[c + 1], s = _rescaled(_right_overlap(R[c + 2], Y[c + 1], X[c + 1]))
                lR[c + 1] = lR[c + 2] + s
    # Y_0 = U S: its norm is ||S_k||, the overlap scale is e^{lL[0] + lR[2]} = e^{lR[2]}
    n0 = float(np.linalg.norm(S))
    Y[0] = Y[0] / n0
    return Y, float(lR[2] + math.log(n0))


def build_env_variational(Jh, Jv, h, beta, chi, sweeps=1):
    """Row environments compressed by two-site variational sweeps (truncate_row_variational)
    instead of successive SVD; everything else as build_env."""
    Jh, Jv, h, Lx, Ly = _check_lattice(Jh, Jv, h)
    env = Env(Lx, Ly, float(beta), int(chi), Jh, Jv, h)
    nxt = None
    for r in range(Ly - 1, -1, -1):
        P = apply_row_mpo(nxt, Jh, Jv, h, beta, r)
        env.M[r], env.log_scale[r] = truncate_row_variational(P, chi, Lx, Ly, r, sweeps, env)
        env.log_lambda[r] = env.log_lambda[r + 1] + env.log_scale[r]
        nxt = env.M[r]
    v = np.ones(1)
    logv = 0.0
    for c in range(Lx):
        v = v @ (env.M[0][c][:, 0, :] + env.M[0][c][:, 1, :])
        m = np.abs(v).max()
        if m > 0:
            v = v / m
            logv += math.log(m)
    env.logZ = env.log_lambda[0] + logv + math.log(v[0]) if v[0] > 0 else float("nan")
    return env
