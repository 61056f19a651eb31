"""Plain FP64 oracle of TNMH on three-dimensional Ising lattices (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may use this module.
numpy loops over layers, rows and sites, vectorised over samples; numpy's QR, SVD and
einsum serve as library steps.

Sec. 3D and App. A (the three-dimensional paragraph, Figs. peps-cutoff2 and
peps-cutoff): the layer transfer operators are PEPOs, the boundary objects PEPS of
bond D, and each layer is sampled through a 2D contraction with boundary MPS of bond chi.

Conventions:
  lattice Lz x Ly x Lx, open boundaries, site (z, y, x); layer z = 0 is sampled first,
  each layer in raster order (rows y, then x);
  Jx[z, y, x] bond (z,y,x)-(z,y,x+1)  shape (Lz, Ly, Lx-1)
  Jy[z, y, x] bond (z,y,x)-(z,y+1,x)  shape (Lz, Ly-1, Lx)
  Jz[z, y, x] bond (z,y,x)-(z+1,y,x)  shape (Lz-1, Ly, Lx)
  h[z, y, x]                          shape (Lz, Ly, Lx)
  H = -sum h s - sum J s s; physical index 0 <-> s = -1, 1 <-> s = +1.
PEPS site tensors A[s, u, l, d, r]: u to row y-1, l to column x-1, d to row y+1, r to
column x+1 (dimension 1 on the open edges).

Layer environment (sample independent, bottom-up):
  env_{Lz-1} = the exact weight of layer Lz-1 (fields and in-layer bonds),
  env_z      = T_D[ D_z H_z V_z env_{z+1} ],
with V_z the sum over layer z+1 through W(s, s') = exp(beta Jz s s') (no bond growth),
D_z the fields, H_z the in-layer bonds as copy structure (each bond doubles: the spin of
the site on the left / above is carried along the bond and weighted at the other end),
and T_D the paper's renormalisation: every column is read as an MPS whose bonds are the
column's vertical bonds and whose physical index lumps the spin with the two horizontal
bonds, and compressed by successive SVD (QR sweep down, SVD sweep up keeping
min(D, rank bound) values); then every row likewise along its horizontal bonds.

Sampling layer z (per sample): with the spins of layer z-1 fixed, site (y, x) of layer z
carries the field factor f(s) = exp(beta Jz[z-1, y, x] s_{z-1,y,x} s).  The layer is
the 2D network of the tensors A f.  Row y is sampled from the sandwich
  Top_y (rows < y, spins fixed; MPS over row y's u-bonds, bond chi)
  x row y (tensors A f, spin open)
  x Bot_y (rows > y, spins summed; MPS over row y's d-bonds, bond chi),
  Bot_{Ly-1} = 1,  Bot_y = T_chi[ S_{y+1} Bot_{y+1} ],  S = sum_s A f,
  Top_0 = 1,       Top_{y+1} = T_chi[ Top_y F_y ],      F = A f at the drawn spins,
with T_chi successive SVD (QR sweep right, SVD sweep left).  Site conditionals are
normalised after clamping at zero, drawn with the Philox word of site
z Ly Lx + y Lx + x, as in two dimensions.  Without truncation (D and chi at the exact
ranks) q = pi.
"""
import math

import numpy as np

from . import philox
from .tnmc import threshold_plus, vertical_split, F_BAD

SPIN = np.array([-1.0, 1.0])


def check_lattice3d(Jx, Jy, Jz, h):
    h = np.asarray(h, dtype=np.float64)
    Lz, Ly, Lx = h.shape
    Jx = np.asarray(Jx, dtype=np.float64).reshape(Lz, Ly, max(Lx - 1, 0))
    Jy = np.asarray(Jy, dtype=np.float64).reshape(Lz, max(Ly - 1, 0), Lx)
    Jz = np.asarray(Jz, dtype=np.float64).reshape(max(Lz - 1, 0), Ly, Lx)
    return Jx, Jy, Jz, h, Lz, Ly, Lx


def energy3d(Jx, Jy, Jz, h, spins):
    """H (Sec. 2, eq. ising on the cubic lattice) of configurations [B, Lz, Ly, Lx]."""
    Jx, Jy, Jz, h, Lz, Ly, Lx = check_lattice3d(Jx, Jy, Jz, h)
    s = np.asarray(spins, dtype=np.float64)
    E = -(h[None] * s).sum(axis=(1, 2, 3))
    E -= (Jx[None] * s[..., :-1] * s[..., 1:]).sum(axis=(1, 2, 3))
    E -= (Jy[None] * s[:, :, :-1, :] * s[:, :, 1:, :]).sum(axis=(1, 2, 3))
    E -= (Jz[None] * s[:, :-1] * s[:, 1:]).sum(axis=(1, 2, 3))
    return E


class Env3D:
    """Layer environments A[z][y][x] (arrays [2, Du, Dl, Dd, Dr]) and their log-scales."""

    def __init__(self, Jx, Jy, Jz, h, beta, D, chi):
        self.Jx, self.Jy, self.Jz, self.h = Jx, Jy, Jz, h
        self.Lz, self.Ly, self.Lx = h.shape
        self.beta, self.D, self.chi = float(beta), int(D), int(chi)
        self.A = [None] * self.Lz
        self.log_scale = np.zeros(self.Lz)


def layer_tensors(env_next, Jx, Jy, Jz, h, beta, z, gauge="spin"):
    """D_z H_z V_z env_{z+1} as PEPS tensors [2, Du, Dl, Dd, Dr] (in-layer bonds doubled).
    gauge "bond": env_{z+1} carries the index rho of the vertical bonds (z, z+1), and V'_z
    applies their lower factor B (vertical_split) instead of summing over layer z+1."""
    _, Ly, Lx = h.shape
    out = [[None] * Lx for _ in range(Ly)]
    for y in range(Ly):
        for x in range(Lx):
            if env_next is None:
                t = np.ones((2, 1, 1, 1, 1))
            elif gauge == "bond":
                Bv, _ = vertical_split(Jz[z, y, x], beta)                   # B[s, rho]
                t = np.einsum("sp,puldr->suldr", Bv, env_next[y][x])
            else:
                W = np.exp(beta * Jz[z, y, x] * np.outer(SPIN, SPIN))        # W[s, s']
                t = np.einsum("ts,suldr->tuldr", W, env_next[y][x])
            t = t * np.exp(beta * h[z, y, x] * SPIN)[:, None, None, None, None]
            _, Du, Dl, Dd, Dr = t.shape
            if y > 0:      # weight of the bond to (y-1, x): its spin k arrives on the u-bond
                G = np.exp(beta * Jy[z, y - 1, x] * np.outer(SPIN, SPIN))   # G[k, s]
                t = np.einsum("suldr,ks->sukldr", t, G).reshape(2, Du * 2, Dl, Dd, Dr)
                Du *= 2
            if x > 0:      # weight of the bond to (y, x-1)
                G = np.exp(beta * Jx[z, y, x - 1] * np.outer(SPIN, SPIN))
                t = np.einsum("suldr,ks->sulkdr", t, G).reshape(2, Du, Dl * 2, Dd, Dr)
                Dl *= 2
            if y < Ly - 1:  # copy the spin onto the d-bond
                t2 = np.zeros((2, Du, Dl, Dd, 2, Dr))
                for s in range(2):
                    t2[s, :, :, :, s, :] = t[s]
                t = t2.reshape(2, Du, Dl, Dd * 2, Dr)
                Dd *= 2
            if x < Lx - 1:  # copy the spin onto the r-bond
                t2 = np.zeros((2, Du, Dl, Dd, Dr, 2))
                for s in range(2):
                    t2[s, :, :, :, :, s] = t[s]
                t = t2.reshape(2, Du, Dl, Dd, Dr * 2)
            out[y][x] = t
    return out


def mps_successive_svd(M, k_max):
    """Successive SVD of an MPS M[i] [Dl, p_i, Dr] (App. A): QR sweep left to right, then
    SVD sweep right to left keeping min(k_max, rank bound) values per bond.  Returns
    (tensors, log of the removed scale); site 0 is left with unit norm."""
    M = list(M)
    n = len(M)
    logs = 0.0
    for i in range(n - 1):
        Dl, p, Dr = M[i].shape
        Q, R = np.linalg.qr(M[i].reshape(Dl * p, Dr))
        M[i] = Q.reshape(Dl, p, Q.shape[1])
        sc = np.abs(R).max()
        if not sc > 0:
            raise FloatingPointError("zero MPS")
        logs += math.log(sc)
        M[i + 1] = np.einsum("ij,jsk->isk", R / sc, M[i + 1])
    for i in range(n - 1, 0, -1):
        Dl, p, Dr = M[i].shape
        U, S, Vh = np.linalg.svd(M[i].reshape(Dl, p * Dr), full_matrices=False)
        k = min(k_max, S.size)
        if not S[0] > 0:
            raise FloatingPointError("zero MPS")
        M[i] = Vh[:k].reshape(k, p, Dr)
        logs += math.log(S[0])
        M[i - 1] = np.einsum("isj,jk->isk", M[i - 1], U[:, :k] * (S[:k] / S[0]))
    n0 = float(np.linalg.norm(M[0]))
    if not n0 > 0:
        raise FloatingPointError("zero MPS")
    M[0] = M[0] / n0
    return M, logs + math.log(n0)


def compress_peps(A, D):
    """T_D of App. A (Fig. peps-cutoff2): columns first (vertical bonds; physical index
    (s, l, r)), then rows (horizontal bonds; physical index (s, u, d)).  Returns (A, log)."""
    Ly, Lx = len(A), len(A[0])
    A = [list(row) for row in A]
    logs = 0.0
    for x in range(Lx):
        col = []
        for y in range(Ly):
            t = A[y][x]                                   # [s, u, l, d, r]
            _, Du, Dl, Dd, Dr = t.shape
            col.append(t.transpose(1, 0, 2, 4, 3).reshape(Du, 2 * Dl * Dr, Dd))
        col, l = mps_successive_svd(col, D)
        logs += l
        for y in range(Ly):
            _, Du, Dl, Dd, Dr = A[y][x].shape
            m = col[y]
            A[y][x] = m.reshape(m.shape[0], 2, Dl, Dr, m.shape[2]).transpose(1, 0, 2, 4, 3)
    for y in range(Ly):
        row = []
        for x in range(Lx):
            t = A[y][x]
            _, Du, Dl, Dd, Dr = t.shape
            row.append(t.transpose(2, 0, 1, 3, 4).reshape(Dl, 2 * Du * Dd, Dr))
        row, l = mps_successive_svd(row, D)
        logs += l
        for x in range(Lx):
            _, Du, Dl, Dd, Dr = A[y][x].shape
            m = row[x]
            A[y][x] = m.reshape(m.shape[0], 2, Du, Dd, m.shape[2]).transpose(1, 2, 0, 3, 4)
    return A, logs


def build_env3d(Jx, Jy, Jz, h, beta, D, chi):
    """All layer environments, bottom-up (App. A, three-dimensional paragraph)."""
    Jx, Jy, Jz, h, Lz, Ly, Lx = check_lattice3d(Jx, Jy, Jz, h)
    env = Env3D(Jx, Jy, Jz, h, beta, D, chi)
    nxt = None
    for z in range(Lz - 1, -1, -1):
        A = layer_tensors(nxt, Jx, Jy, Jz, h, beta, z)
        env.A[z], env.log_scale[z] = compress_peps(A, D)
        nxt = env.A[z]
    return env


def build_env3d_bond(Jx, Jy, Jz, h, beta, D, chi):
    """Layer environments in the bond basis (App. A: vertex tensors from split bond weights;
    in three dimensions the vertical bonds are split as W = B T like the 2D bond gauge).
    env'_z carries the index rho of the vertical bonds (z-1, z):
        env'_z = T_D[ T_{z-1} D_z H_z V'_z env'_{z+1} ]   (V' applies B, T the upper factor),
    and layer z is sampled from the uncompressed PEPS M'_z = D_z H_z V'_z env'_{z+1} of its
    own spins (in-layer bonds up to 2D); the layer above enters through the same fields
    f(s) = W(s_up, s).  env.A[z] holds the M'_z, which run3d samples unchanged."""
    Jx, Jy, Jz, h, Lz, Ly, Lx = check_lattice3d(Jx, Jy, Jz, h)
    env = Env3D(Jx, Jy, Jz, h, beta, D, chi)
    nxt = None
    for z in range(Lz - 1, -1, -1):
        M = layer_tensors(nxt, Jx, Jy, Jz, h, beta, z, gauge="bond")
        env.A[z] = M
        if z > 0:
            X = [[None] * Lx for _ in range(Ly)]
            for y in range(Ly):
                for x in range(Lx):
                    _, Tv = vertical_split(Jz[z - 1, y, x], beta)         # T[rho, s]
                    X[y][x] = np.einsum("ps,suldr->puldr", Tv, M[y][x])
            nxt, env.log_scale[z] = compress_peps(X, D)
    return env


def _batched_successive_svd(M, k_max):
    """mps_successive_svd on a batch: M[i] [B, Dl, p, Dr]; the overall scale is dropped
    (boundaries only enter ratios)."""
    M = list(M)
    n = len(M)
    for i in range(n - 1):
        B, Dl, p, Dr = M[i].shape
        Q, R = np.linalg.qr(M[i].reshape(B, Dl * p, Dr))
        M[i] = Q.reshape(B, Dl, p, Q.shape[2])
        sc = np.abs(R).max(axis=(1, 2))
        sc = np.where(sc > 0, sc, 1.0)
        M[i + 1] = np.einsum("bij,bjsk->bisk", R / sc[:, None, None], M[i + 1])
    for i in range(n - 1, 0, -1):
        B, Dl, p, Dr = M[i].shape
        U, S, Vh = np.linalg.svd(M[i].reshape(B, Dl, p * Dr), full_matrices=False)
        k = min(k_max, S.shape[1])
        M[i] = Vh[:, :k].reshape(B, k, p, Dr)
        s0 = np.where(S[:, 0] > 0, S[:, 0], 1.0)
        M[i - 1] = np.einsum("bisj,bjk->bisk", M[i - 1], U[:, :, :k] * (S[:, None, :k] / s0[:, None, None]))
    n0 = np.sqrt((M[0] ** 2).sum(axis=(1, 2, 3)))
    M[0] = M[0] / np.where(n0 > 0, n0, 1.0)[:, None, None, None]
    return M


def _rescale_vec(v):
    m = np.abs(v).max(axis=1)
    return v / np.where(m > 0, m, 1.0)[:, None]


def run3d(env, B, seed=0, sample_offset=0, forced=None, samples=None):
    """Sequential sampler (forced=None) or evaluator (forced spins [B, Lz, Ly, Lx]).
    Returns (spins int8 [B, Lz, Ly, Lx], logq [B], energy [B], flags [B]); a site with a
    non-positive or non-finite normaliser is drawn with p = 1/2 and flags its sample."""
    Lz, Ly, Lx, beta, chi = env.Lz, env.Ly, env.Lx, env.beta, env.chi
    spins = np.zeros((B, Lz, Ly, Lx), dtype=np.int8) if forced is None else np.array(forced, dtype=np.int8)
    logq = np.zeros(B)
    flags = np.zeros(B, dtype=np.int32)
    if samples is None:
        samples = np.uint64(sample_offset) + np.arange(B, dtype=np.uint64)
    else:
        samples = np.asarray(samples, dtype=np.uint64)
    ar = np.arange(B)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        for z in range(Lz):
            A = env.A[z]
            # field factors f[b, y, x, s] from the fixed layer above
            if z > 0:
                up = spins[:, z - 1].astype(np.float64)
                f = np.exp(beta * env.Jz[z - 1][None, :, :, None] * up[..., None] * SPIN[None, None, None, :])
            else:
                f = np.ones((B, Ly, Lx, 2))
            # bottom boundaries Bot[y][x] [B, bl, d, br] over row y's d-bonds
            Bot = [None] * Ly
            Bot[Ly - 1] = [np.ones((B, 1, 1, 1)) for _ in range(Lx)]
            for y in range(Ly - 2, -1, -1):
                M = []
                for x in range(Lx):
                    S = np.einsum("suldr,bs->buldr", A[y + 1][x], f[:, y + 1, x])
                    # contract S's d-bond with Bot[y+1][x] [B, bl, d, br]
                    N = np.einsum("buldr,bpdq->blpurq", S, Bot[y + 1][x])
                    Bq, Dl, Pl, Du, Dr, Pr = N.shape
                    M.append(N.reshape(Bq, Dl * Pl, Du, Dr * Pr))
                Bot[y] = _batched_successive_svd(M, chi)
            Top = [np.ones((B, 1, 1, 1)) for _ in range(Lx)]       # [B, tl, u, tr]
            for y in range(Ly):
                # sandwich tensors per site and spin: Q[x][s] [B, (tl,l,bl), (tr,r,br)]
                Q = []
                for x in range(Lx):
                    Af = np.einsum("suldr,bs->bsuldr", A[y][x], f[:, y, x])
                    T1 = np.einsum("bauc,bsuldr->bsacldr", Top[x], Af)
                    T2 = np.einsum("bsacldr,bpdq->bsalpcrq", T1, Bot[y][x])
                    Bq, _, a, l, p, c, r, q = T2.shape
                    Q.append(T2.reshape(Bq, 2, a * l * p, c * r * q))
                R = [None] * (Lx + 1)
                R[Lx] = np.ones((B, 1))
                for x in range(Lx - 1, 0, -1):
                    R[x] = _rescale_vec(np.einsum("bsij,bj->bi", Q[x], R[x + 1]))
                Lam = np.ones((B, 1))
                for x in range(Lx):
                    w = np.einsum("bi,bsij,bj->bs", Lam, Q[x], R[x + 1])
                    w = np.maximum(w, 0.0)
                    tot = w[:, 0] + w[:, 1]
                    bad = ~(tot > 0) | ~np.isfinite(tot)
                    pplus = np.where(bad, 0.5, w[:, 1] / tot)
                    pminus = np.where(bad, 0.5, w[:, 0] / tot)
                    if forced is None:
                        xw = philox.draw_words(seed, z * Ly * Lx + y * Lx + x, samples)
                        plus = threshold_plus(pplus, xw)
                        spins[:, z, y, x] = np.where(plus, 1, -1)
                    else:
                        plus = spins[:, z, y, x] > 0
                    logq += np.log(np.where(plus, pplus, pminus))
                    flags |= np.where(bad, F_BAD, 0).astype(np.int32)
                    Lam = _rescale_vec(np.einsum("bi,bij->bj", Lam, Q[x][ar, plus.astype(np.int64)]))
                if y < Ly - 1:
                    M = []
                    for x in range(Lx):
                        idx = (spins[:, z, y, x] > 0).astype(np.int64)
                        F = A[y][x][idx] * f[ar, y, x, idx][:, None, None, None, None]     # [B, u, l, d, r]
                        N = np.einsum("bauc,buldr->baldcr", Top[x], F)
                        Bq, a, l, d, c, r = N.shape
                        M.append(N.reshape(Bq, a * l, d, c * r))
                    Top = _batched_successive_svd(M, chi)
    E = energy3d(env.Jx, env.Jy, env.Jz, env.h, spins)
    return spins, logq, E, flags


def sample3d(env, B, seed=0, sample_offset=0, samples=None):
    """Draw B proposals from the 3D q (Sec. 3D)."""
    return run3d(env, B, seed, sample_offset, samples=samples)


def logq3d(env, spins):
    """Forced evaluation of log q for given configurations."""
    s = np.asarray(spins, dtype=np.int8)
    return run3d(env, s.shape[0], forced=s)
