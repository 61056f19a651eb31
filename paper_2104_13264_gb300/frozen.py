"""Markov chains on closed lattices (cylinder, torus) with the open-boundary move (App. B).

A move freezes a line of spins: column kc when the lattice closes in x, row kr when
it closes in y.  What remains is an open lattice whose edge sites feel the frozen
spins through the cut bonds, as fields J s_frozen.  Its Boltzmann weight is the
conditional law pi(free | frozen), so a TNMH move on it (build the environment, draw
proposals of the free spins, MH against the chain's current free spins) keeps pi
invariant.  The frozen line moves from one iteration to the next (random cuts by
default), so every spin is refreshed.

Each chain has its own frozen spins, hence its own open instance and environment.
One iteration therefore builds one environment per chain in a single batched builder
launch, draws every chain's proposals in one persistent launch, evaluates the current
free spins in forced mode and runs the MH scan -- all in the library's kernels; the
open instances (couplings and fields) are assembled here from the chain spins.

Couplings of the closed lattice: Jh [Ly, Lx] bond (r, c)-(r, c+1 mod Lx), Jv [Ly, Lx]
bond (r, c)-(r+1 mod Ly, c), h [Ly, Lx]; the wrap-around entries (last column of Jh,
last row of Jv) are used only in a closed direction.
"""
import numpy as np

from . import binding
from .instances import Instance


def open_instances(Jh, Jv, h, spins, kr, kc, px, py):
    """The open instances of a batch of configurations [C, Ly, Lx] with row kr frozen (if
    py) and column kc frozen (if px).  Free rows are kr+1, ..., kr-1 (mod Ly), free columns
    likewise.  Returns (rows, cols, Jh_o [ly, lx-1], Jv_o [ly-1, lx], h_o [C, ly, lx])."""
    s = np.asarray(spins, dtype=np.float64)
    C, Ly, Lx = s.shape
    Jh = np.asarray(Jh, dtype=np.float64)
    Jv = np.asarray(Jv, dtype=np.float64)
    rows = (kr + 1 + np.arange(Ly - 1)) % Ly if py else np.arange(Ly)
    cols = (kc + 1 + np.arange(Lx - 1)) % Lx if px else np.arange(Lx)
    Jh_o = Jh[np.ix_(rows, cols[:-1])]                 # bond (r, cols[j]) - (r, cols[j] + 1)
    Jv_o = Jv[np.ix_(rows[:-1], cols)]
    h_o = np.repeat(np.asarray(h, dtype=np.float64)[np.ix_(rows, cols)][None], C, axis=0)
    if px:
        # the frozen column kc sits left of cols[0] = kc + 1 and right of cols[-1] = kc - 1
        h_o[:, :, 0] += Jh[rows, kc][None] * s[:, rows, kc]
        h_o[:, :, -1] += Jh[rows, (kc - 1) % Lx][None] * s[:, rows, kc]
    if py:
        h_o[:, 0, :] += Jv[kr, cols][None] * s[:, kr][:, cols]
        h_o[:, -1, :] += Jv[(kr - 1) % Ly, cols][None] * s[:, kr][:, cols]
    return rows, cols, Jh_o, Jv_o, h_o


class FrozenLineChains:
    """Markov chains of the Boltzmann distributions of D closed lattices (disorder samples
    sharing a shape), C chains each, advanced by frozen-line TNMH moves with T proposals
    per chain and move (sampler arithmetic `precision`).  Jh, Jv, h are [Ly, Lx] arrays or
    [D, Ly, Lx] stacks, beta a scalar or [D]; `start` (int8 [C, Ly, Lx] or [D, C, Ly, Lx])
    is the first state.  `spins` (device int8 [D, C, Ly, Lx]) holds the chain states.

    Chain c of disorder d is instance i = d C + c of each move's batched plan, so its
    proposals use sample indices (i << 40) + k T + t at move k, and its MH uniforms the
    step offsets (i << 40) + k T."""

    def __init__(self, Jh, Jv, h, beta, chi, start, px=True, py=True, precision="f64", proposals=1, seed=0):
        import torch
        self.Jh = np.asarray(Jh, dtype=np.float64)
        single = self.Jh.ndim == 2
        if single:
            self.Jh = self.Jh[None]
        self.Jv = np.asarray(Jv, dtype=np.float64).reshape(self.Jh.shape)
        self.h = np.asarray(h, dtype=np.float64).reshape(self.Jh.shape)
        self.D = self.Jh.shape[0]
        self.beta = np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.D,)).copy()
        self.chi = int(chi)
        self.px, self.py = bool(px), bool(py)
        self.precision, self.T, self.seed = precision, int(proposals), int(seed)
        st = torch.as_tensor(np.asarray(start), dtype=torch.int8)
        if st.dim() == 3:
            st = st[None]
        self.spins = st.to("cuda").contiguous()
        _, self.C, self.Ly, self.Lx = self.spins.shape
        self.k = 0

    def default_cut(self, k):
        """Uniformly random frozen lines for move k (seeded, reproducible)."""
        g = np.random.default_rng([self.seed, k, 13])
        return int(g.integers(self.Ly)), int(g.integers(self.Lx))

    def step(self, cut=None):
        """One move of every chain; returns the accept flags (uint8 cuda tensor [D, C, T])."""
        import torch
        kr, kc = self.default_cut(self.k) if cut is None else cut
        host = self.spins.cpu().numpy()
        insts, rows, cols = [], None, None
        for d in range(self.D):
            rows, cols, Jh_o, Jv_o, h_o = open_instances(self.Jh[d], self.Jv[d], self.h[d], host[d], kr, kc,
                                                         self.px, self.py)
            insts += [Instance("open", Jh_o, Jv_o, h_o[c], float(self.beta[d]), self.chi) for c in range(self.C)]
        envs = binding.build_envs_batched(insts, precisions=tuple(sorted({"f64", self.precision})))
        plan = binding.Batch(envs, self.T, chains=1, precision=self.precision, tile=64, order="instance")
        try:
            plan.set_step(self.seed, self.k)
            prop = plan.alloc_proposals()
            plan.sample(prop)
            r_t = torch.as_tensor(rows, device="cuda")
            c_t = torch.as_tensor(cols, device="cuda")
            n = self.D * self.C
            free = self.spins.view(n, self.Ly, self.Lx).index_select(1, r_t).index_select(2, c_t).contiguous()
            chain = (free.view(-1), torch.empty(n, dtype=torch.float64, device="cuda"),
                     torch.empty(n, dtype=torch.float64, device="cuda"))
            plan.metropolis(chain, 0)          # no sweep: the forced log q and energy of the free spins
            acc = torch.empty(n * self.T, dtype=torch.uint8, device="cuda")
            plan.mh(prop, chain, acc)
            new = chain[0].view(self.D, self.C, len(rows), len(cols))
            self.spins[:, :, r_t.view(-1, 1), c_t.view(1, -1)] = new
        finally:
            plan.free()
            for e in envs:
                e.free()
        self.k += 1
        return acc.view(self.D, self.C, self.T)

    def _bond_products(self, s):
        """s_i s_j over the bonds of the closed lattice: horizontal [.., Ly, Lx or Lx-1] and vertical."""
        hz = s * s.roll(-1, dims=-1) if self.px else s[..., :, :-1] * s[..., :, 1:]
        vt = s * s.roll(-1, dims=-2) if self.py else s[..., :-1, :] * s[..., 1:, :]
        return hz, vt

    def energy(self):
        """H of eq. ising on the closed lattices (float64 cuda tensor [D, C])."""
        import torch
        s = self.spins.double()
        Jh = torch.as_tensor(self.Jh, device="cuda")[:, None]
        Jv = torch.as_tensor(self.Jv, device="cuda")[:, None]
        hz, vt = self._bond_products(s)
        Jh = Jh if self.px else Jh[..., :, :-1]
        Jv = Jv if self.py else Jv[..., :-1, :]
        return (-(torch.as_tensor(self.h, device="cuda")[:, None] * s).sum(dim=(2, 3))
                - (Jh * hz).sum(dim=(2, 3)) - (Jv * vt).sum(dim=(2, 3)))

    def delta(self):
        """The equilibration diagnostic of Sec. 3 (eq. Delta) averaged over the disorder samples:
        (1/|V|)(<H> + beta (|E| - sum <s_i s_j>^2)) with the link overlap from replica pairs
        (2k, 2k+1); |E| counts the closed lattice's bonds.  Returns (mean, per disorder)."""
        import torch
        s = self.spins.double()
        hz, vt = self._bond_products(s)
        q = (hz[:, 0::2] * hz[:, 1::2]).sum(dim=(2, 3)) + (vt[:, 0::2] * vt[:, 1::2]).sum(dim=(2, 3))
        nb = hz[0, 0].numel() + vt[0, 0].numel()
        beta = torch.as_tensor(self.beta, device="cuda")
        d = (self.energy().mean(dim=1) + beta * (nb - q.mean(dim=1))) / (self.Lx * self.Ly)
        return float(d.mean().item()), d
