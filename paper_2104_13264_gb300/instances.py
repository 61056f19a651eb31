"""Seeded synthetic Ising instances (inputs only; none of the method's arithmetic).

The paper's instances are themselves synthetic (Sec. 3, "Models"): the
ferromagnet, +-J and Gaussian Edwards-Anderson spin glasses and the fully
frustrated (Villain) model on open-boundary square lattices.  Couplings are
drawn with numpy's PCG64 generator from a seed; this module is shared by the
tests, the benchmark and the oracle checks and computes nothing else.

Layout: Jh [Ly, Lx-1] (bond (r,c)-(r,c+1)), Jv [Ly-1, Lx] (bond (r,c)-(r+1,c)),
h [Ly, Lx], all float64.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    name: str
    Jh: np.ndarray
    Jv: np.ndarray
    h: np.ndarray
    beta: float
    chi: int
    meta: dict = field(default_factory=dict)

    @property
    def Ly(self):
        return self.h.shape[0]

    @property
    def Lx(self):
        return self.h.shape[1]

    @property
    def integer_couplings(self):
        return all(np.array_equal(a, np.round(a)) for a in (self.Jh, self.Jv, self.h))


def _zeros(Ly, Lx):
    return (np.zeros((Ly, max(Lx - 1, 0))), np.zeros((max(Ly - 1, 0), Lx)), np.zeros((Ly, Lx)))


def ferromagnet(Ly, Lx, beta, chi, J=1.0, hfield=0.0):
    """Uniform ferromagnet (J > 0) or antiferromagnet (J < 0) with a uniform field."""
    Jh, Jv, h = _zeros(Ly, Lx)
    return Instance("ferro", Jh + J, Jv + J, h + hfield, float(beta), int(chi))


def ea_pm(Ly, Lx, beta, chi, seed=0, p=0.5):
    """Edwards-Anderson +-J couplings, J = +1 with probability p."""
    rng = np.random.default_rng([seed, 3])
    Jh, Jv, h = _zeros(Ly, Lx)
    Jh = np.where(rng.random(Jh.shape) < p, 1.0, -1.0)
    Jv = np.where(rng.random(Jv.shape) < p, 1.0, -1.0)
    return Instance("ea_pm", Jh, Jv, h, float(beta), int(chi), {"seed": seed})


def ea_gauss(Ly, Lx, beta, chi, seed=0, float32=True, hscale=0.0):
    """Gaussian N(0,1) Edwards-Anderson couplings (drawn in float32, widened exactly)."""
    rng = np.random.default_rng([seed, 5])
    Jh, Jv, h = _zeros(Ly, Lx)
    dt = np.float32 if float32 else np.float64
    Jh = rng.standard_normal(Jh.shape).astype(dt).astype(np.float64)
    Jv = rng.standard_normal(Jv.shape).astype(dt).astype(np.float64)
    if hscale:
        h = (hscale * rng.standard_normal(h.shape)).astype(dt).astype(np.float64)
    return Instance("ea_gauss", Jh, Jv, h, float(beta), int(chi), {"seed": seed})


def villain(Ly, Lx, beta, chi):
    """Fully frustrated model: every bond +1 except vertical bonds in odd columns (-1).

    Each plaquette then holds exactly one antiferromagnetic bond (Sec. 3,
    fully frustrated case J' = J).
    """
    Jh, Jv, h = _zeros(Ly, Lx)
    Jh = Jh + 1.0
    Jv = Jv + 1.0
    Jv[:, 1::2] = -1.0
    return Instance("villain", Jh, Jv, h, float(beta), int(chi))


def random_small(Ly, Lx, beta, chi, seed=0, hscale=0.3):
    """Gaussian couplings and fields for small parity cases."""
    rng = np.random.default_rng([seed, 7])
    Jh, Jv, h = _zeros(Ly, Lx)
    Jh = rng.standard_normal(Jh.shape)
    Jv = rng.standard_normal(Jv.shape)
    h = hscale * rng.standard_normal(h.shape)
    return Instance("random", Jh, Jv, h, float(beta), int(chi), {"seed": seed})


# ---- the five workloads -------------------------------------------------------

def config1():
    """8x8 ferromagnet, beta = 0.44, chi = 8, 10^4 proposals, one chain."""
    return ferromagnet(8, 8, 0.44, 8)


def config2():
    """32x32 +-J EA, beta = 1.0, chi = 16, B = 65536."""
    return ea_pm(32, 32, 1.0, 16, seed=0)


def config3(n=256, seed=0):
    """Batched Gaussian EA: L in {16,24,32,48,64}, chi in {8,16,32}, beta = 2.0."""
    rng = np.random.default_rng([seed, 4])
    Ls = rng.choice([16, 24, 32, 48, 64], size=n)
    chis = rng.choice([8, 16, 32], size=n)
    return [ea_gauss(int(L), int(L), 2.0, int(c), seed=seed * 100003 + i) for i, (L, c) in enumerate(zip(Ls, chis))]


def config4():
    """64x64 fully frustrated (Villain), beta = 1.5, chi = 32."""
    return villain(64, 64, 1.5, 32)


def gaussian_ea_batch(n=256, L=32, T=0.212, chi=16, seed=0):
    """n Gaussian EA instances on L x L open lattices at temperature T: the setting of the
    paper's equilibration test (Sec. 3, Fig. hb b, Table hb: 32 x 32, T = 0.212, D = 16)."""
    return [ea_gauss(L, L, 1.0 / T, chi, seed=seed * 100003 + 7919 + i) for i in range(n)]


def gaussian_ea_torus_batch(n=32, L=32, T=0.212, seed=0):
    """n Gaussian EA disorder samples on L x L tori (periodic in both directions) at
    temperature T: couplings (Jh, Jv) as [n, L, L] stacks (bond (r, c)-(r, c+1 mod L) and
    (r, c)-(r+1 mod L, c)), N(0, 1) drawn in float32 and widened; h = 0; beta = 1 / T."""
    rng = np.random.default_rng([seed, 17])
    Jh = rng.standard_normal((n, L, L)).astype(np.float32).astype(np.float64)
    Jv = rng.standard_normal((n, L, L)).astype(np.float32).astype(np.float64)
    return Jh, Jv, np.zeros((n, L, L)), 1.0 / T


def config5():
    """256x256 ferromagnet at beta = 0.4407, chi = 64, B = 2^20."""
    return ferromagnet(256, 256, 0.4407, 64)


def config5_strip(Ly=16):
    """The first Ly rows' worth of the 256-wide critical ferromagnet (same Lx, beta, chi):
    a lattice small enough to build in seconds, for profiling the sampler kernels."""
    return ferromagnet(Ly, 256, 0.4407, 64)


def random_tensors(shapes, seed=0, positive=True):
    """Seeded random tensors of the given shapes (inputs for gradient checks)."""
    rng = np.random.default_rng([seed, 11])
    out = []
    for shp in shapes:
        x = rng.standard_normal(shp)
        out.append(np.abs(x) + 0.1 if positive else x)
    return out


@dataclass
class Instance3D:
    """A cubic-lattice instance: Jx [Lz, Ly, Lx-1], Jy [Lz, Ly-1, Lx], Jz [Lz-1, Ly, Lx],
    h [Lz, Ly, Lx]; environment bond D and boundary-MPS bond chi (Sec. 3D)."""
    name: str
    Jx: np.ndarray
    Jy: np.ndarray
    Jz: np.ndarray
    h: np.ndarray
    beta: float
    D: int
    chi: int

    @property
    def shape(self):
        return self.h.shape


def cubic_uniform(L, beta, D, chi, J=1.0, hfield=0.0, name="cubic"):
    """Uniform L^3 lattice with open boundaries: J > 0 ferromagnet, J < 0 antiferromagnet
    (Sec. 3D: the ferromagnet, and the antiferromagnet in a field h = 3)."""
    Lz = Ly = Lx = int(L)
    return Instance3D(name, np.full((Lz, Ly, Lx - 1), float(J)), np.full((Lz, Ly - 1, Lx), float(J)),
                      np.full((Lz - 1, Ly, Lx), float(J)), np.full((Lz, Ly, Lx), float(hfield)), float(beta), int(D),
                      int(chi))


def cubic_ferromagnet(L=16, T=4.6, D=2, chi=2):
    return cubic_uniform(L, 1.0 / T, D, chi, J=1.0, name="ferro3d")


def cubic_antiferromagnet(L=16, T=4.0, D=2, chi=2, hfield=3.0):
    return cubic_uniform(L, 1.0 / T, D, chi, J=-1.0, hfield=hfield, name="antiferro3d_h3")


def cubic_random(Lz, Ly, Lx, beta, D, chi, seed=0, hscale=0.3):
    """Gaussian couplings and fields on an Lz x Ly x Lx box (parity cases)."""
    g = np.random.default_rng(seed)
    return Instance3D("random3d", g.standard_normal((Lz, Ly, Lx - 1)), g.standard_normal((Lz, Ly - 1, Lx)),
                      g.standard_normal((Lz - 1, Ly, Lx)), hscale * g.standard_normal((Lz, Ly, Lx)), float(beta),
                      int(D), int(chi))
