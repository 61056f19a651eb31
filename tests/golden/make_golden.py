"""Write tests/golden/exact_small.json from the oracle's exact references only.

Every value here comes from oracle.exact: brute-force enumeration of all
2^n states (eqs. boltzmann, pf-ising), the row transfer matrix, and the
Onsager / Yang closed forms cited in Sec. 3 (critical point, magnetisation).
The couplings are stored beside the values so the file is self-contained.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import exact  # noqa: E402


def small_cases():
    rng = np.random.default_rng(20210427)
    cases = []
    def add(name, Ly, Lx, beta, Jh, Jv, h):
        cases.append(dict(name=name, Ly=Ly, Lx=Lx, beta=beta, Jh=np.asarray(Jh).tolist(),
                          Jv=np.asarray(Jv).tolist(), h=np.asarray(h).tolist()))
    add("ferro4x4_b044", 4, 4, 0.44, np.ones((4, 3)), np.ones((3, 4)), np.zeros((4, 4)))
    add("gauss3x5_field", 3, 5, 0.9, rng.standard_normal((3, 4)), rng.standard_normal((2, 5)),
        0.3 * rng.standard_normal((3, 5)))
    add("gauss5x3_field", 5, 3, 0.6, rng.standard_normal((5, 2)), rng.standard_normal((4, 3)),
        0.3 * rng.standard_normal((5, 3)))
    add("pmJ4x4_b1", 4, 4, 1.0, np.where(rng.random((4, 3)) < 0.5, 1.0, -1.0),
        np.where(rng.random((3, 4)) < 0.5, 1.0, -1.0), np.zeros((4, 4)))
    Jv = np.ones((3, 4)); Jv[:, 1::2] = -1.0
    add("villain4x4_b15", 4, 4, 1.5, np.ones((4, 3)), Jv, np.zeros((4, 4)))
    add("antiferro4x4_h2", 4, 4, 0.8, -np.ones((4, 3)), -np.ones((3, 4)), 2.0 * np.ones((4, 4)))
    for c in cases:
        Jh, Jv, h = (np.asarray(c[k], dtype=np.float64) for k in ("Jh", "Jv", "h"))
        _, logZ, pi, E = exact.boltzmann(Jh, Jv, h, c["beta"])
        c["logZ"] = logZ
        c["E_mean"] = float(np.dot(pi, E))
    return cases


def main():
    out = {"_source": "oracle.exact (enumeration, transfer matrix, Onsager/Yang closed forms)"}
    out["small"] = small_cases()
    Jh, Jv, h = np.ones((8, 7)), np.ones((7, 8)), np.zeros((8, 8))
    logZ, E, absm = exact.transfer_matrix(Jh, Jv, h, 0.44)
    out["ferro8x8_b044"] = {"logZ": logZ, "E_per_spin": E / 64, "abs_m": absm,
                           "note": "8x8 OBC ferromagnet, beta = 0.44, row transfer matrix"}
    out["beta_c"] = {"value": exact.BETA_C,
                     "note": "T_c = 2 / ln(1 + sqrt 2) quoted in Sec. 3 (critical temperature)"}
    out["onsager_minus_beta_f"] = {str(b): exact.onsager_minus_beta_f(b) for b in (0.3, 0.4407, 0.6)}
    out["onsager_minus_beta_f_at_beta_c"] = {
        "value": exact.onsager_minus_beta_f(exact.BETA_C),
        "closed_form": 0.5 * math.log(2.0) + 2.0 * 0.915965594177219015 / math.pi,
        "note": "ln(2)/2 + 2 G / pi with Catalan's constant G"}
    out["onsager_u"] = {str(b): exact.onsager_energy_per_spin(b) for b in (0.3, 0.44, 0.45, 0.6)}
    out["yang_m_beta_0.6"] = exact.yang_magnetisation(0.6)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
