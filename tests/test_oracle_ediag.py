"""Pins of the oracle's post-hoc diagonalisation diagnostic E_diag = lambda_min(H_VV) (Sec. 3.5):
the textbook H2 full-CI energy, agreement of its dense and iterative routes, and the variational
bound E_S >= E_diag for any amplitudes."""
import os

import numpy as np

from oracle import oracle as O
from paper_2601_21310_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_e_diag_h2_full_ci(olib):
    vals = {}
    with open(os.path.join(GOLDEN, "h2_sto3g.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    h = np.array([[vals["h11"], 0.0], [0.0, vals["h22"]]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0], eri[1, 1, 1, 1] = vals["J11"], vals["J22"]
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = vals["J12"]
    for p, q, r, s in np.ndindex(2, 2, 2, 2):
        if sorted((p, q)) == [0, 1] and sorted((r, s)) == [0, 1]:
            eri[p, q, r, s] = vals["K12"]
    S = synth.full_space(2, 1)
    e = O.e_diag(O.hss(2, h, eri, S))
    assert abs(e - (vals["E_HF"] + vals["E_corr"])) < 3e-4


def test_e_diag_routes_agree_and_bound_E_S(olib):
    p = synth.make_problem("small_n16")
    S = p.S[:5000]
    csr = O.hss(16, p.h, p.eri, S)
    it = O.e_diag(csr)  # 5000 rows: iterative route
    dense = float(np.linalg.eigvalsh(csr.to_scipy().toarray())[0])
    assert abs(it - dense) < 1e-10 * max(1.0, abs(dense))
    rng = np.random.default_rng(0)
    for _ in range(3):
        out, _ = O.energy_from_psi(csr, rng.standard_normal(len(S)))
        assert out[0] >= it - 1e-12
