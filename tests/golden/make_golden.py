"""Writes the stored expected values under tests/golden/ (calls only oracle/).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import green  # noqa: E402


def ghat_quadrature():
    # Set-up of the 32^3 sphere workload: lambda = 0.532 um, eta_b = 1.333, h = lambda/8.
    lam, eta_b = 0.532, 1.333
    kb = green.wavenumber(lam, eta_b)
    h = lam / 8
    R = green.truncation_radius([32 * h] * 3)
    ws = [0.0, 0.25 * kb, 0.9 * kb, kb * (1 - 1e-4), kb, kb * (1 + 1e-4), 1.5 * kb, 2 * kb, np.pi / h]
    vals = green.ghat_t_quadrature(np.array(ws), kb, R, nodes=8192)
    return {
        "source": "numeric radial quadrature of the Fourier transform of g_t (Sec. 3.1 definition of g_t), "
                  "oracle.green.ghat_t_quadrature with 8192 Gauss-Legendre nodes",
        "kb": kb, "R": R, "w": ws,
        "re": [float(v.real) for v in vals], "im": [float(v.imag) for v in vals],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "ghat_t_quadrature.json"), "w") as fh:
        json.dump(ghat_quadrature(), fh, indent=1)
    print("wrote ghat_t_quadrature.json")
