"""Writes tests/golden/dirac_2x2x2x4.txt and laplace_2x2x2x4.txt from the
FP64 oracle alone.

The paper prints no worked example, so these fixtures are regression pins of
the oracle (and fixed targets for the GPU path): a seeded Haar gauge field and
a seeded Gaussian source on a 2x2x2x4 lattice (antiperiodic time, kappa 0.12),
with D psi, D^dag psi and the CGNR solution x = D^{-1} psi at every site, and,
for the covariant Laplacian M, M psi and x = M^{-1} psi by plain CG.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402
from paper_2001_05218_gb300 import inputs as I  # noqa: E402

DIMS = (2, 2, 2, 4)
KAPPA = 0.12
SEED = 12345


def main():
    U = I.gauge_field(DIMS, "haar", SEED, 1)
    psi = I.gaussian_spinor(DIMS, SEED, 2)
    Dpsi = O.dirac(DIMS, KAPPA, U, psi)
    Ddag = O.dirac(DIMS, KAPPA, U, psi, dag=True)
    x, it, rr = O.cgnr(DIMS, KAPPA, U, psi, tol=1e-14)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dirac_2x2x2x4.txt")
    with open(path, "w") as f:
        f.write("# D psi, D^dag psi and x = D^{-1} psi from the FP64 oracle (make_golden.py)\n")
        f.write("# dims %s kappa %.17g seed %d antiperiodic_t 1 cg_iters %d rel_resid %.3e\n"
                % (" ".join(map(str, DIMS)), KAPPA, SEED, it, rr))
        f.write("# columns: site spin colour re(Dpsi) im(Dpsi) re(Ddag psi) im(Ddag psi) re(x) im(x)\n")
        for s in range(I.volume(DIMS)):
            for sp in range(4):
                for c in range(3):
                    f.write("%d %d %d %.17e %.17e %.17e %.17e %.17e %.17e\n" % (
                        s, sp, c, Dpsi[s, sp, c].real, Dpsi[s, sp, c].imag,
                        Ddag[s, sp, c].real, Ddag[s, sp, c].imag, x[s, sp, c].real, x[s, sp, c].imag))


def main_laplace():
    U = I.gauge_field(DIMS, "haar", SEED, 1)
    psi = I.gaussian_spinor(DIMS, SEED, 2)
    Mpsi = O.laplace(DIMS, KAPPA, U, psi)
    x, it, rr = O.cg_laplace(DIMS, KAPPA, U, psi, tol=1e-14)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "laplace_2x2x2x4.txt")
    with open(path, "w") as f:
        f.write("# M psi and x = M^{-1} psi for the covariant Laplacian M = 1 - kappa K, FP64 oracle (make_golden.py)\n")
        f.write("# dims %s kappa %.17g seed %d antiperiodic_t 1 cg_iters %d rel_resid %.3e\n"
                % (" ".join(map(str, DIMS)), KAPPA, SEED, it, rr))
        f.write("# columns: site spin colour re(Mpsi) im(Mpsi) re(x) im(x)\n")
        for s in range(I.volume(DIMS)):
            for sp in range(4):
                for c in range(3):
                    f.write("%d %d %d %.17e %.17e %.17e %.17e\n" % (
                        s, sp, c, Mpsi[s, sp, c].real, Mpsi[s, sp, c].imag, x[s, sp, c].real, x[s, sp, c].imag))


if __name__ == "__main__":
    main()
    main_laplace()
