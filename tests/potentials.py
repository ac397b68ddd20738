"""Per-potential comparison of a GPU solution with the oracle's.

The stated bound holds for each potential separately: the extracellular
potential U (first N entries of X) and the transmembrane potential V (the
N_H entries after it), each as max |X_gpu - X_oracle| over the block divided
by max |X_oracle| over the block.  A single norm over [U; V] would let V,
which sits near v_rest = -90 mV on every heart node, hide an error in U.
"""
import numpy as np


def block_errors(Xg, Xo, N):
    """(error of U, error of V), each relative to the oracle block's largest entry."""
    Xg, Xo = np.asarray(Xg), np.asarray(Xo)
    out = []
    for a, b in ((Xg[:N], Xo[:N]), (Xg[N:], Xo[N:])):
        scale = np.abs(b).max() if b.size else 0.0
        out.append(float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max()))
    return tuple(out)


def assert_potentials_close(Xg, Xo, N, tol, what=""):
    eU, eV = block_errors(Xg, Xo, N)
    assert eU <= tol and eV <= tol, (what, "U", eU, "V", eV)
    return eU, eV
