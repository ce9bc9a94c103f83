"""Dense assembly of the IIM operator for tiny grids (brute-force checks).

Column k of L_Omega is L applied to the k-th unit vector of the unknowns; the
affine data part is excluded (Eq. 7 splits it off).
"""
from __future__ import annotations

import numpy as np


def assemble(op):
    unk = np.nonzero(op.unknown.ravel(order="F"))[0]
    N = op.n ** op.d
    A = np.zeros((unk.size, unk.size))
    e = np.zeros(N)
    for c, k in enumerate(unk):
        e[k] = 1.0
        A[:, c] = op.apply(e)[unk]
        e[k] = 0.0
    return A, unk
