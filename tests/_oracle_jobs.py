"""Oracle solves run in worker processes by the GPU solve-parity tests.

Test infrastructure only: each job draws its slice group from the seeded
generator and runs the FP64 oracle's full reconstruction, so that the long
oracle solves of the large workloads run on the host cores while the GPU
tests proceed.  The workers are started with the spawn method (never forked
from a process that holds a CUDA context).
"""
import numpy as np

import oracle as O
from paper_1901_01893_gb300 import synth


def problem(L, Ns, Nc, N, seed, Ldiv):
    """The seeded slice group and its data at SNR 30, normalised to RMS |y| = 1."""
    g = synth.make_group(L, Ns, Nc, N, seed, field=N >= 128)
    xt, y = O.make_data(g, 30.0, Ldiv=Ldiv)
    sc = np.sqrt(np.mean(np.abs(y) ** 2))
    return g, xt / sc, y / sc


def solve(L, Ns, Nc, N, r, Ldiv, seed, K, J, lam):
    g, xt, y = problem(L, Ns, Nc, N, seed, Ldiv)
    return O.reconstruct(y, g["sens"], r, dict(K=K, J=J, lam=lam), Ldiv=Ldiv)
