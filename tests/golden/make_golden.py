"""Writes the stored expected values of the full-size parity test
(tests/test_gpu_fullsize.py) from the oracle alone.

Workload: the 40-centre s+p chain of the medium Dirac-Coulomb recipe
(synth.medium_dc: nL 160, nS 480, 40 Kramers pairs, Schwarz threshold 1e-12),
Coulomb block (Eqs. DCInt, SchwarzDen).  The oracle's row-streamed transform
(oracle.Transform.packed_streamed) computes the whole packed output (43 MB);
the file keeps a seeded sample of its entries plus whole-array checksums, so
that the GPU test can compare element by element at the full size.

Run from the repository root (about 25 minutes on 8 cores):
    python tests/golden/make_golden.py
Nothing here calls the CUDA library.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2606_04316_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain40_sp_coulomb_sample.txt")
N_RANDOM = 4000
N_LARGEST = 96


def sample_indices(packed):
    rng = np.random.Generator(np.random.PCG64(20261203))
    n = packed.shape[0]
    idx = set(rng.choice(n, size=N_RANDOM, replace=False).tolist())
    idx.update(np.argsort(-np.abs(packed))[:N_LARGEST].tolist())     # the largest entries
    idx.update([0, n - 1])
    return np.array(sorted(idx), dtype=np.int64)


def main():
    O.build()
    p = synth.medium_dc()
    t0 = time.time()
    tr = O.Transform(p)

    def progress(i, n):
        print("  bra shell pair %d / %d, %.0f s" % (i, n, time.time() - t0), flush=True)

    packed = tr.packed_streamed("coulomb", progress=progress).reshape(-1)
    dt = time.time() - t0
    idx = sample_indices(packed)
    kept = tr.mask("coulomb")
    with open(OUT, "w") as f:
        f.write("# Coulomb block (Eqs. DCInt, SchwarzDen) of the 40-centre s+p chain: synth.medium_dc(),\n")
        f.write("# nL 160, nS 480, 40 Kramers pairs, Schwarz threshold 1e-12; packed layout of include/qdt.h.\n")
        f.write("# Written by tests/golden/make_golden.py from oracle.Transform.packed_streamed (oracle only),\n")
        f.write("# %.0f s on %d host threads.\n" % (dt, os.cpu_count()))
        f.write("# doubles %d\n" % packed.shape[0])
        f.write("# kept_shell_quartets %d of %d\n" % (int(kept.sum()), kept.size))
        f.write("# sum %.17g\n" % float(packed.sum()))
        f.write("# sum_abs %.17g\n" % float(np.abs(packed).sum()))
        f.write("# sum_sq %.17g\n" % float((packed * packed).sum()))
        f.write("# index value\n")
        for i in idx:
            f.write("%d %.17g\n" % (i, packed[i]))
    print("wrote %s: %d entries, %.0f s" % (OUT, idx.shape[0], dt))


if __name__ == "__main__":
    main()
