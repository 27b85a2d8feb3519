"""Writes the training targets of the learned Schur scaling: for each of the 16 training grids
(``synth.learned_training_grid``), asinh of the exact ratio (S_T)_ii / (A_TT)_ii computed by the
oracle (``oracle.schur_ratio_target``).  Output: ``paper_1907_04229_gb300/data/schur_targets.npz``
with ``targets`` [16, n] float32 and the grid shape.  The features are not stored: the library
computes them from the regenerated Jacobians.

    python -m oracle.make_schur_targets
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth   # noqa: E402

OUT = os.path.join(os.path.dirname(HERE), "paper_1907_04229_gb300", "data", "schur_targets.npz")


def main():
    shape = (32, 32, 8)
    targets = []
    for k in range(synth.LEARNED_TRAIN_GRIDS):
        t, _ = oracle.schur_ratio_target(synth.learned_training_grid(k, *shape).system())
        targets.append(t)
        print(f"grid {k}: target range {t.min():.3f} .. {t.max():.3f}", flush=True)
    np.savez_compressed(OUT, targets=np.array(targets, np.float32), shape=np.array(shape))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
