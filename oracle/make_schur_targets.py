"""Writes the training targets of the learned Schur scaling: for each of the 16 training grids
(``synth.learned_training_grid``), asinh of the exact ratio (S_T)_ii / B_ii computed by the oracle
(``oracle.schur_ratio_target``) for both base approximations B: the discrete S_e (``targets_se``)
and A_TT (``targets_att``).  Output: ``paper_1907_04229_gb300/data/schur_targets.npz`` with the
two [16, n] float32 arrays and the grid shape.  The features are not stored: the library computes
them from the regenerated Jacobians.

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
    t_se, t_att = [], []
    for k in range(synth.LEARNED_TRAIN_GRIDS):
        sys_k = synth.learned_training_grid(k, *shape).system()
        d = oracle.exact_schur_diag(oracle.Oracle.from_system(sys_k, use_st=False, max_levels=1, dense_max=1,
                                                              stage2=oracle.NONE2), sys_k)
        t_se.append(oracle.schur_ratio_target(sys_k, "se", S_diag=d)[0])
        t_att.append(oracle.schur_ratio_target(sys_k, "att", S_diag=d)[0])
        print(f"grid {k}: S_e target {t_se[-1].min():.4f} .. {t_se[-1].max():.4f}, "
              f"A_TT target {t_att[-1].min():.3f} .. {t_att[-1].max():.3f}", flush=True)
    np.savez_compressed(OUT, targets_se=np.array(t_se, np.float32), targets_att=np.array(t_att, np.float32),
                        shape=np.array(shape))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
