"""The bounds-checking build (libcptr_check.so, compiled with -DCPTR_CHECK): every index that a
hot-path kernel reads from a table is checked against its array. A failed check is recorded, the
access is skipped, and the call returns CPTR_ECHECK. Here the check build runs the configurations
of the parity tests: FP64 and mixed precision, level-set, grouped-level (pairs and groups of three,
four to sixteen lanes per row) and tiled sweeps, multicolour
order, ILU(1), the unknown-based first stage, CPR, b = 4, and an ensemble. Every call must return
without a failed check, and the solves must match the oracle as in the parity tests.

The cases run in a child process: a process loads one library, and this one loads libcptr.so."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    ("ragged", dict(max_levels=3, n_coarse=8)),
    ("ragged", dict(max_levels=3, n_coarse=8, precision=1)),
    ("medium", dict(ilu_sweep=3)),
    ("medium", dict(ilu_sweep=3, ilu_group=3, ilu_lanes=8)),
    ("medium", dict(ilu_sweep=3, ilu_lanes=16)),
    ("medium", dict(ilu_sweep=4, tile_y=2, tile_z=2)),
    ("medium", dict(ilu_sweep=2)),
    ("medium", dict(ilu_order=1)),
    ("medium", dict(ilu_fill=1)),
    ("medium", dict(stage1=6, max_it=20)),
    ("medium", dict(stage1=4)),
    ("three_phase", dict(n_coarse=16)),
    ("three_phase", dict(n_coarse=16, precision=1, ilu_sweep=3)),
    ("three_phase", dict(n_coarse=16, precision=1, ilu_sweep=3, ilu_group=3, ilu_lanes=8)),
]


def _system(name):
    import synth
    if name == "ragged":
        return synth.make_box(7, 5, 3, 3.125, seed=17, heaters=[(11, 80.0, 420.0)]).system()
    if name == "three_phase":
        return synth.make_box(6, 5, 3, 3.125, seed=19, nphase=3, wells="four").system()
    return synth.make_box(40, 40, 10, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                          kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=365 * 86400.0).system()


def run_cases():
    """Child process: the cases on libcptr_check.so against the oracle."""
    import torch

    import oracle
    import paper_1907_04229_gb300 as cp
    cp.select_library("check")
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    for name, opts in CASES:
        s = _system(name)
        S = cp.Solver(**opts)
        S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
                dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
        x, info = S.solve(dev(s["rhs"].reshape(-1)), 1e-8)
        o = oracle.Oracle.from_system(s, **opts)
        xo, io = o.solve(s["rhs"], 1e-8)
        stalls = opts.get("stage1") == 6
        assert info["status"] == ("CPTR_NOT_CONVERGED" if stalls else "CPTR_OK"), (name, opts, info)
        assert abs(info["iters"] - io["iters"]) <= 1, (name, opts, info["iters"], io["iters"])
        xg, b = x.cpu().numpy(), s["b"]
        tol = 1e-4 if opts.get("precision") == 1 else 1e-8
        for u in range(b):
            ref = xo[u::b]
            err = np.linalg.norm(xg[u::b] - ref) / max(np.linalg.norm(ref), 1e-300)
            assert err <= tol, (name, opts, u, err)
        S.close()
        print(f"{name} {opts}: {info['iters']} iterations, no failed index check", flush=True)
    # an ensemble of three instances
    import synth
    insts = [synth.ensemble_member(k, sh).system() for k, sh in enumerate([(6, 5, 3), (10, 8, 2), (4, 4, 4)])]
    S = cp.Solver()
    S.setup_batch(3, [dict(n_cells=t["n"], row_ptr=dev(t["row_ptr"]), col_idx=dev(t["col_idx"]),
                           vals=dev(t["vals"].reshape(-1)), row_weights=dev(t["weights"].reshape(-1)),
                           st_vals=dev(t["st"])) for t in insts], dev(insts[0]["unknown_kind"]))
    xs, status, infos = S.solve_batch([dev(t["rhs"].reshape(-1)) for t in insts], 1e-8)
    assert status == "CPTR_OK", status
    print("ensemble of 3: no failed index check", flush=True)


@pytest.mark.gpu
def test_check_build_runs_the_parity_configurations_clean():
    from paper_1907_04229_gb300 import _build
    _build.build(variant="check")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "run"], cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    print(r.stdout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert r.stdout.count("no failed index check") == len(CASES) + 1


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "run":
    sys.path.insert(0, ROOT)
    run_cases()
