"""The launch-shape autotuner: tuned shapes change only the order of partial sums within a row,
so a tuned solve takes the same iterations as the untuned one and agrees to rounding."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_1907_04229_gb300 as cp  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def setup(s, **opts):
    S = cp.Solver(**opts)
    S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
    return S


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tuned_solve_matches_untuned(precision):
    s = synth.make_box(40, 40, 10, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                       kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=365 * 86400.0).system()
    a = setup(s, precision=cp.PRECISION[precision])
    b = setup(s, precision=cp.PRECISION[precision], autotune=1)
    xa, ia = a.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    xb, ib = b.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ia["status"] == ib["status"] == "CPTR_OK"
    assert abs(ia["iters"] - ib["iters"]) <= (0 if precision == "fp64" else 1)
    err = torch.linalg.norm(xa - xb) / torch.linalg.norm(xa)
    assert err <= (1e-10 if precision == "fp64" else 1e-6), float(err)
    rows = cp.cptr_tuning(b.ctx)
    levels = ia["levels_p"] - 1 + ia["levels_T"] - 1
    assert len(rows) == 3 * levels + 5
    for h, l, k, G, T in rows:
        if k == 3:
            assert h == 2 and T in (64, 128, 256, 512)
        elif k == 4:       # ILU sweeps: poll back-off (ns), persistent grid of the level-set schedule
            assert h == 3 and G in (0, 8, 32, 128, 512) and T in (152, 304, 608, 1216)
        elif k == 5:       # ILU sweeps: level sets (0), chunked wavefront (1), paired levels (2), tiles (3)
            assert h == 3 and G in (0, 1, 2, 3)
        elif k == 6:       # tile shape the autotuner chose (lines per tile along y and z)
            assert h == 3 and 0 < G * T <= 64
        elif k == 7:       # lanes per row of the grouped-level sweeps (0: not in use)
            assert h == 3 and G in (0, 4, 8, 16) and T == 0
        else:
            assert G in (1, 2, 4, 8, 16, 32) and T in (128, 256, 512)
    # untuned: heuristic lanes, 256 threads; level-set sweeps on 608 blocks, 20 ns back-off
    for h, l, k, G, T in cp.cptr_tuning(a.ctx):
        assert (G, T) == {4: (20, 608), 5: (0, 0), 6: (0, 0), 7: (0, 0)}.get(k, (0, 256))
    # a second set-up of the same operators reuses the cached shapes
    b.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
    assert cp.cptr_tuning(b.ctx) == rows


def test_tuned_ensemble_matches_untuned():
    systems = [synth.ensemble_member(k, sh).system() for k, sh in enumerate([(9, 9, 4), (14, 14, 4), (6, 6, 4)])]

    def run(tune):
        S = cp.Solver(autotune=tune, precision=cp.PRECISION["mixed"])
        inst = [dict(n_cells=s["n"], row_ptr=dev(s["row_ptr"]), col_idx=dev(s["col_idx"]),
                     vals=dev(s["vals"].reshape(-1)), row_weights=dev(s["weights"].reshape(-1)), st_vals=dev(s["st"]))
                for s in systems]
        S.setup_batch(3, inst, dev(systems[0]["unknown_kind"]))
        return S.solve_batch([dev(s["rhs"].reshape(-1)) for s in systems], 1e-6)

    _, st0, i0 = run(0)
    _, st1, i1 = run(1)
    assert st0 == st1 == "CPTR_OK"
    for a, b in zip(i0, i1):
        assert abs(a["iters"] - b["iters"]) <= 1 and b["true_rel_res"] <= 1e-6 * 1.05
