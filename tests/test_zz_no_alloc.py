"""cptr_apply_ilu_static: the ILU(0) application for callers that cannot allocate device memory
when they apply the preconditioner (a framework's caching allocator owns the device, a real-time
loop cannot pay for cudaMalloc/cudaFree, or the memory budget is fixed in advance).  Its two
intermediate vectors live in a static device array shared by all calls, instead of context
memory.  It always applies the FP64 factors, so it must give the same result as cptr_apply_ilu
of an FP64 context, call after call, whatever precision and sweep schedule its own context uses;
and it must refuse problems larger than its fixed scratch, and the multicolour ordering.

This file is collected last so that a failure here stops a `-x` run only after every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import paper_1907_04229_gb300 as cp  # noqa: E402

pytestmark = pytest.mark.gpu


def _solver(s, **opts):
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    S = cp.Solver(**opts)
    S.setup(s["n"], s["b"], d(s["row_ptr"]), d(s["col_idx"]), d(s["vals"].reshape(-1)), d(s["unknown_kind"]),
            d(s["weights"].reshape(-1)), d(s["st"]))
    return S


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sweep", ["levels", "paired"])
def test_static_scratch_ilu_matches_context_ilu(precision, sweep):
    s = synth.make_box(7, 5, 3, 3.125, seed=17).system()
    base = dict(max_levels=3, n_coarse=8, ilu_sweep=sweep)
    S = _solver(s, precision=precision, **base)
    ref = S if precision == "fp64" else _solver(s, precision="fp64", **base)
    nb = s["n"] * s["b"]
    for seed in (31, 32):  # two calls in a row: the shared scratch keeps the previous call's data
        r = torch.as_tensor(synth.normal(seed, nb), device="cuda")
        z_ref = torch.empty(nb, dtype=torch.float64, device="cuda")
        z = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
        cp.cptr_apply_ilu(ref.ctx, r, z_ref)
        cp.cptr_apply_ilu_static(S.ctx, r, z)
        err = torch.linalg.norm(z - z_ref) / torch.linalg.norm(z_ref)
        assert float(err) <= 1e-10, float(err)


def test_static_scratch_rejects_multicolour_order():
    s = synth.make_box(7, 5, 3, 3.125, seed=17).system()
    S = _solver(s, max_levels=3, n_coarse=8, ilu_order="multicolor")
    nb = s["n"] * s["b"]
    r = torch.ones(nb, dtype=torch.float64, device="cuda")
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_apply_ilu_static(S.ctx, r, z)
    assert e.value.code == -1 and "natural ILU ordering" in str(e.value)


def test_static_scratch_rejects_oversized_problems():
    # 100 x 100 x 35 cells x 3 unknowns = 1,050,000 > 2^20
    s = synth.make_box(100, 100, 35, 0.5, 0.5, 0.25, seed=3, wells="none").system()
    S = _solver(s, n_coarse=256)
    nb = s["n"] * s["b"]
    r = torch.ones(nb, dtype=torch.float64, device="cuda")
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_apply_ilu_static(S.ctx, r, z)
    assert e.value.code == -1 and "static scratch limit" in str(e.value)
