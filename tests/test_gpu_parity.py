"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (FP64 throughout):
  - set-up arithmetic (decoupling, AMG hierarchy: strength, PMIS, interpolation, Galerkin
    products, smoother diagonals) is ordered identically on both sides: compared bit for bit;
  - one application of an operator (SpMV, V-cycle, ILU, stage 1, two-stage preconditioner):
    relative error <= 1e-10 (different summation order and fused multiply-adds, amplified by the
    conditioning of the coarsest solve and of the triangular solves);
  - the FGMRES solve: iterations equal to the oracle's +-1 and relative solution error <= 1e-8
    per unknown kind (the acceptance bar of the method's parity requirement).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1907_04229_gb300 as cp  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


_SYSTEMS = {}


def system(name):
    if name not in _SYSTEMS:
        if name == "parity":
            r = synth.recipe("parity")
        elif name == "ragged":        # odd sizes: tails in every kernel's tiling
            r = synth.make_box(7, 5, 3, 3.125, seed=17, heaters=[(11, 80.0, 420.0)])
        elif name == "three_phase":   # b = 4
            r = synth.make_box(6, 5, 3, 3.125, seed=19, nphase=3)
        elif name == "medium":        # several AMG levels
            r = synth.make_box(40, 40, 10, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                               kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=365 * 86400.0)
        elif name == "line":
            r = synth.make_box(24, 1, 1, 3.125, seed=4)
        elif name == "cptr200k":
            r = synth.recipe("cptr200k")
        else:
            raise KeyError(name)
        _SYSTEMS[name] = r.system()
    return _SYSTEMS[name]


OPTS = {"parity": dict(max_levels=2), "ragged": dict(max_levels=3, n_coarse=8), "three_phase": dict(n_coarse=16),
        "medium": dict(), "line": dict(max_levels=2, n_coarse=4), "cptr200k": dict()}


def gpu_solver(s, **opts):
    S = cp.Solver(**opts)
    S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
    return S


def pair(name, **extra):
    s = system(name)
    o = {**OPTS[name], **extra}
    return s, oracle.Oracle.from_system(s, **o), gpu_solver(s, **o)


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase"])
def test_weights_and_matrix(name):
    s, o, g = pair(name)
    nb = s["n"] * s["b"]
    rhs = s["rhs"].reshape(-1)
    out = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_weights(g.ctx, dev(rhs), out)
    assert np.array_equal(host(out), o.weight_rhs(rhs))          # same operation order: exact
    x = synth.normal(3, nb)
    y = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_matrix(g.ctx, dev(x), y)
    rp, ci, v = o.matrix()
    absAx = np.array([np.abs(v[rp[i]:rp[i + 1]]) @ np.abs(x[ci[rp[i]:rp[i + 1]]]) for i in range(nb)])
    assert (np.abs(host(y) - o.spmv(x)) <= 1e-14 * absAx).all()


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_amg_hierarchy_bitwise(name):
    s, o, g = pair(name)
    for which in (0, 1):
        lo, lg = o.levels(which), g.hierarchy(which)
        assert len(lo) == len(lg) >= 2
        for a, b in zip(lo, lg):
            assert a["n"] == b["n"]
            for key in ("rp", "ci", "v", "dinv"):
                assert np.array_equal(a[key], b[key]), key
            if "cf" in a:
                for key in ("cf", "Prp", "Pci", "Pv"):
                    assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("name", ["parity", "ragged", "medium"])
@pytest.mark.parametrize("smoother", ["l1", "jacobi"])
def test_vcycle(name, smoother):
    s, o, g = pair(name, smoother=cp.SMOOTHER[smoother])
    for which in (0, 1):
        b = synth.normal(21 + which, s["n"])
        x = torch.empty(s["n"], dtype=torch.float64, device="cuda")
        cp.cptr_apply_vcycle(g.ctx, which, dev(b), x)
        assert relerr(host(x), o.vcycle(which, b)) <= 1e-10


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "line"])
def test_ilu(name):
    s, o, g = pair(name)
    nb = s["n"] * s["b"]
    r = synth.normal(5, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10


@pytest.mark.parametrize("mode", ["full", "upper", "lower", "bd", "cpr", "none"])
def test_stage1_and_precond(mode):
    s, o, g = pair("parity", stage1=cp.STAGE1[mode])
    nb = s["n"] * s["b"]
    v = synth.normal(9, nb)
    x1 = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_stage1(g.ctx, dev(v), x1)
    ref = o.stage1(v)
    if mode == "none":
        assert not host(x1).any()
    else:
        assert relerr(host(x1), ref) <= 1e-10
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_precond(g.ctx, dev(v), z)
    assert relerr(host(z), o.precond(v)) <= 1e-10


def check_solve(s, o, g, rtol, slack=1):
    x_o, info_o = o.solve(s["rhs"], rtol)
    x_g, info_g = g.solve(dev(s["rhs"].reshape(-1)), rtol)
    x_g = host(x_g)
    assert info_g["status"] == "CPTR_OK" and info_o["converged"]
    assert abs(info_g["iters"] - info_o["iters"]) <= slack, (info_g["iters"], info_o["iters"])
    assert info_g["true_rel_res"] <= rtol * 1.05
    b = s["b"]
    for u in range(b):  # per unknown kind: pressure, temperature, saturations
        assert relerr(x_g[u::b], x_o[u::b]) <= 1e-8, (u, relerr(x_g[u::b], x_o[u::b]))
    return info_o, info_g


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
@pytest.mark.parametrize("mode", ["full", "cpr"])
def test_solve(name, mode):
    s, o, g = pair(name, stage1=cp.STAGE1[mode])
    check_solve(s, o, g, 1e-8)


@pytest.mark.parametrize("mode", ["upper", "lower", "bd", "none"])
def test_solve_variants(mode):
    s, o, g = pair("parity", stage1=cp.STAGE1[mode])
    check_solve(s, o, g, 1e-8)


_FULL = {}


def full_size_oracle():
    """The oracle's FP64 solve of the benchmark's workload (100x100x20, 600k unknowns) at the
    benchmark's tolerance, run once for the tests below."""
    if not _FULL:
        s = system("cptr200k")
        o = oracle.Oracle.from_system(s, **OPTS["cptr200k"])
        _FULL["o"] = o
        _FULL["x"], _FULL["info"] = o.solve(s["rhs"], 1e-6)
    return _FULL["o"], _FULL["x"], _FULL["info"]


def check_full_size(g, rtol=1e-6):
    s = system("cptr200k")
    o, x_o, info_o = full_size_oracle()
    x_g, info_g = g.solve(dev(s["rhs"].reshape(-1)), rtol)
    x_g = host(x_g)
    assert info_g["status"] == "CPTR_OK" and info_o["converged"]
    assert abs(info_g["iters"] - info_o["iters"]) <= 1, (info_g["iters"], info_o["iters"])
    assert info_g["true_rel_res"] <= rtol * 1.05
    b = s["b"]
    errs = [relerr(x_g[u::b], x_o[u::b]) for u in range(b)]
    print(f"full size: {info_g['iters']} iterations (oracle {info_o['iters']}), error per unknown kind {errs}")
    for u, e in enumerate(errs):
        assert e <= 1e-8, (u, e)
    return o, info_g


def test_solve_full_size_workload():
    # the benchmark's workload (100x100x20, 600k unknowns), default options, the oracle run in full
    g = gpu_solver(system("cptr200k"), **OPTS["cptr200k"])
    o, info_g = check_full_size(g)
    assert info_g["levels_p"] == len(o.levels(0))


@pytest.mark.parametrize("sweep", ["auto", "paired"])
def test_benchmarked_configuration_full_size(sweep):
    """The headline benchmark's solver exactly as it is timed: launch shapes autotuned at set-up and
    the ILU(0) sweep schedule chosen by the autotuner ("auto"), on the full-size workload, against
    the oracle (iterations +-1, <= 1e-8 per unknown kind); and the paired-level schedule forced,
    since the autotuner picks it on this workload."""
    g = gpu_solver(system("cptr200k"), autotune=1, ilu_sweep=cp.ILU_SWEEP[sweep], **OPTS["cptr200k"])
    sched = [r for r in cp.cptr_tuning(g.ctx) if r[2] == 5][0][3]
    print(f"ILU(0) sweep schedule in use: {sched}")
    if sweep == "paired":
        assert sched == 2
    check_full_size(g)


def test_mixed_full_size_against_fp64_oracle():
    """The mixed-precision form on the full-size workload, autotuned as benchmarked: it must reach
    the FP64 true residual (checked again with the oracle's FP64 matrix on the host), take the
    FP64 oracle's iterations +-1, and its distance from the FP64 oracle's solution is reported.
    Both solutions have relative residual <= 1e-6; their relative distance is bounded by 1e-5
    per unknown kind (measured ~1e-7 .. 1e-6: the FP32 preconditioner only perturbs the Krylov
    space, the outer residual is FP64)."""
    s = system("cptr200k")
    o, x_o, info_o = full_size_oracle()
    g = gpu_solver(s, autotune=1, precision=cp.PRECISION["mixed"], **OPTS["cptr200k"])
    x_g, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-6)
    x_g = host(x_g)
    assert info["status"] == "CPTR_OK" and info["true_rel_res"] <= 1.05e-6
    bw = o.weight_rhs(s["rhs"].reshape(-1))
    assert np.linalg.norm(bw - o.spmv(x_g)) <= 1.05e-6 * np.linalg.norm(bw)
    assert abs(info["iters"] - info_o["iters"]) <= 1, (info["iters"], info_o["iters"])
    b = s["b"]
    errs = [relerr(x_g[u::b], x_o[u::b]) for u in range(b)]
    print(f"mixed full size: {info['iters']} iterations (FP64 oracle {info_o['iters']}), error against the "
          f"FP64 oracle per unknown kind {errs}")
    for u, e in enumerate(errs):
        assert e <= 1e-5, (u, e)


def test_line_grid_converges_in_one_iteration():
    s, o, g = pair("line")
    x, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-10)
    assert info["iters"] == 1 and info["status"] == "CPTR_OK"


def test_restarts_and_iteration_limit():
    s, o, g = pair("parity", stage1=cp.STAGE1["none"], restart=5, max_it=400)
    info_o, info_g = check_solve(s, o, g, 1e-8, slack=1)
    assert info_g["restarts"] >= 1
    # hitting max_it returns NOT_CONVERGED with the same iterate as the oracle
    s, o, g = pair("parity", stage1=cp.STAGE1["none"], restart=5, max_it=12)
    x_o, io = o.solve(s["rhs"], 1e-12)
    x_g, ig = g.solve(dev(s["rhs"].reshape(-1)), 1e-12)
    assert ig["status"] == "CPTR_NOT_CONVERGED" and ig["iters"] == io["iters"] == 12
    assert relerr(host(x_g), x_o) <= 1e-8


def test_zero_rhs():
    s, o, g = pair("parity")
    x, info = g.solve(torch.zeros(s["n"] * s["b"], dtype=torch.float64, device="cuda"), 1e-8)
    assert info["iters"] == 0 and not host(x).any()


def test_host_pointers_match_device_pointers():
    s = system("ragged")
    S = cp.Solver(**OPTS["ragged"])
    S.setup(s["n"], s["b"], s["row_ptr"], s["col_idx"], s["vals"].reshape(-1), s["unknown_kind"],
            s["weights"].reshape(-1), s["st"])
    xh, ih = S.solve(np.ascontiguousarray(s["rhs"].reshape(-1)), 1e-8)
    g = gpu_solver(s, **OPTS["ragged"])
    xd, idv = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ih["iters"] == idv["iters"]
    assert np.array_equal(xh, host(xd))


def test_invalid_inputs_are_rejected():
    s = system("ragged")
    S = cp.Solver()
    with pytest.raises(cp.CptrError) as e:
        S.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert e.value.code == -7                                     # solve before setup
    ci = s["col_idx"].copy()
    ci[[1, 2]] = ci[[2, 1]]                                       # unsorted row
    with pytest.raises(cp.CptrError) as e:
        S.setup(s["n"], s["b"], s["row_ptr"], ci, s["vals"].reshape(-1), s["unknown_kind"])
    assert e.value.code == -1
    v = s["vals"].reshape(-1).copy()
    v[17] = np.nan
    with pytest.raises(cp.CptrError) as e:
        S.setup(s["n"], s["b"], s["row_ptr"], s["col_idx"], v, s["unknown_kind"])
    assert e.value.code == -1 and "non-finite" in str(e.value)
    with pytest.raises(cp.CptrError) as e:
        S.setup(s["n"], s["b"], s["row_ptr"], s["col_idx"], s["vals"].reshape(-1), np.array([0, 2, 2], np.int32))
    assert e.value.code == -1
    # the context is still usable after errors
    S.setup(s["n"], s["b"], s["row_ptr"], s["col_idx"], s["vals"].reshape(-1), s["unknown_kind"],
            s["weights"].reshape(-1), s["st"])
    x, info = S.solve(np.ascontiguousarray(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK"


def test_pattern_errors_name_the_first_bad_row():
    # the pattern is checked on the device; the message names the first failing row and what fails
    kind = system("ragged")["unknown_kind"]
    S = cp.Solver()

    def setup(rp, ci):
        rp, ci = np.asarray(rp, np.int32), np.asarray(ci, np.int32)
        v = np.tile(np.eye(3).reshape(-1), len(ci))
        with pytest.raises(cp.CptrError) as e:
            S.setup(len(rp) - 1, 3, rp, ci, v, kind)
        assert e.value.code == -1
        return str(e.value)

    rp = [0, 2, 5, 7, 9]
    assert "out of range in row 1" in setup(rp, [0, 1, 0, 1, 4, 2, 3, 2, 3])
    assert "not strictly ascending in row 2" in setup(rp, [0, 1, 0, 1, 2, 3, 2, 2, 3])
    assert "missing diagonal block in row 2" in setup(rp, [0, 1, 0, 1, 2, 1, 3, 2, 3])
    # two bad rows: the first one is reported
    assert "not strictly ascending in row 1" in setup(rp, [0, 1, 1, 0, 2, 1, 3, 2, 3])
    assert "row_ptr decreases at row 1" in setup([0, 3, 2, 7, 9], [0, 1, 2, 0, 1, 2, 3, 2, 3])
    # a valid pattern afterwards
    s = system("ragged")
    S.setup(s["n"], s["b"], s["row_ptr"], s["col_idx"], s["vals"].reshape(-1), s["unknown_kind"],
            s["weights"].reshape(-1), s["st"])
    x, info = S.solve(np.ascontiguousarray(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK"


def test_bounded_wait_reports_timeout_and_context_recovers():
    # failure injection without a GPU fault: a row of the ILU sweep waits on a value nobody writes;
    # the wait gives up after ~0.5 s and the call reports CPTR_ETIMEOUT
    s, o, g = pair("parity")
    nb = s["n"] * s["b"]
    cp.cptr_inject_wait_timeout(g.ctx, True)
    r = dev(synth.normal(5, nb))
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_apply_ilu(g.ctx, r, z)
    assert e.value.code == -5
    with pytest.raises(cp.CptrError) as e:
        g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert e.value.code == -5
    cp.cptr_inject_wait_timeout(g.ctx, False)
    check_solve(s, o, g, 1e-8)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_graph_and_direct_launches_agree(use_graph):
    s, o, g = pair("medium", use_graph=use_graph)
    info_o, info_g = check_solve(s, o, g, 1e-8)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_profiling_counts_match_iterations(use_graph):
    s, o, g = pair("parity", use_graph=use_graph)
    cp.cptr_set_profiling(g.ctx, 0b1111111)
    x, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    prof = cp.cptr_profile(g.ctx)
    for fam in ("spmv", "stage1", "stage1_resid", "ilu", "arnoldi", "ilu_fwd", "ilu_bwd"):
        ms, n = prof[fam]
        assert n == info["iters"] and ms > 0.0, (fam, prof[fam])
    l0 = cp.cptr_launch_count()
    g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert cp.cptr_launch_count() - l0 > 20 * info["iters"]


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_multicolour_ilu_and_solve(name):
    s, o, g = pair(name, ilu_order=1)
    nf, nbk = cp.cptr_ilu_levels(g.ctx)
    assert nf == 2 and nbk == 2        # red-black on a 7-point grid
    nb = s["n"] * s["b"]
    r = synth.normal(5, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, g, 1e-8)


# ------------------------------------------------------------------------------------------------
# mixed-precision form: FP32 AMG (BF16 on levels >= 2) and FP32 ILU(0), FP64 Krylov.
# The oracle with precision=1 stores the same rounded values and keeps FP64 arithmetic, so a
# V-cycle differs only by FP32 arithmetic (unit roundoff 6e-8, a few dozen dependent operations
# per entry, amplified by the coarsest solve): 1e-5 relative.  The preconditioner also differs by
# the FP32 ILU factors (the oracle's ILU stays FP64): 1e-4 relative.  Solves must reach the FP64
# true residual; their distance from the FP64 oracle's solution is reported and bounded by
# 1e-4 per unknown kind.
@pytest.mark.parametrize("name", ["parity", "ragged", "medium"])
def test_mixed_vcycle_matches_rounded_oracle(name):
    s, o, g = pair(name, precision=1)
    for which in (0, 1):
        b = synth.normal(21 + which, s["n"])
        x = torch.empty(s["n"], dtype=torch.float64, device="cuda")
        cp.cptr_apply_vcycle(g.ctx, which, dev(b), x)
        assert relerr(host(x), o.vcycle(which, b)) <= 1e-5


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_mixed_preconditioner(name):
    s, o, g = pair(name, precision=1)
    nb = s["n"] * s["b"]
    v = synth.normal(9, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_precond(g.ctx, dev(v), z)
    assert relerr(host(z), o.precond(v)) <= 1e-4


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_mixed_solve_reaches_fp64_residual(name):
    s, o, g = pair(name, precision=1)
    x_g, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK" and info["true_rel_res"] <= 1.05e-8
    xg = host(x_g)
    # independent residual check with the oracle's FP64 matrix on the host
    bw = o.weight_rhs(s["rhs"].reshape(-1))
    assert np.linalg.norm(bw - o.spmv(xg)) <= 1.05e-8 * np.linalg.norm(bw)
    x_o, io = o.solve(s["rhs"], 1e-8)
    assert abs(info["iters"] - io["iters"]) <= 2, (info["iters"], io["iters"])
    o64 = oracle.Oracle.from_system(s, **OPTS[name])
    x64, i64 = o64.solve(s["rhs"], 1e-8)
    b = s["b"]
    for u in range(b):
        assert relerr(xg[u::b], x64[u::b]) <= 1e-4, (u, relerr(xg[u::b], x64[u::b]))


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium", "line"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_chunked_and_level_sweeps_agree(name, precision):
    """The two schedules of the ILU(0) sweeps compute every value with the same operations in the
    same order, so ILU applications agree bit for bit; both match the oracle."""
    s = system(name)
    o = {**OPTS[name], "precision": cp.PRECISION[precision]}
    a = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **o)
    b = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["chunked"], **o)
    assert [r for r in cp.cptr_tuning(b.ctx) if r[2] == 5][0][3] == 1
    assert [r for r in cp.cptr_tuning(a.ctx) if r[2] == 5][0][3] == 0
    r = dev(np.random.default_rng(3).normal(size=s["n"] * s["b"]))
    za, zb = torch.empty_like(r), torch.empty_like(r)
    cp.cptr_apply_ilu(a.ctx, r, za)
    cp.cptr_apply_ilu(b.ctx, r, zb)
    assert torch.equal(za, zb)
    xa, ia = a.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    xb, ib = b.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ia["iters"] == ib["iters"] and torch.equal(xa, xb)


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium", "line"])
def test_paired_level_sweeps(name):
    """Paired levels solve the same triangular systems with the sums grouped differently (a row of
    odd level substitutes its dependencies of the level before): ILU applications agree with the
    level-set sweeps to rounding and with the oracle within the operator tolerance, and solves
    match the oracle."""
    s = system(name)
    a = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **OPTS[name])
    b = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["paired"], **OPTS[name])
    assert [r for r in cp.cptr_tuning(b.ctx) if r[2] == 5][0][3] == 2
    r = np.random.default_rng(4).normal(size=s["n"] * s["b"])
    za, zb = torch.empty(r.size, dtype=torch.float64, device="cuda"), torch.empty(r.size, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(a.ctx, dev(r), za)
    cp.cptr_apply_ilu(b.ctx, dev(r), zb)
    assert relerr(host(zb), host(za)) <= 1e-12
    o = oracle.Oracle.from_system(s, **OPTS[name])
    assert relerr(host(zb), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, b, 1e-8)


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium", "line"])
def test_paired_level_sweeps_mixed(name):
    """The paired-level tables in FP32 (mixed form): against the FP64 ILU(0), the FP32 paired
    sweeps are as accurate as the FP32 level-set sweeps (both carry FP32 rounding through every
    level), and solves converge like them."""
    s = system(name)
    o = {**OPTS[name], "precision": cp.PRECISION["mixed"]}
    a = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **o)
    b = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["paired"], **o)
    f = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **OPTS[name])
    assert [r for r in cp.cptr_tuning(b.ctx) if r[2] == 5][0][3] == 2
    r = dev(np.random.default_rng(5).normal(size=s["n"] * s["b"]))
    za, zb, z64 = torch.empty_like(r), torch.empty_like(r), torch.empty_like(r)
    cp.cptr_apply_ilu(a.ctx, r, za)
    cp.cptr_apply_ilu(b.ctx, r, zb)
    cp.cptr_apply_ilu(f.ctx, r, z64)
    ea, eb = relerr(host(za), host(z64)), relerr(host(zb), host(z64))
    assert ea <= 1e-3 and eb <= 2 * ea + 1e-6, (ea, eb)
    xa, ia = a.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    xb, ib = b.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ib["status"] == "CPTR_OK" and ib["true_rel_res"] <= 1e-8 * 1.05
    assert abs(ia["iters"] - ib["iters"]) <= 1


@pytest.mark.parametrize("name", ["ragged", "three_phase"])
def test_paired_level_sweeps_multicolour(name):
    """Paired levels on the red-black order: every black row substitutes all its red dependencies,
    which depend on nothing, so the forward sweep waits on no other row; the result matches the
    multicolour oracle."""
    s, o, g = pair(name, ilu_order=1, ilu_sweep=cp.ILU_SWEEP["paired"])
    assert [r for r in cp.cptr_tuning(g.ctx) if r[2] == 5][0][3] == 2
    nb = s["n"] * s["b"]
    r = synth.normal(6, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, g, 1e-8)
