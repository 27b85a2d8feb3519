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
        elif name == "ragged_mid":    # 7,659 cells: several levels above the fused size, a partial last warp
            r = synth.make_box(37, 23, 9, 3.125, seed=23, sigma=1.5)
        elif name == "line":
            r = synth.make_box(24, 1, 1, 3.125, seed=4)
        elif name == "cptr200k":
            r = synth.recipe("cptr200k")
        else:
            raise KeyError(name)
        _SYSTEMS[name] = r.system()
    return _SYSTEMS[name]


OPTS = {"parity": dict(max_levels=2), "ragged": dict(max_levels=3, n_coarse=8), "three_phase": dict(n_coarse=16),
        "medium": dict(), "ragged_mid": dict(), "line": dict(max_levels=2, n_coarse=4), "cptr200k": dict()}


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


@pytest.mark.parametrize("name", ["parity", "ragged_mid", "medium"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vcycle_launch_shapes(name, precision):
    """Every lane count of the V-cycle kernels (smoother + residual, restriction, prolongation),
    forced on all levels above the fused size (rows of 7 to ~30 entries; the 7,659-cell box ends in
    a partial warp on every level): all match the oracle's cycle (FP64 1e-10; mixed, against the
    oracle's cycle on the same rounded values, 1e-5: the FP32 bound of the mixed tests below), and
    each agrees with the one-lane cycle to the same bound."""
    s = system(name)
    prec = cp.PRECISION[precision]
    o = oracle.Oracle.from_system(s, precision=prec, **OPTS[name])   # mixed: the oracle's rounded values
    tol = 1e-10 if precision == "fp64" else 1e-5
    for which in (0, 1):
        b = synth.normal(21 + which, s["n"])
        xo = o.vcycle(which, b)
        out = {}
        for lanes in (1, 2, 4, 8, 16, 32):
            g = gpu_solver(s, csr_lanes=lanes, precision=prec, **OPTS[name])
            assert all(r[3] == lanes for r in cp.cptr_tuning(g.ctx) if r[2] in (0, 1, 2) and r[0] == which)
            x = torch.empty(s["n"], dtype=torch.float64, device="cuda")
            cp.cptr_apply_vcycle(g.ctx, which, dev(b), x)
            out[lanes] = host(x)
            assert relerr(out[lanes], xo) <= tol, (lanes, relerr(out[lanes], xo))
        for lanes in (2, 4, 8, 16, 32):
            assert relerr(out[lanes], out[1]) <= tol, (lanes, relerr(out[lanes], out[1]))


@pytest.mark.parametrize("n_levels", [1, 2])
def test_coarsest_inverse_of_many_rows(n_levels):
    """Coarsest matrices larger than one block's shared memory are inverted by the multi-block
    Gauss-Jordan kernel (one grid of resident blocks, two grid barriers per pivot): with one level
    the V-cycle is A^{-1} b on the 1024-cell system, with two levels the coarsest level has a few
    hundred rows; against the oracle's dense LU solve, and A x = b checked on the host."""
    s, o, g = pair("parity", max_levels=n_levels, dense_max=4096)
    for which in (0, 1):
        lev = g.hierarchy(which)
        assert lev[-1]["dense"] and lev[-1]["n"] > 160, [L["n"] for L in lev]
        b = synth.normal(31 + which, s["n"])
        x = torch.empty(s["n"], dtype=torch.float64, device="cuda")
        cp.cptr_apply_vcycle(g.ctx, which, dev(b), x)
        assert relerr(host(x), o.vcycle(which, b)) <= 1e-10
        if n_levels == 1:
            L = lev[0]
            A = np.zeros((L["n"], L["n"]))
            for i in range(L["n"]):
                A[i, L["ci"][L["rp"][i]:L["rp"][i + 1]]] = L["v"][L["rp"][i]:L["rp"][i + 1]]
            assert np.linalg.norm(A @ host(x) - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "line"])
def test_ilu(name):
    s, o, g = pair(name)
    nb = s["n"] * s["b"]
    r = synth.normal(5, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10


def _shuffled_blocks(n, b, seed):
    """Well-conditioned b x b blocks ((b + 1) I + uniform(-1, 1)) with their rows shuffled per
    cell, so that partial pivoting exchanges rows; every fourth block has an exact tie of
    magnitudes (2 and -2) between the first two candidates of its first pivot step."""
    rng = np.random.default_rng(seed)
    D = np.empty((n, b, b))
    for i in range(n):
        while True:
            m = rng.uniform(-1.0, 1.0, (b, b)) + (b + 1.0) * np.eye(b)
            m = m[rng.permutation(b)]
            if i % 4 == 0:
                m[0, 0], m[1, 0] = 2.0, -2.0
                m[2:, 0] = rng.uniform(-1.0, 1.0, b - 2)
            if np.linalg.cond(m) < 1e2:
                break
        D[i] = m
    return D


@pytest.mark.parametrize("b", [3, 4])
def test_pivot_inverses_with_row_exchanges(b):
    """ILU(0) of a block-diagonal matrix is its pivot inverses, so an ILU application gives
    D_i^{-1} r_i.  The blocks need row exchanges (and every fourth one breaks a tie by the lowest
    position).  512 cells, one narrow level, take the row-per-warp factorisation and its warp-wide
    inverse; 4096 cells take the four-lane factorisation.  Both match numpy's solve, and they
    agree bit for bit on the cells they share: the same pivots, ties and operations."""
    kind = system("parity" if b == 3 else "three_phase")["unknown_kind"]
    Dall = _shuffled_blocks(4096, b, 41)
    rall = synth.normal(43, 4096 * b)
    out = {}
    for n in (512, 4096):
        D, r = Dall[:n], rall[:n * b]
        S = cp.Solver(stage1=cp.STAGE1["none"])
        S.setup(n, b, dev(np.arange(n + 1, dtype=np.int32)), dev(np.arange(n, dtype=np.int32)),
                dev(D.reshape(-1)), dev(kind))
        z = torch.empty(n * b, dtype=torch.float64, device="cuda")
        cp.cptr_apply_ilu(S.ctx, dev(r), z)
        ref = np.linalg.solve(D, r.reshape(n, b, 1))[..., 0].reshape(-1)
        assert relerr(host(z), ref) <= 1e-13, (n, relerr(host(z), ref))
        out[n] = host(z)
        S.close()
    assert np.array_equal(out[512], out[4096][:512 * b])


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


@pytest.mark.parametrize("sweep", ["auto", "paired", "grouped3", "tiled"])
def test_benchmarked_configuration_full_size(sweep):
    """The headline benchmark's solver exactly as it is timed: launch shapes autotuned at set-up and
    the ILU(0) sweep schedule chosen by the autotuner ("auto"), on the full-size workload, against
    the oracle (iterations +-1, <= 1e-8 per unknown kind); and the grouped-level (groups of two and
    of three) and tiled schedules forced, the candidates the autotuner picks from on this workload."""
    grp = dict(ilu_group=3) if sweep == "grouped3" else {}
    g = gpu_solver(system("cptr200k"), autotune=1, ilu_sweep=cp.ILU_SWEEP[sweep.replace("grouped3", "paired")],
                   **grp, **OPTS["cptr200k"])
    sched = [r for r in cp.cptr_tuning(g.ctx) if r[2] == 5][0][3:5]
    print(f"ILU(0) sweep schedule in use: {sched}")
    if sweep in ("paired", "grouped3", "tiled"):
        assert sched == {"paired": (2, 2), "grouped3": (2, 3), "tiled": (3, 0)}[sweep]
    check_full_size(g)


def full_size_exact():
    """The oracle's FP64 solution of the full-size workload converged to rtol 1e-12: the reference
    against which solutions at the benchmark's tolerance are measured."""
    if "x_exact" not in _FULL:
        o, _, _ = full_size_oracle()
        x, info = o.solve(system("cptr200k")["rhs"], 1e-12)
        assert info["converged"]
        _FULL["x_exact"] = x
    return _FULL["x_exact"]


def test_mixed_full_size_against_fp64_oracle():
    """The mixed-precision form on the full-size workload, autotuned as benchmarked.  It must reach
    the FP64 true residual (checked again with the oracle's FP64 matrix on the host) in the FP64
    oracle's iterations +-1.  Its solution follows another Krylov path than the FP64 one, so at
    rtol 1e-6 the two differ by up to kappa * 1e-6 (measured: 2.6e-3 in T on this workload, whose
    temperature block is stiff), and that distance is reported, not bounded.  The claim that is
    checked: against the oracle's solution converged to 1e-12, the mixed form's error is at most
    ten times the FP64 oracle's own error at the same tolerance, per unknown kind."""
    s = system("cptr200k")
    o, x_o, info_o = full_size_oracle()
    g = gpu_solver(s, autotune=1, precision=cp.PRECISION["mixed"], **OPTS["cptr200k"])
    x_g, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-6)
    x_g = host(x_g)
    assert info["status"] == "CPTR_OK" and info["true_rel_res"] <= 1.05e-6
    bw = o.weight_rhs(s["rhs"].reshape(-1))
    assert np.linalg.norm(bw - o.spmv(x_g)) <= 1.05e-6 * np.linalg.norm(bw)
    assert abs(info["iters"] - info_o["iters"]) <= 1, (info["iters"], info_o["iters"])
    x_star = full_size_exact()
    b = s["b"]
    e_fp64_path = [relerr(x_g[u::b], x_o[u::b]) for u in range(b)]
    e_mixed = [relerr(x_g[u::b], x_star[u::b]) for u in range(b)]
    e_fp64 = [relerr(x_o[u::b], x_star[u::b]) for u in range(b)]
    print(f"mixed full size: {info['iters']} iterations (FP64 oracle {info_o['iters']}); per unknown kind: "
          f"against the FP64 oracle at 1e-6 {e_fp64_path}, against the converged solution {e_mixed} "
          f"(FP64 oracle at 1e-6: {e_fp64})")
    for u in range(b):
        assert e_mixed[u] <= max(10 * e_fp64[u], 1e-8), (u, e_mixed[u], e_fp64[u])


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


@pytest.mark.parametrize("use_graph", [0, 1, 2])
def test_graph_and_direct_launches_agree(use_graph):
    s, o, g = pair("medium", use_graph=use_graph)
    info_o, info_g = check_solve(s, o, g, 1e-8)


@pytest.mark.parametrize("use_graph", [0, 1, 2])
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


@pytest.mark.parametrize("stage1", ["full", "cpr"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vcycle_kernel_profiling(stage1, precision):
    """Bit 7 of the profiling mask times the four fine-level kernels of every V-cycle: each is
    launched once per V-cycle of its hierarchy, a fixed number of V-cycles per iteration; the
    temperature hierarchy is idle under CPR; the solve is unchanged."""
    s, o, g = pair("medium", stage1=cp.STAGE1[stage1], precision=cp.PRECISION[precision])
    x0, i0 = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    cp.cptr_set_profiling(g.ctx, cp.PROFILE_MASK_VCYCLE)
    x1, i1 = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert i1["iters"] == i0["iters"] and torch.equal(x0, x1)
    vc = cp.cptr_profile_vcycle(g.ctx)
    assert cp.cptr_profile(g.ctx)["spmv"][1] == 0           # bit 7 alone times no family
    for h in ("p", "T"):
        counts = {vc[f"{h}_{k}"][1] for k in ("down", "restrict", "prolong", "post")}
        assert len(counts) == 1, vc
        cnt = counts.pop()
        if h == "T" and stage1 == "cpr":
            assert cnt == 0
        else:
            assert cnt > 0 and cnt % i1["iters"] == 0, vc
            assert all(vc[f"{h}_{k}"][0] > 0.0 for k in ("down", "restrict", "prolong", "post"))
    cp.cptr_set_profiling(g.ctx, 0)


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
@pytest.mark.parametrize("group", [2, 3, 4])
@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_paired_level_sweeps(name, group, lanes):
    """Grouped levels solve the same triangular systems with the sums grouped differently (a row
    substitutes its dependencies inside its group of two, three or four levels, through chains of
    up to group - 1 links; with 8 or 16 lanes a row's slots are split between 2 or 4 parts): ILU
    applications agree with the level-set sweeps to rounding and with the oracle within the
    operator tolerance, and solves match the oracle."""
    s = system(name)
    a = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **OPTS[name])
    b = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["paired"], ilu_group=group, ilu_lanes=lanes, **OPTS[name])
    tun = cp.cptr_tuning(b.ctx)
    assert [r for r in tun if r[2] == 5][0][3:5] == (2, group) and [r for r in tun if r[2] == 7][0][3] == lanes
    r = np.random.default_rng(4).normal(size=s["n"] * s["b"])
    za, zb = torch.empty(r.size, dtype=torch.float64, device="cuda"), torch.empty(r.size, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(a.ctx, dev(r), za)
    cp.cptr_apply_ilu(b.ctx, dev(r), zb)
    assert relerr(host(zb), host(za)) <= 1e-12
    o = oracle.Oracle.from_system(s, **OPTS[name])
    assert relerr(host(zb), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, b, 1e-8)


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium", "line"])
@pytest.mark.parametrize("group", [2, 3])
@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_paired_level_sweeps_mixed(name, group, lanes):
    """The grouped-level tables in FP32 (mixed form): against the FP64 ILU(0), the FP32 grouped
    sweeps are about as accurate as the FP32 level-set sweeps (both carry FP32 rounding through
    every level; pairs over four lanes within twice the level sets' error; groups of three, or a
    row's slots split over parts of four lanes, within ten times: the row then sums terms
    larger than its result (products of three factor blocks, or two partial sums that cancel), each
    rounded to FP32), and solves converge like them."""
    s = system(name)
    o = {**OPTS[name], "precision": cp.PRECISION["mixed"]}
    a = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **o)
    b = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["paired"], ilu_group=group, ilu_lanes=lanes, **o)
    f = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **OPTS[name])
    assert [r for r in cp.cptr_tuning(b.ctx) if r[2] == 5][0][3:5] == (2, group)
    r = dev(np.random.default_rng(5).normal(size=s["n"] * s["b"]))
    za, zb, z64 = torch.empty_like(r), torch.empty_like(r), torch.empty_like(r)
    cp.cptr_apply_ilu(a.ctx, r, za)
    cp.cptr_apply_ilu(b.ctx, r, zb)
    cp.cptr_apply_ilu(f.ctx, r, z64)
    ea, eb = relerr(host(za), host(z64)), relerr(host(zb), host(z64))
    assert ea <= 1e-3 and eb <= (2 if group == 2 and lanes == 4 else 10) * ea + 1e-6, (ea, eb)
    xa, ia = a.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    xb, ib = b.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ib["status"] == "CPTR_OK" and ib["true_rel_res"] <= 1e-8 * 1.05
    assert abs(ia["iters"] - ib["iters"]) <= 1


@pytest.mark.parametrize("name", ["ragged", "three_phase"])
@pytest.mark.parametrize("group", [2, 3])
def test_paired_level_sweeps_multicolour(name, group):
    """Grouped levels on the red-black order (two level sets per sweep, so one group): every black
    row substitutes all its red dependencies, which depend on nothing, so the forward sweep waits
    on no other row; the result matches the multicolour oracle."""
    s = system(name)
    o = oracle.Oracle.from_system(s, ilu_order=1, **OPTS[name])
    g = gpu_solver(s, ilu_order=1, ilu_sweep=cp.ILU_SWEEP["paired"], ilu_group=group, **OPTS[name])
    assert [r for r in cp.cptr_tuning(g.ctx) if r[2] == 5][0][3:5] == (2, group)
    nb = s["n"] * s["b"]
    r = synth.normal(6, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, g, 1e-8)


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium", "line"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(0, 0), (1, 1), (2, 3)])
def test_tiled_and_level_sweeps_agree(name, precision, shape):
    """Tiled sweeps (a block per tile of grid lines, the tile's own level sets inside the block)
    compute every value with the same operations in the same order as the level-set sweeps, so ILU
    applications and solves agree bit for bit, whatever the tile shape: the modelled one (0, 0),
    one line per tile (every y and z dependency crosses blocks), and 2 x 3 lines."""
    s = system(name)
    o = {**OPTS[name], "precision": cp.PRECISION[precision]}
    a = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["levels"], **o)
    b = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["tiled"], tile_y=shape[0], tile_z=shape[1], **o)
    tun = cp.cptr_tuning(b.ctx)
    assert [r for r in tun if r[2] == 5][0][3] == 3
    ty, tz = [r for r in tun if r[2] == 6][0][3:5]
    nx, ny, nz = s["grid"]
    if shape != (0, 0):
        assert (ty, tz) == (min(shape[0], ny), min(shape[1], nz))
    r = dev(np.random.default_rng(3).normal(size=s["n"] * s["b"]))
    for _ in range(2):   # twice: the sweeps reset their vectors and tickets per application
        za, zb = torch.empty_like(r), torch.empty_like(r)
        cp.cptr_apply_ilu(a.ctx, r, za)
        cp.cptr_apply_ilu(b.ctx, r, zb)
        assert torch.equal(za, zb)
    xa, ia = a.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    xb, ib = b.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ia["iters"] == ib["iters"] and torch.equal(xa, xb)


@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_paired_sweeps_timeout_reported_and_context_recovers(lanes):
    """The bounded waits of the grouped-level sweeps (four or eight lanes per row): the injected
    wait on a value nobody writes gives up, the call reports CPTR_ETIMEOUT, and the context solves
    normally afterwards."""
    s = system("medium")
    o = oracle.Oracle.from_system(s, **OPTS["medium"])
    g = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP["paired"], ilu_lanes=lanes, **OPTS["medium"])
    assert [r for r in cp.cptr_tuning(g.ctx) if r[2] == 7][0][3] == lanes
    nb = s["n"] * s["b"]
    cp.cptr_inject_wait_timeout(g.ctx, True)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_apply_ilu(g.ctx, dev(synth.normal(5, nb)), z)
    assert e.value.code == -5
    cp.cptr_inject_wait_timeout(g.ctx, False)
    check_solve(s, o, g, 1e-8)


def test_tiled_sweeps_timeout_reported_and_context_recovers():
    """The bounded waits of the tiled sweeps: the injected wait on a value nobody writes gives up,
    the call reports CPTR_ETIMEOUT, and the context solves normally afterwards."""
    s, o, g = pair("medium", ilu_sweep=cp.ILU_SWEEP["tiled"], tile_y=4, tile_z=2)
    assert [r for r in cp.cptr_tuning(g.ctx) if r[2] == 5][0][3] == 3
    nb = s["n"] * s["b"]
    cp.cptr_inject_wait_timeout(g.ctx, True)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_apply_ilu(g.ctx, dev(synth.normal(5, nb)), z)
    assert e.value.code == -5
    cp.cptr_inject_wait_timeout(g.ctx, False)
    check_solve(s, o, g, 1e-8)


# ------------------------------------------------------------------------------------------------
# unknown-based AMG first stage on A_00 (Sec. 3.4) and the S~_diag Schur approximation (Sec. 3.3.1)
def _bitwise_levels(lo, lg):
    assert len(lo) == len(lg) >= 2
    for a, b in zip(lo, lg):
        assert a["n"] == b["n"]
        for key in ("rp", "ci", "v", "dinv"):
            assert np.array_equal(a[key], b[key]), key
        if "cf" in a:
            for key in ("cf", "Prp", "Pci", "Pv"):
                assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_uamg_hierarchy_bitwise(name):
    """The device's unknown-based hierarchy of A_00 (per-block strength, PMIS and direct
    interpolation, Galerkin product of the coupled matrix) equals the oracle's bit for bit."""
    s, o, g = pair(name, stage1=cp.STAGE1["uamg"])
    _bitwise_levels(o.levels(2), g.hierarchy(0))


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_uamg_vcycle_stage1_precond_and_solve(name):
    """V-cycle, stage 1, two-stage preconditioner and solve of CPTR-uAMG against the oracle.  On the
    conduction-dominated "medium" system (dt = 1 year) CPTR-uAMG with these AMG components stalls
    in the oracle too, so there both stop at the same iteration limit with the same iterate."""
    stalls = name == "medium"
    s, o, g = pair(name, stage1=cp.STAGE1["uamg"], **(dict(max_it=40) if stalls else {}))
    n, nb = s["n"], s["n"] * s["b"]
    b = synth.normal(41, 2 * n)
    x = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    cp.cptr_apply_vcycle(g.ctx, 0, dev(b), x)
    assert relerr(host(x), o.vcycle(2, b)) <= 1e-10
    v = synth.normal(42, nb)
    x1 = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_stage1(g.ctx, dev(v), x1)
    assert relerr(host(x1), o.stage1(v)) <= 1e-10
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_precond(g.ctx, dev(v), z)
    assert relerr(host(z), o.precond(v)) <= 1e-10
    if stalls:
        check_iteration_limit(s, o, g, 1e-8, 40)
    else:
        check_solve(s, o, g, 1e-8)


def check_iteration_limit(s, o, g, rtol, max_it):
    """Both sides stop at max_it Arnoldi steps without converging; the iterates agree."""
    x_o, io = o.solve(s["rhs"], rtol)
    x_g, ig = g.solve(dev(s["rhs"].reshape(-1)), rtol)
    assert ig["status"] == "CPTR_NOT_CONVERGED" and not io["converged"]
    assert ig["iters"] == io["iters"] == max_it
    assert abs(ig["true_rel_res"] - io["true_rel_res"]) <= 1e-6 * io["true_rel_res"]
    x_g = host(x_g)
    b = s["b"]
    for u in range(b):
        assert relerr(x_g[u::b], x_o[u::b]) <= 1e-8, (u, relerr(x_g[u::b], x_o[u::b]))
    return io, ig


def test_uamg_full_size_workload():
    """CPTR-uAMG on the benchmark's 600k-unknown workload against the oracle run in full, to a fixed
    limit of 30 Arnoldi steps: on this conduction-dominated workload the unknown-based first stage
    (with PMIS, direct interpolation and l1-Jacobi in place of BoomerAMG's defaults) stalls, on both
    sides alike; the iterates after 30 steps agree."""
    s = system("cptr200k")
    o = oracle.Oracle.from_system(s, stage1=oracle.UAMG, max_it=30, **OPTS["cptr200k"])
    g = gpu_solver(s, stage1=cp.STAGE1["uamg"], max_it=30, **OPTS["cptr200k"])
    io, ig = check_iteration_limit(s, o, g, 1e-6, 30)
    print(f"CPTR-uAMG full size: residual {ig['true_rel_res']:.3e} after 30 steps (oracle "
          f"{io['true_rel_res']:.3e}), {ig['levels_p']} levels")


@pytest.mark.parametrize("name", ["parity", "ragged"])
def test_uamg_mixed_precision(name):
    """Mixed form of CPTR-uAMG: the V-cycle matches the oracle's rounded hierarchy, and the solve
    reaches the FP64 residual."""
    s, o, g = pair(name, stage1=cp.STAGE1["uamg"], precision=1)
    n = s["n"]
    b = synth.normal(43, 2 * n)
    x = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    cp.cptr_apply_vcycle(g.ctx, 0, dev(b), x)
    assert relerr(host(x), o.vcycle(2, b)) <= 1e-5
    xg, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK" and info["true_rel_res"] <= 1.05e-8


@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
def test_schur_diag_hierarchy_and_solve(name):
    """S~_diag formed on the device (column scaling, SpGEMM, union difference) and its hierarchy
    equal the oracle's bit for bit; the solve matches the oracle.  On the conduction-dominated
    "medium" system S~_diag, like A_TT, performs poorly (Sec. 3.3.1) and stalls on both sides: there
    the iterates after a fixed number of steps agree."""
    stalls = name == "medium"
    s, o, g = pair(name, schur=cp.SCHUR["diag"], **(dict(max_it=40) if stalls else {}))
    _bitwise_levels(o.levels(1), g.hierarchy(1))
    if stalls:
        io, ig = check_iteration_limit(s, o, g, 1e-8, 40)
    else:
        io, ig = check_solve(s, o, g, 1e-8)
    assert ig["schur_used"] == "diag"


# ------------------------------------------------------------------------------------------------
# QI / TI decoupling of the CPR and unknown-based first stages (Sec. 3.1, 3.2)
@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium"])
@pytest.mark.parametrize("decouple", ["qi", "ti"])
@pytest.mark.parametrize("stage1", ["cpr", "uamg"])
def test_decoupled_first_stage(name, decouple, stage1):
    """D_i, the fields of G A', the first-stage hierarchy (bit for bit), the decoupled first stage and
    the solve against the oracle.  CPTR-uAMG on the conduction-dominated "medium" system stalls even
    with TI, on both sides: there the iterates after a fixed number of steps agree."""
    stalls = name == "medium" and stage1 == "uamg"
    extra = dict(max_it=20) if stalls else {}
    s, o, g = pair(name, stage1=cp.STAGE1[stage1], decouple=cp.DECOUPLE[decouple], **extra)
    _bitwise_levels(o.levels(2 if stage1 == "uamg" else 0), g.hierarchy(0))
    nb = s["n"] * s["b"]
    v = synth.normal(52, nb)
    x1 = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_stage1(g.ctx, dev(v), x1)
    assert relerr(host(x1), o.stage1(v)) <= 1e-10
    if stalls:   # (20 steps: the stalled Krylov process amplifies rounding step by step)
        check_iteration_limit(s, o, g, 1e-8, 20)
    else:
        check_solve(s, o, g, 1e-8)


def test_decoupling_rejected_with_the_block_preconditioner():
    with pytest.raises(cp.CptrError):
        cp.Solver(stage1="full", decouple="ti")


# ------------------------------------------------------------------------------------------------
# ILU(1) second stage
@pytest.mark.parametrize("name", ["parity", "ragged", "three_phase", "medium", "line"])
@pytest.mark.parametrize("sweep", ["levels", "paired"])
def test_ilu1_apply_and_solve(name, sweep):
    """Block ILU(1) (fill pattern and factors on the device path, the one-launch factorisation and
    sweeps on the filled pattern) against the oracle's scalar ILU(1): applications to 1e-10, solves
    iterations +-1 and 1e-8; CPR-AMG-ILU(1) as in the paper's comparisons."""
    s, o, g = pair(name, ilu_fill=1, ilu_sweep=cp.ILU_SWEEP[sweep])
    nb = s["n"] * s["b"]
    r = synth.normal(55, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, g, 1e-8)
    s, o, g = pair(name, ilu_fill=1, ilu_sweep=cp.ILU_SWEEP[sweep], stage1=cp.STAGE1["cpr"])
    check_solve(s, o, g, 1e-8)


def test_ilu1_mixed_precision_solve():
    s, o, g = pair("medium", ilu_fill=1, precision=1)
    x, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK" and info["true_rel_res"] <= 1.05e-8


def test_ilu1_rejected_where_unsupported():
    with pytest.raises(cp.CptrError):
        cp.Solver(ilu_fill=1, ilu_order="multicolor")
    s, o, g = pair("ragged", ilu_fill=1)
    nb = s["n"] * s["b"]
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_apply_ilu_static(g.ctx, dev(synth.normal(5, nb)), z)
    assert e.value.code == -1


# ------------------------------------------------------------------------------------------------
# the 2-D mesh-refinement workloads (Sec. 4.1.1) with the paper's six methods
MESH_METHODS = (dict(stage1="cpr"), dict(stage1="cpr", decouple="ti"), dict(stage1="cpr", ilu_fill=1),
                dict(stage1="full"), dict(stage1="uamg"), dict(stage1="uamg", decouple="ti"))


@pytest.mark.parametrize("kind", ["wells", "heaters", "aniso"])
@pytest.mark.parametrize("N", [20, 40])
def test_mesh_refinement_methods_match_oracle(kind, N):
    s = synth.mesh_refinement_case(kind, N).system()
    for opts in MESH_METHODS:
        g = gpu_solver(s, **{k: (cp.STAGE1[v] if k == "stage1" else cp.DECOUPLE[v] if k == "decouple" else v)
                             for k, v in opts.items()})
        o = oracle.Oracle.from_system(s, **{k: (cp.STAGE1[v] if k == "stage1" else cp.DECOUPLE[v] if k == "decouple"
                                                else v) for k, v in opts.items()})
        check_solve(s, o, g, 1e-8)


# ------------------------------------------------------------------------------------------------
# failure paths reached from the host, no GPU fault involved
def test_singular_pivot_block_reports_esingular_and_context_recovers():
    """A zero diagonal block in the first cell's row: ILU(0) meets a singular pivot block at set-up
    (CPTR_ESINGULAR); the context then sets up and solves a valid system."""
    s = system("ragged")
    vals = s["vals"].copy()
    rp, ci = s["row_ptr"], s["col_idx"]
    k0 = [k for k in range(rp[0], rp[1]) if ci[k] == 0][0]
    vals[k0] = 0.0
    S = cp.Solver(stage1="none")
    with pytest.raises(cp.CptrError) as e:
        S.setup(s["n"], s["b"], rp, ci, vals.reshape(-1), s["unknown_kind"])
    assert e.value.code == -6, e.value
    S.setup(s["n"], s["b"], rp, ci, s["vals"].reshape(-1), s["unknown_kind"], s["weights"].reshape(-1), s["st"])
    x, info = S.solve(np.ascontiguousarray(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK"


def test_non_finite_rhs_reports_ebreakdown_and_context_recovers():
    """A NaN in the right-hand side makes the Arnoldi process non-finite: CPTR_EBREAKDOWN; the next
    solve of the same set-up converges."""
    s, o, g = pair("ragged")
    rhs = s["rhs"].reshape(-1).copy()
    rhs[7] = np.nan
    with pytest.raises(cp.CptrError) as e:
        g.solve(dev(rhs), 1e-8)
    assert e.value.code == -4, e.value
    check_solve(s, o, g, 1e-8)


# ------------------------------------------------------------------------------------------------
# set-ups of the same pattern with new values (Newton iterations, time steps): the context keeps the
# pattern-only ILU tables (level sets, tile structure, the grouped-level tables' structure) and
# rebuilds everything that holds values
def _setup_again(S, s, vals):
    S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(vals.reshape(-1)), dev(s["unknown_kind"]),
            dev(s["weights"].reshape(-1)), dev(s["st"]))


@pytest.mark.parametrize("sweep", ["levels", "paired", "grouped3", "tiled"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_set_up_again_with_the_same_pattern_or_another(sweep, precision):
    """A context set up before, then set up with new values on the same pattern, and then with a
    different pattern of the same size (an 8 x 6 x 4 box against a 6 x 8 x 4 one: same cell count,
    same block count), gives bit for bit what a fresh context gives each time: ILU applications
    and solves."""
    o = dict(ilu_sweep=cp.ILU_SWEEP[sweep.replace("grouped3", "paired")], precision=cp.PRECISION[precision],
             n_coarse=16, **(dict(ilu_group=3, ilu_lanes=8) if sweep == "grouped3" else {}))
    s1 = synth.make_box(8, 6, 4, 3.125, seed=23, heaters=[(11, 80.0, 420.0)]).system()
    s2 = synth.make_box(6, 8, 4, 3.125, seed=24, heaters=[(13, 80.0, 420.0)]).system()
    assert s1["n"] == s2["n"] and s1["row_ptr"][-1] == s2["row_ptr"][-1]
    assert not np.array_equal(s1["col_idx"], s2["col_idx"])
    rng = np.random.default_rng(6)
    scale = 1.0 + 0.2 * rng.random(s1["n"])
    rows = np.repeat(np.arange(s1["n"]), np.diff(s1["row_ptr"]))
    vals1b = s1["vals"] * scale[rows][:, None, None]
    S = gpu_solver(s1, **o)
    for s, vals in ((s1, vals1b), (s2, s2["vals"]), (s1, s1["vals"])):
        _setup_again(S, s, vals)
        F = cp.Solver(**o)
        _setup_again(F, s, vals)
        if sweep == "tiled":
            assert [r for r in cp.cptr_tuning(S.ctx) if r[2] == 5][0][3] == 3
        nb = s["n"] * s["b"]
        r = dev(np.random.default_rng(7).normal(size=nb))
        za, zb = torch.empty_like(r), torch.empty_like(r)
        cp.cptr_apply_ilu(S.ctx, r, za)
        cp.cptr_apply_ilu(F.ctx, r, zb)
        assert torch.equal(za, zb)
        xa, ia = S.solve(dev(s["rhs"].reshape(-1)), 1e-8)
        xb, ib = F.solve(dev(s["rhs"].reshape(-1)), 1e-8)
        assert ia["status"] == "CPTR_OK" and ia["iters"] == ib["iters"] and torch.equal(xa, xb)
        F.close()


# ------------------------------------------------------------------------------------------------
# block-Jacobi ILU(0) over a partition of the domain (Sec. 4: the paper's parallel second stage)
def quadrants(nx, ny, nz, px, py):
    i = np.arange(nx * ny * nz)
    x, y = i % nx, (i // nx) % ny
    return ((x * px) // nx + px * ((y * py) // ny)).astype(np.int32)


def bj_solver(s, part, dev_part=True, **opts):
    S = cp.Solver(**opts)
    cp.cptr_set_partition(S.ctx, dev(part) if dev_part else part)
    S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
    return S


@pytest.mark.parametrize("sweep", ["levels", "paired"])
def test_block_jacobi_ilu_matches_oracle(sweep):
    """ILU(0) over 4 x 2 parts of the 40 x 40 x 10 box: the factors drop the couplings between parts,
    the level sets shorten to a part's own, applications match the oracle's block-Jacobi ILU(0)
    within the operator tolerance, and solves match the oracle."""
    s = system("medium")
    part = quadrants(40, 40, 10, 4, 2)
    o = oracle.Oracle.from_system(s, part=part, **OPTS["medium"])
    g = bj_solver(s, part, ilu_sweep=cp.ILU_SWEEP[sweep], **OPTS["medium"])
    glob = gpu_solver(s, ilu_sweep=cp.ILU_SWEEP[sweep], **OPTS["medium"])
    nf, nbk = cp.cptr_ilu_levels(g.ctx)
    nf0, nb0 = cp.cptr_ilu_levels(glob.ctx)
    assert (nf, nbk) == (10 + 20 + 10 - 2, 10 + 20 + 10 - 2) and (nf0, nb0) == (40 + 40 + 10 - 2,) * 2, (nf, nf0)
    nb = s["n"] * s["b"]
    r = synth.normal(63, nb)
    z = torch.empty(nb, dtype=torch.float64, device="cuda")
    cp.cptr_apply_ilu(g.ctx, dev(r), z)
    assert relerr(host(z), o.ilu_apply(r)) <= 1e-10
    check_solve(s, o, g, 1e-8)


def test_block_jacobi_ilu_mixed_and_host_partition():
    """The mixed-precision form with a partition given as a host array reaches the FP64 residual;
    removing the partition restores the global ILU(0) (the same solve as a fresh context)."""
    s = system("medium")
    part = quadrants(40, 40, 10, 2, 2)
    g = bj_solver(s, part, dev_part=False, precision=cp.PRECISION["mixed"])
    x, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["status"] == "CPTR_OK" and info["true_rel_res"] <= 1.05e-8
    cp.cptr_set_partition(g.ctx, None)
    g.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
    f = gpu_solver(s, precision=cp.PRECISION["mixed"])
    xa, ia = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    xb, ib = f.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert ia["iters"] == ib["iters"] and torch.equal(xa, xb)


def test_block_jacobi_ilu_rejected_where_unsupported():
    s = system("ragged")
    part = np.zeros(s["n"], np.int32)
    for opts in (dict(ilu_order=1), dict(ilu_fill=1)):
        S = cp.Solver(**opts)
        cp.cptr_set_partition(S.ctx, part)
        with pytest.raises(cp.CptrError) as e:
            S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
                    dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
        assert e.value.code == -1
    S = cp.Solver()
    cp.cptr_set_partition(S.ctx, np.zeros(s["n"] + 1, np.int32))
    with pytest.raises(cp.CptrError) as e:
        S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
                dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]))
    assert e.value.code == -1
