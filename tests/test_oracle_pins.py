"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks one oracle function against something other than itself: a dense factorisation,
a closed form, an invariant, an exact special case, or the minimal-residual property of GMRES.
"""
import numpy as np
import pytest

import oracle
import synth


# ------------------------------------------------------------------------------------------------
# helpers
def dense_csr(rp, ci, v, n, m=None):
    A = np.zeros((n, n if m is None else m))
    for i in range(n):
        np.add.at(A[i], ci[rp[i]:rp[i + 1]], v[rp[i]:rp[i + 1]])
    return A


def poisson3d(nx, ny, nz, shift=None):
    """7-point Laplacian; Dirichlet-like (diagonal 6) unless shift is given, in which case the
    diagonal is the neighbour count (zero row sums) plus shift[i]."""
    n = nx * ny * nz
    rp, ci, v = [0], [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                nb = []
                if z > 0: nb.append(i - nx * ny)
                if y > 0: nb.append(i - nx)
                if x > 0: nb.append(i - 1)
                if x < nx - 1: nb.append(i + 1)
                if y < ny - 1: nb.append(i + nx)
                if z < nz - 1: nb.append(i + nx * ny)
                diag = 6.0 if shift is None else len(nb) + shift[i]
                cols = sorted(nb + [i])
                for c in cols:
                    ci.append(c)
                    v.append(diag if c == i else -1.0)
                rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)


def bsr_dense(s):
    n, b = s["n"], s["b"]
    A = np.zeros((n * b, n * b))
    rp, ci, J = s["row_ptr"], s["col_idx"], s["vals"]
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i * b:(i + 1) * b, ci[k] * b:(ci[k] + 1) * b] = J[k]
    return A


def tiny(nx=5, ny=4, nz=2, **kw):
    return synth.make_box(nx, ny, nz, 3.125, seed=7, **kw)


def pt_blocks(Ad, b, ps=0, ts=1):
    """A_pp, A_pT, A_Tp, A_TT of a dense interleaved matrix."""
    return Ad[ps::b, ps::b], Ad[ps::b, ts::b], Ad[ts::b, ps::b], Ad[ts::b, ts::b]


def strong_sets(lev, theta=0.25):
    """Strength graph S of a level, recomputed from its matrix (for the PMIS invariants)."""
    n, rp, ci, v = lev["n"], lev["rp"], lev["ci"], lev["v"]
    S = []
    for i in range(n):
        cols, vals = ci[rp[i]:rp[i + 1]], v[rp[i]:rp[i + 1]]
        off = cols != i
        m = (-vals[off]).max() if off.any() else 0.0
        S.append(set(cols[off][-vals[off] >= theta * m].tolist()) if m > 0 else set())
    return S


# ------------------------------------------------------------------------------------------------
# decoupling (eqs. weighted, scaling)
def test_weighting_is_a_row_operation():
    r = tiny()
    s = r.system()
    o = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    A = bsr_dense(s)
    Aw = o.dense()
    b = s["rhs"].reshape(-1)
    bw = o.weight_rhs(b)
    # the solution of the weighted system solves the raw one (normwise backward error)
    x2 = np.linalg.solve(Aw, bw)
    assert np.linalg.norm(A @ x2 - b) <= 1e-13 * np.linalg.norm(A, 2) * np.linalg.norm(x2)
    B = s["b"]
    # energy rows untouched, pressure row = T_ref (c_vw water + c_vo oil), kept mass row = c_ref T_ref water
    assert np.array_equal(Aw[1::B], A[1::B])
    pr = r.T0 * (r.cv_w * A[0::B] + r.cv_o * A[2::B])
    assert np.abs(Aw[0::B] - pr).max() <= 1e-14 * np.abs(pr).max()
    cref = 0.8 * r.cv_o + 0.2 * r.cv_w
    assert np.abs(Aw[2::B] - cref * r.T0 * A[0::B]).max() <= 1e-12 * np.abs(Aw[2::B]).max()


# ------------------------------------------------------------------------------------------------
# ILU(0)
def _lu_from_factors(o):
    rp, ci, _ = o.matrix()
    v = o.ilu_factors()
    n = o.nb
    F = dense_csr(rp, ci, v, n)
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    return L, U, rp, ci


def test_ilu0_product_matches_matrix_on_pattern():
    # the defining property of ILU(0): (L U)_ij = a_ij for every (i, j) in the pattern of A
    o = oracle.Oracle.from_system(tiny().system(), max_levels=1, dense_max=4096)
    L, U, rp, ci = _lu_from_factors(o)
    A = o.dense()
    LU = L @ U
    mask = np.zeros_like(A, dtype=bool)
    for i in range(o.nb):
        mask[i, ci[rp[i]:rp[i + 1]]] = True
    assert np.abs((LU - A)[mask]).max() <= 1e-12 * np.abs(A).max()
    assert np.abs((LU - A)[~mask]).max() > 0  # dropped fill exists on a 2D grid


def test_ilu0_solve_applies_lu_inverse():
    o = oracle.Oracle.from_system(tiny().system(), max_levels=1, dense_max=4096)
    L, U, _, _ = _lu_from_factors(o)
    r = synth.normal(5, o.nb)
    z = o.ilu_apply(r)
    assert np.linalg.norm(L @ (U @ z) - r) <= 1e-10 * np.linalg.norm(r)


def test_ilu0_exact_on_a_line():
    # a 1D grid has a block-tridiagonal Jacobian: ILU(0) has no dropped fill, so it is exact LU
    o = oracle.Oracle.from_system(synth.make_box(12, 1, 1, 3.125, seed=3).system(), max_levels=1)
    A = o.dense()
    r = synth.normal(6, o.nb)
    assert np.linalg.norm(o.ilu_apply(r) - np.linalg.solve(A, r)) <= 1e-9 * np.linalg.norm(np.linalg.solve(A, r))


def test_scalar_ilu0_equals_block_ilu0():
    # with dense b x b blocks, scalar ILU(0) in cell-major order equals block ILU(0) with exact
    # pivot-block inverses; the block form is written here from the textbook definition
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    n, b = s["n"], s["b"]
    rp, ci = s["row_ptr"], s["col_idx"]
    W = s["weights"]
    blocks = {}
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            blocks[(i, int(ci[k]))] = W[i] @ s["vals"][k]
    for i in range(n):
        row = [int(c) for c in ci[rp[i]:rp[i + 1]]]
        for k in [c for c in row if c < i]:
            blocks[(i, k)] = blocks[(i, k)] @ np.linalg.inv(blocks[(k, k)])
            for j in [c for c in row if c > k]:
                if (k, j) in blocks:
                    blocks[(i, j)] = blocks[(i, j)] - blocks[(i, k)] @ blocks[(k, j)]
    r = synth.normal(8, n * b).reshape(n, b)
    y = np.zeros((n, b))
    for i in range(n):
        y[i] = r[i] - sum(blocks[(i, int(k))] @ y[k] for k in ci[rp[i]:rp[i + 1]] if k < i)
    z = np.zeros((n, b))
    for i in reversed(range(n)):
        t = y[i] - sum(blocks[(i, int(k))] @ z[k] for k in ci[rp[i]:rp[i + 1]] if k > i)
        z[i] = np.linalg.solve(blocks[(i, i)], t)
    zo = o.ilu_apply(r.reshape(-1))
    assert np.linalg.norm(zo - z.reshape(-1)) <= 1e-10 * np.linalg.norm(z)


# ------------------------------------------------------------------------------------------------
# AMG
def test_splitmix64_in_oracle():
    assert [oracle.splitmix64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def pmis_reference(S, seed):
    """Brute-force PMIS from its definition (De Sterck, Yang, Heys 2006) on Python sets: each
    round, undecided points whose key (|S^T_i|, top 32 bits of SplitMix64(seed, i), index) beats
    every undecided neighbour in S_i or S^T_i become C; undecided points that strongly depend on a
    C point become F; points with no strong connection at all are F from the start."""
    n = len(S)
    ST = [set() for _ in range(n)]
    for i in range(n):
        for j in S[i]:
            ST[j].add(i)
    h = synth.splitmix64(seed, n) >> np.uint64(32)
    key = [(len(ST[i]), int(h[i]), i) for i in range(n)]
    state = ["F" if not S[i] and not ST[i] else "U" for i in range(n)]
    while "U" in state:
        new = [i for i in range(n) if state[i] == "U"
               and all(key[i] > key[j] for j in S[i] | ST[i] if state[j] == "U")]
        for i in new:
            state[i] = "C"
        for i in range(n):
            if state[i] == "U" and any(state[j] == "C" for j in S[i]):
                state[i] = "F"
    return np.array([1 if t == "C" else 2 for t in state])


@pytest.mark.parametrize("source", ["poisson", "App", "St"])
def test_pmis_splitting(source):
    if source == "poisson":
        levels = oracle.AMG(*poisson3d(10, 10, 6), n_coarse=10).levels()
    else:
        s = synth.recipe("parity").system()
        levels = oracle.Oracle.from_system(s).levels(0 if source == "App" else 1)
    assert len(levels) >= 2
    for l, lev in enumerate(levels[:-1]):
        S = strong_sets(lev)
        cf = lev["cf"]
        assert np.array_equal(cf, pmis_reference(S, l))
        for i in range(lev["n"]):
            if cf[i] == 2 and S[i]:   # every F point with strong couplings has a strong C neighbour
                assert any(cf[j] == 1 for j in S[i]), i
        assert 0 < (cf == 1).sum() < lev["n"]


@pytest.mark.parametrize("source", ["poisson", "App", "St"])
def test_galerkin_coarse_operator(source):
    if source == "poisson":
        levels = oracle.AMG(*poisson3d(8, 8, 6), n_coarse=20).levels()
    else:
        s = synth.recipe("parity").system()
        levels = oracle.Oracle.from_system(s).levels(0 if source == "App" else 1)
    for l in range(len(levels) - 1):
        f, c = levels[l], levels[l + 1]
        A = dense_csr(f["rp"], f["ci"], f["v"], f["n"])
        P = dense_csr(f["Prp"], f["Pci"], f["Pv"], f["n"], f["nc"])
        Ac = dense_csr(c["rp"], c["ci"], c["v"], c["n"])
        ref = P.T @ A @ P
        assert np.abs(Ac - ref).max() <= 1e-13 * np.abs(ref).max()
        # C points inject: their P row is a single 1 at their coarse index, numbered in order
        cidx = np.cumsum(f["cf"] == 1) - 1
        for i in np.nonzero(f["cf"] == 1)[0]:
            assert P[i, cidx[i]] == 1.0 and np.count_nonzero(P[i]) == 1


def test_direct_interpolation_preserves_constants():
    # zero row sums on all rows but a few: F rows with zero row sum interpolate constants exactly
    nx, ny, nz = 9, 8, 5
    shift = np.zeros(nx * ny * nz)
    shift[[0, 100, 250]] = 1.0
    rp, ci, v = poisson3d(nx, ny, nz, shift)
    lev = oracle.AMG(rp, ci, v, n_coarse=10).levels()[0]
    P = dense_csr(lev["Prp"], lev["Pci"], lev["Pv"], lev["n"], lev["nc"])
    rowsum = P.sum(axis=1)
    zero_rows = np.abs(dense_csr(rp, ci, v, lev["n"]).sum(axis=1)) == 0
    F = (lev["cf"] == 2) & zero_rows & (np.count_nonzero(P, axis=1) > 0)
    assert F.sum() > 50
    assert np.abs(rowsum[F] - 1.0).max() <= 1e-14


def test_direct_interpolation_weights_closed_form():
    # F point 0 with strong C neighbours 1, 2 (a = -1.5, -1), a weak negative neighbour 3
    # (a = -0.1) and a positive neighbour 4 (a = +0.2), diagonal 4:
    #   alpha = (-1.5 - 1 - 0.1) / (-1.5 - 1), d = 4 + 0.2, w_0j = -alpha a_0j / d
    # points 1 and 2 are made C by giving each three more points (5-7, 8-10) that depend on them
    rows = {0: {0: 4.0, 1: -1.5, 2: -1.0, 3: -0.1, 4: 0.2},
            1: {0: -0.01, 1: 4.0, 5: -1.0, 6: -1.0, 7: -1.0},
            2: {0: -0.01, 2: 4.0, 8: -1.0, 9: -1.0, 10: -1.0},
            3: {0: -0.1, 3: 4.0}, 4: {0: 0.2, 4: 4.0}}
    for leaf, c in ((5, 1), (6, 1), (7, 1), (8, 2), (9, 2), (10, 2)):
        rows[leaf] = {c: -1.0, leaf: 4.0}
    rp, ci, v = [0], [], []
    for i in range(11):
        for j in sorted(rows[i]):
            ci.append(j)
            v.append(rows[i][j])
        rp.append(len(ci))
    lev = oracle.AMG(np.array(rp), np.array(ci), np.array(v), n_coarse=1, max_levels=2).levels()[0]
    cf = lev["cf"]
    assert cf[1] == 1 and cf[2] == 1 and cf[0] == 2, cf
    P = dense_csr(lev["Prp"], lev["Pci"], lev["Pv"], 11, lev["nc"])
    cidx = np.cumsum(cf == 1) - 1
    alpha = (-1.5 - 1.0 - 0.1) / (-1.5 - 1.0)
    assert abs(P[0, cidx[1]] - (-alpha * -1.5 / 4.2)) < 1e-15
    assert abs(P[0, cidx[2]] - (-alpha * -1.0 / 4.2)) < 1e-15
    assert np.count_nonzero(P[0]) == 2


def test_single_level_vcycle_is_exact():
    rp, ci, v = poisson3d(6, 5, 4)
    h = oracle.AMG(rp, ci, v, max_levels=1, dense_max=4096)
    b = synth.normal(3, 120)
    A = dense_csr(rp, ci, v, 120)
    assert np.linalg.norm(h.vcycle(b) - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(np.linalg.solve(A, b))


@pytest.mark.parametrize("smoother", [oracle.L1, oracle.JACOBI])
def test_vcycle_converges_on_poisson(smoother):
    # textbook behaviour (not a paper number): V(1,1) as a stationary iteration on 3D Poisson
    rp, ci, v = poisson3d(16, 16, 16)
    n = 16 ** 3
    A = dense_csr(rp, ci, v, n)
    h = oracle.AMG(rp, ci, v, n_coarse=50, smoother=smoother)
    assert len(h.levels()) >= 3
    b = np.zeros(n)
    x = synth.normal(4, n)
    e0 = np.linalg.norm(x)
    k = 8
    for _ in range(k):
        x = x + h.vcycle(b - A @ x)
    rho = (np.linalg.norm(x) / e0) ** (1.0 / k)
    assert rho < 0.5, rho


def test_smoother_diagonals():
    rp, ci, v = poisson3d(5, 4, 3)
    lev = oracle.AMG(rp, ci, v, max_levels=1).levels()[0]
    A = dense_csr(rp, ci, v, 60)
    assert np.allclose(lev["dinv"], 1.0 / np.abs(A).sum(axis=1), rtol=1e-15)
    lev = oracle.AMG(rp, ci, v, max_levels=1, smoother=oracle.JACOBI).levels()[0]
    assert np.allclose(lev["dinv"], (2.0 / 3.0) / np.diag(A), rtol=1e-15)


# ------------------------------------------------------------------------------------------------
# the block preconditioner for A_00 (eqs. Afact, Ainv, Aschur) and the two-stage combination
def _exact_setup(r, mode, st="given"):
    s = r.system()
    n, b = s["n"], s["b"]
    o0 = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    Ad = o0.dense()
    App, ApT, ATp, ATT = pt_blocks(Ad, b)
    S_exact = ATT - ATp @ np.linalg.solve(App, ApT)
    if st == "exact":
        full_rp = np.arange(0, n * n + 1, n, dtype=np.int32)
        full_ci = np.tile(np.arange(n, dtype=np.int32), n)
        o = oracle.Oracle(n, b, s["row_ptr"], s["col_idx"], s["vals"], s["weights"], st=S_exact.reshape(-1),
                          st_pattern=(full_rp, full_ci), stage1=mode, max_levels=1, dense_max=4096)
        St = S_exact
    else:
        o = oracle.Oracle.from_system(s, stage1=mode, max_levels=1, dense_max=4096)
        St = dense_csr(s["row_ptr"], s["col_idx"], s["st"], n)
    return s, o, Ad, (App, ApT, ATp, ATT), St


def test_exact_inner_solves_give_exact_block_inverse():
    # eqs. (Afact)/(Ainv): with exact A_pp^{-1} and S~_T = S_T the five steps apply A_00^{-1}
    r = tiny()
    s, o, Ad, (App, ApT, ATp, ATT), St = _exact_setup(r, oracle.CPTR_FULL, st="exact")
    n, b = s["n"], s["b"]
    A00 = np.block([[App, ApT], [ATp, ATT]])
    M1 = np.zeros((2 * n, 2 * n))
    for c in range(2 * n):
        v = np.zeros(n * b)
        v[(c % n) * b + (c // n)] = 1.0
        x1 = o.stage1(v).reshape(n, b)
        M1[:, c] = np.concatenate([x1[:, 0], x1[:, 1]])
        assert np.all(x1[:, 2:] == 0.0)
    assert np.abs(M1 @ A00 - np.eye(2 * n)).max() <= 1e-8


@pytest.mark.parametrize("mode", [oracle.CPTR_FULL, oracle.CPTR_LOWER, oracle.CPTR_UPPER, oracle.BD, oracle.CPR])
def test_stage1_matches_factored_form(mode):
    # eq. (Aschur) with exact A_pp^{-1} and the given S~_T; triangular variants drop a factor
    r = tiny()
    s, o, Ad, (App, ApT, ATp, ATT), St = _exact_setup(r, mode)
    n, b = s["n"], s["b"]
    I, Z = np.eye(n), np.zeros((n, n))
    Ai, Si = np.linalg.inv(App), np.linalg.inv(St)
    left = np.block([[I, -Ai @ ApT], [Z, I]])
    mid = np.block([[Ai, Z], [Z, Si]])
    right = np.block([[I, Z], [-ATp @ Ai, I]])
    ref = {oracle.CPTR_FULL: left @ mid @ right, oracle.CPTR_LOWER: mid @ right, oracle.CPTR_UPPER: left @ mid,
           oracle.BD: mid, oracle.CPR: np.block([[Ai, Z], [Z, Z]])}[mode]
    v = synth.normal(11, n * b)
    x1 = o.stage1(v).reshape(n, b)
    vv = v.reshape(n, b)
    want = ref @ np.concatenate([vv[:, 0], vv[:, 1]])
    got = np.concatenate([x1[:, 0], x1[:, 1]])
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


def test_schur_complement_invariant_to_pressure_row_scaling():
    # S_T = A_TT - A_Tp A_pp^{-1} A_pT does not change when the pressure row is rescaled
    s = tiny().system()
    b = s["b"]
    out = []
    for scale in (1.0, 7.3):
        W = s["weights"].copy()
        W[:, 0, :] *= scale
        o = oracle.Oracle(s["n"], b, s["row_ptr"], s["col_idx"], s["vals"], W, st=s["st"], max_levels=1, dense_max=4096)
        App, ApT, ATp, ATT = pt_blocks(o.dense(), b)
        out.append(ATT - ATp @ np.linalg.solve(App, ApT))
    assert np.abs(out[0] - out[1]).max() <= 1e-10 * np.abs(out[0]).max()


def test_schur_approximation_conditioning_trend():
    # Table (tab:conds) trend: S~_T of eq. (Se) is a much better approximation of S_T than A_TT
    r = synth.make_box(8, 8, 1, 3.125, seed=12, heaters=[(9, 200.0, 450.0), (54, 200.0, 450.0)], dt=86400.0 * 30)
    s = r.system()
    o = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    App, ApT, ATp, ATT = pt_blocks(o.dense(), s["b"])
    S = ATT - ATp @ np.linalg.solve(App, ApT)
    St = dense_csr(s["row_ptr"], s["col_idx"], s["st"], s["n"])
    Sdiag = ATT - ATp @ np.diag(1.0 / np.diag(App)) @ ApT

    def kappa(M):
        ev = np.abs(np.linalg.eigvals(np.linalg.solve(M, S)))
        return ev.max() / ev.min()

    k_st, k_att, k_diag = kappa(St), kappa(ATT), kappa(Sdiag)
    assert k_st < 3.0
    assert k_st <= k_att and k_st <= k_diag


def test_two_stage_formula():
    # M^{-1} = M2^{-1} (I - A M1^{-1}) + M1^{-1}   (Sec. 3, two-stage preconditioners)
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, max_levels=2, n_coarse=4)
    nb = o.nb
    A = o.dense()
    E = np.eye(nb)
    M1 = np.column_stack([o.stage1(E[:, c]) for c in range(nb)])
    M2 = np.column_stack([o.ilu_apply(E[:, c]) for c in range(nb)])
    M = M2 @ (np.eye(nb) - A @ M1) + M1
    v = synth.normal(13, nb)
    assert np.linalg.norm(o.precond(v) - M @ v) <= 1e-10 * np.linalg.norm(M @ v)


def test_exact_two_stage_converges_in_one_iteration():
    # 1D grid: ILU(0) is exact LU, so the two-stage preconditioner is A^{-1} for any first stage
    s = synth.make_box(16, 1, 1, 3.125, seed=4).system()
    for mode in (oracle.CPTR_FULL, oracle.CPR):
        o = oracle.Oracle.from_system(s, stage1=mode, max_levels=2, n_coarse=4)
        x, info = o.solve(s["rhs"], 1e-10)
        assert info["converged"] and info["iters"] == 1, info


# ------------------------------------------------------------------------------------------------
# FGMRES
def test_fgmres_solution_matches_dense_solve():
    s = tiny(6, 5, 3).system()
    o = oracle.Oracle.from_system(s, max_levels=2, n_coarse=8)
    x, info = o.solve(s["rhs"], 1e-10)
    A = o.dense()
    xs = np.linalg.solve(A, o.weight_rhs(s["rhs"].reshape(-1)))
    kappa = np.linalg.cond(A)
    assert info["converged"] and info["true_rel_res"] <= 1e-10 * 1.01
    assert np.linalg.norm(x - xs) <= kappa * 1e-10 * np.linalg.norm(xs)
    assert abs(info["true_rel_res"] - info["est_rel_res"]) <= 1e-3 * info["est_rel_res"] + 1e-14


@pytest.mark.parametrize("mode", [oracle.NONE1, oracle.CPTR_FULL])
def test_gmres_minimal_residual_property(mode):
    # after k steps without restart the residual is min over x in M^{-1} K_k(A M^{-1}, b)
    s = tiny(5, 4, 2).system()
    k = 6
    stage2 = oracle.NONE2 if mode == oracle.NONE1 else oracle.ILU0
    o = oracle.Oracle.from_system(s, stage1=mode, stage2=stage2, max_levels=2, n_coarse=4, max_it=k, restart=30)
    x, info = o.solve(s["rhs"], 1e-30)
    assert info["iters"] == k and not info["converged"]
    nb = o.nb
    A = o.dense()
    Mi = np.column_stack([o.precond(np.eye(nb)[:, c]) for c in range(nb)])
    B = A @ Mi
    b = o.weight_rhs(s["rhs"].reshape(-1))
    K = np.zeros((nb, k))
    v = b / np.linalg.norm(b)
    for j in range(k):
        K[:, j] = v
        v = B @ v
        v = v / np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(B @ Q, b, rcond=None)
    rmin = np.linalg.norm(b - B @ Q @ y) / np.linalg.norm(b)
    assert abs(info["true_rel_res"] - rmin) <= 1e-6 * rmin
    assert abs(info["est_rel_res"] - rmin) <= 1e-6 * rmin


def test_identity_preconditioner_restarted_gmres():
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, stage1=oracle.NONE1, stage2=oracle.ILU0, restart=5, max_it=2000)
    x, info = o.solve(s["rhs"], 1e-9)
    assert info["converged"] and info["restarts"] >= 1
    A = o.dense()
    xs = np.linalg.solve(A, o.weight_rhs(s["rhs"].reshape(-1)))
    assert np.linalg.norm(A @ x - A @ xs) <= 1.01e-9 * np.linalg.norm(A @ xs)


def test_zero_rhs_returns_zero():
    s = tiny(3, 3, 1).system()
    o = oracle.Oracle.from_system(s, max_levels=1)
    x, info = o.solve(np.zeros(o.nb), 1e-8)
    assert info["converged"] and info["iters"] == 0 and not x.any()


def test_cptr_needs_fewer_iterations_than_cpr_when_conduction_dominates():
    # trend of Tables (tab:meshW)-(tab:anisomeshW): with heat diffusion dominant CPTR beats CPR
    r = synth.make_box(24, 24, 4, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1, kT_const=2.0,
                       T_inj=500.0, q_inj=1e-6, dt=365 * 86400.0)
    s = r.system()
    its = {}
    for mode in (oracle.CPTR_FULL, oracle.CPR):
        x, info = oracle.Oracle.from_system(s, stage1=mode, n_coarse=64).solve(s["rhs"], 1e-6)
        assert info["converged"]
        its[mode] = info["iters"]
    assert its[oracle.CPTR_FULL] < its[oracle.CPR], its


# ------------------------------------------------------------------------------------------------
# multicolour ordering of ILU(0) (a reading: the paper does not state the ILU ordering)
def test_multicolour_order_is_red_black_on_a_grid():
    r = tiny(5, 4, 3)
    o = oracle.Oracle.from_system(r.system(), max_levels=1, ilu_order=1)
    order = o.ilu_order()
    idx = np.arange(r.n)
    x, y, z = idx % r.nx, (idx // r.nx) % r.ny, idx // (r.nx * r.ny)
    parity = (x + y + z) % 2
    assert np.array_equal(order, np.concatenate([idx[parity == 0], idx[parity == 1]]))


def _block_ilu_solve(s, order, rvec):
    """Textbook block ILU(0) of the cell-permuted system, then the solve, in original order."""
    n, b = s["n"], s["b"]
    rp, ci, W = s["row_ptr"], s["col_idx"], s["weights"]
    inv = np.empty(n, int)
    inv[order] = np.arange(n)
    blocks, rows = {}, []
    for I in range(n):
        i = order[I]
        cols = []
        for k in range(rp[i], rp[i + 1]):
            J = int(inv[ci[k]])
            blocks[(I, J)] = W[i] @ s["vals"][k]
            cols.append(J)
        rows.append(sorted(cols))
    for I in range(n):
        for K in [c for c in rows[I] if c < I]:
            blocks[(I, K)] = blocks[(I, K)] @ np.linalg.inv(blocks[(K, K)])
            for J in [c for c in rows[I] if c > K]:
                if (K, J) in blocks:
                    blocks[(I, J)] = blocks[(I, J)] - blocks[(I, K)] @ blocks[(K, J)]
    rr = rvec.reshape(n, b)[order]
    yv = np.zeros((n, b))
    for I in range(n):
        yv[I] = rr[I] - sum(blocks[(I, K)] @ yv[K] for K in rows[I] if K < I)
    zv = np.zeros((n, b))
    for I in reversed(range(n)):
        t = yv[I] - sum(blocks[(I, K)] @ zv[K] for K in rows[I] if K > I)
        zv[I] = np.linalg.solve(blocks[(I, I)], t)
    out = np.zeros((n, b))
    out[order] = zv
    return out.reshape(-1)


def test_multicolour_ilu0_equals_block_ilu0_of_permuted_system():
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096, ilu_order=1)
    r = synth.normal(8, s["n"] * s["b"])
    ref = _block_ilu_solve(s, o.ilu_order(), r)
    assert np.linalg.norm(o.ilu_apply(r) - ref) <= 1e-10 * np.linalg.norm(ref)
    # and it is a different operator from the natural-order ILU(0)
    o0 = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    assert np.linalg.norm(o0.ilu_apply(r) - ref) > 1e-6 * np.linalg.norm(ref)


def test_multicolour_cptr_converges():
    s = synth.recipe("parity").system()
    x, info = oracle.Oracle.from_system(s, max_levels=2, ilu_order=1).solve(s["rhs"], 1e-8)
    assert info["converged"] and info["true_rel_res"] <= 1e-8


# ------------------------------------------------------------------------------------------------
# storage rounding of the mixed-precision form
def test_bf16_rounding_closed_forms():
    # bf16 keeps 8 significant bits: spacing 2^-7 in [1, 2); round to nearest, ties to even
    assert oracle.round_bf16(1.0) == 1.0
    assert oracle.round_bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0)
    assert oracle.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7  # tie -> even (odd neighbour up)
    assert oracle.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert oracle.round_bf16(-3.0) == -3.0
    assert oracle.round_bf16(2.0 ** -130) > 0.0                          # subnormal range survives
    for x in synth.normal(3, 1000) * 1e3:
        y = oracle.round_bf16(float(x))
        assert abs(y - x) <= 2.0 ** -8 * abs(x)   # unit roundoff of 8 significant bits


def test_mixed_precision_oracle_rounds_the_hierarchy():
    s = synth.recipe("parity").system()
    o64 = oracle.Oracle.from_system(s, n_coarse=8)
    o16 = oracle.Oracle.from_system(s, n_coarse=8, precision=1)
    l64, l16 = o64.levels(0), o16.levels(0)
    assert len(l64) == len(l16) >= 3
    for l, (a, b) in enumerate(zip(l64, l16)):
        assert np.array_equal(a["ci"], b["ci"])          # same hierarchy, rounded values
        rounded = np.array([oracle.round_bf16(v) for v in a["v"]]) if l >= 2 else a["v"].astype(np.float32).astype(np.float64)
        assert np.array_equal(b["v"], rounded)
    x, info = o16.solve(s["rhs"], 1e-8)
    x64, i64 = o64.solve(s["rhs"], 1e-8)
    assert info["converged"] and abs(info["iters"] - i64["iters"]) <= 2


# ------------------------------------------------------------------------------------------------
# ensemble: FGMRES on one diagonal block of a block-diagonal union
def test_block_solve_of_the_whole_system_is_the_solve():
    s = tiny().system()
    o = oracle.Oracle.from_system(s, n_coarse=16)
    x1, i1 = o.solve(s["rhs"], 1e-10)
    x2, i2 = o.solve_block(0, s["n"], s["rhs"], 1e-10)
    assert i1["iters"] == i2["iters"] and np.array_equal(x1, x2)


def test_block_solve_without_preconditioner_is_the_instance_gmres():
    """With no first and no second stage the preconditioner is the identity, so FGMRES on a block
    of the union is GMRES on the instance alone: the same iterates up to rounding."""
    a = synth.make_box(5, 4, 2, 3.125, seed=3).system()
    c = synth.make_box(3, 6, 2, 3.125, seed=5).system()
    U = synth.concat([a, c])
    opts = dict(stage1=oracle.NONE1, stage2=oracle.NONE2, restart=8)
    ou = oracle.Oracle.from_system(U, **opts)
    for k, s in enumerate((a, c)):
        x_b, i_b = ou.solve_block(int(U["cell0"][k]), s["n"], s["rhs"], 1e-9)
        x_s, i_s = oracle.Oracle.from_system(s, **opts).solve(s["rhs"], 1e-9)
        assert i_b["iters"] == i_s["iters"]
        np.testing.assert_allclose(x_b, x_s, rtol=1e-12, atol=1e-12 * np.abs(x_s).max())


def test_union_preconditioner_is_block_diagonal():
    a = synth.make_box(5, 4, 2, 3.125, seed=3).system()
    c = synth.make_box(3, 6, 2, 3.125, seed=5).system()
    U = synth.concat([a, c])
    ou = oracle.Oracle.from_system(U, n_coarse=8)
    nb0 = a["n"] * a["b"]
    v = np.zeros(U["n"] * U["b"])
    v[:nb0] = np.random.default_rng(1).normal(size=nb0)
    z = ou.precond(v)
    assert np.all(z[nb0:] == 0.0)
    with pytest.raises(ValueError):
        ou.solve_block(1, a["n"], a["rhs"], 1e-8)     # a range that cuts through the coupling


# ------------------------------------------------------------------------------------------------
# Paired levels (the evaluation order of the GPU's ILU(0) sweeps, not a separate method): a row
# of odd level substitutes its dependencies of the level before.  Written here from the algebra
# of the two triangular solves, on textbook block ILU(0) factors, and checked against the plain
# substitution on a random block pattern (dependencies one and several levels back) and on the
# oracle's own ILU solve.
def _block_ilu_factors(n, b, pattern, blocks):
    """Textbook block ILU(0): L_ik = A_ik D_k^-1 (i > k), U_ij (i < j), D_i, in place."""
    F = {key: val.copy() for key, val in blocks.items()}
    for i in range(n):
        row = sorted(pattern[i])
        for k in [c for c in row if c < i]:
            F[(i, k)] = F[(i, k)] @ np.linalg.inv(F[(k, k)])
            for j in [c for c in row if c > k]:
                if (k, j) in F:
                    F[(i, j)] = F[(i, j)] - F[(i, k)] @ F[(k, j)]
    return F


def _levels(n, deps):
    lev = np.zeros(n, int)
    order = range(n) if all(k < i for i in range(n) for k in deps[i]) else reversed(range(n))
    for i in order:
        lev[i] = 1 + max((lev[k] for k in deps[i]), default=-1)
    return lev


def _paired_solves(n, b, pattern, F, r):
    lower = [[k for k in sorted(pattern[i]) if k < i] for i in range(n)]
    upper = [[k for k in sorted(pattern[i]) if k > i] for i in range(n)]
    lf, lb = _levels(n, lower), _levels(n, upper)
    Dinv = {i: np.linalg.inv(F[(i, i)]) for i in range(n)}
    y, ready = np.full((n, b), np.nan), np.full(n, -1)
    for L in range(lf.max() + 1):
        for i in np.flatnonzero(lf == L):
            if L % 2 == 0:
                y[i] = r[i] - sum(F[(i, k)] @ y[k] for k in lower[i])
            else:
                K1 = [k for k in lower[i] if lf[k] == L - 1]
                K0 = [k for k in lower[i] if lf[k] != L - 1]
                c = r[i] - sum((F[(i, k)] @ r[k] for k in K1), np.zeros(b))
                js = sorted(set(K0) | {j for k in K1 for j in lower[k]})
                for j in js:
                    assert lf[j] <= L - 2          # only rows of earlier steps are needed
                    M = F[(i, j)].copy() if j in K0 else np.zeros((b, b))
                    M -= sum((F[(i, k)] @ F[(k, j)] for k in K1 if j in lower[k]), np.zeros((b, b)))
                    c = c - M @ y[j]
                y[i] = c
            ready[i] = L
    z = np.full((n, b), np.nan)
    for L in range(lb.max() + 1):
        for i in np.flatnonzero(lb == L):
            if L % 2 == 0:
                z[i] = Dinv[i] @ (y[i] - sum((F[(i, k)] @ z[k] for k in upper[i]), np.zeros(b)))
            else:
                K1 = [k for k in upper[i] if lb[k] == L - 1]
                K0 = [k for k in upper[i] if lb[k] != L - 1]
                P = {k: F[(i, k)] @ Dinv[k] for k in K1}
                c = y[i] - sum((P[k] @ y[k] for k in K1), np.zeros(b))
                for j in sorted(set(K0) | {j for k in K1 for j in upper[k]}):
                    assert lb[j] <= L - 2
                    M = F[(i, j)].copy() if j in K0 else np.zeros((b, b))
                    M -= sum((P[k] @ F[(k, j)] for k in K1 if j in upper[k]), np.zeros((b, b)))
                    c = c - M @ z[j]
                z[i] = Dinv[i] @ c
    return y, z


def _plain_solves(n, b, pattern, F, r):
    y = np.zeros((n, b))
    for i in range(n):
        y[i] = r[i] - sum((F[(i, k)] @ y[k] for k in pattern[i] if k < i), np.zeros(b))
    z = np.zeros((n, b))
    for i in reversed(range(n)):
        z[i] = np.linalg.solve(F[(i, i)], y[i] - sum((F[(i, k)] @ z[k] for k in pattern[i] if k > i), np.zeros(b)))
    return y, z


def test_paired_levels_equal_plain_substitution_random_pattern():
    rng = np.random.default_rng(7)
    n, b = 60, 3
    pattern = [{i} for i in range(n)]
    for i in range(n):
        for j in rng.choice(n, size=3, replace=False):
            if j != i and abs(int(j) - i) <= 12:
                pattern[i].add(int(j))
                pattern[int(j)].add(i)
    blocks = {}
    for i in range(n):
        for j in pattern[i]:
            blocks[(i, j)] = rng.normal(size=(b, b)) * (0.3 if j != i else 1.0)
        blocks[(i, i)] += 4.0 * b * np.eye(b)
    F = _block_ilu_factors(n, b, pattern, blocks)
    lower = [[k for k in pattern[i] if k < i] for i in range(n)]
    lf = _levels(n, lower)
    # the pattern has dependencies more than one level back (K0 non-empty somewhere)
    assert any(lf[k] < lf[i] - 1 for i in range(n) for k in lower[i])
    r = rng.normal(size=(n, b))
    y0, z0 = _plain_solves(n, b, pattern, F, r)
    y1, z1 = _paired_solves(n, b, pattern, F, r)
    assert np.linalg.norm(y1 - y0) <= 1e-12 * np.linalg.norm(y0)
    assert np.linalg.norm(z1 - z0) <= 1e-12 * np.linalg.norm(z0)


def test_paired_levels_equal_oracle_ilu_on_a_grid():
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    n, b = s["n"], s["b"]
    rp, ci, W = s["row_ptr"], s["col_idx"], s["weights"]
    pattern = [set(int(c) for c in ci[rp[i]:rp[i + 1]]) for i in range(n)]
    blocks = {(i, int(ci[k])): W[i] @ s["vals"][k] for i in range(n) for k in range(rp[i], rp[i + 1])}
    F = _block_ilu_factors(n, b, pattern, blocks)
    r = synth.normal(9, n * b).reshape(n, b)
    _, z = _paired_solves(n, b, pattern, F, r)
    zo = o.ilu_apply(r.reshape(-1))
    assert np.linalg.norm(zo - z.reshape(-1)) <= 1e-10 * np.linalg.norm(zo)


# Grouped levels, the generalisation of the pairs above: the levels of a sweep in groups of g, a
# row substituting the equations of its dependencies inside its group (recursively, through chains
# of up to g - 1 links), so that it depends only on rows of earlier groups.  Written from the
# algebra: with F_ik = L_ik forward, and U_ik D_k^-1 backward for k inside the group (U_ik outside),
#   M_ij = [j outside] F_ij - sum_{k inside} F_ik M_kj,   W_il = [l inside] F_il - sum_{k inside} F_ik W_kl,
#   y_i = r_i - sum_l W_il r_l - sum_j M_ij y_j,   z_i = D_i^-1 (y_i - sum_l W_il y_l - sum_j M_ij z_j).
def _grouped_solves(n, b, pattern, F, r, g, drop_second_order=False):
    lower = [[k for k in sorted(pattern[i]) if k < i] for i in range(n)]
    upper = [[k for k in sorted(pattern[i]) if k > i] for i in range(n)]
    Dinv = {i: np.linalg.inv(F[(i, i)]) for i in range(n)}

    def expansions(deps, lev, backward):
        E = {}
        for L in range(lev.max() + 1):
            G0 = L - L % g
            for i in np.flatnonzero(lev == L):
                M, W = {}, {}
                for k in deps[i]:
                    if lev[k] < G0:
                        M[k] = M.get(k, 0) + F[(i, k)]
                        continue
                    f = F[(i, k)] @ Dinv[k] if backward else F[(i, k)]
                    W[k] = W.get(k, 0) + f
                    Mk, Wk = E[k]
                    for j, blk in Mk.items():
                        M[j] = M.get(j, 0) - f @ blk
                    if not drop_second_order:
                        for l, blk in Wk.items():
                            W[l] = W.get(l, 0) - f @ blk
                assert all(lev[j] < G0 for j in M) and all(G0 <= lev[l] < L for l in W)
                E[i] = (M, W)
        return E

    lf, lb = _levels(n, lower), _levels(n, upper)
    Ef, Eb = expansions(lower, lf, False), expansions(upper, lb, True)
    y = np.full((n, b), np.nan)
    for G0 in range(0, lf.max() + 1, g):   # a group at a time; only earlier groups' y are read
        grp = np.flatnonzero((lf >= G0) & (lf < G0 + g))
        new = {i: r[i] - sum((w @ r[l] for l, w in Ef[i][1].items()), np.zeros(b))
               - sum((m @ y[j] for j, m in Ef[i][0].items()), np.zeros(b)) for i in grp}
        for i, v in new.items():
            y[i] = v
    z = np.full((n, b), np.nan)
    for G0 in range(0, lb.max() + 1, g):
        grp = np.flatnonzero((lb >= G0) & (lb < G0 + g))
        new = {i: Dinv[i] @ (y[i] - sum((w @ y[l] for l, w in Eb[i][1].items()), np.zeros(b))
                             - sum((m @ z[j] for j, m in Eb[i][0].items()), np.zeros(b))) for i in grp}
        for i, v in new.items():
            z[i] = v
    return y, z


def _random_factors(n, b, seed, reach=12):
    rng = np.random.default_rng(seed)
    pattern = [{i} for i in range(n)]
    for i in range(n):
        for j in rng.choice(n, size=3, replace=False):
            if j != i and abs(int(j) - i) <= reach:
                pattern[i].add(int(j))
                pattern[int(j)].add(i)
    blocks = {}
    for i in range(n):
        for j in pattern[i]:
            blocks[(i, j)] = rng.normal(size=(b, b)) * (0.3 if j != i else 1.0)
        blocks[(i, i)] += 4.0 * b * np.eye(b)
    return pattern, _block_ilu_factors(n, b, pattern, blocks), rng.normal(size=(n, b))


@pytest.mark.parametrize("g", [1, 2, 3, 4])
def test_grouped_levels_equal_plain_substitution_random_pattern(g):
    n, b = 60, 3
    pattern, F, r = _random_factors(n, b, 7)
    y0, z0 = _plain_solves(n, b, pattern, F, r)
    y1, z1 = _grouped_solves(n, b, pattern, F, r, g)
    assert np.linalg.norm(y1 - y0) <= 1e-12 * np.linalg.norm(y0)
    assert np.linalg.norm(z1 - z0) <= 1e-12 * np.linalg.norm(z0)
    if g == 2:   # two levels per group are the paired levels
        y2, z2 = _paired_solves(n, b, pattern, F, r)
        assert np.linalg.norm(y1 - y2) <= 1e-13 * np.linalg.norm(y2)
        assert np.linalg.norm(z1 - z2) <= 1e-13 * np.linalg.norm(z2)


def test_grouped_levels_need_the_second_order_terms():
    """A planted mistake: dropping the W terms carried through a chain of two links (a row's
    right-hand-side terms of rows two levels back) breaks groups of three, not groups of two."""
    n, b = 60, 3
    pattern, F, r = _random_factors(n, b, 7)
    y0, z0 = _plain_solves(n, b, pattern, F, r)
    y2, _ = _grouped_solves(n, b, pattern, F, r, 2, drop_second_order=True)
    assert np.linalg.norm(y2 - y0) <= 1e-12 * np.linalg.norm(y0)
    y3, z3 = _grouped_solves(n, b, pattern, F, r, 3, drop_second_order=True)
    assert np.linalg.norm(y3 - y0) > 1e-6 * np.linalg.norm(y0)   # a million times the pass bound
    assert np.linalg.norm(z3 - z0) > 1e-6 * np.linalg.norm(z0)


@pytest.mark.parametrize("g", [3, 4])
def test_grouped_levels_equal_oracle_ilu_on_a_grid(g):
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096)
    n, b = s["n"], s["b"]
    rp, ci, W = s["row_ptr"], s["col_idx"], s["weights"]
    pattern = [set(int(c) for c in ci[rp[i]:rp[i + 1]]) for i in range(n)]
    blocks = {(i, int(ci[k])): W[i] @ s["vals"][k] for i in range(n) for k in range(rp[i], rp[i + 1])}
    F = _block_ilu_factors(n, b, pattern, blocks)
    r = synth.normal(9, n * b).reshape(n, b)
    _, z = _grouped_solves(n, b, pattern, F, r, g)
    zo = o.ilu_apply(r.reshape(-1))
    assert np.linalg.norm(zo - z.reshape(-1)) <= 1e-10 * np.linalg.norm(zo)


# ------------------------------------------------------------------------------------------------
# unknown-based AMG for A_00 (Sec. 3.4) and S~_diag (Sec. 3.3.1)
def _csr_from_dense(M):
    rp, ci, v = [0], [], []
    for i in range(M.shape[0]):
        nz = np.nonzero(M[i])[0]
        ci.extend(nz.tolist())
        v.extend(M[i, nz].tolist())
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)


def _random_mmatrix(nx, ny, nz, seed):
    """A 7-point M-matrix with seeded face weights and a small positive shift (not symmetric)."""
    rp, ci, v = poisson3d(nx, ny, nz)
    n = nx * ny * nz
    A = dense_csr(rp, ci, v, n)
    w = 0.5 + synth.uniform(seed, n * n).reshape(n, n)
    off = (A < 0) * w * A
    return off + np.diag(-off.sum(axis=1) + 0.05 + 0.1 * synth.uniform(seed + 1, n))


def test_uamg_of_a_decoupled_system_is_two_scalar_amgs():
    """With no coupling between the unknowns, unknown-based AMG is classical AMG on each diagonal
    block: hierarchy, V-cycle and all, exactly (Sec. 3.4)."""
    A1, A2 = _random_mmatrix(7, 6, 4, 31), _random_mmatrix(6, 5, 5, 32)
    n1, n2 = A1.shape[0], A2.shape[0]
    A = np.zeros((n1 + n2, n1 + n2))
    A[:n1, :n1], A[n1:, n1:] = A1, A2
    opts = dict(n_coarse=1, max_levels=3)
    hu = oracle.AMG(*_csr_from_dense(A), np_first=n1, **opts)
    h1, h2 = oracle.AMG(*_csr_from_dense(A1), **opts), oracle.AMG(*_csr_from_dense(A2), **opts)
    lu, l1, l2 = hu.levels(), h1.levels(), h2.levels()
    assert len(lu) == len(l1) == len(l2) == 3
    for a, p, t in zip(lu, l1, l2):
        Ad = dense_csr(a["rp"], a["ci"], a["v"], a["n"])
        np1 = p["n"]
        assert np.array_equal(Ad[:np1, :np1], dense_csr(p["rp"], p["ci"], p["v"], p["n"]))
        assert np.array_equal(Ad[np1:, np1:], dense_csr(t["rp"], t["ci"], t["v"], t["n"]))
        assert not Ad[:np1, np1:].any() and not Ad[np1:, :np1].any()
    b = synth.normal(33, n1 + n2)
    x = hu.vcycle(b)
    assert np.array_equal(x[:n1], h1.vcycle(b[:n1])) and np.array_equal(x[n1:], h2.vcycle(b[n1:]))


def test_uamg_hierarchy_of_a_coupled_a00():
    """On the coupled A_00 of a thermal Jacobian: P is block diagonal (no interpolation across
    unknowns), each block is classical direct interpolation of that unknown's diagonal block, the
    coarse pressure points come first, and the coarse operator is the whole Galerkin product
    P^T A_00 P (the coupling blocks stay in the coarse-grid correction)."""
    s = synth.make_box(8, 7, 3, 3.125, seed=21).system()
    o = oracle.Oracle.from_system(s, stage1=oracle.UAMG, n_coarse=20)
    levels = o.levels(2)
    assert len(levels) >= 3
    n = s["n"]
    App, ApT, ATp, ATT = pt_blocks(o.dense(), s["b"])
    A00 = np.block([[App, ApT], [ATp, ATT]])
    lev0 = levels[0]
    assert np.array_equal(dense_csr(lev0["rp"], lev0["ci"], lev0["v"], 2 * n), A00)
    np_l = n
    for l in range(len(levels) - 1):
        f, c = levels[l], levels[l + 1]
        A = dense_csr(f["rp"], f["ci"], f["v"], f["n"])
        P = dense_csr(f["Prp"], f["Pci"], f["Pv"], f["n"], f["nc"])
        ncp = int((f["cf"][:np_l] == 1).sum())
        assert not P[:np_l, ncp:].any() and not P[np_l:, :ncp].any()
        for blk, (r0, r1, c0, c1) in enumerate(((0, np_l, 0, ncp), (np_l, f["n"], ncp, f["nc"]))):
            sub = oracle.AMG(*_csr_from_dense(A[r0:r1, r0:r1]), n_coarse=1, max_levels=2, seed=l).levels()[0]
            assert np.array_equal(f["cf"][r0:r1], sub["cf"])
            assert np.array_equal(P[r0:r1, c0:c1], dense_csr(sub["Prp"], sub["Pci"], sub["Pv"], r1 - r0, c1 - c0))
        Ac = dense_csr(c["rp"], c["ci"], c["v"], c["n"])
        ref = P.T @ A @ P
        assert np.abs(Ac - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.abs(Ac[:ncp, ncp:]).max() > 0.0       # coupling kept on the coarse level
        np_l = ncp


def test_uamg_single_level_is_exact_a00_inverse():
    s = tiny().system()
    o = oracle.Oracle.from_system(s, stage1=oracle.UAMG, max_levels=1, dense_max=4096)
    n, b = s["n"], s["b"]
    App, ApT, ATp, ATT = pt_blocks(o.dense(), b)
    A00 = np.block([[App, ApT], [ATp, ATT]])
    v = synth.normal(34, n * b)
    x1 = o.stage1(v).reshape(n, b)
    vv = v.reshape(n, b)
    want = np.linalg.solve(A00, np.concatenate([vv[:, 0], vv[:, 1]]))
    assert np.linalg.norm(np.concatenate([x1[:, 0], x1[:, 1]]) - want) <= 1e-10 * np.linalg.norm(want)
    assert not x1[:, 2:].any()


def test_cptr_uamg_solve_matches_dense_solve():
    s = synth.make_box(8, 7, 3, 3.125, seed=21).system()
    o = oracle.Oracle.from_system(s, stage1=oracle.UAMG, n_coarse=20)
    x, info = o.solve(s["rhs"], 1e-10)
    assert info["converged"]
    Ad = bsr_dense(s)
    ref = np.linalg.solve(Ad, s["rhs"].reshape(-1))
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)


def test_schur_diag_is_the_schur_complement_with_a_diagonal_pressure_block():
    """S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3.1) is the Schur complement of
    [[diag(A_pp), A_pT], [A_Tp, A_TT]]: its inverse is the T-T block of that matrix's inverse."""
    s = tiny().system()
    o = oracle.Oracle.from_system(s, schur=oracle.SCHUR_DIAG, max_levels=1, dense_max=4096)
    n = s["n"]
    App, ApT, ATp, ATT = pt_blocks(o.dense(), s["b"])
    M = np.block([[np.diag(np.diag(App)), ApT], [ATp, ATT]])
    want = np.linalg.inv(np.linalg.inv(M)[n:, n:])
    lev = o.levels(1)[0]
    got = dense_csr(lev["rp"], lev["ci"], lev["v"], n)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    # its pattern is that of A_TT joined with the pressure couplings two cells away
    assert lev["rp"][-1] > s["row_ptr"][-1]


def test_schur_diag_is_exact_for_one_cell():
    s = synth.make_box(1, 1, 1, 3.125, seed=5, wells="none").system()
    o = oracle.Oracle.from_system(s, schur=oracle.SCHUR_DIAG, max_levels=1)
    App, ApT, ATp, ATT = pt_blocks(o.dense(), s["b"])
    lev = o.levels(1)[0]
    assert abs(lev["v"][0] - (ATT - ATp @ np.linalg.solve(App, ApT))[0, 0]) <= 1e-14 * abs(lev["v"][0])


# ------------------------------------------------------------------------------------------------
# QI / TI decoupling operators (Sec. 3.1 for CPR, extended to the p-T system in Sec. 3.2)
def _dense_decoupling(Ad, n, b, prim, kind):
    """D_i = X_i Y_i^{-1} from the dense A' by numpy: QI from the diagonal block, TI from the sum of
    the blocks of block column i; and G A' with G_i = [I -D_i; 0 I] on the primary rows of cell i."""
    sec = [q for q in range(b) if q not in prim]
    GA = Ad.copy()
    D = np.zeros((n, len(prim), len(sec)))
    for i in range(n):
        cols = [i * b + s for s in sec]
        if kind == "qi":
            X = Ad[np.ix_([i * b + p for p in prim], cols)]
            Y = Ad[np.ix_([i * b + s for s in sec], cols)]
        else:
            X = sum(Ad[np.ix_([j * b + p for p in prim], cols)] for j in range(n))
            Y = sum(Ad[np.ix_([j * b + s for s in sec], cols)] for j in range(n))
        D[i] = np.linalg.solve(Y.T, X.T).T
        for r, p in enumerate(prim):
            GA[i * b + p] = Ad[i * b + p] - sum(D[i, r, t] * Ad[i * b + s] for t, s in enumerate(sec))
    return D, GA, sec


@pytest.mark.parametrize("kind", ["qi", "ti"])
@pytest.mark.parametrize("stage1", ["cpr", "uamg"])
def test_decoupled_first_stage_fields(kind, stage1):
    """The first stage's fields are those of G A': A_pp - D A_sp for CPR (Sec. 3.1), A_00 - D A_s0
    for the p-T first stage (Sec. 3.2), with D_QI / D_TI computed from the dense A' by numpy."""
    s = tiny().system()
    n, b = s["n"], s["b"]
    st1 = oracle.CPR if stage1 == "cpr" else oracle.UAMG
    dec = oracle.DECOUPLE_QI if kind == "qi" else oracle.DECOUPLE_TI
    o = oracle.Oracle.from_system(s, stage1=st1, decouple=dec, max_levels=1, dense_max=4096)
    Ad = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096).dense()
    prim = [0] if stage1 == "cpr" else [0, 1]
    D, GA, sec = _dense_decoupling(Ad, n, b, prim, kind)
    nnzb = int(s["row_ptr"][-1])
    App = dense_csr(s["row_ptr"], s["col_idx"], o.field(0, nnzb), n)
    ApT = dense_csr(s["row_ptr"], s["col_idx"], o.field(1, nnzb), n)
    assert np.abs(App - GA[0::b, 0::b]).max() <= 1e-12 * np.abs(GA[0::b, 0::b]).max()
    assert np.abs(ApT - GA[0::b, 1::b]).max() <= 1e-12 * np.abs(GA[0::b, 1::b]).max()
    if kind == "qi":   # the defining property: no secondary unknown of its own cell in a primary row
        for i in range(n):
            blk = GA[np.ix_([i * b + p for p in prim], [i * b + q for q in sec])]
            assert np.abs(blk).max() <= 1e-12 * np.abs(Ad[i * b:(i + 1) * b, i * b:(i + 1) * b]).max()


@pytest.mark.parametrize("kind", ["qi", "ti"])
def test_decoupled_cpr_stage1_with_exact_inner_solve(kind):
    """With an exact inner solve, the decoupled CPR first stage is x_p = (A_pp - D A_sp)^{-1} (G v)_p
    (Sec. 3.1: M1^{-1} = R_p^T (R_p G A R_p^T)^{-1} R_p G)."""
    s = tiny().system()
    n, b = s["n"], s["b"]
    dec = oracle.DECOUPLE_QI if kind == "qi" else oracle.DECOUPLE_TI
    o = oracle.Oracle.from_system(s, stage1=oracle.CPR, decouple=dec, max_levels=1, dense_max=4096)
    Ad = oracle.Oracle.from_system(s, max_levels=1, dense_max=4096).dense()
    D, GA, sec = _dense_decoupling(Ad, n, b, [0], kind)
    v = synth.normal(51, n * b)
    Gv = v.copy().reshape(n, b)
    for i in range(n):
        Gv[i, 0] = v[i * b] - sum(D[i, 0, t] * v[i * b + q] for t, q in enumerate(sec))
    want = np.linalg.solve(GA[0::b, 0::b], Gv[:, 0])
    x1 = o.stage1(v).reshape(n, b)
    assert np.linalg.norm(x1[:, 0] - want) <= 1e-10 * np.linalg.norm(want)
    assert not x1[:, 1:].any()


def test_decoupling_trend_ti_better_than_qi():
    """Sec. 3.1: TI is superior to QI, which can increase the number of GMRES iterations; TI also
    helps the unknown-based first stage (Tables meshW-anisomeshW, CPTR-uAMG(TI))."""
    s = synth.make_box(40, 40, 10, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                       kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=86400.0).system()
    its = {}
    for st1 in (oracle.CPR, oracle.UAMG):
        for dec in (0, 1, 2):
            x, info = oracle.Oracle.from_system(s, stage1=st1, decouple=dec, max_it=300).solve(s["rhs"], 1e-8)
            assert info["converged"]
            its[st1, dec] = info["iters"]
    assert its[oracle.CPR, 2] <= its[oracle.CPR, 1] and its[oracle.UAMG, 2] <= its[oracle.UAMG, 1]
    assert its[oracle.UAMG, 2] < its[oracle.UAMG, 0]


# ------------------------------------------------------------------------------------------------
# ILU(1) second stage (the CPR-AMG-ILU(1) comparator of Tables meshW-anisomeshW)
def _ilu_lu(o):
    rp, ci = o.ilu_pattern()
    F = dense_csr(rp, ci, o.ilu_factors(), o.nb)
    return np.tril(F, -1) + np.eye(o.nb), np.triu(F), rp, ci


def test_ilu1_pattern_is_a_plus_level_one_fill():
    """The ILU(1) pattern is that of A joined with that of strictlower(A) x strictupper(A) (one
    elimination step from original entries), computed here by a boolean matrix product."""
    o = oracle.Oracle.from_system(tiny().system(), max_levels=1, ilu_fill=1)
    A = o.dense() != 0
    rpA, ciA, _ = o.matrix()
    P = np.zeros_like(A)
    for i in range(o.nb):
        P[i, ciA[rpA[i]:rpA[i + 1]]] = True
    fill = (np.tril(P, -1).astype(int) @ np.triu(P, 1).astype(int)) > 0
    rp, ci = o.ilu_pattern()
    got = np.zeros_like(P)
    for i in range(o.nb):
        got[i, ci[rp[i]:rp[i + 1]]] = True
    assert np.array_equal(got, P | fill) and (got & ~P).any()


def test_ilu1_product_matches_matrix_on_its_pattern():
    o = oracle.Oracle.from_system(tiny().system(), max_levels=1, ilu_fill=1)
    L, U, rp, ci = _ilu_lu(o)
    A = o.dense()
    mask = np.zeros_like(A, dtype=bool)
    for i in range(o.nb):
        mask[i, ci[rp[i]:rp[i + 1]]] = True
    assert np.abs((L @ U - A)[mask]).max() <= 1e-12 * np.abs(A).max()
    r = synth.normal(53, o.nb)
    assert np.linalg.norm(L @ (U @ o.ilu_apply(r)) - r) <= 1e-10 * np.linalg.norm(r)


def test_scalar_ilu1_equals_block_ilu1():
    """With dense b x b blocks, the scalar ILU(1) fill is block fill, and scalar ILU(1) equals the
    textbook block ILU on the block ILU(1) pattern with exact pivot-block inverses."""
    s = tiny(4, 3, 2).system()
    o = oracle.Oracle.from_system(s, max_levels=1, ilu_fill=1)
    n, b = s["n"], s["b"]
    rp, ci, W = s["row_ptr"], s["col_idx"], s["weights"]
    orig = [set(int(c) for c in ci[rp[i]:rp[i + 1]]) for i in range(n)]
    pattern = [set(orig[i]) | {j for k in orig[i] if k < i for j in orig[k] if j > k} for i in range(n)]
    blocks = {(i, j): np.zeros((b, b)) for i in range(n) for j in pattern[i]}
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            blocks[(i, int(ci[k]))] = W[i] @ s["vals"][k]
    F = _block_ilu_factors(n, b, pattern, blocks)
    y, z = _plain_solves(n, b, pattern, F, synth.normal(54, n * b).reshape(n, b))
    zo = o.ilu_apply(synth.normal(54, n * b))
    assert np.linalg.norm(zo - z.reshape(-1)) <= 1e-10 * np.linalg.norm(z)


def test_ilu1_fewer_iterations_than_ilu0_for_cpr():
    """CPR-AMG-ILU(1) takes fewer iterations than CPR-AMG with ILU(0) (Tables meshW-anisomeshW)."""
    s = synth.make_box(40, 40, 10, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                       kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=30 * 86400.0).system()
    its = [oracle.Oracle.from_system(s, stage1=oracle.CPR, ilu_fill=f).solve(s["rhs"], 1e-8)[1]["iters"] for f in (0, 1)]
    assert its[1] < its[0], its


# ------------------------------------------------------------------------------------------------
# Newton's method around the solve (Sec. 3 eq. AXR, Sec. 4)
def test_newton_oracle_solves_the_step_with_quadratic_convergence():
    """The oracle's Newton step drives ||W R|| below 1e-8 of its start (the generator's residual,
    pinned by finite differences, evaluated independently at the result), with full steps near the
    solution and the error ratio of a quadratically convergent method."""
    r = synth.make_box(8, 6, 3, 3.125, seed=17, heaters=[(11, 80.0, 420.0)])
    x, info = oracle.newton_step(r, r.x0.copy(), r.x0, rtol_lin=1e-12)
    assert info["converged"] and info["newton_its"] >= 3
    W = r.weights()
    R = r.evaluate(x, jacobian=False, schur=False)["R"]
    assert np.linalg.norm(np.einsum("nij,nj->ni", W, R)) <= 1e-8 * info["res0"]
    res = [info["res0"]] + [p["res"] for p in info["per_iteration"]]
    assert all(p["alpha"] == 1.0 for p in info["per_iteration"][1:])
    # quadratic: r_{k+1} / r_k^2 stays bounded while r_k falls by orders of magnitude
    rat = [res[k + 1] / res[k] ** 2 for k in range(1, len(res) - 1)]
    assert res[-2] / res[1] < 1e-3 and max(rat[1:]) <= 10 * rat[0] + 1e-30, (res, rat)


# ------------------------------------------------------------------------------------------------
# Block-Jacobi ILU(0) (Sec. 4: the paper's parallel second stage, ILU(k) on each part of the domain)
def _quadrants(nx, ny, nz, px=2, py=2):
    i = np.arange(nx * ny * nz)
    x, y = i % nx, (i // nx) % ny
    return ((x * px) // nx + px * ((y * py) // ny)).astype(np.int32)


def _drop_cross_part_blocks(s, part):
    """The same system with every block between cells of different parts removed from the input."""
    rp, ci, vals = s["row_ptr"], s["col_idx"], s["vals"]
    keep = np.array([part[i] == part[ci[k]] for i in range(s["n"]) for k in range(rp[i], rp[i + 1])])
    rows = np.repeat(np.arange(s["n"]), np.diff(rp))
    out = dict(s)
    out["col_idx"] = ci[keep].astype(np.int32)
    out["vals"] = vals[keep]
    out["row_ptr"] = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=s["n"]))]).astype(np.int32)
    out["st"] = s["st"][keep]
    return out


def test_block_jacobi_ilu_is_ilu_of_the_matrix_without_cross_part_couplings():
    """ILU(0) over parts equals, bit for bit, ILU(0) of the system whose cross-part blocks were
    removed before the set-up; one part gives the global ILU(0)."""
    r = synth.make_box(8, 6, 3, 3.125, seed=21)
    s = r.system()
    part = _quadrants(8, 6, 3)
    o_bj = oracle.Oracle.from_system(s, max_levels=1, part=part)
    o_drop = oracle.Oracle.from_system(_drop_cross_part_blocks(s, part), max_levels=1)
    assert np.array_equal(o_bj.ilu_factors(), o_drop.ilu_factors())
    rp, ci = o_bj.ilu_pattern()
    cells = np.repeat(np.arange(o_bj.nb), np.diff(rp)) // 3
    assert np.all(part[cells] == part[ci // 3])
    v = synth.normal(61, o_bj.nb)
    assert np.array_equal(o_bj.ilu_apply(v), o_drop.ilu_apply(v))
    o_one = oracle.Oracle.from_system(s, max_levels=1, part=np.zeros(s["n"], np.int32))
    o_glob = oracle.Oracle.from_system(s, max_levels=1)
    assert np.array_equal(o_one.ilu_factors(), o_glob.ilu_factors())


def test_block_jacobi_ilu_trend():
    """More parts, a weaker second stage: the solve still converges, in at least as many iterations."""
    s = synth.make_box(40, 40, 10, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                       kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=30 * 86400.0).system()
    its = []
    for px, py in ((1, 1), (2, 2), (4, 4)):
        part = _quadrants(40, 40, 10, px, py)
        x, info = oracle.Oracle.from_system(s, part=part).solve(s["rhs"], 1e-8)
        assert info["converged"]
        its.append(info["iters"])
    assert its[0] <= its[1] <= its[2], its
