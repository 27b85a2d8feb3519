"""Pins of the oracle's learned Schur scaling (features, exact target, network, Adam, BF16
inference) against closed forms, dense linear algebra, finite differences and error bounds.
No GPU."""
import numpy as np
import pytest

import oracle
import synth


def weighted_dense(s):
    """A' = blockdiag(W) A built with numpy from the generator's raw blocks and weights."""
    n, b = s["n"], s["b"]
    A = np.zeros((n * b, n * b))
    rp, ci = s["row_ptr"], s["col_idx"]
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i * b:(i + 1) * b, ci[k] * b:(ci[k] + 1) * b] = s["weights"][i] @ s["vals"][k]
    return A


def three_phase(nx, ny, nz, **kw):
    return synth.make_box(nx, ny, nz, 1.0, 1.0, 0.5, seed=21, sigma=2.5, nphase=3, wells="four",
                          T_inj=500.0, q_inj=4e-6, **kw).system()


def features_of(s, base="att"):
    o = oracle.Oracle.from_system(s, use_st=False, max_levels=1, dense_max=1, stage2=oracle.NONE2)
    return o.schur_features(oracle.schur_base(s, base, o))


def test_features_of_two_cells_closed_form():
    s = synth.make_box(2, 1, 1, 3.125, seed=3, nphase=3, wells="none").system()
    A = weighted_dense(s)
    b = s["b"]
    f = np.sinh(features_of(s))
    blk = lambda i, j: A[i * b:(i + 1) * b, j * b:(j + 1) * b]
    for i, j in ((0, 1), (1, 0)):
        a, c, d = blk(i, i), blk(i, j), blk(j, j)   # diagonal block of i, coupling i->j, diagonal of j
        cT = blk(j, i)                              # coupling j->i (its (p, T) entry is A_pT,ji)
        app, apt, atp, bii = a[0, 0], a[0, 1], a[1, 0], a[1, 1]
        first = atp * apt / app + c[1, 0] * cT[0, 1] / d[0, 0]
        assert f[i, 0] == pytest.approx(first / bii, rel=1e-12)
        assert f[i, 1] == pytest.approx(atp * apt / app / bii, rel=1e-12)
        assert f[i, 2] == pytest.approx(abs(c[0, 0]) / abs(app), rel=1e-12)
        assert f[i, 3] == pytest.approx(abs(c[1, 1]) / abs(bii), rel=1e-12)
        assert f[i, 4] == pytest.approx(c[0, 0] / abs(app), rel=1e-12)
        assert f[i, 5] == pytest.approx(c[1, 1] / abs(bii), rel=1e-12)
        assert f[i, 6] == pytest.approx((abs(atp * apt / app) + abs(c[1, 0] * cT[0, 1] / d[0, 0])) / abs(bii),
                                        rel=1e-12)
        sat = range(2, b)
        assert f[i, 7] == pytest.approx(sum(a[1, k] * a[k, 1] / a[k, k] for k in sat) / bii, rel=1e-12)
        assert f[i, 8] == pytest.approx(sum(a[0, k] * a[k, 0] / a[k, k] for k in sat) / app, rel=1e-12)
        assert f[i, 9] == np.sign(app) and f[i, 10] == np.sign(bii)
        r = np.sqrt(abs(app * bii))
        assert f[i, 11] == pytest.approx(apt / r, rel=1e-12)
        assert f[i, 12] == pytest.approx(atp / r, rel=1e-12)
        assert f[i, 13] == pytest.approx(2 / 7, rel=1e-15)
        assert f[i, 14] == pytest.approx(abs(c[0, 1]) * abs(atp) / abs(app * bii), rel=1e-12)
        assert f[i, 15] == pytest.approx(abs(c[1, 0]) * abs(apt) / abs(app * bii), rel=1e-12)


def test_exact_schur_diagonal_matches_dense_schur_complement():
    s = three_phase(6, 5, 3)
    b = s["b"]
    A = weighted_dense(s)
    App, ApT, ATp, ATT = A[0::b, 0::b], A[0::b, 1::b], A[1::b, 0::b], A[1::b, 1::b]
    S = ATT - ATp @ np.linalg.solve(App, ApT)
    o = oracle.Oracle.from_system(s, use_st=False, max_levels=1, dense_max=1, stage2=oracle.NONE2)
    d = oracle.exact_schur_diag(o, s, chunk=7)
    np.testing.assert_allclose(d, np.diag(S), rtol=1e-10, atol=1e-12 * np.abs(np.diag(S)).max())
    t, _ = oracle.schur_ratio_target(s, "att")
    np.testing.assert_allclose(np.sinh(t), np.diag(S) / np.diag(ATT), rtol=1e-10)
    rp, ci = s["row_ptr"], s["col_idx"]
    se_diag = np.array([s["st"][k] for i in range(s["n"]) for k in range(rp[i], rp[i + 1]) if ci[k] == i])
    t, _ = oracle.schur_ratio_target(s, "se")
    np.testing.assert_allclose(np.sinh(t), np.diag(S) / se_diag, rtol=1e-10)


def test_features_use_the_given_base():
    s = synth.make_box(2, 1, 1, 3.125, seed=3, nphase=3, wells="none").system()
    f = np.sinh(features_of(s, "se"))
    st, rp, ci = s["st"], s["row_ptr"], s["col_idx"]
    for i in range(2):
        row = range(rp[i], rp[i + 1])
        bii = sum(st[k] for k in row if ci[k] == i)
        off = [st[k] for k in row if ci[k] != i]
        assert f[i, 3] == pytest.approx(sum(abs(v) for v in off) / abs(bii), rel=1e-12)
        assert f[i, 5] == pytest.approx(sum(off) / abs(bii), rel=1e-12)
        assert f[i, 10] == np.sign(bii)


def test_exact_schur_of_one_cell_is_the_scalar_schur_complement():
    s = synth.make_box(1, 1, 1, 3.125, seed=4, wells="none").system()
    a = s["weights"][0] @ s["vals"][0]
    t, _ = oracle.schur_ratio_target(s, "att")
    assert np.sinh(t[0]) == pytest.approx((a[1, 1] - a[1, 0] * a[0, 1] / a[0, 0]) / a[1, 1], rel=1e-12)


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(size=oracle.mlp_nparam()) * scale


def test_network_gradient_matches_central_differences():
    s = three_phase(4, 4, 2)
    t, X = oracle.schur_ratio_target(s)
    P = _params(1)
    _, g = oracle.mlp_loss_grad(P, X, t)
    rng = np.random.default_rng(2)
    h = 1e-6
    for k in rng.choice(len(P), 40, replace=False):
        e = np.zeros_like(P)
        e[k] = h
        fd = (oracle.mlp_loss_grad(P + e, X, t)[0] - oracle.mlp_loss_grad(P - e, X, t)[0]) / (2 * h)
        assert fd == pytest.approx(g[k], abs=1e-8 + 1e-6 * abs(g[k]))


def test_network_with_zero_weight_matrices_closed_form():
    nf, nh = oracle.N_FEATURES, oracle.N_HIDDEN
    P = _params(3)
    P[:nh * nf] = 0.0                                  # W1
    P[nh * nf + nh:nh * nf + nh + nh * nh] = 0.0       # W2
    b2 = P[nh * nf + nh + nh * nh:nh * nf + 2 * nh + nh * nh]
    w3 = P[-1 - nh:-1]
    X = np.random.default_rng(4).normal(size=(9, nf))
    t = np.linspace(-1, 1, 9)
    y = P[-1] + w3 @ np.tanh(b2)
    np.testing.assert_allclose(oracle.mlp_forward(P, X), y, rtol=1e-14)
    loss, g = oracle.mlp_loss_grad(P, X, t)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-13)
    assert g[-1] == pytest.approx(2 * np.mean(y - t), rel=1e-12)
    np.testing.assert_allclose(g[-1 - nh:-1], 2 * np.mean(y - t) * np.tanh(b2), rtol=1e-12)
    assert np.all(g[:nh * nf + nh] == 0.0)             # no signal reaches layer 1 through W2 = 0


def test_adam_first_and_second_steps_closed_form():
    P0 = _params(5)
    g1 = _params(6)
    g2 = _params(7)
    P = P0.copy()
    m, v = np.zeros_like(P), np.zeros_like(P)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    oracle.adam_step(P, m, v, g1, 1, lr, b1, b2, eps)
    np.testing.assert_allclose(P, P0 - lr * g1 / (np.abs(g1) + eps), rtol=1e-13, atol=1e-16)
    P1 = P.copy()
    oracle.adam_step(P, m, v, g2, 2, lr, b1, b2, eps)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(P, P1 - lr * mh / (np.sqrt(vh) + eps), rtol=1e-12, atol=1e-16)


def test_training_reduces_the_loss():
    s = three_phase(6, 6, 2, c_o=1e-7, beta_o=5e-2)
    t, X = oracle.schur_ratio_target(s)
    P, losses = oracle.mlp_train(_params(8, 0.1), X, t, steps=60, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]


def test_bf16_inference_within_rounding_bound_of_fp64_network():
    """Every BF16 rounding has relative error <= u = 2^-8; FP32 sums add n * 2^-24 of the absolute
    sum.  The bound below propagates these through the layers (tanh is 1-Lipschitz)."""
    s = three_phase(5, 5, 2)
    _, X = oracle.schur_ratio_target(s, "att")
    nf, nh = oracle.N_FEATURES, oracle.N_HIDDEN
    P = _params(9, 0.1).astype(np.float32).astype(np.float64)
    W1 = P[:nh * nf].reshape(nh, nf)
    b1 = P[nh * nf:nh * nf + nh]
    W2 = P[nh * nf + nh:nh * nf + nh + nh * nh].reshape(nh, nh)
    b2 = P[nh * nf + nh + nh * nh:nh * nf + 2 * nh + nh * nh]
    w3 = P[-1 - nh:-1]
    u, e32 = 2.0 ** -8, 2.0 ** -24
    yb = oracle.mlp_infer_bf16(P.astype(np.float32), X).astype(np.float64)
    yf = oracle.mlp_forward(P, X)
    for i in range(X.shape[0]):
        x = X[i]
        h1 = np.tanh(W1 @ x + b1)
        e1 = np.abs(W1) @ np.abs(x) * (2 * u + u * u) + (nf + 1) * e32 * (np.abs(W1) @ np.abs(x) * 2 + abs(b1))
        dh1 = e1 + u * (np.abs(h1) + e1)                       # tanh, then BF16 rounding of h1
        z2 = W2 @ h1 + b2
        e2 = np.abs(W2) @ (dh1 + u * (np.abs(h1) + dh1)) + (nh + 1) * e32 * (np.abs(W2) @ (np.abs(h1) + dh1) * 2
                                                                                 + abs(b2))
        h2 = np.tanh(z2)
        dh2 = e2 + u * (np.abs(h2) + e2)
        ey = np.abs(w3) @ (dh2 + u * (np.abs(h2) + dh2)) + (nh + 1) * e32 * (np.abs(w3) @ (np.abs(h2) + dh2) * 2
                                                                            + abs(P[-1]))
        assert abs(yb[i] - yf[i]) <= ey
        assert ey < 0.5                                         # the bound is not vacuous
    assert np.abs(yb - yf).max() > 0                            # the BF16 form does round


def test_learned_st_with_constant_output_scales_att():
    s = three_phase(4, 3, 2)
    P = np.zeros(oracle.mlp_nparam(), np.float32)
    P[-1] = np.float32(np.arcsinh(0.5))
    st_se, _, _ = oracle.learned_st(s, P, "se")
    np.testing.assert_allclose(st_se, s["st"] * np.sinh(np.float64(np.float32(np.arcsinh(0.5)))), rtol=1e-15)
    st, sc, y = oracle.learned_st(s, P, "att")
    o = oracle.Oracle.from_system(s, use_st=False, max_levels=1, dense_max=1, stage2=oracle.NONE2)
    np.testing.assert_allclose(sc, np.sinh(np.float64(np.float32(np.arcsinh(0.5)))), rtol=1e-15)
    np.testing.assert_allclose(st, o.att(len(st)) * sc[0], rtol=1e-15)
    A = weighted_dense(s)
    b = s["b"]
    rp, ci = s["row_ptr"], s["col_idx"]
    att = np.array([A[i * b + 1, j * b + 1] for i in range(s["n"]) for j in ci[rp[i]:rp[i + 1]]])
    np.testing.assert_allclose(o.att(len(st)), att, rtol=1e-15)


def test_exact_scaling_rescues_att_on_a_strongly_coupled_case():
    """With strong p-T coupling through the oil (compressible, strongly expanding) the algebraic
    A_TT approximation stalls; the exact diagonal ratio as the row scaling restores convergence.
    This is what the network is trained to predict."""
    s = three_phase(12, 12, 4, c_o=1e-7, beta_o=5e-2)
    t, _ = oracle.schur_ratio_target(s, "att")
    rows = np.repeat(np.arange(s["n"]), np.diff(s["row_ptr"]))
    o = oracle.Oracle.from_system(s, use_st=False, max_levels=1, dense_max=1, stage2=oracle.NONE2)
    att = o.att(int(s["row_ptr"][-1]))
    run = lambda st, **kw: oracle.Oracle.from_system(dict(s, st=st), n_coarse=32, max_it=300, **kw).solve(
        s["rhs"], 1e-6)[1]
    plain = oracle.Oracle.from_system(s, use_st=False, n_coarse=32, max_it=300).solve(s["rhs"], 1e-6)[1]
    scaled = run(att * np.sinh(t)[rows])
    assert not plain["converged"]
    assert scaled["converged"] and scaled["iters"] < 60
