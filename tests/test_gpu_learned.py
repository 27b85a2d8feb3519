"""The learned Schur scaling on the GPU (through the C ABI) against the oracle.

Tolerances:
  - features: FP64 on both sides with the same operation order; asinh may differ in the last
    bits: |difference| <= 1e-13 (1 + |f|);
  - loss and gradient: the GPU computes in FP32 (inputs rounded to FP32 on the device), the oracle
    in FP64 on the same FP32-rounded inputs: relative error <= 1e-4 of the gradient's max norm;
  - BF16 inference: both sides add the same exact BF16 products in the same order in FP32; only
    tanhf may differ by an ulp, which can flip a BF16 rounding of an activation.  At least 99% of
    the outputs agree to 1e-5 (1 + |y|), all within the effect of two such flips;
  - the learned solve: FGMRES iterations equal to the oracle's +-1 on the oracle's own learned
    S~_T, relative solution error <= 1e-8 per unknown kind.
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


def gpu_solver(s, st=True, **opts):
    S = cp.Solver(**opts)
    S.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]) if st else None)
    return S


def gpu_features(S):
    f = torch.zeros((S.n, cp.MLP_FEATURES), dtype=torch.float64, device="cuda")
    cp.cptr_schur_features(S.ctx, f)
    return f


def three_phase(nx, ny, nz, seed=21, **kw):
    return synth.make_box(nx, ny, nz, 1.0, 1.0, 0.5, seed=seed, sigma=2.5, nphase=3, wells="four",
                          T_inj=500.0, q_inj=4e-6, **kw).system()


def oracle_features(s, base):
    o = oracle.Oracle.from_system(s, use_st=False, max_levels=1, dense_max=1, stage2=oracle.NONE2)
    return o.schur_features(oracle.schur_base(s, base, o))


@pytest.mark.parametrize("base", ["se", "att"])
@pytest.mark.parametrize("kind", ["two_phase", "three_phase", "coupled"])
def test_features_match_oracle(kind, base):
    if kind == "two_phase":
        s = synth.make_box(7, 5, 3, 3.125, seed=17).system()
    elif kind == "three_phase":
        s = three_phase(9, 7, 3)
    else:
        s = three_phase(9, 7, 3, c_o=1e-7, beta_o=5e-2)
    S = gpu_solver(s, st=base == "se", n_coarse=16)
    fg = host(gpu_features(S))
    fo = oracle_features(s, base)
    assert np.all(np.abs(fg - fo) <= 1e-13 * (1 + np.abs(fo)))


def _data(n_grids=3, shape=(8, 8, 3), base="att"):
    X, T = [], []
    for k in range(n_grids):
        t, x = oracle.schur_ratio_target(synth.learned_training_grid(k, *shape).system(), base)
        X.append(x)
        T.append(t)
    return np.concatenate(X), np.concatenate(T)


@pytest.mark.parametrize("n", [1, 357, 40000])
def test_loss_and_gradient_match_oracle(n):
    X, T = _data()
    reps = -(-n // len(T))
    X = np.tile(X, (reps, 1))[:n] * (1 + 0.01 * np.arange(n) / n)[:, None]   # distinct samples
    T = np.tile(T, reps)[:n]
    P = synth.mlp_init(5)
    S = cp.Solver()
    g = torch.zeros(cp.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = cp.cptr_mlp_loss_grad(S.ctx, dev(X), dev(T), dev(P), g)
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    loss_o, g_o = oracle.mlp_loss_grad(P.astype(np.float64), X32, T32)
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert np.abs(host(g) - g_o).max() <= 1e-4 * np.abs(g_o).max()


def test_host_and_device_arrays_give_the_same_gradient():
    X, T = _data(1)
    P = synth.mlp_init(6)
    S = cp.Solver()
    g_d = torch.zeros(cp.MLP_NPARAM, dtype=torch.float32, device="cuda")
    g_h = np.zeros(cp.MLP_NPARAM, np.float32)
    l_d = cp.cptr_mlp_loss_grad(S.ctx, dev(X), dev(T), dev(P), g_d)
    l_h = cp.cptr_mlp_loss_grad(S.ctx, X, T, P, g_h)
    assert l_d == l_h and np.array_equal(host(g_d), g_h)


def test_adam_training_follows_the_oracle():
    X, T = _data(2)
    P0 = synth.mlp_init(7)
    S = cp.Solver()
    P = dev(P0.copy())
    steps = 5
    hist = cp.cptr_mlp_train(S.ctx, dev(X), dev(T), P, steps, lr=1e-3)
    X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    P_o, hist_o = oracle.mlp_train(P0.astype(np.float64), X32, T32, steps, lr=1e-3)
    np.testing.assert_allclose(hist, hist_o, rtol=1e-4)
    d = np.abs(host(P) - P_o)
    # Adam's step is lr * m / (sqrt(v) + eps): where the gradient is far from zero both sides take
    # the same step; where it is tiny its sign may differ in FP32.  Every step is at most ~lr.
    assert d.max() <= steps * 1e-3 * 1.01
    assert np.mean(d <= 1e-6) >= 0.95


def test_training_reduces_the_loss_on_the_gpu():
    X, T = _data(3)
    S = cp.Solver()
    P = dev(synth.mlp_init(8))
    hist = cp.cptr_mlp_train(S.ctx, dev(X), dev(T), P, 400, lr=2e-3)
    assert hist[-1] < 0.1 * hist[0]


def _flip_bound(P):
    nf, nh = cp.MLP_FEATURES, cp.MLP_HIDDEN
    P = np.array([oracle.round_bf16(float(v)) for v in P])
    W2 = P[nh * nf + nh:nh * nf + nh + nh * nh].reshape(nh, nh)
    w3 = P[-1 - nh:-1]
    u = 2.0 ** -8
    one = max((np.abs(w3)[:, None] * np.abs(W2)).sum(axis=0).max(), np.abs(w3).max()) * u
    return 2 * one * 1.01


def test_bf16_inference_matches_oracle():
    X, T = _data(3)
    S = cp.Solver()
    P = dev(synth.mlp_init(9))
    cp.cptr_mlp_train(S.ctx, dev(X), dev(T), P, 200, lr=2e-3)
    Ph = host(P)
    cp.cptr_set_mlp(S.ctx, P)
    y = torch.zeros(len(T), dtype=torch.float32, device="cuda")
    cp.cptr_mlp_infer(S.ctx, dev(X), y)
    yg = host(y).astype(np.float64)
    yo = oracle.mlp_infer_bf16(Ph, X).astype(np.float64)
    d = np.abs(yg - yo)
    assert np.mean(d <= 1e-5 * (1 + np.abs(yo))) >= 0.99
    assert d.max() <= _flip_bound(Ph)


def _trained(base, shape=(12, 12, 4), grids=8, steps=1500):
    X, T = _data(grids, shape, base)
    S = cp.Solver()
    P = dev(synth.mlp_init(10))
    hist = cp.cptr_mlp_train(S.ctx, dev(X), dev(T), P, steps, lr=2e-3)
    return host(P), hist


_NET = {}


def trained_net(base):
    if base not in _NET:
        _NET[base] = _trained(base)
    return _NET[base][0]


def learned_solver(s, P, base, **opts):
    g = cp.Solver(schur=cp.SCHUR["learned"], **opts)
    cp.cptr_set_mlp(g.ctx, P)
    g.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]) if base == "se" else None)
    return g


@pytest.mark.parametrize("base", ["se", "att"])
def test_learned_setup_and_solve_match_oracle(base):
    P = trained_net(base)
    s = three_phase(10, 9, 4, seed=33, c_o=3e-8, beta_o=1e-2)
    g = learned_solver(s, P, base, n_coarse=16)
    sg = np.zeros(s["n"])
    cp.cptr_schur_scaling(g.ctx, sg)
    st_o, so, yo = oracle.learned_st(s, P, base)
    ok = np.abs(sg - so) <= 1e-5 * np.abs(so)
    assert np.mean(ok) >= 0.99
    o = oracle.Oracle.from_system(dict(s, st=st_o), n_coarse=16)
    x_o, info_o = o.solve(s["rhs"], 1e-8)
    x_g, info_g = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info_g["schur_used"] == "learned"
    assert info_g["status"] == "CPTR_OK" and info_o["converged"]
    assert abs(info_g["iters"] - info_o["iters"]) <= 1
    if not ok.all():
        # s_i of a few cells differs from the oracle's by a BF16 rounding flip (a hidden unit's
        # FP32 tanh against the FP64 one), so the two preconditioners differ slightly and the
        # iterates at 1e-8 need not agree to 1e-8.  Both solves are then converged to 1e-12, where
        # each solution lies within kappa * 1e-12 of the exact one, and compared there.
        print(f"learned s: {np.count_nonzero(~ok)} of {ok.size} cells differ by more than 1e-5")
        x_o, info_o = o.solve(s["rhs"], 1e-12)
        x_g, info_g = g.solve(dev(s["rhs"].reshape(-1)), 1e-12)
        assert info_g["status"] == "CPTR_OK" and info_o["converged"]
    x_g = host(x_g)
    b = s["b"]
    for u in range(b):
        err = np.linalg.norm(x_g[u::b] - x_o[u::b]) / np.linalg.norm(x_o[u::b])
        assert err <= 1e-8, (u, err)


def _iters(s, mode, P=None, base=None, max_it=300):
    if mode == "learned":
        g = learned_solver(s, P, base, max_it=max_it)
    else:
        g = cp.Solver(schur=cp.SCHUR[mode], max_it=max_it)
        g.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
                dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]) if mode == "given" else None)
    _, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-6)
    if mode == "learned":
        assert info["schur_used"] == "learned"
    return info["iters"] if info["status"] == "CPTR_OK" else None


HELD_OUT = {"coupled": lambda: synth.recipe("three_phase_coupled").system(),
            "mid": lambda: three_phase(16, 16, 4, seed=41, c_o=3e-8, beta_o=1e-2),
            "weak": lambda: three_phase(16, 16, 4, seed=42)}


def test_learned_scaling_of_se_gains_nothing_measurable():
    """The network trained on the exact diagonal ratio (S_T)_ii / (S_e)_ii: the targets stay within
    0.3% of 1 (S_e is close to exact on this model), so the learned form matches S_e's iteration
    count (+-1) and gains nothing measurable; printed for the record."""
    P = trained_net("se")
    out = {}
    for name, mk in HELD_OUT.items():
        s = mk()
        out[name] = (_iters(s, "given"), _iters(s, "learned", P, "se"))
        assert out[name][0] is not None and out[name][1] is not None
        assert abs(out[name][0] - out[name][1]) <= 1
    print("FGMRES iterations (S_e, learned diag(s) S_e):", out)


def test_learned_scaling_of_att_gain():
    """What the network gains over the method without S_e (A_TT, Sec. 3.3.1): on the strongly
    coupled three-phase case A_TT stalls and diag(s) A_TT converges, though in many more
    iterations than S_e; on weakly coupled cases the scaling costs a few iterations.  The paper's
    S_e is the judge; all counts are printed."""
    P = trained_net("att")
    out = {name: {"se": _iters(mk(), "given"), "att": _iters(mk(), "att"), "learned": _iters(mk(), "learned", P, "att")}
           for name, mk in HELD_OUT.items()}
    print("FGMRES iterations (S_e, A_TT, learned diag(s) A_TT):", out)
    assert out["coupled"]["att"] is None                      # A_TT does not converge in 300 steps
    assert out["coupled"]["learned"] is not None              # diag(s) A_TT does
    assert all(v["learned"] is not None for v in out.values())


@pytest.mark.parametrize("with_st", [True, False])
def test_rejected_network_falls_back(with_st):
    s = three_phase(6, 5, 3)
    P = np.zeros(cp.MLP_NPARAM, np.float32)
    P[-1] = 40.0                                  # y = 40 everywhere: |y| > 30 is rejected
    g = gpu_solver(s, st=with_st, schur=cp.SCHUR["learned"], n_coarse=16)
    cp.cptr_set_mlp(g.ctx, P)
    g.setup(s["n"], s["b"], dev(s["row_ptr"]), dev(s["col_idx"]), dev(s["vals"].reshape(-1)),
            dev(s["unknown_kind"]), dev(s["weights"].reshape(-1)), dev(s["st"]) if with_st else None)
    x, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["schur_used"] == ("given" if with_st else "att")
    ref = gpu_solver(s, st=with_st, schur=cp.SCHUR["given" if with_st else "att"], n_coarse=16)
    x_r, info_r = ref.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["iters"] == info_r["iters"] and torch.equal(x, x_r)
    sc = np.zeros(s["n"])
    cp.cptr_schur_scaling(g.ctx, sc)
    assert np.all(sc == 1.0)


def test_learned_without_network_uses_the_fallback():
    s = three_phase(6, 5, 3)
    g = gpu_solver(s, schur=cp.SCHUR["learned"], n_coarse=16)
    _, info = g.solve(dev(s["rhs"].reshape(-1)), 1e-8)
    assert info["schur_used"] == "given"
    with pytest.raises(cp.CptrError):
        cp.cptr_mlp_infer(g.ctx, dev(np.zeros((4, 16))), torch.zeros(4, device="cuda"))
