"""Pins of the seeded input generator (model of Sec. 2 of arXiv 1907.04229)."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(J, rp, ci, n, b):
    A = np.zeros((n * b, n * b))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i * b:(i + 1) * b, ci[k] * b:(ci[k] + 1) * b] = J[k]
    return A


def _dense_scalar(v, rp, ci, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] += v[rp[i]:rp[i + 1]]
    return A


def test_splitmix64_published_outputs():
    # first three outputs of SplitMix64 from state 0 (Vigna's reference implementation)
    assert [int(v) for v in synth.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normals_moments():
    z = synth.normal(123, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_water_correlations_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "water_properties.txt")) if l.strip() and not l.startswith("#")]
    for p, T, rho, trho, mu, tmu, _ in rows:
        r, m = synth.water(float(p), float(T))
        if rho != "nan":
            assert abs(r - float(rho)) <= float(trho) * float(rho), (p, T, r)
        if mu != "nan":
            assert abs(m - float(mu)) <= float(tmu) * float(mu), (p, T, m)


@pytest.mark.parametrize("nphase", [2, 3])
def test_jacobian_matches_central_differences(nphase):
    r = synth.make_box(4, 3, 2, 3.125, seed=5, nphase=nphase, heaters=[(3, 100.0, 400.0)])
    x = r.x0.copy()
    x[:, 1] += 20 * synth.uniform(77, r.n)       # a non-uniform temperature
    x[:, 0] += 1e5 * synth.normal(78, r.n)       # away from x^n, generic upwind directions
    ev = r.evaluate(x)
    n, b = r.n, r.b
    A = _dense(ev["J"], ev["row_ptr"], ev["col_idx"], n, b)
    xf = x.reshape(-1)
    Afd = np.zeros_like(A)
    for c in range(n * b):
        h = 1e-6 * max(abs(xf[c]), 1.0)
        xp, xm = xf.copy(), xf.copy()
        xp[c] += h
        xm[c] -= h
        Afd[:, c] = (r.evaluate(xp, False, False)["R"].reshape(-1) - r.evaluate(xm, False, False)["R"].reshape(-1)) / (2 * h)
    col = np.abs(A).max(axis=0)
    assert (np.abs(A - Afd) / col).max() < 1e-6


def test_flux_jacobian_conserves():
    # with no accumulation (dt -> inf) and no wells, every flux leaves one cell and enters another:
    # each column of each equation family sums to zero
    r = synth.make_box(4, 4, 3, 3.125, seed=9, wells="none", dt=1e300)
    ev = r.evaluate(r.x0)
    A = _dense(ev["J"], ev["row_ptr"], ev["col_idx"], r.n, r.b)
    for eq in range(r.b):
        s = A[eq::r.b].sum(axis=0)
        assert np.abs(s).max() <= 1e-9 * np.abs(A[eq::r.b]).max()
    Se = _dense_scalar(ev["Se"], ev["row_ptr"], ev["col_idx"], r.n)
    assert np.abs(Se.sum(axis=0)).max() <= 1e-9 * np.abs(Se).max()


def test_schur_operator_equals_att_without_thermal_properties():
    # eq. (Se) differentiates only the explicit T factors; if rho, mu do not depend on T and no
    # producer is present, that is exactly the energy/T block of the Jacobian
    r = synth.make_box(5, 4, 3, 3.125, seed=3, wells="none", thermal_props_off=True, heaters=[(7, 50.0, 420.0)])
    r.wells = [(0, 0, 1e-5, 373.15)]
    x = r.x0.copy()
    x[:, 1] += 30 * synth.uniform(5, r.n)
    ev = r.evaluate(x)
    Att = ev["J"][:, 1, 1]
    assert np.abs(ev["Se"] - Att).max() <= 1e-14 * np.abs(Att).max()


def test_schur_operator_differs_with_thermal_properties():
    r = synth.make_box(5, 4, 3, 3.125, seed=3)
    ev = r.evaluate(r.x0)
    assert np.abs(ev["Se"] - ev["J"][:, 1, 1]).max() > 1e-6 * np.abs(ev["J"][:, 1, 1]).max()


def test_schur_operator_symmetric_without_flow():
    # no pressure differences, no gravity, no wells: accumulation + symmetric conduction only
    r = synth.make_box(4, 4, 3, 3.125, seed=4, wells="none", gravity=False, p_sigma=0.0)
    r.x0[:, 0] = synth.P0
    ev = r.evaluate(r.x0)
    S = _dense_scalar(ev["Se"], ev["row_ptr"], ev["col_idx"], r.n)
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    off = S - np.diag(np.diag(S))
    assert (off <= 0).all() and (np.diag(S) > 0).all()


def test_pattern_is_seven_point():
    r = synth.make_box(5, 4, 3, 1.0, seed=1)
    rp, ci = r.pattern()
    assert rp[-1] == 5 * 4 * 3 + 2 * (4 * 4 * 3 + 5 * 3 * 3 + 5 * 4 * 2)
    for i in range(r.n):
        row = ci[rp[i]:rp[i + 1]]
        assert (np.diff(row) > 0).all() and i in row


def test_weights_structure():
    r = synth.recipe("parity")
    W = r.weights()[0]
    Tref = r.T0
    assert W[0, 0] == Tref * r.cv_w and W[0, 2] == Tref * r.cv_o      # eq. (weighted) scaled by T_ref
    assert W[1, 1] == 1.0 and abs(W[1]).sum() == 1.0                    # energy row untouched
    cref = 0.8 * r.cv_o + 0.2 * r.cv_w
    assert abs(W[2, 0] - cref * Tref) < 1e-9 * cref * Tref               # c_ref T_ref on the kept mass row
