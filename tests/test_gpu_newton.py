"""The step either side of the solve on the device: the model's residual, Jacobian and S_e assembled
by the library against the input generator's assembly (which finite differences pin), and Newton's
method with a line search (Sec. 3 eq. AXR, Sec. 4) against the oracle's Newton driver.

Tolerances: the assembly uses the same operations in the same order as the generator, but exp, pow
and the division of the device library may differ from the host's by an ulp: 1e-13 relative to each
array's largest entry.  Newton: equal Newton iteration counts, linear iterations +-1 per Newton
iteration, and the final states within 1e-8 per unknown kind (both converge the residual to 1e-8 of
its start along the same path)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
import paper_1907_04229_gb300 as cp  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def reservoirs():
    return {
        "two_phase_heater": synth.make_box(7, 5, 3, 3.125, seed=17, heaters=[(11, 80.0, 420.0)]),
        "two_phase_wells": synth.make_box(9, 8, 4, 3.125, seed=3),
        "three_phase": synth.make_box(6, 5, 3, 3.125, seed=19, nphase=3, wells="four"),
        "layered_conduction": synth.make_box(12, 10, 5, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True,
                                             kv_ratio=0.1, kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=30 * 86400.0),
        "mesh_aniso": synth.mesh_refinement_case("aniso", 20),
    }


def model_solver(r, **opts):
    S = cp.Solver(**opts)
    cp.cptr_model_set(S.ctx, r.model_fields())
    return S


@pytest.mark.parametrize("name", list(reservoirs()))
def test_assembly_matches_generator(name):
    r = reservoirs()[name]
    S = model_solver(r)
    n, b = r.n, r.b
    rng = np.random.default_rng(8)
    x0 = r.x0.copy()
    # the initial state and a perturbed one (other upwind directions, active producers)
    x1 = x0.copy()
    x1[:, 0] += 2e5 * rng.standard_normal(n)
    x1[:, 1] += 3.0 * rng.standard_normal(n)
    x1[:, 2] += 0.02 * rng.standard_normal(n)
    for x in (x0, x1):
        ev = r.evaluate(x, jacobian=True, schur=True)
        R = torch.empty(n * b, dtype=torch.float64, device="cuda")
        J = torch.empty(ev["J"].size, dtype=torch.float64, device="cuda")
        Se = torch.empty(ev["Se"].size, dtype=torch.float64, device="cuda")
        cp.cptr_assemble(S.ctx, dev(x.reshape(-1)), dev(r.x0.reshape(-1)), R, J, Se)
        for got, want in ((R, ev["R"]), (J, ev["J"]), (Se, ev["Se"])):
            got, want = got.cpu().numpy().reshape(-1), np.asarray(want).reshape(-1)
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err <= 1e-13, err
    # host arrays give the same values
    Rh = np.zeros(n * b)
    cp.cptr_assemble(S.ctx, np.ascontiguousarray(x1.reshape(-1)), np.ascontiguousarray(r.x0.reshape(-1)), Rh)
    R = torch.empty(n * b, dtype=torch.float64, device="cuda")
    cp.cptr_assemble(S.ctx, dev(x1.reshape(-1)), dev(r.x0.reshape(-1)), R)
    assert np.array_equal(Rh, R.cpu().numpy())


@pytest.mark.parametrize("name", ["two_phase_heater", "two_phase_wells", "three_phase", "layered_conduction"])
def test_newton_time_steps_match_oracle(name):
    """Three implicit Euler steps by Newton's method with CPTR-FGMRES, on the device and in the oracle."""
    r = reservoirs()[name]
    opts = dict(n_coarse=16)
    S = model_solver(r, **opts)
    n, b = r.n, r.b
    xg = dev(r.x0.reshape(-1)).clone()
    xo = r.x0.copy()
    for step in range(3):
        xn_g, xn_o = xg.clone(), xo.copy()
        ig = cp.cptr_newton(S.ctx, xg, xn_g, 1e-8, 20)
        xo, io = oracle.newton_step(r, xo, xn_o, 1e-8, **opts)
        print(f"{name} step {step}: Newton {ig['newton_its']} (oracle {io['newton_its']}), linear {ig['linear_its']} "
              f"(oracle {io['linear_its']}), cuts {ig['line_search_cuts']}, ||W R|| {ig['res0']:.3e} -> {ig['res']:.3e}")
        assert ig["status"] == "CPTR_OK" and io["converged"]
        assert ig["newton_its"] == io["newton_its"]
        assert abs(ig["linear_its"] - io["linear_its"]) <= io["newton_its"]
        x = xg.cpu().numpy().reshape(n, b)
        for u in range(b):
            err = np.linalg.norm(x[:, u] - xo[:, u]) / np.linalg.norm(xo[:, u])
            assert err <= 1e-8, (step, u, err)


def test_newton_needs_a_model():
    S = cp.Solver()
    x = torch.zeros(12, dtype=torch.float64, device="cuda")
    with pytest.raises(cp.CptrError) as e:
        cp.cptr_newton(S.ctx, x, x.clone(), 1e-8, 5)
    assert e.value.code == -7
