"""Seeded synthetic inputs for the CPTR solver: thermal multiphase Jacobians on Cartesian grids.

This package is the one module that both the FP64 oracle and the CUDA path are fed from.  It
builds the linear system of one Newton step of the model of arXiv 1907.04229 (Sec. 2: phase mass
+ energy conservation, TPFA, upwinding, implicit Euler) together with the per-cell equation
weights of eqs. (weighted) and (scaling) and the discrete Schur approximation S_e of eq. (Se).
It contains none of the solver's arithmetic: it never applies the weights, extracts blocks,
builds AMG, factors ILU or iterates.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014), the i-th output of stream ``seed`` being
mix64(seed + (i + 1) * 0x9E3779B97F4A7C15); uniforms take the top 53 bits; normals use one
Box-Muller branch per pair of uniforms.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

MD_TO_M2 = 9.869233e-16
GRAV = 9.80665
P0 = 4.1369e7  # initial pressure, Table 1


def build(force: bool = False) -> str:
    """Compile reservoir.c into libsynth.so (plain C, portable flags)."""
    src = os.path.join(_HERE, "reservoir.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_nnzb.restype = ctypes.c_int64
        lib.synth_nnzb.argtypes = [ctypes.c_void_p]
        lib.synth_pattern.restype = None
        lib.synth_pattern.argtypes = [ctypes.c_void_p] * 3
        lib.synth_assemble.restype = ctypes.c_int
        lib.synth_assemble.argtypes = [ctypes.c_void_p] * 8
        lib.synth_water.restype = None
        lib.synth_water.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        _lib = lib
    return _lib


# ----------------------------------------------------------------------------------------------
# counter-based random numbers
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 stream started at state ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from stream ``seed``."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals, Box-Muller cosine branch over consecutive uniform pairs."""
    u = uniform(seed, 2 * n).reshape(n, 2)
    return np.sqrt(-2.0 * np.log(1.0 - u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


# ----------------------------------------------------------------------------------------------
class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("nphase", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("dt", ctypes.c_double), ("phi", ctypes.c_double), ("grav", ctypes.c_double),
        ("kh", ctypes.c_void_p), ("kv", ctypes.c_void_p),
        ("kT_const", ctypes.c_double),
        ("kT_rock", ctypes.c_double), ("kT_w", ctypes.c_double), ("kT_o", ctypes.c_double), ("kT_g", ctypes.c_double),
        ("cv_w", ctypes.c_double), ("cv_o", ctypes.c_double), ("cv_g", ctypes.c_double),
        ("c_rock", ctypes.c_double), ("rho_rock", ctypes.c_double),
        ("mu_o_ref", ctypes.c_double), ("beta_mu", ctypes.c_double), ("T0", ctypes.c_double),
        ("rho_o_ref", ctypes.c_double), ("c_o", ctypes.c_double), ("beta_o", ctypes.c_double), ("p0", ctypes.c_double),
        ("gas_M", ctypes.c_double), ("mu_g", ctypes.c_double),
        ("corey_n", ctypes.c_double),
        ("thermal_props_off", ctypes.c_int32), ("n_wells", ctypes.c_int32),
        ("T_props", ctypes.c_double),
        ("well_cell", ctypes.c_void_p), ("well_kind", ctypes.c_void_p),
        ("well_a", ctypes.c_void_p), ("well_c", ctypes.c_void_p),
        ("heater_cell", ctypes.c_void_p), ("heater_U", ctypes.c_void_p), ("heater_T", ctypes.c_void_p),
        ("n_heaters", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Reservoir:
    """A seeded reservoir state and the physical constants of one implicit Euler step.

    Defaults are Table 1 of the paper (conductivities, specific heats, rock density 2650 kg/m^3,
    initial pressure) and Sec. 4 (porosity 0.2).  The oil, gas and producer laws are stated
    readings because the paper defers them to a companion paper.
    """
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    kh_md: np.ndarray                 # [N] horizontal permeability, mD
    kv_md: np.ndarray                 # [N] vertical permeability, mD
    x0: np.ndarray                    # [N, b] state of the previous step (and the Newton iterate)
    nphase: int = 2
    dt: float = 86400.0
    phi: float = 0.2
    grav: float = GRAV
    kT_const: float = 0.0             # > 0: constant conductivity (W/m/K)
    kT_rock: float = 1.7295772056
    kT_w: float = 0.6005638
    kT_o: float = 0.15
    kT_g: float = 0.03
    cv_w: float = 4181.3
    cv_o: float = 2093.4
    cv_g: float = 2200.0
    c_rock: float = 920.0
    rho_rock: float = 2650.0
    mu_o_ref: float = 1.0             # Pa s at T0 (heavy oil)
    beta_mu: float = 0.03             # 1/K, exponential viscosity-temperature law
    T0: float = 300.0
    rho_o_ref: float = 1000.0         # API 10: oil as dense as water at reference conditions
    c_o: float = 1e-9                 # 1/Pa
    beta_o: float = 5e-4              # 1/K
    p0: float = P0
    gas_M: float = 0.016              # kg/mol, ideal gas
    mu_g: float = 1.5e-5
    corey_n: float = 2.0
    thermal_props_off: bool = False   # densities/viscosities independent of T (test mode)
    T_props: float = 300.0
    wells: list = field(default_factory=list)    # (cell, kind, a, c): kind 0 inj (q, T_inj); 1 prod (WI, p_bh)
    heaters: list = field(default_factory=list)  # (cell, U, T_heater)
    sw0_nominal: float = 0.2
    sg0_nominal: float = 0.0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def b(self) -> int:
        return self.nphase + 1

    def cell(self, x: int, y: int, z: int) -> int:
        return x + self.nx * (y + self.ny * z)

    def depth(self) -> np.ndarray:
        z = np.arange(self.n) // (self.nx * self.ny)
        return (z + 0.5) * self.dz

    # ------------------------------------------------------------------------------------------
    def _struct(self):
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return _ptr(a) if a.size else None

        P = _Problem()
        P.nx, P.ny, P.nz, P.nphase = self.nx, self.ny, self.nz, self.nphase
        P.dx, P.dy, P.dz = self.dx, self.dy, self.dz
        P.dt, P.phi, P.grav = self.dt, self.phi, self.grav
        P.kh = arr(self.kh_md * MD_TO_M2, np.float64)
        P.kv = arr(self.kv_md * MD_TO_M2, np.float64)
        for name in ("kT_const", "kT_rock", "kT_w", "kT_o", "kT_g", "cv_w", "cv_o", "cv_g", "c_rock",
                     "rho_rock", "mu_o_ref", "beta_mu", "T0", "rho_o_ref", "c_o", "beta_o", "p0",
                     "gas_M", "mu_g", "corey_n", "T_props"):
            setattr(P, name, float(getattr(self, name)))
        P.thermal_props_off = int(self.thermal_props_off)
        w = self.wells
        P.n_wells = len(w)
        P.well_cell = arr([c for c, _, _, _ in w], np.int32)
        P.well_kind = arr([k for _, k, _, _ in w], np.int32)
        P.well_a = arr([a for _, _, a, _ in w], np.float64)
        P.well_c = arr([c for _, _, _, c in w], np.float64)
        h = self.heaters
        P.n_heaters = len(h)
        P.heater_cell = arr([c for c, _, _ in h], np.int32)
        P.heater_U = arr([u for _, u, _ in h], np.float64)
        P.heater_T = arr([t for _, _, t in h], np.float64)
        return P, keep

    def pattern(self):
        lib = _load()
        P, keep = self._struct()
        nnzb = lib.synth_nnzb(ctypes.byref(P))
        rp = np.zeros(self.n + 1, np.int32)
        ci = np.zeros(nnzb, np.int32)
        lib.synth_pattern(ctypes.byref(P), _ptr(rp), _ptr(ci))
        return rp, ci

    def evaluate(self, x: np.ndarray, jacobian: bool = True, schur: bool = True, xn: np.ndarray = None):
        """Residual R(x) (raw rows) of the step from xn (default: x0), and optionally the Jacobian
        dR/dx (BSR) and S_e at x."""
        lib = _load()
        P, keep = self._struct()
        rp, ci = self.pattern()
        b = self.b
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.n, b)
        xn = np.ascontiguousarray(self.x0 if xn is None else xn, dtype=np.float64).reshape(self.n, b)
        R = np.zeros((self.n, b))
        J = np.zeros((ci.size, b, b)) if jacobian else None
        Se = np.zeros(ci.size) if schur else None
        rc = lib.synth_assemble(ctypes.byref(P), _ptr(x), _ptr(xn), _ptr(rp), _ptr(ci), _ptr(R),
                                _ptr(J) if jacobian else None, _ptr(Se) if schur else None)
        if rc != 0:
            raise RuntimeError("synth_assemble: inconsistent pattern")
        return dict(R=R, J=J, Se=Se, row_ptr=rp, col_idx=ci)

    def model_fields(self) -> dict:
        """The model as the solver library's cptr_model describes it (SI units, permeabilities in
        m^2, wells and heaters as arrays)."""
        if self.thermal_props_off:
            raise ValueError("the library's model has no property freeze")
        w, h = self.wells, self.heaters
        out = dict(nx=self.nx, ny=self.ny, nz=self.nz, nphase=self.nphase, dx=self.dx, dy=self.dy, dz=self.dz,
                   dt=self.dt, phi=self.phi, grav=self.grav, kh=self.kh_md * MD_TO_M2, kv=self.kv_md * MD_TO_M2,
                   well_cell=np.array([c for c, _, _, _ in w], np.int32),
                   well_kind=np.array([k for _, k, _, _ in w], np.int32),
                   well_a=np.array([a for _, _, a, _ in w], np.float64),
                   well_c=np.array([cc for _, _, _, cc in w], np.float64),
                   heater_cell=np.array([c for c, _, _ in h], np.int32),
                   heater_U=np.array([u for _, u, _ in h], np.float64),
                   heater_T=np.array([t for _, _, t in h], np.float64), weights=self.weights())
        for name in ("kT_const", "kT_rock", "kT_w", "kT_o", "kT_g", "cv_w", "cv_o", "cv_g", "c_rock", "rho_rock",
                     "mu_o_ref", "beta_mu", "T0", "rho_o_ref", "c_o", "beta_o", "p0", "gas_M", "mu_g", "corey_n"):
            out[name] = float(getattr(self, name))
        return out

    def weights(self) -> np.ndarray:
        """Per-cell equation weights W (b x b): decoupled row = W @ raw rows.

        row p = T_ref * sum_alpha c_v,alpha * (mass row alpha)      eq. (weighted), (scaling)
        row T = energy row                                           eq. (scaling)
        row S_w = c_ref * T_ref * (water mass row), S_g likewise     eq. (scaling)
        T_ref = initial reservoir temperature, c_ref = sum_alpha S_alpha^0 c_v,alpha (Sec. 4).
        """
        b = self.b
        Tref = self.T0
        so = 1.0 - self.sw0_nominal - self.sg0_nominal
        cref = so * self.cv_o + self.sw0_nominal * self.cv_w + self.sg0_nominal * (self.cv_g if self.nphase == 3 else 0.0)
        W = np.zeros((b, b))
        # raw rows: 0 water mass, 1 energy, 2 oil mass, 3 gas mass
        W[0, 0] = Tref * self.cv_w
        W[0, 2] = Tref * self.cv_o
        if self.nphase == 3:
            W[0, 3] = Tref * self.cv_g
            W[3, 3] = cref * Tref
        W[1, 1] = 1.0
        W[2, 0] = cref * Tref
        return np.broadcast_to(W, (self.n, b, b)).copy()

    def system(self, schur: bool = True) -> dict:
        """The linear system of the first Newton iteration at x_k = x^n: J dx = -R(x^n).

        Returns n, b, row_ptr, col_idx (int32), vals (raw Jacobian, [nnzb, b, b]), rhs (= -R,
        [n, b]), weights ([n, b, b]), st (S_e on the same pattern, [nnzb]) and unknown_kind.
        """
        ev = self.evaluate(self.x0, jacobian=True, schur=schur)
        kinds = [0, 1] + [2] * (self.b - 2)
        return dict(n=self.n, b=self.b, row_ptr=ev["row_ptr"], col_idx=ev["col_idx"], vals=ev["J"],
                    rhs=-ev["R"], weights=self.weights(), st=ev["Se"], unknown_kind=np.array(kinds, np.int32),
                    grid=(self.nx, self.ny, self.nz))


def water(p: float, T: float):
    """(rho_w, mu_w) of the printed correlations (Appendix A), SI units."""
    lib = _load()
    out = np.zeros(2)
    lib.synth_water(p, T, _ptr(out))
    return float(out[0]), float(out[1])


# ----------------------------------------------------------------------------------------------
# recipes
def _wi(kh_md: np.ndarray, dz: float) -> np.ndarray:
    """Stated producer index WI = 2 pi k_h dz / 5 (m^3), i.e. ln(r_e / r_w) fixed at 5."""
    return 2.0 * math.pi * kh_md * MD_TO_M2 * dz / 5.0


def _initial_state(n, b, depth, seed_s, seed_p, sw0=0.2, sg0=0.0, T0=300.0, p0=P0, sat_amp=0.05, p_sigma=1e4):
    x = np.zeros((n, b))
    x[:, 0] = p0 + 1000.0 * GRAV * depth + p_sigma * normal(seed_p, n)
    x[:, 1] = T0
    x[:, 2] = sw0 + sat_amp * (2.0 * uniform(seed_s, n) - 1.0)
    if b == 4:
        x[:, 3] = sg0 + 0.5 * sat_amp * (2.0 * uniform(seed_s + 1000, n) - 1.0)
    return x


def make_box(nx, ny, nz, dx=3.125, dy=None, dz=None, *, seed=1, sigma=1.0, mean_log=4.0, nphase=2,
             kv_ratio=1.0, layered=False, kT_const=0.0, T_inj=373.15, q_inj=1e-5, dp_prod=5e6,
             wells="corners", heaters=(), thermal_props_off=False, corey_n=2.0, p_sigma=1e4,
             gravity=True, **kw) -> Reservoir:
    """A seeded box reservoir: injector column at (0,0), producer column at (nx-1, ny-1).

    Permeability: ln k_h[mD] = mean_log + sigma * xi with xi iid N(0,1) per cell (stream seed), or
    with ``layered``: xi = 0.8 zeta_layer + 0.6 eta_cell (streams seed, seed+1).  k_v = kv_ratio k_h.
    Initial state: p hydrostatic from P0 plus N(0, p_sigma), T = 300 K, S_w = 0.2 + U(-0.05, 0.05).
    """
    dy = dx if dy is None else dy
    dz = dx if dz is None else dz
    n = nx * ny * nz
    if layered:
        zeta = normal(seed, nz)
        eta = normal(seed + 1, n)
        xi = 0.8 * np.repeat(zeta, nx * ny) + 0.6 * eta
    else:
        xi = normal(seed, n)
    kh = np.exp(mean_log + sigma * xi)
    kv = kh * kv_ratio
    b = nphase + 1
    depth = ((np.arange(n) // (nx * ny)) + 0.5) * dz
    x0 = _initial_state(n, b, depth, seed + 2, seed + 3, sg0=0.05 if nphase == 3 else 0.0, p_sigma=p_sigma)
    r = Reservoir(nx, ny, nz, dx, dy, dz, kh, kv, x0, nphase=nphase, kT_const=kT_const,
                  thermal_props_off=thermal_props_off, corey_n=corey_n,
                  sg0_nominal=0.05 if nphase == 3 else 0.0, **kw)
    if not gravity:
        r.grav = 0.0
    wl = []
    if wells == "corners":
        inj_cols = [(0, 0)]
        prod_cols = [(nx - 1, ny - 1)]
    elif wells == "four":
        # four injectors on the corners of an inner square, four producers at the domain corners
        a, c = nx // 4, (3 * nx) // 4
        ay, cy = ny // 4, (3 * ny) // 4
        inj_cols = [(a, ay), (c, ay), (a, cy), (c, cy)]
        prod_cols = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]
    else:
        inj_cols, prod_cols = [], []
    for (ix, iy) in inj_cols:
        for z in range(nz):
            wl.append((r.cell(ix, iy, z), 0, q_inj / nz, T_inj))
    for (ix, iy) in prod_cols:
        for z in range(nz):
            c = r.cell(ix, iy, z)
            wl.append((c, 1, float(_wi(kh[c:c + 1], dz)[0]), float(x0[c, 0] - dp_prod)))
    r.wells = wl
    r.heaters = list(heaters)
    return r


def recipe(name: str) -> Reservoir:
    """Named workloads.

    parity : 16x16x4 (1024 cells, b=3), lognormal k (mean log 4 mD, sigma 1), 373.15 K injector
             at a corner, producer at the opposite corner, dt = 1 day, Table-1 conductivities.
    cptr200k : 100x100x20 (200k cells, 600k dofs, b=3), layered lognormal k (sigma 2, kv/kh 0.1),
             k_T = 2 W/m/K, 500 K injector, 0.5 x 0.5 x 0.25 m cells.
    three_phase2m : 200x200x50 (2M cells, b=4), lognormal k (sigma 2.5), 4 injectors, 4 producers.
    three_phase_coupled : 16x16x4 three-phase model with c_o = 1e-7 1/Pa, beta_o = 5e-2 1/K.
    """
    if name == "parity":
        return make_box(16, 16, 4, 3.125, seed=1, sigma=1.0)
    if name == "cptr200k":
        return make_box(100, 100, 20, 0.5, 0.5, 0.25, seed=11, sigma=2.0, layered=True, kv_ratio=0.1,
                        kT_const=2.0, T_inj=500.0, q_inj=1e-6, dt=365.0 * 86400.0)
    if name == "three_phase2m":
        return make_box(200, 200, 50, 1.0, 1.0, 0.5, seed=21, sigma=2.5, nphase=3, wells="four",
                        T_inj=500.0, q_inj=4e-6)
    if name == "three_phase_coupled":
        # the three-phase model with a compressible, strongly expanding oil (strong p-T coupling)
        return make_box(16, 16, 4, 1.0, 1.0, 0.5, seed=40, sigma=2.5, nphase=3, wells="four",
                        T_inj=500.0, q_inj=4e-6, c_o=1e-7, beta_o=5e-2)
    raise KeyError(name)


LEARNED_TRAIN_GRIDS = 16


def learned_training_grid(k: int, nx: int = 32, ny: int = 32, nz: int = 8) -> Reservoir:
    """Training grid k of the learned Schur scaling: the three-phase model (sigma 2.5, four
    injectors, four producers, 1 x 1 x 0.5 m cells), permeability seed 101 + k, and the oil's
    compressibility c_o and thermal expansion beta_o drawn log-uniformly per grid from
    [1e-9, 1e-7] 1/Pa and [5e-4, 5e-2] 1/K (uniforms k of stream 900 and of stream 901), so that the
    set spans weak to strong p-T coupling."""
    u1 = float(uniform(900, k + 1)[k])
    u2 = float(uniform(901, k + 1)[k])
    return make_box(nx, ny, nz, 1.0, 1.0, 0.5, seed=101 + k, sigma=2.5, nphase=3, wells="four",
                    T_inj=500.0, q_inj=4e-6, c_o=1e-9 * 100.0 ** u1, beta_o=5e-4 * 100.0 ** u2)


def mlp_init(seed: int, n_features: int = 16, n_hidden: int = 64) -> np.ndarray:
    """Initial parameters of the 16-64-64-1 network (layout W1 | b1 | W2 | b2 | w3 | b3), float32:
    weights N(0, 1/fan_in) from the normal stream ``seed``, biases zero."""
    z = normal(seed, n_hidden * n_features + n_hidden * n_hidden + n_hidden)
    w1 = z[:n_hidden * n_features] / np.sqrt(n_features)
    w2 = z[n_hidden * n_features:n_hidden * n_features + n_hidden * n_hidden] / np.sqrt(n_hidden)
    w3 = z[n_hidden * n_features + n_hidden * n_hidden:] / np.sqrt(n_hidden)
    zero = np.zeros(n_hidden)
    return np.concatenate([w1, zero, w2, zero, w3, [0.0]]).astype(np.float32)


def concat(systems) -> dict:
    """The block-diagonal union of several systems (same b): cells of system k follow those of
    system k - 1.  Returns the union in the layout of ``Reservoir.system()`` plus ``cell0``, the
    first cell of every system and the total at the end."""
    b = systems[0]["b"]
    cell0 = np.zeros(len(systems) + 1, np.int64)
    for k, s in enumerate(systems):
        assert s["b"] == b
        cell0[k + 1] = cell0[k] + s["n"]
    rp, ci, nz = [np.zeros(1, np.int32)], [], 0
    for k, s in enumerate(systems):
        rp.append((s["row_ptr"][1:] + nz).astype(np.int32))
        ci.append((s["col_idx"] + cell0[k]).astype(np.int32))
        nz += int(s["row_ptr"][-1])
    out = {"n": int(cell0[-1]), "b": b, "row_ptr": np.concatenate(rp), "col_idx": np.concatenate(ci),
           "vals": np.concatenate([s["vals"] for s in systems]),
           "weights": np.concatenate([s["weights"] for s in systems]),
           "st": np.concatenate([s["st"] for s in systems]),
           "rhs": np.concatenate([s["rhs"] for s in systems]),
           "unknown_kind": systems[0]["unknown_kind"], "cell0": cell0}
    return out


def mesh_refinement_case(kind: str, N: int) -> Reservoir:
    """The 2-D mesh-refinement workloads (Sec. 4.1.1, Tables meshW, meshH, anisomeshW) on synthetic
    analogues: a 50 m x 50 m square on an N x N grid, represented as an x-z slice one metre thick
    (nx = nz = N, ny = 1) with gravity off, so that the second direction's permeability can differ
    (kind "aniso": 3e-13 m^2 along x, 3e-10 m^2 along the other direction; otherwise 3e-13 m^2
    isotropic), porosity 0.2, initial S_w = 0.1 (S_o = 0.9) with the seeded perturbation, uniform
    initial pressure (1 Pa of seeded noise keeps upwind directions generic), T = 300 K, dt = 10 days.  Six point sources, three on each of two opposite sides (rows N/4, N/2, 3N/4 of
    columns 0 and N-1): kind "heaters" heats all six at 373.15 K (U = 100 W/K each); the well kinds
    inject water at 3e-7 m^3/s and 373.15 K on one side and produce on the other (stated reading:
    producers at a bottom-hole pressure 1 bar below the initial pressure, as the well model here has
    no rate-controlled producer)."""
    d = 50.0 / N
    k_md = 3e-13 / MD_TO_M2
    r = make_box(N, 1, N, d, 1.0, d, seed=61, sigma=0.0, mean_log=math.log(k_md), wells="none", gravity=False,
                 kv_ratio=1000.0 if kind == "aniso" else 1.0, dt=10 * 86400.0, p_sigma=1.0)
    r.x0[:, 0] = P0 + normal(64, N * N)          # uniform initial pressure (no gravity), 1 Pa noise
    r.x0[:, 2] -= 0.1
    rows = [N // 4, N // 2, (3 * N) // 4]
    if kind == "heaters":
        r.heaters = [(r.cell(x, 0, z), 100.0, 373.15) for x in (0, N - 1) for z in rows]
    else:
        wl = [(r.cell(0, 0, z), 0, 3e-7, 373.15) for z in rows]
        for z in rows:
            c = r.cell(N - 1, 0, z)
            wl.append((c, 1, float(_wi(r.kh_md[c:c + 1], 1.0)[0]), float(r.x0[c, 0] - 1e5)))
        r.wells = wl
    return r


def ensemble_sizes(count: int = 64, lo: float = 20e3, hi: float = 500e3, total: float = 4e6, nz: int = 10,
                   seed: int = 31):
    """Cell counts of an ensemble of ``count`` boxes with sizes in [lo, hi] summing to about
    ``total``: N_k = lo (hi / lo)^(u_k^g) with u_k the uniforms of stream ``seed`` and the exponent
    g >= 1 found by bisection so that sum N_k = total (g = 1 is log-uniform; a larger g skews the
    sizes toward lo while keeping the range).  Each instance is an nx x nx x nz box with
    nx = round(sqrt(N_k / nz)).  Returns a list of (nx, ny, nz)."""
    u = uniform(seed, count)
    sizes = lambda g: lo * (hi / lo) ** (u ** g)
    a, b = 1.0, 64.0
    if sizes(a).sum() > total:
        for _ in range(100):
            g = 0.5 * (a + b)
            if sizes(g).sum() > total:
                a = g
            else:
                b = g
    n = sizes(0.5 * (a + b))
    return [(int(round(np.sqrt(v / nz))),) * 2 + (nz,) for v in n]


def ensemble_member(k: int, shape) -> Reservoir:
    """Instance k of the ensemble: the two-phase model of the parity workload (3.125 m cells,
    lognormal permeability sigma 1, corner injector and producer, dt = 1 day) on an
    nx x ny x nz box, permeability seed 100 + k."""
    nx, ny, nz = shape
    return make_box(nx, ny, nz, 3.125, seed=100 + k, sigma=1.0)
