"""FP64 CPU oracle for CPTR/CPR-preconditioned FGMRES (arXiv 1907.04229) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The CUDA library never calls it and shares no code with it.  ``oracle.c`` holds the
arithmetic (every step cites the paper's passage); this module only compiles it and marshals
numpy arrays.

Parity status of each oracle function is pinned by ``tests/test_oracle_pins.py``; nothing here is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

CPTR_FULL, CPTR_UPPER, CPTR_LOWER, BD, CPR, NONE1, UAMG = range(7)
ILU0, NONE2 = 0, 1
SCHUR_GIVEN, SCHUR_ATT, SCHUR_DIAG = 0, 1, 3
DECOUPLE_NONE, DECOUPLE_QI, DECOUPLE_TI = 0, 1, 2
L1, JACOBI = 0, 1


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".tmp"
        subprocess.check_call(["gcc", "-O3", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Opts(ctypes.Structure):
    _fields_ = [("stage1", ctypes.c_int32), ("stage2", ctypes.c_int32), ("schur", ctypes.c_int32),
                ("smoother", ctypes.c_int32), ("omega", ctypes.c_double), ("theta", ctypes.c_double),
                ("n_coarse", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_it", ctypes.c_int32), ("dense_max", ctypes.c_int32), ("seed", ctypes.c_int32),
                ("ilu_order", ctypes.c_int32), ("precision", ctypes.c_int32), ("decouple", ctypes.c_int32),
                ("ilu_fill", ctypes.c_int32), ("part", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("est_rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("bnorm", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.or_create.restype = P
        lib.or_create.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, ctypes.c_int32, ctypes.c_int32,
                                  P, P, P, P]
        lib.or_status.restype = ctypes.c_int
        lib.or_status.argtypes = [P]
        lib.or_destroy.restype = None
        lib.or_destroy.argtypes = [P]
        lib.or_solve.restype = ctypes.c_int
        lib.or_solve.argtypes = [P, P, P, ctypes.c_double, P]
        lib.or_solve_block.restype = ctypes.c_int
        lib.or_solve_block.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_double, P]
        for name in ("or_precond", "or_stage1", "or_ilu_apply", "or_spmv", "or_weight_rhs"):
            getattr(lib, name).restype = None
            getattr(lib, name).argtypes = [P, P, P]
        lib.or_vcycle.restype = None
        lib.or_vcycle.argtypes = [P, ctypes.c_int, P, P]
        lib.or_nlevels.restype = ctypes.c_int
        lib.or_nlevels.argtypes = [P, ctypes.c_int]
        lib.or_hier_level_info.restype = None
        lib.or_hier_level_info.argtypes = [P, ctypes.c_int, P]
        lib.or_hier_level_get.restype = None
        lib.or_hier_level_get.argtypes = [P, ctypes.c_int] + [P] * 8
        lib.or_hierarchy.restype = P
        lib.or_hierarchy.argtypes = [P, ctypes.c_int]
        lib.or_amg_create.restype = P
        lib.or_amg_create.argtypes = [ctypes.c_int32, P, P, P, P, P]
        lib.or_uamg_create.restype = P
        lib.or_uamg_create.argtypes = [ctypes.c_int32, P, P, P, ctypes.c_int32, P, P]
        lib.or_amg_destroy.restype = None
        lib.or_amg_destroy.argtypes = [P]
        lib.or_amg_vcycle.restype = None
        lib.or_amg_vcycle.argtypes = [P, P, P]
        lib.or_amg_nlevels.restype = ctypes.c_int
        lib.or_amg_nlevels.argtypes = [P]
        lib.or_nnz.restype = ctypes.c_int32
        lib.or_nnz.argtypes = [P]
        lib.or_matrix.restype = None
        lib.or_matrix.argtypes = [P, P, P, P]
        lib.or_ilu_nnz.restype = ctypes.c_int32
        lib.or_ilu_nnz.argtypes = [P]
        lib.or_ilu_pattern.restype = None
        lib.or_ilu_pattern.argtypes = [P, P, P]
        lib.or_ilu_order.restype = None
        lib.or_ilu_order.argtypes = [P, P]
        lib.or_ilu_factors.restype = None
        lib.or_ilu_factors.argtypes = [P, P]
        lib.or_field.restype = None
        lib.or_field.argtypes = [P, ctypes.c_int, P]
        lib.or_round_bf16.restype = ctypes.c_double
        lib.or_round_bf16.argtypes = [ctypes.c_double]
        lib.or_splitmix64.restype = ctypes.c_uint64
        lib.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.or_schur_features.restype = None
        lib.or_schur_features.argtypes = [P, P, P]
        lib.or_att.restype = None
        lib.or_att.argtypes = [P, P]
        lib.or_mlp_nparam.restype = ctypes.c_int
        lib.or_mlp_nparam.argtypes = []
        lib.or_mlp_forward.restype = None
        lib.or_mlp_forward.argtypes = [P, P, ctypes.c_int32, P]
        lib.or_mlp_loss_grad.restype = ctypes.c_double
        lib.or_mlp_loss_grad.argtypes = [P, P, P, ctypes.c_int32, P]
        lib.or_adam_step.restype = None
        lib.or_adam_step.argtypes = [P, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double]
        lib.or_mlp_infer_bf16.restype = None
        lib.or_mlp_infer_bf16.argtypes = [P, P, ctypes.c_int32, P]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def default_opts(**kw) -> Opts:
    o = Opts(stage1=CPTR_FULL, stage2=ILU0, schur=SCHUR_GIVEN, smoother=L1, omega=2.0 / 3.0, theta=0.25,
             n_coarse=256, max_levels=25, restart=30, max_it=1000, dense_max=1024, seed=0, ilu_order=0, precision=0,
             decouple=0, ilu_fill=0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Oracle:
    """One CPTR/CPR-FGMRES setup on a BSR Jacobian (raw rows, weights applied inside)."""

    def __init__(self, n, b, row_ptr, col_idx, vals, weights=None, ps=0, ts=1, st=None, st_pattern=None, **opts):
        lib = _load()
        self.n, self.b = int(n), int(b)
        self._keep = []

        def keep(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        rp, ci = keep(row_ptr, np.int32), keep(col_idx, np.int32)
        v = keep(vals, np.float64)
        W = keep(weights, np.float64)
        st_v = keep(st, np.float64)
        if st_pattern is not None:
            st_rp, st_ci = keep(st_pattern[0], np.int32), keep(st_pattern[1], np.int32)
        else:
            st_rp, st_ci = rp, ci
        part = keep(opts.pop("part", None), np.int32)   # block-Jacobi ILU(0) over these parts
        self.opts = default_opts(**opts)
        self.opts.part = _p(part)
        if st_v is None and self.opts.schur == SCHUR_GIVEN:
            self.opts.schur = SCHUR_ATT
        self._c = lib.or_create(self.n, self.b, _p(rp), _p(ci), _p(v), _p(W), ps, ts, _p(st_rp), _p(st_ci),
                                _p(st_v), ctypes.byref(self.opts))
        self.status = lib.or_status(self._c)
        if self.status != 0:
            raise RuntimeError(f"oracle setup failed with status {self.status}")

    @classmethod
    def from_system(cls, sys: dict, use_st: bool = True, **opts) -> "Oracle":
        return cls(sys["n"], sys["b"], sys["row_ptr"], sys["col_idx"], sys["vals"], sys["weights"],
                   st=sys["st"] if use_st else None, **opts)

    def __del__(self):
        if getattr(self, "_c", None):
            _load().or_destroy(self._c)
            self._c = None

    @property
    def nb(self):
        return self.n * self.b

    def solve(self, rhs, rtol=1e-8):
        lib = _load()
        rhs = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
        x = np.zeros(self.nb)
        st = Stats()
        rc = lib.or_solve(self._c, _p(rhs), _p(x), rtol, ctypes.byref(st))
        return x, dict(rc=rc, iters=st.iters, restarts=st.restarts, converged=bool(st.converged),
                       est_rel_res=st.est_rel_res, true_rel_res=st.true_rel_res, bnorm=st.bnorm)

    def solve_block(self, cell0, ncell, rhs, rtol=1e-8):
        """FGMRES on the diagonal block of cells [cell0, cell0 + ncell) of a block-diagonal set-up
        (one instance of an ensemble), with the whole preconditioner restricted to the block."""
        lib = _load()
        rhs = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
        x = np.zeros(ncell * self.b)
        st = Stats()
        rc = lib.or_solve_block(self._c, cell0, ncell, _p(rhs), _p(x), rtol, ctypes.byref(st))
        if rc == -1:
            raise ValueError("the block couples to cells outside it")
        return x, dict(rc=rc, iters=st.iters, restarts=st.restarts, converged=bool(st.converged),
                       est_rel_res=st.est_rel_res, true_rel_res=st.true_rel_res, bnorm=st.bnorm)

    def _vec_op(self, name, v, nout=None):
        lib = _load()
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        out = np.zeros(nout if nout is not None else self.nb)
        getattr(lib, name)(self._c, _p(v), _p(out))
        return out

    def precond(self, v):
        return self._vec_op("or_precond", v)

    def stage1(self, v):
        return self._vec_op("or_stage1", v)

    def ilu_apply(self, r):
        return self._vec_op("or_ilu_apply", r)

    def spmv(self, x):
        return self._vec_op("or_spmv", x)

    def weight_rhs(self, rhs):
        return self._vec_op("or_weight_rhs", rhs)

    def vcycle(self, which, bvec):
        lib = _load()
        bvec = np.ascontiguousarray(bvec, dtype=np.float64)
        x = np.zeros_like(bvec)
        lib.or_vcycle(self._c, which, _p(bvec), _p(x))
        return x

    def matrix(self):
        """Decoupled A' as scalar interleaved CSR (rp, ci, v)."""
        lib = _load()
        nnz = lib.or_nnz(self._c)
        rp = np.zeros(self.nb + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros(nnz)
        lib.or_matrix(self._c, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def dense(self):
        rp, ci, v = self.matrix()
        A = np.zeros((self.nb, self.nb))
        for i in range(self.nb):
            A[i, ci[rp[i]:rp[i + 1]]] += v[rp[i]:rp[i + 1]]
        return A

    def ilu_order(self):
        """Cell order of the ILU(0) factorisation: new index -> original cell."""
        out = np.zeros(self.n, np.int32)
        _load().or_ilu_order(self._c, _p(out))
        return out

    def ilu_factors(self):
        """Values of the ILU factors on their pattern (that of A', or the ILU(1) fill pattern)."""
        lib = _load()
        nnz = lib.or_ilu_nnz(self._c)
        v = np.zeros(nnz)
        lib.or_ilu_factors(self._c, _p(v))
        return v

    def ilu_pattern(self):
        lib = _load()
        nnz = lib.or_ilu_nnz(self._c)
        rp, ci = np.zeros(self.nb + 1, np.int32), np.zeros(nnz, np.int32)
        lib.or_ilu_pattern(self._c, _p(rp), _p(ci))
        return rp, ci

    def field(self, f, nnz):
        lib = _load()
        v = np.zeros(nnz)
        lib.or_field(self._c, f, _p(v))
        return v

    def schur_features(self, base):
        """The 16 local features of every cell for the learned Schur scaling, [n, 16] FP64, with
        the base approximation B given by its values on the cell pattern."""
        base = np.ascontiguousarray(base, np.float64)
        f = np.zeros((self.n, 16))
        _load().or_schur_features(self._c, _p(base), _p(f))
        return f

    def att(self, nnz):
        """A_TT of A' on the cell pattern."""
        v = np.zeros(nnz)
        _load().or_att(self._c, _p(v))
        return v

    def levels(self, which):
        """AMG hierarchy of A_pp (which=0), S~_T (which=1) or, with the uAMG first stage, of A_00 in
        unknown-wise order (which=2): list of dicts per level."""
        lib = _load()
        return _levels(lib.or_hierarchy(self._c, which), lib.or_nlevels(self._c, which))


def _levels(h, nlev):
    lib = _load()
    out = []
    for l in range(nlev):
        info = np.zeros(5, np.int32)
        lib.or_hier_level_info(h, l, _p(info))
        n, nnz, nnzP, nc, dense = (int(t) for t in info)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1))
        dinv = np.zeros(max(n, 1))
        coarse = nc > 0
        cf = np.zeros(n, np.int32) if coarse else None
        Prp = np.zeros(n + 1, np.int32) if coarse else None
        Pci = np.zeros(max(nnzP, 1), np.int32) if coarse else None
        Pv = np.zeros(max(nnzP, 1)) if coarse else None
        lib.or_hier_level_get(h, l, _p(rp), _p(ci), _p(v), _p(dinv), _p(cf), _p(Prp), _p(Pci), _p(Pv))
        lev = dict(n=n, rp=rp, ci=ci[:nnz], v=v[:nnz], dinv=dinv[:n], dense=bool(dense))
        if coarse:
            lev.update(cf=cf, nc=nc, Prp=Prp, Pci=Pci[:nnzP], Pv=Pv[:nnzP])
        out.append(lev)
    return out


class AMG:
    """Standalone oracle AMG hierarchy on a scalar CSR matrix (strength, PMIS, direct
    interpolation, Galerkin RAP, smoother diagonal, dense coarsest solve).  With ``np`` given, the
    unknown-based AMG of Sec. 3.4 on a matrix in unknown-wise order whose first ``np`` rows are the
    first unknown."""

    def __init__(self, rp, ci, v, np_first=None, **opts):
        lib = _load()
        self._keep = [np.ascontiguousarray(rp, np.int32), np.ascontiguousarray(ci, np.int32),
                      np.ascontiguousarray(v, np.float64)]
        self.n = len(rp) - 1
        self.opts = default_opts(**opts)
        st = ctypes.c_int(0)
        if np_first is None:
            self._h = lib.or_amg_create(self.n, *(_p(a) for a in self._keep), ctypes.byref(self.opts),
                                        ctypes.byref(st))
        else:
            self._h = lib.or_uamg_create(self.n, *(_p(a) for a in self._keep), int(np_first),
                                         ctypes.byref(self.opts), ctypes.byref(st))
        if st.value != 0:
            raise RuntimeError(f"oracle AMG setup failed with status {st.value}")

    def __del__(self):
        if getattr(self, "_h", None):
            _load().or_amg_destroy(self._h)
            self._h = None

    def vcycle(self, bvec):
        bvec = np.ascontiguousarray(bvec, dtype=np.float64)
        x = np.zeros_like(bvec)
        _load().or_amg_vcycle(self._h, _p(bvec), _p(x))
        return x

    def levels(self):
        lib = _load()
        return _levels(self._h, lib.or_amg_nlevels(self._h))


def round_bf16(x: float) -> float:
    return float(_load().or_round_bf16(x))


def splitmix64(seed: int, i: int) -> int:
    return int(_load().or_splitmix64(seed, i))


# ---------------------------------------------------------------------------------------------
# learned diagonal scaling of the Schur approximation (network 16-64-64-1, tanh)

N_FEATURES, N_HIDDEN = 16, 64


def mlp_nparam() -> int:
    return int(_load().or_mlp_nparam())


def mlp_forward(params, X):
    P = np.ascontiguousarray(params, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    y = np.zeros(X.shape[0])
    _load().or_mlp_forward(_p(P), _p(X), X.shape[0], _p(y))
    return y


def mlp_loss_grad(params, X, t):
    """(loss, gradient) of the mean squared error of the FP64 network."""
    P = np.ascontiguousarray(params, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    t = np.ascontiguousarray(t, np.float64)
    g = np.zeros(mlp_nparam())
    loss = _load().or_mlp_loss_grad(_p(P), _p(X), _p(t), X.shape[0], _p(g))
    return float(loss), g


def adam_step(params, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on FP64 arrays (step number t >= 1)."""
    for a in (params, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    _load().or_adam_step(_p(params), _p(m), _p(v), _p(g), len(params), t, lr, beta1, beta2, eps)


def mlp_train(params, X, t, steps, lr=1e-3):
    """Full-batch Adam from zero moments; returns (trained params, loss before each step)."""
    P = np.array(params, np.float64)
    m, v = np.zeros_like(P), np.zeros_like(P)
    losses = []
    for k in range(1, steps + 1):
        loss, g = mlp_loss_grad(P, X, t)
        losses.append(loss)
        adam_step(P, m, v, g, k, lr)
    return P, np.array(losses)


def mlp_infer_bf16(params32, X):
    """Network output as the BF16 inference form computes it (FP32 result)."""
    P = np.ascontiguousarray(params32, np.float32)
    X = np.ascontiguousarray(X, np.float64)
    y = np.zeros(X.shape[0], np.float32)
    _load().or_mlp_infer_bf16(_p(P), _p(X), X.shape[0], _p(y))
    return y


def exact_schur_diag(o: "Oracle", sys: dict, chunk: int = 512):
    """Diagonal of the exact S_T = A_TT - A_Tp A_pp^{-1} A_pT of A' (Sec. 3.2 eq. A00 and the Schur
    complement of Sec. 3.3), with A_pp^{-1} applied by a sparse LU factorisation (library step), in
    column chunks: (A_Tp X)_ii with X = A_pp^{-1} A_pT[:, chunk]."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n, rp, ci = sys["n"], sys["row_ptr"], sys["col_idx"]
    nnz = int(rp[-1])
    mk = lambda v: sp.csr_matrix((v, ci, rp), shape=(n, n))
    App, ApT, ATp = (mk(o.field(f, nnz)) for f in range(3))
    ATT = mk(o.att(nnz))
    lu = spl.splu(App.tocsc())
    ApTc = ApT.tocsc()
    d = np.zeros(n)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        X = lu.solve(ApTc[:, c0:c1].toarray())
        d[c0:c1] = np.einsum("ij,ji->i", ATp[c0:c1, :].toarray(), X)
    return ATT.diagonal() - d


def _fields_oracle(sys):
    return Oracle.from_system(sys, use_st=False, max_levels=1, dense_max=1, stage2=NONE2)


def schur_base(sys: dict, base: str, o: "Oracle" = None):
    """Base approximation B of the learned scaling on the cell pattern: the caller's S_e
    (base="se", the generator's "st") or A_TT of A' (base="att")."""
    if base == "se":
        return np.ascontiguousarray(sys["st"], np.float64)
    o = o or _fields_oracle(sys)
    return o.att(int(sys["row_ptr"][-1]))


def schur_ratio_target(sys: dict, base: str = "se", S_diag=None):
    """Training target of the learned scaling, asinh((S_T)_ii / B_ii), and the features.
    S_diag (the exact diagonal of S_T) is computed when not given."""
    o = _fields_oracle(sys)
    B = schur_base(sys, base, o)
    rp, ci = sys["row_ptr"], sys["col_idx"]
    diag = np.array([B[rp[i] + np.searchsorted(ci[rp[i]:rp[i + 1]], i)] for i in range(sys["n"])])
    if S_diag is None:
        S_diag = exact_schur_diag(o, sys)
    return np.arcsinh(S_diag / diag), o.schur_features(B)


def learned_st(sys: dict, params32, base: str = "se"):
    """S~_T = diag(s) B with s = sinh(y) of the BF16 network over the oracle's features;
    returns (st values on the cell pattern, s, y)."""
    o = _fields_oracle(sys)
    B = schur_base(sys, base, o)
    y = mlp_infer_bf16(params32, o.schur_features(B))
    s = np.sinh(y.astype(np.float64))
    rows = np.repeat(np.arange(sys["n"]), np.diff(sys["row_ptr"]))
    return B * s[rows], s, y


def newton_step(reservoir, x, xn, rtol_lin=1e-8, max_newton=20, **opts):
    """One implicit Euler step from state xn by Newton's method with a backtracking line search (Sec. 3
    eq. (AXR), Sec. 4), the oracle's restatement of the library's cptr_newton: F(x) = ||W R(x)||_2
    with the generator's residual (pinned by finite differences); each iteration solves
    J dx = -R with the oracle's CPTR-FGMRES (Jacobian, S_e and weights of the generator) to
    rtol_lin; a = 1, 1/2, ... (at most 10 halvings) until F(x + a dx) <= (1 - 1e-4 a) F(x);
    converged when F <= 1e-8 F(x^0), or when ||a dx|| <= 1e-8 ||x|| with F <= F(x^0).
    Returns (x, dict(newton_its, linear_its, line_search_cuts, converged, res0, res, per_iteration))."""
    W = reservoir.weights()
    n, b = reservoir.n, reservoir.b
    x = np.array(x, dtype=np.float64).reshape(n, b)
    xn = np.asarray(xn, dtype=np.float64).reshape(n, b)

    def F(R):
        return float(np.sqrt(np.sum(np.einsum("nij,nj->ni", W, R) ** 2)))

    F0 = F(reservoir.evaluate(x, jacobian=False, schur=False, xn=xn)["R"])
    Fx, tol = F0, 1e-8
    out = dict(newton_its=0, linear_its=0, line_search_cuts=0, converged=False, res0=F0, per_iteration=[])
    for it in range(max_newton):
        if not Fx > tol * F0:
            out["converged"] = True
            break
        ev = reservoir.evaluate(x, jacobian=True, schur=True, xn=xn)
        o = Oracle(n, b, ev["row_ptr"], ev["col_idx"], ev["J"], W, st=ev["Se"], **opts)
        dx, info = o.solve(-ev["R"].reshape(-1), rtol_lin)
        dx = dx.reshape(n, b)
        out["linear_its"] += info["iters"]
        a, cut = 1.0, 0
        while True:
            xt = x + a * dx
            Ft = F(reservoir.evaluate(xt, jacobian=False, schur=False, xn=xn)["R"])
            if Ft <= (1.0 - 1e-4 * a) * Fx or cut >= 10:
                break
            a *= 0.5
            cut += 1
        out["line_search_cuts"] += cut
        out["per_iteration"].append(dict(linear_its=info["iters"], alpha=a, res=Ft))
        step, xnorm = a * np.linalg.norm(dx), np.linalg.norm(x)
        x, Fx = xt, Ft
        out["newton_its"] = it + 1
        if step <= tol * xnorm:
            out["converged"] = Fx <= F0
            break
    if not out["converged"] and not Fx > tol * F0:
        out["converged"] = True
    out["res"] = Fx
    return x, out

