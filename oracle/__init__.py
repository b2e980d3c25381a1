"""CPU oracle for the periodic Ewald-RPY Brownian-dynamics step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA path.

The heavy parts (D assembly, forces, plain-loop products, the Chebyshev
recurrence, the Euler step, Philox) are in ``bd_oracle.c``, compiled here with
gcc in IEEE binary64 (no fast-math, no FMA contraction).  Exact eigenvalues,
the Cholesky factor and the eigen-decomposition square root used by the pins
come from numpy's LAPACK routines, used as library primitives.

Passages followed (paper sections / equations):
  * D blocks ............ Eq. (Domega), Eq. (DF), Eq. (M1), Eq. (M2),
                          Eqs. (cor1)-(cor5), Eq. (DFmodified)
  * forces .............. Sec. II A (Hookean / FENE springs); narrow-Gaussian EV
  * Chebyshev sqrt ...... Sec. IV, Eqs. (cheb1)-(cheb3), E_f definition
  * Euler step .......... Eq. (sde), FENE rejection (Sec. VII)
  * bounds check ........ Sec. IV, d_max >= lambda_max, d_min <= lambda_min
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_bd.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, defines=()) -> str:
    """Compile bd_oracle.c into oracle/_build/ (gcc, OpenMP).

    ``defines`` names PLANT_* switches; they are used only by the mutation
    test, which builds variants with one deliberate mistake each."""
    os.makedirs(_BUILD, exist_ok=True)
    tag = "".join("_" + d.lower() for d in defines)
    path = os.path.join(_BUILD, f"liboracle_bd{tag}_{platform.machine()}.so")
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", "-D_GNU_SOURCE"]
    cmd += ["-D" + d for d in defines]
    cmd += [_SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("nb", ctypes.c_int32),
        ("L", ctypes.c_double), ("a", ctypes.c_double),
        ("alpha", ctypes.c_double), ("rc", ctypes.c_double),
        ("n2max", ctypes.c_int32), ("overlap_corr", ctypes.c_int32),
        ("spring", ctypes.c_int32), ("fene_b", ctypes.c_double),
        ("ev_on", ctypes.c_int32), ("z_star", ctypes.c_double),
        ("d_star", ctypes.c_double), ("r_ev", ctypes.c_double),
        ("dt", ctypes.c_double),
    ]


def _params(p: dict) -> OracleParams:
    return OracleParams(
        n=int(p["n"]), nb=int(p["nb"]), L=float(p["L"]), a=float(p["a"]),
        alpha=float(p["alpha"]), rc=float(p["rc"]), n2max=int(p["n2max"]),
        overlap_corr=int(p.get("overlap_corr", 1)), spring=int(p.get("spring", 0)),
        fene_b=float(p.get("fene_b", 0.0)), ev_on=int(p.get("ev_on", 0)),
        z_star=float(p.get("z_star", 0.0)), d_star=float(p.get("d_star", 1.0)),
        r_ev=float(p.get("r_ev", 0.0)), dt=float(p.get("dt", 0.0)))


_dp = ctypes.POINTER(ctypes.c_double)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _load(path):
    L = ctypes.CDLL(path)
    P = ctypes.POINTER(OracleParams)
    L.oracle_build_D_rows.argtypes = [P, _dp, ctypes.c_int32, ctypes.c_int32, _dp]
    L.oracle_build_D.argtypes = [P, _dp, _dp]
    L.oracle_D_block.argtypes = [P, _dp, ctypes.c_int32, ctypes.c_int32, _dp]
    L.oracle_forces.argtypes = [P, _dp, _dp]
    L.oracle_forces.restype = ctypes.c_int32
    L.oracle_apply_D.argtypes = [ctypes.c_int32, _dp, _dp, ctypes.c_int32, _dp]
    L.oracle_apply_rows.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    _dp, _dp, ctypes.c_int32, _dp]
    L.oracle_cheb_coeffs.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, _dp]
    L.oracle_cheb_sqrt.argtypes = [ctypes.c_int32, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int32, _dp, ctypes.c_int32, _dp, _dp]
    L.oracle_step.argtypes = [P, _dp, _dp, ctypes.c_int32, ctypes.c_double,
                              ctypes.c_double, ctypes.c_int32, _dp, _dp, _dp]
    L.oracle_step.restype = ctypes.c_int32
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.oracle_wiener_philox.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int64, ctypes.c_double, _dp]
    L.oracle_num_threads.restype = ctypes.c_int32
    L.oracle_grad_DF_R.argtypes = [P, _dp, _dp, _dp, _dp]
    L.oracle_grad_pairs_R.argtypes = [P, _dp, _dp, _dp, ctypes.c_int32, _dp]
    return L


_active = threading.local()


def lib():
    """The loaded oracle library (a planted variant inside ``variant()``)."""
    global _lib
    v = getattr(_active, "lib", None)
    if v is not None:
        return v
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


class variant:
    """Context manager: route this module's functions to a variant build
    with the given PLANT_* switches (mutation test only)."""

    def __init__(self, *defines):
        self.defines = defines

    def __enter__(self):
        self.prev = getattr(_active, "lib", None)
        _active.lib = _load(build(defines=self.defines))
        return self

    def __exit__(self, *exc):
        _active.lib = self.prev
        return False


# --------------------------------------------------------------------------
# Thin numpy wrappers.  Positions R are (n, 3) C-contiguous float64 (bead
# index major, i.e. the 3N vector with index 3*nu + s).  Multi-column vectors
# are stored as (m, 3N) arrays: row j of the array is column j of the 3N x m
# matrix.

def build_D(p: dict, R: np.ndarray) -> np.ndarray:
    """Dense 3N x 3N diffusion tensor, Eq. (DFmodified) block by block."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = int(p["n"])
    D = np.empty((3 * n, 3 * n), dtype=np.float64)
    lib().oracle_build_D(ctypes.byref(_params(p)), _ptr(R), _ptr(D))
    return D


def build_D_rows(p: dict, R: np.ndarray, r0: int, r1: int) -> np.ndarray:
    """Bead rows [r0, r1) of D (3*(r1-r0) x 3N)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = int(p["n"])
    D = np.empty((3 * (r1 - r0), 3 * n), dtype=np.float64)
    lib().oracle_build_D_rows(ctypes.byref(_params(p)), _ptr(R), r0, r1, _ptr(D))
    return D


def D_block(p: dict, R: np.ndarray, nu: int, mu: int) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.float64)
    B = np.empty(9, dtype=np.float64)
    lib().oracle_D_block(ctypes.byref(_params(p)), _ptr(R), int(nu), int(mu), _ptr(B))
    return B.reshape(3, 3)


def forces(p: dict, R: np.ndarray):
    """Spring + excluded-volume forces (3N,) and the over-stretch count."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    F = np.empty(3 * int(p["n"]), dtype=np.float64)
    bad = lib().oracle_forces(ctypes.byref(_params(p)), _ptr(R), _ptr(F))
    return F, int(bad)


def apply_D(D: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = D X by plain loops; X, Y are (m, 3N) (columns as rows)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
    Y = np.empty_like(X)
    lib().oracle_apply_D(D.shape[0], _ptr(D), _ptr(X), X.shape[0], _ptr(Y))
    return Y


def cheb_coeffs(nch: int, dmin: float, dmax: float) -> np.ndarray:
    c = np.empty(nch, dtype=np.float64)
    lib().oracle_cheb_coeffs(int(nch), float(dmin), float(dmax), _ptr(c))
    return c


def cheb_sqrt(D: np.ndarray, dmin: float, dmax: float, nch: int, dW: np.ndarray):
    """Fixman-Chebyshev dS ~ sqrt(D) dW and E_f per column (Sec. IV)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    dW = np.ascontiguousarray(np.atleast_2d(dW), dtype=np.float64)
    dS = np.empty_like(dW)
    Ef = np.empty(dW.shape[0], dtype=np.float64)
    lib().oracle_cheb_sqrt(D.shape[0], _ptr(D), float(dmin), float(dmax), int(nch),
                           _ptr(dW), dW.shape[0], _ptr(dS), _ptr(Ef))
    return dS, Ef


def fixman_bounds(D: np.ndarray, nbeads: int, mode: str, C: float = 0.0):
    """Sec. IV: lambda^F_max = U+.D.U+ / 3N, lambda^F_min = U-.D.U- / 3N
    (Eq. lmax-lmin-dilute; U+ all ones, U- alternating +1, -1).  mode
    'dilute': (d_min, d_max) = (lambda^F_min / 2, 2 lambda^F_max); mode
    'semidilute': lambda_max = 0.35 N^0.6 lambda^F_max (Eq. fmax),
    lambda_min = lambda_max / (C N^0.6) (Eq. fmin), used as the bounds.
    Returns (d_min, d_max, lambda^F_max, lambda^F_min)."""
    n3 = D.shape[0]
    up = np.ones(n3)
    um = np.where(np.arange(n3) % 2 == 0, 1.0, -1.0)
    lmaxF = float(up @ D @ up) / n3
    lminF = float(um @ D @ um) / n3
    if mode == "dilute":
        return 0.5 * lminF, 2.0 * lmaxF, lmaxF, lminF
    n06 = float(nbeads) ** 0.6
    lmax = 0.35 * n06 * lmaxF
    return lmax / (C * n06), lmax, lmaxF, lminF


def nch_initial(dmin: float, dmax: float) -> int:
    """Eq. (nint): N_Ch = nint(sqrt(lambda_max / lambda_min)) + 1, with the
    bounds standing in for the extreme eigenvalues (nint rounds halves up)."""
    return int(math.floor(math.sqrt(dmax / dmin) + 0.5)) + 1


def cheb_sqrt_adaptive(D: np.ndarray, dmin: float, dmax: float, dW: np.ndarray, tol: float,
                       nch_max: int):
    """Sec. IV: start from Eq. (nint) and raise N_Ch by one until E_f < tol in
    every column (at most nch_max).  Each candidate is the full series of
    cheb_sqrt.  Returns (dS, Ef, N_Ch, converged)."""
    n = max(2, min(nch_initial(dmin, dmax), nch_max))
    while True:
        dS, Ef = cheb_sqrt(D, dmin, dmax, n, dW)
        if float(np.max(Ef)) < tol:
            return dS, Ef, n, True
        if n >= nch_max:
            return dS, Ef, n, False
        n += 1


def step(p: dict, R: np.ndarray, dW: np.ndarray, dmin: float, dmax: float, nch: int):
    """One Euler step, Eq. (sde).  Returns (R_new, status, DF, dS, Ef)."""
    Rn = np.ascontiguousarray(R, dtype=np.float64).copy()
    dW = np.ascontiguousarray(np.atleast_2d(dW), dtype=np.float64)
    n3 = 3 * int(p["n"])
    DF = np.zeros(n3)
    dS = np.zeros_like(dW)
    Ef = np.zeros(dW.shape[0])
    st = lib().oracle_step(ctypes.byref(_params(p)), _ptr(Rn), _ptr(dW), dW.shape[0],
                           float(dmin), float(dmax), int(nch), _ptr(DF), _ptr(dS), _ptr(Ef))
    return Rn, int(st), DF, dS, Ef


def grad_DF(p: dict, R: np.ndarray, F: np.ndarray, g: np.ndarray):
    """Gradient of L = g . D(R) F: returns (dL/dR as (N, 3), dL/dF = D g)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    gR = np.empty(3 * int(p["n"]), dtype=np.float64)
    lib().oracle_grad_DF_R(ctypes.byref(_params(p)), _ptr(R), _ptr(F), _ptr(g), _ptr(gR))
    D = build_D(p, R)
    return gR.reshape(-1, 3), D @ g


def grad_pairs(p: dict, R: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """dL/dR when dL/dD = sum_q x_q y_q^T (X, Y of shape (Q, 3N)); (N, 3)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.float64)
    Y = np.ascontiguousarray(np.atleast_2d(Y), dtype=np.float64)
    gR = np.empty(3 * int(p["n"]), dtype=np.float64)
    lib().oracle_grad_pairs_R(ctypes.byref(_params(p)), _ptr(R), _ptr(X), _ptr(Y), X.shape[0],
                              _ptr(gR))
    return gR.reshape(-1, 3)


def cheb_adjoint(D: np.ndarray, dmin: float, dmax: float, nch: int, dW: np.ndarray,
                 h: np.ndarray):
    """Reverse pass of the Chebyshev series of Sec. IV for L(dS) with
    dL/ddS = h (both (m, 3N)), bounds and N_Ch held fixed.  Forward:
    V_0 = dW, V_1 = Y V_0, V_p = 2 Y V_{p-1} - V_{p-2}, dS = sum c_p V_p - c_0/2 V_0,
    Y = s D - t I.  Adjoints U_p = dL/dV_p run the recurrence backwards:
    U_{N-1} = c_{N-1} h, U_p = c_p h + 2 Y U_{p+1} - U_{p+2} (p >= 1), and
    dL/dD = s (U_1 V_0^T + 2 sum_{p>=2} U_p V_{p-1}^T),  dL/ddW = U_0.
    Returns (X, Y) with dL/dD = sum_q X_q Y_q^T, and dL/ddW."""
    dW = np.atleast_2d(dW).astype(np.float64)
    h = np.atleast_2d(h).astype(np.float64)
    c = cheb_coeffs(nch, dmin, dmax)
    s = 2.0 / (dmax - dmin)
    t = (dmax + dmin) / (dmax - dmin)
    Yop = lambda V: s * (V @ D.T) - t * V          # rows are vectors; D symmetric
    V = [dW]
    if nch > 1:
        V.append(Yop(dW))
    for p_ in range(2, nch):
        V.append(2.0 * Yop(V[-1]) - V[-2])
    U = [None] * (nch + 2)
    U[nch] = np.zeros_like(h)
    U[nch + 1] = np.zeros_like(h)
    for p_ in range(nch - 1, 0, -1):
        U[p_] = c[p_] * h + 2.0 * Yop(U[p_ + 1]) - U[p_ + 2]
    # V_1 = Y V_0 has coefficient 1, so U_0 gets Y U_1 (not 2 Y U_1)
    U0 = 0.5 * c[0] * h + (Yop(U[1]) if nch > 1 else 0.0) - (U[2] if nch > 2 else 0.0)
    Xs, Ys = [], []
    if nch > 1:
        Xs.append(s * U[1]); Ys.append(V[0])
    for p_ in range(2, nch):
        Xs.append(2.0 * s * U[p_]); Ys.append(V[p_ - 1])
    m = dW.shape[0]
    X = np.concatenate(Xs, axis=0) if Xs else np.zeros((0, dW.shape[1]))
    Yv = np.concatenate(Ys, axis=0) if Ys else np.zeros((0, dW.shape[1]))
    return X, Yv, U0


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def wiener_philox(seed: int, step_index: int, count: int, dt: float) -> np.ndarray:
    out = np.empty(int(count), dtype=np.float64)
    lib().oracle_wiener_philox(ctypes.c_uint64(seed), ctypes.c_uint64(step_index),
                               int(count), float(dt), _ptr(out))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# --------------------------------------------------------------------------
# Library-primitive helpers used by the pins (numpy LAPACK).

def exact_eigs(D: np.ndarray):
    """Extreme eigenvalues of the symmetric D (Sec. IV, 'exact' eigenvalues)."""
    w = np.linalg.eigvalsh(D)
    return float(w[0]), float(w[-1])


def sqrt_eig(D: np.ndarray) -> np.ndarray:
    """Symmetric square root of D from its eigen-decomposition."""
    w, V = np.linalg.eigh(D)
    return (V * np.sqrt(w)) @ V.T


def cholesky(D: np.ndarray) -> np.ndarray:
    return np.linalg.cholesky(D)
