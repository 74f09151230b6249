"""ctypes + numpy wrapper around ``jacobi_oracle.c`` (test infrastructure only)."""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_LIB = os.path.join(_HERE, "libjacobi_oracle.so")
_lock = threading.Lock()
_lib = None

EPS = 2.0 ** -53


def build_oracle(force=False):
    """Compile jacobi_oracle.c into libjacobi_oracle.so next to it (gcc, -O2, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.oracle_hsvd.argtypes = [I, I, I, P, I, P, D, I, P, I, P, P]
            lib.oracle_hsvd.restype = I
            lib.oracle_eigenpairs.argtypes = [I, I, I, P, I, P, P, P, I, P]
            lib.oracle_eigenpairs.restype = None
            lib.oracle_rotation_params.argtypes = [D, D, D, I, P, P, P]
            lib.oracle_rotation_params.restype = None
            lib.oracle_pairs_modulus.argtypes = [I, I, I, P]
            lib.oracle_pairs_modulus.restype = I
            lib.oracle_pairs_round_robin.argtypes = [I, I, P]
            lib.oracle_pairs_round_robin.restype = I
            lib.oracle_pairs_cycle_weight.argtypes = [I, P, P, P]
            lib.oracle_pairs_cycle_weight.restype = I
            lib.oracle_block_offsets.argtypes = [I, I, P]
            lib.oracle_block_offsets.restype = None
            lib.oracle_check_offdiag.argtypes = [I, I, I, P, I, P, P]
            lib.oracle_check_offdiag.restype = None
            lib.oracle_check_vjv.argtypes = [I, I, P, I, P, P]
            lib.oracle_check_vjv.restype = D
            lib.oracle_check_factor_residual.argtypes = [I, I, I, P, I, P, I, P, I]
            lib.oracle_check_factor_residual.restype = D
            lib.oracle_eig_backward.argtypes = [I, P, P, P, P, D, P]
            lib.oracle_eig_backward.restype = None
            lib.oracle_set_mutation.argtypes = [I]
            lib.oracle_set_mutation.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as_fortran(G):
    """Column-major copy with the interleaved (re, im) layout for complex input."""
    cplx = np.iscomplexobj(G)
    A = np.asfortranarray(G, dtype=np.complex128 if cplx else np.float64).copy(order="F")
    return A, cplx


def set_mutation(k):
    """Plant mistake k in the oracle (0 = none); used only by the mutation tests."""
    load().oracle_set_mutation(int(k))


def hsvd(G, J=None, tol=None, max_sweeps=60, want_v=True):
    """Row-cyclic one-sided Jacobi on a copy of G.  Returns (G_final, V, sweeps, rotations, status)."""
    lib = load()
    A, cplx = _as_fortran(G)
    m, n = A.shape
    if J is None:
        J = np.ones(n, dtype=np.int8)
    J = np.ascontiguousarray(J, dtype=np.int8)
    if tol is None:
        tol = n * EPS
    V = np.zeros((n, n), dtype=A.dtype, order="F") if want_v else None
    sw = ctypes.c_int(0)
    rot = ctypes.c_longlong(0)
    st = lib.oracle_hsvd(m, n, int(cplx), _ptr(A), max(m, 1), _ptr(J), float(tol), int(max_sweeps),
                         _ptr(V) if want_v else None, max(n, 1), ctypes.byref(sw), ctypes.byref(rot))
    if st < 0:
        raise ValueError("oracle_hsvd: invalid argument")
    return A, V, sw.value, rot.value, st


def eigenpairs(Gf, J=None):
    """(lambda ascending, U normalized columns, perm) from a converged factor."""
    lib = load()
    A, cplx = _as_fortran(Gf)
    m, n = A.shape
    if J is None:
        J = np.ones(n, dtype=np.int8)
    J = np.ascontiguousarray(J, dtype=np.int8)
    lam = np.zeros(n)
    U = np.zeros((m, n), dtype=A.dtype, order="F")
    perm = np.zeros(n, dtype=np.int32)
    lib.oracle_eigenpairs(m, n, int(cplx), _ptr(A), max(m, 1), _ptr(J), _ptr(lam), _ptr(U), max(m, 1),
                          _ptr(perm))
    return lam, U, perm


def solve(G, J=None, tol=None, max_sweeps=60, want_v=True):
    """Full oracle solve: dict with lam, U, V (sorted like lam), Gf (sorted), sweeps, rotations, status."""
    Gf, V, sweeps, rot, st = hsvd(G, J, tol, max_sweeps, want_v)
    n = Gf.shape[1]
    if J is None:
        J = np.ones(n, dtype=np.int8)
    lam, U, perm = eigenpairs(Gf, J)
    out = dict(lam=lam, U=U, perm=perm, Gf=Gf[:, perm], sweeps=sweeps, rotations=rot, status=st,
               J=np.asarray(J, dtype=np.int8)[perm])
    out["V"] = V[:, perm] if V is not None else None
    return out


def rotation_params(a, d, beta, hyperbolic):
    lib = load()
    c = ctypes.c_double()
    s = ctypes.c_double()
    t = ctypes.c_double()
    lib.oracle_rotation_params(float(a), float(d), float(beta), int(hyperbolic), ctypes.byref(c),
                               ctypes.byref(s), ctypes.byref(t))
    return c.value, s.value, t.value


def pairs_modulus(nb, k, modified=False):
    lib = load()
    buf = np.zeros(2 * nb, dtype=np.int32)
    np_ = lib.oracle_pairs_modulus(nb, k, int(modified), _ptr(buf))
    return buf[: 2 * np_].reshape(np_, 2)


def pairs_round_robin(nb, s):
    lib = load()
    buf = np.zeros(2 * nb, dtype=np.int32)
    np_ = lib.oracle_pairs_round_robin(nb, s, _ptr(buf))
    return buf[: 2 * np_].reshape(np_, 2)


def pairs_cycle_weight(nb, W):
    """Greedy per-cycle ordering from the weight matrix W (nb x nb, upper triangle used)."""
    lib = load()
    W = np.ascontiguousarray(W, dtype=np.float64)
    npairs = nb * (nb - 1) // 2
    half = nb // 2
    pairs = np.full((npairs * half + half) * 2, -1, dtype=np.int32)
    counts = np.zeros(npairs + 1, dtype=np.int32)
    steps = lib.oracle_pairs_cycle_weight(nb, _ptr(W), _ptr(pairs), _ptr(counts))
    tab = pairs[: steps * half * 2].reshape(steps, half, 2)
    return [tab[s, : counts[s]].copy() for s in range(steps)]


def block_offsets(n, nb):
    lib = load()
    off = np.zeros(nb + 1, dtype=np.int32)
    lib.oracle_block_offsets(n, nb, _ptr(off))
    return off


def check_offdiag(Gf):
    lib = load()
    A, cplx = _as_fortran(Gf)
    m, n = A.shape
    o = ctypes.c_double()
    mx = ctypes.c_double()
    lib.oracle_check_offdiag(m, n, int(cplx), _ptr(A), max(m, 1), ctypes.byref(o), ctypes.byref(mx))
    return o.value, mx.value


def check_vjv(V, J, J_col=None):
    """|| V^* J V - J_col ||_F in long double; J signs V's rows, J_col (default J) its columns."""
    lib = load()
    A, cplx = _as_fortran(V)
    n = A.shape[0]
    J = np.ascontiguousarray(J, dtype=np.int8)
    Jc = J if J_col is None else np.ascontiguousarray(J_col, dtype=np.int8)
    return lib.oracle_check_vjv(n, int(cplx), _ptr(A), max(n, 1), _ptr(J), _ptr(Jc))


def check_factor_residual(G0, V, Gf):
    lib = load()
    A0, cplx = _as_fortran(G0)
    Vv, _ = _as_fortran(V)
    Af, _ = _as_fortran(Gf)
    m, n = A0.shape
    return lib.oracle_check_factor_residual(m, n, int(cplx), _ptr(A0), max(m, 1), _ptr(Vv), max(n, 1),
                                            _ptr(Af), max(m, 1))


def eig_backward(lam, U, lam_bar, U_bar, mask=1e-12):
    """Reference H_bar for L(lambda, U) of a real symmetric H = U diag(lam) U^T (long double)."""
    lib = load()
    n = len(lam)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    U = np.asfortranarray(U, dtype=np.float64)
    lb = np.ascontiguousarray(lam_bar, dtype=np.float64) if lam_bar is not None else None
    Ub = np.asfortranarray(U_bar, dtype=np.float64) if U_bar is not None else None
    H = np.zeros((n, n), order="F")
    lib.oracle_eig_backward(n, _ptr(lam), _ptr(U), _ptr(lb) if lb is not None else None,
                            _ptr(Ub) if Ub is not None else None, float(mask), _ptr(H))
    return H
