"""Thin ctypes binding of libjacobi_gb300.so (include/jacobi_gb300.h).

Argument marshalling only: output tensors are allocated with PyTorch on the input's device,
pointers and the current CUDA stream are passed to the C entry points of the same names, and
every step of the method runs in the library's kernels.  There is no CPU fallback: if the
library is missing or the tensors are not on a CUDA device, the calls raise.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libjacobi_gb300.so")

JAC_OK, JAC_ENOTCONV, JAC_ENOTPD, JAC_ENONFINITE, JAC_ECUDA, JAC_ENOMEM, JAC_EINTERNAL = range(7)
JAC_R64, JAC_C128 = 0, 1
ORDER = {"modulus": 0, "modulus_mod": 1, "round_robin": 2, "cycle_weight": 3}
FACTOR = {"chol": 0, "chol_diagpiv": 1, "chol_signpiv": 2}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_only": 2}
BLOCK_MODE = {"full": 0, "oriented": 1}
F64_PRODUCTS = {"mma": 0, "split16": 1, "split16_tc": 2}
ABI_VERSION = 500  # JAC_VERSION of include/jacobi_gb300.h whose structs JacOpts / JacInfo mirror


class JacOpts(ctypes.Structure):
    _fields_ = [("block_w", ctypes.c_int), ("ordering", ctypes.c_int), ("block_mode", ctypes.c_int),
                ("factor", ctypes.c_int), ("precision", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("want_v", ctypes.c_int), ("tol", ctypes.c_double), ("f64_products", ctypes.c_int),
                ("fused_step", ctypes.c_int)]


class JacInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("steps_per_sweep", ctypes.c_int), ("rotations", ctypes.c_longlong),
                ("pivots_rotated", ctypes.c_longlong), ("max_scaled_off", ctypes.c_double),
                ("off_rel", ctypes.c_double), ("launches", ctypes.c_longlong), ("lowp_sweeps", ctypes.c_int),
                ("global_ns_steps", ctypes.c_int), ("pivot_ns_steps", ctypes.c_longlong),
                ("pivot_cycles", ctypes.c_longlong * 4), ("sweep_max_scaled", ctypes.c_double * 64),
                ("inner_sweeps", ctypes.c_longlong), ("sweep_ms", ctypes.c_double * 64),
                ("pivots_rotated_lowp", ctypes.c_longlong), ("pairs_evaluated", ctypes.c_longlong),
                ("pairs_evaluated_lowp", ctypes.c_longlong)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("pivot_cycles", "sweep_max_scaled", "sweep_ms")}
        d["pivot_cycles"] = list(self.pivot_cycles)
        d["sweep_max_scaled"] = list(self.sweep_max_scaled[: self.sweeps])
        d["sweep_ms"] = list(self.sweep_ms[: self.sweeps])
        return d



class JacobiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (status %d)" % (msg, code))
        self.code = code


_lib = None

EXPORTS = ("jacobi_default_opts", "jacobi_status_string", "jacobi_version", "jacobi_hsvd", "jacobi_eig_pd",
           "jacobi_sched_pairs", "jacobi_profile_begin", "jacobi_profile_read", "jacobi_profile_end",
           "jacobi_sched_pairs_noalloc", "jacobi_eig_batched", "jacobi_eig_backward", "jacobi_autotune_batched")
KERNEL = {"gram": 0, "pivot": 1, "update": 2, "gram_lowp": 3, "update_lowp": 4, "step_fused": 5}


def load_library(path=LIB_PATH):
    """dlopen the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libjacobi_gb300.so not found at %s; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.jacobi_default_opts.argtypes = [ctypes.POINTER(JacOpts)]
    lib.jacobi_default_opts.restype = None
    lib.jacobi_status_string.argtypes = [I]
    lib.jacobi_status_string.restype = ctypes.c_char_p
    lib.jacobi_version.argtypes = []
    lib.jacobi_version.restype = I
    if lib.jacobi_version() // 100 != ABI_VERSION // 100:  # JacOpts / JacInfo mirror this layout
        raise ImportError("libjacobi_gb300.so is version %d, the binding expects %d: rebuild it"
                          % (lib.jacobi_version(), ABI_VERSION))
    lib.jacobi_hsvd.argtypes = [I, I, I, P, I, P, ctypes.POINTER(JacOpts), P, P, I, P, I, ctypes.POINTER(JacInfo), P]
    lib.jacobi_hsvd.restype = I
    lib.jacobi_eig_pd.argtypes = [I, I, I, P, I, ctypes.POINTER(JacOpts), P, P, I, P, I, ctypes.POINTER(JacInfo), P]
    lib.jacobi_eig_pd.restype = I
    lib.jacobi_sched_pairs.argtypes = [I, I, P, P, P, I, ctypes.POINTER(ctypes.c_int), P]
    lib.jacobi_sched_pairs.restype = I
    lib.jacobi_eig_batched.argtypes = [I, P, P, I, P, P, P, ctypes.POINTER(JacOpts), P, P, P, P, P, P, P]
    lib.jacobi_eig_batched.restype = I
    lib.jacobi_autotune_batched.argtypes = [I, I, P, P]
    lib.jacobi_autotune_batched.restype = I
    L = ctypes.c_longlong
    lib.jacobi_eig_backward.argtypes = [I, I, P, L, P, I, L, P, L, P, I, L, D, P, I, L, P, I, L, P, L, P, I, L, P]
    lib.jacobi_eig_backward.restype = I
    lib.jacobi_sched_pairs_noalloc.argtypes = [I, I, P, P, P, I, ctypes.POINTER(ctypes.c_int), P]
    lib.jacobi_sched_pairs_noalloc.restype = I
    lib.jacobi_profile_begin.argtypes = [I]
    lib.jacobi_profile_begin.restype = I
    lib.jacobi_profile_read.argtypes = [I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)]
    lib.jacobi_profile_read.restype = I
    lib.jacobi_profile_end.argtypes = []
    lib.jacobi_profile_end.restype = I
    _lib = lib
    return lib


def default_opts(**kw):
    lib = load_library()
    o = JacOpts()
    lib.jacobi_default_opts(ctypes.byref(o))
    for key, val in kw.items():
        if key == "ordering" and isinstance(val, str):
            val = ORDER[val]
        elif key == "factor" and isinstance(val, str):
            val = FACTOR[val]
        elif key == "precision" and isinstance(val, str):
            val = PRECISION[val]
        elif key == "block_mode" and isinstance(val, str):
            val = BLOCK_MODE[val]
        elif key == "f64_products" and isinstance(val, str):
            val = F64_PRODUCTS[val]
        setattr(o, key, val)
    return o


def status_string(code):
    return load_library().jacobi_status_string(int(code)).decode()


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _check_cuda(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)


def _colmajor(G):
    """Column-major (Fortran-order) float64 / complex128 copy of a 2-D tensor, as the C ABI
    expects (complex: interleaved (re, im) doubles)."""
    dt = torch.complex128 if G.is_complex() else torch.float64
    Gt = G.to(dt).t().contiguous()  # (n, m) row-major == (m, n) column-major
    return Gt


def _call(fn_name, G, J, opts, want_u, raise_on_error):
    lib = load_library()
    _check_cuda(G, "G")
    m, n = G.shape
    dev = G.device
    Gt = _colmajor(G)  # storage: column c at Gt[c]
    if opts is None:
        opts = default_opts()
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    cplx = Gt.is_complex()
    Ut = torch.empty((n, m), dtype=Gt.dtype, device=dev) if want_u else None
    Vt = torch.empty((n, n), dtype=Gt.dtype, device=dev) if opts.want_v else None
    info = JacInfo()
    args = [m, n, JAC_C128 if cplx else JAC_R64, ctypes.c_void_p(Gt.data_ptr()), m]
    if fn_name == "jacobi_hsvd":
        _check_cuda(J, "J")
        Jd = J.to(device=dev, dtype=torch.int8).contiguous()
        args.append(ctypes.c_void_p(Jd.data_ptr()))
    args += [ctypes.byref(opts), ctypes.c_void_p(lam.data_ptr()),
             ctypes.c_void_p(Ut.data_ptr()) if Ut is not None else None, m,
             ctypes.c_void_p(Vt.data_ptr()) if Vt is not None else None, n, ctypes.byref(info), _stream(dev)]
    rc = getattr(lib, fn_name)(*args)
    if rc != JAC_OK and raise_on_error and not (rc == JAC_ENOTCONV and raise_on_error == "allow_notconv"):
        raise JacobiError(rc, status_string(rc))
    out = dict(lam=lam, G=Gt.t(), U=Ut.t() if Ut is not None else None, V=Vt.t() if Vt is not None else None,
               info=info.as_dict(), status=rc)
    return out


def jacobi_hsvd(G, J, opts=None, want_u=True, raise_on_error=True):
    """One-sided hyperbolic block Jacobi (J != I) / trigonometric (J = I) on the factor G of
    H = G J G^T.  G: (m, n) CUDA tensor (not modified; a column-major copy is solved in place);
    J: (n,) +-1.  Returns dict(lam ascending, G = G_in V, U normalized, V, info, status)."""
    return _call("jacobi_hsvd", G, J, opts, want_u, raise_on_error)


def jacobi_eig_pd(G, opts=None, want_u=True, raise_on_error=True):
    """Positive definite H = G G^T: jacobi_hsvd with J = I."""
    return _call("jacobi_eig_pd", G, None, opts, want_u, raise_on_error)


def jacobi_hsvd_raw(m, n, G_ptr, ldg, J_ptr, opts, lam_ptr, U_ptr, ldu, V_ptr, ldv, stream_ptr, dtype=JAC_R64):
    """Direct pointer-level call (used by the end-to-end timing path); returns (status, info).
    dtype JAC_C128: G, U, V hold interleaved (re, im) doubles, leading dimensions in elements."""
    lib = load_library()
    info = JacInfo()
    rc = lib.jacobi_hsvd(m, n, dtype, ctypes.c_void_p(G_ptr), ldg, ctypes.c_void_p(J_ptr), ctypes.byref(opts),
                         ctypes.c_void_p(lam_ptr), ctypes.c_void_p(U_ptr) if U_ptr else None, ldu,
                         ctypes.c_void_p(V_ptr) if V_ptr else None, ldv, ctypes.byref(info),
                         ctypes.c_void_p(stream_ptr))
    return rc, info.as_dict()


def jacobi_eig_batched_raw(m, n, G_ptrs, ldg, J_ptrs, opts, lam_ptrs, U_ptrs, ldu, V_ptrs, ldv, stream_ptr,
                           want_info=True):
    """Pointer-level batched call.  m, n, ldg, ldu, ldv: int32 numpy arrays; *_ptrs: uint64 numpy
    arrays of device addresses (J_ptrs / U_ptrs / V_ptrs may be None).  Returns (status, infos)
    with infos a JacInfo array (or None)."""
    import numpy as np

    lib = load_library()
    batch = len(m)

    def arr(a, dt):
        if a is None:
            return None, None
        a = np.ascontiguousarray(a, dtype=dt)
        return a, ctypes.c_void_p(a.ctypes.data)

    keep = []
    cargs = []
    for a, dt in ((m, np.int32), (n, np.int32)):
        k, c = arr(a, dt)
        keep.append(k)
        cargs.append(c)
    gk, gc = arr(G_ptrs, np.uint64)
    lk, lc = arr(ldg, np.int32)
    jk, jc = arr(J_ptrs, np.uint64)
    lak, lac = arr(lam_ptrs, np.uint64)
    uk, uc = arr(U_ptrs, np.uint64)
    luk, luc = arr(ldu, np.int32)
    vk, vc = arr(V_ptrs, np.uint64)
    lvk, lvc = arr(ldv, np.int32)
    keep += [gk, lk, jk, lak, uk, luk, vk, lvk]
    infos = (JacInfo * batch)() if want_info and batch > 0 else None
    rc = lib.jacobi_eig_batched(batch, cargs[0], cargs[1], JAC_R64, gc, lc, jc, ctypes.byref(opts), lac, uc, luc, vc,
                                lvc, infos, ctypes.c_void_p(stream_ptr))
    del keep
    return rc, infos


def jacobi_eig_batched(Gs, Js=None, opts=None, want_u=False, raise_on_error=True):
    # raise_on_error=False returns the per-problem statuses in info["status"] (argument and
    # call-wide errors raise regardless)
    """Batched solve of independent problems of uneven order (one call, shared launches).
    Gs: list of (m_b, n_b) CUDA tensors on one device; Js: None (every H positive definite) or a
    list whose entries are (n_b,) +-1 tensors or None (J = I for that problem).  opts.block_w is
    ignored (chosen per size class).  Returns (list of dict(lam, G, U, V, info), status)."""
    import numpy as np

    if opts is None:
        opts = default_opts()
    batch = len(Gs)
    if batch == 0:
        return [], JAC_OK
    dev = Gs[0].device
    for i, G in enumerate(Gs):
        _check_cuda(G, "Gs[%d]" % i)
    Gts = [_colmajor(G) for G in Gs]
    ms = np.array([G.shape[0] for G in Gs], dtype=np.int32)
    ns = np.array([G.shape[1] for G in Gs], dtype=np.int32)
    lams = [torch.empty(int(k), dtype=torch.float64, device=dev) for k in ns]
    Uts = [torch.empty((int(k), int(mm)), dtype=torch.float64, device=dev) for mm, k in zip(ms, ns)] if want_u else None
    Vts = [torch.empty((int(k), int(k)), dtype=torch.float64, device=dev) for k in ns] if opts.want_v else None
    Jds = None
    if Js is not None:
        Jds = [None if J is None else J.to(device=dev, dtype=torch.int8).contiguous() for J in Js]
    ptr = lambda ts: np.array([0 if t is None else t.data_ptr() for t in ts], dtype=np.uint64)
    rc, infos = jacobi_eig_batched_raw(
        ms, ns, ptr(Gts), ms, ptr(Jds) if Jds is not None else None, opts, ptr(lams),
        ptr(Uts) if Uts is not None else None, ms if Uts is not None else None,
        ptr(Vts) if Vts is not None else None, ns if Vts is not None else None, _stream(dev).value or 0)
    if rc < 0 or rc in (JAC_ECUDA, JAC_ENOMEM) or (rc != JAC_OK and raise_on_error):
        raise JacobiError(rc, status_string(rc))
    outs = []
    for i in range(batch):
        outs.append(dict(lam=lams[i], G=Gts[i].t(), U=Uts[i].t() if Uts is not None else None,
                         V=Vts[i].t() if Vts is not None else None, info=infos[i].as_dict()))
    return outs, rc


def jacobi_autotune_batched(count=64, precision="fp64", device="cuda"):
    """Measure and install the fastest block-width rule per size class for jacobi_eig_batched on
    `device`; count=0 restores the defaults.  Returns the rule per order n (index 0..128)."""
    import numpy as np

    lib = load_library()
    dev = torch.device(device)
    rules = np.full(129, -1, dtype=np.int32)
    with torch.cuda.device(dev):
        rc = lib.jacobi_autotune_batched(int(count), PRECISION.get(precision, precision),
                                         ctypes.c_void_p(rules.ctypes.data), _stream(dev))
    if rc != JAC_OK:
        raise JacobiError(rc, status_string(rc))
    return rules


def jacobi_eig_batched_uniform(G, J=None, opts=None, want_u=True, raise_on_error=True):
    """Batched solve of a stack of equal-shape problems.  G: (batch, m, n) CUDA tensor, J: None
    (J = I) or (batch, n) signs.  Outputs are written straight into stacked tensors:
    returns dict(lam (batch, n), G (batch, m, n) = G_in V, U (batch, m, n) or None,
    V (batch, n, n) or None, infos, status)."""
    import numpy as np

    if opts is None:
        opts = default_opts()
    _check_cuda(G, "G")
    batch, m, n = G.shape
    dev = G.device
    Gt = G.to(torch.float64).transpose(-1, -2).contiguous()  # (batch, n, m): column-major m x n each
    lam = torch.empty((batch, n), dtype=torch.float64, device=dev)
    Ut = torch.empty((batch, n, m), dtype=torch.float64, device=dev) if want_u else None
    Vt = torch.empty((batch, n, n), dtype=torch.float64, device=dev) if opts.want_v else None
    Jd = None
    if J is not None:
        _check_cuda(J, "J")
        Jd = J.to(device=dev, dtype=torch.int8).reshape(batch, n).contiguous()
    idx = np.arange(batch, dtype=np.uint64)
    ptrs = lambda t, per: (np.uint64(t.data_ptr()) + idx * np.uint64(per)).astype(np.uint64)
    ms = np.full(batch, m, dtype=np.int32)
    ns = np.full(batch, n, dtype=np.int32)
    rc, infos = jacobi_eig_batched_raw(
        ms, ns, ptrs(Gt, 8 * m * n), ms, ptrs(Jd, n) if Jd is not None else None, opts, ptrs(lam, 8 * n),
        ptrs(Ut, 8 * m * n) if Ut is not None else None, ms if Ut is not None else None,
        ptrs(Vt, 8 * n * n) if Vt is not None else None, ns if Vt is not None else None, _stream(dev).value or 0)
    if rc < 0 or rc in (JAC_ECUDA, JAC_ENOMEM) or (rc != JAC_OK and raise_on_error):
        raise JacobiError(rc, status_string(rc))
    return dict(lam=lam, G=Gt.transpose(-1, -2), U=Ut.transpose(-1, -2) if Ut is not None else None,
                V=Vt.transpose(-1, -2) if Vt is not None else None, infos=infos, status=rc)


def jacobi_eig_backward(lam, U, lam_bar=None, U_bar=None, deg_tol=1e-12, G=None, J=None):
    """Adjoint of the eigendecomposition of square problems.  lam (batch, n), U (batch, n, n)
    (or unbatched (n,), (n, n)); lam_bar / U_bar like them or None.  With G (the input factor,
    same shape as U) and J ((batch, n) signs or None) also returns G_bar = 2 H_bar G J.
    Returns (H_bar, G_bar or None), shaped like U."""
    lib = load_library()
    _check_cuda(U, "U")
    unbatched = U.dim() == 2
    if unbatched:
        lam, U = lam.unsqueeze(0), U.unsqueeze(0)
        lam_bar = lam_bar.unsqueeze(0) if lam_bar is not None else None
        U_bar = U_bar.unsqueeze(0) if U_bar is not None else None
        G = G.unsqueeze(0) if G is not None else None
        J = J.unsqueeze(0) if J is not None else None
    batch, n, n2 = U.shape
    if n2 != n:
        raise ValueError("U must be square (m = n)")
    dev = U.device
    cm = lambda X: X.to(torch.float64).transpose(-1, -2).contiguous()  # column-major storage
    lamc = lam.to(torch.float64).contiguous()
    Uc = cm(U)
    lbc = lam_bar.to(device=dev, dtype=torch.float64).contiguous() if lam_bar is not None else None
    Ubc = cm(U_bar.to(dev)) if U_bar is not None else None
    Gc = cm(G.to(dev)) if G is not None else None
    Jc = J.to(device=dev, dtype=torch.int8).reshape(batch, n).contiguous() if J is not None else None
    Hb = torch.empty((batch, n, n), dtype=torch.float64, device=dev)
    Gb = torch.empty((batch, n, n), dtype=torch.float64, device=dev) if G is not None else None
    vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    nn = n * n
    rc = lib.jacobi_eig_backward(batch, n, vp(lamc), n, vp(Uc), n, nn, vp(lbc), n, vp(Ubc), n, nn, float(deg_tol),
                                 vp(Hb), n, nn, vp(Gc), n, nn, vp(Jc), n, vp(Gb), n, nn, _stream(dev))
    if rc != JAC_OK:
        raise JacobiError(rc, status_string(rc))
    Hb = Hb.transpose(-1, -2)
    Gb = Gb.transpose(-1, -2) if Gb is not None else None
    if unbatched:
        Hb = Hb[0]
        Gb = Gb[0] if Gb is not None else None
    return Hb, Gb


def jacobi_sched_pairs(nb, ordering, weights=None, device="cuda", max_steps=None, noalloc=False):
    """Device scheduler: list of (count, 2) int tensors, one per step of a cycle.  noalloc=True
    calls jacobi_sched_pairs_noalloc (library-resident scratch, no device allocation)."""
    lib = load_library()
    if isinstance(ordering, str):
        ordering = ORDER[ordering]
    half = nb // 2
    if max_steps is None:
        max_steps = 2 * nb
    pairs = torch.full((max_steps * half * 2,), -7, dtype=torch.int32, device=device)
    counts = torch.zeros(max_steps, dtype=torch.int32, device=device)
    w = None
    if weights is not None:
        w = weights.to(device=device, dtype=torch.float64).contiguous()
    ns = ctypes.c_int(0)
    fn = lib.jacobi_sched_pairs_noalloc if noalloc else lib.jacobi_sched_pairs
    rc = fn(nb, ordering, ctypes.c_void_p(w.data_ptr()) if w is not None else None,
                                ctypes.c_void_p(pairs.data_ptr()), ctypes.c_void_p(counts.data_ptr()), max_steps,
                                ctypes.byref(ns), _stream(torch.device(device)))
    if rc != JAC_OK:
        raise JacobiError(rc, "jacobi_sched_pairs%s failed" % ("_noalloc" if noalloc else ""))
    tab = pairs.view(max_steps, half, 2).cpu()
    cnt = counts.cpu()
    return [tab[s, : int(cnt[s])].clone() for s in range(ns.value)]


def jacobi_profile_begin(kernels=("gram", "pivot", "update")):
    mask = 0
    for k in kernels:
        mask |= 1 << KERNEL[k]
    rc = load_library().jacobi_profile_begin(mask)
    if rc != 0:
        raise JacobiError(rc, "jacobi_profile_begin")


def jacobi_profile_read(kernel):
    """(total milliseconds, launches) of one kernel since jacobi_profile_begin."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    rc = load_library().jacobi_profile_read(KERNEL[kernel], ctypes.byref(ms), ctypes.byref(n))
    if rc != 0:
        raise JacobiError(rc, "jacobi_profile_read")
    return ms.value, n.value


def jacobi_profile_end():
    load_library().jacobi_profile_end()
