"""The C ABI library builds, loads and exports every function declared in include/*.h (no GPU).

Only host-side functions (defaults, status strings, version, profile bookkeeping) are called.
"""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(jacobi_[A-Za-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("jacobi_hsvd", "jacobi_eig_pd", "jacobi_sched_pairs", "jacobi_default_opts"):
        assert required in names


def test_library_exports_all_declared(lib_built):
    from paper_1008_0201_gb300 import binding

    lib = binding.load_library()
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTS) <= declared_functions()


def test_host_only_calls(lib_built):
    from paper_1008_0201_gb300 import binding

    o = binding.default_opts()
    assert (o.block_w, o.ordering, o.factor, o.max_sweeps, o.want_v) == (32, 2, 2, 50, 1)
    assert binding.status_string(0) == "ok"
    assert "invalid" in binding.status_string(-3)
    assert binding.load_library().jacobi_version() >= 100
    binding.jacobi_profile_begin(("pivot",))
    assert binding.jacobi_profile_read("pivot") == (0.0, 0)
    binding.jacobi_profile_end()
    # the extension is not a CPU fallback: a CPU tensor is rejected before any call
    import pytest
    import torch

    with pytest.raises(ValueError):
        binding.jacobi_eig_pd(torch.zeros(4, 4, dtype=torch.float64))


def test_library_is_sm103a_only(lib_built):
    from paper_1008_0201_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_opts_layout_matches_header(lib_built):
    """jacobi_default_opts writes exactly the bytes of the ctypes mirror (no more), and its last
    field lands where the mirror expects it: the binding's JacOpts has the header's layout."""
    from paper_1008_0201_gb300 import binding

    lib = binding.load_library()
    n = ctypes.sizeof(binding.JacOpts)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
    lib.jacobi_default_opts(ctypes.cast(buf, ctypes.POINTER(binding.JacOpts)))
    assert bytes(buf[n:]) == b"\xa5" * 64
    o = binding.JacOpts.from_buffer_copy(bytes(buf[:n]))
    assert o.f64_products == binding.F64_PRODUCTS["split16"]
    assert o.precision == binding.PRECISION["fp64"] and o.tol == 0.0
    assert lib.jacobi_version() == binding.ABI_VERSION


def test_info_layout_matches_header(lib_built):
    """An argument error returns before any CUDA call, after clearing *info: the cleared bytes are
    exactly the ctypes mirror's, and the status lands in its field."""
    from paper_1008_0201_gb300 import binding

    lib = binding.load_library()
    n = ctypes.sizeof(binding.JacInfo)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
    info = ctypes.cast(buf, ctypes.POINTER(binding.JacInfo))
    rc = lib.jacobi_hsvd(0, 1, 0, None, 1, None, None, None, None, 0, None, 0, info, None)
    assert rc == -1
    assert bytes(buf[n:]) == b"\xa5" * 64
    got = binding.JacInfo.from_buffer_copy(bytes(buf[:n]))
    assert got.status == -1 and got.sweeps == 0 and got.launches == 0
    assert all(v == 0.0 for v in got.sweep_ms) and all(v == 0.0 for v in got.sweep_max_scaled)
