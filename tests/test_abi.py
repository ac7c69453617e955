"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every entry point that include/snn.h declares; the binding
declares exactly that set.  No compute calls (there is no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snn.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(snn_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2109_12855_gb300 import build
    return build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (snn_[a-z_0-9]+)\b", out))
    declared = set(_declared())
    assert declared, "no declarations parsed"
    assert declared <= exported, sorted(declared - exported)


def test_checked_variant_exports_the_same_symbols(libpath):
    """libsnn_check.so (SNN_CHECK bounds checks) is built beside libsnn.so
    with the same ABI; each reports which variant it is."""
    import ctypes
    from paper_2109_12855_gb300 import native
    assert os.path.exists(native.LIB_CHECKED)
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_CHECKED],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (snn_[a-z_0-9]+)\b", out))
    assert set(_declared()) <= exported
    prod = ctypes.CDLL(native.LIB)
    chk = ctypes.CDLL(native.LIB_CHECKED)
    assert prod.snn_checked() == 0 and chk.snn_checked() == 1
    f = prod.snn_debug_poke_record
    f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                  ctypes.c_uint32]
    assert f(None, 0, 0, 0) != 0  # refused: null net


def test_binding_covers_the_header(libpath):
    from paper_2109_12855_gb300 import snn
    assert sorted(snn.EXPORTS) == _declared()
    L = snn.lib()
    for name in snn.EXPORTS:
        assert getattr(L, name) is not None


def test_library_loads_and_reports_version_without_gpu(libpath):
    from paper_2109_12855_gb300 import snn
    assert snn.snn_abi_version() == 1
    p = snn.snn_default_params()
    assert (p.n_exc, p.n_inh, p.n_slots) == (1000, 250, 32)


def test_struct_layouts_match_header(libpath):
    """sizeof of the C structs as compiled (g++) equals the ctypes mirrors."""
    import ctypes
    from paper_2109_12855_gb300 import snn
    src = ('#include "snn.h"\n#include <stdio.h>\nint main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu",'
           'sizeof(snn_params),sizeof(snn_conn_params),sizeof(snn_stats),'
           'sizeof(snn_request),sizeof(snn_result),sizeof(snn_server_stats),'
           'sizeof(snn_stdp_params),sizeof(snn_bounds));}')
    exe = os.path.join(ROOT, "paper_2109_12855_gb300", "_build", "sizes")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    r = subprocess.run(["gcc", "-x", "c", "-I", os.path.join(ROOT, "include"),
                        "-o", exe, "-"], input=src, text=True,
                       capture_output=True)
    assert r.returncode == 0, r.stderr
    sizes = [int(x) for x in subprocess.run([exe], capture_output=True,
                                            text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(snn.snn_params),
                     ctypes.sizeof(snn.snn_conn_params),
                     ctypes.sizeof(snn.snn_stats),
                     ctypes.sizeof(snn.snn_request),
                     ctypes.sizeof(snn.snn_result),
                     ctypes.sizeof(snn.snn_server_stats),
                     ctypes.sizeof(snn.snn_stdp_params),
                     ctypes.sizeof(snn.snn_bounds)]


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2109_12855_gb300.snn as snn
    monkeypatch.setattr(snn, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(snn, "_lib", None)
    with pytest.raises(ImportError):
        snn.lib()


def test_binding_constants_match_header(libpath):
    """The binding's copies of the header's constants (the allocation-free
    scratch capacity, the status codes, the probe patterns) equal the
    compiled values."""
    from paper_2109_12855_gb300 import snn
    src = ('#include "snn.h"\n#include <stdio.h>\nint main(){printf("%u %d %d %d %u %d %d",'
           '(unsigned)SNN_NOALLOC_MAX_SPIKES,SNN_E_ARG,SNN_E_STATE,SNN_E_TIMEOUT,'
           '(unsigned)SNN_ERRF_CHECK,SNN_PROBE_SCATTER,SNN_PROBE_SWEEP);}')
    exe = os.path.join(ROOT, "paper_2109_12855_gb300", "_build", "consts")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    r = subprocess.run(["gcc", "-x", "c", "-I", os.path.join(ROOT, "include"),
                        "-o", exe, "-"], input=src, text=True,
                       capture_output=True)
    assert r.returncode == 0, r.stderr
    vals = [int(x) for x in subprocess.run([exe], capture_output=True,
                                           text=True).stdout.split()]
    assert vals == [snn.SNN_NOALLOC_MAX_SPIKES, snn.SNN_E_ARG, snn.SNN_E_STATE,
                    snn.SNN_E_TIMEOUT, snn.SNN_ERRF_CHECK, snn.SNN_PROBE_SCATTER,
                    snn.SNN_PROBE_SWEEP]
