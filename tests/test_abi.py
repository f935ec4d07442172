"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/kclique.h (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(kc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_2002_10047_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("kc_orient", "kc_count", "kc_count_per_vertex", "kc_count_per_arc", "kc_count_roots", "kc_dag_free",
                 "kc_dag_n", "kc_dag_m", "kc_strerror", "kc_dag_export", "kc_dag_get_stats"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (kc_\w+)", out))
    assert declared_functions() <= exported


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.kc_strerror.restype = ctypes.c_char_p
    lib.kc_kernel_launches.restype = ctypes.c_uint64
    before = lib.kc_kernel_launches()
    for code in range(7):
        assert lib.kc_strerror(code)
    assert lib.kc_kernel_launches() == before  # no device work behind these calls


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2002_10047_gb300 import build, kclique
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(kclique, "_lib", None)
    with pytest.raises(RuntimeError):
        kclique._load()


def test_binding_checks_arguments_before_any_device_call(lib_path):
    """The binding rejects host tensors and mismatched shapes itself (no
    device is touched), for every entry point that takes tensors."""
    torch = pytest.importorskip("torch")
    from paper_2002_10047_gb300 import kclique as kc
    rp = torch.zeros(5, dtype=torch.int64)
    col = torch.zeros(0, dtype=torch.int32)
    with pytest.raises(ValueError):
        kc.orient(rp, col, 4)
    with pytest.raises(ValueError):
        kc.Batch(torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.uint8))
    with pytest.raises(ValueError):
        kc.count_colorful(rp, col, 3, 2, 1)
    with pytest.raises(ValueError):
        kc.peel(rp, col, None, 3)
    with pytest.raises(ValueError):
        kc.count_roots(None, 4, torch.zeros(3, dtype=torch.int32))


def test_binding_constants_match_the_header():
    """The Python binding's constants are the header's (status codes, k range,
    orientation methods and flags, warp-root orders)."""
    from paper_2002_10047_gb300 import kclique as kc
    text = open(os.path.join(ROOT, "include", "kclique.h")).read()
    defines = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define (KC_\w+) (0x[0-9a-fA-F]+|\d+)\b", text)}
    for name in ("KC_KMAX", "KC_ORIENT_DEGREE", "KC_ORIENT_GP", "KC_ORIENT_BE", "KC_VALIDATE_SYMMETRY",
                 "KC_CORE_BITS", "KC_NO_CORE_BITS", "KC_LIGHT_BY_DEGREE", "KC_LIGHT_BY_ID"):
        assert getattr(kc, name) == defines[name], name
    enum = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"(KC_E?\w+) = (\d+)", text))
    for name in ("KC_OK", "KC_EINVAL", "KC_ERANGE", "KC_ENOMEM", "KC_ETIMEDOUT", "KC_ECUDA", "KC_ECAPACITY"):
        assert getattr(kc, name) == enum[name], name
    assert kc._METHODS == {"degree": defines["KC_ORIENT_DEGREE"], "gp": defines["KC_ORIENT_GP"],
                           "be": defines["KC_ORIENT_BE"]}


def test_orient_rejects_bad_flags_without_gpu(lib_path):
    """kc_orient checks its method flags before any device call: unknown bits
    and KC_CORE_BITS together with KC_NO_CORE_BITS give KC_EINVAL."""
    lib = ctypes.CDLL(lib_path)
    lib.kc_kernel_launches.restype = ctypes.c_uint64

    class Csr(ctypes.Structure):
        _fields_ = [("n", ctypes.c_uint32), ("nnz", ctypes.c_uint64), ("rp", ctypes.c_void_p),
                    ("col", ctypes.c_void_p)]

    g = Csr(0, 0, None, None)
    h = ctypes.c_void_p()
    before = lib.kc_kernel_launches()
    assert lib.kc_orient(ctypes.byref(g), 0x200 | 0x400, ctypes.byref(h), None) == 1
    assert lib.kc_orient(ctypes.byref(g), 0x800, ctypes.byref(h), None) == 1
    assert lib.kc_orient(ctypes.byref(g), 3, ctypes.byref(h), None) == 1
    assert h.value is None
    assert lib.kc_kernel_launches() == before

