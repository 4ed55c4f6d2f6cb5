"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/cem.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="cem.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(cem_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cem_mesh_create", "cem_set_material", "cem_set_bc", "cem_step",
                     "cem_get_fields", "cem_get_crack_tips", "cem_mesh_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2509_01827_gb300 import build
    from paper_2509_01827_gb300 import cem
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared entry points
    assert sorted(cem.SIGNATURES) == declared_functions()


def test_surrogate_abi_exported_and_bound():
    from paper_2509_01827_gb300 import build
    from paper_2509_01827_gb300 import surrogate
    lib = ctypes.CDLL(build.build())
    names = declared_functions("cem_surrogate.h")
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(surrogate.SG_SIGNATURES) == names


def test_surrogate_argument_checks_without_gpu():
    """Shape checks come before any launch: bad channel counts are errors."""
    from paper_2509_01827_gb300 import surrogate
    L = surrogate.sg()
    assert L.cem_sg_conv3x3(1, 1, 4, 4, 3, 3, 1, None, 8, 0, None, 0, 1, 8, 0, None) == -1  # Cin % 8
    assert L.cem_sg_wgrad_workspace(1, 4, 4, 8, 8) > 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2509_01827_gb300 import cem
    monkeypatch.setattr(cem, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(cem, "_LIB", None)
    with pytest.raises(RuntimeError):
        cem.lib()


def test_create_error_path_without_gpu_is_an_error_not_a_crash():
    """Argument validation happens before any device call."""
    from paper_2509_01827_gb300 import cem
    d = cem.cem_mesh_desc()
    d.nx, d.ny, d.hx, d.hy = 0, 4, 1e-3, 1e-3
    with pytest.raises(cem.CemError) as ei:
        cem.cem_mesh_create(d)
    assert ei.value.code == cem.CEM_ERR_ARG
