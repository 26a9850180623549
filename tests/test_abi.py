"""The C-ABI library builds, loads and exports every symbol declared in include/*.h."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*(rbf_[a-z_0-9]+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rbf_create", "rbf_operator_init", "rbf_assemble", "rbf_gkb", "rbf_hkt",
                     "rbf_ine_tsvd", "rbf_tikhonov", "rbf_evaluate", "rbf_projected_svd"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2511_09798_gb300 import build
    lib_path = build.build()
    import ctypes
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2511_09798_gb300 import rbfkr
    assert set(declared_functions()) <= set(rbfkr.EXPORTS)


def test_package_path_has_no_oracle_import():
    # the product path must not reach the oracle
    for f in glob.glob(os.path.join(ROOT, "paper_2511_09798_gb300", "**", "*.py"), recursive=True):
        src = open(f).read()
        assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, flags=re.M), f


def test_oracle_does_not_import_the_package():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        mods = re.findall(r"^\s*(?:from|import)\s+([\w.]+)", open(f).read(), flags=re.M)
        assert not any(m.startswith("paper_2511_09798_gb300") for m in mods), f


def test_checked_library_builds_and_exports_the_same_symbols():
    from paper_2511_09798_gb300 import build
    lib_path = build.build(checked=True)
    import ctypes
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.rbf_checked_build() == 1
