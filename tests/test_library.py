"""The C-ABI boundary without a GPU: the library builds for sm_103a, loads with
every symbol bound at load time, exports every function include/*.h declares,
and the Python binding declares the same set.  The oracle library builds and
loads too.  No compute call is made."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(dwf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("dwf_create", "dwf_apply", "dwf_cg", "dwf_mspcg", "dwf_batch_mspcg",
              "dwf_set_reduced_ls", "dwf_destroy", "dwf_last_error"):
        assert n in names
    assert len(names) >= 30


def test_library_loads_and_exports_every_declared_function():
    from paper_2104_05615_gb300 import build
    lib_path = build.build()
    # RTLD_NOW: an unresolved reference fails here, not at its first call
    lib = ctypes.CDLL(lib_path, mode=ctypes.RTLD_LOCAL | os.RTLD_NOW)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_function():
    from paper_2104_05615_gb300 import binding
    src = open(binding.__file__).read()
    missing = [n for n in sorted(declared_functions()) if f'"{n}"' not in src]
    assert not missing, missing


def test_oracle_library_builds_and_loads():
    import oracle
    path = oracle.build()
    ctypes.CDLL(path, mode=ctypes.RTLD_LOCAL | os.RTLD_NOW)
