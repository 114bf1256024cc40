"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/pg.h declares. No compute calls are
made here (there may be no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:pg_status|void|const char \*)\s*\*?\s*(pg_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1705_02313_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ["pg_ctx_create", "pg_ctx_destroy", "pg_set_stream", "pg_last_error", "pg_load_csr",
                     "pg_game_free", "pg_solve", "pg_best_response", "pg_valuate"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    from paper_1705_02313_gb300 import pg
    missing = [n for n in declared_functions() if not hasattr(pg, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_1705_02313_gb300 import pg
    monkeypatch.setattr(pg, "_lib", None)
    monkeypatch.setattr(pg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(pg.PgUnavailable):
        pg.lib()
