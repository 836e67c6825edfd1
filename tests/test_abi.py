"""Host-side checks of the C ABI: the library builds, loads and exports every
function include/msa.h declares; the size helpers are plain arithmetic."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(msa_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2601_15458_gb300 import build, _lib
    build.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert "msa_lev_batch" in declared and "msa_pack" in declared
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2601_15458_gb300 import _lib
    assert _declared() == set(_lib.SIGNATURES)


def test_size_helpers(lib):
    assert lib.msa_code_bytes(0) == 32
    assert lib.msa_code_bytes(33) == 96
    assert lib.msa_plane_words(64, 0) == (2 + 1) * 2
    assert lib.msa_plane_words(65, 1) == (3 + 1) * 5
    assert lib.msa_lev_workspace_bytes(1000, 10) > 1000 * 8
    for n, ns in [(0, 1), (1, 1), (1000, 10), (123457, 50000)]:
        # the pair list (2 int32 per target, 256-byte rounded) plus the batch's own workspace
        assert lib.msa_lev_one_to_many_workspace_bytes(n, ns) == \
            (8 * n + 255) // 256 * 256 + lib.msa_lev_workspace_bytes(n, ns)
    assert b"sm_103a" in lib.msa_version()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2601_15458_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "SO_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.lib()
