"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "gift.h")).read()
    return sorted(set(re.findall(r"^GIFT_API\s+[\w\s\*]*?\b(gift_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_01879_gb300 import build
    build.build()
    import paper_1604_01879_gb300 as gift
    return gift.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for must in ("gift_build_index", "gift_query", "gift_rerank", "gift_match_forward", "gift_match_backward",
                 "gift_destroy_index", "gift_last_error"):
        assert must in syms


def test_every_declared_symbol_is_exported(lib):
    import paper_1604_01879_gb300 as gift
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in gift.SYMBOLS, f"binding lacks {name}"


def test_error_path_without_gpu(lib):
    # argument checks run before any CUDA call
    assert lib.gift_query(None, None, None, 0, 0, 0, None, None, None) == 1
    assert b"NULL" in lib.gift_last_error()
    assert lib.gift_version() >= 100


def test_binding_refuses_missing_library(tmp_path):
    import paper_1604_01879_gb300 as gift
    saved = gift._lib
    gift._lib = None
    try:
        with pytest.raises(RuntimeError):
            gift.load(str(tmp_path / "missing.so"))
    finally:
        gift._lib = saved
