"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, and
exports every entry point that include/gedwalk.h declares; the product path never imports
the oracle and refuses to run without its CUDA library."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gedwalk.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"GEDWALK_API\s+[\w\s\*]+?\b(gedwalk_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_13874_gb300 import build, gedwalk

    build.build()
    return gedwalk.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gedwalk_graph_upload", "gedwalk_score", "gedwalk_score_batch", "gedwalk_maximize",
                 "gedwalk_serve_create", "gedwalk_serve_submit", "gedwalk_serve_poll", "gedwalk_serve_destroy"):
        assert must in names


def _declaration_comments():
    """(name, the comment blocks between the previous declaration and this one) per entry point."""
    text = open(HEADER).read()
    out, prev = [], 0
    for m in re.finditer(r"GEDWALK_API\s+[\w\s\*]+?\b(gedwalk_\w+)\s*\(", text):
        blocks = " ".join(re.findall(r"/\*.*?\*/", text[prev:m.start()], re.S))
        out.append((m.group(1), re.sub(r"\s*\n\s*\*?\s*", " ", blocks)))  # one line, no margin stars
        prev = text.index(";", m.end())
    return out


def test_every_entry_point_cites_its_passage_or_says_it_has_none():
    cite = re.compile(r"Section \d|Eq\. |Algorithm \d|Lemma |Def\. |Prop\. |Appendix |problem \(|"
                      r"no counterpart")
    decls = _declaration_comments()
    assert len(decls) == len(_declared())
    for name, comment in decls:
        assert comment.strip(), name
        assert cite.search(comment), name


def test_library_exports_every_declared_symbol(lib):
    from paper_1910_13874_gb300 import gedwalk

    names = _declared()
    assert sorted(gedwalk.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", gedwalk.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r"\bT (gedwalk_\w+)", out)))
    assert exported == names  # nothing else leaks from the C++ internals


def test_params_default_and_last_error(lib):
    from paper_1910_13874_gb300 import gedwalk

    p = gedwalk.make_params()
    assert p.epsilon == 1e-4 and p.L == 0 and p.precision == gedwalk.FP32 and p.alpha == 0.0
    assert lib.gedwalk_last_error() is not None
    # argument errors are reported before any device work
    import ctypes

    st = lib.gedwalk_graph_upload(None, None, 0, 0, 0, ctypes.byref(ctypes.c_void_p()))
    assert st == gedwalk.ERR_INVALID
    assert b"n must be" in lib.gedwalk_last_error()


def test_product_path_never_imports_the_oracle():
    code = ("import sys; import paper_1910_13874_gb300 as p; import paper_1910_13874_gb300.build; "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), 'oracle imported'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_1910_13874_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "oracle_impl" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    code = ("import paper_1910_13874_gb300.gedwalk as g\n"
            f"try:\n    g.load({str(tmp_path / 'nope.so')!r})\nexcept RuntimeError as e:\n"
            "    assert 'no CPU fallback' in str(e); print('raised')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "raised" in out.stdout, out.stderr
