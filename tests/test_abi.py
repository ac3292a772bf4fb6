"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/domagg.h declares (no GPU needed: no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "domagg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(domagg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2305_16751_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("domagg_create", "domagg_destroy", "domagg_forward", "domagg_backward", "domagg_batch"):
        assert name in fns


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    from paper_2305_16751_gb300 import domagg
    assert sorted(domagg.SIGNATURES) == declared_functions()
    L = domagg.lib()
    for name in declared_functions():
        assert hasattr(L, name)
    assert "sm_103a" in domagg.domagg_version()


def test_library_is_built_for_sm_103a(libpath):
    # the fatbinary lists the architectures it carries; read only the listing
    r = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in r.stdout


def test_no_oracle_in_the_product_path():
    pkg = os.path.join(ROOT, "paper_2305_16751_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "domagg_oracle" not in text, f


def _header_enum(name):
    """{enumerator: value} of the typedef'd enum `name` in the header."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef\s+enum\s*\{([^}]*)\}\s*" + name + r"\s*;", src, flags=re.S)
    assert m, name
    out, nxt = {}, 0
    for item in [x.strip() for x in m.group(1).split(",") if x.strip()]:
        k, _, v = item.partition("=")
        nxt = int(v.strip()) if v.strip() else nxt
        out[k.strip()] = nxt
        nxt += 1
    return out


def test_binding_enums_match_the_header():
    """The ctypes binding's op, dtype, variant and status codes are the
    header's enumerators (the binding passes plain ints across the ABI)."""
    from paper_2305_16751_gb300 import domagg
    ops = _header_enum("domagg_op")
    assert {k: ops["DOMAGG_" + k.upper()] for k in domagg.OPS} == domagg.OPS
    dts = _header_enum("domagg_dtype")
    assert {k: dts["DOMAGG_" + k.upper()] for k in domagg.DTYPES} == domagg.DTYPES
    var = _header_enum("domagg_variant")
    assert {k: var["DOMAGG_" + k.upper()] for k in domagg.VARIANTS} == domagg.VARIANTS
    assert len(var) == len(domagg.VARIANTS)
    st = _header_enum("domagg_status")
    assert {v: "DOMAGG_" + ("ERR_" if v else "") + n for v, n in domagg.STATUS.items()} == \
        {v: k for k, v in st.items()}
