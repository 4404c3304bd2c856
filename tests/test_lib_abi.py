"""The C-ABI library builds, loads and exports every entry point include/lcq.h declares;
host-only queries agree with the oracle (no GPU compute in this file)."""
import os
import re

import numpy as np
import pytest

from oracle import rules

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lcq():
    import __graft_entry__ as g
    g.build()
    from paper_2006_02545_gb300 import lcq as mod
    return mod


def declared_functions():
    with open(os.path.join(ROOT, "include", "lcq.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lcq_[A-Za-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lcq):
    names = declared_functions()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(lcq._lib, nm), nm
    assert set(names) == set(lcq.SYMBOLS)


@pytest.mark.parametrize("d", range(1, 11))
def test_ref_nodes_match_oracle(lcq, d):
    u, v, w = lcq.ref_nodes(d)
    ou, ov = rules.interp_nodes(d)
    assert np.abs(u - ou).max() < 1e-14 and np.abs(v - ov).max() < 1e-14
    assert np.abs(w - rules.interp_weights(d)).max() < 1e-14


def test_params_and_status_strings(lcq):
    p = lcq.params(1e-9)
    assert p.eps == 1e-9 and p.eta == -1.0 and p.eta1 == 1.25 and p.max_depth == 24
    assert p.m_max == 24 and p.self_order == 0 and p.leaf_order == 0
    assert lcq._lib.lcq_status_string(0) == b"ok"
    assert b"max_depth" in lcq._lib.lcq_status_string(4)
    assert lcq._lib.lcq_status_string(99) == b"unknown status"


def test_bad_degree_rejected_on_host(lcq):
    with pytest.raises(lcq.LCQError):
        lcq.ref_nodes(11)


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """Without liblcq.so the binding raises on import: there is no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    shutil.copy(os.path.join(ROOT, "paper_2006_02545_gb300", "lcq.py"), pkg / "lcq.py")
    r = subprocess.run([sys.executable, "-c", "import pkg.lcq"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "liblcq.so not built" in r.stderr


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """Each entry point's comment in include/lcq.h names the paper's passage (section,
    equation or table) or states that the paper has no counterpart."""
    with open(os.path.join(ROOT, "include", "lcq.h")) as f:
        text = f.read()
    decls = list(re.finditer(r"^(?:const char\*|void|lcq_status)\s+(lcq_[A-Za-z0-9_]+)\s*\(",
                             text, re.M))
    assert len(decls) >= 30
    for m in decls:
        before = text[:m.start()]
        end = before.rfind("*/")
        comment = before[before.rfind("/*", 0, end):end]
        assert re.search(r"Sec\.|Eq\.|Table|counterpart|extension|library facility", comment), \
            m.group(1)
