"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/cqp.h declares (no GPU needed: nothing is called that touches a device)."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names.update(re.findall(r"\b(cqp_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def cqplib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2608_09159_gb300 as g
    g.build()
    return g.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cqp_setup", "cqp_solve", "cqp_kkt", "cqp_free", "cqp_spmv", "cqp_project"):
        assert required in names


def test_library_exports_every_declared_symbol(cqplib):
    missing = [n for n in _declared() if not hasattr(cqplib, n)]
    assert not missing, missing


def test_defaults_match_paper_table(cqplib):
    import paper_2608_09159_gb300 as g
    o = g.cqp_default_options()
    # Table "practical-defaults"
    assert o.ruiz_iters == 10 and o.pc_alpha == 1.0 and o.bound_obj == 1
    assert (o.eps0_in, o.gamma_in, o.eps_min_in) == (1e-3, 5e-4, 1e-9)
    assert o.jacobi == 1 and o.rho == 1.0
    assert (o.beta_s, o.beta_n, o.beta_a) == (0.2, 0.8, 0.36)
    assert (o.beta_I, o.K_P, o.K_I, o.K_D) == (0.3, 0.99, 0.01, 0.0)
    assert o.step_factor == 0.998


def test_status_strings(cqplib):
    import paper_2608_09159_gb300 as g
    assert g.cqp_status_string(0) == "converged"
    assert g.cqp_status_string(-1) == "invalid input"


def test_oracle_not_imported_by_product():
    # the product package never references the oracle
    pkg = os.path.join(ROOT, "paper_2608_09159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".inc")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "oracle.h" not in txt, f
