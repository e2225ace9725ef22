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


def _header_fields(header, struct_name):
    """(name, C type, array length) of the fields of `typedef struct { ... } struct_name;`."""
    import re
    end = header.index("} %s;" % struct_name)
    start = header.rindex("typedef struct {", 0, end)
    body = re.sub(r"/\*.*?\*/", "", header[start + len("typedef struct {"):end], flags=re.S)
    out = []
    for line in body.splitlines():
        m = re.match(r"\s*(int32_t|int64_t|double|void\*|cqp_kkt_report|cqp_csr|const \w+\*)\s+(.+);", line)
        if not m:
            continue
        for nm in m.group(2).split(","):
            nm = nm.strip()
            a = re.match(r"(\w+)\[(\d+)\]", nm)
            out.append((a.group(1), m.group(1), int(a.group(2))) if a else (nm, m.group(1), 1))
    return out


def test_ctypes_mirrors_follow_the_header():
    # the binding's option and result structures must match include/cqp.h field by field
    # (order, C type, array length); a mismatch would shift every later field across the ABI
    import ctypes as C
    import paper_2608_09159_gb300 as g
    header = open(os.path.join(ROOT, "include", "cqp.h")).read()
    ctype = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double, "void*": C.c_void_p}
    for struct_name, py in (("cqp_options", g.Options), ("cqp_result", g.Result), ("cqp_kkt_report", g.KKTReport),
                            ("cqp_csr", g.CSR), ("cqp_qop", g.QOp), ("cqp_cones", g.Cones), ("cqp_bounds", g.Bounds),
                            ("cqp_batch", g.Batch), ("cqp_instance_result", g.InstanceResult)):
        fields = _header_fields(header, struct_name)
        assert [f[0] for f in fields] == [f for f, _ in py._fields_], struct_name
        for (name, ty, n), (_, pty) in zip(fields, py._fields_):
            if ty == "cqp_kkt_report":
                assert pty is g.KKTReport, name
            elif ty == "cqp_csr":
                assert pty is g.CSR, name
            elif ty.startswith("const "):
                assert pty is C.c_void_p, (struct_name, name)   # device or host pointer
            elif n > 1:
                assert pty._type_ is ctype[ty] and pty._length_ == n, name
            else:
                assert pty is ctype[ty], (struct_name, name)
