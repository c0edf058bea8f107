"""CPU checks of the C-ABI boundary: the library builds, loads and exports every entry point
that include/rpca.h declares, and argument checking that needs no GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1702_02241_gb300 import build, rpca
    build.build()
    return rpca.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rpca.h")).read()
    return sorted(set(re.findall(r"RPCA_API\s+[\w\s\*]+?\b(rpca_\w+)\s*\(", txt)))


def test_header_declares_the_four_named_entry_points():
    syms = declared_symbols()
    for s in ["rpca_create", "rpca_fg", "rpca_solve", "rpca_certificate", "rpca_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    for s in declared_symbols():
        assert hasattr(lib, s), s
        assert isinstance(getattr(lib, s), ctypes._CFuncPtr)


def test_binding_names_match_header(lib):
    from paper_1702_02241_gb300 import rpca
    assert sorted(rpca.EXPORTED) == declared_symbols()
    for s in declared_symbols():
        assert callable(getattr(rpca, s))


def test_default_options_and_version(lib):
    from paper_1702_02241_gb300 import rpca
    o = rpca.rpca_default_options()
    assert o.lbfgs_mem == 10 and o.cert_tol == 1e-4 and o.max_iter > 0
    assert "sm_103a" in rpca.rpca_version()


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    from paper_1702_02241_gb300 import rpca
    cases = [
        dict(m=0, n=5, X=16, ldx=4, k=1, lam_L=1.0, lam_S=1.0),
        dict(m=8, n=5, X=0, ldx=8, k=1, lam_L=1.0, lam_S=1.0),
        dict(m=8, n=5, X=16, ldx=4, k=1, lam_L=1.0, lam_S=1.0),
        dict(m=8, n=5, X=16, ldx=8, k=6, lam_L=1.0, lam_S=1.0),
        dict(m=8, n=5, X=16, ldx=8, k=1, lam_L=0.0, lam_S=1.0),
        dict(m=8, n=5, X=16, ldx=8, k=1, lam_L=1.0, lam_S=-1.0),
        dict(m=8, n=5, X=12, ldx=8, k=1, lam_L=1.0, lam_S=1.0),     # misaligned X
        dict(m=7, n=5, X=16, ldx=7, k=1, lam_L=1.0, lam_S=1.0),     # ldx*4 not 16-byte multiple
    ]
    for cs in cases:
        with pytest.raises(rpca.RpcaError) as ei:
            rpca.rpca_create(cs["m"], cs["n"], cs["X"], cs["ldx"], None, 0, cs["k"], cs["lam_L"], cs["lam_S"])
        assert ei.value.status == rpca.RPCA_EINVAL, cs
        assert rpca.rpca_last_error(None)
    with pytest.raises(rpca.RpcaError) as ei:  # factor ranks above 256 are not built
        rpca.rpca_create(512, 512, 16, 512, None, 0, 257, 1.0, 1.0)
    assert ei.value.status == rpca.RPCA_EUNSUPPORTED


def test_entry_points_reject_null_context(lib):
    from paper_1702_02241_gb300 import rpca
    assert lib.rpca_fg(None, None, None, None, None, None) == rpca.RPCA_EINVAL
    assert lib.rpca_solve(None, None, None, None) == rpca.RPCA_EINVAL
    assert lib.rpca_certificate(None, None, None, None) == rpca.RPCA_EINVAL
    lib.rpca_destroy(None)


def test_inject_fault_arguments_without_a_gpu(lib):
    from paper_1702_02241_gb300 import rpca
    assert lib.rpca_inject_fault(None, rpca.RPCA_FAULT_FG_STARVE, 1) == rpca.RPCA_EINVAL  # needs a context
    assert lib.rpca_inject_fault(None, 99, 1) == rpca.RPCA_EINVAL
    assert lib.rpca_inject_fault(None, rpca.RPCA_FAULT_ALLOC, -1) == rpca.RPCA_EINVAL
    assert lib.rpca_inject_fault(None, rpca.RPCA_FAULT_ALLOC, 0) == rpca.RPCA_OK
