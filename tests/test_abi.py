"""Host-only checks of the C-ABI library (no GPU needed): it builds, loads, exports every
function that include/dg.h declares, validates arguments before touching the device, and
its own table derivation agrees with the oracle's independent one."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1904_11147_gb300 as dgl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    l = dgl.lib()
    names = _declared()
    assert "dg_mesh_create" in names and "dg_cswenolimit" in names
    for n in names:
        assert hasattr(l, n), n


@pytest.mark.parametrize("N", [1, 2, 3])
def test_library_tables_match_oracle(N):
    """The library derives its tables by a different route (closed-form nodes, Bonnet
    recurrence, primitive-function interpolation, back substitution, quadrature); the
    oracle by monomial moments.  Both must agree to rounding."""
    a = dgl.limiter_tables(N)
    b = oracle.weno_tables(N)
    np.testing.assert_allclose(a["pt"], b["pt"], atol=1e-15)
    np.testing.assert_allclose(a["wt"], b["wt"], atol=1e-15)
    np.testing.assert_allclose(a["gam"], b["gam"], atol=1e-13)
    np.testing.assert_allclose(a["SA"], b["SA"], atol=1e-15)
    for i in range(N + 1):
        np.testing.assert_allclose(a["C"][i], b["C"][i][:, i:i + N + 1], atol=1e-13)
        np.testing.assert_allclose(a["B"][i], b["B"][i][i:i + N + 1, i:i + N + 1], atol=1e-11)


def test_argument_validation_without_device():
    l = dgl.lib()
    h = ctypes.c_void_p()
    nx = (ctypes.c_int * 1)(8)
    box = (ctypes.c_double * 4)(0, 1, 0, 1)
    for dim, pde, N, bc, gam in [(3, 0, 2, 0, 1.4), (1, 5, 2, 0, 1.4), (1, 0, 4, 0, 1.4), (1, 0, 0, 0, 1.4),
                                 (1, 0, 2, 7, 1.4), (1, 1, 2, 0, 0.5)]:
        s = l.dg_mesh_create(dim, pde, N, 1, nx, nx, box, bc, gam, None, ctypes.byref(h))
        assert s == dgl.DG_EINVAL
        assert l.dg_last_error()
    assert l.dg_mesh_create(1, 0, 2, 0, nx, nx, box, 0, 1.4, None, ctypes.byref(h)) == dgl.DG_EINVAL
    assert l.dg_mesh_create(1, 0, 2, 1, nx, nx, box, 0, 1.4, None, None) == dgl.DG_EINVAL
    assert l.dg_rk_stage(None, 1, 0.1) == dgl.DG_EINVAL
    assert l.dg_cswenolimit(None) == dgl.DG_EINVAL
    assert l.dg_mesh_destroy(None) == dgl.DG_OK
