"""The autotuner (dg_autotune): its choices are valid, it leaves u^n alone, and the results
of the method do not depend on the launch configuration it picks."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_choices_and_state():
    n = 192
    w = W.euler_2d_quadrant(n, 2, seed=5)
    g = dgl.Mesh(2, 1, 2, [n], [n], w.box, bc=1)
    g.project_ic(w.ic, w.params[0])
    u0 = g.get_modes()
    ws = g.max_wavespeed()[0]
    dt = 0.1 / (ws[0] * n + ws[1] * n)
    g.rk_stage(1, dt)
    before = g.get_modes()
    g.set_modes(u0)
    ty, mult, pers = g.autotune(dt)
    assert ty in (0, 4, 8) and mult in (2, 4, 8, 16) and pers in (0, 1)
    assert np.array_equal(g.get_modes(), u0)  # u^n untouched
    g.rk_stage(1, dt)
    # the split and fused stage forms sum in different orders: equal up to rounding
    after = g.get_modes()
    scale = np.abs(before).max(axis=(0, 2))
    assert (np.abs(after - before).max(axis=(0, 2)) / scale).max() <= 1e-14


@pytest.mark.parametrize("form", ["4 2 1", "8 8 0", "0 8 0"])
def test_stage_forms_match_oracle_in_fresh_process(tmp_path, form):
    """Force a stage form through the tuning file -- fused with 4-row tiles and the
    persistent tile queue, fused with 8-row tiles one block per tile, or split into the face
    and cell passes -- and check a stage, the flags and the limiter against the oracle on a
    ragged 2D Euler P2 mesh."""
    f = tmp_path / "tune.txt"
    nx, ny = 70, 45
    cls = int(np.floor(np.log2(nx * ny)))
    f.write_text("2 1 2 %d %s\n" % (cls, form))
    code = textwrap.dedent("""
        import sys, numpy as np
        sys.path.insert(0, %r)
        import oracle, paper_1904_11147_gb300 as dgl
        from paper_1904_11147_gb300 import workloads as W
        nx, ny = %d, %d
        o = oracle.Mesh(2, 1, 2, nx, ny, box=(0, 1.3, 0, 0.9), bc=1)
        g = dgl.Mesh(2, 1, 2, [nx], [ny], [(0, 1.3, 0, 0.9)], bc=1)
        u = W.random_modes(2, 1, 2, nx * ny, np.random.default_rng(3), smooth=0.02)
        g.set_modes(u)
        g.rk_stage(1, 1e-4)
        s1 = o.rk_stage(1, 1e-4, u, u)
        got = g.get_modes()
        assert np.abs(got - s1).max() <= 1e-13 * np.abs(s1).max()
        fl, nf, nn = g.flag_cells(dgl.IND_TVB, 0.01, want=True)
        fo, nfo, nno = o.flag_tvb(s1, 0.01)
        assert nf == nfo and np.array_equal(fl, fo)
        g.cswenolimit()
        ref = o.limit(s1, fo)
        assert np.abs(g.get_modes() - ref).max() <= 1e-11 * np.abs(ref).max()
        print("ok")
    """) % (ROOT, nx, ny)
    env = dict(os.environ, DG_AUTOTUNE_FILE=str(f))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
