"""Stage-by-stage shadow comparison of the CUDA path with the oracle (GPU tests only).

Every step of the GPU trajectory is replayed through the per-call entry points, and each
sub-step is recomputed by the oracle from the GPU's own input to it, so that every
comparison starts from identical doubles:
  - the stage output (dg_rk_stage) within 1e-13 (relative, per variable),
  - the troubled-cell flags (dg_flag_cells) identical: the indicator's decision is taken
    in the same FP64 operations on both sides, so identical inputs give identical flags,
  - the limited state (dg_cswenolimit) within 1e-11 of the variable's scale, and its modes
    n >= 1 within HI_TOL of their own largest magnitude,
  - optionally the positivity-preserving scaling (dg_positivity_limit) within 1e-11.
The CUDA-graph step (dg_step) from the same state must then reproduce the stage-level
result bitwise: it launches the same kernels in the same order.
"""
import numpy as np

import paper_1904_11147_gb300 as dgl


from parity_cases import rel, rel_hi  # noqa: E402

# limited modes n >= 1 against the largest |U_n|, n >= 1, of their variable
HI_TOL = 1e-11


def shadow_stages(o, g, u0, dt, steps, M=0.01, pp_eps=None, graph_check=True, stop_on_nonfinite=False, t_end=None,
                  indicator="tvb", limiter="csweno"):
    """dt: a number or a function of (step, state).  With t_end the last step is cut to
    end there.  stop_on_nonfinite: a stage output that is not finite on both sides ends
    the run (it must be non-finite on both).  indicator: "tvb" (flags identical) or
    "kxrcf" (flags identical up to the oracle's near-threshold cells: the two sides'
    basis values at the Gauss points are derived independently and may differ in the last
    bit).  Returns (worst stage deviation, worst limited deviation, flagged cells in
    total, steps done, time reached).  limiter: "csweno" or "parent" (parent WENO)."""
    ind = dgl.IND_KXRCF if indicator == "kxrcf" else dgl.IND_TVB
    parent = limiter == "parent"
    g.set_limiter(dgl.LIM_PARENT if parent else dgl.LIM_CSWENO)
    g.set_modes(u0)
    if pp_eps is not None:
        g.set_positivity(True, pp_eps)
    worst_stage = worst_lim = worst_hi = 0.0
    flagged = 0
    t = 0.0
    for k in range(steps):
        prev = g.get_modes()
        if t_end is not None and t >= t_end - 1e-14:
            return worst_stage, worst_lim, flagged, k, t
        h = dt(k, prev) if callable(dt) else dt
        if t_end is not None:
            h = min(h, t_end - t)
        us = prev
        for s in (1, 2, 3):
            g.rk_stage(s, h)
            got = g.get_modes()
            ref = o.rk_stage(s, h, prev, us)
            if stop_on_nonfinite and not (np.isfinite(got).all() and np.isfinite(ref).all()):
                assert not np.isfinite(got).all() and not np.isfinite(ref).all(), (k, s)
                return worst_stage, worst_lim, flagged, k, t
            d = rel(got, ref)
            assert d <= 1e-13, (k, s, "stage", d)
            worst_stage = max(worst_stage, d)
            fl_g, nf, _, near_g = g.flag_cells(ind, M, near_cells=True)
            if ind == dgl.IND_KXRCF:
                fl_o, nf_o, _, _, near_o = o.flag_kxrcf(got, near_cells=True)
                bad = (fl_g != fl_o) & (near_o == 0) & (near_g == 0)
                assert not bad.any(), (k, s, "flags", int(bad.sum()))
            else:
                fl_o, nf_o, _, near_o = o.flag_tvb(got, M, near_cells=True)
                assert nf == nf_o and np.array_equal(fl_g, fl_o), (k, s, "flags", int((fl_g != fl_o).sum()))
                assert np.all(near_g >= near_o), (k, s, "near")
            flagged += nf
            if parent:
                g.parent_wenolimit()
            else:
                g.cswenolimit()
            lim = g.get_modes()
            lref = o.parent_limit(got, fl_g) if parent else o.limit(got, fl_g)
            d = rel(lim, lref)
            assert d <= 1e-11, (k, s, "limiter", d)
            worst_lim = max(worst_lim, d)
            # the rewritten modes n >= 1 against their own scale
            dh = rel_hi(lim, lref)
            assert dh <= HI_TOL, (k, s, "limiter modes n >= 1", dh)
            worst_hi = max(worst_hi, dh)
            if pp_eps is not None:
                g.positivity_limit(pp_eps)
                scaled = g.get_modes()
                ref_pp, _, bad = o.positivity_limit(lim, pp_eps)
                assert bad == 0
                d = rel(scaled, ref_pp)
                assert d <= 1e-11, (k, s, "positivity", d)
                lim = scaled
            us = lim
        assert np.isfinite(us).all(), k
        if graph_check:
            g.set_modes(prev)
            g.step(h, ind, M)
            assert np.array_equal(g.get_modes(), us), (k, "graph step differs from the stage calls")
        else:
            g.set_modes(us)
        t += h
    print("shadow: worst limited deviation of the modes n >= 1 (own scale) %.2e" % worst_hi)
    return worst_stage, worst_lim, flagged, steps, t
