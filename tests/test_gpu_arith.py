"""The refined FP64 reciprocal and square root of the stage and limiter kernels against
IEEE arithmetic: special values give the IEEE result, and normal arguments are within two
units in the last place (relative error <= 2^-51) of the correctly rounded value."""
import numpy as np
import pytest

import paper_1904_11147_gb300 as dgl

pytestmark = pytest.mark.gpu

SPECIAL = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-310, 2.0 ** 1022, -2.0 ** 1022,
           1.7976931348623157e308, -1.7976931348623157e308, np.inf, -np.inf, np.nan, -1.0, -3.7, 1.0, 3.7,
           2.0 ** 1021, 2.0 ** -1021]


def _run(op, x):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    out = torch.empty_like(t)
    dgl.refined_arith(op, t, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _same(a, b):
    return (np.isnan(a) & np.isnan(b)) | (a == b) & (np.signbit(a) == np.signbit(b))


def test_special_values_reciprocal():
    x = np.array(SPECIAL)
    got = _run(0, x)
    with np.errstate(divide="ignore"):
        want = 1.0 / x
    big = np.abs(x) >= 2.0 ** 1022
    tiny = (np.abs(x) < 2.0 ** -1022)
    special = big | tiny | ~np.isfinite(x)
    assert np.all(_same(got[special], want[special])), (x[special], got[special], want[special])
    rel = np.abs(got[~special] - want[~special]) / np.abs(want[~special])
    assert rel.max() <= 2.0 ** -51


def test_special_values_square_root():
    x = np.array(SPECIAL)
    got = _run(1, x)
    with np.errstate(invalid="ignore"):
        want = np.sqrt(x)
    special = ~(np.isfinite(x) & (x >= 2.0 ** -1022))
    assert np.all(_same(got[special], want[special])), (x[special], got[special], want[special])
    rel = np.abs(got[~special] - want[~special]) / np.abs(want[~special])
    assert rel.max() <= 2.0 ** -51


@pytest.mark.parametrize("op", [0, 1])
def test_accuracy_over_the_normal_range(op):
    rng = np.random.default_rng(31 + op)
    x = np.exp(rng.uniform(np.log(1e-300), np.log(1e300), 2_000_000))
    if op == 0:
        x *= rng.choice([-1.0, 1.0], x.size)
    got = _run(op, x)
    want = 1.0 / x if op == 0 else np.sqrt(x)
    rel = np.abs(got - want) / np.abs(want)
    print("max relative error %.3e" % rel.max())
    assert rel.max() <= 2.0 ** -51
