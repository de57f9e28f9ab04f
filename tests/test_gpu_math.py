"""FP64 reciprocal, square root and logarithm of the FP64 flux arithmetic
(Newton-Raphson, Goldschmidt, Tang's table-driven logarithm) against
reference values: within 2 ulp of the correctly rounded 1/x and sqrt(x)
(IEEE double in numpy) and of ln x evaluated in extended precision."""
import numpy as np
import pytest

from paper_2607_06045_b300 import idp

pytestmark = pytest.mark.gpu


def _inputs(rng, n):
    a = 10.0 ** rng.uniform(-300, 300, n)                  # wide range
    b = 10.0 ** rng.uniform(-8, 8, n)                      # physical range
    c = 1.0 + rng.uniform(-1e-3, 1e-3, n) * 10.0 ** rng.uniform(-12, 0, n)   # near 1
    d = np.nextafter(np.ldexp(1.0, rng.integers(-60, 60, n)), rng.choice([0.0, np.inf], n))  # near powers of 2
    return np.concatenate([a, b, c, d, [1.0, 2.0, 0.5, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53, 1.4, 116.5]])


def _ulp(v):
    return np.spacing(np.abs(v).astype(np.float64))


def _eval(fn, x):
    import torch
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    idp.idp_eval_math(fn, xd, yd)
    return yd.cpu().numpy()


@pytest.mark.parametrize("fn", [0, 1, 2])
def test_fast_math_ulp(fn):
    rng = np.random.default_rng(7 + fn)
    x = _inputs(rng, 200000)
    y = _eval(fn, x)
    if fn == 0:
        ref = 1.0 / x
        err = np.abs(y - ref) / _ulp(ref)
    elif fn == 1:
        ref = np.sqrt(x)
        err = np.abs(y - ref) / _ulp(ref)
    else:
        xl = x.astype(np.longdouble)
        refl = np.log(xl)
        ref = refl.astype(np.float64)
        nz = ref != 0.0
        err = np.abs((y[nz].astype(np.longdouble) - refl[nz]) / _ulp(ref[nz]).astype(np.longdouble)).astype(np.float64)
        assert np.all(y[~nz] == 0.0)
    assert np.all(np.isfinite(y))
    assert err.max() <= 2.0, (fn, float(err.max()), x[np.argmax(err)])
