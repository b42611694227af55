"""The oracle's FP32-storage option (reading A13): the arithmetic stays FP64,
and what is stored between steps is each post-collision population's
deviation from the rest state w_i(r), rounded to the nearest float32.  Pinned
against the same rounding done outside the oracle by numpy, step by step,
through the oracle's population get / set; a slip (rounding the populations
themselves rather than their deviations) is shown to fail the comparison.
"""
import numpy as np
import pytest

S = pytest.importorskip("oracle.stepper")


def _params(**kw):
    base = dict(nx=23, ny=17, r=0.5, gamma=0.25, nu=0.01, u_lid=0.04)
    base.update(kw)
    return S.OracleParams(**base)


def _numpy_rounded_run(p, steps, shifted=True):
    o = S.Oracle(p)
    w = S.rest_weights(p)[:, None, None]
    for _ in range(steps):
        o.step(1)
        f = o.populations()
        if shifted:
            f = w + (f - w).astype(np.float32).astype(np.float64)
        else:
            f = f.astype(np.float32).astype(np.float64)
        o.set_populations(f)
    return o.populations()


@pytest.mark.parametrize("r,gamma", [(0.5, 0.25), (2.0, 1.0), (1.0, 0.1)])
def test_storage_f32_rounds_the_shifted_populations_every_step(r, gamma):
    p = _params(r=r, gamma=gamma)
    want = _numpy_rounded_run(p, 30)
    o = S.Oracle(_params(r=r, gamma=gamma, storage_f32=1))
    o.step(30)
    got = o.populations()
    assert np.array_equal(got, want)
    # what is stored is a float32 deviation from the rest state
    w = S.rest_weights(p)[:, None, None]
    d = got - w
    assert np.array_equal(d.astype(np.float32).astype(np.float64), d)
    # and it is not the plain FP64 run
    f64 = S.Oracle(p)
    f64.step(30)
    assert not np.array_equal(got, f64.populations())
    rel = np.linalg.norm(got - f64.populations()) / np.linalg.norm(f64.populations() - w)
    assert 1e-9 < rel < 1e-5, rel


def test_rounding_the_populations_themselves_is_caught():
    p = _params()
    slip = _numpy_rounded_run(p, 30, shifted=False)
    o = S.Oracle(_params(storage_f32=1))
    o.step(30)
    assert not np.array_equal(o.populations(), slip)
