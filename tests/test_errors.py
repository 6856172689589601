"""The parity metrics reject NaN and infinity: a result that is NaN anywhere
fails the finiteness assertion, and a running maximum that has seen NaN stays
NaN, so a bound ``worst < tol`` is false.  Host-made arrays only."""
import numpy as np
import pytest

from tests._errors import Worst, assert_finite, max_abs_rel, rel_l2, rel_l2_field


def _fields():
    rng = np.random.default_rng(0)
    ref = rng.normal(size=(3, 4, 5))
    return ref + 1e-9 * rng.normal(size=ref.shape), ref


def test_finite_inputs_give_the_plain_metrics():
    got, ref = _fields()
    e = [np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c]) for c in range(3)]
    assert rel_l2(got, ref) == pytest.approx(max(e), rel=1e-12)
    assert rel_l2_field(got, ref) == pytest.approx(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert max_abs_rel(got, ref) == pytest.approx(np.abs(got - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("metric", [rel_l2, rel_l2_field, max_abs_rel])
def test_non_finite_result_fails(bad, metric):
    got, ref = _fields()
    got[1, 2, 3] = bad
    with pytest.raises(AssertionError, match="not finite"):
        metric(got, ref)
    with pytest.raises(AssertionError, match="not finite"):
        metric(np.full_like(ref, bad), ref)


def test_assert_finite_counts_every_bad_value():
    a = np.zeros(10)
    a[[2, 7]] = np.nan
    with pytest.raises(AssertionError, match="2 of 10"):
        assert_finite(a)


def test_running_maximum_keeps_nan():
    assert max(0.0, float("nan")) == 0.0          # the pitfall the helper exists for
    w = Worst()
    w.update(1e-7)
    w.update(float("nan"))
    w.update(2e-7)
    assert np.isnan(w.value)
    assert not (w < 1e-5)
    w2 = Worst()
    for x in (3e-7, 1e-7, 5e-7):
        w2.update(x)
    assert w2.value == 5e-7 and w2 < 1e-5
