"""The generators' elementary functions (workloads.detmath) are built from IEEE add, subtract, multiply and
divide only, so the inputs are bit-identical on every machine. Here they are held to a few ulps of the
platform's own functions, and the generated problems are checked to depend on nothing else."""
import numpy as np
import pytest

from workloads import detmath, input_hash, poisson2d


def _ulps(got, want):
    want = np.asarray(want, dtype=np.float64)
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), np.finfo(np.float64).tiny) / np.finfo(np.float64).eps)


@pytest.mark.parametrize("name,lo,hi,bound", [
    ("exp", -30.0, 30.0, 4), ("expm1", -2.0, 2.0, 4), ("tanh", -8.0, 8.0, 6),
    ("log", 1e-12, 1.0, 4), ("cos", 0.0, 7.0, 4)])
def test_close_to_platform(name, lo, hi, bound):
    x = np.random.default_rng(0).uniform(lo, hi, 20000)
    ref = {"exp": np.exp, "expm1": np.expm1, "tanh": np.tanh, "log": np.log, "cos": np.cos}[name]
    assert _ulps(getattr(detmath, name)(x), ref(x)) <= bound


def test_sin_absolute_on_the_generator_range():
    # sin(a pi x) with a <= 8 and x in [0, 1]: absolute error at the rounding level
    x = np.random.default_rng(1).uniform(0.0, 8.0 * np.pi, 20000)
    assert np.max(np.abs(detmath.sin(x) - np.sin(x))) <= 4e-16


def test_special_values():
    assert detmath.exp(np.array([0.0]))[0] == 1.0
    assert detmath.tanh(np.array([0.0]))[0] == 0.0
    assert detmath.tanh(np.array([40.0, -40.0])).tolist() == [1.0, -1.0]
    assert detmath.log(np.array([1.0]))[0] == 0.0
    assert detmath.sin(np.array([0.0]))[0] == 0.0 and detmath.cos(np.array([0.0]))[0] == 1.0
    t = np.linspace(-3, 3, 101)
    assert np.array_equal(detmath.tanh(-t), -detmath.tanh(t))      # odd
    assert abs(detmath.pow10(np.array([-10.0]))[0] / 1e-10 - 1) < 1e-14


def test_generator_is_reproducible():
    a = poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7)
    b = poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7)
    assert input_hash(a) == input_hash(b)
    c = poisson2d(3, 2, 37, 11, 9, R=1.5, seed=8)
    assert input_hash(a) != input_hash(c)
