"""A seeded stand-in for the few hypothesis features that
``test_oracle_properties.py`` uses, for machines where hypothesis is not
installed: the same strategies, drawn from a fixed-seed numpy generator per
test (no shrinking, no example database), so the property pins still run
there instead of being skipped."""
import zlib

import numpy as np


class _Strategy:
    def __init__(self, fn):
        self._fn = fn

    def draw(self, rng):
        return self._fn(rng)


class st:  # noqa: N801 -- mirrors the hypothesis.strategies module name
    @staticmethod
    def integers(lo, hi):
        return _Strategy(lambda rng: int(rng.integers(lo, hi + 1)))

    @staticmethod
    def sampled_from(xs):
        xs = list(xs)
        return _Strategy(lambda rng: xs[int(rng.integers(len(xs)))])

    @staticmethod
    def composite(fn):
        def make(*args, **kw):
            return _Strategy(lambda rng: fn(lambda s: s.draw(rng), *args, **kw))
        return make


class HealthCheck:
    too_slow = "too_slow"


def event(_msg):
    pass


def settings(max_examples=20, **_kw):
    def deco(f):
        f._max_examples = max_examples
        return f
    return deco


def given(*strategies):
    def deco(f):
        def run():
            rng = np.random.default_rng(zlib.crc32(f.__name__.encode()))
            for _ in range(getattr(run, "_max_examples", 20)):
                f(*[s.draw(rng) for s in strategies])
        run.__name__ = f.__name__
        run.__doc__ = f.__doc__
        return run
    return deco
