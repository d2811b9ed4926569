"""Cartesian component bookkeeping for the generator: component (i, j, k) of
degree l, ordered by x exponent descending then y descending."""
from functools import lru_cache


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nsph(l: int) -> int:
    return 2 * l + 1


@lru_cache(maxsize=None)
def tuples(l: int):
    return tuple((i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1))


def index(t) -> int:
    """Position of tuple t within its degree."""
    jk = t[1] + t[2]
    return jk * (jk + 1) // 2 + t[2]


@lru_cache(maxsize=None)
def range_tuples(lo: int, hi: int):
    """All tuples with lo <= degree <= hi, stacked by degree."""
    out = []
    for n in range(lo, hi + 1):
        out.extend(tuples(n))
    return tuple(out)


def sub(t, i, k=1):
    u = list(t)
    u[i] -= k
    return tuple(u)


def add(t, i, k=1):
    u = list(t)
    u[i] += k
    return tuple(u)
