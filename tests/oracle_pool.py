"""Runs oracle calls over every host core (test infrastructure).

The oracle is a C library called through ctypes, which releases the GIL for
the duration of each foreign call, so a pool of threads runs that many
generations of the oracle at once.  Threads, not processes: nothing is forked
after the tests have initialised CUDA.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import oracle


def workers() -> int:
    return max(1, os.cpu_count() or 1)


def pmap(fn, items):
    """[fn(x) for x in items], evaluated on every host core (in order)."""
    items = list(items)
    oracle.build()
    with ThreadPoolExecutor(max_workers=min(workers(), max(1, len(items)))) as ex:
        return list(ex.map(fn, items))


def mismatches(fn, items):
    """Indices i of items for which fn(items[i]) is false."""
    return [i for i, ok in enumerate(pmap(fn, items)) if not ok]
