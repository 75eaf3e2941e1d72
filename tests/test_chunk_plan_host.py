"""Omega-chunk planning of the FP32 path, on the host (no GPU).

The library's split search (sc_plan_omega_chunks) must give the same chunks
as the search written again in tune_chunks.py, on the throughput tables
compiled into the library (read from its source), for every count up to
3000 omegas and both request sizes.  The search itself is pinned on
synthetic tables: with equal throughput for every count a request stays one
chunk, a much faster 1- and 32-omega class splits 33 as 1 + 32, and the
per-chunk charge keeps near-ties whole.
"""
import os
import re

import pytest

import paper_1609_08146_gb300 as sc
from paper_1609_08146_gb300 import tune_chunks as tc

SRC = os.path.join(os.path.dirname(sc.__file__), "csrc", "sc_batch.cpp")


def _tables():
    text = open(SRC).read()
    small = re.search(r"kRateSmall\[65\] = \{(.*?)\};", text, re.S).group(1)
    full = re.search(r"kRateFull\[6\] = \{(.*?)\};", text, re.S).group(1)
    num = lambda t: [float(x.rstrip("f")) for x in re.findall(r"[0-9]+\.[0-9]*f?", re.sub(r"//[^\n]*", "", t))]
    small, full = num(small), num(full)
    assert len(small) == 65 and len(full) == 6
    return small, full


@pytest.mark.parametrize("small_cuts", [True, False])
def test_library_plan_equals_the_python_search(small_cuts):
    small, full = _tables()
    first = tc.first_chunks(small, full, small_cuts=small_cuts)
    pairs = 1 << 30 if small_cuts else 1000
    for n in range(1, 3001):
        got = sc.plan_omega_chunks(n, pairs)
        assert got == tc.plan(n, first), n
        assert sum(got) == n and all(1 <= c <= 2048 for c in got)


def test_uniform_throughput_keeps_one_chunk():
    small = [0.0] + [1.0] * 64
    full = [float(c) for c in tc.FULL]  # a grouped chunk of capacity c at rate c: cost 1 per omega slot
    first = tc.first_chunks(small, full)
    assert first[1:65] == list(range(1, 65))


def test_fast_classes_are_split_out():
    small = [0.0] + [1.0] * 64
    small[1] = small[32] = 10.0
    full = [float(c) for c in tc.FULL]
    first = tc.first_chunks(small, full)
    assert tc.plan(33, first) == [1, 32]


def test_extra_chunk_is_charged():
    small = [0.0] + [1.0] * 64
    small[32] = 1.01  # 1% faster: less than the 2% charge of an extra chunk
    full = [float(c) for c in tc.FULL]
    first = tc.first_chunks(small, full)
    assert first[33] == 33


def test_idle_grouped_slots_are_cut_off():
    # 65 omegas on 16 threads of 8 would leave 7 idle: a full 64 and a rest
    assert sorted(sc.plan_omega_chunks(65, 1000)) == [1, 64]
    assert sorted(sc.plan_omega_chunks(129, 1000)) == [1, 128]


def test_plan_errors():
    lib = sc.load()
    import ctypes

    sizes = (ctypes.c_int * 4)()
    n = ctypes.c_int()
    assert lib.sc_plan_omega_chunks(None, 0, 1, sizes, 4, ctypes.byref(n)) == sc.SC_ERR_INVALID
    assert lib.sc_plan_omega_chunks(None, 5000, 1 << 30, sizes, 1, ctypes.byref(n)) == sc.SC_ERR_INVALID
    assert n.value > 1  # the count is reported even when the sizes do not fit
