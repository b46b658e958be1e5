"""The C-ABI library loads on any machine and exports every declared entry point.

CPU-only: no call here launches GPU work.  Argument errors are rejected on
the host before anything is launched, so they can be checked without a GPU.
"""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1601_07789_gb300 import build, flyte

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols() -> set[str]:
    text = open(os.path.join(ROOT, "include", "flyte.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(flyte_[a-z_0-9]+)\s*\(", text))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return flyte.lib()


def test_header_declares_the_boundary():
    assert declared_symbols() == set(flyte.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_version(lib):
    assert lib.flyte_version() >= 100


@pytest.mark.parametrize("k,base", [(0, 0), (5, 0), (9, 1), (2, 7), (-1, 1)])
def test_bad_format_rejected_on_host(lib, k, base):
    st = lib.flyte_pack(None, None, 10, flyte.Fmt(k, base), 1, 1, 0, None)
    assert st == 1
    assert b"format" in lib.flyte_last_error_string()
    assert lib.flyte_unpack(None, None, 10, flyte.Fmt(k, base), 1, 1, None) == 1


def test_bad_sizes_strides_modes_rejected_on_host(lib):
    f = flyte.Fmt(3, 1)
    assert lib.flyte_pack(None, None, -1, f, 1, 1, 0, None) == 1
    assert lib.flyte_pack(None, None, 10, f, 0, 1, 0, None) == 1
    assert lib.flyte_pack(None, None, 10, f, 1, -2, 0, None) == 1
    assert lib.flyte_pack(None, None, 10, f, 1, 1, 9, None) == 1
    assert lib.flyte_pack(None, None, 10, f, 1, 1, 0, None) == 1      # null pointers
    assert lib.flyte_unpack(None, None, 10, f, 1, 1, None) == 1


def test_zero_length_is_a_noop(lib):
    f = flyte.Fmt(3, 1)
    assert lib.flyte_pack(None, None, 0, f, 1, 1, 0, None) == 0
    assert lib.flyte_unpack(None, None, 0, f, 1, 1, None) == 0


def test_batch_job_layout_and_host_validation(lib):
    assert ctypes.sizeof(flyte.Job) == 88
    bad = (flyte.Job * 1)(flyte.Job(9, 0, flyte.Fmt(3, 1), flyte.Fmt(3, 1), 0, 10, None, None, None, None, 0.0, 0.0))
    assert lib.flyte_batch_workspace_bytes(bad, 1) == ctypes.c_size_t(-1).value
    assert lib.flyte_batch_prepare(bad, 1, None, 0, None) == 1
    assert b"job 0" in lib.flyte_last_error_string()
    big = (flyte.Job * 1)(flyte.Job(3, 0, flyte.Fmt(3, 1), flyte.Fmt(3, 1), 4, 5000, 1, 1, 1, None, 1.0, 0.0))
    assert lib.flyte_batch_prepare(big, 1, None, 0, None) == 2     # gemv side above the batch limit
    ok = (flyte.Job * 1)(flyte.Job(0, 0, flyte.Fmt(3, 1), flyte.Fmt(3, 1), 0, 1000, 16, None, 16, None, 0.0, 0.0))
    assert 0 < lib.flyte_batch_workspace_bytes(ok, 1) < 4096


def test_batch_plan_reserves_the_split_x_of_gemv_n_jobs(lib):
    """The planner (host code) keeps a binary32 pair slot, 8 bytes per entry of x, for each gemv 'N' job
    on the double-word path, split once per launch; a job too short for that path (binary64 row sums)
    gets none."""
    def ws(n, count):
        jobs = (flyte.Job * count)(*[flyte.Job(3, 0, flyte.Fmt(4, 1), flyte.Fmt(4, 1), 64, n, 1, 1, 1, None, 1.0,
                                               0.0) for _ in range(count)])
        return lib.flyte_batch_workspace_bytes(jobs, count)

    long_rows = ws(2048, 2) - ws(2048, 1)     # n = 2048: the double-word path
    short_rows = ws(300, 2) - ws(300, 1)      # n = 300: too short for its bound
    assert long_rows >= 8 * 2048
    assert short_rows < 8 * 300               # its job and tile entries only, no x slot
