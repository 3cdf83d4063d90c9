"""Partitioning constraints of Section 3.1 — test infrastructure only (see ``oracle/__init__``).

The paper requires that every vector V_i shared by two consecutive kernels be
split into the same p partitions V_i^j, that the partitions cover V_i, and that
each partition respect the vector's elementary partitioning unit epu(V_i), the
number of elements nu(V_i, K) each thread of kernel K computes, and the
work-group size wgs_j(K). The right-hand side of the printed condition is
garbled ("#V mod (epu/nu)"); the executor reads it as: a partition holds a
whole number of elementary units, and epu is a multiple of nu, so every
thread's elements lie inside one unit. On a GPU the work-group condition
(#V_i^j / nu divisible by the block size) is replaced by masking the last
block's idle threads, so it is checked only where the plan claims it.

`check_plan` takes a list of partitions as (start, length) element ranges.
"""
from __future__ import annotations


def check_plan(total: int, parts, epu: int, nu: int, block: int | None = None,
               ragged_tail_ok: bool = True) -> list[str]:
    """Return a list of violated constraints (empty when the plan is valid)."""
    errs = []
    if epu <= 0 or nu <= 0:
        return ["epu and nu must be positive"]
    if epu % nu:
        errs.append(f"epu {epu} is not a multiple of nu {nu}")
    cur = 0
    for k, (s, n) in enumerate(sorted(parts)):
        if s != cur:
            errs.append(f"partition {k} starts at {s}, expected {cur} (gap or overlap)")
        last = (s + n == total)
        if n % epu and not (ragged_tail_ok and last and total % epu):
            errs.append(f"partition {k} of {n} elements is not a whole number of units of {epu}")
        if block is not None and (n // nu) % block and not (ragged_tail_ok and last):
            errs.append(f"partition {k}: {n // nu} threads is not a multiple of the block size {block}")
        cur = s + n
    if cur != total:
        errs.append(f"partitions cover {cur} of {total} elements")
    return errs
