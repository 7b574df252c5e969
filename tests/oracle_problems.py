"""Bridges the shared workload descriptions to the oracle's Problem type (tests only)."""
from oracle.fem import Problem
from paper_2407_13997_gb300.inputs import KIND_NAMES


def oracle_problem(w):
    return Problem(kind=KIND_NAMES[w.kind], nu=w.nu, conv=w.conv, T=w.T, steady=w.steady,
                   mx=w.mx, my=w.my, amp=w.amp, t0=w.t0)
