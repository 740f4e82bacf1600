"""The OpenMP build of the oracle (the same source compiled with -fopenmp:
faces, cells and the cells of each sweep diagonal spread over threads) must
give the serial build's results bit for bit: each face and cell is computed by
one thread with the same arithmetic, and the sweep visits the cells of one
anti-diagonal at a time, an order the serial build is pinned to reproduce
(test_sgs_wavefront_equals_serial_bitwise)."""
import os

import numpy as np
import pytest

import oracle
from paper_1704_03151_gb300 import workloads as wl


def cases():
    body = wl.square_cylinder(ma=2.0, kn=0.5, nvel=13, vmax=8.0, levels=2, nx_side=8, nx_sq=4, ny_side=8,
                              ny_sq=4, half=3.0, dtn_growth=0.0)
    sym = wl.couette(n=10, nvel=12, kn=0.3, t_bottom=1.0, t_top=1.3, u_top=0.2, nx=6)
    return {"cavity_L3": wl.cavity(n=24, nvel=12, kn=0.5, lid=0.2, levels=3), "square_L2": body, "couette": sym}


@pytest.mark.parametrize("name", ["cavity_L3", "square_L2", "couette"])
def test_openmp_build_matches_serial_bitwise(name, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    case = cases()[name]
    fields = wl.initial_fields(case) if case.get("rear") else wl.random_fields(case, 3, amp=0.08)
    a, b = oracle.Oracle(case), oracle.Oracle(case, omp=True)
    for o in (a, b):
        o.init_fields(*fields)
    ra, rb = a.step(3), b.step(3)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.get_f(), b.get_f())
    for k, v in a.macro().items():
        assert np.array_equal(v, b.macro()[k]), k
