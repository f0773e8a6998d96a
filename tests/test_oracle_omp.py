"""The all-cores build of the oracle (liboracle_omp.so: the same source with
-fopenmp) computes the same states as the serial build, bit for bit, in 2D,
3D and on a stretched z-grid: its pragmas only split per-node loops."""
import os

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("cfg", [O.Config(nx=96, nz=33, Ra=1e7, pert_amp=1e-2),
                                 O.Config(nx=24, ny=16, nz=13, ndim=3, Ra=1e6, pert_amp=1e-2),
                                 O.Config(nx=64, nz=29, Ra=1e6, zstretch=1.5, pert_amp=1e-2)])
def test_openmp_build_is_bit_identical(cfg, monkeypatch):
    path = O.build_omp()
    if path is None:
        pytest.skip("gcc has no OpenMP here")
    monkeypatch.setenv("OMP_NUM_THREADS", str(max(2, min(8, os.cpu_count() or 2))))
    X0 = O.init(cfg)
    A, tA, dA = O.step(cfg, X0, 4)
    with O.library(path):
        B, tB, dB = O.step(cfg, X0, 4)
    assert np.array_equal(A, B) and tA == tB and np.array_equal(dA, dB)
