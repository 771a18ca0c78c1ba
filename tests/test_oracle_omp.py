"""The OpenMP build of the oracle (the multi-core CPU baseline) gives the plain
build's results bit for bit: its parallel loops (the per-particle push, the
Yee stages by row) have independent iterations and the deposit stays serial,
so no sum changes its order."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("three", [False, True], ids=["2d3v", "3d3v"])
def test_openmp_oracle_is_bit_identical(oracle_mod, three):
    wl = W.small_case3(nx=30, ny=16, nz=12, ppc=2, u_th=0.3, a0=3.0) if three else \
        W.small_case(nx=48, ny=32, ppc=3, u_th=0.3, a0=3.0, two_species=True)
    parts = W.generate_particles(wl)
    plain = oracle_mod.OracleSim(wl, parts, step=5)
    plain.step(6)
    with oracle_mod.parallel() as nthreads:
        par = oracle_mod.OracleSim(wl, parts, step=5)
        par.step(6)
    assert nthreads >= 1
    for k in plain.f:
        assert np.array_equal(plain.f[k], par.f[k]), k
    for a, b in zip(plain.p, par.p):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert (~plain.p[0]["alive"].astype(bool)).sum() >= 0
