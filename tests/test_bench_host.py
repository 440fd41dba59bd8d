"""Host-side pieces of bench.py (no GPU): every workload builds inputs of the
stated shape with the compatibility condition met exactly, and names itself."""

import importlib.util
import math
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,n", [("stokes_tp", 4096), ("stokes_dp_slab", 4096), ("stokes_tp_batch16", 2048),
                                    ("laplace_tp_multi", 6), ("stokes_chebyshev", 9), ("stokes_lognormal", 3000),
                                    ("stokes_tp_pressure", 2048)])
def test_workloads_shapes_and_neutrality(name, n):
    b = _bench()
    wl = b.WORKLOADS[name]
    x, d, off, desc = b.workload(name, n, 0)
    k = 1 if wl["kernel"] in (0, 2) else 3  # source density components
    assert x.ndim == 2 and x.shape[1] == 3 and d.shape == (wl["nrhs"], len(x), k)
    assert np.all((x >= 0) & (x <= 1))
    segs = [(0, len(x))] if off is None else list(zip(off[:-1], off[1:]))
    for r in range(wl["nrhs"]):
        for a, c in segs:
            for comp in range(k):
                assert math.fsum(d[r, a:c, comp]) == 0.0
    assert isinstance(desc, str) and desc
    assert b.workload_name(name, wl, n, wl["p"], wl["leaf"]).startswith(name.split("_")[0])


def test_traffic_note_requires_matching_source():
    b = _bench()
    assert b.m2l_traffic("no_such_workload") is None


def test_oracle_sample_velocity_pressure():
    # the reference values of the velocity-pressure workload: (u, p) per target
    import oracle
    b = _bench()
    wl = b.WORKLOADS["stokes_tp_pressure"]
    x, d, off, _ = b.workload("stokes_tp_pressure", 300, 0)
    idx, ref = b.oracle_sample(wl, x, d, off, 5, np.random.default_rng(0))
    assert ref.shape == (5, 4)
    np.testing.assert_allclose(ref[:, :3], oracle.stokes_tp(x, d[0], x[idx]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(ref[:, 3], oracle.stokes_pressure(7, x, d[0], x[idx]), rtol=0, atol=1e-13)
