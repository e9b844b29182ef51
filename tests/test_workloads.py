"""Seeded synthetic workloads (CPU): every workload the benchmark accepts exists, states its
grid in its name and is reproduced exactly from its seeds."""
import importlib.util
import os

import numpy as np

from paper_2505_10168_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bench_workloads_resolve_and_name_their_grid():
    bench = _bench()
    for name in bench.WORKLOADS:
        fn = getattr(wl, name)
        small = fn() if name == "rod_blocks" else fn(N=64, NT=128)
        assert "%dx%d" % (small["N"], small["NT"]) in small["name"], small["name"]
        q = np.asarray(small["q"])
        assert q.shape == (small["NT"] + 1, small["N"])


def test_workloads_are_reproducible():
    a, b = wl.filtered_simp(N=64, NT=32), wl.filtered_simp(N=64, NT=32)
    np.testing.assert_array_equal(a["chi"], b["chi"])
    r1, r2 = wl.serving_requests(16), wl.serving_requests(16)
    assert [(r["N"], r["NT"], r["kmin"], r["adjoint"]) for r in r1] == [(r["N"], r["NT"], r["kmin"], r["adjoint"]) for r in r2]
    k1, k2 = wl.request_fields(r1[3])[0], wl.request_fields(r2[3])[0]
    np.testing.assert_array_equal(k1, k2)
    assert set(np.unique(k1)) <= {r1[3]["kmin"], 1.0}
