"""The request loop over resident solvers (hbs_server_*): single-angle requests arriving at
random times, 10 % of them exactly at Wood's anomalies, batched while other batches run;
every result must equal the same angle solved alone."""
import math
import threading
import time

import numpy as np
import pytest

from paper_1301_1247_gb300 import inputs

from gpu_util import relerr, require_lib

pytestmark = pytest.mark.gpu


def _geometries():
    specs = [(inputs.wiggly(11, 0.35, 20, 0.03), 2000, 20.0), (inputs.star(0.3, 0.25, 4), 4000, 30.0),
             (inputs.wiggly(12, 0.3, 30, 0.04), 1200, 10.0)]
    return [o.sample(n) for o, n, _ in specs], [w for _, _, w in specs]


def _angle(rng, omega):
    if rng.random() < 0.1:
        ns = [n for n in range(1, 20) if 1.0 - 2.0 * math.pi * n / omega > -1.0]
        n = int(rng.choice(ns))
        return -math.acos(1.0 - 2.0 * math.pi * n / omega)  # Wood's anomaly of order n
    return float(rng.uniform(-math.pi / 2 + 0.05, -0.05))


def test_serving_results_alone_and_in_the_mix():
    hbs = require_lib()
    geoms, omegas = _geometries()
    handles = hbs.build_batch(geoms, omegas, 1.0, 1e-12)
    sv = hbs.Server(slots=3, max_batch=64)
    gids = [sv.add(h) for h in handles]
    rng = np.random.default_rng(7)
    reqs = []
    lock = threading.Lock()

    def client(seed, count):
        r = np.random.default_rng(seed)
        for _ in range(count):
            gi = int(r.integers(0, len(handles)))
            th = _angle(r, omegas[gi])
            rid = sv.submit(gids[gi], th)
            with lock:
                reqs.append((rid, gi, th))
            time.sleep(float(r.exponential(5e-4)))

    threads = [threading.Thread(target=client, args=(int(rng.integers(1 << 30)), 100)) for _ in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    got = {rid: sv.wait(rid, 300.0) for rid, _, _ in reqs}
    st = sv.stats()
    assert st["submitted"] == st["completed"] == 300
    assert st["batches"] < 300 and st["mean_batch"] > 1.0
    assert 0.0 < st["p50_latency_s"] <= st["p99_latency_s"] <= st["max_latency_s"]
    assert st["solves_per_s"] > 0.0
    for rid, gi, th in reqs:
        o1, c1, d1, f1 = got[rid]
        o2, c2, d2, f2 = handles[gi].solve([th]).bragg(0)
        assert list(o1) == list(o2)
        assert relerr(np.concatenate([c1, d1]), np.concatenate([c2, d2])) < 1e-12
        assert abs(f1 - f2) < 1e-12
    sv.close()


def test_server_admission_by_device_memory():
    hbs = require_lib()
    geoms, omegas = _geometries()
    a = hbs.Handle(*geoms[2], 1.0, omegas[2], 1e-12)
    b = hbs.Handle(*geoms[0], 1.0, omegas[0], 1e-12)
    ia, ib = a.info(), b.info()
    sv = hbs.Server(hbm_budget_bytes=ia["device_bytes"] + ib["device_bytes"] // 2, slots=1)
    ga = sv.add(a)
    with pytest.raises(hbs.HbsError):
        sv.add(b)
    assert sv.stats()["resident_bytes"] == ia["device_bytes"]
    rid = sv.submit(ga, -0.7)
    sv.wait(rid, 60.0)
    sv.remove(ga)
    gb = sv.add(b)
    assert sv.stats()["resident_bytes"] == ib["device_bytes"]
    sv.wait(sv.submit(gb, -0.9), 60.0)
    sv.close()
