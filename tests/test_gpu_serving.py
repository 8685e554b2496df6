"""Served replicas against the same replicas run alone: bit-identical states.

The server admits requests as they arrive into the slots of one batch and steps all
admitted replicas together in chunks (fused launches over every replica); a replica's
trajectory must not depend on what runs beside it, and admissions and retirements keep
the batch's captured graphs."""
import numpy as np
import pytest

from paper_2606_14073_gb300 import nep_params
from paper_2606_14073_gb300.serving import GpuBackend, Request, Server

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("creators", [0, 2])
def test_each_result_same_alone_and_in_the_mix(creators):
    params = nep_params.load()
    reqs = [Request(0, cells=6, T=300.0, B=(0, 0, 0.2), n_steps=60, arrival=0.0, replica=0),
            Request(1, cells=4, T=150.0, B=(0, 0, 0.0), n_steps=35, arrival=0.0, replica=1),
            Request(2, cells=5, T=250.0, B=(0, 0, 0.4), n_steps=47, arrival=0.02, replica=2),
            Request(3, cells=7, T=80.0, B=(0, 0, 0.1), n_steps=23, arrival=0.05, replica=3),
            Request(4, cells=4, T=320.0, B=(0, 0, 0.5), n_steps=71, arrival=0.08, replica=4)]
    be = GpuBackend(params, reserve_bytes=0)
    out = Server(be, max_active=3, chunk=20, creators=creators).run(reqs)
    assert out["requests"] == len(reqs)
    st = be.batch_stats()
    assert st["fused_captures"] == 1 and st["replica_calls"] == 0 and st["fused_calls"] > 1
    for d in out["done"]:
        req = reqs[d.rid]
        h = be.create(req)
        be.attach(h)
        h.step(req.n_steps, req.dt, req.T, req.B)
        alone = be.result(h)
        be.destroy(h)
        for k in ("positions", "spins", "velocities"):
            assert np.array_equal(alone[k], d.result[k]), (d.rid, k)
        assert alone["step"] == d.result["step"] == req.n_steps
    assert out["latency_p99_s"] >= out["latency_p50_s"] > 0
    be.close()
