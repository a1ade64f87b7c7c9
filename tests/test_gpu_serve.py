"""The continuous-batching solve server (mb_server_*): a request's result is
the same alone and in a mix of concurrent requests, admission respects the
device-memory budget, and served eigenvalues match the dense oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import eigen as E
from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    mb.load(build_if_missing=True)
    return mb


def _requests():
    tiny = W.tiny()
    slab = W.scaled(W.slab(), ecut=5.0, n_int=21, nbands=6, name="slab-small")
    gra = W.scaled(W.graphene(), ecut=2.5, n_int=13, nbands=10, name="graphene-small")
    tiny_k = dataclasses.replace(tiny, kpts=np.array([[0.2, -0.1], [0.05, 0.3]]))
    return [(tiny, 8, "fp32"), (slab, 6, "fp64"), (gra, 10, "fp32"), (tiny_k, 5, "fp64")]


def test_results_alone_equal_results_in_the_mix(mbmod):
    reqs = _requests()
    alone = []
    srv = mbmod.Server(slots=1, hbm_budget_bytes=200e9)
    for w, nb, prec in reqs:
        rc, ev, info, lat = srv.wait(srv.submit(w, nb, 1e-7, prec))
        assert rc == 0
        alone.append(ev)
    srv.close()
    srv = mbmod.Server(slots=4, hbm_budget_bytes=200e9)
    noise = [srv.submit(W.scaled(W.tiny(), n_int=50 + i, nbands=6), 6, 1e-7, "fp32") for i in range(3)]
    tickets = [srv.submit(w, nb, 1e-7, prec) for w, nb, prec in reqs]
    mixed = []
    for t in tickets:
        rc, ev, info, lat = srv.wait(t)
        assert rc == 0
        mixed.append(ev)
    for t in noise:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    srv.close()
    assert st["peak_running"] > 1          # the work of several requests was in flight together
    for a, b in zip(alone, mixed):
        assert np.array_equal(a, b)        # bitwise: private state, fixed reduction orders
    # and the served values are the eigenvalues
    w, nb, prec = reqs[0]
    m = Hm.model_from_workload(w)
    ref = E.generalized_lowest(m.dense_H(), m.dense_S(), nb)
    assert np.abs(alone[0][0] - ref).max() < 1e-6


def test_admission_respects_the_memory_budget(mbmod):
    w = W.tiny()
    srv = mbmod.Server(slots=4, hbm_budget_bytes=200e9)
    probe = srv.submit(w, 8, 1e-6, "fp32")
    srv.wait(probe)
    srv.close()
    # a budget that holds one such request at a time serializes them
    srv = mbmod.Server(slots=4, hbm_budget_bytes=1.2e9)
    try:
        ts = [srv.submit(W.scaled(w, n_int=37 + i), 8, 1e-6, "fp32") for i in range(4)]
    except mbmod.MBError as e:
        pytest.skip("footprint estimate exceeds the test budget: %s" % e)
    for t in ts:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    srv.close()
    assert st["peak_bytes"] <= 1.2e9
    # a request that can never fit is refused at submission
    srv = mbmod.Server(slots=2, hbm_budget_bytes=1e6)
    with pytest.raises(mbmod.MBError):
        srv.submit(w, 8, 1e-6, "fp32")
    srv.close()
