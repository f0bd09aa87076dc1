"""GPU tests of the continuous-batching request engine: every result equals the same request run
alone (through a plan), requests on different cells overlap, resident S-matrices are reused by
key, admission respects the HBM budget, and impossible requests fail cleanly."""
import threading

import numpy as np
import pytest
import torch

from paper_1702_01904_gb300 import prism as P
from paper_1702_01904_gb300.runtime import PrismSimulation, Server

from test_gpu_parity import DET, c_grid, det_c, grid_dict, rand_v

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    from paper_1702_01904_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()
    yield
    torch.cuda.synchronize()


def cells():
    """Uneven cells: grid, cell size, slices, f, seed."""
    out = []
    for i, (n, cell, H, f) in enumerate([(64, 8.0, 3, 2), (128, 12.8, 5, 4), (256, 16.0, 8, 4), (64, 6.4, 2, 1),
                                           (128, 16.0, 4, 2), (256, 32.0, 6, 8)]):
        g = grid_dict(n, n, cell, cell, H, 2.0, f)
        V = torch.from_numpy(rand_v(H, n, n, 40 + i)).pin_memory()
        out.append((g, V))
    return out


def requests_for(g, i):
    rng = np.random.Generator(np.random.PCG64(60 + i))
    n = 7 + 5 * i
    x0 = rng.uniform(0, g["cell_x"], n)
    y0 = rng.uniform(0, g["cell_y"], n)
    probe = P.make_probe(20.0 if i % 2 == 0 else 15.0, c1=10.0 * i)
    return probe, x0, y0


def alone(g, V, probe, x0, y0):
    sim = PrismSimulation(c_grid(g))
    sim.build(V.cuda())
    out = sim.scan(probe, x0, y0, det_c(DET)).cpu().numpy()
    sim.close()
    return out


def test_results_identical_alone_and_in_the_mix():
    cs = cells()
    refs = []
    for i, (g, V) in enumerate(cs):
        probe, x0, y0 = requests_for(g, i)
        refs.append(alone(g, V, probe, x0, y0))
    srv = Server(max_inflight=4)
    tickets = []
    for i, (g, V) in enumerate(cs):       # all submitted at once: they are admitted as slots free up
        probe, x0, y0 = requests_for(g, i)
        tickets.append(srv.submit(c_grid(g), V, probe, x0, y0, det_c(DET), key=0))
    for (t, out), ref in zip(tickets, refs):
        srv.wait(t)
        assert np.array_equal(out, ref)
    info = srv.stats()
    assert info.completed == len(cs) and info.running == 0 and info.pending == 0
    srv.close()


def test_resident_smatrix_is_reused_by_key():
    g = grid_dict(128, 128, 12.8, 12.8, 4, 2.0, 2)
    V = torch.from_numpy(rand_v(4, 128, 128, 70)).pin_memory()
    srv = Server(max_inflight=2)
    probes = [P.make_probe(20.0), P.make_probe(12.0, c1=50.0), P.make_probe(18.0, c3=1e4)]
    x0, y0 = np.linspace(0, 12.8, 9), np.linspace(3, 9, 9)
    first = srv.submit(c_grid(g), V, probes[0], x0, y0, det_c(DET), key=7)
    st = srv.wait(first[0])
    assert st.smatrix_reused == 0
    for pr in probes:
        t, out = srv.submit(c_grid(g), V, pr, x0, y0, det_c(DET), key=7)
        st = srv.wait(t)
        assert st.smatrix_reused == 1
        assert np.array_equal(out, alone(g, V, pr, x0, y0))
    assert srv.stats().resident == 1
    # the same key with another grid is refused
    g2 = grid_dict(64, 64, 12.8, 12.8, 4, 2.0, 2)
    t, _ = srv.submit(c_grid(g2), V, probes[0], x0, y0, det_c(DET), key=7)
    with pytest.raises(P.PrismError) as e:
        srv.wait(t)
    assert e.value.status == P.PRISM_ERR_INVALID
    srv.close()


def test_admission_under_a_tight_budget_and_concurrent_submitters():
    cs = cells()[:4]
    budget = 160 << 20  # fits about one 256^2 cell at a time
    srv = Server(hbm_budget_bytes=budget, max_inflight=4)
    results = {}

    def client(i):
        g, V = cs[i]
        probe, x0, y0 = requests_for(g, i)
        t, out = srv.submit(c_grid(g), V, probe, x0, y0, det_c(DET))
        srv.wait(t)
        results[i] = (out, alone(g, V, probe, x0, y0))

    threads = [threading.Thread(target=client, args=(i,)) for i in range(len(cs))]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert len(results) == len(cs)
    for out, ref in results.values():
        assert np.array_equal(out, ref)
    info = srv.stats()
    assert info.peak_bytes <= budget
    srv.close()


def test_request_larger_than_budget_fails_cleanly():
    g = grid_dict(256, 256, 16.0, 16.0, 8, 2.0, 4)
    V = torch.zeros((8, 256, 256)).pin_memory()
    srv = Server(hbm_budget_bytes=8 << 20, max_inflight=1)
    t, _ = srv.submit(c_grid(g), V, P.make_probe(20.0), [1.0], [1.0], det_c(DET))
    with pytest.raises(P.PrismError) as e:
        srv.wait(t)
    assert e.value.status == P.PRISM_ERR_BUDGET
    srv.close()
