"""Continuous-batching server and batched/captured calls: every result is the
same alone and in the mix (bit-exact)."""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_29651_gb300 as ni
    ni.build()
    return ni


def _graphs(count, seed):
    u = gg.uniform(seed, 3, 3 * count)
    out = []
    for i in range(count):
        n = int(np.exp(np.log(20) + u[i] * (np.log(4000) - np.log(20))))
        if u[count + i] < 0.5:
            out.append(gg.er_mean_degree(n, 4 + 20 * u[2 * count + i], seed * 1000 + i))
        else:
            out.append(gg.chunglu(n, 2.2 + 0.8 * u[2 * count + i], 8.0, seed * 1000 + i))
    return out


def _alone(ni, rp, ci):
    dev = torch.device("cuda:0")
    out = ni.count(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev))
    ni.check()
    return out.cpu().numpy()


def test_server_results_equal_alone(ni):
    from paper_2606_29651_gb300.serve import Server
    graphs = _graphs(80, 5)
    futs = [None] * len(graphs)
    with Server(0, mem_budget=256 << 20, streams=3, max_batch_graphs=16) as srv:
        def client(lo, hi):
            for i in range(lo, hi):
                futs[i] = srv.submit(*graphs[i])
                time.sleep(0.0005 * (i % 3))
        ts = [threading.Thread(target=client, args=(k * 20, (k + 1) * 20)) for k in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        res = [f.result(timeout=300) for f in futs]
        assert srv.batches < len(graphs)          # requests were batched together
    for i, (rp, ci) in enumerate(graphs):
        assert np.array_equal(res[i], _alone(ni, rp, ci)), i
        if len(rp) < 800:
            assert np.array_equal(res[i], oracle.count(rp, ci)), i


def test_server_rejects_oversized_request(ni):
    from paper_2606_29651_gb300 import NiorcaError
    from paper_2606_29651_gb300.serve import Server
    rp, ci = gg.er(3000, 0.01, 1)
    with Server(0, mem_budget=64 << 10, streams=1) as srv:
        f = srv.submit(rp, ci)
        with pytest.raises(NiorcaError):
            f.result(timeout=60)


def test_batch_in_captured_cuda_graph(ni):
    graphs = _graphs(40, 9)
    rowptr, colidx, vo, eo = gg.pack(graphs)
    dev = torch.device("cuda:0")
    d_rp = torch.from_numpy(rowptr.astype(np.int32)).to(dev)
    d_ci = torch.from_numpy(colidx).to(dev)
    d_vo, d_eo = torch.from_numpy(vo).to(dev), torch.from_numpy(eo).to(dev)
    out = torch.zeros((len(rowptr) - 1, 15), dtype=torch.int64, device=dev)
    ref = ni.count_batch(d_rp, d_ci, d_vo, d_eo).cpu()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ni.count_batch(d_rp, d_ci, d_vo, d_eo, out)     # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ni.count_batch(d_rp, d_ci, d_vo, d_eo, out)
    for _ in range(3):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out.cpu(), ref)
    ni.check()


def test_tuning_knobs_do_not_change_counts(ni, tmp_path, monkeypatch):
    from paper_2606_29651_gb300 import autotune
    monkeypatch.setenv("NIORCA_TUNING_CACHE", str(tmp_path / "tuning.json"))
    rp, ci = gg.rmat(13, 16, seed=21)
    exp = _alone(ni, rp, ci)
    saved = ni.get_tuning()
    try:
        for knobs in ({"warp_maxd": 2, "c4_warp_maxw": 2, "long_row_class": 1},
                      {"grid_tri": 1, "grid_c4": 1, "grid_relabel": 1, "grid_agg": 1, "grid_solve": 1},
                      {"warp_maxd": 33, "c4_warp_maxw": 100, "long_row_class": 20}):
            ni.set_tuning(**knobs)
            assert np.array_equal(_alone(ni, rp, ci), exp), knobs
        dev = torch.device("cuda:0")
        res = autotune.tune_graph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), reps=1)
        assert set(res["params"]) == set(saved) and not res["cached"]
        assert np.array_equal(_alone(ni, rp, ci), exp)
        again = autotune.tune_graph(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev))
        assert again["cached"] and again["params"] == res["params"]
    finally:
        ni.set_tuning(**saved)
