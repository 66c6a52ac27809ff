"""Device-detected errors are reported per stream: a malformed graph on one
stream never fails, or clears the error of, a call on another stream, and
the server isolates a malformed request from the others of its batch."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_29651_gb300 as ni
    ni.build()
    return ni


def _batch(graphs, dev):
    rowptr, colidx, vo, eo = gg.pack(graphs)
    return (torch.from_numpy(rowptr.astype(np.int32)).to(dev), torch.from_numpy(colidx).to(dev),
            torch.from_numpy(vo).to(dev), torch.from_numpy(eo).to(dev))


def _bad_graph():
    # 40 vertices; vertex 3's row names vertex 57, outside the graph (EINVAL)
    rp, ci = gg.er(40, 0.2, 3)
    ci = ci.copy()
    ci[rp[3]] = 57
    return rp, ci


def test_concurrent_batches_report_separately(ni):
    from paper_2606_29651_gb300 import Status
    dev = torch.device("cuda:0")
    good = [gg.er(int(n), 0.05, i) for i, n in enumerate((300, 900, 50, 2000))]
    bad = good[:2] + [_bad_graph()] + good[2:]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ni.last_status(s1)
    ni.last_status(s2)
    a, b = _batch(good, dev), _batch(bad, dev)
    torch.cuda.synchronize()
    for rep in range(3):
        oa = ni.count_batch(*a, stream=s1)
        ob = ni.count_batch(*b, stream=s2)
        # the clean stream is read first, while the malformed batch may still run
        assert ni.last_status(s1) == Status.OK, rep
        assert ni.last_status(s2) == Status.EINVAL, rep
        assert ni.last_status(s2) == Status.OK          # read clears the word
    torch.cuda.synchronize()
    ref = ni.count_batch(*a)
    ni.check()
    assert torch.equal(oa, ref)


def test_server_isolates_a_malformed_request(ni):
    from paper_2606_29651_gb300 import NiorcaError, Status
    from paper_2606_29651_gb300.serve import Server
    dev = torch.device("cuda:0")
    graphs = [gg.er(int(n), 0.03, 10 + i) for i, n in enumerate(np.linspace(50, 2500, 30).astype(int))]
    reqs = graphs[:17] + [_bad_graph()] + graphs[17:]
    with Server(0, mem_budget=256 << 20, streams=3, max_batch_graphs=8) as srv:
        futs = [srv.submit(rp, ci) for rp, ci in reqs]
        res = []
        for i, f in enumerate(futs):
            if i == 17:
                with pytest.raises(NiorcaError) as e:
                    f.result(timeout=300)
                assert e.value.status == Status.EINVAL
                res.append(None)
            else:
                res.append(f.result(timeout=300))
    for i, (rp, ci) in enumerate(reqs):
        if i == 17:
            continue
        exp = ni.count(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev))
        ni.check()
        assert np.array_equal(res[i], exp.cpu().numpy()), i
