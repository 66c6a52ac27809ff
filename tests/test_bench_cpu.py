"""bench.py pieces that run without a GPU: the reference (oracle) arm, the
algorithmic byte counts, and the max-over-ranks timing reduction of the
multi-GPU (replica) path, exercised with gloo ranks on the CPU."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import graphgen as gg  # noqa: E402


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["metric"] == bench.METRIC and rec["unit"] == "edges/s"
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_bytes_small_cases():
    # a triangle: one oriented edge pair closes it; no 4-cycle wedge pair
    rp, ci = gg.complete(3)
    ab = bench.algorithmic_bytes(rp, ci)
    assert ab["B_csr"] == 4 * 4 + 4 * 6
    assert ab["B_out"] == 360
    # the 4-cycle 0-1-2-3: root 3 has wedges 3-0-1 and 3-2-1, root 2 has 2-1-0
    ab = bench.algorithmic_bytes(*gg.cycle(4))
    assert ab["W_c4"] == 3


@pytest.mark.parametrize("pad", [0, (1 << 21) + 5000 - 3000])
def test_four_cycle_tiers_partition_the_wedges(pad):
    # Every live root's wedges go to exactly one 4-cycle kernel, so the
    # per-kernel bytes add up to B_c4 (less the roots with W < 2 or fewer
    # than two in-neighbours, which no kernel walks), with packed tables
    # and, past 2^21 vertices, split ones.
    rp, ci = gg.er_mean_degree(6000, 48, 5)
    rp = np.concatenate([rp, np.full(pad, rp[-1], rp.dtype)])
    ab = bench.algorithmic_bytes(rp, ci)
    tiers = {k: v for k, v in ab["per_kernel"].items() if k.startswith("k_c4")}
    assert set(tiers) == {"k_c4_warp", "k_c4_warp_big", "k_c4_mid", "k_c4_cta", "k_c4_tiled"}
    assert 0 < sum(tiers.values()) <= ab["B_c4"]
    assert ab["B_c4"] - sum(tiers.values()) < 0.001 * ab["B_c4"]
    assert tiers["k_c4_warp"] > 0 and tiers["k_c4_warp_big"] > 0
    if pad:   # split tables: the warp tiers stop at W = 576 and 768
        assert tiers["k_c4_mid"] > 0


def test_hub_roots_go_to_the_key_tiled_tier():
    # a root with more than 1024 in-neighbours is routed to the key-tiled
    # tier whatever its wedge count (no one-warp search of its rows for W)
    rp, ci = gg.er_mean_degree(6000, 4, 3)
    n = len(rp) - 1
    hub_edges = [(v, n) for v in range(0, 6000, 4)]   # 1500 neighbours, all below the hub in any order
    rows = [list(ci[rp[v]:rp[v + 1]]) for v in range(n)] + [[]]
    for v, h in hub_edges:
        rows[v].append(h)
        rows[h].append(v)
    rp2 = np.zeros(n + 2, np.int64)
    rp2[1:] = np.cumsum([len(r) for r in rows])
    ci2 = np.concatenate([np.array(sorted(r), np.int32) for r in rows]).astype(np.int32)
    sh = bench.Shape(rp2.astype(np.int32), ci2)
    t = sh.c4_tiers()
    hub = int(np.flatnonzero(sh.order == n)[0])   # relabelled id of the hub
    assert sh.din[hub] > 1024 and t["k_c4_tiled"][hub]
    assert not any(t[k][hub] for k in t if k != "k_c4_tiled")


def test_small_graph_four_cycle_roots_above_256_wedges_leave_the_warp_tiers():
    # fewer vertices than 32 warps per SM: the warp tiers stop at W = 256
    rp, ci = gg.er_mean_degree(3000, 48, 5)
    sh = bench.Shape(rp, ci)
    t = sh.c4_tiers()
    assert not t["k_c4_warp_big"].any()
    assert (sh.w_root[t["k_c4_warp"]] <= 256).all() and t["k_c4_warp"].any()
    assert t["k_c4_mid"].any() or t["k_c4_midp"].any()


def test_deg_class_matches_library_rule():
    d = np.array([0, 1, 7, 8, 9, 10, 12, 15, 16, 20, 1 << 20, (1 << 20) + (1 << 19)])
    c = bench.deg_class(d)
    assert c.tolist()[:3] == [0, 1, 7]
    assert c[3] == 8 and c[4] == 8 and c[5] == 9 and c[6] == 10 and c[7] == 11 and c[8] == 12
    assert (np.diff(bench.deg_class(np.arange(0, 5000))) >= 0).all()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q.put((rank, bench.reduce_max(1.0 + rank * 2.5, world)))
    dist.destroy_process_group()


def test_reduce_max_over_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(v == pytest.approx(3.5) for _, v in res)
