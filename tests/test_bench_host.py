"""Host-side logic of bench.py (no GPU): roofline arithmetic, the traffic record
lookup, and the max/sum reductions over ranks with gloo at world size 2."""
import json
import os
import socket

import pytest

import bench
from workloads import cavity64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_roofline_hbm_and_alu():
    d = cavity64().desc
    pk = {"hbm_gbs": 6775.3, "hbm_src": "measured", "fp32_tflops": 80.5, "fp64_tflops": 1.26}
    r = bench.roofline("krylov_dot", 10, 2.0, 13.55e9, d, pk)  # 13.55 GB in 2 ms
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(6775.0, rel=1e-3)
    assert r["frac"] == pytest.approx(1.0, rel=1e-3)
    # the projections' second roof: one float64 FMA per float64 read
    assert r["alu_fp64"]["achieved"] == pytest.approx(13.55e9 / 8 * 2 / 2e-3 / 1e12, rel=1e-3)
    # a float32 basis (the inner solves of refinement) has no float64 roof
    assert "alu_fp64" not in bench.roofline("krylov_dot", 10, 2.0, 13.55e9, d, pk, basis_f64=False)
    r = bench.roofline("ns_jvp_f32", 4, 1.0, 0.0, d, pk)
    flops = 8 * (486 + 114) * d.ne
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(flops / 250e-6 / 1e12, rel=1e-3)
    assert bench.roofline("stage", 0, 0.0, 0.0, d, pk) is None


def test_roofline_picks_the_binding_roof():
    """The NS product declares its coefficient stream: the float32 product is bound by
    HBM (1.26 GFLOP against 80 TFLOP/s takes less than 0.38 GB against 6.8 TB/s), the
    float64 one by the float64 FMA rate; the other roof is reported beside it."""
    d = cavity64().desc
    pk = {"hbm_gbs": 6775.3, "hbm_src": "measured", "fp32_tflops": 80.5, "fp64_tflops": 1.26,
          "alu_src": "test"}
    r32 = bench.roofline("ns_jvp_f32", 10, 1.0, 10 * 383e6, d, pk)
    assert r32["bound"] == "hbm" and r32["other_roof"]["bound"] == "alu"
    assert r32["achieved"] == pytest.approx(383e6 / 100e-6 / 1e9, rel=1e-3)
    r64 = bench.roofline("ns_jvp_f64", 10, 10.0, 10 * 760e6, d, pk)
    assert r64["bound"] == "alu" and r64["other_roof"]["bound"] == "hbm"


def test_traffic_record_requires_matching_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel")
    import hashlib
    (tmp_path / "profiles").mkdir()
    rec = {"krylov_dot": {"sources": ["k.cu"], "sha256": hashlib.sha256(b"kernel").hexdigest(),
                          "traffic_ratio": 1.02, "note": "n"}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("krylov_dot")["traffic_ratio"] == 1.02
    d = cavity64().desc
    pk = {"hbm_gbs": 6775.3, "hbm_src": "measured", "fp32_tflops": 80.5, "fp64_tflops": 1.26}
    assert bench.roofline("krylov_dot", 10, 2.0, 1.0e9, d, pk)["traffic"] == round(1.02 * 1.0e8)
    src.write_text("changed kernel")
    assert bench.traffic_record("krylov_dot") is None


def _worker(rank, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    q.put((rank, bench.reduce_max(1.0 + rank, 2), bench.reduce_sum(10.0 * (rank + 1), 2)))
    dist.destroy_process_group()


def test_rank_reductions_gloo_world_size_2():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
    assert all(r[1] == 2.0 and r[2] == 30.0 for r in res)


def test_operator_rates():
    prof = {"ns_jvp_f32": (10, 2.0), "ns_jvp_f64": (2, 12.0), "ac_residual": (4, 0.4), "b_jvp_f32": (3, 0.6),
            "krylov_dot": (100, 5.0), "ns_diag": (1, 0.1), "stage": (0, 0.0)}
    r = bench.operator_rates(prof, 1000)
    assert set(r) == {"ns_jvp_f32", "ns_jvp_f64", "ac_residual", "b_jvp_f32"}
    assert r["ns_jvp_f32"]["gdofs"] == pytest.approx(4000 * 10 / 2e-3 / 1e9, rel=1e-3)
    assert r["ac_residual"]["gdofs"] == pytest.approx(1000 * 4 / 0.4e-3 / 1e9, rel=1e-3)
    assert r["b_jvp_f32"]["gdofs"] == pytest.approx(6000 * 3 / 0.6e-3 / 1e9, rel=1e-3)
    assert r["ns_jvp_f64"]["us_per_launch"] == pytest.approx(6000.0)

