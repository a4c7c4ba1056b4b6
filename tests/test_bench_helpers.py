"""The bench's roofline bookkeeping (host logic, no GPU): algorithmic work per
launch kind, the mapping of ncu kernel names to kinds, and the traffic file
written from an ncu log, which leaves out launches that returned at once."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HBM, ALU = 6783.5, 40.27


def test_algorithmic_bytes_and_ops():
    n, es = bench.N_VOX, bench.ES
    # a plain filter reads and writes the volume once; the gate-first pass of the
    # five filters reads once and writes five outputs
    assert bench.algorithmic("filter:mean", 0, HBM, ALU) == ("hbm", n * es * 2)
    assert bench.algorithmic("filter:ours", 0, HBM, ALU) == ("hbm", n * es * 2)
    assert bench.algorithmic("gate:ours", 0, HBM, ALU) == ("hbm", n * es * 2)
    assert bench.algorithmic("filter:gate", 0, HBM, ALU) == ("hbm", n * es * 6)
    assert bench.algorithmic("stats", 0, HBM, ALU) == ("hbm", n * es)
    # sigma and Okada: ALU work of the voxels passing the gate, when it outlasts the bytes
    few = n // 100
    assert bench.algorithmic("filter:sigma", few, HBM, ALU)[0] == "hbm"
    bound, ops = bench.algorithmic("filter:sigma", n, HBM, ALU)
    assert bound == "alu" and ops == 4 * (2 * bench.RADIUS + 1) ** 3 * n
    bound, ops = bench.algorithmic("filter:okada", n, HBM, 1.0)
    assert bound == "alu" and ops == 4 * (6 * bench.RADIUS + 1) * n
    assert bench.algorithmic("params", 0, HBM, ALU) == (None, None)


def test_kind_of_kernel():
    k = bench.kind_of_kernel
    assert k("void <unnamed>::k_fast2<unsigned short, 2, 1, 0>(CUtensorMap_st, <unnamed>::Args2)") == "filter:sigma"
    assert k("void <unnamed>::k_fast2<unsigned char, 1, 0, 1>(CUtensorMap_st, <unnamed>::Args2)") == "filter:mean"
    assert k("void gatek::k_gate<unsigned short, 2, 3>(gatek::GateArgs)") == "filter:gate"
    assert k("void gatek::k_gate<unsigned char, 4, 1>(gatek::GateArgs)") == "gate:ours"
    assert k("void gatek::k_gate<unsigned short, 1, 2>(gatek::GateArgs)") == "gate:cube"
    assert k("void <unnamed>::k_ours_fast<unsigned short, 2, 0>(CUtensorMap_st, <unnamed>::FastArgs)") == "filter:ours"
    assert k("void at::native::vectorized_elementwise_kernel<4>(int)") is None


def test_record_traffic_leaves_out_launches_that_returned(tmp_path, monkeypatch):
    rows = [
        ("1", "void gatek::k_gate<unsigned short, 2, 3>(X)", 150e6, 600e6),
        ("2", "void <unnamed>::k_fast2<unsigned short, 2, 1, 0>(X)", 0.0, 0.0),   # returned at once
        ("3", "void <unnamed>::k_ours_fast<unsigned short, 2, 0>(X)", 151e6, 105e6),
        ("4", "void gatek::k_gate<unsigned short, 2, 3>(X)", 152e6, 602e6),
    ]
    lines = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i, name, rd, wr in rows:
        lines.append(f'"{i}","{name}","dram__bytes_read.sum","byte","{rd:.0f}"')
        lines.append(f'"{i}","{name}","dram__bytes_write.sum","byte","{wr:.0f}"')
    csv = tmp_path / "traffic.csv"
    csv.write_text("\n".join(lines) + "\n")
    out = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(out))
    bench.record_traffic(str(csv), 2.0)
    got = {ln.split()[0]: int(ln.split()[1]) for ln in out.read_text().splitlines()}
    assert set(got) == {"filter:gate", "filter:ours"}
    assert got["filter:gate"] == round((150e6 + 600e6 + 152e6 + 602e6) / 2 * 2.0)
    assert got["filter:ours"] == round((151e6 + 105e6) * 2.0)
