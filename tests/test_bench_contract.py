"""The benchmark's host-side contract on the CPU: the byte model behind the
roofline fractions, and the reference arm (the FP64 oracle timed on the host
cores) with its one JSON line on rank 0 and silence on the other ranks."""
import json

import pytest

import bench


def test_algorithmic_bytes_per_voxel():
    """Bytes per voxel of each kernel for the 1 mm protocol (K = 4 maps, C = 3
    contrasts, I = 22 images, float32; T = 10 Hessian entries), counted from
    each kernel's operand list."""
    ab = bench.algorithmic_bytes(4, 3, 22)
    assert ab["grad_hess"] == 22 * 4 + 4 * 4 + 4 + 3 * 4 + 4 * 4 + 10 * 4   # x, y, b1+, b1-; g, H
    assert ab["grad_hess"] == 176
    assert ab["jtv"] == 20                                  # y in, w out
    assert ab["pcg_init"] == 148                            # w, g, y, H in; L, r, p out
    assert ab["pcg_matvec"] == 76                           # p, H, w in; q out
    assert ab["pcg_update"] == 104                          # q, r, L in; r, z out
    assert ab["uncertainty"] == 60                          # H, w in; var out
    # direction, 29 passes per 30-iteration solve: 15 odd passes (z, p in; p out),
    # pass 2 (also p_{k-2} in, x out) and 13 later even passes (also x in)
    assert ab["pcg_direction_per_solve"] == 15 * 48 + 80 + 13 * 96
    # final: x (folded through pass 28), the two pending directions, y in and out
    assert ab["pcg_final"] == 16 + 2 * 16 + 2 * 16
    assert bench.algorithmic_bytes(4, 3, 22, echo_bytes=2)["grad_hess"] == 176 - 22 * 2


@pytest.fixture
def single_rank(monkeypatch):
    for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)


def test_reference_arm_prints_one_line(monkeypatch, capsys, single_rank):
    monkeypatch.setattr(bench, "SHAPE", (176, 240, 4))
    monkeypatch.setattr(bench, "REF_SAMPLE_Z", 1)
    assert bench.main(["--impl", "reference", "--steps", "2", "--warmup", "1"]) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "176x240x1" in d["config"]["workload"]


def test_reference_arm_other_ranks_are_silent(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
