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


def _ncu_csv(path, launches):
    """A log in `ncu --csv --metrics ...` form: one row per launch and metric,
    between the profiler's own lines and the program's output."""
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
            '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
            '"Metric Value"\n')
    with open(path, "w") as f:
        f.write("==PROF== Connected to process 1\n")
        f.write('{"metric": "the program\'s own output"}\n')
        f.write(head)
        for i, (name, rd, wr) in enumerate(launches):
            for metric, val in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr),
                                ("gpu__time_duration.sum", 1000)):
                f.write(f'"{i}","1","python3","127.0.0.1","{name}","1","7","(256, 1, 1)",'
                        f'"(1216, 1, 1)","0","10.3","Command line profiler metrics","{metric}",'
                        f'"byte","{val:,}"\n')


def test_write_traffic_takes_the_timed_fit(tmp_path):
    """DRAM bytes per launch come from the last whole fit of the plain capture
    (after the second-to-last k_uncertainty) and from the second half of the
    moved-scan capture; warm-up and autotuning launches do not count."""
    upd = "void k_pcg_update<4, 4>(DevProblem, int, float *, Reduce)"
    unc = "void k_uncertainty<4>(DevProblem, const float *, float *)"
    plain = [("void k_pcg_matvec_tma<4, 16, 16>(DevProblem, int)", 9e9, 9e9),   # autotuner
             (upd, 5e9, 5e9), (unc, 7e9, 7e9),                                 # warm-up fit
             ("void k_jtv<4>(DevProblem, const float *)", 100, 20),              # timed fit
             (upd, 1000, 200), (upd, 1100, 300), (unc, 600, 40)]
    moved = [("void k_grad_hess_proj<4, 0, float>(DevProblem)", 8e9, 8e9),
             ("void k_push_all<4>(DevProblem)", 8e9, 8e9),
             ("void k_grad_hess_proj<4, 0, float>(DevProblem)", 500, 70),
             ("void k_push_all<4>(DevProblem)", 900, 100)]
    _ncu_csv(tmp_path / "plain.csv", plain)
    _ncu_csv(tmp_path / "moved.csv", moved)
    out = tmp_path / "traffic.json"
    doc = bench.write_traffic(str(tmp_path / "plain.csv"), str(tmp_path / "moved.csv"),
                              n_vox=10, out=str(out), commands=["cmd"])
    k = json.load(open(out))["kernels"]
    assert doc["kernels"] == k and json.load(open(out))["capture"] == ["cmd"]
    assert k["pcg_update"]["launches"] == 2 and k["pcg_update"]["dram_bytes_per_launch"] == 1300
    assert k["pcg_update"]["dram_bytes_per_voxel"] == 130.0
    assert k["jtv"]["dram_bytes_per_launch"] == 120
    assert k["uncertainty"] == {"launches": 1, "dram_bytes_per_launch": 640,
                                "dram_bytes_per_voxel": 64.0,
                                "source_hash": bench.kernel_source_hash("uncertainty")}
    assert "pcg_matvec" not in k
    assert k["grad_hess_proj"]["dram_bytes_per_launch"] == 570
    assert k["reslice"]["dram_bytes_per_launch"] == 1000


def test_launch_table_shares(tmp_path):
    _ncu_csv(tmp_path / "t.csv", [("void k_a<1>(int)", 10, 0), ("void k_b(int)", 20, 0),
                                  ("void k_a<1>(int)", 30, 0)])
    rows = bench.launch_table(bench.read_ncu_csv(str(tmp_path / "t.csv"))).splitlines()
    assert rows[0].startswith("3 launches")
    assert rows[1].split()[:2] == ["k_a", "2"] and "66.7%" in rows[1]   # 2 of 3 us
    assert rows[2].split()[:2] == ["k_b", "1"] and "33.3%" in rows[2]
