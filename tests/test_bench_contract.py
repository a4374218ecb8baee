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
    assert ab["pcg_init"] == 92                             # w, g, y, H in; z_0 out
    assert ab["uncertainty"] == 60                          # H, w in; var out
    # PCG iterations of a 30-iteration solve: j = 0 (z_0, w, H in; p_0, v_0 out),
    # 29 later ones (z, v, p, w, H in; z, v, p out), the x fold at j = 2 (p_0 in,
    # x out) and at the 13 even j > 2 (p_{j-2}, x in; x out)
    assert bench.step_bytes(0, 4) == 92
    assert bench.step_bytes(1, 4) == 140
    assert bench.step_bytes(2, 4) == 172 and bench.step_bytes(4, 4) == 188
    assert ab["pcg_step_per_solve"] == 92 + 29 * 140 + 32 + 13 * 48
    assert ab["pcg_step"] == ab["pcg_step_per_solve"] / 30
    # final: x (folded through iteration 28), the two pending directions, y in and out
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
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
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


def _capture(path, launches, voxels, hashes=None):
    """An ncu log of one kernel kind with the captured program's own lines."""
    _ncu_csv(path, launches)
    with open(path, "a") as f:
        if hashes is not None:
            f.write(json.dumps({"kernel_source_hashes": hashes}) + "\n")
        f.write(json.dumps({"metric": "m", "config": {"voxels": voxels}}) + "\n")


def test_write_traffic_per_kind_captures(tmp_path):
    """DRAM bytes per launch are the mean over each capture's launches of its
    kind, per voxel of that capture's volume; the kind's source hash comes
    from the captured program's own output."""
    hashes = {k: bench.kernel_source_hash(k) for k in bench.KIND_SOURCES}
    step = "void mpm::k_pcg_step_tma<4, 32, 8, 1>(mpm::DevProblem, int, int, int)"
    _capture(tmp_path / "step.csv", [(step, 1000, 200), (step, 1100, 300)], 10, hashes)
    _capture(tmp_path / "jtv.csv", [("void k_jtv<4>(DevProblem, const float *)", 100, 20)], 4, hashes)
    out = tmp_path / "traffic.json"
    doc = bench.write_traffic([str(tmp_path / "step.csv"), str(tmp_path / "jtv.csv")],
                              out=str(out), commands=["cmd"])
    k = json.load(open(out))["kernels"]
    assert doc["kernels"] == k and json.load(open(out))["capture"] == ["cmd"]
    assert k["pcg_step"]["launches"] == 2 and k["pcg_step"]["dram_bytes_per_launch"] == 1300
    assert k["pcg_step"]["dram_bytes_per_voxel"] == 130.0 and k["pcg_step"]["voxels"] == 10
    assert k["pcg_step"]["source_hash"] == hashes["pcg_step"]
    assert k["jtv"]["dram_bytes_per_voxel"] == 30.0
    assert set(k) == {"pcg_step", "jtv"}
    # a later capture of one kind replaces that kind and keeps the others
    _capture(tmp_path / "jtv2.csv", [("void k_jtv<4>(DevProblem, const float *)", 50, 10)], 4, hashes)
    k2 = bench.write_traffic([str(tmp_path / "jtv2.csv")], out=str(out))["kernels"]
    assert k2["jtv"]["dram_bytes_per_voxel"] == 15.0 and k2["pcg_step"] == k["pcg_step"]


def test_write_traffic_refuses_stale_or_unlabelled_captures(tmp_path):
    """A capture taken from other sources than the current ones, or one whose
    log lacks the program's hashes, is refused rather than stored as current."""
    step = "void k_pcg_step_tma<4, 32, 8>(DevProblem, int, int, int)"
    stale = {k: bench.kernel_source_hash(k) for k in bench.KIND_SOURCES}
    stale["pcg_step"] = "0123456789abcdef"
    _capture(tmp_path / "stale.csv", [(step, 1000, 200)], 10, stale)
    with pytest.raises(ValueError, match="pcg_step was captured"):
        bench.write_traffic([str(tmp_path / "stale.csv")], out=str(tmp_path / "t.json"))
    _capture(tmp_path / "bare.csv", [(step, 1000, 200)], 10, None)
    with pytest.raises(ValueError, match="no source hashes"):
        bench.write_traffic([str(tmp_path / "bare.csv")], out=str(tmp_path / "t.json"))
    assert not (tmp_path / "t.json").exists()


def test_traffic_commands_are_single_kernel_small_captures():
    """Every committed capture names one kernel, a few launches (a whole
    30-iteration solve for the PCG iteration), the clock-control flag and the
    176 x 240 x 128 volume, never the full-size fit."""
    for kind, cmd in zip(bench.TRAFFIC_CAPTURES, bench.TRAFFIC_COMMANDS):
        assert "--clock-control none" in cmd and "-k regex:" in cmd
        assert "--shape 176,240,128" in cmd and "--print-hashes" in cmd
        count = int(cmd.split(" -c ")[1].split()[0])
        assert count <= (30 if kind == "pcg_step" else 3)
    assert bench.TRAFFIC_COMMANDS[-1].startswith("python bench.py --write-traffic")


def test_launch_table_shares(tmp_path):
    _ncu_csv(tmp_path / "t.csv", [("void k_a<1>(int)", 10, 0), ("void k_b(int)", 20, 0),
                                  ("void k_a<1>(int)", 30, 0)])
    rows = bench.launch_table(bench.read_ncu_csv(str(tmp_path / "t.csv"))).splitlines()
    assert rows[0].startswith("3 launches")
    assert rows[1].split()[:2] == ["k_a", "2"] and "66.7%" in rows[1]   # 2 of 3 us
    assert rows[2].split()[:2] == ["k_b", "1"] and "33.3%" in rows[2]
