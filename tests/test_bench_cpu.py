"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic table written from an
ncu CSV capture and read back, scaled, by the bench line's `traffic` fields."""
import json

import pytest

import bench

HDR = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
       '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _line(i, name, metric, value):
    return (f'"{i}","1","python3.12","127.0.0.1","{name}","1","13","(128, 1, 1)","(516, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","byte","{value}"')


def _csv(tmp_path, launches):
    lines = ["==PROF== Connected to process 1", HDR]
    for i, (name, rd, wr) in enumerate(launches):
        lines += [_line(i, name, "dram__bytes_read.sum", f"{rd:,}"), _line(i, name, "dram__bytes_write.sum", wr),
                  _line(i, name, "gpu__time_duration.sum", 1000)]
    p = tmp_path / "t.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


W = dict(N=64, Nx=4, Nz=4, nu=1e-3, dt=1e-3)          # 3 x 4 = 12 modes, 768 rows


def test_write_and_read_back(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    rows = bench.n_modes_of(W) * W["N"]
    assert rows == 768
    path = _csv(tmp_path, [
        # ncu prints nested template names in several forms: match on the base name
        ("void unnamed>::bih_df_kernel<0>(Plan, const int *, long, long, const double *, double *, float4 *)",
         768 * 40, 768 * 40),
        ("void unnamed>::bih_df_kernel<0>(Plan, const int *, long, long, const double *, double *, float4 *)",
         768 * 42, 768 * 40),
        ("void unnamed>::bih_df_kernel<1>(Plan, const int *, long, long, const double *, double *, float4 *)",
         1, 1),                                                          # other shape: not the table's
        ("void shen::<unnamed>::transform_kernel<1, 1, 0>(shen::<unnamed>::TrArgs, const double *, double *)",
         768 * 16, 768 * 16),
        ("void shen::<unnamed>::transform_kernel<2, 1, 0>(shen::<unnamed>::TrArgs, const double *, double *)",
         768 * 16, 768 * 15),
    ])
    out = bench.write_traffic(path, W)
    bpr = out["bytes_per_row"]
    assert bpr["biharmonic:df"] == pytest.approx(81.0)                   # mean of 80 and 82
    assert bpr["transform:scalar_dirichlet"] == pytest.approx(32.0)
    assert bpr["transform:forward_dirichlet"] == pytest.approx(31.0)
    assert "helmholtz:df" not in bpr
    assert out["launches"]["bih_df_kernel<0>"] == 2
    saved = json.loads((tmp_path / "traffic.json").read_text())
    assert saved["sources_sha1"] == {g: bench.sources_sha1(n) for g, n in bench.TRAFFIC_SOURCES.items()}
    # read back, scaled to another workload's rows
    assert bench.measured_traffic("biharmonic:df", 1000) == pytest.approx(81000.0)
    assert bench.measured_traffic("transform:forward_dirichlet", 10) == pytest.approx(310.0)
    assert bench.measured_traffic("helmholtz:df", 10) is None


def test_stale_sources_give_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    bench.write_traffic(_csv(tmp_path, [("void unnamed>::velocity_df_kernel(Plan)", 768 * 50, 768 * 44)]), W)
    assert bench.measured_traffic("velocity:df", 1) == pytest.approx(94.0)
    t = json.loads((tmp_path / "traffic.json").read_text())
    t["sources_sha1"]["velocity"] = "0" * 40                            # the kernel changed since the capture
    (tmp_path / "traffic.json").write_text(json.dumps(t))
    assert bench.measured_traffic("velocity:df", 1) is None
    assert bench.traffic_group("matvec_helmholtz:df") == "matvec"
    assert bench.traffic_group("transform:inverse_dirichlet") == "transform"
    assert bench.traffic_group("helmholtz:df") == "df"


def test_reference_arm_times_whole_sampled_steps():
    """--impl reference times K sampled steps of the oracle on the host cores: ms_per_step is
    a measured step (so steps x ms_per_step fits inside the run's own wall time), and the
    whole-workload figure is labelled as extrapolated."""
    import os
    import subprocess
    import sys
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    t = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "small",
                        "--steps", "4", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    wall = time.perf_counter() - t
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 4
    assert 0 < line["ms_per_step"] * line["steps"] / 1e3 < wall
    assert line["value"] == pytest.approx(2 * line["config"]["sample_rows"] / (line["ms_per_step"] * 1e-3), rel=1e-6)
    assert line["full_step_ms_extrapolated"] >= line["ms_per_step"] * 0.999
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_traffic_from_one_capture_per_kernel(tmp_path, monkeypatch):
    """Captures taken one kernel at a time restart their launch IDs: each file's launches
    stay apart."""
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "traffic.json"))
    a = tmp_path / "a"
    b = tmp_path / "b"
    a.mkdir()
    b.mkdir()
    pa = _csv(a, [("void unnamed>::bih_df_kernel<0>(Plan)", 768 * 40, 768 * 40)])
    pb = _csv(b, [("void unnamed>::helm_df_kernel<0>(Plan)", 768 * 30, 768 * 30)])
    bpr = bench.write_traffic([pa, pb], W)["bytes_per_row"]
    assert bpr["biharmonic:df"] == pytest.approx(80.0)
    assert bpr["helmholtz:df"] == pytest.approx(60.0)


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    """The traffic table stays valid across comment edits of unchanged kernel code, and
    turns stale when the code changes."""
    csrc = tmp_path / "paper_1701_03787_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "k.cu").write_text("// one\nint a = 1; /* two\nlines */ int b = 2;\n")
    h0 = bench.sources_sha1(("k.cu",))
    (csrc / "k.cu").write_text("// reworded\nint a = 1; /* other */ int b = 2;\n")
    assert bench.sources_sha1(("k.cu",)) == h0
    (csrc / "k.cu").write_text("// reworded\nint a = 3; /* other */ int b = 2;\n")
    assert bench.sources_sha1(("k.cu",)) != h0


def test_precision_per_problem():
    """A refinement precision names the fused Helmholtz kernels; the biharmonic solve of the
    step then runs in float-float (its plain solve has no fused refinement)."""
    assert bench.resolve_precision("df_r1") == {"helmholtz": "df_r1", "biharmonic": "df"}
    assert bench.resolve_precision("fp32_r1") == {"helmholtz": "fp32_r1", "biharmonic": "df"}
    for p in ("fp64", "df"):
        assert bench.resolve_precision(p) == {"helmholtz": p, "biharmonic": p}
    assert set(bench.resolve_precision("auto")) == {"helmholtz", "biharmonic"}
