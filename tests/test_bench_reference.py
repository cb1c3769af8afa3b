"""The reference arm of bench.py (`--impl reference`: the FP64 oracle timed on
the host cores), with the oracle's sample replaced by a stand-in of known
cost so that the sizing of the sample and the printed line can be checked
without spending minutes of CPU time."""
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2503_10148_gb300 import inputs  # noqa: E402


class _Cam:
    width, height = 64, 48


@pytest.fixture
def stand_in(monkeypatch):
    """A sample costs 2 s plus 1 ms per pixel per view (4 views)."""
    calls = []

    def fake_sample(scene_np, cams, n_pix, seed):
        calls.append(n_pix)
        return 2.0 + 1e-3 * n_pix

    monkeypatch.setattr(bench, "_oracle_sample", fake_sample)
    monkeypatch.setattr(inputs, "clusters_1p5m_4views", lambda: ({"n": 1_500_000}, [_Cam()] * 4))
    return calls


def test_reference_arm_sizes_its_sample_from_two_pilots(stand_in, monkeypatch, capsys):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = types.SimpleNamespace(steps=4, warmup=3, workload="clusters_1p5m_4views")
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    # step budget min(6 s, 150 s / 7 steps) = 6 s: (6 - 2) s / 1 ms = 4000 pixels per view
    # (the fitted cost per pixel may round a pixel away)
    n = stand_in[2]
    assert stand_in[:2] == [8, 40] and 3990 <= n <= 4000
    assert stand_in[2:] == [n] * 5  # one more warm-up, then the 4 timed steps
    assert line["impl"] == "reference" and line["unit"] == "Mpix/s" and line["higher_is_better"] is True
    assert line["steps"] == 4 and line["warmup"] == 3 and line["n_gpus"] == 1
    t = 2.0 + 1e-3 * n
    assert line["value"] == pytest.approx(n * 4 / t / 1e6, rel=1e-5)
    assert line["ms_per_step"] == pytest.approx(t * 1e3, abs=0.1)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert f"{n} seeded pixels per view" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["metric"] == bench.METRIC


def test_reference_arm_keeps_at_least_32_pixels_when_the_projection_fills_the_step(stand_in, monkeypatch,
                                                                                   capsys):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    # 200 steps: budget max(1 s, 150 s / 203) = 1 s, below the 2 s projection
    bench.run_reference(types.SimpleNamespace(steps=200, warmup=3, workload="clusters_1p5m_4views"))
    assert set(stand_in[2:]) == {32}
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert "32 seeded pixels per view" in line["cpu_baseline"]["sample"]


def test_reference_arm_prints_only_on_rank_0(stand_in, monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(types.SimpleNamespace(steps=2, warmup=3, workload="clusters_1p5m_4views"))
    assert capsys.readouterr().out == ""
    assert stand_in == []  # no oracle work on the other ranks


def test_kernels_per_step_counts_every_launch_of_the_timed_step():
    """35 launches per step on the 1.5M-component workload (588 list tiles:
    10 tile bits, two radix passes), as the launch list of the captured step
    shows: project; depth sort (init, 4 x (histogram, scan, scatter)),
    pair count, scan, finish, emission; tile sort (2 x 3, range init and
    fix-up); render_fwd; SSIM value, finish, gradient; render_bwd;
    project_bwd; SGHMC, Adam rows, step-counter advance."""
    plan = types.SimpleNamespace(tile_bits=10)
    assert bench.kernels_per_step(plan, "autograd", "full") == 35
    assert bench.kernels_per_step(types.SimpleNamespace(tile_bits=13), "autograd", "full") == 35
    assert bench.kernels_per_step(types.SimpleNamespace(tile_bits=17), "autograd", "full") == 38  # 3 passes
    assert bench.kernels_per_step(plan, "autograd", "l1") == 34
    assert bench.kernels_per_step(plan, "direct", "l1") == 33


def test_alu_roofline_follows_the_per_pair_work_and_device_ceiling():
    """The render roofline: 50 FP32 flops + 2 MUFU per contributing pair for
    the backward, the FP32 pipe binding (50 / (152 x 128 x 2) > 2 / (152 x
    16)); at 1.314e9 pairs in 5.684 ms on 152 SMs at 2070 MHz that is 0.143
    of the ceiling.  The ceiling scales with the SM count it is given."""
    import bench
    r = bench.roofline("render_bwd", 5.684, None, (1_313_980_094, 0), {}, "measured", 152, 2070.0)
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(0.1435, abs=5e-4)
    assert r["peak"] == pytest.approx(80.548, abs=1e-3)
    assert r["detailed_count"]["frac"] == pytest.approx(0.2152, abs=5e-4)
    half = bench.roofline("render_bwd", 5.684, None, (1_313_980_094, 0), {}, "measured", 76, 2070.0)
    assert half["frac"] == pytest.approx(2 * r["frac"], rel=1e-3)
    f = bench.roofline("render_fwd", 2.0, None, (1_000_000_000, 2_000_000_000), {}, "measured", 152, 2070.0)
    # 8 x 2e9 + 12 x 1e9 = 28e9 flops (0.348 ms of FP32) vs 2e9 MUFU (0.397 ms): the MUFU pipe binds
    assert f["frac"] == pytest.approx(2e9 / (152 * 16 * 2.07e9) / 2e-3, rel=1e-3)


def test_profile_code_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    """The DRAM traffic recorded with an ncu capture stays valid through an
    edit of a comment, and not through a change of the code."""
    csrc = tmp_path / "paper_2503_10148_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (csrc / "k.cu").write_text("// header\nint f(int a) {\n  return a + 1;  /* one */\n}\n")
    h0 = bench.code_hash(["k.cu"])
    (csrc / "k.cu").write_text("// a longer header\n// over two lines\nint f(int a) {\n    return a + 1;\n}\n")
    assert bench.code_hash(["k.cu"]) == h0
    (csrc / "k.cu").write_text("// header\nint f(int a) {\n  return a + 2;\n}\n")
    assert bench.code_hash(["k.cu"]) != h0
