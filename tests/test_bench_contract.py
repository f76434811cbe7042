"""Host-side checks of bench.py (no GPU): the committed ncu traffic belongs to
the prox kernel's current code, a comment edit does not change the kernel's
digest, and the reference arm (the FP64 oracle on the host cores) prints one
JSON line with the contract's keys, from rank 0 only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_traffic_matches_the_kernel_code():
    """profiles/traffic.json was captured from the prox kernel as it is now,
    so bench.py reports its DRAM traffic instead of null.  A launch reads the
    occupancy bitmap of Omega and writes that of Omega+ (p^2 / 8 bytes each)
    at the least."""
    t = bench.profiled_traffic("tc_gemm_prox", bench.kernel_digest())
    assert t is not None and t > 40000 ** 2 / 4


def test_digest_ignores_comments_and_blank_space():
    code = "int f(int x) {\n  return x + 1;  // add one\n}\n"
    commented = "/* the successor */\nint f(int x) {\n\n  return x + 1;\n}\n"
    changed = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._code_only(code) == bench._code_only(commented)
    assert bench._code_only(code) != bench._code_only(changed)


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == "hubblock_p40000_n1000"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_profile_summaries_quote_commands_bench_accepts():
    """Every ncu summary under profiles/ names the command that produced it,
    and each bench.py command it quotes parses with today's bench.py."""
    import glob
    import re
    import shlex
    mds = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert mds
    for md in mds:
        txt = open(md).read()
        cmds = re.findall(r"python bench\.py([^`\n]*)", txt)
        assert cmds or "ncu" in txt, md
        assert "ncu " in txt and "--clock-control none" in txt, md
        for c in cmds:
            args = bench.parse(shlex.split(c.replace("\\", " ")))
            assert args.impl == "ours", (md, c)


def test_clock_sampler_parses_clocks_and_throttle_reasons(monkeypatch, tmp_path):
    """ClockSampler reads nvidia-smi's CSV: the median SM clock under load, the
    maximum clock, and every throttle reason seen Active ("Not Active" is not
    one).  Here a fake nvidia-smi on PATH prints the rows."""
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!/bin/sh\n"
        "echo '0, 1900, 2070, 1200.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
        "echo '0, 1800, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
        "echo '0, 2000, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
        "echo '0, [N/A], 2070, 900.0, 0x0, Not Active, Active, Not Active, Not Active'\n"
        "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    cs = bench.ClockSampler(0)
    cs.start()
    for _ in range(100):
        if os.path.getsize(cs.path) > 0 and open(cs.path).read().count("\n") >= 4:
            break
        time.sleep(0.05)
    got = cs.stop()
    assert got["samples"] == 4
    assert got["sm_mhz"] == 1900.0 and got["sm_max_mhz"] == 2070.0   # the N/A sample is skipped
    assert got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() is None
    assert not os.path.exists(cs.path)          # no temp file left behind


def test_refresh_cost_leg_alternates_and_reports_the_difference():
    """The refresh-cost leg alternates fits without and with the refresh of Y,
    ends on the default (so the caller's Omega buffer holds its estimate), and
    reports the median times and their difference."""
    calls = []

    class Stats:
        def __init__(self, yr):
            self.y_refreshes, self.iters, self.n_prox_gemm, self.kkt = (2, 41, 46, 9e-5) if yr else (0, 41, 45, 8e-5)

    class FakeLib:
        @staticmethod
        def accord_fit(X, lam, y_refresh, **kw):
            assert kw == {"precision": "mixed"} and lam == 0.1
            calls.append(y_refresh)
            return None, Stats(y_refresh)

    ms = {0: iter([300.0, 302.0, 301.0]), 32: iter([311.0, 309.0, 310.0])}

    def time_fit(fn):
        res = fn()
        return next(ms[calls[-1]]), res

    out = bench.refresh_cost_leg(FakeLib, "X", 0.1, {"precision": "mixed"}, 3, time_fit)
    assert calls == [0, 32] * 3
    assert out["fit_ms_with"] == 310.0 and out["fit_ms_without"] == 301.0 and out["cost_ms_per_fit"] == 9.0
    assert (out["refreshes_per_fit"], out["prox_launches_with"], out["prox_launches_without"]) == (2, 46, 45)
    assert out["fits_each"] == 3 and out["final_kkt_without"] == 8e-5
