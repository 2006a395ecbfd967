"""bench.py on the CPU.  The reference arm (the FP64 oracle timed on this
host's cores) prints one JSON line with the keys of the benchmark contract,
and ranks other than 0 exit quietly (the line is printed once per job).  The
clock sampler of the timed region parses nvidia-smi's samples (a stand-in
script here)."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
       "--warmup", "0", "--n", "2048"]


def _env(**kw):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(kw)
    return env


def test_reference_arm_prints_the_contract_line():
    res = subprocess.run(CMD, capture_output=True, text=True, timeout=300, env=_env(), cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "blob-pair interactions/s" and d["unit"] == "pairs/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 0)
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "workload" in d["config"] and d["config"]["n_blobs"] == 2048
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and "targets" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    res = subprocess.run(CMD, capture_output=True, text=True, timeout=120,
                         env=_env(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"), cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    assert not [ln for ln in res.stdout.splitlines() if ln.startswith("{")]


FAKE_SMI = """#!/bin/sh
# stands in for nvidia-smi --query-gpu=... --format=csv,noheader,nounits -lms 200
echo "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "0, 1980, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
exec sleep 30
"""


def test_clock_sampler_reads_nvidia_smi_samples(tmp_path, monkeypatch):
    """The clock record of the timed region: median SM clock, maximum, and the
    throttle reasons seen, parsed from nvidia-smi's CSV samples."""
    import bench

    smi = tmp_path / "nvidia-smi"
    smi.write_text(FAKE_SMI)
    smi.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    for path in (str(tmp_path / "out" / "clocks.csv"), None):
        s = bench.ClockSampler(0, path)
        s.start()
        deadline = time.time() + 10
        while time.time() < deadline:
            if os.path.exists(s.path) and open(s.path).read().count("\n") >= 3:
                break
            time.sleep(0.05)
        rec = s.stop()
        assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                       "samples": 3}
        assert os.path.exists(s.path)
        if path is None:
            os.remove(s.path)


def test_accuracy_and_flop_helpers():
    """The matvec accuracy figures compare against the oracle rows as stated,
    and the setup flop count is n^3 per body of n = 3 n_p rows (Cholesky,
    inverse factor and inverse product, n^3 / 3 each)."""
    import numpy as np

    import bench

    ref = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    got = ref + np.array([[0.0, 1e-6, 0.0], [0.0, 0.0, 0.0]])
    c = bench.compare_rows(got, ref)
    assert c["rows"] == 2
    assert abs(c["rel_l2_vs_oracle"] - 1e-6 / np.sqrt(5.0)) < 1e-15
    assert abs(c["max_abs_vs_oracle"] - 1e-6) < 1e-18
    assert abs(c["max_abs_over_max_ref"] - 0.5e-6) < 1e-18
    f = bench.setup_flops([162, 162])
    assert f["total"] == 2 * 486.0 ** 3 and f["cholesky"] == 2 * 486.0 ** 3 / 3.0


def test_serving_requests_from_the_process_pool_equal_direct_ones():
    """Serving requests generated by the spawned pool are the seeded
    requests themselves."""
    import numpy as np

    import bench
    from paper_1602_02170_gb300 import inputs as I

    seeds = list(range(500, 520))
    pooled = bench._gen_requests(seeds)
    for sd, s in zip(seeds[:4], pooled[:4]):
        d = I.config_serving_request(sd)
        for k in ("q", "theta", "blob_start", "rho", "F", "T"):
            np.testing.assert_array_equal(getattr(s, k), getattr(d, k))
