"""The benchmark's JSON contract on the host: the reference arm (the FP64
oracle timed on every host core, one worker process per core) prints one line
with the keys the native arm also carries, and its rank > 0 processes print
nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600,
                         check=True).stdout.strip().splitlines()
    lines = [json.loads(x) for x in out if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "SBIM mode-history MACs/s"
    assert d["unit"] == "MAC/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_are_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT="29581")
    r = subprocess.run([sys.executable, "-c",
                        "import bench, sys; sys.argv = ['bench.py', '--impl', 'reference']; "
                        "a = bench.parse(); a.warmup = 3; "
                        "bench.dist_setup = lambda args: (2, 1, 1); bench.run_reference(a)"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120, check=True)
    assert r.stdout.strip() == ""


def test_tpv3_workload_uses_the_papers_parameters():
    """tests/golden/tpv3_parameters.txt holds the TPV3 values Section 3 prints;
    the benchmark's TPV3 and coupled workloads take theirs from bench.TPV3."""
    import bench
    golden = {}
    with open(os.path.join(ROOT, "tests", "golden", "tpv3_parameters.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (x.strip() for x in line.split("="))
                golden[k] = float(v)
    assert set(golden) == set(bench.TPV3)
    for k, v in golden.items():
        assert bench.TPV3[k] == v, k
    import numpy as np
    x = np.array([0.0, 1000.0, 1600.0, 14000.0, 16000.0])
    X1, X3 = np.meshgrid(x, np.zeros(1))
    mu_s, tau0, mu_k, Dc, sigma0 = bench.tpv3_law(X1, X3)
    assert list(mu_s[0]) == [0.677, 0.677, 0.677, 0.677, bench.TPV3_UNBREAKABLE_MU_S]
    assert tau0[0, 0] == tau0[0, 1] > 0.677 * 120e6 and tau0[0, 2] == 70e6
    assert (mu_k, Dc, sigma0) == (0.525, 0.4, 120e6)


def test_oracle_pool_adds_up_its_workers():
    """Two spawned oracle workers on disjoint mode samples: the aggregate rate is
    all MACs over the slower worker's time."""
    import bench
    c = dict(bench.config_large(), n1=32, n3=32, L1=3200.0, L3=3200.0, n_cut=64)
    pool = bench.OraclePool(c, 2, 16, seed=1)
    try:
        rate, secs = pool.run(min_reps=3)
    finally:
        pool.close()
    assert rate > 0 and secs > 0
    assert rate >= 2 * 16 * 64 * bench.MACS_PER_PAIR * 3 / secs * (1 - 1e-9)
