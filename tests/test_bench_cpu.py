"""bench.py's host-side contract, on the CPU: the reference arm (the FP64 oracle on the host cores)
prints exactly one JSON line carrying the fields of the benchmark contract, and under a
multi-rank launch only rank 0 works and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=900)


def json_lines(out):
    return [json.loads(line) for line in out.splitlines() if line.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    """About 30 s of oracle time (the arm sizes its sample to that)."""
    r = run_bench({}, "--steps", "3", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1, r.stdout
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("spinodal decomposition 4096x4096")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--gpus", "2", "--steps", "3",
                  "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    assert json_lines(r.stdout) == []


def test_kernel_choices_name_library_variants():
    """bench.py --kernel maps each choice to a step kernel the C ABI declares, with that kernel's
    default tile, and the ncu traffic of the 16-bit and FP32 steps is keyed on different sources."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1803_11345_gb300 import build
    build.build()
    from paper_1803_11345_gb300 import lbm
    variants = {name: spec[0](lbm) for name, spec in bench.KERNELS.items()}
    assert variants == {"generic": lbm.LBM_KERNEL_GENERIC, "pair": lbm.LBM_KERNEL_PAIR,
                        "pair_staged": lbm.LBM_KERNEL_PAIR_STAGED}
    assert bench.KERNELS["pair"][1:3] == (128, 1) and bench.KERNELS["pair_staged"][1:3] == (128, 1)
    assert bench.kernel_source_hash("fp16s") != bench.kernel_source_hash("fp32")
