"""The benchmark's reference arm (the oracle timed on the host cores) runs
without a GPU and prints one JSON line with the keys the benchmark contract
names, on the same metric and unit as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    line = json.loads(lines[-1])
    assert line["impl"] == "reference"
    import bench
    assert line["metric"] == bench.METRIC and line["unit"] == "frames/s"    # the native arm's string
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["cpu_model"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("1080p")


def test_roofline_kernel_follows_the_tuned_full_search_form():
    """The bench's roofline names the kernel of the full-search form the tuner
    chose for the step (read from its record), with a DRAM traffic constant
    for each pipelined kernel it may pick."""
    import bench
    log = ("fsbm 1920x1088 16x16 p=32 K=59 tuned: model=pipe T=13 chosen=pipetab B=12 | "
           "pipe T=13 8.3412 ms | pipetab B=12 7.8221 ms | group T=13 G=32 thr=256 9.4666 ms")
    t = bench.parse_tune_log(log)
    assert len(t) == 1 and t[0]["shape"] == "fsbm 1920x1088 16x16 p=32 K=59"
    assert t[0]["chosen"] == "pipetab B=12" and t[0]["ms"]["pipe T=13"] == 8.3412
    kern = {name: next(k for pre, k in bench.FSBM_FORM_KERNEL if name.startswith(pre))
            for name in t[0]["ms"]}
    assert kern == {"pipe T=13": "k_fsbm_pipe", "pipetab B=12": "k_fsbm_pipe_tab",
                    "group T=13 G=32 thr=256": "k_fsbm_seq"}
    for k in ("k_fsbm_pipe", "k_fsbm_pipe_tab"):
        assert bench.FSBM_SEQ_DRAM_BYTES_PER_FRAME[k] * 13 > 27e6
