"""Host-side logic of bench.py that shapes the reported roofline (no GPU).

The roofline's numerator sums the oracle's word-op counts over the width
classes of the measured launch, so bench.py's class table must be the
engine's, and the per-launch sum must take exactly the classes in range.
"""
import json
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def engine_class_widths():
    """Padded words per row of each width class, read from the CUDA source."""
    src = open(os.path.join(ROOT, "paper_2212_01473_gb300", "csrc", "mce_internal.cuh")).read()
    body = re.search(r"constexpr int class_wp\(int c\) \{(.*?)\}", src, re.S).group(1)
    n = int(re.search(r"constexpr int kNumClasses = (\d+);", src).group(1))
    pairs = {int(c): int(w) for c, w in re.findall(r"c == (\d+) \? (\d+)", body)}
    last = int(re.search(r": (\d+);", body).group(1))
    return [pairs.get(c, last) for c in range(n)]


def test_bench_width_classes_are_the_engines():
    assert bench.WP_CLASSES == engine_class_widths()


def test_wp_of_words_picks_the_narrowest_class_that_fits():
    assert [bench.wp_of_words(w) for w in (1, 2, 3, 4, 5, 12, 13, 20, 21, 132)] == [1, 2, 4, 4, 12, 12, 20, 20, 28, 132]
    assert bench.wp_of_words(133) is None


def test_launch_word_ops_takes_the_classes_in_range():
    by_w = {"0": 5, "1": 1, "2": 2, "3": 4, "4": 8, "5": 16, "12": 32, "13": 64}
    # one launch for every one-warp class (widths 1..12); W = 0 roots never launch
    assert bench.launch_word_ops(by_w, 1, 12) == 1 + 2 + 4 + 8 + 16 + 32
    assert bench.launch_word_ops(by_w, 12, 12) == 16 + 32
    assert bench.launch_word_ops(by_w, 4, 4) == 4 + 8
    assert bench.launch_word_ops(by_w, 20, 20) == 64


def test_chunglu_1m_golden_covers_the_merged_launch():
    # every root of chunglu_1m with later neighbours has |P0| <= 340 (the
    # degeneracy), i.e. at most 11 words: all of it is the one-warp launch
    with open(os.path.join(ROOT, "tests", "golden", "chunglu_1m.json")) as f:
        gold = json.load(f)
    by_w = gold["word_ops_by_W"]
    assert max(int(w) for w, v in by_w.items() if v) <= (gold["degeneracy"] + 31) // 32
    total = sum(v for w, v in by_w.items() if int(w) > 0)
    assert total == gold["word_ops"]
    assert bench.launch_word_ops(by_w, 1, 12) == total


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference times the CPU oracle and prints one JSON line
    # with the keys the benchmark contract names (run here on a small graph)
    import subprocess
    import sys
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "er_2000", "--cpu-sample", "0.5"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "maximal cliques/sec" and d["value"] > 0
    assert d["config"]["workload"] == "er_2000"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


class MCEError(RuntimeError):
    """Stands in for the engine's error type (bench.py matches it by name)."""


def test_one_gpu_run_measures_once_more_after_an_engine_error(monkeypatch):
    calls = []

    def fake_run_ours(args):
        calls.append(getattr(args, "retried_after", None))
        if len(calls) == 1:
            raise MCEError("MCE_ETIMEOUT: a wait gave up")
        return 0

    monkeypatch.setattr(bench, "run_ours", fake_run_ours)
    monkeypatch.setattr(bench.sys, "argv", ["bench.py"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main() == 0
    # the second measurement knows which error it follows, for its line
    assert calls == [None, "MCEError: MCE_ETIMEOUT: a wait gave up"]


def test_other_errors_are_not_retried(monkeypatch):
    def fake_run_ours(args):
        raise ValueError("not an engine error")

    monkeypatch.setattr(bench, "run_ours", fake_run_ours)
    monkeypatch.setattr(bench.sys, "argv", ["bench.py"])
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    try:
        bench.main()
    except ValueError:
        pass
    else:
        raise AssertionError("a non-engine error must propagate")
