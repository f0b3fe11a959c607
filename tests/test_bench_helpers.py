"""CPU checks of bench.py's helpers: the Table 1 fixture reader, the symmetry
images used to compare a found sequence with Table 1's, the work unit of the
roofline accounting, the size of the oracle's timed sample and the JSON line
of the reference arm (the oracle, which needs no GPU)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_table1_rows_read_the_fixture():
    rows = bench.table1_rows()
    assert len(rows) == 17
    assert rows[171][0] == 1669 and rows[247][0] == 3259 and rows[247][2] == 13.0


def test_symmetry_images_keep_energy_and_skew_symmetry(oracle_mod):
    import paper_2210_15962_gb300 as m
    for L, (E, _, _, hx) in bench.table1_rows().items():
        s = m.from_hex(hx, L)
        imgs = bench.symmetry_orbit(s)
        assert len(imgs) == 8 and any(np.array_equal(i, s) for i in imgs)
        D = (L + 1) // 2
        for i in imgs:
            assert oracle_mod.energy(i) == E
            assert np.array_equal(oracle_mod.skew_expand(i[:D], L), i)  # still skew-symmetric
        assert len({i.tobytes() for i in imgs}) >= 4


def test_roofline_unit_counts_the_lags_of_each_space():
    # 4 LOP3 per 32 lags and digit plane: (L-1)/2 even lags of a skew sequence, L-1 lags in the full space
    assert bench.core_alu_ops_per_eval(121, 5.0) == 4.0 * 5.0 * 60 / 32
    assert bench.core_alu_ops_per_eval(121, 5.0, full=True) == 4.0 * 5.0 * 120 / 32


def test_popcount_count_of_the_skew_scan():
    # counted by hand: L=5 (D=3) has one one-sided word at flips 0 and 2 and
    # none at flip 1 (its only y lag is its own mirror pair); at L=27 (one
    # word) every flip has a valid lag and flips 2..12 have both sides
    assert bench.popc_words_per_step(5) == (2, 0)
    assert bench.popc_words_per_step(27) == (14, 11)
    # per evaluation: TP counts per word with lags + 2 per two-sided word
    assert bench.popc_needed(27, 14, 5) == 5 * 14 + 2 * 11
    # the walk kernel's ncu profile at L=121 (5.0 digit planes) counted 11.5
    # POPC per warp-flip; the formulation's count is within 1% of it
    per_eval = bench.popc_needed(121, 61 * 1000, 5 * 1000) / (61 * 1000)
    assert abs(per_eval - 11.5) / 11.5 < 0.01
    assert abs(bench.popc_peak_tops() - 152 * 16 * 2.07e9 / 1e12) < 1e-9


def test_cpu_sample_is_bounded_and_whole_per_core():
    def work(n, L, wl, full=False):
        flips = L if full else (L + 1) // 2
        lags = L - 1 if full else (L - 1) // 2
        return n * wl * (flips * lags + bench.CPU_STEP_OVERHEAD)
    target = bench.CPU_SAMPLE_LAG_UPDATES
    for L, wl, cores, full in [(121, 8192, 16, False), (27, 4096, 16, False), (449, 16384, 16, False),
                               (128, 2048, 8, True), (64, 4096, 12, True)]:
        n = bench.cpu_sample_walks(L, wl, cores, full)
        assert n % cores == 0 and n >= cores
        # just enough whole walks per core to reach the target work
        assert work(n, L, wl, full) >= target or n == cores
        assert work(n - cores, L, wl, full) < target
    assert 16 * 16 <= bench.cpu_sample_walks(121, 8192, 16) <= 64 * 16  # ~13 s of oracle work
    assert bench.cpu_sample_walks(449, 10 ** 7, 16) == 16               # one walk per core at least
    assert bench.cpu_sample_walks(27, 4096, 16, total_walks=64) == 64   # never more than the workload


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-walks", "4"], capture_output=True, text=True, check=True,
                         cwd=ROOT, timeout=600).stdout
    lines = [x for x in out.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "neighbour_evals_per_s" and d["unit"] == "neighbour_evals/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["config"]["workload"] == "plain_L121_131072x8192_budget1e11"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "4 of the 131072" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_cpu_baseline_reports_all_cores_and_one_core():
    cores = os.cpu_count() or 1
    cb = bench.cpu_baseline(n_walks=8 * cores, walk_len=256, L=27, total_walks=64 * cores, one_core=True)
    assert cb["kind"] == "oracle" and cb["unit"] == "neighbour_evals/s" and cb["cores"] == cores
    assert cb["value"] > 0 and ("%d of the %d walks" % (8 * cores, 64 * cores)) in cb["sample"]
    assert cb["one_core"]["value"] > 0 and cb["one_core"]["sample"].startswith("1 walks")
