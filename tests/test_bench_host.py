"""bench.py's host arithmetic without a GPU: the roofline records of the
circuit kernel (useful flops against the derived FP32 peak, warp instructions
against the derived issue peak), the update's algorithmic bytes, and the
launches counted per generation."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1809_11134_gb300 import workloads as W  # noqa: E402


def test_circuit_roofline_and_issue_rate():
    searches = W.config(2)
    pk = {"hbm_gbs": 6802.0, "sm_max_mhz": 2070.0}
    roof = bench.roofline("circuits", 0.025, 13.5e6, searches, pk, traffic=41.5e6)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["peak"] - peak) < 1e-9
    assert abs(roof["achieved"] - 13.5e6 / 25e-6 / 1e12) < 1e-12
    assert abs(roof["frac"] - roof["achieved"] / peak) < 1e-12
    assert roof["traffic"] == 41.5e6
    iss = bench.issue_roofline(roof, 11330413)
    assert abs(iss["peak"] - 152 * 4 * 2.07) < 1e-9
    assert abs(iss["achieved_ginst_per_s"] - 11330413 / 25e-6 / 1e9) < 1e-6
    assert 0 < iss["frac"] < 1
    assert bench.issue_roofline(roof, None)["frac"] is None


def test_update_bytes_counts_slots_segments_and_mutations():
    s = W.Search(3, 4, 8, W.LIB_NCV | W.LIB_HT, W.cknot(3), p_mutation=0.5)
    sid = np.arange(32, dtype=np.uint32).reshape(8, 4)
    sid[1, 0] = sid[0, 0]  # one segment used by two slots
    R = 3 * 2 + 3
    got = bench.update_bytes([s], [{"seg_id": sid}])
    want = 32 * 8 + 31 * (32 + 32 + 4) + 0.5 * 8 * R * 4 * (32 + 32 + 4 + 4)
    assert got == want


def test_launches_per_generation():
    # one circuit kernel group, two update roles, selection, one rescoring
    # width, sort, finish
    assert bench.launches_per_generation(W.config(2)) == 7
    # three widths and one binary64 group: four circuit kernels, three rescoring widths
    mixed = W.config(4)[:40] + [W.Search(3, 5, 64, W.LIB_NCV, W.cknot(3), precision=W.PREC_FP64)]
    widths = len(set(s.n for s in mixed if s.precision != W.PREC_FP64))
    groups = len(set((s.n, s.precision == W.PREC_FP64) for s in mixed))
    assert bench.launches_per_generation(mixed) == groups + 2 + 1 + widths + 1 + 1


def test_rank_count_must_match_gpus():
    """Under a launcher, --gpus must equal the launched world size (a silent
    single-process run of --gpus 8 would report n_gpus 1)."""
    import subprocess
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "1",
                        "--impl", "reference", "--steps", "1"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode != 0 and "launcher started 2 ranks" in r.stderr


def test_oracle_generation_threads_match_the_oracle_step():
    """The threaded generation of the CPU baseline computes what the oracle's
    own generation step computes (same state afterwards)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    s = W.config(2)[0]
    p = oracle.make_problem(s.n, s.L, 300, s.library, s.perm, seed=s.seed)
    a = oracle.init_state(p)
    b = tuple(x.copy() for x in a)
    rep = oracle.new_report()
    with ThreadPoolExecutor(4) as pool:
        for g in range(3):
            bench.oracle_generation(oracle, p, a, g, pool)
            oracle.step(p, *b, g, 32, rep)
    for x, y in zip(a, b):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))


def test_by_qubits_table():
    """the flat n = 3/4/5 table is read off the per-set results, binary32
    against plain binary64, and tolerates a missing arithmetic"""
    def r(k, g):
        return {"circuit_kernel_circuits_per_s": k, "generation_circuits_per_s": g}
    pc = {"config2": {"fp32": r(600.0, 300.0), "fp64": r(90.0, 75.0)},
          "config3": {"fp32": r(290.0, 140.0), "fp64": r(14.0, 14.0)},
          "config5": {"fp32": r(87.0, 50.0)},
          "config4": {"fp32": r(230.0, 100.0)}}
    t = bench.by_qubits(pc)
    assert sorted(t) == ["3", "4", "5"]
    assert t["3"] == {"fp32_circuit_kernel": 600.0, "fp32_generation": 300.0,
                      "fp64_circuit_kernel": 90.0, "fp64_generation": 75.0,
                      "fp32_over_fp64_generation": 4.0}
    assert t["4"]["fp32_over_fp64_generation"] == 10.0
    assert t["5"] == {"fp32_circuit_kernel": 87.0, "fp32_generation": 50.0}
