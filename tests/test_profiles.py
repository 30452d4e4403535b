"""The committed ncu summaries under profiles/ belong to the current sweep
kernel: bench.py reports a capture's DRAM traffic only while the hash of the
sweep's sources equals the one recorded in the summary, so a kernel change
without a fresh capture shows up here (and as traffic = null in the bench
line). Also checks the algorithmic op counts the roofline divides by."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sweep_profiles_match_current_sources():
    for name in ("sweep_kernel_L65536.md", "sweep_kernel_general_L65536.md"):
        traffic = bench.measured_traffic(65536, name)
        assert traffic is not None, f"profiles/{name} was captured on other sources"
        # one bit read and one written per site: the capture's DRAM bytes are
        # at least the algorithmic bytes and within a small factor of them
        alg = 0.25 * 65536 ** 2
        assert alg <= traffic <= 1.5 * alg


def test_profiles_name_their_commands():
    for name in os.listdir(os.path.join(ROOT, "profiles")):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert "--clock-control none" in txt, name
        assert "python " in txt, name


def test_algorithmic_op_counts():
    # p = 1: 19 three-input ops per round and 32-cell word, 20 Philox xors per
    # 128 random bits at 2 bits per attempt, one funnel shift per staged word
    assert bench.K_ALG_ALU == 19 / 32 + 20 / 64 + 1 / 32 == 0.9375
    # general rates: 30 ops per round and word plus the acceptance bits
    extra = bench.K_ALG_ALU_GENERAL - (30 / 32 + 20 / 64 + 1 / 32)
    assert abs(extra - bench.C_CAND * 2 * (20 / 128 + 2 / 32)) < 1e-12
