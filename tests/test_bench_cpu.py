"""bench.py's accounting, on CPU: the models the roofline and the tensor
figures are computed from, pinned to what the GPU counters measured.

* tensor_stage_ops / 8192 is the number of mma.sync m16n8k32 instructions
  the tensor-core stages issue; ncu counted, for one large_dense product
  (profiles/ncu_tensor_stages_large_dense.md),
  sm__inst_executed_pipe_tensor_subpipe_imma = 3,145,728 (forward),
  18,874,368 (middle) and 3,145,680 (inverse).
* algorithmic_bytes: the DRAM bytes every pass must move; ncu's DRAM reads
  of the middle and inverse passes on two degree-262143 polynomials of
  1024-bit coefficients (profiles/traffic_huge_dense.md: 805.75 MB and
  422.41 MB) match the reads the model assigns them (2 r Y 2K words, r Y 2K
  words plus the inverse tiles' twiddle tables).
* stage_bits follows the radix split of the stage code (at most 4 bits a
  stage, as even as possible, larger stages first).
"""
import pytest

import bench
import paper_1612_05778_gb300 as ipm


@pytest.fixture(scope="module")
def large_dense_info():
    return ipm.choose(32768, 32768, 4096, 4096, K=128)


def test_tensor_stage_model_matches_imma_counter(large_dense_info):
    ops = bench.tensor_stage_ops(large_dense_info, 32768, 32768)
    assert [o // 8192 for o in ops] == [3145728, 18874368, 3145680]
    assert all(o % 8192 == 0 for o in ops)


def test_algorithmic_bytes_match_measured_reads():
    I = ipm.choose(262144, 262144, 1024, 1024, K=32, s=4)
    fwd, mid, inv = bench.algorithmic_bytes(I)
    z = I["r"] * I["Y"] * 2 * I["K"] * 4
    assert mid == 3 * z
    # measured DRAM reads: the middle pass reads both operands' transforms,
    # the inverse pass the product's (and its tiles' twiddle tables)
    assert abs(805.747456e6 - 2 * z) / (2 * z) < 0.002
    assert 0 <= (422.409728e6 - z) / z < 0.08
    assert fwd > 2 * z and inv > z


@pytest.mark.parametrize("logL,want", [(0, []), (1, [1]), (4, [4]), (5, [3, 2]), (7, [4, 3]), (8, [4, 4]),
                                       (9, [3, 3, 3]), (11, [4, 4, 3]), (12, [4, 4, 4]), (21, [4, 4, 4, 3, 3, 3])])
def test_stage_bits(logL, want):
    assert bench.stage_bits(logL) == want
    assert sum(want) == logL


@pytest.mark.parametrize("workload", ["taylor", "paper_table", "families"])
def test_single_gpu_workloads_leave_other_ranks_idle(workload, monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--workload", workload, "--gpus", "2"]) == 0


def test_schedule_bytes_are_eight_slabs_plus_io(large_dense_info):
    """The method's three-pass schedule moves in + out + 8R, R = r Y K 4
    bytes (K1 writes 2R, K2 reads 2R and writes 2R, K3 reads 2R); this
    implementation moves in + out + 12R (both x halves of both operands
    leave the first pass)."""
    I = large_dense_info
    R = I["r"] * I["Y"] * I["K"] * 4
    inp, out = bench.io_bytes(I)
    s = bench.schedule_bytes(I)
    a = bench.algorithmic_bytes(I)
    assert s == [inp + 2 * R, 4 * R, 2 * R + out]
    assert sum(s) == inp + out + 8 * R and sum(a) == inp + out + 12 * R
    assert abs(sum(s) - 0.906e9) / 0.906e9 < 0.01  # 0.91 GB for d = 32768, 4096-bit


def test_both_arms_print_the_same_config():
    """The reference arm (the oracle, on a bounded sample) and our arm build
    `config` from the same function, so the driver sees one workload."""
    import io
    import json
    from contextlib import redirect_stdout
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.main(["--impl", "reference", "--workload", "small_dense", "--steps", "1", "--warmup", "0"]) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    name, sh, _, _ = bench.workload("small_dense")
    assert line["config"] == bench.workload_config(name, sh)
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
