"""Host-side logic of bench.py on the CPU: the max over ranks of the timed
region with two gloo ranks (the N > 1 replicas path), the reference arm's
non-zero ranks, the work count of a V-cycle and the kernel-source fingerprint
that keys the recorded ncu traffic."""
import os
import shutil
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_max(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.barrier_max(values[rank], world, "cpu")
    finally:
        dist.destroy_process_group()


def test_barrier_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    out = mp.Manager().dict()
    values = [3.25, 3.5]
    port = _free_port()
    procs = [mp.Process(target=_rank_max, args=(r, 2, port, values, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == 3.5


def test_barrier_max_single_rank_is_identity():
    assert bench.barrier_max(1.25, 1, "cpu") == 1.25


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        workload, steps, warmup = "c2", 2, 3
    assert bench.run_reference(A(), bench.WORKLOADS["c2"], 2, 1) == 0
    assert capsys.readouterr().out == ""


def test_dof_sweeps_per_vcycle():
    # 64x64 elements, P{3-2-1-0}, I{5-10-20-40}: 4 E sum_l N_l s_l with
    # s_l = 2 n_l above the coarsest level and n_L on it
    E = 64 * 64
    assert bench.dof_sweeps_per_vcycle(E, [3, 2, 1, 0], [5, 10, 20, 40]) == 4 * E * (16 * 10 + 9 * 20 + 4 * 40 + 1 * 40)


def test_fingerprint_ignores_comments_and_blank_space(tmp_path):
    src = os.path.join(ROOT, "paper_1908_03972_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    ref = bench.csrc_fingerprint(str(dst))
    assert ref == bench.csrc_fingerprint(src)
    f = dst / "k_fused.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n\n" + text.replace(";\n", ";   /* trailing */\n", 3))
    assert bench.csrc_fingerprint(str(dst)) == ref
    f.write_text(text.replace("namespace pmg {", "namespace pmg {\nconstexpr int kProbe = 1;", 1))
    assert bench.csrc_fingerprint(str(dst)) != ref
    (dst / "api.cu").write_text("host code changes do not count\n")
    (dst / "k_blocks.cu").write_text("nor do kernels whose counters are not recorded\n")
    f.write_text(text)
    assert bench.csrc_fingerprint(str(dst)) == ref
