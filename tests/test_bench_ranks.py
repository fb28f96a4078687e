"""The bench's multi-rank logic on CPU: world size 2 over gloo, replicas with no
data-path collective, the job time is the slowest rank's, the rate counts all replicas."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(torch, 1.0 + rank, "cpu")
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.0
    import bench
    assert bench.aggregate_rate(2, 128000, 10, 2.0) == pytest.approx(2 * 128000 * 10 / 2.0)
    assert bench.max_over_ranks(torch, 3.5, "cpu") == 3.5      # single process: unchanged


def test_roofline_line_from_stage_events():
    """The roofline entry divides the algorithmic work of one launch (the per-atom count
    times the compacted atoms) by the CUDA-event average of the timed launches; the entry for
    the kernel alone does the same with the per-stage pass's average."""
    import bench
    from paper_2505_12958_gb300.workload import ace_contract_flops_per_atom
    atoms = list(range(1000))
    prof = {"ace": (2.5, 5)}                          # 5 launches, 0.5 ms each
    r = bench.ace_kernel_roofline(prof, 5, None, {"sm_max_mhz": 2000.0}, "test", atoms, fma_peak=80.0,
                                  alone_ms=0.4)
    flops = ace_contract_flops_per_atom() * 1000
    assert r["algorithmic_flops_per_launch"] == flops and r["timed_launches"] == 5
    assert abs(r["achieved"] - flops / 0.5e-3 / 1e12) < 1e-9 and abs(r["frac"] - r["achieved"] / 80.0) < 1e-12
    assert abs(r["alone"]["achieved"] - flops / 0.4e-3 / 1e12) < 1e-9
    assert r["alone"]["frac"] > r["frac"]
    assert r["peak"] == 80.0 and abs(r["peak_derived_unit_count"] - 152 * 128 * 2 * 2.0e9 / 1e12) < 1e-9
    assert bench.ace_kernel_roofline(prof, 5, None, {}, "test", atoms, fma_peak=80.0)["alone"] is None
    # the split by pipe: FP32-lane work against the FP32 peak, tensor-core products against the
    # TF32 peak (measured BF16 x 1.1 / 2.25)
    from paper_2505_12958_gb300.workload import ace_tc_contract_work
    w = ace_tc_contract_work()
    r = bench.ace_kernel_roofline(prof, 5, None, {"bf16_tflops": 2000.0}, "test", atoms, fma_peak=80.0)
    assert abs(r["fp32_lanes"]["achieved"] - w["fp32"] * 1000 / 0.5e-3 / 1e12) < 1e-9
    assert abs(r["tensor"]["peak"] - 2000.0 * 1.1 / 2.25) < 1e-9
    assert abs(r["tensor"]["frac_executed"] - w["tensor_executed"] * 1000 / 0.5e-3 / 1e12 / r["tensor"]["peak"]) < 1e-12


def test_eam_roofline_from_stage_times():
    """The EAM entry divides the passes' minimum HBM bytes (the per-atom model at the mean list
    length, counted here by brute force on a small periodic cell) by their per-stage times."""
    import numpy as np

    import bench
    import synth
    from paper_2505_12958_gb300.workload import eam_bytes_per_atom
    c = synth.configs.w_bulk(ncell=6)                 # 432 atoms, 19 A periodic box
    x = c["x"]
    L = np.asarray(c["box"]["h"]).reshape(3, 3)[0, 0]
    rc = max(max(c["eam"]["phi_d"]), max(c["eam"]["rho_d"]), c["ace"]["rc"]) + 1.0
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.round(d / L)                          # periodic in all three directions
    cnt = (np.linalg.norm(d, axis=2) < rc).sum(axis=1) - 1
    r = bench.eam_roofline({"eam_density": 0.01, "eam_force": 0.03}, c, {"hbm_gbs": 5000.0}, "test")
    assert abs(r["mean_list_length"] - cnt.mean()) < 1e-9
    assert abs(r["algorithmic_bytes_per_step"] - len(x) * eam_bytes_per_atom(cnt.mean())) < 1e-6
    assert abs(r["achieved"] - r["algorithmic_bytes_per_step"] / 0.04e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12 and r["unit"] == "GB/s"
