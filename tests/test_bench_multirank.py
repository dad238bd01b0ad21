"""The multi-rank (replicas) path of bench.py on the CPU: two gloo ranks.
Each rank advances its own replica, the job time is the slowest rank's, the
job's ns/day is the sum over ranks, each rank builds its own seeded
replica, and the reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 17.25][rank]
    out[rank] = bench.max_over_ranks(local_ms, world, "cpu")
    d, _ = bench.make_workload("c0", rank)
    out[10 + rank] = float(np.asarray(d["pos"]).sum())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_replicas():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 17.25
    assert out[10] != out[11]          # the replicas are different seeded systems
    one = bench.weak_scaling_ns_day(0.001, 0.15, 1)
    assert bench.weak_scaling_ns_day(0.001, 0.15, 2) == pytest.approx(2 * one)
    assert one == pytest.approx(0.001 * 1e-3 * 86400.0 / 0.15e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "c0"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""


def test_reference_arm_line_carries_the_contract_keys(monkeypatch, capsys):
    import json
    import sys
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "c0",
                                      "--steps", "1", "--warmup", "0"])
    bench.run_reference(bench.parse())
    lines = [l for l in capsys.readouterr().out.split("\n") if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in rec, k
    assert rec["impl"] == "reference" and rec["unit"] == "ns/day" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["cpu_baseline"]["cores"] >= 1
    assert rec["e2e"] == {"value": rec["value"], "unit": "ns/day", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    # the driver's K and W are honoured, and the workload is described exactly
    # as in the GPU arm's line
    assert rec["steps"] == 1 and rec["warmup"] == 0
    assert rec["config"] == bench.run_config(*bench.make_workload("c0", 0))


def test_output_errors_of_the_oracle_against_itself_vanish():
    from oracle import reference as R
    from paper_2608_12691_b300 import systems as S
    d = S.make_c0()
    lam = 0.6
    _, _, res = bench.oracle_timed(d, 2, 1)
    E, F0, Fuv, Fs, Ub, Fb = res
    hA, hB, dA, dB = R.switching(lam)
    terms = {"U": E["U_vv"] + E["U_uu"] + hA * E["U_uv"] + hB * E["U_soft"] + Ub,
             "dUdl": dA * E["U_uv"] + dB * E["U_soft"], "U_vv": E["U_vv"], "U_uu": E["U_uu"],
             "U_uv": E["U_uv"], "U_soft": E["U_soft"], "U_bonded": Ub}
    F = F0 + hA * Fuv + hB * Fs + Fb
    out = bench.output_errors(terms, F, res, lam, d["solute"])
    assert out["F_rel_rms"] == 0.0 and out["F_rel_rms_solute"] == 0.0 and out["F_max_over_rms"] == 0.0
    assert all(out[k]["abs"] == 0.0 for k in terms)
    # a perturbed solute force shows in the solute norm far more than in the total
    F2 = F.copy()
    F2[np.flatnonzero(d["solute"])[0]] *= 1.0 + 1e-4
    out2 = bench.output_errors(terms, F2, res, lam, d["solute"])
    assert out2["F_rel_rms_solute"] > 2 * out2["F_rel_rms"] > 0
