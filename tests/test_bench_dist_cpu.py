"""Host logic of bench.py for N > 1 ranks, on two CPU processes over gloo:
each rank gets its own independent job (no data-path collective), the timed
region is closed by a barrier, the job time is the maximum over ranks and the
throughput counts the LED updates of all ranks."""

import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), FPM_BENCH_BACKEND="gloo")
    import bench
    w, r, local, pg = bench.dist_setup()
    c, nominal, truth = bench.workload(seed_shift=r)
    sched = bench.full_batches(c.n_leds, c.B, 20, c.seed)
    bench.barrier(pg)
    t_rank = 1.0 + r                                    # stands in for this rank's timed region
    t_max = bench.allreduce_max(pg, t_rank, "cpu")
    bench.barrier(pg)
    value = w * 20 * c.B / t_max                        # the formula of the engine arm
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump(dict(world=w, rank=r, seed=c.seed, t_max=t_max, value=value,
                       first=sched[0].tolist(), leds=int(c.n_leds), B=int(c.B)), fh)
    pg.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [x["world"] for x in res] == [2, 2]
    assert res[0]["seed"] != res[1]["seed"]             # independent jobs
    assert res[0]["t_max"] == res[1]["t_max"] == 2.0    # max over ranks, seen by every rank
    assert res[0]["value"] == pytest.approx(2 * 20 * res[0]["B"] / 2.0)
    for x in res:                                       # each rank's batches are valid schedules
        b = np.array(x["first"])
        assert len(set(b.tolist())) == x["B"] and b.min() >= 0 and b.max() < x["leds"]


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse_args(["--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"])
    bench.reference_arm(args)
    assert capsys.readouterr().out == ""
