"""The multi-rank path on the CPU: two gloo ranks each decode their contiguous
shard of a batch with the oracle, gather the outputs and sum the error counts;
the merged result equals the unsharded decode, and the timing reduction takes
the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

from paper_cs_0609090_gb300 import shard


def test_frame_range_partition():
    for F in (0, 1, 2, 7, 1000, 4097):
        for world in (1, 2, 3, 8):
            ranges = [shard.frame_range(F, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == F
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [e - s for s, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.frame_range(5, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_cs_0609090_gb300 import inputs as I
        w = I.make_workload("reg36_n1008", n_frames=37, ebn0_db=1.5)
        s, e = shard.frame_range(w.n_frames, world, rank)
        p = w.params
        o = oracle.decode_int(w.code, w.q0[s:e], form="ss_1bit", rule=p["rule"], offset=p["offset"],
                              msg_sat=p["msg_sat"], max_iter=p["max_iter"], early_stop=1)
        full = shard.gather_outputs({"bits": o.bits, "iters": o.iters, "ok": o.ok, "z": o.z}, w.n_frames)
        frame_err = int(np.any(o.bits != w.codewords[s:e], axis=1).sum())
        counts = shard.sum_counts([frame_err, e - s])
        t = shard.max_over_ranks([1.0 + rank, 5.0 - rank])
        if rank == 0:
            ref = oracle.decode_int(w.code, w.q0, form="ss_1bit", rule=p["rule"], offset=p["offset"],
                                    msg_sat=p["msg_sat"], max_iter=p["max_iter"], early_stop=1)
            ok = (np.array_equal(full["bits"], ref.bits) and np.array_equal(full["iters"], ref.iters)
                  and np.array_equal(full["ok"], ref.ok) and np.array_equal(full["z"], ref.z)
                  and counts[0] == int(np.any(ref.bits != w.codewords, axis=1).sum())
                  and counts[1] == w.n_frames and list(t) == [float(world), 5.0])
            open(result_path, "w").write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_unsharded(tmp_path):
    import torch.multiprocessing as mp
    path = str(tmp_path / "result")
    mp.start_processes(_rank_main, args=(2, _free_port(), path), nprocs=2, join=True, start_method="spawn")
    assert open(path).read() == "ok"
