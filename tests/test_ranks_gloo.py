"""The multi-rank path on the host: the pattern split, the CSR slices each
rank matches, the max-over-ranks timing and the rank gating of the bench's
reference arm, with two gloo ranks on CPU.  The per-pattern work on each rank
is the oracle's match, standing in for the GPU call it would make."""

import json
import os
import socket

import numpy as np
import pytest

from paper_2111_00171_gb300 import ranks


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n", [0, 1, 7, 64, 65, 1000])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_pattern_range_tiles(n, world):
    spans = [ranks.pattern_range(n, world, r) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (lo0, hi0), (lo1, hi1) in zip(spans, spans[1:]):
        assert hi0 == lo1
    sizes = [hi - lo for lo, hi in spans]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_pattern_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        ranks.pattern_range(10, 2, 2)
    with pytest.raises(ValueError):
        ranks.pattern_range(10, 0, 0)


def test_csr_slice_is_csr_and_covers_scan():
    import synth
    scan = synth.random_patterns(5, n_patterns=11)
    pieces = [ranks.csr_slice(scan.row_ptr, scan.qx, scan.qy, scan.I, 3, r) for r in range(3)]
    for rp, qx, qy, I, lo, hi in pieces:
        assert rp[0] == 0 and len(rp) == hi - lo + 1
        assert np.all(np.diff(rp) >= 0) and rp[-1] == len(qx) == len(qy) == len(I)
        for j, b in enumerate(range(lo, hi)):
            ref = scan.pattern(b)
            got = (qx[rp[j]:rp[j + 1]], qy[rp[j]:rp[j + 1]], I[rp[j]:rp[j + 1]])
            for a, c in zip(got, ref):
                np.testing.assert_array_equal(a, c)
    assert sum(hi - lo for *_, lo, hi in pieces) == scan.n_patterns


def test_csr_slice_torch_tensors():
    torch = pytest.importorskip("torch")
    rp = torch.tensor([0, 2, 2, 5, 9], dtype=torch.int64)
    q = torch.arange(9, dtype=torch.float32)
    r0 = ranks.csr_slice(rp, q, q, q, 2, 0)
    r1 = ranks.csr_slice(rp, q, q, q, 2, 1)
    assert r0[0].tolist() == [0, 2, 2] and r0[1].tolist() == [0.0, 1.0]
    assert r1[0].tolist() == [0, 3, 7] and r1[1].tolist() == [2.0, 3, 4, 5, 6, 7, 8]


def test_single_process_reductions():
    assert ranks.max_over_ranks(3.5) == 3.5
    assert ranks.sum_over_ranks(2.0) == 2.0
    ranks.barrier()


def _oracle_plan():
    from oracle import acom_oracle as O
    refl = O.reflections(np.eye(3) * 4.08, [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]],
                         [79.0] * 4, [0.25] * 4, 1.5)
    v0, v1, v2, om = O.cubic_triangle()
    za = O.zone_axis_grid(v0, v1, v2, 6.0, om)
    return O.orientation_plan(refl, za, O.PlanParams(40, 0.0375, 72, 0.08, lam=0.01969))


def _match_all(plan, rp, qx, qy, I):
    from oracle import acom_oracle as O
    out = []
    for b in range(len(rp) - 1):
        s, e = rp[b], rp[b + 1]
        m = O.match_pattern(plan, qx[s:e], qy[s:e], I[s:e])
        out.append([int(m.za), int(m.k), int(m.mirror), float(m.score)])
    return out


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist

    import synth
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        assert ranks.rank_env() == (world, rank, rank)
        scan = synth.random_patterns(11, n_patterns=7)
        rp, qx, qy, I, lo, hi = ranks.csr_slice(scan.row_ptr, scan.qx, scan.qy, scan.I,
                                                world, rank)
        res = _match_all(_oracle_plan(), rp, qx, qy, I)
        gathered = [None] * world
        dist.all_gather_object(gathered, {"lo": lo, "hi": hi, "res": res})
        t_max = ranks.max_over_ranks(10.0 + rank)
        n_tot = ranks.sum_over_ranks(hi - lo)
        ranks.barrier()
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"gathered": gathered, "t_max": t_max, "n_tot": n_tot}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_their_slices():
    """Two ranks each match their slice of one scan with no collective on the
    data path; the gathered results equal one process matching everything,
    and the timing reduction is the maximum over ranks."""
    import tempfile

    import torch.multiprocessing as mp

    import synth
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, free_port(), d), nprocs=world,
                           start_method="spawn", join=True)
        outs = [json.load(open(os.path.join(d, f"rank{r}.json"))) for r in range(world)]
    scan = synth.random_patterns(11, n_patterns=7)
    ref = _match_all(_oracle_plan(), scan.row_ptr, scan.qx, scan.qy, scan.I)
    for o in outs:
        assert o["t_max"] == 10.0 + world - 1
        assert o["n_tot"] == scan.n_patterns
        g = o["gathered"]
        assert [x["lo"] for x in g] == [0, 4] and [x["hi"] for x in g] == [4, 7]
        assert [r for x in g for r in x["res"]] == ref


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.reference_arm(argparse.Namespace(warmup=3, steps=2, gpus=2))
    assert capsys.readouterr().out == ""


def test_bench_rank_seeds_distinct():
    import bench
    seeds = [bench.rank_seed(r) for r in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == bench.W["seed"]
