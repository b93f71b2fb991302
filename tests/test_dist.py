"""Host-side logic of the multi-process benchmark path on CPU (gloo,
world size 2): every rank runs an independent replica, the job time is the
maximum over ranks and the job value counts the units of all ranks.  No
collective touches the data path."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        t_local = 1.0 + rank  # rank 1 is the slower replica
        t_max = bench.max_over_ranks(t_local, dist, "cpu")
        value = bench.job_value(w, 100.0, t_max)
        out[rank] = (w, r, local, t_max, value)
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_units():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank, (w, r, local, t_max, value) in res.items():
        assert (w, r, local) == (2, rank, rank)
        assert t_max == pytest.approx(2.0)
        assert value == pytest.approx(2 * 100.0 / 2.0)


def test_single_process_defaults():
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 10.0, 2.0) == 5.0


def test_roofline_helpers():
    """The issue view: 152 SMs x 4 schedulers x 1 warp instruction per
    cycle; the committed ncu record is used only on matching sources and
    split."""
    r = bench.issue_roofline(608e6, 1e-3, 2000.0)
    assert r["peak"] == pytest.approx(152 * 4 * 2.0)
    assert r["achieved"] == pytest.approx(608.0)
    assert r["frac"] == pytest.approx(0.5)
    assert bench.ncu_record("kr_mpa", "no such workload", "x") == {}
    assert bench.ncu_traffic("no_such_kernel", "w", "s") is None


def test_l2_resident_levels_report_the_issue_roofline():
    """A level whose node spectra fit in L2 reports the issue view as its
    roofline ("alu") and keeps the HBM figures beside it; a larger level,
    or a line without the issue view, keeps the HBM roofline."""
    prof = {"kn_mpa": (10.0, 100, 1.75e10), "scan": (2.0, 100, 1e9)}
    hbm, _ = bench.hbm_roofline(prof, 6786.9, "measured", {"dram_bytes_per_launch": 1.49e8})
    hbm["issue"] = bench.issue_roofline(74.9e6, 10.0e-3 / 100, 2070.0)
    small = bench.l2_resident_roofline(hbm, 801 * (1 << 14) * 8.0)
    assert small["bound"] == "alu" and small["kernel"] == "kn_mpa"
    assert small["frac"] == hbm["issue"]["frac"] and small["peak"] == pytest.approx(152 * 4 * 2.07, abs=0.1)
    assert small["hbm"]["frac"] == hbm["frac"] and small["traffic"] == 1.49e8
    assert bench.l2_resident_roofline(hbm, 126 * (1 << 20) * 8.0) is hbm
    plain, _ = bench.hbm_roofline(prof, 6786.9, "measured")
    assert bench.l2_resident_roofline(plain, 1e6) is plain


def test_clock_samples_are_parsed():
    """The clocks record: median SM clock of the loaded samples, the maximum
    clock, and every throttle reason that was active in any sample."""
    idle = "0, 345, 2070, 120.5, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active"
    busy = "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1965, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1800, 2070, 1400.0, 0x0000000000000020, Not Active, Not Active, Active, Not Active"
    r = bench.parse_clock_samples("\n".join([idle, busy, busy, capped, "garbage line", ""]))
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 4
    assert r["reasons"] == ["sw_power_cap"]
    assert bench.parse_clock_samples(hot)["reasons"] == ["sw_thermal_slowdown"]
    assert bench.parse_clock_samples("")["reasons"] == ["no samples"]
