"""Slice sharding across processes (gloo, world size 2 and 3, on CPU).

The per-rank partial sums come from the oracle's slice terms here (no GPU); the test
checks the range split and the exchange: the sharded amplitude equals the single-process
one, and a rank that fails to join makes the others fail instead of hanging."""
import math
import os
import socket

import numpy as np
import pytest

import circuitgen as cg
from paper_1805_01450_gb300.distributed import compensated_sum, slice_range


def test_slice_ranges_partition():
    for total in (1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            got = [slice_range(total, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == total
            assert all(got[i][1] == got[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1


def test_compensated_sum_is_exact_on_cancelling_terms():
    parts = np.array([[1e16 + 1j], [1.0 + 1e-16j], [-1e16 - 1j]])
    out = compensated_sum(parts)
    assert out[0].real == 1.0
    assert math.isclose(out[0].imag, 1e-16)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    from datetime import timedelta
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
    try:
        from oracle import ve as VE
        from paper_1805_01450_gb300.distributed import sharded_amplitude
        import paper_1805_01450_gb300 as qv
        circ = cg.grid_circuit(4, 4, 12, 7)
        plan = qv.Plan(circ, n_slices=5)
        xs = cg.random_bitstrings(16, 3, 8)

        def partial(begin, count):
            ids = np.arange(begin, begin + count, dtype=np.int64)
            return np.array([VE.exact_sum(VE.slice_terms(circ, x, plan.order, plan.slices, slice_ids=ids))
                             for x in xs])
        q.put((rank, sharded_amplitude(partial, 1 << len(plan.slices))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_amplitude_matches_single_process(world):
    import multiprocessing as mp
    from oracle import statevector as SV
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circ = cg.grid_circuit(4, 4, 12, 7)
    psi = SV.final_state(circ)
    want = psi[cg.random_bitstrings(16, 3, 8)]
    for r in range(world):
        assert np.max(np.abs(res[r] - want)) < 1e-14
        assert np.array_equal(res[r], res[0])


class _HostStandIn:
    """Stands in for a GPU plan in plan_partial: the same amplitude(bitstrings, slice_begin,
    slice_count) contract (a complex128 tensor of partial sums), computed by the oracle on
    the host, and a record of the slice ranges it was asked for."""

    def __init__(self, plan, circ):
        self.plan, self.circ, self.calls = plan, circ, []

    def amplitude(self, bitstrings, slice_begin=0, slice_count=None):
        import torch
        from oracle import ve as VE
        self.calls.append((slice_begin, slice_count))
        ids = np.arange(slice_begin, slice_begin + slice_count, dtype=np.int64)
        vals = [VE.exact_sum(VE.slice_terms(self.circ, x, self.plan.order, self.plan.slices, slice_ids=ids))
                if slice_count else 0j for x in bitstrings]
        return torch.tensor(vals, dtype=torch.complex128)


def _plan_partial_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    from datetime import timedelta
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
    try:
        from paper_1805_01450_gb300.distributed import plan_partial, sharded_amplitude
        import paper_1805_01450_gb300 as qv
        circ = cg.grid_circuit(4, 5, 12, 17)
        plan = qv.Plan(circ, n_slices=4)
        xs = cg.random_bitstrings(20, 2, 18)
        stand_in = _HostStandIn(plan, circ)
        amps = sharded_amplitude(plan_partial(stand_in, xs), plan.n_slice_terms)
        q.put((rank, amps, stand_in.calls))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_plan_partial_contract_over_gloo_ranks(world):
    import multiprocessing as mp
    from oracle import statevector as SV
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_plan_partial_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {r: (a, calls) for r, a, calls in (q.get(timeout=120) for _ in range(world))}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circ = cg.grid_circuit(4, 5, 12, 17)
    want = SV.final_state(circ)[cg.random_bitstrings(20, 2, 18)]
    for r in range(world):
        # each rank asked for exactly its contiguous share of the 16 slice terms, once
        b, e = slice_range(16, r, world)
        assert res[r][1] == [(b, e - b)]
        assert np.max(np.abs(res[r][0] - want)) < 1e-14
        assert np.array_equal(res[r][0], res[0][0])


def _lonely_worker(port, q):
    import torch.distributed as dist
    from datetime import timedelta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=0, world_size=2, timeout=timedelta(seconds=3))
        q.put("joined")
    except Exception as e:    # the second rank never joins: the rendezvous times out
        q.put(type(e).__name__)


def test_missing_rank_times_out_instead_of_hanging():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_lonely_worker, args=(_free_port(), q))
    p.start()
    out = q.get(timeout=120)
    p.join(timeout=30)
    assert out != "joined"
