"""The y-slab decomposition of one lattice (halo.py) on CPU ranks.

Each gloo rank steps the FP64 oracle on its band (its rows plus two ghost
rows each side) and exchanges halo rows with its neighbours after every step
through ``halo.exchange``; the owned rows are gathered and compared with the
undecomposed oracle run, bit for bit.  A droplet straddles the periodic wrap
in y (Eq. 1), so the exchange between the last rank and rank 0 carries it.
(The oracle is this test's engine: it stores the state after streaming, the
CUDA library before it, and both need the same two ghost rows per side.)
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from oracle import theory as th
from paper_1204_4098_gb300 import halo, inputs

NX, T, STEPS = 24, 0.85, 25


def initial_field(ny, seed=2):
    """Droplet centred on the y wrap (centre row 0), small random velocities."""
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(T)))
    rho = inputs.droplet(NX, ny, rg, rl, 7.0, W=4.0, x0=NX / 2.0, y0=0.0)
    rng = np.random.default_rng(seed)
    return rho, 0.01 * rng.uniform(-1, 1, rho.shape), 0.01 * rng.uniform(-1, 1, rho.shape)


def whole_run(ny, scheme, tau, sigma):
    rho, ux, uy = initial_field(ny)
    lat = oracle.Lattice(NX, ny, T)
    lat.init_density(rho, ux, uy)
    assert lat.step(STEPS, scheme, tau, sigma)[0] == 0
    return lat.f


def band_run(rank, world, ny, scheme, tau, sigma, window=False):
    """This rank's band stepped by the oracle with halo exchanges; returns
    its owned rows [9][rows][nx]."""
    y0, rows = halo.band_partition(ny, world)[rank]
    rho, ux, uy = initial_field(ny)
    f0 = oracle.init_equilibrium(rho, ux, uy)
    lat = oracle.Lattice(NX, rows + 2 * halo.GHOST_ROWS, T)
    lat.f = halo.with_halo(f0, y0, rows)
    g = halo.GHOST_ROWS
    for _ in range(STEPS):
        assert lat.step(1, scheme, tau, sigma)[0] == 0
        lo = torch.from_numpy(np.ascontiguousarray(lat.f[:, g:2 * g]))
        hi = torch.from_numpy(np.ascontiguousarray(lat.f[:, rows:rows + g]))
        below, above = halo.exchange(lo, hi, rank, world)
        lat.f[:, 0:g] = below.numpy()
        lat.f[:, rows + g:rows + 2 * g] = above.numpy()
    own = lat.f[:, g:g + rows].copy()
    if window:  # the window diagnostics in one FP64 all-reduce
        return halo.window_reduce(own.sum(0), y0, ny, world)
    return own


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, ny, case, q, window=False):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own = band_run(rank, world, ny, *case, window=window)
        if window:
            q.put((rank, own))
            return
        parts = [None] * world
        dist.all_gather_object(parts, own)
        if rank == 0:
            q.put(np.concatenate(parts, 1))
    finally:
        dist.destroy_process_group()


def _spawn(world, ny, case, window=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ny, case, q, window))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)] if window else q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world,ny", [(2, 30), (4, 31)])
@pytest.mark.parametrize("case", [(oracle.IMPROVED, 0.8, 0.1), (oracle.SC, 1.0, 0.0)],
                         ids=["improved", "shan-chen"])
def test_decomposed_run_matches_whole_lattice_bitwise(world, ny, case):
    got = _spawn(world, ny, case)
    want = whole_run(ny, *case)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_single_rank_is_the_periodic_self_exchange():
    ny, case = 20, (oracle.IMPROVED, 0.8, 0.1)
    assert np.array_equal(band_run(0, 1, ny, *case), whole_run(ny, *case))


def test_band_partition_and_halo_rows():
    assert halo.band_partition(10, 1) == [(0, 10)]
    assert halo.band_partition(31, 4) == [(0, 8), (8, 8), (16, 8), (24, 7)]
    parts = halo.band_partition(1000, 7)
    assert sum(n for _, n in parts) == 1000 and max(n for _, n in parts) - \
        min(n for _, n in parts) <= 1
    with pytest.raises(ValueError):
        halo.band_partition(7, 4)  # a band needs two rows to serve as a halo
    field = np.arange(6 * 3, dtype=float).reshape(6, 3)
    h = halo.with_halo(field, 0, 2)  # rows 4, 5 | 0, 1 | 2, 3
    assert np.array_equal(h[:, 0], [12.0, 15.0, 0.0, 3.0, 6.0, 9.0])
    assert halo.neighbours(0, 4) == (3, 1) and halo.neighbours(3, 4) == (2, 0)


def test_window_reduce_gives_every_rank_the_whole_lattice_diagnostics():
    """One FP64 all-reduce per window: every rank gets the whole lattice's
    mass and row means, equal to those of the undecomposed run (the mass to
    rounding, the row means exactly: each row is summed by one rank)."""
    ny, case = 31, (oracle.IMPROVED, 0.8, 0.1)
    got = _spawn(4, ny, case, window=True)
    rho = whole_run(ny, *case).sum(0)
    for rank, (mass, means) in got:
        assert mass == pytest.approx(rho.sum(), rel=1e-13)
        assert np.array_equal(means, rho.sum(1) / NX)
    g, l = halo.coexistence(rho.mean(1))
    assert halo.coexistence(got[0][1][1]) == (g, l)
    mass, means = halo.window_reduce(rho[3:9], 3, ny, 1)  # one rank: its rows only
    assert mass == pytest.approx(rho[3:9].sum(), rel=1e-14)
    assert np.array_equal(means[3:9], rho[3:9].sum(1) / NX) and not means[:3].any()
