"""Decomposition of one lattice into y-slabs (bands of rows), one per rank,
with halo rows exchanged every step.

A band owns a contiguous range of rows and keeps two ghost rows below and
two above them (the pull of Eq. 1 reaches one row, the Eq. 3 force's density
one row more).  After each step a band sends its two lowest owned rows to the
band below and its two highest to the band above, and receives the matching
rows into its ghost rows; the band below rank 0 is the last rank's, which is
the periodic wrap of Eq. 1 in y.  Every owned row then evaluates exactly what
the undecomposed lattice evaluates there, so the result is bit-identical.

* ``band_partition`` -- rows of each rank (as even as possible, >= 2 each).
* ``with_halo`` -- a band's initial field: its rows plus two wrapped rows on
  each side.
* ``exchange`` -- one halo exchange over ``torch.distributed`` (point to
  point; gloo for host tensors, NCCL for device tensors), or the periodic
  self-exchange of a single rank.
* ``window_reduce`` -- the window diagnostics of the whole lattice (mass
  and the row means of the density, hence the coexistence densities) from
  the bands' owned rows, in one FP64 all-reduce.
* ``BandLattice`` -- a band of the CUDA library (``lbm_create_band``) with
  its halo buffers; ``step`` computes the boundary rows, packs them, sends
  them on a second stream while the interior rows are computed, and unpacks
  (or, without overlap, step, pack, exchange, unpack).
* ``LocalBands`` -- several bands of one lattice on one GPU in one process,
  exchanging by device copies (each band's kernels run to completion before
  the copies; nothing waits on another kernel).

The engine of a band is anything with the four halo operations; the tests
drive the same ``exchange`` with the FP64 oracle on CPU ranks.
"""
from __future__ import annotations

import numpy as np

from . import lbm

GHOST_ROWS = 2
TAG_UP, TAG_DOWN = 1, 2  # messages to the band above / below


def band_partition(ny, world):
    """[(y0, rows)] of each rank: contiguous, covering 0 .. ny - 1, the first
    ny % world ranks one row longer; every band needs >= 2 rows."""
    if world < 1 or ny < GHOST_ROWS * world:
        raise ValueError(f"{ny} rows cannot give {world} bands of >= {GHOST_ROWS} rows")
    base, extra = divmod(ny, world)
    out, y0 = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((y0, n))
        y0 += n
    return out


def with_halo(field, y0, rows):
    """Rows y0 - 2 .. y0 + rows + 1 (wrapped in y) of a [..., ny, nx] field."""
    ny = field.shape[-2]
    idx = np.arange(y0 - GHOST_ROWS, y0 + rows + GHOST_ROWS) % ny
    return np.ascontiguousarray(np.take(field, idx, axis=-2))


def neighbours(rank, world):
    """(rank below, rank above) in the periodic ring of bands."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(lo, hi, rank, world, group=None, out=None):
    """One halo exchange: send `hi` (this band's two highest rows) to the
    band above and `lo` to the band below; return (from_below, from_above),
    the band below's `hi` and the band above's `lo` (received into `out`
    when given).  Tensors of equal shape and type on the device the process
    group serves.  A single rank is its own neighbour: (hi, lo)."""
    if world == 1:
        return hi, lo
    import torch
    import torch.distributed as dist
    below, above = neighbours(rank, world)
    from_below, from_above = out if out is not None else (torch.empty_like(hi),
                                                          torch.empty_like(lo))
    ops = [dist.P2POp(dist.isend, hi, above, group, TAG_UP),
           dist.P2POp(dist.irecv, from_below, below, group, TAG_UP),
           dist.P2POp(dist.isend, lo, below, group, TAG_DOWN),
           dist.P2POp(dist.irecv, from_above, above, group, TAG_DOWN)]
    for w in dist.batch_isend_irecv(ops):
        w.wait()
    return from_below, from_above


def window_reduce(rho_own, y0, ny, world, group=None, device=None):
    """(mass, row means [ny]) of the whole lattice from this rank's owned
    density rows `rho_own` [rows][nx] starting at row y0: every rank fills
    its rows of an FP64 vector [mass, row sums ...] and one all-reduce (sum)
    completes it.  The coexistence densities of a slab follow from the row
    means (gas: rows 0 and ny - 1, liquid: rows ny/2 - 1 and ny/2)."""
    import torch
    rho_own = np.asarray(rho_own, dtype=np.float64)
    rows, nx = rho_own.shape
    v = np.zeros(ny + 1)
    sums = rho_own.sum(1)
    v[0] = sums.sum()
    v[1 + y0:1 + y0 + rows] = sums
    t = torch.from_numpy(v).to(device if device is not None else "cpu")
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.cpu().numpy()
    return float(v[0]), v[1:] / nx


def coexistence(row_means):
    """(rho_g, rho_l) of a slab whose liquid fills the middle rows."""
    ny = len(row_means)
    lo = ny // 2 - 1 if ny >= 2 else 0
    return (0.5 * (row_means[0] + row_means[-1]),
            0.5 * (row_means[lo] + row_means[ny // 2]))


class BandLattice:
    """This rank's band of an nx x ny lattice on its GPU, stepped with halo
    exchanges over the default process group (NCCL for the device buffers).
    `density` is the whole initial field (every rank passes the same)."""

    def __init__(self, nx, ny, T_over_Tc, density, rank=0, world=1, precision=lbm.FP32,
                 device=0, at_rest=False, group=None, **kw):
        import torch
        self.torch = torch
        self.rank, self.world, self.group = rank, world, group
        self.ny, self.device = ny, device
        self.y0, self.rows = band_partition(ny, world)[rank]
        self.stream = torch.cuda.Stream(device=device)
        self.lat = lbm.Lattice(nx, self.rows, T_over_Tc, precision=precision, device=device,
                               stream=self.stream.cuda_stream, band=True, **kw)
        rho = with_halo(np.asarray(density, dtype=np.float64), self.y0, self.rows)
        if at_rest:
            self.lat.init_density_at_rest(rho)
        else:
            self.lat.init_density(rho)
        n = self.lat.halo_bytes()
        dev = torch.device("cuda", device)
        self.lo = torch.empty(n, dtype=torch.uint8, device=dev)
        self.hi = torch.empty(n, dtype=torch.uint8, device=dev)
        self.recv = (torch.empty(n, dtype=torch.uint8, device=dev),
                     torch.empty(n, dtype=torch.uint8, device=dev))
        self.comm = torch.cuda.Stream(device=device)
        self.exchange()  # ghost rows from the neighbours' exact boundary rows

    def exchange(self):
        """Pack, exchange and unpack the halo rows (on the band's stream)."""
        with self.torch.cuda.stream(self.stream):
            self.lat.halo_pack(self.lo.data_ptr(), self.hi.data_ptr())
            below, above = exchange(self.lo, self.hi, self.rank, self.world, self.group,
                                    self.recv)
            self.lat.halo_unpack(below.data_ptr(), above.data_ptr())

    def step(self, n, scheme, tau, sigma=0.0, overlap=None):
        """n steps, each followed by a halo exchange; returns the status of
        the last step (lbm_sync_status).  With `overlap` the boundary rows
        are computed and packed first, and the exchange runs on a second
        stream while the interior rows are computed (lbm_band_step_overlap);
        the next step waits for the unpack.  By default overlap is on when
        there is a transfer to hide (world > 1): a single band's
        self-exchange copies nothing, and the split costs two small launches."""
        torch = self.torch
        if overlap is None:
            overlap = self.world > 1
        for _ in range(n):
            if not overlap:
                with torch.cuda.stream(self.stream):
                    self.lat.step_async(1, scheme, tau, sigma)
                self.exchange()
                continue
            with torch.cuda.stream(self.stream):
                self.lat.step_overlap(scheme, tau, sigma, self.lo.data_ptr(), self.hi.data_ptr(),
                                      self.comm.cuda_stream)
            with torch.cuda.stream(self.comm):
                below, above = exchange(self.lo, self.hi, self.rank, self.world, self.group,
                                        self.recv)
            self.stream.wait_stream(self.comm)
            with torch.cuda.stream(self.stream):
                self.lat.halo_unpack(below.data_ptr(), above.data_ptr())
        return self.lat.sync()

    def observe(self):
        """(rho, vx, vy) of the owned rows."""
        return self.lat.observe()

    def window(self):
        """(mass, rho_g, rho_l) of the whole lattice: one FP64 all-reduce over
        the ranks (window_reduce), on the device the process group serves."""
        self.lat.sync()
        dev = self.torch.device("cuda", self.device) if self.world > 1 else None
        mass, means = window_reduce(self.observe()[0], self.y0, self.ny, self.world,
                                    self.group, dev)
        return (mass, *coexistence(means))

    def close(self):
        self.lat.close()


class LocalBands:
    """`k` bands of one nx x ny lattice on one GPU, one stream, exchanging
    halos by device copies after every step (a single-GPU run of the
    decomposed path; with k = 1 it is the periodic self-exchange)."""

    def __init__(self, nx, ny, T_over_Tc, density, k, precision=lbm.FP32, device=0,
                 at_rest=False, **kw):
        import torch
        self.torch = torch
        self.k = k
        self.parts = band_partition(ny, k)
        self.stream = torch.cuda.Stream(device=device)
        dev = torch.device("cuda", device)
        density = np.asarray(density, dtype=np.float64)
        self.lats, self.lo, self.hi = [], [], []
        for y0, rows in self.parts:
            lat = lbm.Lattice(nx, rows, T_over_Tc, precision=precision, device=device,
                              stream=self.stream.cuda_stream, band=True, **kw)
            rho = with_halo(density, y0, rows)
            if at_rest:
                lat.init_density_at_rest(rho)
            else:
                lat.init_density(rho)
            n = lat.halo_bytes()
            self.lats.append(lat)
            self.lo.append(torch.empty(n, dtype=torch.uint8, device=dev))
            self.hi.append(torch.empty(n, dtype=torch.uint8, device=dev))
        self.exchange()  # ghost rows from the neighbours' exact boundary rows

    def set_variant(self, variant):
        for lat in self.lats:
            lat.set_variant(variant)

    def exchange(self):
        """Every band packs its boundary rows, then unpacks its neighbours'."""
        for lat, lo, hi in zip(self.lats, self.lo, self.hi):
            lat.halo_pack(lo.data_ptr(), hi.data_ptr())
        for b, lat in enumerate(self.lats):
            below, above = (b - 1) % self.k, (b + 1) % self.k
            lat.halo_unpack(self.hi[below].data_ptr(), self.lo[above].data_ptr())

    def step(self, n, scheme, tau, sigma=0.0, overlap=False):
        """n steps of every band with an exchange after each; returns the
        worst band status.  `overlap` takes the boundary-rows-first path
        (lbm_band_step_overlap; on one stream the order only changes)."""
        for _ in range(n):
            if overlap:
                for lat, lo, hi in zip(self.lats, self.lo, self.hi):
                    lat.step_overlap(scheme, tau, sigma, lo.data_ptr(), hi.data_ptr())
                for b, lat in enumerate(self.lats):
                    below, above = (b - 1) % self.k, (b + 1) % self.k
                    lat.halo_unpack(self.hi[below].data_ptr(), self.lo[above].data_ptr())
                continue
            for lat in self.lats:
                lat.step_async(1, scheme, tau, sigma)
            self.exchange()
        return max(lat.sync() for lat in self.lats)

    def observe(self):
        """(rho, vx, vy) of the whole lattice, the bands' owned rows stacked."""
        parts = [lat.observe() for lat in self.lats]
        return tuple(np.concatenate([p[i] for p in parts], 0) for i in range(3))

    def populations(self):
        return np.concatenate([lat.populations() for lat in self.lats], 1)

    def mass(self):
        return sum(lat.mass() for lat in self.lats)

    def close(self):
        for lat in self.lats:
            lat.close()
