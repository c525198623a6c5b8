"""One lattice split into row slabs (Sec. 3, the aggregated algorithm over a partition of
the array; the trajectory does not depend on the partition, the remark after Fig. 3.6).

Slab i owns rows [row0_i, row0_i + nrows_i) of the torus.  Each step advances every slab by
R exact synchronous rounds (ac_slab_step: one temporal-blocked launch over the slab's tiles,
reading the R rows above and below the slab from the handle's current state).  After the
step every slab sends its first R rows to the slab above (they are that slab's halo below)
and its last R rows to the slab below (its halo above).  Every slab's halo is then the
neighbours' state after the same number of steps, so each step is R global synchronous
rounds and the union of the slabs' own rows is the exact trajectory.

`plan` gives the split and the exchange; `run_on_one_gpu` runs all slabs as handles of
one process on one GPU, exchanging halo rows by device copies; `exchange_distributed`
and `run_distributed` do the same with one slab per rank over torch.distributed
(send / recv of the halo rows; a max-reduction of the live flags ends the run).
"""
from __future__ import annotations

from dataclasses import dataclass

BYTES_PER_CELL = 12          # exported rows: uint64 keys, then uint32 counts


@dataclass(frozen=True)
class Slab:
    index: int
    row0: int
    nrows: int
    above: int               # index of the slab above (its last R rows are this slab's halo above)
    below: int               # index of the slab below


def plan(rows: int, nslabs: int, R: int) -> list[Slab]:
    """Equal split of the torus rows into `nslabs` slabs (the first rows % nslabs one row
    taller); every slab needs R <= nrows <= rows - 2R, so that its halo lies in its two
    neighbours."""
    if nslabs < 1:
        raise ValueError("at least one slab")
    q, rm = divmod(rows, nslabs)
    out, r0 = [], 0
    for i in range(nslabs):
        n = q + (i < rm)
        if not (R <= n <= rows - 2 * R):
            raise ValueError(f"slab {i} has {n} rows: needs {R} <= rows <= {rows - 2 * R}")
        out.append(Slab(i, r0, n, (i - 1) % nslabs, (i + 1) % nslabs))
        r0 += n
    return out


def halo_rows(slab: Slab, rows: int, R: int):
    """Rows of this slab's halo: (first row above, first row below), R rows each (the torus
    rows just outside the slab; a halo never wraps inside itself since R <= nrows)."""
    return (slab.row0 - R) % rows, (slab.row0 + slab.nrows) % rows


def send_rows(slab: Slab, R: int):
    """Rows this slab sends: (its first R rows, for the slab above; its last R rows, for the
    slab below)."""
    return slab.row0, slab.row0 + slab.nrows - R


def _copy_rows(export, imp, src_row: int, dst_row: int, R: int, rows: int, buf) -> None:
    """Copy R torus rows starting at src_row of one handle into rows starting at dst_row of
    another, splitting where either range crosses the last row."""
    done = 0
    while done < R:
        s = (src_row + done) % rows
        d = (dst_row + done) % rows
        n = min(R - done, rows - s, rows - d)
        export(s, n, buf)
        imp(d, n, buf)
        done += n


def run_on_one_gpu(ac, sims, slabs: list[Slab], R: int, t_end: int, max_steps: int = 1 << 20) -> int:
    """Advance the handles `sims` (each the whole lattice, one per slab, configured with
    `rounds` = R) to t_end as row slabs on one GPU.  Returns the number of steps."""
    import torch
    rows, cols = sims[0].rows, sims[0].cols
    for sim, sl in zip(sims, slabs):
        ac.ac_slab_configure(sim.handle, sl.row0, sl.nrows)
    buf = torch.empty(R * cols * BYTES_PER_CELL, dtype=torch.uint8, device="cuda")
    steps = 0
    while steps < max_steps:
        live = [ac.ac_slab_step(sim.handle, t_end) for sim in sims]
        steps += 1
        if not any(live):
            break
        for sim, sl in zip(sims, slabs):
            top, bottom = send_rows(sl, R)
            up, down = sims[sl.above], sims[sl.below]
            # this slab's first rows are the halo below of the slab above, its last rows the
            # halo above of the slab below
            _copy_rows(lambda r, n, b: ac.ac_slab_export(sim.handle, r, n, b.data_ptr()),
                       lambda r, n, b: ac.ac_slab_import(up.handle, r, n, b.data_ptr()), top, top, R, rows, buf)
            _copy_rows(lambda r, n, b: ac.ac_slab_export(sim.handle, r, n, b.data_ptr()),
                       lambda r, n, b: ac.ac_slab_import(down.handle, r, n, b.data_ptr()), bottom, bottom, R, rows,
                       buf)
    for sim in sims:
        ac.ac_slab_configure(sim.handle, 0, 0)
    return steps


def exchange_distributed(export_rows, import_rows, slab: Slab, R: int, nbytes: int, device, dist) -> None:
    """One halo exchange for the calling rank's slab over torch.distributed.

    export_rows(row, buf) fills `buf` (nbytes, uint8) with R rows starting at `row`;
    import_rows(row, buf) writes them into the state.  Every rank sends its first R rows to
    the rank above and its last R rows to the rank below, in that order, and receives the
    rank below's first rows (its halo below) and the rank above's last rows (its halo
    above), in that order, so the pairing also holds with two ranks (above == below)."""
    import torch
    top, bottom = send_rows(slab, R)
    above_row, below_row = (slab.row0 - R), (slab.row0 + slab.nrows)
    s_top = torch.empty(nbytes, dtype=torch.uint8, device=device)
    s_bot = torch.empty(nbytes, dtype=torch.uint8, device=device)
    r_below = torch.empty(nbytes, dtype=torch.uint8, device=device)
    r_above = torch.empty(nbytes, dtype=torch.uint8, device=device)
    export_rows(top, s_top)
    export_rows(bottom, s_bot)
    ops = [dist.P2POp(dist.isend, s_top, slab.above), dist.P2POp(dist.isend, s_bot, slab.below),
           dist.P2POp(dist.irecv, r_below, slab.below), dist.P2POp(dist.irecv, r_above, slab.above)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    import_rows(below_row, r_below)
    import_rows(above_row, r_above)


def run_distributed(ac, sim, rank: int, world: int, R: int, t_end: int, max_steps: int = 1 << 20) -> int:
    """One slab per rank (the handle holds the whole lattice, configured with rounds = R):
    steps, halo exchanges over torch.distributed and a max-reduction of the live flags."""
    import torch
    import torch.distributed as dist
    rows, cols = sim.rows, sim.cols
    slabs = plan(rows, world, R)
    sl = slabs[rank]
    ac.ac_slab_configure(sim.handle, sl.row0, sl.nrows)
    nbytes = R * cols * BYTES_PER_CELL
    device = torch.device("cuda", torch.cuda.current_device())

    # R torus rows from `row` as chunks of whole rows (two where they cross the last row), each
    # chunk in the exported layout: its keys, then its counts
    def chunks(row):
        done = 0
        while done < R:
            r = (row + done) % rows
            n = min(R - done, rows - r)
            yield r, n, done * cols * BYTES_PER_CELL
            done += n

    def export_rows(row, buf):
        for r, n, off in chunks(row):
            ac.ac_slab_export(sim.handle, r, n, buf[off:].data_ptr())

    def import_rows(row, buf):
        for r, n, off in chunks(row):
            ac.ac_slab_import(sim.handle, r, n, buf[off:].data_ptr())

    steps = 0
    flag = torch.zeros(1, dtype=torch.int32, device=device)
    while steps < max_steps:
        live = ac.ac_slab_step(sim.handle, t_end)
        steps += 1
        flag.fill_(1 if live else 0)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX)
        if int(flag.item()) == 0:
            break
        exchange_distributed(export_rows, import_rows, sl, R, nbytes, device, dist)
    ac.ac_slab_configure(sim.handle, 0, 0)
    return steps
