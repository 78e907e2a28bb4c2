"""1-D domain decomposition of one ring road over ranks (grid layout).

The paper lists distributed memory among its variations; for the grid
representation the natural split is by cells.  Rank r of `world` owns the
contiguous cells [a_r, a_{r+1}) with a_r = floor(r L / world), and keeps
them in a buffer with H = round_up(k vmax, 16) halo cells on each side:

    buffer index:  0 .. H-1       H .. H+owned-1      H+owned .. W-1
    ring cell:     a-H .. a-1     a .. b-1            b .. b+H-1     (mod L)

Cell j at step t+1 depends on cells j - vmax .. j + vmax at step t (a car
arriving from behind, the gap ahead), so k steps of the owned cells need
exactly these halos.  Before every launch of k steps each rank sends its
first H owned cells to its left neighbour (that rank's right halo) and its
last H owned cells to its right neighbour (that rank's left halo), and
receives its own halos likewise: one point-to-point exchange per k steps,
never a collective on the data path.  The per-step statistics of a rank
count the cars whose cell at the start of a step it owns, so the ranks'
series add up to the whole road's (a sum over ranks, or a gather).

Two ways to run it:
  * run_rank: this process is one rank of a torch.distributed group; the
    halo exchange is point-to-point send/receive (NCCL between GPUs, gloo
    between CPU processes);
  * run_local: every rank's buffer lives in this process and the exchange is
    a copy between buffers (one GPU holding all the ranks' segments one
    after another, for tests and for a one-GPU run of the same code).
The k steps themselves are a callable, step_fn(seg, buf_in, buf_out, k,
step0, rank) -> (sum_v[k], crossings[k]) or None, so the same exchange
drives the library's segment kernel (nasch_segment_run) or any other
stepper of a buffer laid out as above.
"""
from __future__ import annotations

from dataclasses import dataclass


def halo_cells(k: int, vmax: int) -> int:
    """Halo cells per side for k fused steps: k vmax rounded up to 16."""
    return (k * vmax + 15) // 16 * 16


def owned_range(L: int, world: int, rank: int) -> tuple[int, int]:
    """Cells [a, b) owned by `rank`: a = floor(rank L / world)."""
    return rank * L // world, (rank + 1) * L // world


@dataclass(frozen=True)
class RingSegment:
    L: int
    world: int
    rank: int
    k: int
    vmax: int

    def __post_init__(self):
        if not (1 <= self.world <= self.L and 0 <= self.rank < self.world):
            raise ValueError("need 1 <= world <= L and 0 <= rank < world")
        if self.k < 1:
            raise ValueError("k >= 1")
        if self.L // self.world < self.H:
            raise ValueError(f"each rank must own at least H = {self.H} cells (L // world = {self.L // self.world})")

    @property
    def H(self) -> int:
        return halo_cells(self.k, self.vmax)

    @property
    def a(self) -> int:
        return owned_range(self.L, self.world, self.rank)[0]

    @property
    def b(self) -> int:
        return owned_range(self.L, self.world, self.rank)[1]

    @property
    def owned(self) -> int:
        return self.b - self.a

    @property
    def W(self) -> int:
        """Buffer length: owned cells and a halo on each side."""
        return self.owned + 2 * self.H

    @property
    def first_buffer_cell(self) -> int:
        """Ring cell of buffer index 0."""
        return (self.a - self.H) % self.L

    @property
    def left(self) -> int:
        return (self.rank - 1) % self.world

    @property
    def right(self) -> int:
        return (self.rank + 1) % self.world

    def ring_cells(self) -> list[int]:
        """Ring cell of every buffer index (for filling a buffer from a whole road)."""
        return [(self.a - self.H + i) % self.L for i in range(self.W)]

    # slices of the buffer
    def left_halo(self):
        return slice(0, self.H)

    def right_halo(self):
        return slice(self.H + self.owned, self.W)

    def first_owned(self):
        """The first H owned cells: the left neighbour's right halo."""
        return slice(self.H, 2 * self.H)

    def last_owned(self):
        """The last H owned cells: the right neighbour's left halo."""
        return slice(self.owned, self.owned + self.H)

    def owned_part(self):
        return slice(self.H, self.H + self.owned)


def segments(L: int, world: int, k: int, vmax: int) -> list[RingSegment]:
    return [RingSegment(L, world, r, k, vmax) for r in range(world)]


def exchange_local(segs: list[RingSegment], bufs: list) -> None:
    """Halo exchange between buffers held in one process (every rank's)."""
    if segs[0].H == 0:
        return
    sends = [(b[s.first_owned()].clone() if hasattr(b, "clone") else b[s.first_owned()].copy(),
              b[s.last_owned()].clone() if hasattr(b, "clone") else b[s.last_owned()].copy())
             for s, b in zip(segs, bufs)]
    for s, b in zip(segs, bufs):
        b[s.left_halo()] = sends[s.left][1]     # the left neighbour's last owned cells
        b[s.right_halo()] = sends[s.right][0]   # the right neighbour's first owned cells


def exchange_dist(seg: RingSegment, buf, dist, group=None) -> None:
    """Halo exchange of this rank's buffer (a torch tensor) by point-to-point
    messages.  Sends and receives are posted in one fixed order on every rank
    (to the right, then to the left; from the left, then from the right), so
    that messages between the same two ranks match in order even when the
    left and right neighbours are the same rank (world = 2)."""
    if seg.H == 0:
        return
    if seg.world == 1:
        first = buf[seg.first_owned()].clone()
        last = buf[seg.last_owned()].clone()
        buf[seg.left_halo()] = last
        buf[seg.right_halo()] = first
        return
    send_right = buf[seg.last_owned()].contiguous()
    send_left = buf[seg.first_owned()].contiguous()
    recv_left = buf.new_empty(seg.H)
    recv_right = buf.new_empty(seg.H)
    ops = [dist.P2POp(dist.isend, send_right, seg.right, group, tag=1),
           dist.P2POp(dist.isend, send_left, seg.left, group, tag=2),
           dist.P2POp(dist.irecv, recv_left, seg.left, group, tag=1),
           dist.P2POp(dist.irecv, recv_right, seg.right, group, tag=2)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    buf[seg.left_halo()] = recv_left
    buf[seg.right_halo()] = recv_right


def chunks(steps: int, k: int, step0: int = 0):
    """(first step, steps) of each launch: k steps at a time."""
    s = 0
    while s < steps:
        kk = min(k, steps - s)
        yield step0 + s, kk
        s += kk


def run_local(segs: list[RingSegment], bufs: list, steps: int, step_fn, step0: int = 0, spare=None):
    """Run `steps` steps of every rank's segment held in this process.
    bufs[r]: rank r's buffer with its owned cells at step0 (halos are filled
    here).  Returns (bufs, per-rank statistics) with the owned cells at
    step0 + steps; statistics are lists of step_fn's per-launch results."""
    k = segs[0].k
    outs = spare if spare is not None else [b.clone() if hasattr(b, "clone") else b.copy() for b in bufs]
    stats = [[] for _ in segs]
    for s0, kk in chunks(steps, k, step0):
        exchange_local(segs, bufs)
        for r, s in enumerate(segs):
            stats[r].append(step_fn(s, bufs[r], outs[r], kk, s0, r))
        bufs, outs = outs, bufs
    return bufs, stats


def run_rank(seg: RingSegment, buf, steps: int, step_fn, dist, group=None, step0: int = 0, spare=None):
    """Run `steps` steps of this rank's segment, exchanging halos with its
    ring neighbours before every launch.  Returns (buffer, statistics)."""
    out = spare if spare is not None else buf.clone()
    stats = []
    for s0, kk in chunks(steps, seg.k, step0):
        exchange_dist(seg, buf, dist, group)
        stats.append(step_fn(seg, buf, out, kk, s0, seg.rank))
        buf, out = out, buf
    return buf, stats


def library_step(L: int, vmax: int, p: float, seed: int, road_id: int = 0, stream=None):
    """step_fn for torch CUDA buffers: the library's segment kernel
    (nasch_segment_run); returns the launch's (sum_v, crossings) as device
    tensors of length k."""
    import torch

    from . import nasch as NS

    def step(seg: RingSegment, buf_in, buf_out, k: int, step0: int, rank: int):
        sv = torch.zeros(k, dtype=torch.int64, device=buf_in.device)
        cr = torch.zeros(k, dtype=torch.int64, device=buf_in.device)
        NS.segment_run(buf_in.data_ptr(), buf_out.data_ptr(), seg.owned, seg.H, seg.a, L, vmax, p, seed, road_id,
                       step0, k, sv.data_ptr(), cr.data_ptr(),
                       stream if stream is not None else torch.cuda.current_stream())
        return sv, cr

    return step
