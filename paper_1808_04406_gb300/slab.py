"""Domain decomposition of a periodic D3Q27 grid into slabs along z.

Streaming moves every population by its velocity, one node per step (Sec. II.A,
the final update of Sec. II.C), so a slab of the grid needs one ghost plane on
each side.  Each rank holds its nzl planes as local planes 1 .. nzl of a grid
of nzl + 2 planes and sweeps only those (lbm_set_active_planes).

In the AA pattern the even sweep touches only a node's own slots; the odd sweep
reads and writes slot (x + e_j, j) of every population j.  So only odd sweeps
reach into a ghost plane, and only for the nine populations whose e_z points
out of the slab (UP: e_z = +1 into the top ghost, DOWN: e_z = -1 into the
bottom ghost).  Around each odd sweep a rank
  before: receives the neighbour's boundary plane of those nine populations
          into its ghost plane (the neighbour's even sweep wrote them), and
  after:  sends the ghost plane back; the neighbour stores it in its boundary
          plane (the slots the odd sweep wrote belong to the neighbour's nodes).
Each slot is touched by exactly one node per sweep, so the neighbour's own
copy of those slots is neither read nor written meanwhile.  Nothing here does
arithmetic of the method: the sweeps are the library's kernels, and this
module only moves planes: between ranks one contiguous slice per population
and plane, within a process one strided copy of the nine planes.

After an even sweep (odd parity) some populations of a boundary node sit in a
ghost plane; refresh_ghosts() fills it before the slab's state is read.

Transports: torch.distributed point-to-point (NCCL between GPUs, gloo on CPU),
a local copy when one rank holds the whole periodic grid, and LocalGroup,
which runs all slabs of a grid in one process.
"""
import numpy as np

# velocity index i = sum_d (e_id + 1) 3^d: e_z = i // 9 - 1, so the nine
# populations crossing a face are one contiguous index range
UP = tuple(range(18, 27))    # e_z = +1
DOWN = tuple(range(0, 9))    # e_z = -1


def split(nz, world):
    """(z0, count) of each rank's planes: contiguous, sizes differ by at most one."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz (every slab holds at least one plane)")
    base, extra = divmod(nz, world)
    out, z0 = [], 0
    for r in range(world):
        c = base + (1 if r < extra else 0)
        out.append((z0, c))
        z0 += c
    return out


def messages(nzl, phase):
    """The plane copies of one odd step for a slab of nzl owned planes, in the
    canonical order both ends of a message use.  phase "pre" (before the odd
    sweep) or "post" (after it).  Returns (sends, recvs), each a list of
    (towards, pops, local_plane): towards is "down" (to or from the rank below)
    or "up"; a send to "down" is matched by the lower rank's receive from "up",
    message by message in this order."""
    top_ghost = nzl + 1
    if phase == "pre":
        sends = [("down", UP, 1), ("up", DOWN, nzl)]
        recvs = [("up", UP, top_ghost), ("down", DOWN, 0)]
    elif phase == "post":
        sends = [("down", DOWN, 0), ("up", UP, top_ghost)]
        recvs = [("up", DOWN, nzl), ("down", UP, 1)]
    else:
        raise ValueError(phase)
    return sends, recvs


def _peer_of(towards):
    return "up" if towards == "down" else "down"


def _tag(phase, towards_of_sender, k):
    """Message tag: the sender's direction decides it, so both ends agree."""
    return (0 if phase == "pre" else 100) + (0 if towards_of_sender == "down" else 10) + k


def plane_view(pop, j, plane, plane_elems):
    """Population j of one local plane: a contiguous slice of the (Q, N) buffer."""
    return pop[j, plane * plane_elems:(plane + 1) * plane_elems]


def planes_view(pop, pops, plane, plane_elems):
    """The nine populations `pops` (a contiguous index range) of one local
    plane: a strided (9, plane_elems) view, copied in one operation."""
    return pop[pops[0]:pops[-1] + 1, plane * plane_elems:(plane + 1) * plane_elems]


class SlabRun:
    """One rank's slab.  sim: a D3Q27 object with step(n), step_count and
    raw_populations() (the (Q, N) storage view; lbm.Simulation on a GPU) over a
    local grid (nx, ny, nzl + 2) whose sweeps cover local planes 1 .. nzl only.
    transport: run(ops) for lists of (kind, tensor, peer, tag); None when one
    rank holds the whole grid (the neighbour is the slab itself) or when a
    LocalGroup steps the slabs."""

    def __init__(self, sim, global_dims, rank, world, transport=None):
        self.sim = sim
        self.nx, self.ny, self.nz = (int(v) for v in global_dims)
        self.rank, self.world = int(rank), int(world)
        self.z0, self.nzl = split(self.nz, self.world)[self.rank]
        self.plane = self.nx * self.ny
        self.transport = transport
        self.peers = {"down": (self.rank - 1) % self.world, "up": (self.rank + 1) % self.world}

    @classmethod
    def create(cls, global_dims, tau_per_order, storage, rank, world, transport=None, device=None, stream=None):
        """A slab on the GPU through the library."""
        from .lbm import Simulation
        nx, ny, nz = (int(v) for v in global_dims)
        z0, nzl = split(nz, world)[rank]
        sim = Simulation("D3Q27", (nx, ny, nzl + 2), tau_per_order, storage=storage, device=device, stream=stream)
        sim.set_active_planes(1, nzl)
        return cls(sim, global_dims, rank, world, transport)

    # fields --------------------------------------------------------------------
    def local_planes(self):
        """Global plane index of each local plane 0 .. nzl + 1 (ghosts wrap)."""
        return [(self.z0 - 1 + k) % self.nz for k in range(self.nzl + 2)]

    def local_fields(self, rho, u):
        """The slab's part (with ghost planes) of global fields rho[N], u[3, N]."""
        rho = np.asarray(rho).reshape(self.nz, self.plane)
        u = np.asarray(u).reshape(3, self.nz, self.plane)
        idx = self.local_planes()
        return rho[idx].reshape(-1), u[:, idx].reshape(3, -1)

    def owned(self, local_array, comps):
        """Owned planes of a local (comps, nzl + 2 planes) array."""
        a = np.asarray(local_array).reshape(comps, self.nzl + 2, self.plane)
        return a[:, 1:self.nzl + 1].reshape(comps, -1)

    # stepping ------------------------------------------------------------------
    def _exchange(self, phase):
        pop = self.sim.raw_populations()
        sends, recvs = messages(self.nzl, phase)
        if self.world == 1:
            # the slab is its own neighbour on both sides: match each send with
            # the receive of the opposite end
            for (to, pops, src), (fr, pops2, dst) in zip(sends, recvs):
                assert fr == _peer_of(to) and pops == pops2
                planes_view(pop, pops, dst, self.plane).copy_(planes_view(pop, pops, src, self.plane))
            return
        if self.transport is None:
            raise ValueError("a slab of a decomposed grid steps through a transport or a LocalGroup")
        ops = []
        for to, pops, pl in sends:
            for k, j in enumerate(pops):
                ops.append(("send", plane_view(pop, j, pl, self.plane), self.peers[to], _tag(phase, to, k)))
        for fr, pops, pl in recvs:
            for k, j in enumerate(pops):
                # the message comes from the neighbour on side `fr`, which sent it towards the other side
                ops.append(("recv", plane_view(pop, j, pl, self.plane), self.peers[fr], _tag(phase, _peer_of(fr), k)))
        self.transport.run(ops)

    def refresh_ghosts(self):
        """Before reading the slab's state (populations, fields, totals) after an
        even sweep: in the odd-parity layout some populations of boundary nodes
        sit in the ghost planes, which the next odd sweep's exchange would fill;
        this does that exchange now (repeating it later is harmless)."""
        if self.sim.step_count & 1:
            self._exchange("pre")

    def step(self, n=1, sweep=None):
        """n steps; sweep() runs one sweep of the slab (default sim.step(1); e.g.
        sim.step_totals_async to log totals), with the exchanges around odd ones."""
        sweep = sweep or (lambda: self.sim.step(1))
        for _ in range(int(n)):
            odd = self.sim.step_count & 1
            if odd:
                self._exchange("pre")
            sweep()
            if odd:
                self._exchange("post")


class TorchTransport:
    """Point-to-point plane exchange through torch.distributed (NCCL between GPUs,
    gloo on CPU): every message of one exchange is posted in one batch, then
    waited for.  On a GPU the waits order the exchange on the current stream, so
    call it with the sweeps' stream current."""

    def __init__(self, dist):
        self.dist = dist

    def run(self, ops):
        d = self.dist
        p2p = [d.P2POp(d.isend if kind == "send" else d.irecv, t, peer, tag=tag) for kind, t, peer, tag in ops]
        for req in d.batch_isend_irecv(p2p):
            req.wait()


class LocalGroup:
    """All slabs of one grid in one process, stepped in lockstep; an exchange is
    one copy per population and plane from the sender's buffer to the
    receiver's.  The slabs share one stream (or run on the host), so the copies
    are ordered between the sweeps."""

    def __init__(self, runs):
        self.runs = list(runs)
        self.world = len(self.runs)

    def _exchange(self, phase):
        pops_of = [r.sim.raw_populations() for r in self.runs]
        for r, run in enumerate(self.runs):
            sends, _ = messages(run.nzl, phase)
            for to, pops, src in sends:
                peer = self.runs[run.peers[to]]
                _, precv = messages(peer.nzl, phase)
                # the peer receives from the side we are on
                fr = _peer_of(to)
                (dst,) = [pl for side, pp, pl in precv if side == fr and pp == pops]
                planes_view(pops_of[peer.rank], pops, dst, peer.plane).copy_(
                    planes_view(pops_of[r], pops, src, run.plane))

    def refresh_ghosts(self):
        """As SlabRun.refresh_ghosts, for every slab."""
        if self.runs[0].sim.step_count & 1:
            self._exchange("pre")

    def step(self, n=1):
        for _ in range(int(n)):
            odd = self.runs[0].sim.step_count & 1
            if odd:
                self._exchange("pre")
            for run in self.runs:
                run.sim.step(1)
            if odd:
                self._exchange("post")
