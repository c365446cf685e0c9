"""Domain decomposition of the lattice along T: the host-side logic of the
multi-GPU layout (one T-slab per rank), which the paper names as its next
step (Sec. 6) and whose exchange follows its spin projection (Sec. 4.3,
App. B): a rank needs, per dslash, only the projected boundary spinors of its
two neighbours.

Each rank owns the slices t0 .. t0 + nt - 1 (nt even, so t0 is even and a
site's even-odd parity is the same locally and globally).  For the stencil it
needs one halo slice on each side:

* below (t0 - 1): for the backward hop (1 + s gamma_4) U_4^dag(x - 4) psi(x - 4)
  it receives P_+ psi = (1 + s gamma_4)/2 psi of the lower neighbour's last
  slice, and the link slice U_4(t0 - 1);
* above (t0 + nt): for the forward hop (1 - s gamma_4) U_4(x) psi(x + 4) it
  receives P_- psi = (1 - s gamma_4)/2 psi of the upper neighbour's first slice;

with s = +1 for D and -1 for D^dag.  Because P_{+-} is idempotent, applying the
hop's own projector (1 -+ s gamma_4) to the received P psi gives the same
result as applying it to psi: the projected face carries all the hop needs
and has rank 2 (12 reals per site instead of 24).  Across the global boundary
t = T - 1 <-> 0 an antiperiodic time direction multiplies the halo by -1.

The exchange uses torch.distributed point-to-point messages (gloo on CPU,
NCCL on GPUs); with one rank the halos are the rank's own opposite slices.

On the GPU (``SlabDslash``) the library packs the projected faces and runs the
stencil: faces are packed by a kernel (``wd_slab_pack_faces``), travel on a
communication stream into buffers in the receiving GPU's own memory, and the
interior slices are computed while they travel (``wd_dslash_slab`` region 0);
the two boundary slices follow once the halos have arrived (region 1).  The
numpy functions below are the host-side form of the same exchange, used with
the CPU oracle.
"""
from __future__ import annotations

import numpy as np

# gamma_4 of the DeGrand-Rossi set (the host basis), read off the App. B projectors
GAMMA4_DR = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=np.complex128)


def slab_range(T: int, world: int, rank: int) -> tuple[int, int]:
    """(t0, nt) of a rank's slab; T must split into even slabs."""
    if T % world or (T // world) % 2:
        raise ValueError(f"T = {T} does not split into {world} slabs of even thickness")
    nt = T // world
    return rank * nt, nt


def face_projector(sign: int) -> np.ndarray:
    """(1 + sign gamma_4) / 2, a rank-2 projector on spin."""
    return 0.5 * (np.eye(4) + sign * GAMMA4_DR)


def project(face: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to a slice (sites, 4, 3)."""
    return np.einsum("ab,sbc->sac", P, face)


def halo_signs(rank: int, world: int, antiperiodic: bool) -> tuple[float, float]:
    """Sign of the lower and upper halo: -1 where the halo crosses t = T-1 <-> 0."""
    lo = -1.0 if (antiperiodic and rank == 0) else 1.0
    hi = -1.0 if (antiperiodic and rank == world - 1) else 1.0
    return lo, hi


def exchange_faces(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None) -> None:
    """Move torch tensors between time neighbours: send_lo (my first slice's
    face) to the lower neighbour, where it arrives as its recv_hi; send_hi (my
    last slice's face) to the upper neighbour, where it arrives as its
    recv_lo.  One rank: the halos are my own opposite faces (a copy).

    The messages are posted in one fixed order on every rank -- upward (hi to
    the upper neighbour, lo halo from the lower one), then downward -- with
    tag 0 for the upward and 1 for the downward direction.  Backends that
    match point-to-point messages between a pair of ranks in posting order
    (NCCL) then pair them correctly even with two ranks, where the lower and
    upper neighbour are the same rank; gloo matches on the tags.  Returns once
    the transfers are complete (CPU tensors) or, for CUDA tensors, once the
    current stream is ordered after them."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist
    down, up = (rank - 1) % world, (rank + 1) % world
    ops = [dist.P2POp(dist.isend, send_hi, up, group, tag=0), dist.P2POp(dist.irecv, recv_lo, down, group, tag=0),
           dist.P2POp(dist.isend, send_lo, down, group, tag=1), dist.P2POp(dist.irecv, recv_hi, up, group, tag=1)]
    for q in dist.batch_isend_irecv(ops):
        q.wait()


def send_up(send, recv, rank: int, world: int, group=None) -> None:
    """send (my last slice's link face) to the upper neighbour; recv <- the
    lower neighbour's.  One rank: a copy."""
    if world == 1:
        recv.copy_(send)
        return
    import torch.distributed as dist
    down, up = (rank - 1) % world, (rank + 1) % world
    ops = [dist.P2POp(dist.isend, send, up, group, tag=2), dist.P2POp(dist.irecv, recv, down, group, tag=2)]
    for q in dist.batch_isend_irecv(ops):
        q.wait()


def _exchange(lo_send: np.ndarray, hi_send: np.ndarray, rank: int, world: int):
    """numpy form of exchange_faces: returns (from the lower neighbour, from
    the upper neighbour)."""
    import torch
    t_lo = torch.from_numpy(np.ascontiguousarray(lo_send).view(np.float64).copy())
    t_hi = torch.from_numpy(np.ascontiguousarray(hi_send).view(np.float64).copy())
    r_lo, r_hi = torch.empty_like(t_hi), torch.empty_like(t_lo)
    exchange_faces(t_lo, t_hi, r_lo, r_hi, rank, world)
    shape = lo_send.shape
    return r_lo.numpy().view(np.complex128).reshape(shape), r_hi.numpy().view(np.complex128).reshape(shape)


def spinor_halos(psi_slab: np.ndarray, slice_sites: int, rank: int, world: int, dagger: bool = False,
                 antiperiodic: bool = False):
    """Projected halo slices of a (nt * slice_sites, 4, 3) slab: returns
    (below, above), each (slice_sites, 4, 3): below = sign P_+ psi of the lower
    neighbour's last slice, above = sign P_- psi of the upper neighbour's first."""
    s = -1 if dagger else 1
    first, last = psi_slab[:slice_sites], psi_slab[-slice_sites:]
    # what the upper neighbour needs from me (its lower halo) and the lower one (its upper halo)
    to_up = project(last, face_projector(+s))
    to_down = project(first, face_projector(-s))
    below, above = _exchange(to_down, to_up, rank, world)
    lo_sign, hi_sign = halo_signs(rank, world, antiperiodic)
    return lo_sign * below, hi_sign * above


def link_halo(U_slab: np.ndarray, slice_sites: int, rank: int, world: int) -> np.ndarray:
    """The lower neighbour's last link slice (slice_sites, 4, 3, 3): the
    backward temporal hop of the first local slice uses U_4(t0 - 1)."""
    below, _ = _exchange(U_slab[:slice_sites], U_slab[-slice_sites:], rank, world)
    return below


def extended_parity(global_parity: int, t0: int) -> int:
    """Parity, in the extended slab (one halo slice below), of a site of the
    given global parity: the local time index is t - t0 + 1."""
    return global_parity ^ ((1 - t0) & 1)


class SlabDslash:
    """The dslash of one rank's T-slab on its GPU, with the face exchange.

    ``wd`` is the rank's ``WilsonDirac`` context, created with the slab's dims
    ``(X, Y, Z, nt)`` and loaded with the slab's links; ``rank`` / ``world``
    place the slab at t0 = rank * nt of a lattice of T = world * nt slices.
    With ``world`` > 1 the faces travel by torch.distributed (the process
    group must be initialised: NCCL for CUDA tensors).  One apply():

    1. pack both projected faces of the input (library stream);
    2. on the communication stream, after the pack: exchange the faces into
       this GPU's halo buffers;
    3. meanwhile, on the library stream: the interior slices (region 0);
    4. the library stream waits for the exchange, then the two boundary
       slices (region 1).
    """

    def __init__(self, wd, rank: int, world: int, t_antiperiodic: bool = False, group=None, overlap: bool = True):
        import torch
        self.wd, self.rank, self.world, self.group = wd, rank, world, group
        self.torch = torch
        lo_sign, hi_sign = halo_signs(rank, world, t_antiperiodic)
        self.flip_lo, self.flip_hi = lo_sign < 0, hi_sign < 0
        self.overlap = overlap
        self.comm = torch.cuda.Stream() if overlap else wd.stream
        self._faces = {}
        self._links = {}

    def _buf(self, n):
        return self.torch.empty(n, dtype=self.torch.uint8, device="cuda")

    def faces(self, prec: int):
        """(send_lo, send_hi, halo_lo, halo_hi) device buffers of one precision."""
        if prec not in self._faces:
            n = self.wd.slab_face_bytes(prec)
            self._faces[prec] = tuple(self._buf(n) for _ in range(4))
        return self._faces[prec]

    def link_halo(self, prec: int):
        """The lower neighbour's link face (exchanged once per precision)."""
        if prec not in self._links:
            n = self.wd.slab_link_face_bytes(prec)
            send, recv = self._buf(n), self._buf(n)
            self.wd.slab_pack_link_face(send, prec)
            s = self.wd.stream
            with self.torch.cuda.stream(s):
                send_up(send, recv, self.rank, self.world, self.group)
            self._links[prec] = (send, recv)
        return self._links[prec][1]

    def apply(self, out, inp, out_parity: int, dagger: bool, prec: int):
        torch = self.torch
        wd, s = self.wd, self.wd.stream
        link = self.link_halo(prec)
        send_lo, send_hi, halo_lo, halo_hi = self.faces(prec)
        wd.slab_pack_faces(send_lo, send_hi, inp, dagger, prec)
        packed = torch.cuda.Event()
        packed.record(s)
        with torch.cuda.stream(self.comm):
            self.comm.wait_event(packed)
            exchange_faces(send_lo, send_hi, halo_lo, halo_hi, self.rank, self.world, self.group)
            arrived = torch.cuda.Event()
            arrived.record(self.comm)
        wd.dslash_slab(out, inp, None, None, None, False, False, out_parity, dagger, prec, 0)
        s.wait_event(arrived)
        wd.dslash_slab(out, inp, halo_lo, halo_hi, link, self.flip_lo, self.flip_hi, out_parity, dagger, prec, 1)
