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
This module holds no compute of the stencil itself: the caller applies its
own dslash to the extended slab.
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


def _exchange(lo_send: np.ndarray, hi_send: np.ndarray, rank: int, world: int):
    """Send lo_send to the lower neighbour and hi_send to the upper one;
    return (from the lower neighbour, from the upper neighbour)."""
    if world == 1:
        return hi_send.copy(), lo_send.copy()
    import torch
    import torch.distributed as dist
    down, up = (rank - 1) % world, (rank + 1) % world
    t_lo = torch.from_numpy(np.ascontiguousarray(lo_send).view(np.float64).copy())
    t_hi = torch.from_numpy(np.ascontiguousarray(hi_send).view(np.float64).copy())
    r_lo, r_hi = torch.empty_like(t_hi), torch.empty_like(t_lo)
    # tag 0: a lower halo travelling up; tag 1: an upper halo travelling down
    # (with two ranks the lower and upper neighbour are the same rank)
    reqs = [dist.isend(t_lo, down, tag=1), dist.isend(t_hi, up, tag=0),
            dist.irecv(r_lo, down, tag=0), dist.irecv(r_hi, up, tag=1)]
    for q in reqs:
        q.wait()
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
