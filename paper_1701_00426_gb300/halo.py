"""Host-side logic of a t-slab decomposition of the even/odd lattice over
ranks: which sites a rank owns, which face it exchanges with each neighbour
per D_eo / D_oe application, where the antiperiodic boundary falls in a
rank's slab, and a rank-ordered FP64 sum for the two reductions of a CG
iteration (<p, q> and ||r||^2).

Layout fact this rests on (half index of Eq. lexicographic_eo, t = x3 the
slowest coordinate): the sites of either parity in the t-slices [ta, tb)
are exactly the half indices [ta S/2, tb S/2), S = N0 N1 N2, in the same
order for every slice.  So a rank's part of a field is one contiguous range,
a face is one contiguous block of S/2 sites, and the exchange is one plain
copy each way with no gather or scatter.  Links, in the full lexicographic
order [4][V][3][3], slice the same way with S sites per slice.

A rank's extended slab has GHOST = 2 slices on each side: with an even slab
extent nt, t0 - GHOST is even, so a site's parity in the extended slab is
its global parity and the half-index order within a slice is the global one.
The D_eo / D_oe hops of the nt owned slices reach only the innermost ghost
slice on each side, which is what the exchange fills; the outer ghost slices
stay zero.

Nothing here touches a GPU.  Every machine this code runs on has one GPU, so
the exchange is exercised by CPU ranks over torch.distributed (gloo)."""
from __future__ import annotations

import numpy as np

GHOST = 2


def check_slab(dims, world: int) -> int:
    """Slab extent nt = Lt / world; it must be even and >= 2 (parity of the
    slab origin) and divide Lt."""
    Lt = int(dims[3])
    if world < 1 or Lt % world:
        raise ValueError(f"Lt = {Lt} is not divisible by {world} ranks")
    nt = Lt // world
    if nt < 2 or nt % 2:
        raise ValueError(f"slab extent {nt} must be even and >= 2")
    return nt


def slab(dims, world: int, rank: int) -> tuple[int, int]:
    """(t0, nt): rank owns the global t-slices [t0, t0 + nt)."""
    nt = check_slab(dims, world)
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank * nt, nt


def slice_sites(dims) -> int:
    """S = N0 N1 N2: sites per t-slice (S/2 per parity)."""
    return int(dims[0]) * int(dims[1]) * int(dims[2])


def half_range(dims, ta: int, tb: int) -> tuple[int, int]:
    """Half-index range of the sites of either parity in t-slices [ta, tb)."""
    h = slice_sites(dims) // 2
    return ta * h, tb * h


def ext_dims(dims, world: int) -> tuple[int, int, int, int]:
    """Dimensions of a rank's extended slab (owned slices + ghosts)."""
    return (int(dims[0]), int(dims[1]), int(dims[2]), check_slab(dims, world) + 2 * GHOST)


def local_part(field, dims, world: int, rank: int) -> np.ndarray:
    """The rank's slices of a global half field [Vh][3] (a view)."""
    t0, nt = slab(dims, world, rank)
    lo, hi = half_range(dims, t0, t0 + nt)
    return field[lo:hi]


def extended_links(links, dims, world: int, rank: int) -> np.ndarray:
    """Links [4][V_ext][3][3] of the extended slab: global slices
    t0 - GHOST .. t0 + nt + GHOST - 1, periodic in t.  Links are static
    during a solve, so a rank holds its ghost links once; nothing is
    exchanged per iteration."""
    t0, nt = slab(dims, world, rank)
    S, Lt = slice_sites(dims), int(dims[3])
    U = np.asarray(links).reshape(4, Lt, S, 3, 3)
    ts = [(t0 - GHOST + k) % Lt for k in range(nt + 2 * GHOST)]
    return np.ascontiguousarray(U[:, ts]).reshape(4, len(ts) * S, 3, 3)


def boundary_slices(dims, world: int, rank: int) -> list[int]:
    """Local slices of the extended slab, among those the owned sites' hops
    use (GHOST - 1 .. GHOST + nt), whose t-link U_3 is the global one at
    x3 = Lt - 1 and so carries the antiperiodic sign."""
    t0, nt = slab(dims, world, rank)
    Lt = int(dims[3])
    return [k for k in range(GHOST - 1, GHOST + nt + 1) if (t0 - GHOST + k) % Lt == Lt - 1]


def faces(local, dims, world: int) -> tuple[np.ndarray, np.ndarray]:
    """(bottom, top): the owned slices a rank sends down (to rank - 1, whose
    upper ghost it becomes) and up (to rank + 1, its lower ghost)."""
    h = slice_sites(dims) // 2
    nt = check_slab(dims, world)
    local = np.asarray(local)
    assert local.shape[0] == nt * h
    return local[:h], local[(nt - 1) * h:]


def exchange(local, dims, world: int, rank: int) -> tuple[np.ndarray, np.ndarray]:
    """Fill the innermost ghost slices of a half field: returns (lower,
    upper), the neighbours' faces (periodic in t).  One send and one receive
    each way; with one rank the faces wrap onto the rank itself."""
    bottom, top = faces(local, dims, world)
    if world == 1:
        return top.copy(), bottom.copy()
    import torch
    import torch.distributed as dist
    below, above = (rank - 1) % world, (rank + 1) % world

    def as_real(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy())

    lower = torch.empty_like(as_real(top))
    upper = torch.empty_like(as_real(bottom))
    reqs = [dist.isend(as_real(top), above), dist.isend(as_real(bottom), below),
            dist.irecv(lower, below), dist.irecv(upper, above)]
    for r in reqs:
        r.wait()
    return lower.numpy().view(np.complex128), upper.numpy().view(np.complex128)


def extend(local, lower, upper, dims, world: int) -> np.ndarray:
    """Extended half field: [zero][lower][owned slices][upper][zero]."""
    h = slice_sites(dims) // 2
    local = np.asarray(local)
    z = np.zeros((h * (GHOST - 1),) + local.shape[1:], local.dtype)
    return np.concatenate([z, lower, local, upper, z])


def interior(ext, dims, world: int) -> np.ndarray:
    """The owned slices of an extended half field."""
    h = slice_sites(dims) // 2
    nt = check_slab(dims, world)
    return ext[GHOST * h:(GHOST + nt) * h]


def ordered_sum(partial: float, world: int) -> float:
    """Sum of one FP64 partial per rank, added in rank order on every rank,
    so every rank holds the same bits whatever the arrival order."""
    if world == 1:
        return float(partial)
    import torch
    import torch.distributed as dist
    out = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(out, torch.tensor([float(partial)], dtype=torch.float64))
    s = 0.0
    for t in out:
        s += float(t[0])
    return s
