"""Cell-ordered particle storage (Sections 2.1 and 2.3.1).

Particles are stored sorted by their parent coarse cell; a particle's cell is
implied by its index and the per-cell counts rho_c: particle i is in cell c
iff offset[c] <= i < offset[c+1], offset = exclusive prefix sum of the counts
in storage order.

Storage order of coarse cells (a reading; the paper fixes only "the same
memory layout as rho_c"): the N_c^3 cells are grouped into cubic bricks of
B^3 cells; bricks are ordered x-fastest, and cells inside a brick are
x-fastest.  B = N_c gives plain x-fastest order.
"""
import numpy as np


def auto_brick(n_coarse):
    """Default brick side: 4, else 2, else 1 -- the largest that divides N_c
    and leaves at least three bricks per side."""
    for b in (4, 2, 1):
        if n_coarse % b == 0 and n_coarse // b >= 3:
            return b
    raise ValueError("need at least 3 coarse cells per side")


def storage_index(cx, cy, cz, n_coarse, brick):
    """Storage rank of coarse cell (cx, cy, cz) (periodically wrapped)."""
    nb = n_coarse // brick
    cx = np.mod(cx, n_coarse)
    cy = np.mod(cy, n_coarse)
    cz = np.mod(cz, n_coarse)
    bx, by, bz = cx // brick, cy // brick, cz // brick
    lx, ly, lz = cx % brick, cy % brick, cz % brick
    b = bx + nb * (by + nb * bz)
    loc = lx + brick * (ly + brick * lz)
    return (b * brick ** 3 + loc).astype(np.int64)


def cell_coords(index, n_coarse, brick):
    """Inverse of storage_index: (cx, cy, cz) of storage rank `index`."""
    index = np.asarray(index, dtype=np.int64)
    nb = n_coarse // brick
    b, loc = index // brick ** 3, index % brick ** 3
    lx, ly, lz = loc % brick, (loc // brick) % brick, loc // (brick * brick)
    bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
    return bx * brick + lx, by * brick + ly, bz * brick + lz


def offsets_from_counts(counts):
    """Exclusive prefix sum (length N_cc + 1)."""
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


def particle_cells(counts):
    """Storage rank of the cell of every stored particle (cell-ordered format)."""
    return np.repeat(np.arange(len(counts), dtype=np.int64), counts)


def stable_order(keys):
    """Permutation that sorts `keys` and keeps equal keys in their input order
    (numpy's stable argsort)."""
    return np.argsort(np.asarray(keys, dtype=np.int64), kind="stable")
