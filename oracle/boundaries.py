"""Non-periodic boundaries for the oracle -- TEST INFRASTRUCTURE ONLY.

Ghost cells, written plainly in numpy around the periodic stage of oracle.cpp.  A
direction whose boundary is not periodic is padded with two ghost cells on each side
(the PLM stencil reaches two cells), and the padded grid is stepped as a periodic one.
Before every stage the ghosts are refilled from the interior, direction by direction
(x, then y, then z, each over the full padded extent of the others, so edge and corner
ghosts come out consistent).  The wrap-around of the periodic stage only ever touches
ghost cells, whose results are discarded by the next refill.

Kinds (per direction, both sides):
  OUTFLOW    zero-gradient: a ghost cell copies the nearest interior cell (cell fields
             and the transverse face fields stored with it); the normal field on the
             ghost faces copies the boundary face.
  REFLECTING mirror image about the boundary face, with the normal momentum and the
             normal field reversed and everything else copied (a rigid, perfectly
             conducting wall: v_n = B_n = 0 on it).
The paper names outflow boundaries (Sec. 4.1, the spherical blast); the reflecting wall is
the usual mirror condition of Godunov MHD codes.

Layout of a non-periodic direction d in the user arrays: n_d cells, and n_d + 1 faces for
the normal field B_d (faces i = 0 .. n_d, the last being the upper boundary face).  In the
padded arrays interior cell i is i + 2 and face i is face i + 2 (the lower face of cell
i + 2); faces 0, 1 and n_d + 3 are ghosts, face n_d + 2 is the upper boundary face.
"""
import numpy as np

PERIODIC, OUTFLOW, REFLECTING = 0, 1, 2
NG = 2

# numpy axis of direction d in the (nz, ny, nx) layout
AXIS = (2, 1, 0)


def _take(a, axis, idx):
    sl = [slice(None)] * 3
    sl[axis] = idx
    return a[tuple(sl)]


def _put(a, axis, idx, v):
    sl = [slice(None)] * 3
    sl[axis] = idx
    a[tuple(sl)] = v


def padded_shape(shape, bc):
    s = list(shape)
    for d in range(3):
        if bc[d] != PERIODIC:
            s[AXIS[d]] += 2 * NG
    return tuple(s)


def pad(fields, bc):
    """User layout (cell fields n, normal face field n + 1 along non-periodic d) -> padded
    arrays with zero ghosts; fill_ghosts makes them valid."""
    cell_shape = fields[0].shape
    out = []
    for f in range(8):
        a = np.asarray(fields[f], dtype=np.float64)
        p = np.zeros(padded_shape(cell_shape, bc))
        # interior cells i -> i + 2; along non-periodic d the normal field's n + 1 faces
        # -> padded faces 2 .. n + 2
        sl = [slice(None) if bc[AXIS.index(ax)] == PERIODIC else slice(NG, NG + a.shape[ax])
              for ax in range(3)]
        p[tuple(sl)] = a
        out.append(p)
    return out


def unpad(padded, bc, cell_shape):
    out = []
    for f in range(8):
        sl = []
        for ax in range(3):
            d = AXIS.index(ax)
            n = cell_shape[ax]
            if bc[d] == PERIODIC:
                sl.append(slice(None))
            elif f == 5 + d:
                sl.append(slice(NG, NG + n + 1))
            else:
                sl.append(slice(NG, NG + n))
        out.append(np.ascontiguousarray(padded[f][tuple(sl)]))
    return out


def fill_ghosts(u, bc):
    """Refill the ghost cells of a padded state (conserved or primitive: the only sign
    changes are of the normal momentum/velocity and the normal field) in place."""
    for d in range(3):
        kind = bc[d]
        if kind == PERIODIC:
            continue
        ax = AXIS[d]
        n = u[0].shape[ax] - 2 * NG          # interior cells along d
        lo_cells, hi_cells = (0, 1), (n + 2, n + 3)
        for f in range(8):
            a = u[f]
            normal_face = f == 5 + d
            flip = (f == 1 + d) or normal_face
            if kind == OUTFLOW:
                if normal_face:
                    for g in (0, 1):
                        _put(a, ax, g, _take(a, ax, 2))
                    _put(a, ax, n + 3, _take(a, ax, n + 2))
                else:
                    for g in lo_cells:
                        _put(a, ax, g, _take(a, ax, 2))
                    for g in hi_cells:
                        _put(a, ax, g, _take(a, ax, n + 1))
            else:  # REFLECTING
                s = -1.0 if flip else 1.0
                if normal_face:
                    # faces mirror about the boundary faces 2 and n + 2
                    _put(a, ax, 1, s * _take(a, ax, 3))
                    _put(a, ax, 0, s * _take(a, ax, 4))
                    _put(a, ax, n + 3, s * _take(a, ax, n + 1))
                else:
                    # cells mirror about the boundary faces: 1 <-> 2, 0 <-> 3, n+2 <-> n+1, n+3 <-> n
                    _put(a, ax, 1, s * _take(a, ax, 2))
                    _put(a, ax, 0, s * _take(a, ax, 3))
                    _put(a, ax, n + 2, s * _take(a, ax, n + 1))
                    _put(a, ax, n + 3, s * _take(a, ax, n))
    return u


def padded_lengths(lengths, cell_shape, bc):
    L = list(lengths)
    for d in range(3):
        if bc[d] != PERIODIC:
            n = cell_shape[AXIS[d]]
            L[d] = L[d] * (n + 2 * NG) / n
    return tuple(L)
