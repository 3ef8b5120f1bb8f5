"""Single-interface oracle values for sampled comparisons at full size."""
import numpy as np


def oracle_face_flux(orc, st, axis, i, j, k):
    """Oracle eq. FWENO flux through the lower face of cell (i, j, k) along
    axis, in the library's component order (rho, mx, my, mz, E, B_t1, B_t2)."""
    n, t1, t2 = axis, (axis + 1) % 3, (axis + 2) % 3
    perm = [0, 1 + n, 1 + t1, 1 + t2, 4 + n, 4 + t1, 4 + t2, 7]
    nx, ny, nz = st.dims
    dims = (nx, ny, nz)
    Us = np.empty((6, 8))
    for m in range(6):
        q = [i, j, k]
        q[axis] = (q[axis] + m - 3) % dims[axis]
        Us[m] = st.U[perm, q[2], q[1], q[0]]
    Fh = orc.interface_flux(Us, st.gamma)
    out = np.empty(7)
    out[0] = Fh[0]
    for gq in range(3):
        out[1 + gq] = Fh[perm.index(1 + gq)]
    out[4] = Fh[7]
    out[5] = Fh[5]
    out[6] = Fh[6]
    return out
