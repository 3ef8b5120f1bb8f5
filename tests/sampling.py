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


def bf16(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def learned_params_as_run(params):
    """The network parameters as the tensor-core sweep uses them: it stores
    the first layer (weights and bias, the bias fed as a weight) times
    k = 0.851 in BF16, the hidden weights halved in BF16, the hidden bias
    times k in FP32, the output weights divided by 2 k in BF16 and the output
    bias in FP32 (the GELU's argument constant folded into the weights); the
    values returned are those divided back by the same factors."""
    from oracle import learned as Lr

    k = np.float32(0.851)
    p32 = np.asarray(params, np.float32).reshape(7, Lr.NPARAM)
    P = np.asarray(params, np.float64).reshape(7, Lr.NPARAM).copy()
    n1 = 32 * 6 + 32                                   # W1 and b1
    P[:, :n1] = bf16(p32[:, :n1] * k) / np.float64(k)
    o2 = n1
    P[:, o2:o2 + 32 * 32] = bf16(p32[:, o2:o2 + 32 * 32] * np.float32(0.5)) * 2.0
    ob2 = o2 + 32 * 32
    P[:, ob2:ob2 + 32] = (p32[:, ob2:ob2 + 32] * k).astype(np.float64) / np.float64(k)
    o3 = ob2 + 32
    k2 = np.float32(2.0) * k
    P[:, o3:o3 + 3 * 32] = bf16(p32[:, o3:o3 + 3 * 32] / k2) * np.float64(k2)
    return P


def oracle_face_flux_learned(st, axis, i, j, k, P, kappa, pjump, margins=None, smooth=0.0):
    """Learned-weight eq. FWENO flux through the lower face of cell (i, j, k)
    (library component order), from the FP64 reference network."""
    from oracle import learned as Lr

    n, t1, t2 = axis, (axis + 1) % 3, (axis + 2) % 3
    perm = [0, 1 + n, 1 + t1, 1 + t2, 4 + n, 4 + t1, 4 + t2, 7]
    dims = st.dims
    Us = np.empty((6, 8))
    for m in range(6):
        q = [i, j, k]
        q[axis] = (q[axis] + m - 3) % dims[axis]
        Us[m] = st.U[perm, q[2], q[1], q[0]]
    Fh = Lr.interface_flux_learned(Us, st.gamma, P, kappa, pjump, margins, smooth=smooth)
    r = np.empty(7)
    r[0] = Fh[0]
    for gq in range(3):
        r[1 + gq] = Fh[perm.index(1 + gq)]
    r[4], r[5], r[6] = Fh[7], Fh[5], Fh[6]
    return r
