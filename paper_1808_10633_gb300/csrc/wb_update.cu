// wb_update.cu -- per-cell stage update: flux difference of the WENO face
// fluxes (Sec. 2.2: the fluxes "rotated back" and the update performed),
// constrained transport of the face-centred field on the staggered mesh
// (Sec. 2.1), and the Runge-Kutta stage combination.
//
// Two kernels per stage.  emf_kernel: one thread per cell forms the three
// edge EMFs at the cell's own edge index (E_x at (i, j-1/2, k-1/2), E_y at
// (i-1/2, j, k-1/2), E_z at (i-1/2, j-1/2, k)), each from the stored face
// fluxes:
//   E_z(i-1/2, j-1/2) from -F_x(B_y) on the two x faces and F_y(B_x) on the
//   two y faces next to the edge, and cyclically for E_x, E_y;
//   emf_mode 0: E = 1/2 (sum of the 4 face values) - 1/4 (sum of the 4 cell
//   values of -v x B), which reduces to the 1-D upwind flux for flow that
//   does not vary across the edge; emf_mode 1: E = 1/4 (sum of the 4 face
//   values).
// update_kernel: one thread per cell updates the cell's (rho, m, E) and its
// three lower faces (bx at i-1/2, by at j-1/2, bz at k-1/2).  Face rates are
// -curl E by Stokes' theorem on each face (four edge EMFs per face), so the
// face divergence of b is unchanged to round-off.  Forming every EMF once
// (instead of nine times per cell inside the update) keeps the update's loads
// few and independent, so it runs near HBM bandwidth.
#include "wb_internal.h"

namespace wb {
namespace {

// Cell (i, j, k) of patch p, where an index one step outside the patch
// wraps round a periodic patch or, with LINKED, reaches the neighbouring
// patch through the link table.
template <class T, bool LINKED>
struct Geo {
    const PatchDev P;
    const PatchDev* __restrict__ patches;
    const int* __restrict__ links;
    int p;
    __device__ __forceinline__ long long at(int i, int j, int k) const {
        if constexpr (LINKED) {
            return locate(patches, links, p, P, i, j, k);
        } else {
            i = i < 0 ? i + P.nx : (i >= P.nx ? i - P.nx : i);
            j = j < 0 ? j + P.ny : (j >= P.ny ? j - P.ny : j);
            k = k < 0 ? k + P.nz : (k >= P.nz ? k - P.nz : k);
            return P.off + ((long long)k * P.ny + j) * P.nx + i;
        }
    }
};

// Flux array layout per axis: rho, mx, my, mz, E, B_t1, B_t2 with
// (t1, t2) = (y, z) for x faces, (z, x) for y faces, (x, y) for z faces.
// EMF at the edge of cell-index (i, j, k): E_z at (i-1/2, j-1/2, k).
template <class T, bool LINKED>
__device__ __forceinline__ T emf_z(const UpdateArgs<T>& A, const Geo<T, LINKED>& G, int i, int j, int k) {
    const long long N = A.ncells;
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const int im = i - 1, jm = j - 1;
    const long long c = G.at(i, j, k), cjm = G.at(i, jm, k), cim = G.at(im, j, k);
    const T fsum = -Fx[5 * N + cjm] - Fx[5 * N + c] + Fy[6 * N + cim] + Fy[6 * N + c];
    if (A.emf_mode == 1) return T(0.25) * fsum;
    const T* __restrict__ Er = A.er + 2 * N;
    const T esum = Er[G.at(im, jm, k)] + Er[cjm] + Er[cim] + Er[c];
    return T(0.5) * fsum - T(0.25) * esum;
}

// E_y at (i-1/2, j, k-1/2)
template <class T, bool LINKED>
__device__ __forceinline__ T emf_y(const UpdateArgs<T>& A, const Geo<T, LINKED>& G, int i, int j, int k) {
    const long long N = A.ncells;
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fz = A.flux + 14 * N;
    const int im = i - 1, km = k - 1;
    const long long c = G.at(i, j, k), ckm = G.at(i, j, km), cim = G.at(im, j, k);
    const T fsum = Fx[6 * N + ckm] + Fx[6 * N + c] - Fz[5 * N + cim] - Fz[5 * N + c];
    if (A.emf_mode == 1) return T(0.25) * fsum;
    const T* __restrict__ Er = A.er + N;
    const T esum = Er[G.at(im, j, km)] + Er[ckm] + Er[cim] + Er[c];
    return T(0.5) * fsum - T(0.25) * esum;
}

// E_x at (i, j-1/2, k-1/2)
template <class T, bool LINKED>
__device__ __forceinline__ T emf_x(const UpdateArgs<T>& A, const Geo<T, LINKED>& G, int i, int j, int k) {
    const long long N = A.ncells;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    const int jm = j - 1, km = k - 1;
    const long long c = G.at(i, j, k), ckm = G.at(i, j, km), cjm = G.at(i, jm, k);
    const T fsum = -Fy[5 * N + ckm] - Fy[5 * N + c] + Fz[6 * N + cjm] + Fz[6 * N + c];
    if (A.emf_mode == 1) return T(0.25) * fsum;
    const T* __restrict__ Er = A.er;
    const T esum = Er[G.at(i, jm, km)] + Er[ckm] + Er[cjm] + Er[c];
    return T(0.5) * fsum - T(0.25) * esum;
}

// Stage combination for one value.
//   SSP-RK3: stage 0: un + dt L; 1: 3/4 un + 1/4 (uk + dt L);
//            2: 1/3 un + 2/3 (uk + dt L).
//   RK4 (acc = running un + dt/6 sum w_i k_i):
//            stage 0: acc = un + dt/6 L, out = un + dt/2 L;
//            stage 1: acc += dt/3 L, out = un + dt/2 L;
//            stage 2: acc += dt/3 L, out = un + dt L;
//            stage 3: out = acc + dt/6 L.
template <class T>
__device__ __forceinline__ T combine(const UpdateArgs<T>& A, long long o, T L, T dt) {
    const T un = A.un[o];
    if (A.integrator == 0) {
        if (A.stage == 0) return un + dt * L;
        const T uk = A.uk[o];
        if (A.stage == 1) return T(0.75) * un + T(0.25) * (uk + dt * L);
        return T(1.0 / 3.0) * un + T(2.0 / 3.0) * (uk + dt * L);
    }
    const T dt6 = dt * T(1.0 / 6.0);
    if (A.stage == 0) { A.acc[o] = un + dt6 * L; return un + T(0.5) * dt * L; }
    if (A.stage == 1) { A.acc[o] = A.acc[o] + T(2) * dt6 * L; return un + T(0.5) * dt * L; }
    if (A.stage == 2) { A.acc[o] = A.acc[o] + T(2) * dt6 * L; return un + dt * L; }
    return A.acc[o] + dt6 * L;
}

template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock) emf_kernel(const UpdateArgs<T> A) {
    const CellBlock cb = A.blocks[blockIdx.x];
    const Geo<T, LINKED> G{A.patches[cb.x], A.patches, A.links, cb.x};
    const int local = cb.y + threadIdx.x;
    const int nxy = G.P.nx * G.P.ny;
    if (local >= nxy * G.P.nz) return;
    const int k = local / nxy;
    const int rem = local - k * nxy;
    const int j = rem / G.P.nx;
    const int i = rem - j * G.P.nx;
    const long long N = A.ncells;
    const long long c = G.P.off + local;
    A.emf[c] = emf_x(A, G, i, j, k);
    A.emf[N + c] = emf_y(A, G, i, j, k);
    A.emf[2 * N + c] = emf_z(A, G, i, j, k);
}

template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock, 4) update_kernel(const UpdateArgs<T> A) {
    const CellBlock cb = A.blocks[blockIdx.x];
    const Geo<T, LINKED> G{A.patches[cb.x], A.patches, A.links, cb.x};
    const int local = cb.y + threadIdx.x;
    const int nxy = G.P.nx * G.P.ny;
    if (local >= nxy * G.P.nz) return;
    const int k = local / nxy;
    const int rem = local - k * nxy;
    const int j = rem / G.P.nx;
    const int i = rem - j * G.P.nx;
    const long long N = A.ncells;
    const long long c = G.P.off + local;
    const long long cx = G.at(i + 1, j, k);
    const long long cy = G.at(i, j + 1, k);
    const long long cz = G.at(i, j, k + 1);
    const T dt = T(*A.dt);
    const T idx = T(A.idx), idy = T(A.idy), idz = T(A.idz);
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;

    // (rho, mx, my, mz, E): L = -sum_d (F_d(c + e_d) - F_d(c)) / dx_d, x then y then z
#pragma unroll
    for (int q = 0; q < 5; q++) {
        const long long o = q * N;
        T L = T(0);
        L -= (Fx[o + cx] - Fx[o + c]) * idx;
        L -= (Fy[o + cy] - Fy[o + c]) * idy;
        L -= (Fz[o + cz] - Fz[o + c]) * idz;
        A.dst[o + c] = combine(A, o + c, L, dt);
    }
    // faces: -curl E
    const T* __restrict__ Ex = A.emf;
    const T* __restrict__ Ey = A.emf + N;
    const T* __restrict__ Ez = A.emf + 2 * N;
    const T ex = Ex[c], ey = Ey[c], ez = Ez[c];
    const T Lbx = -((Ez[cy] - ez) * idy - (Ey[cz] - ey) * idz);
    const T Lby = -((Ex[cz] - ex) * idz - (Ez[cx] - ez) * idx);
    const T Lbz = -((Ey[cx] - ey) * idx - (Ex[cy] - ex) * idy);
    A.dst[5 * N + c] = combine(A, 5 * N + c, Lbx, dt);
    A.dst[6 * N + c] = combine(A, 6 * N + c, Lby, dt);
    A.dst[7 * N + c] = combine(A, 7 * N + c, Lbz, dt);
}

}  // namespace

template <class T>
cudaError_t launch_emf(const UpdateArgs<T>& a, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (a.links) emf_kernel<T, true><<<nblocks, kCellBlock, 0, s>>>(a);
    else emf_kernel<T, false><<<nblocks, kCellBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_update(const UpdateArgs<T>& a, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (a.links) update_kernel<T, true><<<nblocks, kCellBlock, 0, s>>>(a);
    else update_kernel<T, false><<<nblocks, kCellBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_emf<float>(const UpdateArgs<float>&, int, cudaStream_t);
template cudaError_t launch_emf<double>(const UpdateArgs<double>&, int, cudaStream_t);
template cudaError_t launch_update<float>(const UpdateArgs<float>&, int, cudaStream_t);
template cudaError_t launch_update<double>(const UpdateArgs<double>&, int, cudaStream_t);

}  // namespace wb
