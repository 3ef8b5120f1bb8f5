// wb_update.cu -- per-cell stage update: flux difference of the WENO face
// fluxes (Sec. 2.2: the fluxes "rotated back" and the update performed),
// constrained transport of the face-centred field on the staggered mesh
// (Sec. 2.1), and the Runge-Kutta stage combination.
//
// Two kernels per stage.  The EMF kernel forms the three edge EMFs at each
// cell's own edge index (E_x at (i, j-1/2, k-1/2), E_y at (i-1/2, j, k-1/2),
// E_z at (i-1/2, j-1/2, k)), each from the stored face fluxes:
//   E_z(i-1/2, j-1/2) from -F_x(B_y) on the two x faces and F_y(B_x) on the
//   two y faces next to the edge, and cyclically for E_x, E_y;
//   emf_mode 0: E = 1/2 (sum of the 4 face values) - 1/4 (sum of the 4 cell
//   values of -v x B), which reduces to the 1-D upwind flux for flow that
//   does not vary across the edge; emf_mode 1: E = 1/4 (sum of the 4 face
//   values).
// The update kernel updates each cell's (rho, m, E) and its three lower faces
// (bx at i-1/2, by at j-1/2, bz at k-1/2).  Face rates are -curl E by Stokes'
// theorem on each face (four edge EMFs per face), so the face divergence of b
// is unchanged to round-off.
//
// Three forms of each kernel share the per-value arithmetic below (written
// with explicit roundings, so all give identical bits): for periodic patches
// whose x extent is a multiple of the vector width, one thread per 16-byte
// vector of cells along x (4 in FP32, 2 in FP64), which keeps four times the
// bytes in flight per thread on these bandwidth-bound kernels; otherwise (any
// patch, linked patches) two cells per thread with the loads of both issued
// before the first store (FP32), or one cell per thread (FP64, whose doubled
// registers would spill).
#include "wb_internal.h"

// FP32 grids whose per-cell kernels cannot use the vector forms run the
// two-cells-per-thread forms (0: one cell per thread)
#ifndef WB_UPDATE_PAIRS
#define WB_UPDATE_PAIRS 1
#endif

namespace wb {
namespace {

// ---- arithmetic with explicit rounding (no contraction) ---------------------
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// L = -sum_d (F_d(c + e_d) - F_d(c)) / dx_d, x then y then z
template <class T>
__device__ __forceinline__ T flux_rate(T fxp, T fxc, T fyp, T fyc, T fzp, T fzc, T idx, T idy, T idz) {
    T L = -rmul(rsub(fxp, fxc), idx);
    L = rsub(L, rmul(rsub(fyp, fyc), idy));
    return rsub(L, rmul(rsub(fzp, fzc), idz));
}

// Face rate -((Ea(c + e_a) - Ea(c)) / dx_a - (Eb(c + e_b) - Eb(c)) / dx_b)
template <class T>
__device__ __forceinline__ T face_rate(T ap, T ac, T ia, T bp, T bc, T ib) {
    return -rsub(rmul(rsub(ap, ac), ia), rmul(rsub(bp, bc), ib));
}

// Edge EMF from its four signed face values, fsum = ((s0 + s1) + s2) + s3,
// and the four cell values of -v x B.
template <class T>
__device__ __forceinline__ T edge_emf(T s0, T s1, T s2, T s3, T e0, T e1, T e2, T e3, int mode) {
    const T fsum = radd(radd(radd(s0, s1), s2), s3);
    if (mode == 1) return rmul(T(0.25), fsum);
    const T esum = radd(radd(radd(e0, e1), e2), e3);
    return rsub(rmul(T(0.5), fsum), rmul(T(0.25), esum));
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
__device__ __forceinline__ T combine_value(int integrator, int stage, T un, T uk, T& acc, T L, T dt) {
    if (integrator == 0) {
        if (stage == 0) return rfma(dt, L, un);
        const T s = rfma(dt, L, uk);
        if (stage == 1) return rfma(T(0.75), un, rmul(T(0.25), s));
        return rfma(T(1.0 / 3.0), un, rmul(T(2.0 / 3.0), s));
    }
    const T dt6 = rmul(dt, T(1.0 / 6.0));
    const T half = rmul(T(0.5), dt);
    if (stage == 0) { acc = rfma(dt6, L, un); return rfma(half, L, un); }
    if (stage == 1) { acc = rfma(rmul(T(2), dt6), L, acc); return rfma(half, L, un); }
    if (stage == 2) { acc = rfma(rmul(T(2), dt6), L, acc); return rfma(dt, L, un); }
    return rfma(dt6, L, acc);
}

// ---- one thread per cell -------------------------------------------------------

// Cell (i, j, k) of patch p, where an index one step outside the patch
// wraps round a periodic patch or, with LINKED, reaches the neighbouring
// patch through the link table.
template <class T, bool LINKED>
struct Geo {
    const PatchDev P;
    const PatchDev* __restrict__ patches;
    const int* __restrict__ links;
    int p;
    long long N;
    unsigned int* flag;
    __device__ __forceinline__ long long at(int i, int j, int k) const {
        if constexpr (LINKED) {
            return chk(locate(patches, links, p, P, i, j, k), N, flag);
        } else {
            i = i < 0 ? i + P.nx : (i >= P.nx ? i - P.nx : i);
            j = j < 0 ? j + P.ny : (j >= P.ny ? j - P.ny : j);
            k = k < 0 ? k + P.nz : (k >= P.nz ? k - P.nz : k);
            return chk(P.off + ((long long)k * P.ny + j) * P.nx + i, N, flag);
        }
    }
};

// Flux array layout per axis: rho, mx, my, mz, E, B_t1, B_t2 with
// (t1, t2) = (y, z) for x faces, (z, x) for y faces, (x, y) for z faces.
template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock) emf_kernel(const UpdateArgs<T> A) {
    const CellBlock cb = A.blocks[blockIdx.x];
    const Geo<T, LINKED> G{A.patches[cb.x], A.patches, A.links, cb.x, A.ncells, A.flag};
    const int local = cb.y + threadIdx.x;
    const int nxy = G.P.nx * G.P.ny;
    if (local >= nxy * G.P.nz) return;
    const int k = local / nxy;
    const int rem = local - k * nxy;
    const int j = rem / G.P.nx;
    const int i = rem - j * G.P.nx;
    const long long N = A.ncells;
    const long long c = chk(G.P.off + local, N, A.flag);
    const long long cim = G.at(i - 1, j, k), cjm = G.at(i, j - 1, k), ckm = G.at(i, j, k - 1);
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    const T* __restrict__ Er = A.er;
    const bool m0 = A.emf_mode == 0;
    // E_x at (i, j-1/2, k-1/2): -F_y(B_z) on y faces, F_z(B_y) on z faces
    A.emf[c] = edge_emf(-Fy[5 * N + ckm], -Fy[5 * N + c], Fz[6 * N + cjm], Fz[6 * N + c],
                        m0 ? Er[G.at(i, j - 1, k - 1)] : T(0), m0 ? Er[ckm] : T(0),
                        m0 ? Er[cjm] : T(0), m0 ? Er[c] : T(0), A.emf_mode);
    // E_y at (i-1/2, j, k-1/2): F_x(B_z) on x faces, -F_z(B_x) on z faces
    A.emf[N + c] = edge_emf(Fx[6 * N + ckm], Fx[6 * N + c], -Fz[5 * N + cim], -Fz[5 * N + c],
                            m0 ? Er[N + G.at(i - 1, j, k - 1)] : T(0), m0 ? Er[N + ckm] : T(0),
                            m0 ? Er[N + cim] : T(0), m0 ? Er[N + c] : T(0), A.emf_mode);
    // E_z at (i-1/2, j-1/2, k): -F_x(B_y) on x faces, F_y(B_x) on y faces
    A.emf[2 * N + c] = edge_emf(-Fx[5 * N + cjm], -Fx[5 * N + c], Fy[6 * N + cim], Fy[6 * N + c],
                                m0 ? Er[2 * N + G.at(i - 1, j - 1, k)] : T(0), m0 ? Er[2 * N + cjm] : T(0),
                                m0 ? Er[2 * N + cim] : T(0), m0 ? Er[2 * N + c] : T(0), A.emf_mode);
}

// Two cells per thread (t and t + 128 of a 256-cell block), the loads of
// both issued before the first store; the same arithmetic as emf_kernel.
template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock / 2) emf_kernel2(const UpdateArgs<T> A) {
    constexpr int H = kCellBlock / 2;
    const CellBlock cb = A.blocks[blockIdx.x];
    const Geo<T, LINKED> G{A.patches[cb.x], A.patches, A.links, cb.x, A.ncells, A.flag};
    const int nxy = G.P.nx * G.P.ny, np = nxy * G.P.nz;
    const int local0 = cb.y + threadIdx.x;
    if (local0 >= np) return;
    const bool has1 = local0 + H < np;
    const long long N = A.ncells;
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    const T* __restrict__ Er = A.er;
    const bool m0 = A.emf_mode == 0;
    long long c[2];
    T e[2][3];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int local = u == 1 && has1 ? local0 + H : local0;
        const int k = local / nxy;
        const int rem = local - k * nxy;
        const int j = rem / G.P.nx;
        const int i = rem - j * G.P.nx;
        c[u] = chk(G.P.off + local, N, A.flag);
        const long long cc = c[u];
        const long long cim = G.at(i - 1, j, k), cjm = G.at(i, j - 1, k), ckm = G.at(i, j, k - 1);
        e[u][0] = edge_emf(-Fy[5 * N + ckm], -Fy[5 * N + cc], Fz[6 * N + cjm], Fz[6 * N + cc],
                           m0 ? Er[G.at(i, j - 1, k - 1)] : T(0), m0 ? Er[ckm] : T(0),
                           m0 ? Er[cjm] : T(0), m0 ? Er[cc] : T(0), A.emf_mode);
        e[u][1] = edge_emf(Fx[6 * N + ckm], Fx[6 * N + cc], -Fz[5 * N + cim], -Fz[5 * N + cc],
                           m0 ? Er[N + G.at(i - 1, j, k - 1)] : T(0), m0 ? Er[N + ckm] : T(0),
                           m0 ? Er[N + cim] : T(0), m0 ? Er[N + cc] : T(0), A.emf_mode);
        e[u][2] = edge_emf(-Fx[5 * N + cjm], -Fx[5 * N + cc], Fy[6 * N + cim], Fy[6 * N + cc],
                           m0 ? Er[2 * N + G.at(i - 1, j - 1, k)] : T(0), m0 ? Er[2 * N + cjm] : T(0),
                           m0 ? Er[2 * N + cim] : T(0), m0 ? Er[2 * N + cc] : T(0), A.emf_mode);
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
        if (u == 1 && !has1) break;
#pragma unroll
        for (int d = 0; d < 3; d++) A.emf[d * N + c[u]] = e[u][d];
    }
}

template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock, 4) update_kernel(const UpdateArgs<T> A) {
    const CellBlock cb = A.blocks[blockIdx.x];
    const Geo<T, LINKED> G{A.patches[cb.x], A.patches, A.links, cb.x, A.ncells, A.flag};
    const int local = cb.y + threadIdx.x;
    const int nxy = G.P.nx * G.P.ny;
    if (local >= nxy * G.P.nz) return;
    const int k = local / nxy;
    const int rem = local - k * nxy;
    const int j = rem / G.P.nx;
    const int i = rem - j * G.P.nx;
    const long long N = A.ncells;
    const long long c = chk(G.P.off + local, N, A.flag);
    const long long cx = G.at(i + 1, j, k);
    const long long cy = G.at(i, j + 1, k);
    const long long cz = G.at(i, j, k + 1);
    const T dt = T(*A.dt);
    const T idx = T(A.idx), idy = T(A.idy), idz = T(A.idz);
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    T Lq[8];
#pragma unroll
    for (int q = 0; q < 5; q++) {
        const long long o = q * N;
        Lq[q] = flux_rate(Fx[o + cx], Fx[o + c], Fy[o + cy], Fy[o + c], Fz[o + cz], Fz[o + c], idx, idy, idz);
    }
    const T* __restrict__ Ex = A.emf;
    const T* __restrict__ Ey = A.emf + N;
    const T* __restrict__ Ez = A.emf + 2 * N;
    const T ex = Ex[c], ey = Ey[c], ez = Ez[c];
    Lq[5] = face_rate(Ez[cy], ez, idy, Ey[cz], ey, idz);
    Lq[6] = face_rate(Ex[cz], ex, idz, Ez[cx], ez, idx);
    Lq[7] = face_rate(Ey[cx], ey, idx, Ex[cy], ex, idy);
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const long long o = q * N + c;
        const T un = A.un[o];
        const T uk = A.stage > 0 && A.integrator == 0 ? A.uk[o] : T(0);
        T acc = A.integrator == 1 && A.stage > 0 ? A.acc[o] : T(0);
        const T out = combine_value(A.integrator, A.stage, un, uk, acc, Lq[q], dt);
        if (A.integrator == 1 && A.stage < 3) A.acc[o] = acc;
        A.dst[o] = out;
    }
}

// Two cells per thread (cells t and t + 128 of a 256-cell block): all loads
// of both cells are issued before the first store, so each thread keeps
// twice the bytes in flight of update_kernel (same arithmetic, same bits).
template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock / 2, 6) update_kernel2(const UpdateArgs<T> A) {
    constexpr int H = kCellBlock / 2;
    const CellBlock cb = A.blocks[blockIdx.x];
    const Geo<T, LINKED> G{A.patches[cb.x], A.patches, A.links, cb.x, A.ncells, A.flag};
    const int nxy = G.P.nx * G.P.ny, np = nxy * G.P.nz;
    const int local0 = cb.y + threadIdx.x;
    if (local0 >= np) return;
    const bool has1 = local0 + H < np;
    const long long N = A.ncells;
    long long c[2], cx[2], cy[2], cz[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int local = u == 1 && has1 ? local0 + H : local0;
        const int k = local / nxy;
        const int rem = local - k * nxy;
        const int j = rem / G.P.nx;
        const int i = rem - j * G.P.nx;
        c[u] = chk(G.P.off + local, N, A.flag);
        cx[u] = G.at(i + 1, j, k);
        cy[u] = G.at(i, j + 1, k);
        cz[u] = G.at(i, j, k + 1);
    }
    const T dt = T(*A.dt);
    const T idx = T(A.idx), idy = T(A.idy), idz = T(A.idz);
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    const T* __restrict__ Ex = A.emf;
    const T* __restrict__ Ey = A.emf + N;
    const T* __restrict__ Ez = A.emf + 2 * N;
    T Lq[2][8];
#pragma unroll
    for (int u = 0; u < 2; u++) {
#pragma unroll
        for (int q = 0; q < 5; q++) {
            const long long o = q * N;
            Lq[u][q] = flux_rate(Fx[o + cx[u]], Fx[o + c[u]], Fy[o + cy[u]], Fy[o + c[u]], Fz[o + cz[u]],
                                 Fz[o + c[u]], idx, idy, idz);
        }
        const T ex = Ex[c[u]], ey = Ey[c[u]], ez = Ez[c[u]];
        Lq[u][5] = face_rate(Ez[cy[u]], ez, idy, Ey[cz[u]], ey, idz);
        Lq[u][6] = face_rate(Ex[cz[u]], ex, idz, Ez[cx[u]], ez, idx);
        Lq[u][7] = face_rate(Ey[cx[u]], ey, idx, Ex[cy[u]], ex, idy);
    }
    T un[2][8], uk[2][8], acc[2][8];
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const long long o = q * N + c[u];
            un[u][q] = A.un[o];
            uk[u][q] = A.stage > 0 && A.integrator == 0 ? A.uk[o] : T(0);
            acc[u][q] = A.integrator == 1 && A.stage > 0 ? A.acc[o] : T(0);
        }
#pragma unroll
    for (int u = 0; u < 2; u++) {
        if (u == 1 && !has1) break;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const long long o = q * N + c[u];
            const T out = combine_value(A.integrator, A.stage, un[u][q], uk[u][q], acc[u][q], Lq[u][q], dt);
            if (A.integrator == 1 && A.stage < 3) A.acc[o] = acc[u][q];
            A.dst[o] = out;
        }
    }
}

// ---- one thread per vector of V cells along x (periodic patches) -------------
template <class T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int V = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int V = 2; };

template <class T>
__device__ __forceinline__ void vload(const T* __restrict__ p, T (&v)[Vec<T>::V]) {
    const typename Vec<T>::type w = *reinterpret_cast<const typename Vec<T>::type*>(p);
    if constexpr (Vec<T>::V == 4) { v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w; }
    else { v[0] = w.x; v[1] = w.y; }
}

template <class T>
__device__ __forceinline__ void vstore(T* __restrict__ p, const T (&v)[Vec<T>::V]) {
    typename Vec<T>::type w;
    if constexpr (Vec<T>::V == 4) { w.x = v[0]; w.y = v[1]; w.z = v[2]; w.w = v[3]; }
    else { w.x = v[0]; w.y = v[1]; }
    *reinterpret_cast<typename Vec<T>::type*>(p) = w;
}

// Geometry of a thread's vector: cells i0 .. i0+V-1 of row (j, k) and the
// first cells of the neighbouring vectors and rows (periodic wrap).
struct VRow {
    long long c;              // first cell of the vector
    long long cxm, cxp;       // cells i0-1 and i0+V
    long long cym, cyp;       // rows j-1, j+1
    long long czm, czp;       // planes k-1, k+1
    long long cymzm;          // (j-1, k-1)
    long long cxmym, cxmzm;   // cells (i0-1, j-1) and (i0-1, k-1)
};

template <int V>
__device__ __forceinline__ bool vrow(const CellBlock& cb, const PatchDev& P, int tid, VRow& r, long long N,
                                     unsigned int* flag) {
    const int local = cb.y + tid * V;
    const int nxy = P.nx * P.ny;
    if (local >= nxy * P.nz) return false;
    const int k = local / nxy;
    const int rem = local - k * nxy;
    const int j = rem / P.nx;
    const int i = rem - j * P.nx;
    const int im = i == 0 ? P.nx - 1 : i - 1;
    const int ip = i + V == P.nx ? 0 : i + V;
    const int jm = j == 0 ? P.ny - 1 : j - 1, jp = j + 1 == P.ny ? 0 : j + 1;
    const int km = k == 0 ? P.nz - 1 : k - 1, kp = k + 1 == P.nz ? 0 : k + 1;
    auto at = [&](int a, int b, int cc) { return P.off + ((long long)cc * P.ny + b) * P.nx + a; };
    r.c = P.off + local;
    r.cxm = at(im, j, k);
    r.cxp = at(ip, j, k);
    r.cym = at(i, jm, k);
    r.cyp = at(i, jp, k);
    r.czm = at(i, j, km);
    r.czp = at(i, j, kp);
    r.cymzm = at(i, jm, km);
    r.cxmym = at(im, jm, k);
    r.cxmzm = at(im, j, km);
#if WB_BOUNDS_CHECK
    // every vector inside the arrays and aligned, every scalar neighbour inside
    auto vec_ok = [&](long long a) { return a >= 0 && a + V <= N && a % V == 0; };
    auto one_ok = [&](long long a) { return a >= 0 && a < N; };
    if (!(vec_ok(r.c) && vec_ok(r.cym) && vec_ok(r.cyp) && vec_ok(r.czm) && vec_ok(r.czp) &&
          vec_ok(r.cymzm) && one_ok(r.cxm) && one_ok(r.cxp) && one_ok(r.cxmym) && one_ok(r.cxmzm))) {
        if (flag) atomicOr(flag, kFlagBounds);
        return false;
    }
#else
    (void)N;
    (void)flag;
#endif
    return true;
}

template <class T>
__global__ void __launch_bounds__(kCellBlock) emf_kernel_vec(const UpdateArgs<T> A) {
    constexpr int V = Vec<T>::V;
    const CellBlock cb = A.blocks[blockIdx.x];
    const PatchDev P = A.patches[cb.x];
    VRow r;
    if (!vrow<V>(cb, P, threadIdx.x, r, A.ncells, A.flag)) return;
    const long long N = A.ncells;
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    const T* __restrict__ Er = A.er;
    const bool m0 = A.emf_mode == 0;
    T a[V], b[V], d[V], e[V], o[V];
    T e0[V], e1[V], e2[V], e3[V];
#pragma unroll
    for (int v = 0; v < V; v++) e0[v] = e1[v] = e2[v] = e3[v] = T(0);
    // E_x: -Fy5(k-1), -Fy5(k), Fz6(j-1), Fz6(j); er0 at (j-1,k-1), (k-1), (j-1), own
    vload(Fy + 5 * N + r.czm, a);
    vload(Fy + 5 * N + r.c, b);
    vload(Fz + 6 * N + r.cym, d);
    vload(Fz + 6 * N + r.c, e);
    if (m0) {
        vload(Er + r.cymzm, e0);
        vload(Er + r.czm, e1);
        vload(Er + r.cym, e2);
        vload(Er + r.c, e3);
    }
#pragma unroll
    for (int v = 0; v < V; v++) o[v] = edge_emf(-a[v], -b[v], d[v], e[v], e0[v], e1[v], e2[v], e3[v], A.emf_mode);
    vstore(A.emf + r.c, o);
    // E_y: Fx6(k-1), Fx6(k), -Fz5(i-1), -Fz5(i); er1 at (i-1,k-1), (k-1), (i-1), own
    vload(Fx + 6 * N + r.czm, a);
    vload(Fx + 6 * N + r.c, b);
    vload(Fz + 5 * N + r.c, e);
    const T fz_im = Fz[5 * N + r.cxm];
    T er_a = T(0), er_b = T(0);
    if (m0) {
        vload(Er + N + r.czm, e1);
        vload(Er + N + r.c, e3);
        er_a = Er[N + r.cxmzm];
        er_b = Er[N + r.cxm];
    }
#pragma unroll
    for (int v = 0; v < V; v++)
        o[v] = edge_emf(a[v], b[v], -(v == 0 ? fz_im : e[v - 1]), -e[v], v == 0 ? er_a : e1[v - 1], e1[v],
                        v == 0 ? er_b : e3[v - 1], e3[v], A.emf_mode);
    vstore(A.emf + N + r.c, o);
    // E_z: -Fx5(j-1), -Fx5(j), Fy6(i-1), Fy6(i); er2 at (i-1,j-1), (j-1), (i-1), own
    vload(Fx + 5 * N + r.cym, a);
    vload(Fx + 5 * N + r.c, b);
    vload(Fy + 6 * N + r.c, e);
    const T fy_im = Fy[6 * N + r.cxm];
    if (m0) {
        vload(Er + 2 * N + r.cym, e1);
        vload(Er + 2 * N + r.c, e3);
        er_a = Er[2 * N + r.cxmym];
        er_b = Er[2 * N + r.cxm];
    }
#pragma unroll
    for (int v = 0; v < V; v++)
        o[v] = edge_emf(-a[v], -b[v], v == 0 ? fy_im : e[v - 1], e[v], v == 0 ? er_a : e1[v - 1], e1[v],
                        v == 0 ? er_b : e3[v - 1], e3[v], A.emf_mode);
    vstore(A.emf + 2 * N + r.c, o);
}

template <class T>
__global__ void __launch_bounds__(kCellBlock, 4) update_kernel_vec(const UpdateArgs<T> A) {
    constexpr int V = Vec<T>::V;
    const CellBlock cb = A.blocks[blockIdx.x];
    const PatchDev P = A.patches[cb.x];
    VRow r;
    if (!vrow<V>(cb, P, threadIdx.x, r, A.ncells, A.flag)) return;
    const long long N = A.ncells;
    const T dt = T(*A.dt);
    const T idx = T(A.idx), idy = T(A.idy), idz = T(A.idz);
    const T* __restrict__ Fx = A.flux;
    const T* __restrict__ Fy = A.flux + 7 * N;
    const T* __restrict__ Fz = A.flux + 14 * N;
    T L[8][V];
#pragma unroll
    for (int q = 0; q < 5; q++) {
        const long long o = q * N;
        T xc[V], yc[V], yp[V], zc[V], zp[V];
        vload(Fx + o + r.c, xc);
        const T xn = Fx[o + r.cxp];
        vload(Fy + o + r.c, yc);
        vload(Fy + o + r.cyp, yp);
        vload(Fz + o + r.c, zc);
        vload(Fz + o + r.czp, zp);
#pragma unroll
        for (int v = 0; v < V; v++)
            L[q][v] = flux_rate(v + 1 < V ? xc[v + 1] : xn, xc[v], yp[v], yc[v], zp[v], zc[v], idx, idy, idz);
    }
    {
        T ex[V], ey[V], ez[V], ezy[V], eyz[V], exz[V], exy[V];
        vload(A.emf + r.c, ex);
        vload(A.emf + N + r.c, ey);
        vload(A.emf + 2 * N + r.c, ez);
        vload(A.emf + 2 * N + r.cyp, ezy);
        vload(A.emf + N + r.czp, eyz);
        vload(A.emf + r.czp, exz);
        vload(A.emf + r.cyp, exy);
        const T ezx = A.emf[2 * N + r.cxp];
        const T eyx = A.emf[N + r.cxp];
#pragma unroll
        for (int v = 0; v < V; v++) {
            L[5][v] = face_rate(ezy[v], ez[v], idy, eyz[v], ey[v], idz);
            L[6][v] = face_rate(exz[v], ex[v], idz, v + 1 < V ? ez[v + 1] : ezx, ez[v], idx);
            L[7][v] = face_rate(v + 1 < V ? ey[v + 1] : eyx, ey[v], idx, exy[v], ex[v], idy);
        }
    }
    const bool rk3 = A.integrator == 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const long long o = q * N + r.c;
        T un[V], uk[V], acc[V], out[V];
#pragma unroll
        for (int v = 0; v < V; v++) uk[v] = acc[v] = T(0);
        vload(A.un + o, un);
        if (A.stage > 0 && rk3) vload(A.uk + o, uk);
        if (!rk3 && A.stage > 0) vload(A.acc + o, acc);
#pragma unroll
        for (int v = 0; v < V; v++) out[v] = combine_value(A.integrator, A.stage, un[v], uk[v], acc[v], L[q][v], dt);
        if (!rk3 && A.stage < 3) vstore(A.acc + o, acc);
        vstore(A.dst + o, out);
    }
}

}  // namespace

template <class T>
cudaError_t launch_emf(const UpdateArgs<T>& a, int nblocks, cudaStream_t s) {
    if (a.vblocks) {
        UpdateArgs<T> v = a;
        v.blocks = a.vblocks;
        if (a.nvblocks > 0) emf_kernel_vec<T><<<a.nvblocks, kCellBlock, 0, s>>>(v);
        return cudaGetLastError();
    }
    if (nblocks <= 0) return cudaSuccess;
    if constexpr (WB_UPDATE_PAIRS && sizeof(T) == 4) {
        if (a.links) emf_kernel2<T, true><<<nblocks, kCellBlock / 2, 0, s>>>(a);
        else emf_kernel2<T, false><<<nblocks, kCellBlock / 2, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.links) emf_kernel<T, true><<<nblocks, kCellBlock, 0, s>>>(a);
    else emf_kernel<T, false><<<nblocks, kCellBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_update(const UpdateArgs<T>& a, int nblocks, cudaStream_t s) {
    if (a.vblocks) {
        UpdateArgs<T> v = a;
        v.blocks = a.vblocks;
        if (a.nvblocks > 0) update_kernel_vec<T><<<a.nvblocks, kCellBlock, 0, s>>>(v);
        return cudaGetLastError();
    }
    if (nblocks <= 0) return cudaSuccess;
    if constexpr (WB_UPDATE_PAIRS && sizeof(T) == 4) {
        if (a.links) update_kernel2<T, true><<<nblocks, kCellBlock / 2, 0, s>>>(a);
        else update_kernel2<T, false><<<nblocks, kCellBlock / 2, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.links) update_kernel<T, true><<<nblocks, kCellBlock, 0, s>>>(a);
    else update_kernel<T, false><<<nblocks, kCellBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int update_vector_width(bool fp64) { return fp64 ? Vec<double>::V : Vec<float>::V; }

template cudaError_t launch_emf<float>(const UpdateArgs<float>&, int, cudaStream_t);
template cudaError_t launch_emf<double>(const UpdateArgs<double>&, int, cudaStream_t);
template cudaError_t launch_update<float>(const UpdateArgs<float>&, int, cudaStream_t);
template cudaError_t launch_update<double>(const UpdateArgs<double>&, int, cudaStream_t);

}  // namespace wb
