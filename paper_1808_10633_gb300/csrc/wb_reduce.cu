// wb_reduce.cu -- CFL time step (FP64 max reduction with warp shuffles),
// deterministic FP64 conserved totals, and the FP64 <-> state conversions
// used at the ABI.
#include "wb_internal.h"

#include <cfloat>
#include <limits>

namespace wb {
namespace {

// dt rule: s = sum_d (|v_d| + c_f,d) / dx_d per cell, maximised over cells;
// the fast speed along d uses B_d as the normal field.  The per-cell speed is
// taken in the state's precision (FP32 in FP32 mode: FP64 division and square
// root run at a small fraction of the FP32 rate on this GPU); the maximum is
// reduced in FP64, which is exact.
// Upper neighbour of cell (i, j, k) of patch p along each axis: the wrap
// round a periodic patch, or the link table's neighbour.
template <bool LINKED>
__device__ __forceinline__ long long upper(const PatchDev* __restrict__ patches,
                                           const int* __restrict__ links, int p, const PatchDev& P,
                                           int i, int j, int k) {
    if constexpr (LINKED) return locate(patches, links, p, P, i, j, k);
    i = i == P.nx ? 0 : i;
    j = j == P.ny ? 0 : j;
    k = k == P.nz ? 0 : k;
    return P.off + ((long long)k * P.ny + j) * P.nx + i;
}

// Folds one cell's signal rate into the running maximum s (kept in T: the
// largest of FP32 values converted to FP64 once is the largest of their FP64
// conversions, the conversion being exact and monotonic, so FP32 grids keep
// the FP64 pipe out of the loop); flags NaN/Inf and rho, p <= 0.
template <class T>
__device__ __forceinline__ void fold_signal(T& s, T rho, T m0, T m1, T m2, T E, T B0, T B1, T B2,
                                            T g, T id0, T id1, T id2, unsigned int* flag) {
    T p;
    T sc = cell_signal<T>(rho, m0, m1, m2, E, B0, B1, B2, g, id0, id1, id2, p);
    unsigned int bad = 0;
    if (!(sc <= std::numeric_limits<T>::max())) bad |= 1u;   // NaN or Inf
    if (!(rho > T(0)) || !(p > T(0))) bad |= 2u;
    if (bad) {
        atomicOr(flag, bad);
        sc = T(0);
    }
    s = sc > s ? sc : s;
}

// Block maximum of s, folded into *smax_bits as an FP64 bit pattern (s >= 0,
// so the IEEE bit patterns order like the values).
template <class T>
__device__ __forceinline__ void block_max_out(T s, unsigned long long* smax_bits) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T r = __shfl_xor_sync(0xffffffffu, s, o);
        s = r > s ? r : s;
    }
    __shared__ T red[kCellBlock / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < kCellBlock / 32 ? red[threadIdx.x] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T r = __shfl_xor_sync(0xffffffffu, s, o);
            s = r > s ? r : s;
        }
        if (threadIdx.x == 0)
            atomicMax(smax_bits, (unsigned long long)__double_as_longlong(double(s)));
    }
}

// One thread per cell, any patches (linked ones too).
template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock)
cfl_kernel(const T* __restrict__ q, const CellBlock* __restrict__ blocks, int nblocks,
           const PatchDev* __restrict__ patches, const int* __restrict__ links, long long N,
           double idx, double idy, double idz, double gamma, unsigned long long* smax_bits,
           unsigned int* flag) {
    T s = T(0);
    const T g = T(gamma), i0 = T(idx), i1 = T(idy), i2 = T(idz);
    // grid-stride over the cell blocks: one atomic per resident block, not
    // one per 256 cells (same-address atomics serialise in L2)
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const CellBlock cb = blocks[b];
        const PatchDev P = patches[cb.x];
        const int local = cb.y + threadIdx.x;
        const int nxy = P.nx * P.ny;
        if (local < nxy * P.nz) {
            const int k = local / nxy;
            const int rem = local - k * nxy;
            const int j = rem / P.nx;
            const int i = rem - j * P.nx;
            const long long c = chk(P.off + local, N, flag);
            const long long cx = chk(upper<LINKED>(patches, links, cb.x, P, i + 1, j, k), N, flag);
            const long long cy = chk(upper<LINKED>(patches, links, cb.x, P, i, j + 1, k), N, flag);
            const long long cz = chk(upper<LINKED>(patches, links, cb.x, P, i, j, k + 1), N, flag);
            fold_signal<T>(s, q[c], q[N + c], q[2 * N + c], q[3 * N + c], q[4 * N + c],
                           rn::mul(T(0.5), rn::add(q[5 * N + c], q[5 * N + cx])),
                           rn::mul(T(0.5), rn::add(q[6 * N + c], q[6 * N + cy])),
                           rn::mul(T(0.5), rn::add(q[7 * N + c], q[7 * N + cz])), g, i0, i1, i2, flag);
        }
    }
    block_max_out<T>(s, smax_bits);
}

template <class T> struct CflVec;
template <> struct CflVec<float> { using type = float4; static constexpr int V = 4; };
template <> struct CflVec<double> { using type = double2; static constexpr int V = 2; };

template <class T, int V>
__device__ __forceinline__ void vget(const T* __restrict__ p, T (&v)[V]) {
    const typename CflVec<T>::type x = *reinterpret_cast<const typename CflVec<T>::type*>(p);
    if constexpr (V == 4) { v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; }
    else { v[0] = x.x; v[1] = x.y; }
}

// One thread per 16-byte vector of cells along x, for periodic patches whose
// x extent is a multiple of the vector width (vector blocks of the grid):
// four times the bytes in flight per thread, the same per-cell arithmetic.
template <class T>
__global__ void __launch_bounds__(kCellBlock)
cfl_kernel_vec(const T* __restrict__ q, const CellBlock* __restrict__ vblocks, int nvblocks,
               const PatchDev* __restrict__ patches, long long N, double idx, double idy, double idz,
               double gamma, unsigned long long* smax_bits, unsigned int* flag) {
    constexpr int V = CflVec<T>::V;
    T s = T(0);
    const T g = T(gamma), i0 = T(idx), i1 = T(idy), i2 = T(idz);
    for (int b = blockIdx.x; b < nvblocks; b += gridDim.x) {
        const CellBlock cb = vblocks[b];
        const PatchDev P = patches[cb.x];
        const int local = cb.y + threadIdx.x * V;
        const int nxy = P.nx * P.ny;
        if (local < nxy * P.nz) {
            const int k = local / nxy;
            const int rem = local - k * nxy;
            const int j = rem / P.nx;
            const int i = rem - j * P.nx;
            const int ip = i + V == P.nx ? 0 : i + V;
            const int jp = j + 1 == P.ny ? 0 : j + 1, kp = k + 1 == P.nz ? 0 : k + 1;
            auto at = [&](int a, int bb, int cc) { return P.off + ((long long)cc * P.ny + bb) * P.nx + a; };
            const long long c = P.off + local, cxp = at(ip, j, k), cyp = at(i, jp, k), czp = at(i, j, kp);
#if WB_BOUNDS_CHECK
            auto vec_ok = [&](long long a) { return a >= 0 && a + V <= N && a % V == 0; };
            if (!(vec_ok(c) && vec_ok(cyp) && vec_ok(czp) && cxp >= 0 && cxp < N)) {
                atomicOr(flag, kFlagBounds);
                continue;
            }
#endif
            T rho[V], m0[V], m1[V], m2[V], E[V], bx[V], by[V], bz[V], byp[V], bzp[V];
            vget<T, V>(q + c, rho);
            vget<T, V>(q + N + c, m0);
            vget<T, V>(q + 2 * N + c, m1);
            vget<T, V>(q + 3 * N + c, m2);
            vget<T, V>(q + 4 * N + c, E);
            vget<T, V>(q + 5 * N + c, bx);
            vget<T, V>(q + 6 * N + c, by);
            vget<T, V>(q + 7 * N + c, bz);
            vget<T, V>(q + 6 * N + cyp, byp);
            vget<T, V>(q + 7 * N + czp, bzp);
            const T bx_next = q[5 * N + cxp];
#pragma unroll
            for (int v = 0; v < V; v++) {
                const T bxu = v + 1 < V ? bx[v + 1] : bx_next;
                fold_signal<T>(s, rho[v], m0[v], m1[v], m2[v], E[v], rn::mul(T(0.5), rn::add(bx[v], bxu)),
                               rn::mul(T(0.5), rn::add(by[v], byp[v])), rn::mul(T(0.5), rn::add(bz[v], bzp[v])),
                               g, i0, i1, i2, flag);
            }
        }
    }
    block_max_out<T>(s, smax_bits);
}

// Face divergence of b per cell (the quantity constrained transport keeps at
// round-off, Sec. 2.1): (bx(i+1) - bx(i))/dx + (by(j+1) - by(j))/dy +
// (bz(k+1) - bz(k))/dz, in FP64; out_bits[0] = max |div b|, out_bits[1] =
// max |b| over the faces, both as FP64 bit patterns (non-negative values, so
// an integer maximum orders them).
template <class T, bool LINKED>
__global__ void __launch_bounds__(kCellBlock)
divb_kernel(const T* __restrict__ q, const CellBlock* __restrict__ blocks, int nblocks,
            const PatchDev* __restrict__ patches, const int* __restrict__ links, long long N,
            double idx, double idy, double idz, unsigned long long* out_bits, unsigned int* flag) {
    double dmax = 0.0, bmax = 0.0;
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const CellBlock cb = blocks[b];
        const PatchDev P = patches[cb.x];
        const int local = cb.y + threadIdx.x;
        const int nxy = P.nx * P.ny;
        if (local < nxy * P.nz) {
            const int k = local / nxy;
            const int rem = local - k * nxy;
            const int j = rem / P.nx;
            const int i = rem - j * P.nx;
            const long long c = chk(P.off + local, N, flag);
            const long long cx = chk(upper<LINKED>(patches, links, cb.x, P, i + 1, j, k), N, flag);
            const long long cy = chk(upper<LINKED>(patches, links, cb.x, P, i, j + 1, k), N, flag);
            const long long cz = chk(upper<LINKED>(patches, links, cb.x, P, i, j, k + 1), N, flag);
            const double bx = double(q[5 * N + c]), by = double(q[6 * N + c]), bz = double(q[7 * N + c]);
            const double d = (double(q[5 * N + cx]) - bx) * idx + (double(q[6 * N + cy]) - by) * idy
                           + (double(q[7 * N + cz]) - bz) * idz;
            dmax = fmax(dmax, fabs(d));
            bmax = fmax(bmax, fmax(fabs(bx), fmax(fabs(by), fabs(bz))));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out_bits, (unsigned long long)__double_as_longlong(dmax));
        atomicMax(out_bits + 1, (unsigned long long)__double_as_longlong(bmax));
    }
}

__global__ void set_dt_kernel(const unsigned long long* smax_bits, double cfl, double fixed_dt,
                              double* dt, double* time) {
    double d = fixed_dt;
    if (!(fixed_dt > 0.0)) {
        const double smax = __longlong_as_double((long long)*smax_bits);
        d = smax > 0.0 ? cfl / smax : 0.0;
    }
    *dt = d;
    *time += d;
}

// Totals: sum over cells of rho, m, E and of the face fields (for a periodic
// patch the sum of the face means equals the sum over faces).  Pass 1: each
// block reduces a fixed contiguous chunk in a fixed order; pass 2: one block
// reduces the partials.  Same order on every call, so bitwise repeatable.
// The FP64 value of an FP32 number, formed from its bits with integer
// operations (IEEE 754 binary32 -> binary64 is exact: sign kept, exponent
// rebiased by 1023 - 127, mantissa widened by 29 zero bits; subnormals
// normalised, zero, infinities and NaN mapped to their binary64 forms).  The
// conversion instruction would run on the FP64 pipe, which is narrow on this
// GPU; here only the sums do.
__device__ __forceinline__ double widen(float x) {
    const unsigned int u = __float_as_uint(x);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned int e = (u >> 23) & 0xffu;
    unsigned int m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) {                       // infinity or NaN
        bits = sign | (0x7ffull << 52) | ((unsigned long long)m << 29);
    } else if (e != 0u) {                   // normal
        bits = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {                   // signed zero
        bits = sign;
    } else {                                // subnormal: value m 2^-149
        const int sh = __clz(m) - 8;        // shifts that bring the top bit to bit 23
        m = (m << sh) & 0x7fffffu;
        bits = sign | ((unsigned long long)(897 - sh) << 52) | ((unsigned long long)m << 29);
    }
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double x) { return x; }

template <class T>
__global__ void __launch_bounds__(256)
totals_pass1(const T* __restrict__ q, long long N, long long chunk, double* __restrict__ partial) {
    const long long beg = (long long)blockIdx.x * chunk;
    long long end = beg + chunk;
    if (end > N) end = N;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long c = beg + threadIdx.x; c < end; c += 256) {
#pragma unroll
        for (int f = 0; f < 8; f++) acc[f] += widen(q[f * N + c]);
    }
    __shared__ double red[8][256];
#pragma unroll
    for (int f = 0; f < 8; f++) red[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int f = 0; f < 8; f++) red[f][threadIdx.x] += red[f][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) partial[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(256)
totals_pass2(const double* __restrict__ partial, int npartial, double dV, double* __restrict__ out) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < npartial; b += 256) {
#pragma unroll
        for (int f = 0; f < 8; f++) acc[f] += partial[b * 8 + f];
    }
    __shared__ double red[8][256];
#pragma unroll
    for (int f = 0; f < 8; f++) red[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
#pragma unroll
            for (int f = 0; f < 8; f++) red[f][threadIdx.x] += red[f][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // state order rho, mx, my, mz, E, bx, by, bz -> ABI order
        // rho, mx, my, mz, Bx, By, Bz, E
        out[0] = red[0][0] * dV;
        out[1] = red[1][0] * dV;
        out[2] = red[2][0] * dV;
        out[3] = red[3][0] * dV;
        out[4] = red[5][0] * dV;
        out[5] = red[6][0] * dV;
        out[6] = red[7][0] * dV;
        out[7] = red[4][0] * dV;
    }
}

// ABI layout (FP64, or FP32 for the FP32 entry points, type H): U[patch][8][cells]
// with (rho, mx, my, mz, Bx, By, Bz, E), b[patch][3][cells]; state layout:
// field-major over all patches.
template <class T, class H>
__global__ void __launch_bounds__(kCellBlock)
import_kernel(const H* __restrict__ U, const H* __restrict__ b, T* __restrict__ q,
              const CellBlock* __restrict__ blocks, const PatchDev* __restrict__ patches,
              long long N) {
    const CellBlock cb = blocks[blockIdx.x];
    const PatchDev P = patches[cb.x];
    const long long np = (long long)P.nx * P.ny * P.nz;
    const int local = cb.y + threadIdx.x;
    if (local >= np) return;
    const long long c = P.off + local;
    const H* u = U + 8 * P.off + local;
    const H* bb = b + 3 * P.off + local;
    q[c] = T(u[0]);
    q[N + c] = T(u[np]);
    q[2 * N + c] = T(u[2 * np]);
    q[3 * N + c] = T(u[3 * np]);
    q[4 * N + c] = T(u[7 * np]);
    q[5 * N + c] = T(bb[0]);
    q[6 * N + c] = T(bb[np]);
    q[7 * N + c] = T(bb[2 * np]);
}

template <class T, class H, bool LINKED>
__global__ void __launch_bounds__(kCellBlock)
export_kernel(const T* __restrict__ q, H* __restrict__ U, H* __restrict__ b,
              const CellBlock* __restrict__ blocks, const PatchDev* __restrict__ patches,
              const int* __restrict__ links, long long N) {
    const CellBlock cb = blocks[blockIdx.x];
    const PatchDev P = patches[cb.x];
    const int nxy = P.nx * P.ny;
    const long long np = (long long)nxy * P.nz;
    const int local = cb.y + threadIdx.x;
    if (local >= np) return;
    const int k = local / nxy;
    const int rem = local - k * nxy;
    const int j = rem / P.nx;
    const int i = rem - j * P.nx;
    const long long c = P.off + local;
    const long long cx = upper<LINKED>(patches, links, cb.x, P, i + 1, j, k);
    const long long cy = upper<LINKED>(patches, links, cb.x, P, i, j + 1, k);
    const long long cz = upper<LINKED>(patches, links, cb.x, P, i, j, k + 1);
    if (U) {
        H* u = U + 8 * P.off + local;
        u[0] = H(double(q[c]));
        u[np] = H(double(q[N + c]));
        u[2 * np] = H(double(q[2 * N + c]));
        u[3 * np] = H(double(q[3 * N + c]));
        u[4 * np] = H(0.5 * (double(q[5 * N + c]) + double(q[5 * N + cx])));
        u[5 * np] = H(0.5 * (double(q[6 * N + c]) + double(q[6 * N + cy])));
        u[6 * np] = H(0.5 * (double(q[7 * N + c]) + double(q[7 * N + cz])));
        u[7 * np] = H(double(q[4 * N + c]));
    }
    if (b) {
        H* o = b + 3 * P.off + local;
        o[0] = H(double(q[5 * N + c]));
        o[np] = H(double(q[6 * N + c]));
        o[2 * np] = H(double(q[7 * N + c]));
    }
}

// Face fluxes of one axis to the ABI's patch-major FP64 layout [7][cells].
template <class T>
__global__ void __launch_bounds__(kCellBlock)
export_flux_kernel(const T* __restrict__ F, double* __restrict__ out,
                   const CellBlock* __restrict__ blocks, const PatchDev* __restrict__ patches,
                   long long N) {
    const CellBlock cb = blocks[blockIdx.x];
    const PatchDev P = patches[cb.x];
    const long long np = (long long)P.nx * P.ny * P.nz;
    const int local = cb.y + threadIdx.x;
    if (local >= np) return;
    const long long c = P.off + local;
    double* o = out + 7 * P.off + local;
#pragma unroll
    for (int q = 0; q < 7; q++) o[q * np] = double(F[q * N + c]);
}

}  // namespace

template <class T>
cudaError_t launch_export_flux(const T* flux, double* out, const CellBlock* blocks,
                               const PatchDev* patches, long long ncells, int nblocks,
                               cudaStream_t s) {
    export_flux_kernel<T><<<nblocks, kCellBlock, 0, s>>>(flux, out, blocks, patches, ncells);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_cfl(const T* state, const CellBlock* blocks, const PatchDev* patches,
                       const int* links, long long ncells, int nblocks, const CellBlock* vblocks,
                       int nvblocks, double idx, double idy, double idz, double gamma,
                       unsigned long long* smax_bits, unsigned int* flag, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = 8 * (nsm > 0 ? nsm : 152);      // one wave of 256-thread blocks
    }
    if (vblocks && nvblocks > 0 && !links) {
        const int vgrid = nvblocks < grid_cap ? nvblocks : grid_cap;
        cfl_kernel_vec<T><<<vgrid, kCellBlock, 0, s>>>(state, vblocks, nvblocks, patches, ncells, idx, idy,
                                                       idz, gamma, smax_bits, flag);
        return cudaGetLastError();
    }
    const int grid = nblocks < grid_cap ? nblocks : grid_cap;
    if (links)
        cfl_kernel<T, true><<<grid, kCellBlock, 0, s>>>(state, blocks, nblocks, patches, links, ncells,
                                                        idx, idy, idz, gamma, smax_bits, flag);
    else
        cfl_kernel<T, false><<<grid, kCellBlock, 0, s>>>(state, blocks, nblocks, patches, links, ncells,
                                                         idx, idy, idz, gamma, smax_bits, flag);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_divb(const T* state, const CellBlock* blocks, const PatchDev* patches,
                        const int* links, long long ncells, int nblocks, double idx, double idy,
                        double idz, unsigned long long* out_bits, unsigned int* flag, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out_bits, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cap = 8 * (nsm > 0 ? nsm : 152);
    const int grid = nblocks < cap ? nblocks : cap;
    if (links)
        divb_kernel<T, true><<<grid, kCellBlock, 0, s>>>(state, blocks, nblocks, patches, links, ncells,
                                                         idx, idy, idz, out_bits, flag);
    else
        divb_kernel<T, false><<<grid, kCellBlock, 0, s>>>(state, blocks, nblocks, patches, links, ncells,
                                                          idx, idy, idz, out_bits, flag);
    return cudaGetLastError();
}

cudaError_t launch_set_dt(const unsigned long long* smax_bits, double cfl, double fixed_dt,
                          double* dt, double* time, cudaStream_t s) {
    set_dt_kernel<<<1, 1, 0, s>>>(smax_bits, cfl, fixed_dt, dt, time);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_totals(const T* state, const PatchDev*, int, long long ncells,
                          double* partial, int npartial, double dV, double* out, cudaStream_t s) {
    const long long chunk = (ncells + npartial - 1) / npartial;
    totals_pass1<T><<<npartial, 256, 0, s>>>(state, ncells, chunk, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    totals_pass2<<<1, 256, 0, s>>>(partial, npartial, dV, out);
    return cudaGetLastError();
}

template <class T, class H>
cudaError_t launch_import(const H* U, const H* b, T* state, const CellBlock* blocks,
                          const PatchDev* patches, long long ncells, int nblocks, cudaStream_t s) {
    import_kernel<T, H><<<nblocks, kCellBlock, 0, s>>>(U, b, state, blocks, patches, ncells);
    return cudaGetLastError();
}

template <class T, class H>
cudaError_t launch_export(const T* state, H* U, H* b, const CellBlock* blocks,
                          const PatchDev* patches, const int* links, long long ncells, int nblocks,
                          cudaStream_t s) {
    if (links)
        export_kernel<T, H, true><<<nblocks, kCellBlock, 0, s>>>(state, U, b, blocks, patches, links, ncells);
    else
        export_kernel<T, H, false><<<nblocks, kCellBlock, 0, s>>>(state, U, b, blocks, patches, links, ncells);
    return cudaGetLastError();
}

#define WB_INST(T)                                                                            \
    template cudaError_t launch_cfl<T>(const T*, const CellBlock*, const PatchDev*, const int*, \
                                       long long, int, const CellBlock*, int, double, double, \
                                       double, double, unsigned long long*, unsigned int*,    \
                                       cudaStream_t);                                         \
    template cudaError_t launch_divb<T>(const T*, const CellBlock*, const PatchDev*, const int*, \
                                        long long, int, double, double, double,              \
                                        unsigned long long*, unsigned int*, cudaStream_t);    \
    template cudaError_t launch_totals<T>(const T*, const PatchDev*, int, long long, double*, \
                                          int, double, double*, cudaStream_t);                \
    template cudaError_t launch_import<T, double>(const double*, const double*, T*,          \
                                                  const CellBlock*, const PatchDev*, long long, \
                                                  int, cudaStream_t);                          \
    template cudaError_t launch_export<T, double>(const T*, double*, double*, const CellBlock*, \
                                                  const PatchDev*, const int*, long long, int,  \
                                                  cudaStream_t);                                \
    template cudaError_t launch_export_flux<T>(const T*, double*, const CellBlock*,           \
                                               const PatchDev*, long long, int, cudaStream_t);
WB_INST(float)
template cudaError_t launch_import<float, float>(const float*, const float*, float*, const CellBlock*,
                                                 const PatchDev*, long long, int, cudaStream_t);
template cudaError_t launch_export<float, float>(const float*, float*, float*, const CellBlock*,
                                                 const PatchDev*, const int*, long long, int, cudaStream_t);
WB_INST(double)
#undef WB_INST

}  // namespace wb
