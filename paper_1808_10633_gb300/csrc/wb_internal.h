// wb_internal.h -- types shared by the CUDA translation units of the library
// (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace wb {

// One periodic patch of the world grid (Sec. 2.2 "patches"); a single grid
// is one patch.  Field f of the state lives at base + f*ncells + off + local.
struct PatchDev {
    int nx, ny, nz, pad;
    long long off;
};

// Cell addressing across patch boundaries.  Sec. 2.2 resolves each patch
// with the ghost zones its neighbours provide; here a patch reads its
// neighbours' cells in place.  links == nullptr: every patch is periodic on
// itself.  Otherwise links[27 p + 9 (oz+1) + 3 (oy+1) + (ox+1)] is the patch
// that continues patch p in direction (ox, oy, oz) in {-1, 0, 1}^3; the host
// has checked that linked patches agree in the extents they share and are at
// least 3 cells deep wherever a stencil crosses into them.  (i, j, k) may lie
// up to 3 cells outside patch p; the result is the flat cell index.
__device__ __forceinline__ int wrap_cell(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ long long locate(const PatchDev* __restrict__ patches,
                                            const int* __restrict__ links, int p,
                                            const PatchDev& P, int i, int j, int k) {
    const int ox = i < 0 ? -1 : (i >= P.nx ? 1 : 0);
    const int oy = j < 0 ? -1 : (j >= P.ny ? 1 : 0);
    const int oz = k < 0 ? -1 : (k >= P.nz ? 1 : 0);
    if ((ox | oy | oz) == 0) return P.off + ((long long)k * P.ny + j) * P.nx + i;
    if (links == nullptr)
        return P.off + ((long long)wrap_cell(k, P.nz) * P.ny + wrap_cell(j, P.ny)) * P.nx +
               wrap_cell(i, P.nx);
    const int q = links[27 * p + 9 * (oz + 1) + 3 * (oy + 1) + (ox + 1)];
    const PatchDev Q = patches[q];
    i = ox < 0 ? i + Q.nx : (ox > 0 ? i - P.nx : i);
    j = oy < 0 ? j + Q.ny : (oy > 0 ? j - P.ny : j);
    k = oz < 0 ? k + Q.nz : (oz > 0 ? k - P.nz : k);
    // a patch linked to itself along an axis shorter than the stencil reach
    if (i < 0 || i >= Q.nx) i = wrap_cell(i, Q.nx);
    if (j < 0 || j >= Q.ny) j = wrap_cell(j, Q.ny);
    if (k < 0 || k >= Q.nz) k = wrap_cell(k, Q.nz);
    return Q.off + ((long long)k * Q.ny + j) * Q.nx + i;
}

// Bounds-checked builds (WB_BOUNDS_CHECK=1, the library's "check" variant):
// each global or shared index the solver kernels form is tested against its
// array; an index outside it sets kFlagBounds in the grid's status word and
// is replaced by 0 (an in-range access), and the host reports the run as
// WB_EINTERNAL.  In normal builds chk() is the identity.
#ifndef WB_BOUNDS_CHECK
#define WB_BOUNDS_CHECK 0
#endif
constexpr unsigned int kFlagBounds = 4u;
// A bounded wait of a kernel on the tensor cores ran out (WB_ETIMEOUT).
constexpr unsigned int kFlagTimeout = 8u;

__device__ __forceinline__ long long chk(long long i, long long n, unsigned int* flag) {
#if WB_BOUNDS_CHECK
    if (i < 0 || i >= n) {
        if (flag) atomicOr(flag, kFlagBounds);
        return 0;
    }
#else
    (void)n;
    (void)flag;
#endif
    return i;
}

// Sweep tile: x = patch, y = start along the sweep axis, z = start along the
// pencil axis, w = fixed third coordinate.
using Tile = int4;

// Cell block for the per-cell kernels: x = patch, y = first local cell.
using CellBlock = int2;

constexpr int kCellBlock = 256;   // cells per block of the per-cell kernels

// Operations with explicit rounding (no contraction into FMAs), for values
// that several kernels must compute to the same bits.
namespace rn {
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
}  // namespace rn

// The CFL signal rate of one cell, sum over the axes d of
// (|v_d| + c_f,d) / dx_d with c_f,d the fast speed along d, from its rho,
// momentum, total energy and cell-centred B (the CFL rule; the paper states
// none).  Every operation is rounded explicitly, so the scalar and the vector
// CFL kernels agree to the bit.  p receives the gas pressure.
template <class T>
__device__ __forceinline__ T cell_signal(T rho, T m0, T m1, T m2, T E, T B0, T B1, T B2, T g,
                                         T id0, T id1, T id2, T& p) {
    const T rinv = rn::div(T(1), rho);
    const T v0 = rn::mul(m0, rinv), v1 = rn::mul(m1, rinv), v2 = rn::mul(m2, rinv);
    const T bb = rn::add(rn::add(rn::mul(B0, B0), rn::mul(B1, B1)), rn::mul(B2, B2));
    const T vv = rn::add(rn::add(rn::mul(v0, v0), rn::mul(v1, v1)), rn::mul(v2, v2));
    const T kin = rn::mul(rn::mul(T(0.5), rho), vv);
    p = rn::mul(rn::sub(g, T(1)), rn::sub(rn::sub(E, kin), rn::mul(T(0.5), bb)));
    const T a2 = rn::mul(rn::mul(g, p), rinv);
    const T q[3] = {rn::mul(B0, B0), rn::mul(B1, B1), rn::mul(B2, B2)};
    const T vd[3] = {v0, v1, v2}, id[3] = {id0, id1, id2};
    T sp = T(0);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        // cf^2 = (a^2 + ca^2 + t + D)/2, D^2 = (a^2 - ca^2)^2 + t (2 (a^2 + ca^2) + t),
        // t = B_perp^2 / rho: non-negative terms only (no cancellation)
        const T ca2 = rn::mul(q[d], rinv);
        const T t = rn::mul(rn::add(q[(d + 1) % 3], q[(d + 2) % 3]), rinv);
        const T dA = rn::sub(a2, ca2), sA = rn::add(a2, ca2);
        const T D = rn::sqrt(rn::add(rn::mul(dA, dA), rn::mul(t, rn::add(rn::mul(T(2), sA), t))));
        const T cf = rn::sqrt(rn::mul(T(0.5), rn::add(rn::add(sA, t), D)));
        const T av = vd[d] < T(0) ? -vd[d] : vd[d];
        sp = rn::add(sp, rn::mul(rn::add(av, cf), id[d]));
    }
    return sp;
}

// Number of state arrays: rho, mx, my, mz, E (cell) + bx, by, bz (faces).
constexpr int kNState = 8;
// Stored flux components per axis: rho, mx, my, mz, E, B_t1, B_t2.
constexpr int kNFlux = 7;

template <class T>
struct SweepArgs {
    const T* __restrict__ src;     // state base (kNState arrays)
    T* __restrict__ flux;          // flux base of this axis (kNFlux arrays)
    T* __restrict__ er;            // cell -v x B (3 arrays) or nullptr
    const Tile* __restrict__ tiles;
    const PatchDev* __restrict__ patches;
    const int* __restrict__ links = nullptr;   // patch links (see locate) or nullptr
    long long ncells;              // stride between arrays
    double gamma;
    int zweights = 0;              // 1: WENO-Z weights instead of Jiang-Shu
    unsigned long long* lstats = nullptr;   // learned sweep: detector firings, decisions
    int* queue = nullptr;          // persistent sweep: tile counter of this launch (or fixed stride)
    int split[3] = {0, 0, 0};      // tiles of shape 0, 1, 2 of a table sorted by shape
                                   // (one fixed launch per shape, a tile per block);
                                   // all 0: the persistent runtime-shape launch
    unsigned int* flag = nullptr;  // status word (bounds-checked builds)
};

template <class T>
struct UpdateArgs {
    const T* un;                   // state at t^n (may alias dst)
    const T* uk;                   // stage state the fluxes were taken from (may alias dst)
    T* dst;                        // output stage state (may alias uk or un)
    T* acc;                        // RK4 accumulator (may be null)
    const T* __restrict__ flux;    // 3 axes x kNFlux arrays
    const T* __restrict__ er;      // 3 arrays (emf_mode 0) or nullptr
    T* emf;                        // 3 arrays of edge EMFs (E_x, E_y, E_z)
    const CellBlock* __restrict__ blocks;
    const CellBlock* __restrict__ vblocks;   // blocks of 256 vectors of cells along x, or nullptr
    int nvblocks;
    const PatchDev* __restrict__ patches;
    const int* __restrict__ links; // patch links (see locate) or nullptr
    const double* __restrict__ dt; // device scalar
    long long ncells;
    double idx, idy, idz;
    int stage;                     // SSP-RK3: 0,1,2; RK4: 0..3
    int integrator;
    int emf_mode;
    unsigned int* flag;            // status word (bounds-checked builds)
};

// Sets the calling thread's wb_last_error() message and returns `code`.
int set_last_error(int code, const char* msg);

// ---- launchers (one per translation unit) ---------------------------------
template <class T>
cudaError_t launch_sweep(int axis, const SweepArgs<T>& a, int ntiles, cudaStream_t s);
template <class T>
cudaError_t prepare_sweep_kernels();
// Tile shape s (0 = default, kNTileShape alternatives) of the sweep along
// `axis`: ta interfaces along the axis times tp pencils (ta * tp = 256).
constexpr int kNTileShape = 3;
void sweep_shape(int axis, int s, int* ta, int* tp);
// Tile of the learned-weight sweep along `axis` (one shape, 256 threads).
void learned_shape(int axis, int* ta, int* tp);

template <class T>
cudaError_t launch_emf(const UpdateArgs<T>& a, int nblocks, cudaStream_t s);
template <class T>
cudaError_t launch_update(const UpdateArgs<T>& a, int nblocks, cudaStream_t s);
// Cells per thread of the vector forms of the EMF and update kernels (16 bytes).
int update_vector_width(bool fp64);

cudaError_t prepare_sweep_learned();
cudaError_t launch_sweep_learned(int axis, const SweepArgs<float>& a, int ntiles, const uint32_t* mlp,
                                 float kappa, float pjump, float smooth, cudaStream_t s);
void mlp_fragments(const float* params, uint32_t* out);
size_t mlp_fragment_words();
// The learned sweep on the 5th-generation tensor cores (wb_sweep_learned_tc.cu).
void learned_tc_shape(int axis, int* ta, int* tp);
cudaError_t prepare_sweep_learned_tc();
cudaError_t launch_sweep_learned_tc(int axis, const SweepArgs<float>& a, int ntiles, const void* image,
                                    float kappa, float pjump, float smooth, cudaStream_t s);
size_t mlp_tc_image_bytes();
void mlp_tc_image(const float* params, unsigned char* out);

template <class T>
cudaError_t launch_harvest(const T* src, long long ncells, const PatchDev& P, int axis,
                           const long long* cells, long long n, const double* hU, const double* hF,
                           double gamma, double kappa, double pjump, float* out, cudaStream_t s);

template <class T>
cudaError_t launch_cell_state_flux(const T* src, long long ncells, const PatchDev& P, int axis,
                                   double gamma, double* X, double* F, cudaStream_t s);

template <class T>
cudaError_t launch_cfl(const T* state, const CellBlock* blocks, const PatchDev* patches,
                       const int* links, long long ncells, int nblocks, const CellBlock* vblocks,
                       int nvblocks, double idx, double idy, double idz, double gamma,
                       unsigned long long* smax_bits, unsigned int* flag, cudaStream_t s);
template <class T>
cudaError_t launch_divb(const T* state, const CellBlock* blocks, const PatchDev* patches,
                        const int* links, long long ncells, int nblocks, double idx, double idy,
                        double idz, unsigned long long* out_bits, unsigned int* flag, cudaStream_t s);
cudaError_t launch_set_dt(const unsigned long long* smax_bits, double cfl, double fixed_dt,
                          double* dt, double* time, cudaStream_t s);

template <class T>
cudaError_t launch_totals(const T* state, const PatchDev* patches, int npatch,
                          long long ncells, double* partial, int npartial,
                          double dV, double* out, cudaStream_t s);

template <class T, class H>
cudaError_t launch_import(const H* U, const H* b, T* state,
                          const CellBlock* blocks, const PatchDev* patches,
                          long long ncells, int nblocks, cudaStream_t s);
template <class T>
cudaError_t launch_export_flux(const T* flux, double* out, const CellBlock* blocks,
                               const PatchDev* patches, long long ncells, int nblocks,
                               cudaStream_t s);
template <class T, class H>
cudaError_t launch_export(const T* state, H* U, H* b,
                          const CellBlock* blocks, const PatchDev* patches, const int* links,
                          long long ncells, int nblocks, cudaStream_t s);

}  // namespace wb
