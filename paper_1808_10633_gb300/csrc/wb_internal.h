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
                                 float kappa, float pjump, cudaStream_t s);
void mlp_fragments(const float* params, uint32_t* out);
size_t mlp_fragment_words();

template <class T>
cudaError_t launch_harvest(const T* src, long long ncells, const PatchDev& P, int axis,
                           const long long* cells, long long n, const double* hU, const double* hF,
                           double gamma, double kappa, double pjump, float* out, cudaStream_t s);

template <class T>
cudaError_t launch_cfl(const T* state, const CellBlock* blocks, const PatchDev* patches,
                       const int* links, long long ncells, int nblocks, double idx, double idy, double idz,
                       double gamma, unsigned long long* smax_bits, unsigned int* flag,
                       cudaStream_t s);
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
