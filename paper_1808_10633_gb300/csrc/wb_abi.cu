// wb_abi.cu -- the C ABI (include/wombat_gb300.h): grid lifecycle and the
// stream-ordered step sequence.
//
// Device state per grid (field-major over all patches, N cells in total):
//   un   8 arrays  rho, mx, my, mz, E, bx, by, bz at t^n
//   uk   8 arrays  Runge-Kutta stage state
//   acc  8 arrays  RK4 accumulator (RK4 only)
//   flux 21 arrays 7 face-flux components per axis
//   er   3 arrays  cell -v x B for the edge EMFs (emf_mode 0 only)
//   emf  3 arrays  edge EMFs of the current stage
// One step = [CFL reduction + dt] + per stage: x, y, z sweeps, the edge-EMF
// kernel and the update kernel.  A step is captured once as a CUDA graph and replayed.
#include "../../include/wombat_gb300.h"
#include "wb_internal.h"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define WB_CK(call)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? WB_ENOMEM : WB_ECUDA,      \
                        "%s:%d: %s: %s", __FILE__, __LINE__, #call,                  \
                        cudaGetErrorString(e_));                                     \
    } while (0)

constexpr int kPartials = 1024;

// Engine of the learned-weight sweep: 0 per warp with mma.sync
// (wb_sweep_learned.cu, the default: measured 6.3 ms per 256^3 launch), 1 per
// block on the 5th-generation tensor cores (tcgen05, wb_sweep_learned_tc.cu:
// 11.9 ms, its three block-wide rounds per field leave the MMA latency
// exposed); the build's "tc" variant compiles the library with engine 1.
#ifndef WB_LEARNED_ENGINE
#define WB_LEARNED_ENGINE 0
#endif

cudaError_t launch_learned(wb_grid* g, int axis, const wb::SweepArgs<float>& a);

// Optional per-launch CUDA-event timing (wb_step_profiled): an event pair is
// recorded on the grid's stream around each kernel launch.
struct Prof {
    std::vector<cudaEvent_t> ev;   // 2 per launch
    std::vector<int> cls;
    size_t used = 0;
};

int prof_begin(Prof* pf, cudaStream_t s) {
    if (!pf) return WB_OK;
    if (pf->used + 2 > pf->ev.size()) return fail(WB_EINTERNAL, "profiler event pool exhausted");
    WB_CK(cudaEventRecord(pf->ev[pf->used], s));
    return WB_OK;
}

int prof_end(Prof* pf, cudaStream_t s, int cls) {
    if (!pf) return WB_OK;
    WB_CK(cudaEventRecord(pf->ev[pf->used + 1], s));
    pf->cls.push_back(cls);
    pf->used += 2;
    return WB_OK;
}

}  // namespace

struct wb_grid {
    int npatch = 0;
    long long N = 0;
    double dx = 0, dy = 0, dz = 0, gamma = 0;
    int precision = 0, integrator = 0, emf_mode = 0, weights = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t tsize = 8;
    void* un = nullptr;
    void* uk = nullptr;
    void* acc = nullptr;
    void* flux = nullptr;
    void* er = nullptr;
    void* emf = nullptr;
    uint32_t* d_mlp = nullptr;            // learned weights, fragment order
    void* d_mlp_tc = nullptr;             // learned weights, tensor-core shared-memory image
    unsigned long long* d_lstats = nullptr;   // detector firings, decisions (learned grids)
    int* d_queue = nullptr;               // per-axis tile counters of the persistent sweeps
    int step_totals = 0;                  // 1: every step also takes the totals of its start state
    cudaStream_t side = nullptr;          // stream the per-step totals run on
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double kappa = 4.0, pjump = 0.5, smooth = 1.03;   // detector thresholds, smoothness gate
    int tile_policy[3] = {-2, -2, -2};    // build_tiles policy of each axis' table
    int tile_split[3][3] = {};            // per axis: tiles of each shape of a table sorted
                                          // by shape, or all 0 (wb::SweepArgs::split)
    wb::PatchDev* d_patches = nullptr;
    std::vector<wb::PatchDev> h_patches;
    int* d_links = nullptr;               // 27 per patch (wb::locate) or nullptr
    wb::Tile* d_tiles[3] = {nullptr, nullptr, nullptr};
    int ntiles[3] = {0, 0, 0};
    wb::CellBlock* d_blocks = nullptr;
    int nblocks = 0;
    wb::CellBlock* d_vblocks = nullptr;   // vector blocks of the per-cell kernels (periodic grids)
    int nvblocks = 0;
    double* d_scalars = nullptr;          // dt, time
    unsigned long long* d_smax = nullptr;
    unsigned int* d_flag = nullptr;
    double* d_partial = nullptr;          // totals partials and result slots (kTotalsSlot ...)
    double* d_io = nullptr;               // FP64 staging, 11 N
    double* h_small = nullptr;            // pinned scratch for scalars
    cudaGraphExec_t graph = nullptr;
    int graph_mode = -1;                  // 0 fixed dt, 1 cfl
    double graph_value = 0;
    long long steps = 0;
    long long bytes = 0;
};

namespace {

constexpr int kNTileCandidate = WB_NTILE_CANDIDATE;   // tile tables wb_autotune times per axis
static_assert(WB_NTILE_SHAPE == wb::kNTileShape, "tile shape count");

// Tiles of each shape when the table is sorted by shape (then each shape
// runs as its own fixed-shape launch), else all 0.
void tile_split(const std::vector<wb::Tile>& t, int split[3]) {
    split[0] = split[1] = split[2] = 0;
    int prev = 0;
    for (const wb::Tile& x : t) {
        const int sh = (int)((unsigned)x.x >> 24);
        if (sh < prev || sh >= wb::kNTileShape) {
            split[0] = split[1] = split[2] = 0;
            return;
        }
        split[sh]++;
        prev = sh;
    }
}

template <class T>
void set_split(wb::SweepArgs<T>& a, const int split[3]) {
    for (int i = 0; i < 3; i++) a.split[i] = split[i];
}

template <class T>
int enqueue_stages(wb_grid* g, Prof* pf) {
    const long long N = g->N;
    T* un = static_cast<T*>(g->un);
    T* uk = static_cast<T*>(g->uk);
    T* acc = static_cast<T*>(g->acc);
    T* flux = static_cast<T*>(g->flux);
    T* er = static_cast<T*>(g->er);
    const int nstage = g->integrator == WB_RK4 ? 4 : 3;
    for (int st = 0; st < nstage; st++) {
        // per-step totals read un on the side stream; the last stage writes un
        if (st == nstage - 1 && g->step_totals && !pf) WB_CK(cudaStreamWaitEvent(g->stream, g->ev_join, 0));
        const T* src = st == 0 ? un : uk;
        for (int axis = 0; axis < 3; axis++) {
            wb::SweepArgs<T> a;
            a.src = src;
            a.flux = flux + (long long)axis * wb::kNFlux * N;
            a.er = (axis == 0 && g->emf_mode == 0) ? er : nullptr;
            a.tiles = g->d_tiles[axis];
            a.patches = g->d_patches;
    a.links = g->d_links;
            a.ncells = N;
            a.gamma = g->gamma;
            a.zweights = g->weights;
            set_split(a, g->tile_split[axis]);
            a.lstats = g->d_lstats;
            a.queue = g->d_queue + axis;
            a.flag = g->d_flag;
            int rc = prof_begin(pf, g->stream);
            if (rc != WB_OK) return rc;
            if constexpr (sizeof(T) == 4) {
                if (g->precision == WB_FP32_LEARNED)
                    WB_CK(launch_learned(g, axis, a));
                else
                    WB_CK(wb::launch_sweep<T>(axis, a, g->ntiles[axis], g->stream));
            } else {
                WB_CK(wb::launch_sweep<T>(axis, a, g->ntiles[axis], g->stream));
            }
            if ((rc = prof_end(pf, g->stream, WB_K_SWEEP_X + axis)) != WB_OK) return rc;
        }
        wb::UpdateArgs<T> u;
        u.un = un;
        u.uk = src;
        u.dst = (st == nstage - 1) ? un : uk;
        u.acc = acc;
        u.flux = flux;
        u.er = g->emf_mode == 0 ? er : nullptr;
        u.blocks = g->d_blocks;
        u.patches = g->d_patches;
        u.links = g->d_links;
        u.vblocks = g->d_vblocks;
        u.nvblocks = g->nvblocks;
        u.flag = g->d_flag;
        u.dt = g->d_scalars;
        u.ncells = N;
        u.idx = 1.0 / g->dx;
        u.idy = 1.0 / g->dy;
        u.idz = 1.0 / g->dz;
        u.stage = st;
        u.integrator = g->integrator;
        u.emf_mode = g->emf_mode;
        u.emf = static_cast<T*>(g->emf);
        int rc = prof_begin(pf, g->stream);
        if (rc != WB_OK) return rc;
        WB_CK(wb::launch_emf<T>(u, g->nblocks, g->stream));
        if ((rc = prof_end(pf, g->stream, WB_K_EMF)) != WB_OK) return rc;
        if ((rc = prof_begin(pf, g->stream)) != WB_OK) return rc;
        WB_CK(wb::launch_update<T>(u, g->nblocks, g->stream));
        if ((rc = prof_end(pf, g->stream, WB_K_UPDATE)) != WB_OK) return rc;
    }
    return WB_OK;
}

int enqueue_cfl(wb_grid* g, Prof* pf = nullptr) {
    int rc = prof_begin(pf, g->stream);
    if (rc != WB_OK) return rc;
    WB_CK(cudaMemsetAsync(g->d_smax, 0, sizeof(unsigned long long), g->stream));
    if (g->precision == WB_FP64)
        WB_CK(wb::launch_cfl<double>(static_cast<const double*>(g->un), g->d_blocks, g->d_patches, g->d_links,
                                     g->N, g->nblocks, g->d_vblocks, g->nvblocks, 1.0 / g->dx,
                                     1.0 / g->dy, 1.0 / g->dz, g->gamma, g->d_smax, g->d_flag,
                                     g->stream));
    else
        WB_CK(wb::launch_cfl<float>(static_cast<const float*>(g->un), g->d_blocks, g->d_patches, g->d_links,
                                    g->N, g->nblocks, g->d_vblocks, g->nvblocks, 1.0 / g->dx,
                                    1.0 / g->dy, 1.0 / g->dz, g->gamma, g->d_smax, g->d_flag,
                                    g->stream));
    return prof_end(pf, g->stream, WB_K_CFL);
}

// d_partial: kPartials*8 pass-1 partials, then 8 totals (wb_conserved_totals),
// 8 per-step totals, 2 words of the div b maxima.
constexpr int kTotalsSlot = kPartials * 8, kStepTotalsSlot = kPartials * 8 + 8, kDivbSlot = kPartials * 8 + 16;

int enqueue_totals(wb_grid* g, Prof* pf = nullptr, cudaStream_t st = nullptr, int slot = kTotalsSlot) {
    if (!st) st = g->stream;
    double* res = g->d_partial + slot;
    const double dV = g->dx * g->dy * g->dz;
    int rc = prof_begin(pf, st);
    if (rc != WB_OK) return rc;
    if (g->precision == WB_FP64)
        WB_CK(wb::launch_totals<double>(static_cast<const double*>(g->un), g->d_patches, g->npatch,
                                        g->N, g->d_partial, kPartials, dV, res, st));
    else
        WB_CK(wb::launch_totals<float>(static_cast<const float*>(g->un), g->d_patches, g->npatch,
                                       g->N, g->d_partial, kPartials, dV, res, st));
    return prof_end(pf, st, WB_K_TOTALS);
}

// One step: mode 0 fixed dt = value, mode 1 dt = value / smax.
int enqueue_step(wb_grid* g, int mode, double value, Prof* pf = nullptr) {
    int rc;
    if (g->step_totals && !pf) {
        // totals of the step's start state, beside the CFL kernel and the
        // first stages (joined before the last stage overwrites the state)
        WB_CK(cudaEventRecord(g->ev_fork, g->stream));
        WB_CK(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        if ((rc = enqueue_totals(g, nullptr, g->side, kStepTotalsSlot)) != WB_OK) return rc;
        WB_CK(cudaEventRecord(g->ev_join, g->side));
    }
    if (mode == 1) {
        if ((rc = enqueue_cfl(g, pf)) != WB_OK) return rc;
        if ((rc = prof_begin(pf, g->stream)) != WB_OK) return rc;
        WB_CK(wb::launch_set_dt(g->d_smax, value, 0.0, g->d_scalars, g->d_scalars + 1, g->stream));
    } else {
        if ((rc = prof_begin(pf, g->stream)) != WB_OK) return rc;
        WB_CK(wb::launch_set_dt(g->d_smax, 0.0, value, g->d_scalars, g->d_scalars + 1, g->stream));
    }
    if ((rc = prof_end(pf, g->stream, WB_K_DT)) != WB_OK) return rc;
    return g->precision == WB_FP64 ? enqueue_stages<double>(g, pf) : enqueue_stages<float>(g, pf);
}

int capture_step(wb_grid* g, int mode, double value) {
    if (g->graph && g->graph_mode == mode && g->graph_value == value) return WB_OK;
    if (g->graph) {
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    WB_CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(g, mode, value);
    cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
    if (rc != WB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    WB_CK(ce);
    cudaError_t ie = cudaGraphInstantiate(&g->graph, graph, 0);
    cudaGraphDestroy(graph);
    WB_CK(ie);
    g->graph_mode = mode;
    g->graph_value = value;
    return WB_OK;
}

int run_steps(wb_grid* g, int mode, double value, int nsteps) {
    if (g->precision == WB_FP32_LEARNED && !g->d_mlp)
        return fail(WB_EINVAL, "learned grid: install the networks with wb_set_mlp first");
    WB_CK(cudaSetDevice(g->device));
    int rc = capture_step(g, mode, value);
    if (rc != WB_OK) return rc;
    for (int s = 0; s < nsteps; s++) WB_CK(cudaGraphLaunch(g->graph, g->stream));
    g->steps += nsteps;
    return WB_OK;
}

int check_flag(wb_grid* g) {
    WB_CK(cudaMemcpyAsync(g->h_small, g->d_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                          g->stream));
    WB_CK(cudaStreamSynchronize(g->stream));
    unsigned int f = *reinterpret_cast<unsigned int*>(g->h_small);
    if (f) {
        WB_CK(cudaMemsetAsync(g->d_flag, 0, sizeof(unsigned int), g->stream));
        WB_CK(cudaStreamSynchronize(g->stream));
        if (f & wb::kFlagBounds)
            return fail(WB_EINTERNAL, "a kernel formed an index outside its array (bounds-checked build)");
        if (f & wb::kFlagTimeout)
            return fail(WB_ETIMEOUT, "a learned sweep's wait for the tensor cores ran out");
        return fail(WB_ENONFINITE, "state holds %s",
                    (f & 1u) ? "NaN/Inf values" : "non-positive density or pressure");
    }
    return WB_OK;
}

cudaError_t launch_learned(wb_grid* g, int axis, const wb::SweepArgs<float>& a) {
    if (WB_LEARNED_ENGINE == 1)
        return wb::launch_sweep_learned_tc(axis, a, g->ntiles[axis], g->d_mlp_tc, (float)g->kappa,
                                           (float)g->pjump, (float)g->smooth, g->stream);
    return wb::launch_sweep_learned(axis, a, g->ntiles[axis], g->d_mlp, (float)g->kappa, (float)g->pjump,
                                    (float)g->smooth, g->stream);
}

// The address under which the grid's device reads or writes a host array in
// place: page-locked memory mapped at the same address (cudaHostAlloc
// memory under unified addressing, e.g. a pinned torch tensor), allocated
// while that device was current.  nullptr for pageable memory, which is
// staged through a copy instead.
template <class P>
P* mapped(const wb_grid* g, P* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer != static_cast<const void*>(host) ||
        a.device != g->device)
        return nullptr;
    return host;
}

int upload(wb_grid* g, const double* U, const double* b) {
    const long long N = g->N;
    if (mapped(g, U) && mapped(g, b)) {      // the import kernel reads the host arrays in place
        if (g->precision == WB_FP64)
            WB_CK((wb::launch_import<double, double>(U, b, static_cast<double*>(g->un), g->d_blocks,
                                                     g->d_patches, N, g->nblocks, g->stream)));
        else
            WB_CK((wb::launch_import<float, double>(U, b, static_cast<float*>(g->un), g->d_blocks,
                                                    g->d_patches, N, g->nblocks, g->stream)));
        return WB_OK;
    }
    WB_CK(cudaMemcpyAsync(g->d_io, U, sizeof(double) * 8 * N, cudaMemcpyHostToDevice, g->stream));
    WB_CK(cudaMemcpyAsync(g->d_io + 8 * N, b, sizeof(double) * 3 * N, cudaMemcpyHostToDevice,
                          g->stream));
    if (g->precision == WB_FP64)
        WB_CK((wb::launch_import<double, double>(g->d_io, g->d_io + 8 * N, static_cast<double*>(g->un),
                                        g->d_blocks, g->d_patches, N, g->nblocks, g->stream)));
    else
        WB_CK((wb::launch_import<float, double>(g->d_io, g->d_io + 8 * N, static_cast<float*>(g->un),
                                       g->d_blocks, g->d_patches, N, g->nblocks, g->stream)));
    return WB_OK;
}

void release(wb_grid* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    if (g->side) cudaStreamSynchronize(g->side);
    void* ptrs[] = {g->un, g->uk, g->acc, g->flux, g->er, g->emf, g->d_mlp, g->d_mlp_tc, g->d_lstats, g->d_queue,
                    g->d_patches, g->d_links, g->d_tiles[0], g->d_tiles[1], g->d_tiles[2], g->d_blocks,
                    g->d_vblocks, g->d_scalars, g->d_smax, g->d_flag, g->d_partial, g->d_io};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->h_small) cudaFreeHost(g->h_small);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->side) cudaStreamDestroy(g->side);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

// Sweep tiles of `axis` for every patch.  policy >= 0: that tile shape
// everywhere; policy < 0: per patch the shape needing the fewest thread slots
// (ragged tiles at the patch edges idle threads), ties to the lower shape;
// policy -2 then orders the table by shape (a fixed-shape launch per shape).
// The shape goes into the top byte of the tile's patch field.
std::vector<wb::Tile> build_tiles(const wb_grid* g, int axis, int policy) {
    std::vector<wb::Tile> out;
    for (int p = 0; p < g->npatch; p++) {
        const wb::PatchDev& P = g->h_patches[p];
        const int na = axis == 0 ? P.nx : (axis == 1 ? P.ny : P.nz);
        const int npn = axis == 0 ? P.ny : P.nx;
        const int n3 = axis == 0 ? P.nz : (axis == 1 ? P.nz : P.ny);
        int best = policy;
        if (policy < 0) {
            long long slots = -1;
            for (int sh = 0; sh < wb::kNTileShape; sh++) {
                int ta, tp;
                wb::sweep_shape(axis, sh, &ta, &tp);
                const long long n = (long long)((na + ta - 1) / ta) * ((npn + tp - 1) / tp) * n3;
                if (slots < 0 || n < slots) { slots = n; best = sh; }
            }
        }
        int ta, tp;
        if (g->precision == WB_FP32_LEARNED) {
            // the learned sweep's own tile
            if (WB_LEARNED_ENGINE == 1) wb::learned_tc_shape(axis, &ta, &tp);
            else wb::learned_shape(axis, &ta, &tp);
            best = 0;
        } else {
            wb::sweep_shape(axis, best, &ta, &tp);
        }
        const int px = p | (best << 24);
        if (axis == 0) {
            for (int z = 0; z < P.nz; z++)
                for (int y0 = 0; y0 < P.ny; y0 += tp)
                    for (int x0 = 0; x0 < P.nx; x0 += ta) out.push_back(wb::Tile{px, x0, y0, z});
        } else if (axis == 1) {
            for (int z = 0; z < P.nz; z++)
                for (int y0 = 0; y0 < P.ny; y0 += ta)
                    for (int x0 = 0; x0 < P.nx; x0 += tp) out.push_back(wb::Tile{px, y0, x0, z});
        } else {
            for (int y = 0; y < P.ny; y++)
                for (int z0 = 0; z0 < P.nz; z0 += ta)
                    for (int x0 = 0; x0 < P.nx; x0 += tp) out.push_back(wb::Tile{px, z0, x0, y});
        }
    }
    if (policy == -2)
        std::stable_sort(out.begin(), out.end(), [](const wb::Tile& a, const wb::Tile& b) {
            return ((unsigned)a.x >> 24) < ((unsigned)b.x >> 24);
        });
    return out;
}

// Checks a patch link table (layout of wb::locate): every entry names a
// patch, the centre entry is the patch itself, links are reciprocal, a
// diagonal link is the composition of single-axis moves in any order,
// linked patches agree in their extents along the axes they are not offset
// in, and a patch met across an axis from a different patch is at least 3
// cells deep along it (the stencil reach), as is the patch left behind.
int check_links(const std::vector<wb::PatchDev>& P, const int* L) {
    const long long n = (long long)P.size();
    auto at = [&](long long p, int ox, int oy, int oz) {
        return L[27 * p + 9 * (oz + 1) + 3 * (oy + 1) + (ox + 1)];
    };
    auto ext = [&](long long p, int d) { return d == 0 ? P[p].nx : (d == 1 ? P[p].ny : P[p].nz); };
    for (long long p = 0; p < n; p++)
        for (int oz = -1; oz <= 1; oz++)
            for (int oy = -1; oy <= 1; oy++)
                for (int ox = -1; ox <= 1; ox++) {
                    const int q = at(p, ox, oy, oz);
                    if (q < 0 || q >= n)
                        return fail(WB_EINVAL, "links: patch %lld direction (%d,%d,%d) names patch %d",
                                    p, ox, oy, oz, q);
                }
    for (long long p = 0; p < n; p++) {
        if (at(p, 0, 0, 0) != p) return fail(WB_EINVAL, "links: centre entry of patch %lld is not itself", p);
        for (int oz = -1; oz <= 1; oz++)
            for (int oy = -1; oy <= 1; oy++)
                for (int ox = -1; ox <= 1; ox++) {
                    if (!ox && !oy && !oz) continue;
                    const int o[3] = {ox, oy, oz};
                    const int q = at(p, ox, oy, oz);
                    if (at(q, -ox, -oy, -oz) != p)
                        return fail(WB_EINVAL, "links: patch %lld -> %d along (%d,%d,%d) is not reciprocal",
                                    p, q, ox, oy, oz);
                    for (int d = 0; d < 3; d++) {
                        if (o[d] == 0) {
                            if (ext(q, d) != ext(p, d))
                                return fail(WB_EINVAL, "links: patches %lld and %d differ in extent %d",
                                            p, q, d);
                            continue;
                        }
                        int e[3] = {0, 0, 0}, r[3] = {ox, oy, oz};
                        e[d] = o[d];
                        r[d] = 0;
                        const int f = at(p, e[0], e[1], e[2]);
                        if (at(f, r[0], r[1], r[2]) != q)
                            return fail(WB_EINVAL, "links: patch %lld direction (%d,%d,%d) is not the "
                                        "composition of its moves", p, ox, oy, oz);
                        if (f != p && (ext(p, d) < 3 || ext(f, d) < 3))
                            return fail(WB_EINVAL, "links: patches %lld and %d meet along axis %d with "
                                        "fewer than 3 cells", p, f, d);
                    }
                }
    }
    return WB_OK;
}

// 1 when every tile uses shape 0 (then one tile per block, no dispatch).
template <class P>
int dmalloc(wb_grid* g, P** p, size_t bytes) {
    WB_CK(cudaMalloc(reinterpret_cast<void**>(p), bytes));
    g->bytes += (long long)bytes;
    return WB_OK;
}

template <class T>
int face_fluxes_impl(wb_grid* g, int axis, double* F_out) {
    const long long N = g->N;
    T* flux = static_cast<T*>(g->flux) + (long long)axis * wb::kNFlux * N;
    wb::SweepArgs<T> a;
    a.src = static_cast<const T*>(g->un);
    a.flux = flux;
    a.er = nullptr;
    a.tiles = g->d_tiles[axis];
    a.patches = g->d_patches;
    a.links = g->d_links;
    a.ncells = N;
    a.gamma = g->gamma;
    a.zweights = g->weights;
    set_split(a, g->tile_split[axis]);
    a.flag = g->d_flag;
    if constexpr (sizeof(T) == 4) {
        if (g->precision == WB_FP32_LEARNED) {
            if (!g->d_mlp) return fail(WB_EINVAL, "learned grid: install the networks with wb_set_mlp first");
            WB_CK(launch_learned(g, axis, a));
        } else {
            WB_CK(wb::launch_sweep<T>(axis, a, g->ntiles[axis], g->stream));
        }
    } else {
        WB_CK(wb::launch_sweep<T>(axis, a, g->ntiles[axis], g->stream));
    }
    // 7 N doubles fit the 11 N staging buffer
    WB_CK(wb::launch_export_flux<T>(flux, g->d_io, g->d_blocks, g->d_patches, N, g->nblocks,
                                    g->stream));
    WB_CK(cudaMemcpyAsync(F_out, g->d_io, sizeof(double) * 7 * N, cudaMemcpyDeviceToHost,
                          g->stream));
    WB_CK(cudaStreamSynchronize(g->stream));
    return check_flag(g);        // a bounds or tensor-core wait failure of the sweep
}

template <class T>
int time_sweep(wb_grid* g, int axis, const wb::Tile* tiles, int ntiles, const int split[3], float* ms) {
    wb::SweepArgs<T> a;
    a.src = static_cast<const T*>(g->un);
    a.flux = static_cast<T*>(g->flux) + (long long)axis * wb::kNFlux * g->N;
    a.er = nullptr;
    a.tiles = tiles;
    a.patches = g->d_patches;
    a.links = g->d_links;
    a.ncells = g->N;
    a.gamma = g->gamma;
    a.zweights = g->weights;
    set_split(a, split);
    a.queue = g->d_queue + axis;
    a.flag = g->d_flag;
    cudaEvent_t e0, e1;
    WB_CK(cudaEventCreate(&e0));
    WB_CK(cudaEventCreate(&e1));
    WB_CK(wb::launch_sweep<T>(axis, a, ntiles, g->stream));
    WB_CK(cudaEventRecord(e0, g->stream));
    WB_CK(wb::launch_sweep<T>(axis, a, ntiles, g->stream));
    WB_CK(wb::launch_sweep<T>(axis, a, ntiles, g->stream));
    WB_CK(cudaEventRecord(e1, g->stream));
    WB_CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(ms, e0, e1);
    *ms *= 0.5f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return WB_OK;
}

}  // namespace

int wb::set_last_error(int code, const char* msg) {
    g_err = msg;
    return code;
}

extern "C" {

const char* wb_last_error(void) { return g_err.c_str(); }

const char* wb_version(void) { return "wombat-gb300 0.1 (sm_103a)"; }

int wb_init_grid(const wb_grid_desc* d, const double* U0, const double* b0, void* cuda_stream,
                 wb_grid** out) {
    g_err.clear();
    if (!d || !U0 || !b0 || !out) return fail(WB_EINVAL, "null argument");
    *out = nullptr;
    if (d->npatch < 1 || !d->dims) return fail(WB_EINVAL, "npatch must be >= 1 with dims");
    // a sweep tile keeps its patch index in 24 bits (the top byte holds the shape)
    if (d->npatch >= (1 << 24)) return fail(WB_EINVAL, "npatch must be < 2^24, got %d", d->npatch);
    if (d->ghost != 3) return fail(WB_EINVAL, "ghost must be 3 (WENO5 stencil), got %d", d->ghost);
    if (!(d->dx > 0) || !(d->dy > 0) || !(d->dz > 0)) return fail(WB_EINVAL, "dx, dy, dz must be > 0");
    if (!(d->gamma > 1.0)) return fail(WB_EINVAL, "gamma must be > 1");
    if (d->precision != WB_FP64 && d->precision != WB_FP32 && d->precision != WB_FP32_LEARNED)
        return fail(WB_EINVAL, "unknown precision %d", d->precision);
    if (d->integrator != WB_SSPRK3 && d->integrator != WB_RK4)
        return fail(WB_EINVAL, "unknown integrator %d", d->integrator);
    if (d->emf_mode != 0 && d->emf_mode != 1) return fail(WB_EINVAL, "unknown emf_mode %d", d->emf_mode);
    if (d->weights != 0 && d->weights != 1) return fail(WB_EINVAL, "unknown weights %d", d->weights);
    if (d->weights == 1 && d->precision == WB_FP32_LEARNED)
        return fail(WB_EINVAL, "WENO-Z weights and learned weights exclude each other");

    wb_grid* g = new (std::nothrow) wb_grid();
    if (!g) return fail(WB_ENOMEM, "host allocation failed");
    g->npatch = d->npatch;
    g->dx = d->dx; g->dy = d->dy; g->dz = d->dz; g->gamma = d->gamma;
    g->precision = d->precision; g->integrator = d->integrator; g->emf_mode = d->emf_mode;
    g->weights = d->weights;
    g->tsize = d->precision == WB_FP64 ? 8 : 4;
    long long off = 0;
    for (int p = 0; p < d->npatch; p++) {
        const int nx = d->dims[3 * p], ny = d->dims[3 * p + 1], nz = d->dims[3 * p + 2];
        if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096) {
            delete g;
            return fail(WB_EINVAL, "patch %d: sizes (%d,%d,%d) outside [1,4096]", p, nx, ny, nz);
        }
        const long long np = (long long)nx * ny * nz;
        if (np >= (1LL << 31)) {
            delete g;
            return fail(WB_EINVAL, "patch %d: more than 2^31-1 cells", p);
        }
        g->h_patches.push_back(wb::PatchDev{nx, ny, nz, 0, off});
        off += np;
    }
    g->N = off;
    if (d->links) {
        const int lrc = check_links(g->h_patches, d->links);
        if (lrc != WB_OK) {
            delete g;
            return lrc;
        }
    }

    int rc;
    auto bail = [&](int code) { release(g); return code; };
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return fail(WB_ECUDA, "no CUDA device available");
    }
    if (cuda_stream) {
        g->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete g;
            return fail(WB_ECUDA, "stream creation failed");
        }
        g->own_stream = true;
    }
    // tiles and cell blocks
    std::vector<wb::Tile> tiles[3];
    std::vector<wb::CellBlock> blocks;
    for (int a = 0; a < 3; a++) tiles[a] = build_tiles(g, a, g->precision == WB_FP32_LEARNED ? 0 : -2);
    for (int p = 0; p < g->npatch; p++) {
        const wb::PatchDev& P = g->h_patches[p];
        const long long np = (long long)P.nx * P.ny * P.nz;
        for (long long c = 0; c < np; c += wb::kCellBlock) blocks.push_back(wb::CellBlock{p, (int)c});
    }
    for (int a = 0; a < 3; a++) {
        if (tiles[a].size() > 0x7fffffffULL) return bail(fail(WB_EINVAL, "grid too large"));
        g->ntiles[a] = (int)tiles[a].size();
        tile_split(tiles[a], g->tile_split[a]);
    }
    g->nblocks = (int)blocks.size();
    // vector blocks: periodic patches whose x extent is a multiple of the width
    std::vector<wb::CellBlock> vblocks;
    {
        const int V = wb::update_vector_width(g->precision == WB_FP64);
        bool ok = d->links == nullptr;
        for (const wb::PatchDev& P : g->h_patches) ok = ok && P.nx % V == 0;
        if (ok)
            for (int p = 0; p < g->npatch; p++) {
                const wb::PatchDev& P = g->h_patches[p];
                const long long np = (long long)P.nx * P.ny * P.nz;
                for (long long c = 0; c < np; c += (long long)wb::kCellBlock * V)
                    vblocks.push_back(wb::CellBlock{p, (int)c});
            }
        g->nvblocks = (int)vblocks.size();
    }

    const size_t T = g->tsize;
    const long long N = g->N;
    if ((rc = dmalloc(g, &g->un, T * 8 * N))) return bail(rc);
    if ((rc = dmalloc(g, &g->uk, T * 8 * N))) return bail(rc);
    if (g->integrator == WB_RK4 && (rc = dmalloc(g, &g->acc, T * 8 * N))) return bail(rc);
    if ((rc = dmalloc(g, &g->flux, T * 3 * wb::kNFlux * N))) return bail(rc);
    if (g->emf_mode == 0 && (rc = dmalloc(g, &g->er, T * 3 * N))) return bail(rc);
    if ((rc = dmalloc(g, &g->emf, T * 3 * N))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_patches, sizeof(wb::PatchDev) * g->npatch))) return bail(rc);
    if (d->links && (rc = dmalloc(g, &g->d_links, sizeof(int) * 27 * (size_t)g->npatch))) return bail(rc);
    for (int a = 0; a < 3; a++)
        if ((rc = dmalloc(g, &g->d_tiles[a], sizeof(wb::Tile) * tiles[a].size()))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_blocks, sizeof(wb::CellBlock) * blocks.size()))) return bail(rc);
    if (!vblocks.empty() &&
        (rc = dmalloc(g, &g->d_vblocks, sizeof(wb::CellBlock) * vblocks.size()))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_scalars, sizeof(double) * 2))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_smax, sizeof(unsigned long long)))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_flag, sizeof(unsigned int)))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_partial, sizeof(double) * (kPartials * 8 + 18)))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_io, sizeof(double) * 11 * N))) return bail(rc);
    if (g->precision == WB_FP32_LEARNED &&
        (rc = dmalloc(g, &g->d_lstats, sizeof(unsigned long long) * 2))) return bail(rc);
    if ((rc = dmalloc(g, &g->d_queue, sizeof(int) * 3))) return bail(rc);
    if (cudaMallocHost(reinterpret_cast<void**>(&g->h_small), 256) != cudaSuccess)
        return bail(fail(WB_ENOMEM, "pinned host allocation failed"));

    auto cp = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, g->stream);
    };
    if (d->links && cp(g->d_links, d->links, sizeof(int) * 27 * (size_t)g->npatch) != cudaSuccess)
        return bail(fail(WB_ECUDA, "link upload failed"));
    if (cp(g->d_patches, g->h_patches.data(), sizeof(wb::PatchDev) * g->npatch) != cudaSuccess ||
        cp(g->d_blocks, blocks.data(), sizeof(wb::CellBlock) * blocks.size()) != cudaSuccess ||
        (!vblocks.empty() &&
         cp(g->d_vblocks, vblocks.data(), sizeof(wb::CellBlock) * vblocks.size()) != cudaSuccess))
        return bail(fail(WB_ECUDA, "table upload failed: %s", cudaGetErrorString(cudaGetLastError())));
    for (int a = 0; a < 3; a++)
        if (cp(g->d_tiles[a], tiles[a].data(), sizeof(wb::Tile) * tiles[a].size()) != cudaSuccess)
            return bail(fail(WB_ECUDA, "tile upload failed"));
    if ((g->d_lstats &&
         cudaMemsetAsync(g->d_lstats, 0, sizeof(unsigned long long) * 2, g->stream) != cudaSuccess) ||
        cudaMemsetAsync(g->d_scalars, 0, sizeof(double) * 2, g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->d_flag, 0, sizeof(unsigned int), g->stream) != cudaSuccess ||
        cudaMemsetAsync(g->flux, 0, T * 3 * wb::kNFlux * N, g->stream) != cudaSuccess)
        return bail(fail(WB_ECUDA, "memset failed"));
    cudaError_t pe = g->precision == WB_FP64 ? wb::prepare_sweep_kernels<double>()
                                             : wb::prepare_sweep_kernels<float>();
    if (pe == cudaSuccess && g->precision == WB_FP32_LEARNED)
        pe = WB_LEARNED_ENGINE == 1 ? wb::prepare_sweep_learned_tc() : wb::prepare_sweep_learned();
    if (pe != cudaSuccess) return bail(fail(WB_ECUDA, "kernel attributes: %s", cudaGetErrorString(pe)));
    if ((rc = upload(g, U0, b0)) != WB_OK) return bail(rc);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess)
        return bail(fail(WB_ECUDA, "init: %s", cudaGetErrorString(cudaGetLastError())));
    *out = g;
    return WB_OK;
}

int wb_set_state(wb_grid* g, const double* U, const double* b) {
    g_err.clear();
    if (!g || !U || !b) return fail(WB_EINVAL, "null argument");
    WB_CK(cudaSetDevice(g->device));
    return upload(g, U, b);
}

int wb_step(wb_grid* g, double dt, int nsteps) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    if (!(dt > 0) || nsteps < 0) return fail(WB_EINVAL, "need dt > 0 and nsteps >= 0");
    return run_steps(g, 0, dt, nsteps);
}

int wb_step_cfl(wb_grid* g, double cfl, int nsteps) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    if (!(cfl > 0) || nsteps < 0) return fail(WB_EINVAL, "need cfl > 0 and nsteps >= 0");
    return run_steps(g, 1, cfl, nsteps);
}

int wb_step_profiled(wb_grid* g, double cfl, int nsteps, int with_totals, double* kernel_ms,
                     int* launches, double* total_ms) {
    g_err.clear();
    if (!g || !kernel_ms || !launches || !total_ms) return fail(WB_EINVAL, "null argument");
    if (!(cfl > 0) || nsteps < 1) return fail(WB_EINVAL, "need cfl > 0 and nsteps >= 1");
    WB_CK(cudaSetDevice(g->device));
    const int per_step = 2 + (g->integrator == WB_RK4 ? 4 : 3) * 5 + (with_totals ? 1 : 0);
    Prof pf;
    pf.ev.resize((size_t)2 * per_step * nsteps, nullptr);
    int rc = WB_OK;
    for (auto& e : pf.ev) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            rc = fail(WB_ECUDA, "event creation failed");
            break;
        }
    }
    for (int s = 0; s < nsteps && rc == WB_OK; s++) {
        rc = enqueue_step(g, 1, cfl, &pf);
        if (rc == WB_OK && with_totals) rc = enqueue_totals(g, &pf);
    }
    if (rc == WB_OK && cudaStreamSynchronize(g->stream) != cudaSuccess)
        rc = fail(WB_ECUDA, "profiled step: %s", cudaGetErrorString(cudaGetLastError()));
    if (rc == WB_OK) {
        for (int k = 0; k < WB_NKERNEL; k++) { kernel_ms[k] = 0.0; launches[k] = 0; }
        for (size_t l = 0; l < pf.cls.size(); l++) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, pf.ev[2 * l], pf.ev[2 * l + 1]);
            kernel_ms[pf.cls[l]] += ms;
            launches[pf.cls[l]] += 1;
        }
        float tot = 0.f;
        cudaEventElapsedTime(&tot, pf.ev[0], pf.ev[pf.used - 1]);
        *total_ms = tot;
        g->steps += nsteps;
    }
    for (auto& e : pf.ev)
        if (e) cudaEventDestroy(e);
    if (rc != WB_OK) return rc;
    return check_flag(g);
}

int wb_cfl_dt(wb_grid* g, double cfl, double* dt_out) {
    g_err.clear();
    if (!g || !dt_out) return fail(WB_EINVAL, "null argument");
    if (!(cfl > 0)) return fail(WB_EINVAL, "need cfl > 0");
    WB_CK(cudaSetDevice(g->device));
    int rc = enqueue_cfl(g);
    if (rc != WB_OK) return rc;
    WB_CK(cudaMemcpyAsync(g->h_small + 1, g->d_smax, sizeof(double), cudaMemcpyDeviceToHost,
                          g->stream));
    if ((rc = check_flag(g)) != WB_OK) return rc;
    double smax;
    std::memcpy(&smax, g->h_small + 1, sizeof(double));
    if (!(smax > 0)) return fail(WB_ENONFINITE, "no positive signal speed in the state");
    *dt_out = cfl / smax;
    return WB_OK;
}

int wb_set_step_totals(wb_grid* g, int on) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    WB_CK(cudaSetDevice(g->device));
    on = on ? 1 : 0;
    if (on && !g->side) {
        WB_CK(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
        WB_CK(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
        WB_CK(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
    }
    if (on != g->step_totals) {
        WB_CK(cudaStreamSynchronize(g->stream));
        g->step_totals = on;
        if (g->graph) {             // the step changed: capture again
            cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
        }
    }
    return WB_OK;
}

int wb_step_totals(wb_grid* g, double out[8]) {
    g_err.clear();
    if (!g || !out) return fail(WB_EINVAL, "null argument");
    if (!g->step_totals) return fail(WB_EINVAL, "step totals are off (wb_set_step_totals)");
    WB_CK(cudaSetDevice(g->device));
    WB_CK(cudaMemcpyAsync(g->h_small + 2, g->d_partial + kStepTotalsSlot, sizeof(double) * 8,
                          cudaMemcpyDeviceToHost, g->stream));
    const int rc = check_flag(g);
    if (rc != WB_OK) return rc;
    std::memcpy(out, g->h_small + 2, sizeof(double) * 8);
    return WB_OK;
}

int wb_div_b(wb_grid* g, double out[2]) {
    g_err.clear();
    if (!g || !out) return fail(WB_EINVAL, "null argument");
    WB_CK(cudaSetDevice(g->device));
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(g->d_partial + kDivbSlot);
    if (g->precision == WB_FP64)
        WB_CK(wb::launch_divb<double>(static_cast<const double*>(g->un), g->d_blocks, g->d_patches,
                                      g->d_links, g->N, g->nblocks, 1.0 / g->dx, 1.0 / g->dy,
                                      1.0 / g->dz, bits, g->d_flag, g->stream));
    else
        WB_CK(wb::launch_divb<float>(static_cast<const float*>(g->un), g->d_blocks, g->d_patches,
                                     g->d_links, g->N, g->nblocks, 1.0 / g->dx, 1.0 / g->dy,
                                     1.0 / g->dz, bits, g->d_flag, g->stream));
    WB_CK(cudaMemcpyAsync(g->h_small + 2, bits, sizeof(double) * 2, cudaMemcpyDeviceToHost, g->stream));
    const int rc = check_flag(g);
    if (rc != WB_OK) return rc;
    std::memcpy(out, g->h_small + 2, sizeof(double) * 2);
    return WB_OK;
}

int wb_conserved_totals(wb_grid* g, double out[8]) {
    g_err.clear();
    if (!g || !out) return fail(WB_EINVAL, "null argument");
    WB_CK(cudaSetDevice(g->device));
    double* res = g->d_partial + kPartials * 8;
    int rc = enqueue_totals(g);
    if (rc != WB_OK) return rc;
    WB_CK(cudaMemcpyAsync(g->h_small + 2, res, sizeof(double) * 8, cudaMemcpyDeviceToHost, g->stream));
    rc = check_flag(g);
    if (rc != WB_OK) return rc;
    std::memcpy(out, g->h_small + 2, sizeof(double) * 8);
    return WB_OK;
}

int wb_set_state_f32(wb_grid* g, const float* U, const float* b) {
    g_err.clear();
    if (!g || !U || !b) return fail(WB_EINVAL, "null argument");
    if (g->precision == WB_FP64) return fail(WB_EINVAL, "set_state_f32: the grid holds FP64");
    WB_CK(cudaSetDevice(g->device));
    const long long N = g->N;
    if (mapped(g, U) && mapped(g, b)) {      // the import kernel reads the host arrays in place
        WB_CK((wb::launch_import<float, float>(U, b, static_cast<float*>(g->un), g->d_blocks,
                                              g->d_patches, N, g->nblocks, g->stream)));
        return WB_OK;
    }
    float* io = reinterpret_cast<float*>(g->d_io);
    WB_CK(cudaMemcpyAsync(io, U, sizeof(float) * 8 * N, cudaMemcpyHostToDevice, g->stream));
    WB_CK(cudaMemcpyAsync(io + 8 * N, b, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, g->stream));
    WB_CK((wb::launch_import<float, float>(io, io + 8 * N, static_cast<float*>(g->un), g->d_blocks,
                                          g->d_patches, N, g->nblocks, g->stream)));
    return WB_OK;
}

int wb_get_state_f32(wb_grid* g, float* U_out, float* b_out) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    if (g->precision == WB_FP64) return fail(WB_EINVAL, "get_state_f32: the grid holds FP64");
    WB_CK(cudaSetDevice(g->device));
    const long long N = g->N;
    if ((!U_out || mapped(g, U_out)) && (!b_out || mapped(g, b_out))) {
        // the export kernel writes the host arrays in place
        WB_CK((wb::launch_export<float, float>(static_cast<const float*>(g->un), U_out, b_out, g->d_blocks,
                                              g->d_patches, g->d_links, N, g->nblocks, g->stream)));
        return check_flag(g);
    }
    float* io = reinterpret_cast<float*>(g->d_io);
    float* dU = U_out ? io : nullptr;
    float* db = b_out ? io + 8 * N : nullptr;
    WB_CK((wb::launch_export<float, float>(static_cast<const float*>(g->un), dU, db, g->d_blocks,
                                          g->d_patches, g->d_links, N, g->nblocks, g->stream)));
    if (U_out)
        WB_CK(cudaMemcpyAsync(U_out, dU, sizeof(float) * 8 * N, cudaMemcpyDeviceToHost, g->stream));
    if (b_out)
        WB_CK(cudaMemcpyAsync(b_out, db, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, g->stream));
    return check_flag(g);
}

int wb_get_state(wb_grid* g, double* U_out, double* b_out) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    WB_CK(cudaSetDevice(g->device));
    const long long N = g->N;
    const bool in_place = (!U_out || mapped(g, U_out)) && (!b_out || mapped(g, b_out));
    double* dU = U_out ? (in_place ? U_out : g->d_io) : nullptr;
    double* db = b_out ? (in_place ? b_out : g->d_io + 8 * N) : nullptr;
    if (g->precision == WB_FP64)
        WB_CK((wb::launch_export<double, double>(static_cast<const double*>(g->un), dU, db, g->d_blocks,
                                        g->d_patches, g->d_links, N, g->nblocks, g->stream)));
    else
        WB_CK((wb::launch_export<float, double>(static_cast<const float*>(g->un), dU, db, g->d_blocks,
                                       g->d_patches, g->d_links, N, g->nblocks, g->stream)));
    if (U_out && !in_place)
        WB_CK(cudaMemcpyAsync(U_out, dU, sizeof(double) * 8 * N, cudaMemcpyDeviceToHost, g->stream));
    if (b_out && !in_place)
        WB_CK(cudaMemcpyAsync(b_out, db, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, g->stream));
    return check_flag(g);
}

int wb_face_fluxes(wb_grid* g, int axis, double* F_out) {
    g_err.clear();
    if (!g || !F_out) return fail(WB_EINVAL, "null argument");
    if (axis < 0 || axis > 2) return fail(WB_EINVAL, "axis must be 0, 1 or 2");
    WB_CK(cudaSetDevice(g->device));
    return g->precision == WB_FP64 ? face_fluxes_impl<double>(g, axis, F_out)
                                   : face_fluxes_impl<float>(g, axis, F_out);
}

int wb_harvest(wb_grid* g, int axis, const long long* cells, long long n, const double* hU,
               const double* hF, double kappa, double pjump, float* records_out) {
    g_err.clear();
    if (!g || !cells || !hU || !hF || !records_out || n < 1)
        return fail(WB_EINVAL, "harvest: null argument or no samples");
    if (g->precision != WB_FP64) return fail(WB_EINVAL, "harvest: needs an FP64 grid");
    if (axis < 0 || axis > 2) return fail(WB_EINVAL, "harvest: axis must be 0, 1 or 2");
    if (g->d_links) return fail(WB_EINVAL, "harvest: needs a periodic patch 0 (grid has links)");
    const wb::PatchDev& P = g->h_patches[0];
    const long long np = (long long)P.nx * P.ny * P.nz;
    for (long long t = 0; t < n; t++)
        if (cells[t] < 0 || cells[t] >= np) return fail(WB_EINVAL, "harvest: cell index outside patch 0");
    WB_CK(cudaSetDevice(g->device));
    long long* dc = nullptr;
    double* dh = nullptr;
    float* dout = nullptr;
    const size_t nrec = (size_t)n * 14 * WB_MLP_RECORD;
    cudaError_t e = cudaMalloc(&dc, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dh, sizeof(double) * 14 * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(float) * nrec);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, cells, sizeof(long long) * n, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dh, hU, sizeof(double) * 7 * n, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dh + 7 * n, hF, sizeof(double) * 7 * n, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = wb::launch_harvest<double>(static_cast<const double*>(g->un), g->N, P, axis, dc, n, dh,
                                       dh + 7 * n, g->gamma, kappa, pjump, dout, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(records_out, dout, sizeof(float) * nrec, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (dc) cudaFree(dc);
    if (dh) cudaFree(dh);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) return fail(WB_ECUDA, "harvest: %s", cudaGetErrorString(e));
    return WB_OK;
}

int wb_cell_state_flux(wb_grid* g, int axis, double* X_out, double* F_out) {
    g_err.clear();
    if (!g || !X_out || !F_out) return fail(WB_EINVAL, "cell_state_flux: null argument");
    if (g->precision != WB_FP64) return fail(WB_EINVAL, "cell_state_flux: needs an FP64 grid");
    if (axis < 0 || axis > 2) return fail(WB_EINVAL, "cell_state_flux: axis must be 0, 1 or 2");
    if (g->d_links) return fail(WB_EINVAL, "cell_state_flux: needs a periodic patch 0 (grid has links)");
    const wb::PatchDev& P = g->h_patches[0];
    const long long np = (long long)P.nx * P.ny * P.nz;
    WB_CK(cudaSetDevice(g->device));
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * 14 * np);
    if (e == cudaSuccess)
        e = wb::launch_cell_state_flux<double>(static_cast<const double*>(g->un), g->N, P, axis, g->gamma,
                                               d, d + 7 * np, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(X_out, d, sizeof(double) * 7 * np, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(F_out, d + 7 * np, sizeof(double) * 7 * np, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return fail(WB_ECUDA, "cell_state_flux: %s", cudaGetErrorString(e));
    return WB_OK;
}

int wb_set_mlp(wb_grid* g, const float* params, double kappa, double pjump) {
    g_err.clear();
    if (!g || !params) return fail(WB_EINVAL, "null argument");
    if (g->precision != WB_FP32_LEARNED) return fail(WB_EINVAL, "wb_set_mlp needs a WB_FP32_LEARNED grid");
    if (!(kappa > 0) || !(pjump > 0)) return fail(WB_EINVAL, "kappa and pjump must be > 0");
    WB_CK(cudaSetDevice(g->device));
    const size_t words = wb::mlp_fragment_words();
    std::vector<uint32_t> frag(words);
    wb::mlp_fragments(params, frag.data());
    if (!g->d_mlp) {
        int rc = dmalloc(g, &g->d_mlp, sizeof(uint32_t) * words);
        if (rc != WB_OK) return rc;
    }
    WB_CK(cudaMemcpyAsync(g->d_mlp, frag.data(), sizeof(uint32_t) * words, cudaMemcpyHostToDevice, g->stream));
    const size_t tcb = wb::mlp_tc_image_bytes();
    std::vector<unsigned char> img(tcb);
    wb::mlp_tc_image(params, img.data());
    if (!g->d_mlp_tc) {
        int rc = dmalloc(g, &g->d_mlp_tc, tcb);
        if (rc != WB_OK) return rc;
    }
    WB_CK(cudaMemcpyAsync(g->d_mlp_tc, img.data(), tcb, cudaMemcpyHostToDevice, g->stream));
    WB_CK(cudaStreamSynchronize(g->stream));
    g->kappa = kappa;
    g->pjump = pjump;
    if (g->graph) {              // kernel arguments changed: capture again
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    return WB_OK;
}

int wb_set_mlp_gate(wb_grid* g, double smooth) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    if (g->precision != WB_FP32_LEARNED) return fail(WB_EINVAL, "wb_set_mlp_gate needs a WB_FP32_LEARNED grid");
    if (!(smooth >= 0) || !(smooth < 1e30)) return fail(WB_EINVAL, "smooth must be >= 0 and finite");
    g->smooth = smooth;
    if (g->graph) {              // kernel arguments changed: capture again
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    return WB_OK;
}

namespace {

// build_tiles policy of wb_autotune's candidate table c: 0 the per-patch
// model (one persistent launch), 1..3 each fixed shape, 4 the per-patch
// model ordered by shape (a launch per shape)
int candidate_policy(int c) { return c == 0 ? -1 : (c <= wb::kNTileShape ? c - 1 : -2); }

// Builds and uploads the tile table of `axis` for `policy` (synchronous).
int install_tiles(wb_grid* g, int axis, int policy) {
    std::vector<wb::Tile> t = build_tiles(g, axis, policy);
    // the new table is uploaded into its own buffer first: on failure the
    // grid keeps its current table
    wb::Tile* d = nullptr;
    WB_CK(cudaMalloc(&d, sizeof(wb::Tile) * t.size()));
    if (cudaMemcpy(d, t.data(), sizeof(wb::Tile) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return fail(WB_ECUDA, "tile table upload failed");
    }
    cudaFree(g->d_tiles[axis]);
    g->d_tiles[axis] = d;
    g->ntiles[axis] = (int)t.size();
    g->tile_policy[axis] = policy;
    tile_split(t, g->tile_split[axis]);
    if (g->graph) {              // tile tables changed: capture again
        cudaGraphExecDestroy(g->graph);
        g->graph = nullptr;
    }
    return WB_OK;
}

}  // namespace

int wb_autotune(wb_grid* g, double* ms_out) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    if (g->precision == WB_FP32_LEARNED) return fail(WB_EINVAL, "autotune: learned grids use the default tiles");
    WB_CK(cudaSetDevice(g->device));
    WB_CK(cudaStreamSynchronize(g->stream));
    for (int axis = 0; axis < 3; axis++) {
        float best_ms = -1.f;
        int best = -1;
        for (int c = 0; c < kNTileCandidate; c++) {
            // 0: per-patch model (one persistent launch), 1..3: each fixed
            // shape, 4: the per-patch model sorted by shape (a launch per shape)
            const int policy = candidate_policy(c);
            std::vector<wb::Tile> t = build_tiles(g, axis, policy);
            wb::Tile* d = nullptr;
            WB_CK(cudaMalloc(&d, sizeof(wb::Tile) * t.size()));
            int rc = WB_OK;
            float ms = 0.f;
            if (cudaMemcpy(d, t.data(), sizeof(wb::Tile) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                rc = fail(WB_ECUDA, "autotune: tile upload failed");
            int split[3];
            tile_split(t, split);
            if (rc == WB_OK)
                rc = g->precision == WB_FP64 ? time_sweep<double>(g, axis, d, (int)t.size(), split, &ms)
                                             : time_sweep<float>(g, axis, d, (int)t.size(), split, &ms);
            cudaFree(d);
            if (rc != WB_OK) return rc;
            if (ms_out) ms_out[axis * kNTileCandidate + c] = ms;
            if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = policy; }
        }
        const int rc = install_tiles(g, axis, best);
        if (rc != WB_OK) return rc;
    }
    return WB_OK;
}

int wb_set_tiles(wb_grid* g, int candidate) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    if (g->precision == WB_FP32_LEARNED) return fail(WB_EINVAL, "set_tiles: learned grids use the default tiles");
    if (candidate < 0 || candidate >= kNTileCandidate)
        return fail(WB_EINVAL, "set_tiles: candidate %d outside [0, %d)", candidate, kNTileCandidate);
    WB_CK(cudaSetDevice(g->device));
    WB_CK(cudaStreamSynchronize(g->stream));
    for (int axis = 0; axis < 3; axis++) {
        const int rc = install_tiles(g, axis, candidate_policy(candidate));
        if (rc != WB_OK) return rc;
    }
    return WB_OK;
}

int wb_learned_stats(wb_grid* g, long long out[2], int reset) {
    g_err.clear();
    if (!g || !out) return fail(WB_EINVAL, "null argument");
    if (!g->d_lstats) return fail(WB_EINVAL, "learned_stats: not a learned-weights grid");
    WB_CK(cudaSetDevice(g->device));
    unsigned long long h[2];
    WB_CK(cudaMemcpyAsync(g->h_small, g->d_lstats, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    if (reset) WB_CK(cudaMemsetAsync(g->d_lstats, 0, sizeof(h), g->stream));
    WB_CK(cudaStreamSynchronize(g->stream));
    std::memcpy(h, g->h_small, sizeof(h));
    out[0] = (long long)h[0];
    out[1] = (long long)h[1];
    return check_flag(g);
}

int wb_sync(wb_grid* g) {
    g_err.clear();
    if (!g) return fail(WB_EINVAL, "null grid");
    WB_CK(cudaSetDevice(g->device));
    return check_flag(g);
}

int wb_get_info(wb_grid* g, wb_grid_info* info) {
    g_err.clear();
    if (!g || !info) return fail(WB_EINVAL, "null argument");
    WB_CK(cudaSetDevice(g->device));
    WB_CK(cudaMemcpyAsync(g->h_small, g->d_scalars, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                          g->stream));
    WB_CK(cudaStreamSynchronize(g->stream));
    info->npatch = g->npatch;
    info->ncells = g->N;
    info->precision = g->precision;
    info->integrator = g->integrator;
    info->emf_mode = g->emf_mode;
    info->device_bytes = g->bytes;
    info->time = g->h_small[1];
    info->steps = g->steps;
    return WB_OK;
}

int wb_destroy(wb_grid* g) {
    g_err.clear();
    release(g);
    return WB_OK;
}

}  // extern "C"
